"""Saving and resuming a run: the state (FP64 subcell means, element-major), its
configuration, the step count and the simulated time, in one directory of plain
files (state.npy and run.json). Host-side bookkeeping only; the state is copied
to / from the device by the caller (numpy or torch)."""
import json
import os

import numpy as np


def save_state(path, u, cfg, step=0, time=0.0, extra=None):
    """Write u ([E][d+2][M^d] array or CUDA tensor), cfg (the configuration dict), the
    step count and time to directory `path` (created if missing); files are replaced
    atomically."""
    os.makedirs(path, exist_ok=True)
    arr = u.detach().cpu().numpy() if hasattr(u, "detach") else np.asarray(u)
    if arr.dtype != np.float64:
        raise ValueError("the state is FP64")
    tmp = os.path.join(path, "state.npy.tmp")
    with open(tmp, "wb") as fh:
        np.save(fh, arr)
    os.replace(tmp, os.path.join(path, "state.npy"))
    meta = {"config": {k: (list(v) if isinstance(v, tuple) else v) for k, v in dict(cfg).items()},
            "step": int(step), "time": float(time), "shape": list(arr.shape), "extra": extra or {}}
    tmp = os.path.join(path, "run.json.tmp")
    with open(tmp, "w") as fh:
        json.dump(meta, fh)
    os.replace(tmp, os.path.join(path, "run.json"))


def load_state(path):
    """(u, cfg, step, time, extra) from a directory written by save_state; tuples of the
    configuration come back as tuples."""
    with open(os.path.join(path, "run.json")) as fh:
        meta = json.load(fh)
    u = np.load(os.path.join(path, "state.npy"))
    if list(u.shape) != meta["shape"]:
        raise ValueError("state and run record disagree")
    cfg = {k: (tuple(v) if isinstance(v, list) else v) for k, v in meta["config"].items()}
    return u, cfg, meta["step"], meta["time"], meta["extra"]
