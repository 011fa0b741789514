"""The bounds-checked build (-DSESC_BOUNDS, libsesc_bounds.so): every computed
global index of the kernels (neighbour elements of a face, halo rows, face-flux rows,
element indices) is checked against its buffer, and one outside would record
SESC_EBOUNDS in the status word instead of being accessed.

The same script runs in two child processes, one per library (selected by
SESC_LIBRARY), over the code paths of the parity suite: both precisions, 2D and 3D,
walls / periodic / outflow, a mesh split into parts (halo reads), a batch in one
launch per stage, and the adjoint. The checked build must report no index out of
range and give the regular build's results bit for bit."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import sys
import numpy as np
import torch
from paper_2011_03338_gb300 import Batch, Solver, inputs
from paper_2011_03338_gb300.shard import LocalGroup

out, codes = {}, {}

def steps(name, cfg, u0, n=2):
    s = Solver(cfg)
    u = torch.from_numpy(u0).cuda()
    v = torch.empty_like(u)
    r = torch.empty_like(u)
    s.rhs(u, r)
    out[name + "_rhs"] = r.cpu().numpy()
    for _ in range(n):
        s.rk3_step(u, v)
        u, v = v, u
    out[name + "_u"] = u.cpu().numpy()
    codes[name] = s.status()[0]
    return s, u

split = dict(precision="fp32_split")
steps("sedov2d_m8_fp64", *inputs.sedov(2, 8, 12))
steps("sedov2d_m8_split", *inputs.sedov(2, 8, 12, **split))
steps("sedov3d_m4_fp64", *inputs.sedov(3, 4, 5))
steps("quad_m4_split", *inputs.quadrants(4, 10, seed=1, **split))
s, u = steps("kh_m8_fp64", *inputs.kelvin_helmholtz(8, 6))
# adjoint of the right-hand side
g = torch.from_numpy(np.random.default_rng(3).standard_normal(tuple(u.shape))).cuda()
ub = torch.empty_like(u)
s.rhs_vjp(u, g, ub)
out["kh_vjp"] = ub.cpu().numpy()
codes["kh_vjp"] = s.status()[0]
# one mesh in three parts (halo rows of the face-flux kernel)
cfg, u0 = inputs.sedov(2, 4, 9)
lg = LocalGroup(cfg, 3)
u = torch.from_numpy(u0).cuda()
r = torch.empty_like(u)
lg.rhs(lg.split(u), lg.split(r))
out["parts_rhs"] = r.cpu().numpy()
for k, p in enumerate(lg.parts):
    codes[f"part{k}"] = p.solver.status()[0]
# a batch of uneven problems, default launch mode
probs = [inputs.sedov(2, 4, 6), inputs.quadrants(4, 7, seed=2, **split), inputs.sedov(2, 8, 5, seed=7)]
b = Batch([c for c, _ in probs])
ub = torch.empty(b.total, dtype=torch.float64, device="cuda")
for k, (_, uk) in enumerate(probs):
    b.view(ub, k).copy_(torch.from_numpy(uk))
vb = torch.empty_like(ub)
b.rk3_step(ub, vb)
out["batch_u"] = vb.cpu().numpy()
codes["batch"] = b.status()[0]
torch.cuda.synchronize()
np.savez(sys.argv[1], **out)
print(";".join(f"{k}={v}" for k, v in codes.items()))
"""


def _run(tmp_path, tag, lib):
    script = tmp_path / "bounds_case.py"
    script.write_text(SCRIPT)
    env = dict(os.environ)
    env["PYTHONPATH"] = ROOT + os.pathsep + env.get("PYTHONPATH", "")
    if lib:
        env["SESC_LIBRARY"] = lib
    else:
        env.pop("SESC_LIBRARY", None)
    res = subprocess.run([sys.executable, str(script), str(tmp_path / f"{tag}.npz")], env=env, cwd=ROOT,
                         capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stdout[-2000:] + res.stderr[-4000:]
    codes = dict(kv.split("=") for kv in res.stdout.strip().splitlines()[-1].split(";"))
    return np.load(tmp_path / f"{tag}.npz"), {k: int(v) for k, v in codes.items()}


def test_bounds_checked_build_reports_nothing_and_matches(tmp_path):
    from paper_2011_03338_gb300 import build
    lib = build.build(bounds=True)
    ref, ref_codes = _run(tmp_path, "regular", None)
    got, codes = _run(tmp_path, "bounds", lib)
    assert all(c == 0 for c in ref_codes.values()), ref_codes
    assert all(c == 0 for c in codes.values()), codes   # in particular no SESC_EBOUNDS
    assert sorted(ref.files) == sorted(got.files)
    for k in ref.files:
        assert np.array_equal(ref[k].view(np.int64), got[k].view(np.int64)), k
