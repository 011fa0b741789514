"""Saving and resuming a run (paper_2011_03338_gb300.checkpoint): the state comes back
bit for bit with its configuration, step and time."""
import numpy as np

from paper_2011_03338_gb300 import inputs
from paper_2011_03338_gb300.checkpoint import load_state, save_state


def test_state_round_trip(tmp_path):
    cfg, u = inputs.sedov(2, 4, 6, precision="fp32_split")
    save_state(str(tmp_path / "run"), u, cfg, step=17, time=0.0123, extra={"seed": 0})
    v, c, step, t, extra = load_state(str(tmp_path / "run"))
    assert np.array_equal(v.view(np.int64), u.view(np.int64))
    assert c == cfg and step == 17 and t == 0.0123 and extra == {"seed": 0}
    save_state(str(tmp_path / "run"), u * 2.0, cfg, step=18)      # replaced in place
    v, _, step, _, _ = load_state(str(tmp_path / "run"))
    assert step == 18 and np.array_equal(v, u * 2.0)
