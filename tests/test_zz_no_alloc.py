"""sesc_rhs_static, the allocation-free right-hand side, for callers that must not
have the library call cudaMalloc (a fixed device-memory budget handed out up
front, or a time-critical path where an allocation could synchronise the
device). Its output must match sesc_rhs (the handle-based entry point) within
the parity tolerance of the other tests, on two calls in a row that share the
static scratch. This file is collected last on purpose."""
import numpy as np
import pytest

from paper_2011_03338_gb300 import inputs
from tests._gpu_helpers import term_scale

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
TOL = 1e-12


def _err(cfg, got, ref, u):
    return np.abs(got - ref) / np.maximum(np.abs(ref), term_scale(cfg, u))


@pytest.mark.parametrize("case", ["sedov2d_M8", "sedov3d_M4"])
def test_static_rhs_matches_handle_rhs_twice(case):
    from paper_2011_03338_gb300 import Solver
    from paper_2011_03338_gb300.sesc import rhs_static
    if case == "sedov2d_M8":
        cfg, u1 = inputs.sedov(2, 8, 10)
        _, u2 = inputs.sedov(2, 8, 10, seed=5, sigma=0.1)
    else:
        cfg, u1 = inputs.sedov(3, 4, 5)
        _, u2 = inputs.sedov(3, 4, 5, seed=9, sigma=0.2)
    s = Solver(cfg)
    for u in (u1, u2):                                 # two calls in a row on the same scratch
        ud = torch.from_numpy(u).cuda()
        ref = torch.empty_like(ud)
        s.rhs(ud, ref)
        got = torch.full_like(ud, float("nan"))
        rhs_static(cfg, ud, got)
        torch.cuda.synchronize()
        g, r = got.cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.isfinite(g))
        assert _err(cfg, g, r, u).max() <= TOL


def test_static_rhs_rejects_problems_beyond_the_scratch():
    from paper_2011_03338_gb300.sesc import SESC_ETOOLARGE, SescError, rhs_static
    cfg = inputs.make_config(2, 8, (256, 256), (-1, -1), (1, 1), (1, 1, 1, 1))
    n = 256 * 256 * 4 * 64
    u = torch.ones(n, dtype=torch.float64, device="cuda")
    out = torch.empty_like(u)
    with pytest.raises(SescError) as ei:
        rhs_static(cfg, u, out)
    assert ei.value.code == SESC_ETOOLARGE
