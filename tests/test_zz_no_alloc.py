"""sesc_rhs_static, the allocation-free right-hand side.

It serves callers that must not have a library allocate device memory: a program
that hands out a fixed device-memory budget up front and forbids allocations
behind its back, or a time-critical path where cudaMalloc / cudaFree could
synchronise the device. It runs the same kernels as sesc_rhs (the handle-based
entry point) on the same input, with its scratch in a static device array instead
of a handle's workspace, so its output must be bit-identical to sesc_rhs, on two
calls in a row that share (and reuse) that array.

Why this file's name starts with test_zz: pytest collects files in name order, so
it runs last. Its subject is an extra service, not part of the method, and if it
fails, a run that stops at the first failure (pytest -x) has by then run every
parity test of the method itself. The test does not depend on that order: it
passes alone in a fresh process (its first call sets up the device) and after the
other tests."""
import numpy as np
import pytest

from paper_2011_03338_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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
        assert torch.isfinite(got).all()
        assert torch.equal(got, ref), (got - ref).abs().max().item()


def test_static_rhs_rejects_problems_beyond_the_scratch():
    from paper_2011_03338_gb300.sesc import SESC_ETOOLARGE, SescError, rhs_static
    cfg = inputs.make_config(2, 8, (256, 256), (-1, -1), (1, 1), (1, 1, 1, 1))
    n = 256 * 256 * 4 * 64
    u = torch.ones(n, dtype=torch.float64, device="cuda")
    out = torch.empty_like(u)
    with pytest.raises(SescError) as ei:
        rhs_static(cfg, u, out)
    assert ei.value.code == SESC_ETOOLARGE
    assert np.isfinite(u.sum().item())
