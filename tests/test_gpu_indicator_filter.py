"""Certified FP32 pass of the FP64 indicator (sesc_set_indicator_filter).

The pass decides a blending factor of eq. calc-blending-factor only where the
error bound of its FP32 smoothness statistics (eq. L1-norm-slope) puts the ratio
outside the transition band; every other element is evaluated in FP64 from the
start. So the coefficients, the blending weights, the decisions, the element-face
states and the right-hand side must be the same bits with the pass on and off, on
every workload: the benchmark's Sedov blast at full size after some steps, 3D, the
Kelvin-Helmholtz and four-quadrant workloads, Gauss-Lobatto nodes, the single-level
scheme, and transition bands wide enough that the pass leaves most factors open."""
import numpy as np
import pytest

from paper_2011_03338_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _advance(s, u, steps):
    ua = torch.from_numpy(u).cuda()
    ub = torch.empty_like(ua)
    for _ in range(steps):
        s.rk3_step(ua, ub)
        ua, ub = ub, ua
    torch.cuda.synchronize()
    rc, _ = s.status()
    assert rc == 0
    return ua


def _evaluate(s, u, on):
    s.set_indicator_filter(on)
    s.reset_status()
    dev = "cuda"
    coeffs = torch.full((s.E, 2, s.S), float("nan"), dtype=torch.float64, device=dev)
    theta = torch.full((s.E, s.nl, s.md), float("nan"), dtype=torch.float64, device=dev)
    dec = torch.zeros(s.E, dtype=torch.uint8, device=dev)
    abar = torch.full((s.E, s.md), float("nan"), dtype=torch.float64, device=dev)
    s.indicator(u, coeffs, theta, dec, abar)
    r = torch.full_like(u, float("nan"))
    s.rhs(u, r)
    torch.cuda.synchronize()
    rc, cnt = s.status()
    assert rc == 0
    return (coeffs, theta, dec, abar, r), cnt


def _check_same_bits(cfg, u, steps, min_share=None, max_share=None):
    from paper_2011_03338_gb300 import Solver
    s = Solver(dict(cfg, precision="fp64"))
    ua = _advance(s, u, steps)
    got_on, c_on = _evaluate(s, ua, True)
    got_off, c_off = _evaluate(s, ua, False)
    for name, a, b in zip(("coeffs", "theta", "decision", "abar", "rhs"), got_on, got_off):
        assert torch.equal(a, b), f"{name} differs with the FP32 pass on"
    assert torch.isfinite(got_on[4]).all()
    # the same counters apart from the pass's own count (two indicator evaluations each)
    assert c_on[:12] == c_off[:12] and c_on[13:] == c_off[13:]
    assert c_off[12] == 0
    share = c_on[12] / (2.0 * s.E)
    print(f"FP32 pass decided {share:.3f} of the element evaluations")
    if min_share is not None:
        assert share >= min_share
    if max_share is not None:
        assert share <= max_share
    s.close()
    return share


def test_same_bits_on_the_benchmark_workload_at_size():
    cfg, u = inputs.sedov(2, 8, 256)
    _check_same_bits(cfg, u, 6, min_share=0.5)


@pytest.mark.parametrize("case", ["sedov2d_M4_32", "sedov2d_M8_48_lgl", "sedov3d_M4_12", "sedov3d_M8_6",
                                  "kh_M8_32", "quadrants_M4_40", "quadrants_M8_24", "sedov2d_M8_32_single"])
def test_same_bits_across_workloads(case):
    kw = {}
    if case.endswith("_lgl"):
        kw["family"] = "lgl"
    if case.endswith("_single"):
        kw["scheme"] = "single_level"
    if case.startswith("sedov2d_M4"):
        cfg, u = inputs.sedov(2, 4, 32, **kw)
    elif case.startswith("sedov2d_M8_48"):
        cfg, u = inputs.sedov(2, 8, 48, **kw)
    elif case.startswith("sedov2d_M8_32"):
        cfg, u = inputs.sedov(2, 8, 32, **kw)
    elif case == "sedov3d_M4_12":
        cfg, u = inputs.sedov(3, 4, 12)
    elif case == "sedov3d_M8_6":
        cfg, u = inputs.sedov(3, 8, 6)
    elif case == "kh_M8_32":
        cfg, u = inputs.kelvin_helmholtz(8, 32, seed=3)
    elif case == "quadrants_M4_40":
        cfg, u = inputs.quadrants(4, 40, seed=11)
    else:
        cfg, u = inputs.quadrants(8, 24, seed=5)
    _check_same_bits(cfg, u, 4)


@pytest.mark.parametrize("tauS,tauA", [(0.0, 1.0), (0.02, 4.0), (0.05, 1e4)])
def test_same_bits_when_the_band_leaves_factors_open(tauS, tauA):
    """(0, 1): the band covers every possible ratio, so the pass decides nothing and
    every element goes through the FP64 evaluation; (0.02, 4): a wide band, elements
    decided at one level and open at the next; (0.05, 1e4): a band of width 1e-4."""
    cfg, u = inputs.sedov(2, 8, 40, tauS=tauS, tauA=tauA)
    share = _check_same_bits(cfg, u, 3)
    if tauS == 0.0:
        assert share == 0.0


def test_same_bits_near_vacuum_and_with_squeezing():
    """Densities down to 1e-6 next to a strong blast: levels to squeeze and
    densities the FP32 bound cannot resolve take the FP64 evaluation."""
    cfg, u = inputs.sedov(2, 8, 24, energy=50.0, sigma=0.1)
    rng = np.random.default_rng(4)
    u = u.copy()
    low = rng.random(u.shape[0]) < 0.2
    u[low, 0, :] *= 1e-6
    u[low, 1:3, :] *= 1e-6
    _check_same_bits(cfg, u, 0)
