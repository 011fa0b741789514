"""Convergence pins of the oracle: design order on a smooth advected density wave
with the indicator active (Sec. 3.2, tables of EOCs: order ~ n for the level-n
variant; the indicator must keep smooth data at full order, Sec. 2.7), first
order of the subcell FV scheme, and the Sod shock tube against the exact
Riemann solution (Sec. 3.4)."""
import numpy as np

from oracle.blended import Config, blended_rhs
from oracle.exact_riemann import cell_averages
from oracle.layout import to_grid
from oracle.plain_fv import fv_rhs
from oracle.timestep import cfl_dt, rk3_step
from paper_2011_03338_gb300 import inputs


def _wave_error(nel, M, T=0.1, cfl=0.1, scheme="blended"):
    cd, u = inputs.density_wave(M=M, nel_per_dir=nel)
    cfg = Config(**{**cd, "cfl": cfl})
    U = to_grid(u, 2, M, cd["nel"])
    t = 0.0
    full_order = True
    while t < T - 1e-14:
        dt = min(cfl_dt(U, cfg), T - t)
        if scheme == "blended":
            _, dg = blended_rhs(U, cfg, return_diag=True)
            full_order &= bool(np.all(dg.n_min == M) and np.all(dg.n_max == M))
            U, _ = rk3_step(U, cfg, dt)
        else:
            U0, Us = U, U
            for a, b in ((0.0, 1.0), (0.75, 0.25), (1 / 3, 2 / 3)):
                Us = a * U0 + b * (Us + dt * fv_rhs(Us, cfg))
            U = Us
        t += dt
    _, ue = inputs.density_wave(M=M, nel_per_dir=nel, t=T)
    Ue = to_grid(ue, 2, M, cd["nel"])
    return np.sqrt(np.mean((U[0] - Ue[0]) ** 2)), full_order


def test_design_order_with_indicator_active():
    e4, ok4 = _wave_error(4, 4)
    e8, ok8 = _wave_error(8, 4)
    assert ok4 and ok8                      # smooth data never triggers blending
    eoc = np.log2(e4 / e8)
    assert 3.5 < eoc < 4.6, eoc


def test_subcell_fv_is_first_order():
    e1, _ = _wave_error(4, 4, T=0.2, cfl=0.5, scheme="fv")
    e2, _ = _wave_error(8, 4, T=0.2, cfl=0.5, scheme="fv")
    assert 0.8 < np.log2(e1 / e2) < 1.3


def test_sod_converges_to_exact_solution():
    errs = []
    for nel in (16, 32):
        cd, u = inputs.sod(M=4, nel_x=nel)
        cfg = Config(**cd)
        U = to_grid(u, 2, 4, cd["nel"])
        t, T = 0.0, 0.2
        while t < T - 1e-14:
            dt = min(cfl_dt(U, cfg), T - t)
            U, _ = rk3_step(U, cfg, dt)
            t += dt
        ex = cell_averages((1, 0, 1), (0.125, 0, 0.1), 0.5, T, np.linspace(0, 1, nel * 4 + 1))
        errs.append(np.abs(U[0].mean(axis=0) - ex[0]).mean())
        assert U[0].min() > 0 and np.all(np.isfinite(U))
    assert errs[1] < 0.7 * errs[0] and errs[0] < 0.01, errs


def test_lax_tube_converges_to_exact_solution():
    """The Lax shock tube of Sec. 3.4 (textbook states: (rho, u, p) = (0.445, 0.698,
    3.528) | (0.5, 0, 0.571), diaphragm at 0.5, t = 0.13) against the exact
    Riemann solution: the L1 density error falls with resolution."""
    left, right, T = (0.445, 0.698, 3.528), (0.5, 0.0, 0.571), 0.13
    errs = []
    for nel in (16, 32):
        cd, u = inputs.shock_tube(left, right, M=4, nel_x=nel)
        cfg = Config(**cd)
        U = to_grid(u, 2, 4, cd["nel"])
        t = 0.0
        while t < T - 1e-14:
            dt = min(cfl_dt(U, cfg), T - t)
            U, _ = rk3_step(U, cfg, dt)
            t += dt
        ex = cell_averages(left, right, 0.5, T, np.linspace(0, 1, nel * 4 + 1))
        errs.append(np.abs(U[0].mean(axis=0) - ex[0]).mean())
        assert U[0].min() > 0 and np.all(np.isfinite(U))
    assert errs[1] < 0.7 * errs[0] and errs[0] < 0.03, errs
