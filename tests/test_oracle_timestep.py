"""Pins of the oracle's time integrators: the SSP-RK(5,4) coefficients satisfy the
fourth-order conditions of the Butcher tableau they define, are consistent and
nonnegative (strong-stability preserving, SSP coefficient above 1.5), and the
step converges at fourth order on a linear ODE with a closed-form solution; the
SSP-RK3 stages are the classical third-order method."""
import numpy as np

from oracle.timestep import RK3_STAGES, SSPRK54_ALPHA, SSPRK54_BETA, shu_osher_step


def _butcher(alpha, beta):
    """Butcher matrix of a Shu-Osher method: u_i = u + dt sum_j A_ij L(u_j)."""
    s = len(alpha)
    A = np.zeros((s + 1, s + 1))
    for i in range(1, s + 1):
        for k in range(i):
            A[i] += alpha[i - 1][k] * A[k]
            A[i, k] += beta[i - 1][k]
    return A[:s, :s], A[s, :s]


def test_ssprk54_order_conditions():
    A, b = _butcher(SSPRK54_ALPHA, SSPRK54_BETA)
    c = A.sum(axis=1)
    cond = {
        "b": (b.sum(), 1.0), "bc": (b @ c, 1 / 2), "bc2": (b @ c ** 2, 1 / 3), "bAc": (b @ A @ c, 1 / 6),
        "bc3": (b @ c ** 3, 1 / 4), "bcAc": (b @ (c * (A @ c)), 1 / 8), "bAc2": (b @ A @ c ** 2, 1 / 12),
        "bAAc": (b @ A @ A @ c, 1 / 24),
    }
    for k, (got, want) in cond.items():
        assert abs(got - want) < 1e-13, (k, got, want)


def test_ssprk54_is_consistent_and_ssp():
    for row in SSPRK54_ALPHA:
        assert abs(sum(row) - 1.0) < 1e-14
    ratios = []
    for ar, br in zip(SSPRK54_ALPHA, SSPRK54_BETA):
        for a, b in zip(ar, br):
            assert a >= 0.0 and b >= 0.0
            if b > 0.0:
                ratios.append(a / b)
    assert 1.50 < min(ratios) < 1.51                      # the published SSP coefficient, about 1.508


def test_ssprk54_fourth_order_on_linear_ode():
    lam = -1.3 + 0.7j
    errs = []
    for n in (10, 20, 40):
        dt, y = 1.0 / n, 1.0 + 0.0j
        for _ in range(n):
            y = shu_osher_step(y, lambda v: lam * v, dt, SSPRK54_ALPHA, SSPRK54_BETA)
        errs.append(abs(y - np.exp(lam)))
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(3.8 < r < 4.3 for r in rates), rates


def test_rk3_stages_are_the_third_order_ssp_method():
    alpha = [(1.0,), (0.75, 0.25), (1 / 3, 0.0, 2 / 3)]
    beta = [(1.0,), (0.0, 0.25), (0.0, 0.0, 2 / 3)]
    assert [tuple(x) for x in RK3_STAGES] == [(0.0, 1.0), (0.75, 0.25), (1 / 3, 2 / 3)]
    A, b = _butcher(alpha, beta)
    c = A.sum(axis=1)
    assert abs(b.sum() - 1) < 1e-15 and abs(b @ c - 0.5) < 1e-15
    assert abs(b @ c ** 2 - 1 / 3) < 1e-15 and abs(b @ A @ c - 1 / 6) < 1e-15


def _cfl_case(dim, M):
    """Two elements along x; every mean at state A (rho 1, p 5/7, so c = 1, and
    velocity components of largest magnitude 2: lambda = 3) except one subcell of
    the second element at state B (rho 1/4, p 5/7: c = 2, one velocity component
    of magnitude 3: lambda = 5), eq. euler-max-eigenvalue."""
    from oracle.blended import Config
    from oracle.euler import conserved
    g = 1.4
    if dim == 2:
        cfg = Config(dim=2, M=M, nel=(2, 1), xlo=(0.0, 0.0), xhi=(2.0, 0.5), bc=(1, 1, 1, 1))
        wA, wB = [1.0, 0.5, -2.0, 5 / 7], [0.25, 0.0, 3.0, 5 / 7]
        shape = (M, 2 * M)
    else:
        cfg = Config(dim=3, M=M, nel=(2, 1, 1), xlo=(0.0, 0.0, 0.0), xhi=(2.0, 1.0, 0.25), bc=(1,) * 6)
        wA, wB = [1.0, 0.5, -2.0, 1.0, 5 / 7], [0.25, 0.0, 0.0, -3.0, 5 / 7]
        shape = (M, M, 2 * M)
    W = np.empty((dim + 2,) + shape)
    W[:] = np.array(wA).reshape((-1,) + (1,) * dim)
    idx = (slice(None),) + (1,) * (dim - 1) + (M + 2,)           # a subcell of element 2
    W[idx] = wB
    return cfg, conserved(W, g)


def test_cfl_dt_against_hand_values():
    """eq. cfl-condition: dt = CFL min_q dx_q / (2^(d-1) (2M - 1) lambda_q), CFL 0.5,
    lambda = 5 (the element holding state B), dx_q the smallest edge:
      2D, M = 4, dx = (1, 1/2):       0.5 (1/2) / (2 * 7 * 5)  = 1/280
      2D, M = 8:                       0.5 (1/2) / (2 * 15 * 5) = 1/600
      3D, M = 4, dx = (1, 1, 1/4):    0.5 (1/4) / (4 * 7 * 5)  = 1/1120
    A factor 2^d, (2M + 1), the largest edge or the mean wave speed would each
    move the value."""
    from oracle.euler import max_wave_speed
    from oracle.timestep import cfl_dt
    for dim, M, want in ((2, 4, 1 / 280), (2, 8, 1 / 600), (3, 4, 1 / 1120)):
        cfg, U = _cfl_case(dim, M)
        lam = max_wave_speed(U, cfg.gamma)
        assert abs(lam.max() - 5.0) < 1e-14 and abs(np.sort(lam.ravel())[-2] - 3.0) < 1e-14
        assert abs(cfl_dt(U, cfg) - want) < 1e-17, (dim, M, cfl_dt(U, cfg), want)
