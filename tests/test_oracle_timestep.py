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
