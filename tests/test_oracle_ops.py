"""Pins of the oracle's 1D operators against what the paper and mathematics fix."""
import os

import numpy as np
import pytest

from oracle.ops import (element_surface_operator, fv_difference_matrices, gauss_nodes,
                        lagrange_matrix, level_ops, lgl_nodes)

GOLD = os.path.join(os.path.dirname(__file__), "golden")
LEVELS = (2, 4, 8)


def test_gauss_nodes_match_tabulated_rule():
    x, w = np.loadtxt(os.path.join(GOLD, "gauss_legendre_4.txt")).T
    gx, gw = gauss_nodes(4)
    assert np.allclose(gx, 0.5 * x, atol=1e-15, rtol=0)
    assert np.allclose(gw, 0.5 * w, atol=1e-15, rtol=0)
    x2, w2 = gauss_nodes(2)
    assert np.allclose(x2, [-1 / (2 * np.sqrt(3)), 1 / (2 * np.sqrt(3))], atol=1e-16)
    assert np.allclose(w2, [0.5, 0.5])


def test_lgl_nodes_closed_form():
    x, w = lgl_nodes(3)
    assert np.allclose(x, [-0.5, 0.0, 0.5]) and np.allclose(w, [1 / 6, 4 / 6, 1 / 6])
    x, w = lgl_nodes(2)
    assert np.allclose(x, [-0.5, 0.5]) and np.allclose(w, [0.5, 0.5])


def test_projection_closed_form_n2():
    # P^(2) from its definition with nodes +-1/(2 sqrt 3) (Sec. 2.3), by hand.
    P = level_ops(2).P
    a, b = 0.5 + np.sqrt(3) / 4, 0.5 - np.sqrt(3) / 4
    assert np.allclose(P, [[a, b], [b, a]], atol=1e-15, rtol=0)


@pytest.mark.parametrize("n", LEVELS)
@pytest.mark.parametrize("family", ["gauss", "lgl"])
def test_paper_identities(n, family):
    o = level_ops(n, family)
    one = np.ones(n)
    # eq. dg-vol-mat-property: w^T Dvol = 0
    assert np.abs(o.w @ o.Dvol).max() < 1e-13
    # eq. projection-mat-property: 1^T P = n w^T
    assert np.abs(one @ o.P - n * o.w).max() < 1e-13
    # eq. reconstruction-mat-property: w^T R = w^T R^(beta) = 1^T / n
    assert np.abs(o.w @ o.R - one / n).max() < 1e-13
    for beta in (0.0, 0.3, 0.97):
        Rb = (1 - beta) / n * np.outer(one, one) + beta * o.R
        assert np.abs(o.w @ Rb - one / n).max() < 1e-13
    # eq. dg-surf-mat-property: w^T B0 = 1^T Delta^(S)
    _, DV, DS = fv_difference_matrices(n)
    assert np.abs(o.w @ o.B0 - np.ones(n) @ DS).max() < 1e-13
    # eq. fv-vol-mat-property: 1^T Delta^(V) = 0
    assert np.abs(np.ones(n) @ DV).max() == 0.0
    # R is the inverse of P
    assert np.abs(o.R @ o.P - np.eye(n)).max() < 1e-12
    # D 1 = 0 (derivative of a constant)
    assert np.abs(o.Dnodal @ one).max() < 1e-12


@pytest.mark.parametrize("n", LEVELS)
def test_operators_exact_on_polynomials(n):
    """D, P, I+-, b+- are exact for polynomials of degree < n (brute force against
    closed-form derivatives, antiderivatives and point values)."""
    o = level_ops(n)
    xi = o.nodes
    edges = -0.5 + np.arange(n + 1) / n
    for k in range(n):
        vals = xi ** k
        dk = k * xi ** (k - 1) if k > 0 else 0 * xi
        assert np.allclose(o.Dnodal @ vals, dk, atol=1e-11)
        means = n * (edges[1:] ** (k + 1) - edges[:-1] ** (k + 1)) / (k + 1)
        assert np.allclose(o.P @ vals, means, atol=1e-12)
        assert np.allclose(o.R @ means, vals, atol=1e-10)
        assert np.allclose(o.Iminus @ vals, edges[:-1] ** k, atol=1e-11)
        assert np.allclose(o.Iplus @ vals, edges[1:] ** k, atol=1e-11)
        assert np.isclose(o.bminus @ vals, (-0.5) ** k) and np.isclose(o.bplus @ vals, 0.5 ** k)


def test_lagrange_is_cardinal():
    x, _ = gauss_nodes(8)
    assert np.allclose(lagrange_matrix(x, x), np.eye(8), atol=1e-14)


@pytest.mark.parametrize("n", LEVELS)
def test_surface_operator_sparsity_matches_appendix(n):
    """[I_{8/n} (x) Bhat^(n)]^(0) in R^{8x9}: nonzeros only in the columns of the
    sub-element boundary interfaces, block by block (appendix boundary-eval-op)."""
    S = element_surface_operator(8, n)
    expected = np.zeros((8, 9), dtype=bool)
    for s in range(8 // n):
        expected[s * n:(s + 1) * n, s * n] = True
        expected[s * n:(s + 1) * n, s * n + n] = True
    assert np.array_equal(np.abs(S) > 1e-14, expected)


def test_dvol_is_weak_derivative():
    """Dvol = M^-1 D^T M: for nodal f, g of degree < n, w^T (g * Dvol f) equals the
    exact integral of g' f (integration by parts without boundary terms is the
    adjoint relation sum_i w_i g_i (Dvol f)_i = sum_j w_j f_j (D g)_j)."""
    o = level_ops(6)
    rng = np.random.default_rng(1)
    f, gv = rng.standard_normal(6), rng.standard_normal(6)
    lhs = o.w @ (gv * (o.Dvol @ f))
    rhs = o.w @ (f * (o.Dnodal @ gv))
    assert np.isclose(lhs, rhs, rtol=1e-12)
