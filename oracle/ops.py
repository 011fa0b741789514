"""1D operators of one level of the hierarchy (test infrastructure: oracle).

Everything lives on a (sub-)element reference interval xi in [-1/2, 1/2] with
``n`` collocation nodes, as in Sec. 2.2 (eq. sub-element, eq. lagrange-function).
Definitions followed:

* Gauss-Legendre nodes and weights, weights summing to 1 (Sec. 2.2: "The nodes
  are the Gauss-Legendre quadrature nodes"; appendix 3D extension).
  Legendre-Gauss-Lobatto nodes are provided as a variant.
* D_ij = l_j'(xi_i), the nodal differentiation matrix (Sec. 2.2).
* Dvol = M^-1 D^T M, Bsurf = M^-1 B with B the boundary evaluation matrix
  (eq. boundary-evalution-matrix, eq. semi-discrete-dg).
* b+- = l_j(+-1/2) (eq. boundary-interpolation-operators).
* P_ij = n_mu * int over subcell i of l_j (Sec. 2.3, projection operator).
* R = P^-1 (eq. trafo-mv-nodal).
* B0: Bsurf with a column of zeros inserted (eq. tweak-boundary-evaluation-matrix)
  generalised to n x (n+1); Dhat = P Dvol, Bhat = P B0 (eq. dgfv-operators).
* I+- : values at the right / left interface of each subcell
  (eq. subcell-fv-interpolation-operator).
* Delta, Delta^(V), Delta^(S): FV difference matrix and its split
  (eqs. fv-diff-matrix, fv-vol-surf-matrices).
"""
from dataclasses import dataclass

import numpy as np
from numpy.polynomial import legendre as npleg


def gauss_nodes(n):
    """n Gauss-Legendre nodes on [-1/2, 1/2] and weights that sum to 1."""
    x, w = npleg.leggauss(n)
    return 0.5 * x, 0.5 * w


def lgl_nodes(n):
    """n Legendre-Gauss-Lobatto nodes on [-1/2, 1/2] and weights that sum to 1.

    Nodes: the end points and the roots of P'_{n-1}; weights
    2 / (n (n-1) P_{n-1}(x)^2) on [-1, 1] (textbook LGL rule)."""
    if n < 2:
        raise ValueError("LGL needs n >= 2")
    cn = np.zeros(n)
    cn[-1] = 1.0  # coefficients of P_{n-1}
    interior = np.sort(np.real(npleg.legroots(npleg.legder(cn)))) if n > 2 else np.array([])
    x = np.concatenate(([-1.0], interior, [1.0]))
    w = 2.0 / (n * (n - 1) * npleg.legval(x, cn) ** 2)
    return 0.5 * x, 0.5 * w


def lagrange_matrix(nodes, x):
    """L[i, j] = l_j(x_i) with l_j the Lagrange polynomial of eq. lagrange-function."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    out = np.ones((len(x), n))
    for j in range(n):
        for k in range(n):
            if k != j:
                out[:, j] *= (x - nodes[k]) / (nodes[j] - nodes[k])
    return out


def lagrange_derivative_matrix(nodes, x):
    """L'[i, j] = l_j'(x_i), from the product rule applied to eq. lagrange-function."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    out = np.zeros((len(x), n))
    for j in range(n):
        for m in range(n):
            if m == j:
                continue
            term = np.full(len(x), 1.0 / (nodes[j] - nodes[m]))
            for k in range(n):
                if k != j and k != m:
                    term *= (x - nodes[k]) / (nodes[j] - nodes[k])
            out[:, j] += term
    return out


def projection_matrix(nodes, n_mu):
    """P^(n -> n_mu)_ij = n_mu * int_{mu_{i-1/2}}^{mu_{i+1/2}} l_j(xi) dxi (Sec. 2.3).

    The integral is taken exactly with an n-point Gauss rule on each subcell
    (l_j has degree n-1)."""
    n = len(nodes)
    gx, gw = npleg.leggauss(n)
    P = np.zeros((n_mu, n))
    for i in range(n_mu):
        a = -0.5 + i / n_mu
        b = a + 1.0 / n_mu
        xq = 0.5 * (a + b) + 0.5 * (b - a) * gx
        wq = 0.5 * (b - a) * gw
        P[i, :] = n_mu * (wq @ lagrange_matrix(nodes, xq))
    return P


def fv_difference_matrices(n):
    """Delta, Delta^(V), Delta^(S) in R^{n x (n+1)} (eqs. fv-diff-matrix, fv-vol-surf-matrices)."""
    Delta = np.zeros((n, n + 1))
    for i in range(n):
        Delta[i, i] = -1.0
        Delta[i, i + 1] = 1.0
    DeltaS = np.zeros((n, n + 1))
    DeltaS[0, 0] = -1.0
    DeltaS[n - 1, n] = 1.0
    DeltaV = Delta - DeltaS
    return Delta, DeltaV, DeltaS


@dataclass
class LevelOps:
    n: int
    nodes: np.ndarray      # xi_i on [-1/2, 1/2]
    w: np.ndarray          # omega_i, sum 1
    Dnodal: np.ndarray     # D_ij = l_j'(xi_i)
    Dvol: np.ndarray       # M^-1 D^T M
    Bmat: np.ndarray       # boundary evaluation matrix (n x n)
    Bsurf: np.ndarray      # M^-1 B (n x n)
    B0: np.ndarray         # Bsurf with the zero column inserted (n x (n+1))
    bminus: np.ndarray     # l_j(-1/2)
    bplus: np.ndarray      # l_j(+1/2)
    P: np.ndarray          # projection nodal -> n subcell means
    R: np.ndarray          # P^-1
    Dhat: np.ndarray       # P Dvol
    Bhat: np.ndarray       # P B0
    Iminus: np.ndarray     # (I^-)_ij = l_j(mu_{i-1/2})
    Iplus: np.ndarray      # (I^+)_ij = l_j(mu_{i+1/2})


def level_ops(n, family="gauss"):
    """All 1D operators of the level with n >= 2 nodes / n subcells per sub-element."""
    if n < 2:
        raise ValueError("DG levels have n >= 2; level 1 is the subcell FV scheme")
    if family == "gauss":
        nodes, w = gauss_nodes(n)
    elif family == "lgl":
        nodes, w = lgl_nodes(n)
    else:
        raise ValueError(family)
    Dn = lagrange_derivative_matrix(nodes, nodes)
    Mass = np.diag(w)
    Minv = np.diag(1.0 / w)
    Dvol = Minv @ Dn.T @ Mass
    bminus = lagrange_matrix(nodes, [-0.5])[0]
    bplus = lagrange_matrix(nodes, [0.5])[0]
    Bmat = np.zeros((n, n))
    Bmat[:, 0] = -bminus
    Bmat[:, n - 1] += bplus
    Bsurf = Minv @ Bmat
    B0 = np.zeros((n, n + 1))
    B0[:, 0] = Bsurf[:, 0]
    B0[:, n] = Bsurf[:, n - 1]
    P = projection_matrix(nodes, n)
    R = np.linalg.inv(P)
    left = -0.5 + np.arange(n) / n
    right = left + 1.0 / n
    return LevelOps(
        n=n, nodes=nodes, w=w, Dnodal=Dn, Dvol=Dvol, Bmat=Bmat, Bsurf=Bsurf, B0=B0,
        bminus=bminus, bplus=bplus, P=P, R=R, Dhat=P @ Dvol, Bhat=P @ B0,
        Iminus=lagrange_matrix(nodes, left), Iplus=lagrange_matrix(nodes, right),
    )


def element_surface_operator(M, n, family="gauss"):
    """[I_{M/n} (x) Bhat^(n)]^(0) in R^{M x (M+1)}: the level-n surface operator acting
    on the M+1 subcell interface fluxes of an element, with Bhat's first and last
    columns placed on each sub-element's boundary interfaces (appendix on boundary
    evaluation operators)."""
    op = level_ops(n, family)
    out = np.zeros((M, M + 1))
    for s in range(M // n):
        out[s * n:(s + 1) * n, s * n:s * n + n + 1] += op.Bhat
    return out
