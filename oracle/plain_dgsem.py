"""Independent nodal DGSEM on Gauss nodes (test infrastructure: oracle).

Sec. 2.2: on every element of size dx with n Gauss nodes per direction,
du~/dt = (1/dx) (Dvol f~ - Bsurf f*) per direction (eq. semi-discrete-dg, tensor
product for d > 1), f* the HLL flux evaluated pointwise at the face nodes between
b+^T u~ of the left and b-^T u~ of the right element (eqs. dg-surface-flux,
dg-boundary-values). Boundary ghosts as in the blended scheme.

Pins: with the top-level blending weight 1 everywhere the blended scheme equals
P (DGSEM(R u)) (Sec. 2.5 remark: alpha = 1 recovers pure DG); with level n forced
everywhere it equals this DGSEM on the mesh of level-n sub-elements.
"""
import numpy as np

from .euler import hll_flux, mirror, physical_flux
from .ops import level_ops

PERIODIC, WALL, OUTFLOW = 0, 1, 2


def _mode(X, A, axis, n):
    X = np.moveaxis(X, axis, -1)
    sh = X.shape
    Y = np.einsum("...bj,kj->...bk", X.reshape(sh[:-1] + (sh[-1] // n, n)), A)
    return np.moveaxis(Y.reshape(sh[:-1] + (sh[-1] // n * A.shape[0],)), -1, axis)


def dgsem_rhs(Ut, cfg, n, family="gauss"):
    """Nodal DGSEM RHS; Ut has n nodes per element along each axis on a grid of
    G_a / n elements per direction (element size (xhi-xlo) n / G_a)."""
    d = cfg.dim
    o = level_ops(n, family)
    R = np.zeros_like(Ut)
    for a in range(d):
        ax = d - a
        G = Ut.shape[ax]
        ne = G // n
        h = (cfg.xhi[a] - cfg.xlo[a]) / ne
        vol = _mode(physical_flux(Ut, a, cfg.gamma), o.Dvol, ax, n)
        # boundary values of every element along a
        Xm = np.moveaxis(Ut, ax, -1)
        blocks = Xm.reshape(Xm.shape[:-1] + (ne, n))
        uminus = np.einsum("...ej,j->...e", blocks, o.bminus)  # left face of each element
        uplus = np.einsum("...ej,j->...e", blocks, o.bplus)    # right face of each element
        lo, hi = cfg.bc[2 * a], cfg.bc[2 * a + 1]
        # faces 0..ne: left state / right state
        if lo == PERIODIC:
            gl = uplus[..., -1:]
        elif lo == WALL:
            gl = mirror(uminus[..., :1], a)
        else:
            gl = uminus[..., :1]
        if hi == PERIODIC:
            gr = uminus[..., :1]
        elif hi == WALL:
            gr = mirror(uplus[..., -1:], a)
        else:
            gr = uplus[..., -1:]
        left = np.concatenate([gl, uplus], axis=-1)
        right = np.concatenate([uminus, gr], axis=-1)
        F = hll_flux(left, right, a, cfg.gamma)                 # (..., ne+1) with variable axis first
        Fl = F[..., :-1]
        Fr = F[..., 1:]
        surf = (Fl[..., None] * o.Bsurf[:, 0] + Fr[..., None] * o.Bsurf[:, n - 1])  # (..., ne, n)
        surf = surf.reshape(surf.shape[:-2] + (G,))
        surf = np.moveaxis(surf, -1, ax)
        R += (vol - surf) / h
    return R


def projected_dgsem_rhs(U, cfg, n, family="gauss"):
    """P(DGSEM(R u)) on the mesh of level-n sub-elements of the means U."""
    o = level_ops(n, family)
    d = cfg.dim
    Ut = U
    for a in range(d):
        Ut = _mode(Ut, o.R, d - a, n)
    R = dgsem_rhs(Ut, cfg, n, family)
    for a in range(d):
        R = _mode(R, o.P, d - a, n)
    return R
