"""Independent first-order subcell finite volume scheme (test infrastructure: oracle).

Eq. fv-simple-form on the global subcell grid, every direction:
du_i/dt = -(M/dx) (f*(u_i, u_{i+1}) - f*(u_{i-1}, u_i)), f* the HLL flux, with the
same boundary ghosts as the blended scheme (wall mirror, outflow copy, periodic
wrap). With all blending factors zero the blended scheme must reduce to this
(Sec. 2.5 remark: alpha = 0 recovers the pure subcell FV discretisation).
"""
import numpy as np

from .euler import hll_flux, mirror

PERIODIC, WALL, OUTFLOW = 0, 1, 2


def fv_rhs(U, cfg):
    d = cfg.dim
    R = np.zeros_like(U)
    for a in range(d):
        ax = d - a
        G = U.shape[ax]
        first = np.take(U, [0], axis=ax)
        last = np.take(U, [G - 1], axis=ax)
        lo, hi = cfg.bc[2 * a], cfg.bc[2 * a + 1]
        gl = last if lo == PERIODIC else (mirror(first, a) if lo == WALL else first)
        gr = first if hi == PERIODIC else (mirror(last, a) if hi == WALL else last)
        ext = np.concatenate([gl, U, gr], axis=ax)
        left = np.take(ext, np.arange(0, G + 1), axis=ax)
        right = np.take(ext, np.arange(1, G + 2), axis=ax)
        F = hll_flux(left, right, a, cfg.gamma)
        h = (cfg.xhi[a] - cfg.xlo[a]) / G
        R -= np.diff(F, axis=ax) / h
    return R
