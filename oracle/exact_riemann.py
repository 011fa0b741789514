"""Exact solution of the 1D Riemann problem of the ideal-gas Euler equations
(test infrastructure: oracle; pin for the Sod shock tube of Sec. 3.4).

Textbook method (Toro, "Riemann Solvers and Numerical Methods for Fluid
Dynamics", ch. 4): the star pressure is the root of
f_L(p) + f_R(p) + (u_R - u_L) = 0 with the shock / rarefaction branches of f_K,
found by Newton iteration; the solution is then sampled on x/t.
"""
import numpy as np


def _fk(p, rho, pk, ck, g):
    if p > pk:   # shock
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        sq = np.sqrt(A / (p + B))
        return (p - pk) * sq, sq * (1.0 - 0.5 * (p - pk) / (B + p))
    # rarefaction
    pr = p / pk
    f = 2.0 * ck / (g - 1.0) * (pr ** ((g - 1.0) / (2.0 * g)) - 1.0)
    df = 1.0 / (rho * ck) * pr ** (-(g + 1.0) / (2.0 * g))
    return f, df


def star_state(left, right, g=1.4, tol=1e-14, maxit=100):
    """(p*, u*) for left/right primitive states (rho, u, p)."""
    rL, uL, pL = left
    rR, uR, pR = right
    cL, cR = np.sqrt(g * pL / rL), np.sqrt(g * pR / rR)
    p = max(tol, 0.5 * (pL + pR) - 0.125 * (uR - uL) * (rL + rR) * (cL + cR))
    for _ in range(maxit):
        fL, dL = _fk(p, rL, pL, cL, g)
        fR, dR = _fk(p, rR, pR, cR, g)
        pn = p - (fL + fR + uR - uL) / (dL + dR)
        pn = max(pn, tol)
        if abs(pn - p) <= tol * 0.5 * (pn + p):
            p = pn
            break
        p = pn
    fL, _ = _fk(p, rL, pL, cL, g)
    fR, _ = _fk(p, rR, pR, cR, g)
    u = 0.5 * (uL + uR) + 0.5 * (fR - fL)
    return p, u


def sample(left, right, xi, g=1.4):
    """Primitive solution (rho, u, p) at similarity coordinates xi = (x - x0)/t."""
    rL, uL, pL = left
    rR, uR, pR = right
    cL, cR = np.sqrt(g * pL / rL), np.sqrt(g * pR / rR)
    ps, us = star_state(left, right, g)
    xi = np.atleast_1d(np.asarray(xi, dtype=np.float64))
    out = np.zeros((3, len(xi)))
    gm = (g - 1.0) / (g + 1.0)
    for i, s in enumerate(xi):
        if s <= us:   # left of contact
            if ps > pL:
                SL = uL - cL * np.sqrt((g + 1.0) / (2 * g) * ps / pL + (g - 1.0) / (2 * g))
                if s <= SL:
                    out[:, i] = (rL, uL, pL)
                else:
                    out[:, i] = (rL * (ps / pL + gm) / (gm * ps / pL + 1.0), us, ps)
            else:
                cs = cL * (ps / pL) ** ((g - 1.0) / (2 * g))
                SH, ST = uL - cL, us - cs
                if s <= SH:
                    out[:, i] = (rL, uL, pL)
                elif s >= ST:
                    out[:, i] = (rL * (ps / pL) ** (1.0 / g), us, ps)
                else:
                    fac = 2.0 / (g + 1.0) + gm / cL * (uL - s)
                    out[:, i] = (rL * fac ** (2.0 / (g - 1.0)),
                                 2.0 / (g + 1.0) * (cL + (g - 1.0) / 2 * uL + s),
                                 pL * fac ** (2 * g / (g - 1.0)))
        else:         # right of contact
            if ps > pR:
                SR = uR + cR * np.sqrt((g + 1.0) / (2 * g) * ps / pR + (g - 1.0) / (2 * g))
                if s >= SR:
                    out[:, i] = (rR, uR, pR)
                else:
                    out[:, i] = (rR * (ps / pR + gm) / (gm * ps / pR + 1.0), us, ps)
            else:
                cs = cR * (ps / pR) ** ((g - 1.0) / (2 * g))
                SH, ST = uR + cR, us + cs
                if s >= SH:
                    out[:, i] = (rR, uR, pR)
                elif s <= ST:
                    out[:, i] = (rR * (ps / pR) ** (1.0 / g), us, ps)
                else:
                    fac = 2.0 / (g + 1.0) - gm / cR * (uR - s)
                    out[:, i] = (rR * fac ** (2.0 / (g - 1.0)),
                                 2.0 / (g + 1.0) * (-cR + (g - 1.0) / 2 * uR + s),
                                 pR * fac ** (2 * g / (g - 1.0)))
    return out


def cell_averages(left, right, x0, t, edges, g=1.4, npts=64):
    """Averages of the exact (rho, rho u, E) over the cells [edges[i], edges[i+1]]."""
    gx, gw = np.polynomial.legendre.leggauss(npts)
    out = np.zeros((3, len(edges) - 1))
    for i in range(len(edges) - 1):
        a, b = edges[i], edges[i + 1]
        x = 0.5 * (a + b) + 0.5 * (b - a) * gx
        r, u, p = sample(left, right, (x - x0) / t, g)
        cons = np.stack([r, r * u, p / (g - 1.0) + 0.5 * r * u * u])
        out[:, i] = cons @ (0.5 * gw)
    return out
