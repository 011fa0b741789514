"""Compressible Euler physics and the HLL flux (test infrastructure: oracle).

* Conserved variables u = (rho, rho v_1..rho v_d, E) (eq. comp-euler-conservative).
* Ideal-gas pressure p = (gamma-1) (E - rho |v|^2 / 2) (eq. equation-of-state).
* Permissible states: rho > 0 and p > 0 (Sec. 3.1).
* Interface flux: HLL (Harten, Lax, van Leer) with Einfeldt signal speeds
  (Sec. 3, "HLL approximate Riemann solver with Einfeldt signal speed estimates").
  The paper does not print the speeds; the textbook HLLE form is used:
  Roe averages of the normal velocity and of the enthalpy,
  c_hat^2 = (gamma-1)(H_hat - |v_hat|^2/2), sound speeds sqrt(max(gamma p / rho, 0))
  (a squeezed state targets p = 1e-20, which rounding can leave slightly below
  zero; its sound speed is then 0 rather than NaN),
  S_L = min(v_L - c_L, v_hat - c_hat), S_R = max(v_R + c_R, v_hat + c_hat),
  F = f_L if S_L >= 0, f_R if S_R <= 0, else the HLL average state flux.
* Largest wave speed on mean values (eq. euler-max-eigenvalue).

Arrays carry the variable index on axis 0: u[0] = rho, u[1..d] = momentum,
u[d+1] = E. Direction ``a`` = 0 is x.
"""
import numpy as np


def pressure(u, gamma):
    d = u.shape[0] - 2
    rho = u[0]
    kin = sum(u[1 + k] ** 2 for k in range(d)) / rho
    return (gamma - 1.0) * (u[d + 1] - 0.5 * kin)


def primitives(u, gamma):
    """(rho, v_1..v_d, p) from conserved variables, pointwise."""
    d = u.shape[0] - 2
    rho = u[0]
    out = np.empty_like(u)
    out[0] = rho
    for k in range(d):
        out[1 + k] = u[1 + k] / rho
    out[d + 1] = pressure(u, gamma)
    return out


def conserved(w, gamma):
    """Conserved variables from (rho, v_1..v_d, p)."""
    d = w.shape[0] - 2
    rho = w[0]
    out = np.empty_like(w)
    out[0] = rho
    kin = 0.0
    for k in range(d):
        out[1 + k] = rho * w[1 + k]
        kin = kin + w[1 + k] ** 2
    out[d + 1] = w[d + 1] / (gamma - 1.0) + 0.5 * rho * kin
    return out


def physical_flux(u, a, gamma):
    """Euler flux in direction a: (rho v_a, rho v_a v + p e_a, v_a (E + p))."""
    d = u.shape[0] - 2
    rho = u[0]
    va = u[1 + a] / rho
    p = pressure(u, gamma)
    f = np.empty_like(u)
    f[0] = u[1 + a]
    for k in range(d):
        f[1 + k] = u[1 + k] * va
    f[1 + a] = f[1 + a] + p
    f[d + 1] = va * (u[d + 1] + p)
    return f


def einfeldt_speeds(uL, uR, a, gamma):
    """Signal speed estimates (S_L, S_R) of Einfeldt's HLLE flux in direction a,
    pointwise over trailing axes: Roe averages weighted by sqrt(rho) of the
    velocity and the enthalpy H = (E + p) / rho, c_hat^2 = (gamma-1)(H_hat -
    |v_hat|^2/2), S_L = min(v_L - c_L, v_hat - c_hat), S_R = max(v_R + c_R, v_hat + c_hat)."""
    d = uL.shape[0] - 2
    rhoL, rhoR = uL[0], uR[0]
    pL, pR = pressure(uL, gamma), pressure(uR, gamma)
    vL = [uL[1 + k] / rhoL for k in range(d)]
    vR = [uR[1 + k] / rhoR for k in range(d)]
    cL = np.sqrt(np.maximum(gamma * pL / rhoL, 0.0))
    cR = np.sqrt(np.maximum(gamma * pR / rhoR, 0.0))
    HL = (uL[d + 1] + pL) / rhoL
    HR = (uR[d + 1] + pR) / rhoR
    sL = np.sqrt(rhoL)
    sR = np.sqrt(rhoR)
    vhat = [(sL * vL[k] + sR * vR[k]) / (sL + sR) for k in range(d)]
    Hhat = (sL * HL + sR * HR) / (sL + sR)
    c2hat = (gamma - 1.0) * (Hhat - 0.5 * sum(vh ** 2 for vh in vhat))
    chat = np.sqrt(np.maximum(c2hat, 0.0))
    SL = np.minimum(vL[a] - cL, vhat[a] - chat)
    SR = np.maximum(vR[a] + cR, vhat[a] + chat)
    return SL, SR


def hll_flux(uL, uR, a, gamma):
    """HLL flux with Einfeldt speeds in direction a, pointwise over trailing axes."""
    SL, SR = einfeldt_speeds(uL, uR, a, gamma)
    fL = physical_flux(uL, a, gamma)
    fR = physical_flux(uR, a, gamma)
    with np.errstate(divide="ignore", invalid="ignore"):
        fmid = (SR * fL - SL * fR + SL * SR * (uR - uL)) / (SR - SL)
    return np.where(SL >= 0.0, fL, np.where(SR <= 0.0, fR, fmid))


def max_wave_speed(u, gamma):
    """max over directions of |v_a| + sqrt(gamma p / rho), pointwise (eq. euler-max-eigenvalue)."""
    d = u.shape[0] - 2
    rho = u[0]
    c = np.sqrt(gamma * pressure(u, gamma) / rho)
    lam = np.abs(u[1] / rho) + c
    for k in range(1, d):
        lam = np.maximum(lam, np.abs(u[1 + k] / rho) + c)
    return lam


def mirror(u, a):
    """Reflecting-wall ghost state: normal momentum negated."""
    g = u.copy()
    g[1 + a] = -g[1 + a]
    return g
