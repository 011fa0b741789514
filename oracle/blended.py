"""Multi-level blended DG/FV right-hand side R(u) (test infrastructure: oracle).

Plain FP64 restatement, on the global subcell grid, of
  * Sec. 2.5 single-level blending (common surface flux, eq. dgfv-scheme-1d),
  * Sec. 2.6 multi-level blending (eqs. reco-2nd-order ... multilevel-blending-
    discretizations, subcell-fv-interpolation-operator and the blended interface
    values that follow it),
  * Sec. 2.7 blending factor (eqs. L1-norm-slope, calc-blending-factor),
  * the appendix 3D extension (eqs. 3D-nodal-reconstruction, dgfv-scheme-3d,
    3D-prolongation, 3D-boundary-value-recon, 3D-interface-fluxes,
    3D-blend-interface-fluxes) and the multi-level algorithm sketch,
  * Sec. 3.4 blending weights theta (eq. blending-weights) and the weighted
    blending factor (eq. order-estimate).

Readings of passages the paper leaves open:
  R1 multi-D multi-level face states: at every subcell face, in every direction,
     Ubar = sum_n theta^(n) U^(n), U^(1) the subcell mean, U^(n) the face-mean of the
     beta-limited level-n polynomial (interface value along the direction, subcell
     mean across it).
  R2 face flux: Fbar = sum_n w^(n) F^(n), w^(n) = (theta_L^(n) + theta_R^(n)) / 2,
     F^(1) = f*(Ubar_L, Ubar_R) pointwise, F^(n) = P f*(R Ubar_L R^T, R Ubar_R R^T) P^T
     on transverse level-n blocks; a block whose reconstructed point states are not
     all permissible uses F^(1) instead.
  R3 sigma = h_n^(d-1) sum_dir sum_nodes W_k |d_xi v|_k on the sub-element's own
     Gauss nodes (h_n = n/M), primitives taken pointwise from the unlimited
     reconstruction; a non-finite ratio gives alpha = 0.
  R4 beta is checked at the nodes and at every subcell-face mean value of the
     sub-element in every direction; each ratio in beta is 1 when its minimum is
     >= eps; the pressure ratio is taken on the density-squeezed values, where a
     value whose density rounding left <= 0 counts as pressure -inf (see
     squeeze_beta); a non-permissible sub-element average gives beta = 0.
  R5 snapping: a level snaps to 1 (and ends the loop) only when all its
     sub-elements exceed alpha_H, to 0 only when all are below alpha_L.
  R6 boundary ghosts: wall = mirror of the interior face state (normal momentum
     negated) with the interior theta; outflow = copy; periodic = wrap.
  R7 a level or face candidate whose weight is zero contributes nothing (the
     algorithm sketch skips levels outside n_min..n_max), so values computed for
     a dropped level never enter the result, even when they are not finite.
"""
from dataclasses import dataclass, field

import numpy as np

from .euler import hll_flux, mirror, physical_flux, pressure, primitives
from .ops import level_ops

PERIODIC, WALL, OUTFLOW, HALO = 0, 1, 2, 3


@dataclass
class Config:
    dim: int
    M: int
    nel: tuple                 # elements per direction (x, y[, z])
    xlo: tuple
    xhi: tuple
    bc: tuple                  # (x-lo, x-hi, y-lo, y-hi[, z-lo, z-hi]); 0 periodic, 1 wall, 2 outflow
    gamma: float = 1.4
    tauA: float = 100.0
    tauS: float = 0.05
    alphaH: float = 0.99
    alphaL: float = 0.01
    betaL: float = 0.95
    cfl: float = 0.5
    family: str = "gauss"
    scheme: str = "multi_level"   # or "single_level" (Sec. 2.5, eq. dgfv-scheme-3d)
    elem_size: tuple = None       # element edges when given (a part of a partitioned mesh), else box / nel

    @property
    def nv(self):
        return self.dim + 2

    @property
    def levels(self):
        """DG levels from the top down: M, M/2, ..., 2."""
        out, n = [], self.M
        while n >= 2:
            out.append(n)
            n //= 2
        return out

    @property
    def dx(self):
        if self.elem_size is not None:
            return [float(self.elem_size[a]) for a in range(self.dim)]
        return [(self.xhi[a] - self.xlo[a]) / self.nel[a] for a in range(self.dim)]


# ----------------------------------------------------------------------------
# tensor helpers (the n-mode product of the appendix, applied blockwise)
# ----------------------------------------------------------------------------

def blockwise(X, A, axis, n):
    """n-mode product of X along `axis` with I (x) A: each block of n consecutive
    entries along the axis is mapped by A (K x n) to K entries."""
    X = np.moveaxis(X, axis, -1)
    sh = X.shape
    Xb = X.reshape(sh[:-1] + (sh[-1] // n, n))
    Y = np.einsum("...bj,kj->...bk", Xb, A)
    Y = Y.reshape(sh[:-1] + (sh[-1] // n * A.shape[0],))
    return np.moveaxis(Y, -1, axis)


def block_reduce(X, n, axes, fn):
    """Reduce blocks of n consecutive entries along each of `axes` with fn."""
    for ax in axes:
        X = np.moveaxis(X, ax, -1)
        sh = X.shape
        X = fn(X.reshape(sh[:-1] + (sh[-1] // n, n)), axis=-1)
        X = np.moveaxis(X, -1, ax)
    return X


def expand(S, n, axes):
    """Repeat every entry n times along each of `axes` (sub-element value -> subcells)."""
    for ax in axes:
        S = np.repeat(S, n, axis=ax)
    return S


def weighted(w, X):
    """w * X where w != 0, exactly 0 where w == 0 (reading R7)."""
    with np.errstate(invalid="ignore", over="ignore"):
        return np.where(w != 0.0, w * X, 0.0)


def permissible(u, gamma):
    return (u[0] > 0.0) & (pressure(u, gamma) > 0.0)


def squeeze_beta(avg, points, gamma, n, saxes):
    """Squeezing parameter beta per sub-element (eq. calc-squeezing-parameter,
    reading R4).

    avg: sub-element averages (nv, sub-grid); points: list of arrays (nv, grid)
    of the unlimited values at the checked points (nodes and subcell faces).
    eps = min(1e-20, <rho>, <p>) with <p> = p(<u>).
    Step 1 (density): beta_rho = (<rho> - eps) / (<rho> - rho_min), 1 if rho_min >= eps.
    Step 2 (pressure): p_min over the density-squeezed points
    (1 - beta_rho) <u> + beta_rho u~, beta_p = (<p> - eps) / (<p> - p_min), 1 if
    p_min >= eps. beta = beta_rho * beta_p. Where the unlimited density stays
    >= eps this is exactly the printed min-formula; where it does not, the
    pressure of the unlimited state is meaningless and the pressure ratio is
    taken after the density step, as in the Zhang-Shu procedure the paper cites.
    The density step puts the lowest point at rho = eps = 1e-20 only up to
    rounding; a squeezed point whose density comes out <= 0 is not in the
    permissible set, and its pressure counts as -inf (for rho < 0 the formula
    (gamma-1)(E - |m|^2 / (2 rho)) would instead be large and positive and let
    the point pass). A non-permissible average gives beta = 0."""
    rho_avg = avg[0]
    p_avg = pressure(avg, gamma)
    eps = np.minimum(np.minimum(1e-20, rho_avg), p_avg)
    rho_min = None
    for x in points:
        r = block_reduce(x[0], n, saxes, np.min)
        rho_min = r if rho_min is None else np.minimum(rho_min, r)
    with np.errstate(divide="ignore", invalid="ignore"):
        b_rho = np.where(rho_min >= eps, 1.0, (rho_avg - eps) / (rho_avg - rho_min))
    b_rho = np.minimum(b_rho, 1.0)
    bexp = expand(b_rho, n, saxes)[None]
    aexp = expand(avg, n, [ax + 1 for ax in saxes])
    p_min = None
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        for x in points:
            sq = (1.0 - bexp) * aexp + bexp * x
            # a squeezed point whose density rounding left <= 0 is outside the
            # permissible set: its pressure counts as -inf (reading R4)
            q = block_reduce(np.where(sq[0] > 0.0, pressure(sq, gamma), -np.inf), n, saxes, np.min)
            p_min = q if p_min is None else np.minimum(p_min, q)
        b_p = np.where(p_min >= eps, 1.0, (p_avg - eps) / (p_avg - p_min))
    b_p = np.minimum(b_p, 1.0)
    beta = b_rho * b_p
    bad = ~((rho_avg > 0.0) & (p_avg > 0.0))
    beta = np.where(bad | ~np.isfinite(beta), 0.0, beta)
    return np.maximum(beta, 0.0), b_rho


# ----------------------------------------------------------------------------
# the right-hand side
# ----------------------------------------------------------------------------

@dataclass
class Diagnostics:
    alpha: dict = field(default_factory=dict)       # level n -> per-sub-element alpha (grid of sub-elements)
    beta: dict = field(default_factory=dict)        # level n -> per-sub-element beta
    beta_rho: dict = field(default_factory=dict)    # level n -> density step of beta (1: density not squeezed)
    alpha_raw: dict = field(default_factory=dict)   # before snapping
    sigma: dict = field(default_factory=dict)       # level n -> (nv, sub-element grid)
    theta: dict = field(default_factory=dict)       # level n (1 included) -> per-subcell weight
    abar: np.ndarray = None                         # weighted blending factor per subcell
    n_min: np.ndarray = None                        # per element
    n_max: np.ndarray = None
    dropped_blocks: int = 0                          # DG face candidates replaced by F^(1)
    Fbar: list = None                               # interface fluxes per direction
    nonpermissible_means: int = 0
    boundary_states: dict = field(default_factory=dict)   # (a, side) -> (face states, thetas) of the outer faces


def _grid_axes(cfg):
    d = cfg.dim
    vax = lambda a: d - a        # direction a in arrays with a leading variable axis
    sax = lambda a: d - 1 - a    # direction a in scalar arrays
    return vax, sax


def _element_view(S, cfg, k):
    """(G/n grid) -> (elements..., k^d) per-element view of a sub-element array."""
    d = cfg.dim
    nel = [cfg.nel[a] for a in range(d)][::-1]   # slow -> fast
    sh = []
    for e in nel:
        sh += [e, k]
    X = S.reshape(sh)
    perm = list(range(0, 2 * d, 2)) + list(range(1, 2 * d, 2))
    return X.transpose(perm).reshape(tuple(nel) + (k ** d,))


def _from_element_view(X, cfg, k):
    d = cfg.dim
    nel = [cfg.nel[a] for a in range(d)][::-1]
    X = X.reshape(tuple(nel) + (k,) * d)
    perm = []
    for i in range(d):
        perm += [i, d + i]
    X = X.transpose(perm)
    return X.reshape([e * k for e in nel])


def indicator(U, cfg, ops=None):
    """Steps (I)-(II) of the multi-level sketch: reconstruction, positivity
    squeezing and blending factors per level, then the high-to-low snapping loop.

    Returns (alpha, beta, alpha_raw, sigma, recon, beta_rho) with per-sub-element
    arrays indexed by level, recon[n] = (unlimited nodal values, averages, face
    values) and beta_rho the density step of the squeezing (1: not squeezed)."""
    d, M, g = cfg.dim, cfg.M, cfg.gamma
    vax, sax = _grid_axes(cfg)
    ops = ops or {n: level_ops(n, cfg.family) for n in cfg.levels}
    vaxes = [vax(a) for a in range(d)]
    saxes = [sax(a) for a in range(d)]
    recon, beta, sigma, beta_rho = {}, {}, {}, {}
    for n in cfg.levels:
        o = ops[n]
        ut = U
        for a in range(d):                                   # eq. 3D-nodal-reconstruction
            ut = blockwise(ut, o.R, vax(a), n)
        avg = block_reduce(U, n, vaxes, np.mean)             # eq. element-average
        faces = {}
        for a in range(d):                                   # values at every subcell face
            for side, I in (("-", o.Iminus), ("+", o.Iplus)):
                y = blockwise(ut, I, vax(a), n)              # eq. subcell-fv-interpolation-operator
                for b in range(d):
                    if b != a:
                        y = blockwise(y, o.P, vax(b), n)     # face-mean across (eq. 3D-prolongation)
                faces[(a, side)] = y
        recon[n] = (ut, avg, faces)
        # eq. positivity-limiter-2 / calc-squeezing-parameter at nodes and face values
        beta[n], beta_rho[n] = squeeze_beta(avg, [ut] + list(faces.values()), g, n, saxes)
        # eq. L1-norm-slope on the unlimited polynomial, primitives taken pointwise
        with np.errstate(divide="ignore", invalid="ignore"):
            w = primitives(ut, g)
            Wn = np.ones(())
            for a in range(d - 1, -1, -1):                   # tensor Gauss weights (sum 1 per sub-element)
                Wn = np.multiply.outer(Wn, np.tile(o.w, cfg.nel[a] * M // n))
            s = 0.0
            for a in range(d):
                dw = blockwise(w, o.Dnodal, vax(a), n)
                s = s + block_reduce(np.abs(dw) * Wn, n, vaxes, np.sum)
            sigma[n] = (n / M) ** (d - 1) * s
    alpha_raw = {}
    for n in cfg.levels:
        if n == 2:
            a_n = beta[2].copy()                             # alpha^(2) := beta^(2) (Sec. 2.7)
        else:
            child = block_reduce(sigma[n // 2], 2, vaxes, np.sum)
            s = sigma[n]
            with np.errstate(divide="ignore", invalid="ignore"):
                ratio = np.abs(s - child) / np.maximum(np.maximum(s, child), 1.0)
                a_var = 1.0 - np.clip(cfg.tauA * (ratio - cfg.tauS), 0.0, 1.0)  # eq. calc-blending-factor
            a_var = np.where(np.isfinite(ratio), a_var, 0.0)
            a_n = a_var.min(axis=0)                          # smallest over primitive variables
        a_n = np.where(beta[n] < cfg.betaL, 0.0, a_n)        # beta below beta_L: level dropped
        alpha_raw[n] = a_n
    # high-to-low loop with snapping (appendix multi-level sketch, step II)
    nel_shape = tuple(cfg.nel[a] for a in range(d))[::-1]
    stopped = np.zeros(nel_shape, dtype=bool)
    alpha = {}
    for n in cfg.levels:
        k = M // n
        ae = _element_view(alpha_raw[n], cfg, k).copy()
        ae[stopped] = 0.0                                    # levels never reached
        all_hi = np.all(ae > cfg.alphaH, axis=-1) & ~stopped
        all_lo = np.all(ae < cfg.alphaL, axis=-1) & ~stopped
        ae[all_hi] = 1.0
        ae[all_lo] = 0.0
        stopped |= all_hi
        alpha[n] = _from_element_view(ae, cfg, k)
    if cfg.scheme == "single_level":
        # single-level scheme (Sec. 2.5, sketch of Sec. 2.8): one blending factor per
        # element, from the indicator of the top level; the levels below stay off
        for n in cfg.levels[1:]:
            alpha[n] = np.zeros_like(alpha[n])
    return alpha, beta, alpha_raw, sigma, recon, beta_rho


def blending_weights(alpha, cfg):
    """theta^(n) per subcell (eq. blending-weights, any M): theta^(M) = alpha^(M),
    theta^(n) = alpha^(n) prod_{m>n} (1 - alpha^(m)), theta^(1) = prod_m (1 - alpha^(m))."""
    _, sax = _grid_axes(cfg)
    saxes = [sax(a) for a in range(cfg.dim)]
    theta = {}
    rest = 1.0
    for n in cfg.levels:
        A = expand(alpha[n], n, saxes)
        theta[n] = A * rest
        rest = rest * (1.0 - A)
    theta[1] = rest * np.ones_like(theta[cfg.M])
    return theta


def _interface_states(Up, Um, th_p, th_m, a, cfg, ghost=None):
    """Left/right states and thetas at the G_a + 1 interfaces along direction a
    (neighbour append of Sec. 2.6, reading R6 for physical boundaries).

    Up / Um: blended state at the right / left face of every subcell. A HALO side
    takes its outer state and thetas from ghost[(a, side)] = (U, theta dict): the
    face states of the neighbouring part of a partitioned mesh (the face-centred
    means and blending factors a part exchanges, appendix 3D extension)."""
    vax, sax = _grid_axes(cfg)
    av, asx = vax(a), sax(a)
    lo, hi = cfg.bc[2 * a], cfg.bc[2 * a + 1]
    take = lambda X, i, ax: np.take(X, [i], axis=ax)
    G = Up.shape[av]
    if lo == PERIODIC:
        gL = take(Up, G - 1, av)
        tL = {n: take(t, G - 1, asx) for n, t in th_p.items()}
    elif lo == HALO:
        gL, tL = ghost[(a, 0)]
    else:
        first = take(Um, 0, av)
        gL = mirror(first, a) if lo == WALL else first.copy()
        tL = {n: take(t, 0, asx) for n, t in th_m.items()}
    if hi == PERIODIC:
        gR = take(Um, 0, av)
        tR = {n: take(t, 0, asx) for n, t in th_m.items()}
    elif hi == HALO:
        gR, tR = ghost[(a, 1)]
    else:
        last = take(Up, G - 1, av)
        gR = mirror(last, a) if hi == WALL else last.copy()
        tR = {n: take(t, G - 1, asx) for n, t in th_p.items()}
    UL = np.concatenate([gL, Up], axis=av)
    UR = np.concatenate([Um, gR], axis=av)
    thL = {n: np.concatenate([tL[n], th_p[n]], axis=asx) for n in th_p}
    thR = {n: np.concatenate([th_m[n], tR[n]], axis=asx) for n in th_m}
    return UL, UR, thL, thR


def _apply_surface(Fa, Bhat, axis, n):
    """[I (x) Bhat^(n)]^(0) along `axis`: Fa holds the G+1 interface fluxes; block s
    uses interfaces s*n ... s*n+n (appendix on boundary evaluation operators)."""
    X = np.moveaxis(Fa, axis, -1)
    G = X.shape[-1] - 1
    nb = G // n
    idx = (np.arange(nb)[:, None] * n + np.arange(n + 1)[None, :])
    Xb = X[..., idx]                                          # (..., nb, n+1)
    Y = np.einsum("...bj,kj->...bk", Xb, Bhat).reshape(X.shape[:-1] + (G,))
    return np.moveaxis(Y, -1, axis)


def blended_rhs(U, cfg, frozen=None, return_diag=False, ghost=None):
    """R(u) of the multi-level blended scheme on the global subcell grid.

    U: (nv, G_{d-1}, ..., G_0) subcell means.
    frozen: optional (alpha, beta) dicts level -> per-sub-element arrays; when given
    the indicator is skipped and these (already snapped) values are used.
    ghost: outer face states of HALO sides (see _interface_states); the states of
    this part's own boundary faces are in diag.boundary_states."""
    d, M, g = cfg.dim, cfg.M, cfg.gamma
    vax, sax = _grid_axes(cfg)
    saxes = [sax(a) for a in range(d)]
    ops = {n: level_ops(n, cfg.family) for n in cfg.levels}
    diag = Diagnostics()
    alpha, beta, alpha_raw, sigma, recon, diag.beta_rho = indicator(U, cfg, ops)
    if frozen is not None:
        alpha = {n: np.asarray(frozen[0][n], dtype=np.float64) for n in cfg.levels}
        beta = {n: np.asarray(frozen[1][n], dtype=np.float64) for n in cfg.levels}
    diag.alpha, diag.beta, diag.alpha_raw, diag.sigma = alpha, beta, alpha_raw, sigma
    theta = blending_weights(alpha, cfg)
    diag.theta = theta
    diag.abar = theta[1] + sum(n * theta[n] for n in cfg.levels)   # eq. order-estimate, any M
    # per element level bounds: lowest / highest level with a nonzero weight
    all_levels = [1] + sorted(cfg.levels)
    used = np.stack([_element_view(block_reduce(theta[n] != 0.0, M, saxes, np.any), cfg, 1)[..., 0]
                     for n in all_levels])
    lv = np.array(all_levels)[:, None]
    flat = used.reshape(len(all_levels), -1)
    diag.n_min = np.where(flat, lv, 10 ** 6).min(axis=0)
    diag.n_max = np.where(flat, lv, 0).max(axis=0)
    # beta-limited values (eq. positivity-limiter-applied): (1-beta) <u> + beta u~
    utb, facesb = {}, {}
    for n in cfg.levels:
        ut, avg, faces = recon[n]
        bexp = expand(beta[n], n, saxes)[None]
        aexp = expand(avg, n, [vax(a) for a in range(d)])
        utb[n] = (1.0 - bexp) * aexp + bexp * ut
        facesb[n] = {k: (1.0 - bexp) * aexp + bexp * f for k, f in faces.items()}
    Fbar = []
    for a in range(d):
        av = vax(a)
        # blended state at every subcell face (reading R1)
        Up = weighted(theta[1][None], U)
        Um = weighted(theta[1][None], U)
        for n in sorted(cfg.levels):
            Up = Up + weighted(theta[n][None], facesb[n][(a, "+")])
            Um = Um + weighted(theta[n][None], facesb[n][(a, "-")])
        th = {1: theta[1], **{n: theta[n] for n in cfg.levels}}
        G = Up.shape[av]
        diag.boundary_states[(a, 0)] = (np.take(Um, [0], axis=av), {n: np.take(t, [0], axis=sax(a)) for n, t in th.items()})
        diag.boundary_states[(a, 1)] = (np.take(Up, [G - 1], axis=av),
                                        {n: np.take(t, [G - 1], axis=sax(a)) for n, t in th.items()})
        UL, UR, thL, thR = _interface_states(Up, Um, th, th, a, cfg, ghost)
        with np.errstate(divide="ignore", invalid="ignore"):
            F1 = hll_flux(UL, UR, a, g)
        F = weighted(0.5 * (thL[1] + thR[1])[None], F1)
        for n in sorted(cfg.levels):
            o = ops[n]
            w_n = 0.5 * (thL[n] + thR[n])[None]
            rL, rR = UL, UR
            others = [b for b in range(d) if b != a]
            for b in others:                                  # eq. 3D-boundary-value-recon
                rL = blockwise(rL, o.R, vax(b), n)
                rR = blockwise(rR, o.R, vax(b), n)
            ok = permissible(rL, g) & permissible(rR, g)
            ok_blk = expand(block_reduce(ok, n, [sax(b) for b in others], np.all), n, [sax(b) for b in others])
            with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
                Fn = hll_flux(rL, rR, a, g)                  # eq. 3D-interface-fluxes
            for b in others:
                Fn = blockwise(Fn, o.P, vax(b), n)           # P f* P^T (eq. 3D-blend-interface-fluxes)
            Fn = np.where(ok_blk[None], Fn, F1)
            diag.dropped_blocks += int((~ok_blk).sum() // max(1, n ** (d - 1)))
            F = F + weighted(w_n, Fn)
        if cfg.scheme == "single_level":
            # inner subcell interfaces: the flux of the raw subcell means (eq.
            # assemble-boundary-values / common-surface-flux; the inner interface
            # fluxes of the 3D form); element faces keep the blend above
            G = U.shape[av]
            with np.errstate(divide="ignore", invalid="ignore"):
                Fi = hll_flux(np.take(U, np.arange(G - 1), axis=av), np.take(U, np.arange(1, G), axis=av), a, g)
            k = np.arange(1, G)
            inner = k[k % M != 0]
            F = np.moveaxis(F, av, -1).copy()
            F[..., inner] = np.moveaxis(Fi, av, -1)[..., inner - 1]
            F = np.moveaxis(F, -1, av)
        Fbar.append(F)
    # level right-hand sides and their blend (eq. multilevel-blending-scheme, dgfv-scheme-3d)
    rhs1 = 0.0
    for a in range(d):
        rhs1 = rhs1 - (M / cfg.dx[a]) * np.diff(Fbar[a], axis=vax(a))
    R = weighted(theta[1][None], rhs1)
    for n in sorted(cfg.levels):
        o = ops[n]
        rhs_n = 0.0
        for a in range(d):
            vol = blockwise(physical_flux(utb[n], a, g), o.Dhat, vax(a), n)
            for b in range(d):
                if b != a:
                    vol = blockwise(vol, o.P, vax(b), n)
            surf = _apply_surface(Fbar[a], o.Bhat, vax(a), n)
            rhs_n = rhs_n + ((M / n) / cfg.dx[a]) * (vol - surf)
        R = R + weighted(theta[n][None], rhs_n)
    diag.nonpermissible_means = int((~permissible(U, g)).sum())
    diag.Fbar = Fbar
    if return_diag:
        return R, diag
    return R
