"""Helpers of the GPU parity tests: oracle runs in the library's layout,
coefficient layout conversion, tolerances."""
import numpy as np

from oracle.blended import Config, blended_rhs
from oracle.layout import sub_from_elements, sub_to_elements, to_elements, to_grid


def levels(M):
    out, n = [], M
    while n >= 2:
        out.append(n)
        n //= 2
    return out


def oracle_rhs(cfg, u, frozen=None):
    """Oracle R(u) in the element layout, plus its diagnostics."""
    c = Config(**cfg)
    U = to_grid(u, cfg["dim"], cfg["M"], cfg["nel"])
    fz = None if frozen is None else coeffs_to_levels(cfg, frozen)
    R, dg = blended_rhs(U, c, frozen=fz, return_diag=True)
    return to_elements(R, cfg["dim"], cfg["M"], cfg["nel"]), dg


def levels_to_coeffs(cfg, alpha, beta):
    """Per-level grids -> (E, 2, S) coefficient layout of the library."""
    d, M, nel = cfg["dim"], cfg["M"], cfg["nel"]
    a = np.concatenate([sub_to_elements(alpha[n], d, M // n, nel) for n in levels(M)], axis=1)
    b = np.concatenate([sub_to_elements(beta[n], d, M // n, nel) for n in levels(M)], axis=1)
    return np.ascontiguousarray(np.stack([a, b], axis=1))


def coeffs_to_levels(cfg, c):
    d, M, nel = cfg["dim"], cfg["M"], cfg["nel"]
    al, be, off = {}, {}, 0
    for n in levels(M):
        k = (M // n) ** d
        al[n] = sub_from_elements(c[:, 0, off:off + k], d, M // n, nel)
        be[n] = sub_from_elements(c[:, 1, off:off + k], d, M // n, nel)
        off += k
    return al, be


def near_threshold(cfg, dg, tol=1e-10):
    """Elements with a raw alpha within tol of alpha_H / alpha_L, or a beta within
    tol of beta_L, at any level (their decisions may legitimately differ)."""
    d, M, nel = cfg["dim"], cfg["M"], cfg["nel"]
    E = int(np.prod(nel))
    near = np.zeros(E, dtype=bool)
    for n in levels(M):
        ar = sub_to_elements(dg.alpha_raw[n], d, M // n, nel)
        b = sub_to_elements(dg.beta[n], d, M // n, nel)
        near |= np.any((np.abs(ar - cfg["alphaH"]) < tol) | (np.abs(ar - cfg["alphaL"]) < tol)
                       | (np.abs(b - cfg["betaL"]) < tol), axis=1)
    return near


def scaled_error(got, ref):
    """|g - o| / max(|o|, 1e-3 ||o_var||_inf) per entry (the parity metric)."""
    floor = 1e-3 * np.abs(ref).max(axis=(0, 2), keepdims=True)
    return np.abs(got - ref) / np.maximum(np.abs(ref), np.maximum(floor, 1e-300))


def decisions_from_diag(dg):
    lo = np.log2(dg.n_min).astype(int)
    hi = np.log2(dg.n_max).astype(int)
    return (lo | (hi << 4)).astype(np.uint8)


def term_scale(cfg, u):
    """Term scale of every (element, variable): (M / dx_min) times the largest
    sum_a |f_a,v| + lambda |u_v| over the means and over the nodal values of every
    level's reconstruction, in the element and its face neighbours. Every RHS
    entry is a combination, with O(1) operator weights, of terms of this size
    (physical fluxes at means and nodes, and the S u parts of the HLL flux), so two
    FP64 evaluations in a different order differ by ~1e-16 of it, whatever the
    size of the result."""
    from oracle.blended import Config, indicator
    from oracle.euler import max_wave_speed, physical_flux
    d, M, nel = cfg["dim"], cfg["M"], cfg["nel"]
    g = cfg["gamma"]

    def mag_of(q):                                               # q: (nv, ...)
        with np.errstate(all="ignore"):
            lam = max_wave_speed(q, g)
            lam = np.where(np.isfinite(lam), lam, 0.0)
            m = lam[None] * np.abs(q)
            for a in range(d):
                m = m + np.abs(physical_flux(q, a, g))
        return np.where(np.isfinite(m), m, 0.0)

    q = np.moveaxis(np.asarray(u), 1, 0)                          # (nv, E, M^d)
    el = mag_of(q).max(axis=2).T                                  # (E, nv)
    recon = indicator(to_grid(u, d, M, nel), Config(**cfg))[4]
    for n, (ut, _, _) in recon.items():
        nodal = to_elements(mag_of(ut), d, M, nel)                # (E, nv, M^d)
        el = np.maximum(el, nodal.max(axis=2))
    E = el.shape[0]
    idx = np.arange(E)
    coords = [idx % nel[0], (idx // nel[0]) % nel[1]] + ([idx // (nel[0] * nel[1])] if d == 3 else [])
    out = el.copy()
    for ax in range(d):
        for sh in (-1, 1):
            cc = [x.copy() for x in coords]
            cc[ax] = np.clip(cc[ax] + sh, 0, nel[ax] - 1)
            nb = cc[0] + nel[0] * (cc[1] + (nel[1] * cc[2] if d == 3 else 0))
            out = np.maximum(out, el[nb])
    dxmin = min((cfg["xhi"][a] - cfg["xlo"][a]) / nel[a] for a in range(d))
    return (M / dxmin) * out[:, :, None]


def face_neighbours(cfg, flags):
    """flags OR-ed with the flags of the face neighbours (periodic wrap is harmless
    for a test mask)."""
    d, nel = cfg["dim"], cfg["nel"]
    E = len(flags)
    idx = np.arange(E)
    coords = [idx % nel[0], (idx // nel[0]) % nel[1]] + ([idx // (nel[0] * nel[1])] if d == 3 else [])
    out = flags.copy()
    for a in range(d):
        for sh in (-1, 1):
            cc = [x.copy() for x in coords]
            cc[a] = (cc[a] + sh) % nel[a]
            nb = cc[0] + nel[0] * (cc[1] + (nel[1] * cc[2] if d == 3 else 0))
            out |= flags[nb]
    return out


def density_squeezed_active(cfg, dg, coeffs):
    """Elements where a level whose density had to be squeezed (beta_rho < 1) carries
    weight. There the limited density reaches eps = 1e-20 at a point up to rounding,
    and the flux m / rho at that point amplifies a one-ulp change of beta without
    bound (checked: one ulp moves R by O(||R||)), so those elements and their face
    neighbours are counted and left out of the 1e-12 comparison."""
    d, M, nel = cfg["dim"], cfg["M"], cfg["nel"]
    E = int(np.prod(nel))
    rest = np.ones((E, M ** d))
    flag = np.zeros(E, dtype=bool)
    off = 0
    for n in levels(M):
        k = M // n
        a_sub = coeffs[:, 0, off:off + k ** d]
        off += k ** d
        # expand the sub-element alpha to subcells
        A = np.zeros((E, M ** d))
        t = np.arange(M ** d)
        cx, cy = t % M, (t // M) % M
        cz = t // (M * M) if d == 3 else 0 * t
        sub = cx // n + k * (cy // n) + (k * k * (cz // n) if d == 3 else 0)
        A = a_sub[:, sub]
        th = A * rest
        rest = rest * (1.0 - A)
        br = sub_to_elements(dg.beta_rho[n], d, k, nel)[:, sub]
        flag |= np.any((th != 0.0) & (br < 1.0), axis=1)
    return face_neighbours(cfg, flag)


def window(cfg, u, lo, hi, halo):
    """The elements lo[a] - halo <= e_a < hi[a] + halo (clipped at the mesh) as a
    problem of their own: (cfg_w, u_w, inner, glob) with inner the indices, in the
    window's element order, of the elements lo <= e_a < hi and glob their indices
    in the whole mesh. Window sides inside the
    mesh get outflow boundaries; sides on the mesh boundary keep its condition
    (periodic meshes only for windows that stay inside). The right-hand side of an
    element depends on its own means and on the face states of its face neighbours,
    which depend on their own means alone, so the oracle's R on the window is exact
    on elements at least one element away from an artificial side (k stages of an
    RK step: k elements)."""
    d, nel = cfg["dim"], cfg["nel"]
    a0 = [max(0, lo[a] - halo) for a in range(d)]
    a1 = [min(nel[a], hi[a] + halo) for a in range(d)]
    dx = [(cfg["xhi"][a] - cfg["xlo"][a]) / nel[a] for a in range(d)]
    bc = []
    for a in range(d):
        for side, edge in ((0, a0[a] == 0), (1, a1[a] == nel[a])):
            b = cfg["bc"][2 * a + side]
            if edge:
                assert b != 0, "periodic sides must stay outside the window"
                bc.append(b)
            else:
                bc.append(2)
    wn = tuple(a1[a] - a0[a] for a in range(d))
    cw = dict(cfg, nel=wn, bc=tuple(bc), elem_size=tuple(dx),
              xlo=tuple(cfg["xlo"][a] + a0[a] * dx[a] for a in range(d)),
              xhi=tuple(cfg["xlo"][a] + a1[a] * dx[a] for a in range(d)))
    grids = np.meshgrid(*[np.arange(a0[a], a1[a]) for a in range(d)], indexing="ij")
    # element index e = ex + nx (ey + ny ez), window order x fastest
    idx = grids[0] + nel[0] * grids[1] + (nel[0] * nel[1] * grids[2] if d == 3 else 0)
    idx = np.transpose(idx, tuple(range(d))[::-1]).ravel()
    uw = np.ascontiguousarray(np.asarray(u)[idx])
    loc = np.meshgrid(*[np.arange(wn[a]) for a in range(d)], indexing="ij")
    ins = np.ones(loc[0].shape, dtype=bool)
    for a in range(d):
        ins &= (loc[a] + a0[a] >= lo[a]) & (loc[a] + a0[a] < hi[a])
    inner = np.flatnonzero(np.transpose(ins, tuple(range(d))[::-1]).ravel())
    glob = idx[inner]
    return cw, uw, inner, glob


def entry_sensitivity(cfg, u, ref, keep=None, seeds=(1, 2)):
    """Conditioning of the per-entry metric on this input: the largest change, per
    variable, of the oracle's own R in scaled_error units when every input mean is
    perturbed by a random relative amount in {-1, 0, 1} x 2^-52 (one unit in the
    last place), over a few seeds. An evaluation in another order of the same FP64
    arithmetic differs from the oracle by rounding of the same size in its
    intermediate values, so its per-entry error can reach a small multiple of this
    and no less; where the result is a small remainder of large terms (the energy
    right-hand side of a blast at rest, v = 0) this is far above 1e-12."""
    keep = np.ones(len(u), dtype=bool) if keep is None else keep
    out = 0.0
    for sd in seeds:
        rng = np.random.default_rng(sd)
        up = np.asarray(u) * (1.0 + 2.0 ** -52 * rng.integers(-1, 2, size=np.shape(u)))
        rp, _ = oracle_rhs(cfg, up)
        out = np.maximum(out, scaled_error(rp[keep], ref[keep]).max(axis=(0, 2), initial=0.0))
    return out
