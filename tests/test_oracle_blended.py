"""Pins of the oracle's blended right-hand side against what the paper fixes:
the FV and DG limits (Sec. 2.5 remark), forced intermediate levels (brute-force
sub-element DGSEM), free-stream preservation, discrete conservation for
arbitrary blending factors (Sec. 2.5 lemma, Sec. 3.3), the unit sum of the
blending weights (eq. blending-weights-unit-property), the limits of the
weighted blending factor (eq. order-estimate), mirror / transpose symmetry, and
the indicator on a linear ramp and on a step."""
import numpy as np
import pytest

from oracle.blended import Config, blended_rhs, indicator
from oracle.euler import conserved, pressure
from oracle.plain_dgsem import projected_dgsem_rhs
from oracle.plain_fv import fv_rhs
from tests._oracle_cases import cfg2, cfg3, frozen, smooth_state


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


CASES = [
    ("2d_M4_wall", lambda: cfg2(M=4, bc=(1, 1, 1, 1))),
    ("2d_M8_periodic_outflow", lambda: cfg2(M=8, nel=(2, 2), bc=(0, 0, 2, 2))),
    ("3d_M4_mixed", lambda: cfg3(M=4)),
]


@pytest.mark.parametrize("name,mk", CASES)
def test_alpha_zero_is_subcell_fv(name, mk):
    cfg = mk()
    U = smooth_state(cfg, seed=3, noise=0.05)
    R = blended_rhs(U, cfg, frozen=frozen(cfg, lambda n: 0.0))
    assert rel(R, fv_rhs(U, cfg)) < 1e-13


@pytest.mark.parametrize("name,mk", CASES)
def test_top_level_is_projected_dgsem(name, mk):
    cfg = mk()
    U = smooth_state(cfg, seed=4)
    R = blended_rhs(U, cfg, frozen=frozen(cfg, lambda n: 1.0 if n == cfg.M else "random", seed=5))
    assert rel(R, projected_dgsem_rhs(U, cfg, cfg.M)) < 1e-12


@pytest.mark.parametrize("name,mk", CASES)
def test_forced_intermediate_level_is_subelement_dgsem(name, mk):
    cfg = mk()
    U = smooth_state(cfg, seed=6)
    for n in cfg.levels[1:]:
        fz = frozen(cfg, lambda m: 1.0 if m == n else (0.0 if m > n else "random"), seed=n)
        R = blended_rhs(U, cfg, frozen=fz)
        assert rel(R, projected_dgsem_rhs(U, cfg, n)) < 1e-12, n


@pytest.mark.parametrize("name,mk", CASES)
def test_free_stream_with_random_blending(name, mk):
    cfg = mk()
    G = [cfg.nel[a] * cfg.M for a in range(cfg.dim)][::-1]
    w = np.empty((cfg.nv,) + tuple(G))
    w[0], w[-1] = 1.3, 0.7
    for k in range(cfg.dim):
        w[1 + k] = 0.0 if cfg.bc[2 * k] == 1 else 0.3 + 0.1 * k   # walls need v_n = 0
    U = conserved(w, cfg.gamma)
    rng = np.random.default_rng(7)
    al, be = frozen(cfg, lambda n: "random", seed=8)
    be = {n: rng.uniform(0.95, 1.0, b.shape) for n, b in be.items()}
    R = blended_rhs(U, cfg, frozen=(al, be))
    assert np.abs(R).max() < 1e-12


@pytest.mark.parametrize("M,d", [(4, 2), (8, 2), (4, 3)])
def test_conservation_with_random_blending_each_stage(M, d):
    """Periodic mesh, blending factors drawn at random per sub-element and level
    (the stress test of Sec. 3.3): the change of bulk (eq. change-of-bulk) is at
    FP64 roundoff."""
    if d == 2:
        cfg = Config(dim=2, M=M, nel=(3, 2), xlo=(0, 0), xhi=(1.5, 1.0), bc=(0,) * 4)
    else:
        cfg = Config(dim=3, M=M, nel=(2, 2, 2), xlo=(0, 0, 0), xhi=(1, 1, 1), bc=(0,) * 6)
    U = smooth_state(cfg, seed=9, noise=0.1)
    for stage in range(3):
        al, _ = frozen(cfg, lambda n: "random", seed=10 + stage)
        be = indicator(U, cfg)[1]                             # squeezing keeps face states permissible
        R = blended_rhs(U, cfg, frozen=(al, be))
        bulk = R.reshape(cfg.nv, -1).sum(axis=1) / cfg.M ** d
        scale = np.abs(R).reshape(cfg.nv, -1).sum(axis=1) / cfg.M ** d
        assert np.all(np.abs(bulk) <= 1e-13 * scale), (bulk, scale)


def test_conservation_with_indicator_on_shock_state():
    cfg = Config(dim=2, M=8, nel=(3, 3), xlo=(0, 0), xhi=(1, 1), bc=(0,) * 4)
    U = smooth_state(cfg, seed=11)
    U[:, 8:20, 5:13] *= 3.0                                  # strong discontinuities
    R, dg = blended_rhs(U, cfg, return_diag=True)
    assert (dg.n_min < cfg.M).any()                           # blending really active
    bulk = R.reshape(cfg.nv, -1).sum(axis=1)
    assert np.all(np.abs(bulk) <= 1e-13 * np.abs(R).reshape(cfg.nv, -1).sum(axis=1))


def test_theta_sums_to_one_and_abar_limits():
    cfg = cfg2(M=8, nel=(2, 2))
    U = smooth_state(cfg, seed=12)
    _, dg = blended_rhs(U, cfg, frozen=frozen(cfg, lambda n: "random", seed=13), return_diag=True)
    total = sum(dg.theta.values())
    assert np.abs(total - 1.0).max() < 1e-15
    _, dg0 = blended_rhs(U, cfg, frozen=frozen(cfg, lambda n: 0.0), return_diag=True)
    _, dg1 = blended_rhs(U, cfg, frozen=frozen(cfg, lambda n: 1.0), return_diag=True)
    assert np.all(dg0.abar == 1.0) and np.all(dg1.abar == cfg.M)
    assert np.all(dg0.n_min == 1) and np.all(dg0.n_max == 1)
    assert np.all(dg1.n_min == cfg.M) and np.all(dg1.n_max == cfg.M)


def _mirror_x(X, cfg, vector=True):
    Y = np.flip(X, axis=-1).copy()
    if vector:
        Y[1] = -Y[1]
    return Y


@pytest.mark.parametrize("M", [4, 8])
def test_mirror_symmetry(M):
    """x -> -x with symmetric walls: R(mirror u) = mirror R(u). A swapped I+/I-,
    b+/b- or a wrong surface column breaks this."""
    cfg = Config(dim=2, M=M, nel=(3, 2), xlo=(-1, 0), xhi=(1, 1), bc=(1, 1, 1, 1))
    U = smooth_state(cfg, seed=14, noise=0.2)
    R = blended_rhs(U, cfg)
    Rm = blended_rhs(_mirror_x(U, cfg), cfg)
    assert rel(Rm, _mirror_x(R, cfg)) < 1e-12


def test_transpose_symmetry():
    cfg = Config(dim=2, M=8, nel=(2, 2), xlo=(0, 0), xhi=(1, 1), bc=(1, 2, 1, 2))
    U = smooth_state(cfg, seed=15, noise=0.3)
    sw = lambda X: np.swapaxes(X, 1, 2)[[0, 2, 1, 3]]
    assert rel(blended_rhs(sw(U), cfg), sw(blended_rhs(U, cfg))) < 1e-12


def test_periodic_translation_by_one_element():
    cfg = Config(dim=2, M=4, nel=(3, 3), xlo=(0, 0), xhi=(1, 1), bc=(0,) * 4)
    U = smooth_state(cfg, seed=16, noise=0.3)
    sh = lambda X: np.roll(X, 4, axis=-1)
    assert rel(blended_rhs(sh(U), cfg), sh(blended_rhs(U, cfg))) < 1e-13


def test_indicator_linear_ramp_keeps_full_order():
    """A linear profile is reproduced exactly by every level, so sigma^(n) equals
    the sum over its children and alpha = 1 (tau_S > 0, Sec. 2.7)."""
    cfg = Config(dim=2, M=8, nel=(2, 2), xlo=(0, 0), xhi=(1, 1), bc=(2,) * 4)
    G = 16
    x = (np.arange(G) + 0.5) / G
    w = np.zeros((4, G, G))
    w[0] = 1.0 + 0.5 * x[None, :] + 0.25 * x[:, None]
    w[1], w[2], w[3] = 0.3, -0.2, 1.0
    U = conserved(w, cfg.gamma)
    alpha, beta, alpha_raw, _, _, _ = indicator(U, cfg)
    for n in cfg.levels:
        assert np.all(alpha_raw[n] == 1.0) or np.abs(alpha_raw[n] - 1).max() < 1e-12
        assert np.all(beta[n] == 1.0)
    assert np.all(alpha[cfg.M] == 1.0)


def test_indicator_step_drops_top_level():
    cfg = Config(dim=2, M=8, nel=(2, 2), xlo=(0, 0), xhi=(1, 1), bc=(2,) * 4)
    w = np.zeros((4, 16, 16))
    w[0], w[3] = 1.0, 1.0
    w[0][:, 11:] = 0.3                                        # a density step inside element x=1
    U = conserved(w, cfg.gamma)
    alpha, _, alpha_raw, _, _, _ = indicator(U, cfg)
    assert alpha_raw[8][0, 1] == 0.0 and alpha[8][0, 1] == 0.0
    assert alpha[8][0, 0] == 1.0                              # the smooth element keeps full order


def _cubic_means(c):
    """Subcell means of c * y^3 over the four quarters of y in [-1/2, 1/2]:
    (b^4 - a^4) / (4 (b - a)) = c * (-15, -1, 1, 15) / 256."""
    return c * np.array([-15.0, -1.0, 1.0, 15.0]) / 256.0


@pytest.mark.parametrize("two_d", [False, True])
def test_blending_factor_inside_the_transition_band_closed_form(two_d):
    """eqs. L1-norm-slope and calc-blending-factor evaluated by hand inside the band.

    M = 4; every element holds the subcell means of rho = 1 + c y^3 (y the element's
    reference coordinate along x in [-1/2, 1/2]), v = 0, p = 1; with two_d the
    same cubic is added along the other axis as well. The degree-3 reconstruction
    reproduces the cubic, so sigma^(4) = its total variation along each axis: c/4
    per axis. A level-2 child reproduces the linear function through its two means,
    whose total variation is twice their difference: 2 (14 c / 256) per child, so the
    children sum to 7 c / 32 per axis (in 2D the children's factor n/M = 1/2 and the
    two children across each axis give the same sum). For c/4 per axis below 1 the
    ratio of eq. calc-blending-factor is (c/32 per axis) / 1; c = 1.76 in 1D form
    (0.88 per axis in 2D) puts it at 0.055, inside (tau_S, tau_S + 1/tau_A) =
    (0.05, 0.06): alpha^(4) = 1 - 100 (0.055 - 0.05) = 0.5, not snapped (between
    alpha_L and alpha_H). v and p are constant (sigma = 0, alpha = 1), so the
    minimum over the primitive variables is rho's."""
    cfg = Config(dim=2, M=4, nel=(2, 2), xlo=(0, 0), xhi=(1, 1), bc=(2,) * 4)
    c = 0.88 if two_d else 1.76
    mx = np.tile(_cubic_means(c), 2)                        # both elements along x
    w = np.zeros((4, 8, 8))
    w[0] = 1.0 + mx[None, :] + (mx[:, None] if two_d else 0.0)
    w[3] = 1.0
    U = conserved(w, cfg.gamma)
    alpha, beta, alpha_raw, sigma, _, _ = indicator(U, cfg)
    per_axis = 2 if two_d else 1
    assert np.allclose(sigma[4][0], per_axis * c / 4, rtol=0, atol=1e-13)          # density, every element
    children = sigma[2][0].reshape(2, 2, 2, 2).sum(axis=(1, 3))    # [element y][element x]
    assert np.allclose(children, per_axis * 7 * c / 32, rtol=0, atol=1e-13)
    assert np.all(beta[4] == 1.0) and np.all(beta[2] == 1.0)
    assert np.abs(alpha_raw[4] - 0.5).max() < 1e-11
    assert np.abs(alpha[4] - 0.5).max() < 1e-11


def test_blending_factor_inside_the_transition_band_closed_form_3d():
    """The 1D-form in-band case of eqs. L1-norm-slope / calc-blending-factor in 3D
    (reading R3 with d = 3): rho = 1 + c y^3 along x in every M = 4 element, c = 1.76.
    sigma^(4) = c/4 (factor (4/4)^2 = 1); each of the eight level-2 children carries
    (2/4)^2 = 1/4 of the total variation of its line, four children per half along x,
    so the children sum to the 1D value 7c/32 again, and alpha^(4) = 0.5."""
    cfg = Config(dim=3, M=4, nel=(2, 1, 1), xlo=(0, 0, 0), xhi=(1, 0.5, 0.5), bc=(2,) * 6)
    c = 1.76
    mx = np.tile(_cubic_means(c), 2)
    w = np.zeros((5, 4, 4, 8))
    w[0] = 1.0 + mx[None, None, :]
    w[4] = 1.0
    U = conserved(w, cfg.gamma)
    alpha, beta, alpha_raw, sigma, _, _ = indicator(U, cfg)
    assert np.allclose(sigma[4][0], c / 4, rtol=0, atol=1e-13)
    children = sigma[2][0].reshape(1, 2, 1, 2, 2, 2).sum(axis=(1, 3, 5))
    assert np.allclose(children, 7 * c / 32, rtol=0, atol=1e-13)
    assert np.abs(alpha_raw[4] - 0.5).max() < 1e-11 and np.abs(alpha[4] - 0.5).max() < 1e-11


def test_mixed_level_face_fluxes_closed_form():
    """Readings R1 / R2 (multi-D face states and candidate fluxes of mixed-level
    elements) against a construction by hand, with numpy polynomial fits instead of
    the oracle's operator matrices.

    One M = 4 element, frozen factors alpha^(4) = 0.6, alpha^(2) = 1 on the two level-2
    sub-elements of the left half (x) and 1/2 on those of the right half, beta = 1:
    theta^(4, 2, 1) = (0.6, 0.4, 0) left and (0.6, 0.2, 0.2) right. rho = 1 + c X^2 + e Y
    on the reference square [-1/2, 1/2]^2, v = (1/2, 0), p = 1, so every conserved
    variable is an affine function of rho. At the inner x-interfaces X_k = -1/2 + k/4:
      * level 4 reproduces the data: face value 1 + c X_k^2 + e Y;
      * a level-2 sub-element (2 x 2 subcells) is the bilinear polynomial with its
        four subcell means, here the line through its two x-means (at the subcell
        centres) plus e Y;
      * the FV level contributes the subcell mean;
      * U = sum_n theta^(n) U^(n), from the subcell left (its right face) and right
        (its left face) of the interface, as a face mean over each transverse subcell;
      * candidate 1: the HLL flux of those face means; candidate n >= 2: the point
        values of U at the level-n Gauss nodes of each transverse block (exact, U
        being linear in Y), the HLL flux there, then the subcell means of the
        interpolant through those nodal fluxes;
      * flux = sum_n w^(n) F^(n), w^(n) = (theta_L^(n) + theta_R^(n)) / 2.
    The HLL flux is the oracle's (pinned by its own tests), used as a library step."""
    from oracle.euler import hll_flux
    cfg = Config(dim=2, M=4, nel=(1, 1), xlo=(0, 0), xhi=(1, 1), bc=(1,) * 4)
    g = cfg.gamma
    c, e = 0.8, 0.3
    h = 0.25
    cen = -0.5 + h * (np.arange(4) + 0.5)                      # subcell centres (X or Y)
    lo_, hi_ = cen - h / 2, cen + h / 2
    mx2 = (hi_ ** 3 - lo_ ** 3) / (3 * h)                     # subcell means of X^2
    w = np.zeros((4, 4, 4))
    w[0] = 1.0 + c * mx2[None, :] + e * cen[:, None]          # [j (y)][i (x)]
    w[1], w[2], w[3] = 0.5, 0.0, 1.0
    U = conserved(w, g)

    def state(rho):                                           # conserved state of rho (affine)
        rho = np.asarray(rho, dtype=float)
        return np.stack([rho, 0.5 * rho, 0.0 * rho, 1.0 / (g - 1) + 0.125 * rho])

    def fit2(i, X):                                           # level-2 line in x of the sub-element of subcell i
        i0 = 2 * (i // 2)
        m0, m1 = 1.0 + c * mx2[i0], 1.0 + c * mx2[i0 + 1]
        return m0 + (m1 - m0) * (X - cen[i0]) / h

    theta = {i: ((0.6, 0.4, 0.0) if i < 2 else (0.6, 0.2, 0.2)) for i in range(4)}   # (theta4, theta2, theta1)
    al = {4: np.full((1, 1), 0.6), 2: np.array([[1.0, 0.5], [1.0, 0.5]])}
    be = {4: np.ones((1, 1)), 2: np.ones((2, 2))}
    _, dg = blended_rhs(U, cfg, frozen=(al, be), return_diag=True)
    assert np.allclose(dg.theta[2][0], [0.4, 0.4, 0.2, 0.2]) and np.allclose(dg.theta[1][0], [0, 0, 0.2, 0.2])
    Fx = dg.Fbar[0]                                           # (nv, G_y, G_x + 1)
    for k in (1, 2, 3):
        Xk = -0.5 + k * h

        def rho_face(i, Y):                                    # U of subcell i at X_k, at height Y
            t4, t2, t1 = theta[i]
            return t4 * (1.0 + c * Xk ** 2 + e * Y) + t2 * (fit2(i, Xk) + e * Y) + t1 * (1.0 + c * mx2[i] + e * Y)
        wts = [(theta[k - 1][q] + theta[k][q]) / 2 for q in range(3)]
        expect = wts[2] * hll_flux(state(rho_face(k - 1, cen)), state(rho_face(k, cen)), 0, g)
        for n, wn in ((4, wts[0]), (2, wts[1])):
            nodes = np.polynomial.legendre.leggauss(n)[0]
            for b in range(4 // n):                           # transverse blocks of n subcells
                Yn = -0.5 + b * n * h + n * h * (nodes + 1) / 2
                Fn = hll_flux(state(rho_face(k - 1, Yn)), state(rho_face(k, Yn)), 0, g)
                for v in range(4):
                    P = np.polyint(np.polyfit(Yn, Fn[v], n - 1))   # interpolant through the nodal fluxes
                    for j in range(b * n, (b + 1) * n):
                        expect[v, j] += wn * (np.polyval(P, hi_[j]) - np.polyval(P, lo_[j])) / h
        got = Fx[:, :, k]
        assert np.abs(got - expect).max() < 1e-13 * np.abs(expect).max(), (k, got - expect)


def test_positivity_squeeze_makes_checked_points_permissible():
    cfg = Config(dim=2, M=8, nel=(1, 1), xlo=(0, 0), xhi=(1, 1), bc=(2,) * 4)
    w = np.zeros((4, 8, 8))
    w[0], w[3] = 1.0, 1.0
    w[0][3, 4] = 1e-3
    w[3][3, 4] = 1e-4
    U = conserved(w, cfg.gamma)
    _, beta, _, _, recon, _ = indicator(U, cfg)
    assert beta[8][0, 0] < 1.0
    ut, avg, faces = recon[8]
    b = beta[8][0, 0]
    eps = min(1e-20, avg[0].min(), pressure(avg, cfg.gamma).min())
    for vals in [ut] + list(faces.values()):
        lim = (1 - b) * avg[:, :, :] + b * vals
        assert lim[0].min() >= eps * (1 - 1e-12) - 1e-15
        assert pressure(lim, cfg.gamma).min() >= -1e-14


@pytest.mark.parametrize("variable", ["density", "pressure"])
def test_squeezing_parameter_closed_form(variable):
    """eqs. positivity-limiter-2 / calc-squeezing-parameter by hand. One variable is
    q = a + b X along x (X in [-1/2, 1/2] on the element, a = 0.3, b = 0.64): the
    density (v = 0, E = 2.5), or the pressure (rho = 1, v = 0, E = q / (gamma - 1)).
    Every level reproduces the line; its lowest checked point in a sub-element is the
    value at the sub-element's left face, a - b/2 = -0.02 for the sub-elements
    touching X = -1/2, while every subcell mean stays positive (a - 7b/16 = 0.02).
    The step of that variable gives beta = (<q> - eps) / (<q> - q_min), eps = 1e-20:
    0.3 / 0.32 = 0.9375 for the element (level 8), 0.14 / 0.16 = 0.875 for the left
    level-4 sub-elements, 0.06 / 0.08 = 0.75 for the left level-2 column, and 1 for
    every other sub-element. The density case is checked on the density step alone:
    it puts the lowest point at rho = eps only up to rounding, where reading R4 may
    still take the final beta to 0 (the pressure step of that point); the pressure
    case is linear in beta (rho = 1, no momentum), so its step is the final beta."""
    cfg = Config(dim=2, M=8, nel=(1, 1), xlo=(0, 0), xhi=(1, 1), bc=(2,) * 4)
    a, b = 0.3, 0.64
    X = -0.5 + (np.arange(8) + 0.5) / 8
    q = a + b * X[None, :] + np.zeros((8, 1))
    U = np.zeros((4, 8, 8))
    if variable == "density":
        U[0], U[3] = q, 2.5
    else:
        U[0], U[3] = 1.0, q / (cfg.gamma - 1.0)
    _, beta, _, _, _, beta_rho = indicator(U, cfg)
    got = beta_rho if variable == "density" else beta
    assert abs(got[8][0, 0] - 0.9375) < 1e-12
    assert np.abs(got[4][:, 0] - 0.875).max() < 1e-12 and np.all(got[4][:, 1] == 1.0)
    assert np.abs(got[2][:, 0] - 0.75).max() < 1e-12 and np.all(got[2][:, 1:] == 1.0)
    if variable == "pressure":
        assert all(np.all(beta_rho[n] == 1.0) for n in cfg.levels)


def test_two_step_squeeze_is_the_printed_formula_when_density_is_not_squeezed():
    """Reading R4 claims: where the density needs no squeezing (every checked
    density >= eps), the two-step beta equals eq. calc-squeezing-parameter as
    printed, beta = min((<rho> - eps)/(<rho> - rho_min), (<p> - eps)/(<p> - p_min), 1)
    with p_min the pressure minimum over the unlimited points. Checked on 300 seeded
    sub-elements of two points each, positive densities and pressures that dip below
    zero at some points; and shown to differ from it where the density is squeezed."""
    from oracle.blended import squeeze_beta
    rng = np.random.default_rng(7)
    K, g = 300, 1.4
    avg = np.zeros((4, K, 1))
    pts = [np.zeros((4, K, 1)) for _ in range(2)]
    avg[0, :, 0] = rng.uniform(0.5, 2.0, K)
    avg[1, :, 0] = rng.uniform(-0.5, 0.5, K)
    avg[2, :, 0] = rng.uniform(-0.5, 0.5, K)
    avg[3, :, 0] = rng.uniform(1.0, 3.0, K)
    for x in pts:
        x[0] = avg[0] * rng.uniform(0.3, 1.7, (K, 1))
        x[1] = avg[1] + rng.uniform(-0.3, 0.3, (K, 1))
        x[2] = avg[2] + rng.uniform(-0.3, 0.3, (K, 1))
        x[3] = avg[3] * rng.uniform(-0.2, 1.2, (K, 1))
    beta, b_rho = squeeze_beta(avg, pts, g, 1, [0, 1])
    assert np.all(b_rho == 1.0)
    p = lambda u: (g - 1.0) * (u[3] - 0.5 * (u[1] ** 2 + u[2] ** 2) / u[0])
    eps = np.minimum(np.minimum(1e-20, avg[0]), p(avg))
    rmin = np.minimum(pts[0][0], pts[1][0])
    pmin = np.minimum(p(pts[0]), p(pts[1]))
    tr = np.where(rmin >= eps, 1.0, (avg[0] - eps) / (avg[0] - rmin))
    tp = np.where(pmin >= eps, 1.0, (p(avg) - eps) / (p(avg) - pmin))
    printed = np.minimum(np.minimum(tr, tp), 1.0)
    assert (printed < 1.0).sum() > 50                          # the pressure step is exercised
    assert np.abs(beta - printed).max() < 1e-15
    # density squeezed: the two-step value is below the printed one (its pressure
    # minimum is taken after the density step)
    pts[0][0, :5] = -0.2 * avg[0, :5]
    beta2, b_rho2 = squeeze_beta(avg, pts, g, 1, [0, 1])
    assert np.all(b_rho2[:5] < 1.0)


def test_squeeze_rejects_points_left_at_nonpositive_density():
    """Sec. 2.4 two-step squeezing, reading R4: the density step puts the lowest
    checked point at rho = eps = 1e-20 only up to rounding, and with momentum there
    that point has a hugely negative pressure, so the pressure step must take beta
    to ~0. When rounding leaves the squeezed density <= 0, the pressure formula
    turns large and positive instead; such a point is outside the permissible set
    and must still squeeze. A sweep of 400 (average, point) pairs lands on both
    sides of 0 (checked below), and every beta must be ~0."""
    from oracle.blended import squeeze_beta
    K = 400
    k = np.arange(K)
    avg = np.zeros((4, K, 1))
    pt = np.zeros((4, K, 1))
    avg[0, :, 0] = 0.2 + 1e-3 * k
    avg[1, :, 0] = 0.01
    avg[3, :, 0] = 1.0
    pt[0, :, 0] = -0.1 - 1.7e-4 * k
    pt[1, :, 0] = 0.05
    pt[2, :, 0] = -0.02
    pt[3, :, 0] = 0.8
    beta, b_rho = squeeze_beta(avg, [pt], 1.4, 1, [0, 1])
    sq = (1 - b_rho) * avg[0] + b_rho * pt[0]
    assert (sq < 0).sum() > 50 and (sq > 0).sum() > 50
    assert np.all(b_rho < 0.8) and beta.max() < 1e-10


def _single_level_direct_2d(U, cfg, alpha_el):
    """Eq. dgfv-scheme-3d in 2D (the single-level scheme of Sec. 2.5 in its
    tensor-product form), written element by element for a periodic mesh:
    face-centred means of eq. 3D-prolongation, candidate fluxes of eq.
    3D-interface-fluxes blended with the mean alpha of the two elements (eq.
    3D-blend-interface-fluxes), inner interfaces with the flux of the raw means."""
    from oracle.euler import hll_flux, physical_flux
    from oracle.ops import level_ops
    M, g = cfg.M, cfg.gamma
    o = level_ops(M, cfg.family)
    nx, ny = cfg.nel
    dx, dy = cfg.dx
    E = U.reshape(4, ny, M, nx, M).transpose(0, 1, 3, 2, 4)          # (v, ey, ex, iy, ix)
    A = alpha_el[None, :, :, None]                                     # (1, ey, ex, 1)
    ut = np.einsum("aj,bk,vqejk->vqeab", o.R, o.R, E)                  # nodal values (v, ey, ex, y, x)
    # face-centred means at the four element faces, per transverse subcell
    xm = (1 - A) * E[..., :, 0] + A * np.einsum("ia,vqeak,k->vqei", o.P, ut, o.bminus)
    xp = (1 - A) * E[..., :, -1] + A * np.einsum("ia,vqeak,k->vqei", o.P, ut, o.bplus)
    ym = (1 - A) * E[..., 0, :] + A * np.einsum("kb,vqeab,a->vqek", o.P, ut, o.bminus)
    yp = (1 - A) * E[..., -1, :] + A * np.einsum("kb,vqeab,a->vqek", o.P, ut, o.bplus)

    def face_flux(UL, UR, aL, aR, d):
        F1 = hll_flux(UL, UR, d, g)
        Fn = np.einsum("ia,v...a->v...i", o.P, hll_flux(np.einsum("ai,v...i->v...a", o.R, UL),
                                                        np.einsum("ai,v...i->v...a", o.R, UR), d, g))
        ab = 0.5 * (aL + aR)[None, ..., None]
        return (1 - ab) * F1 + ab * Fn

    # x: fstar (v, ey, ex, iy, M+1); face k=0 of element ex is shared with ex-1
    fx = np.empty(E.shape[:4] + (M + 1,))
    left = face_flux(np.roll(xp, 1, axis=2), xm, np.roll(alpha_el, 1, axis=1), alpha_el, 0)
    fx[..., 0] = left
    fx[..., M] = np.roll(left, -1, axis=2)
    fx[..., 1:M] = hll_flux(E[..., :-1], E[..., 1:], 0, g)
    fy = np.empty(E.shape[:3] + (M, M + 1))                           # (v, ey, ex, ix, M+1)
    low = face_flux(np.roll(yp, 1, axis=1), ym, np.roll(alpha_el, 1, axis=0), alpha_el, 1)
    fy[..., 0] = low
    fy[..., M] = np.roll(low, -1, axis=1)
    fy[..., 1:M] = np.swapaxes(hll_flux(E[..., :-1, :], E[..., 1:, :], 1, g), -1, -2)
    # x-direction terms: (1 - alpha) FV difference and alpha (volume - surface)
    fv_x = -(M / dx) * np.diff(fx, axis=-1)
    vol_x = np.einsum("ia,bk,vqeak->vqeib", o.P, o.Dhat, physical_flux(ut, 0, g))
    sur_x = np.einsum("bk,vqeik->vqeib", o.Bhat, fx)
    fv_y = -(M / dy) * np.swapaxes(np.diff(fy, axis=-1), -1, -2)
    vol_y = np.einsum("kb,ia,vqeab->vqeik", o.P, o.Dhat, physical_flux(ut, 1, g))
    sur_y = np.einsum("ia,vqeka->vqeik", o.Bhat, fy)
    A5 = A[..., None]
    R = (1 - A5) * (fv_x + fv_y) + A5 * ((vol_x - sur_x) / dx + (vol_y - sur_y) / dy)
    return R.transpose(0, 1, 3, 2, 4).reshape(U.shape)


@pytest.mark.parametrize("M", [4, 8])
def test_single_level_scheme_is_eq_dgfv_scheme_3d(M):
    """Single-level scheme (Sec. 2.5; its tensor-product form eq. dgfv-scheme-3d with
    the face treatment of eqs. 3D-prolongation ... 3D-blend-interface-fluxes) with
    seeded per-element blending factors on a smooth periodic state (no squeezing,
    every candidate permissible) against that equation written element by element."""
    cfg = cfg2(M=M, nel=(3, 2), bc=(0, 0, 0, 0), scheme="single_level")
    U = smooth_state(cfg, seed=11)
    rng = np.random.default_rng(12)
    a_el = rng.uniform(0, 1, (cfg.nel[1], cfg.nel[0]))
    al, be = frozen(cfg, lambda n: 0.0)
    al[M] = a_el.copy()
    R = blended_rhs(U, cfg, frozen=(al, be))
    assert rel(R, _single_level_direct_2d(U, cfg, a_el)) < 1e-12


def test_single_level_indicator_keeps_lower_levels_off():
    """Single-level scheme: the blending factor of the top level is the multi-level
    one (same indicator, eq. calc-blending-factor, Sec. 2.7 remark), every level
    below it is off."""
    cfg_m = cfg2(M=8, nel=(3, 2), bc=(1, 1, 1, 1))
    cfg_s = cfg2(M=8, nel=(3, 2), bc=(1, 1, 1, 1), scheme="single_level")
    U = smooth_state(cfg_m, seed=13, noise=0.08)
    am = indicator(U, cfg_m)[0]
    a_s = indicator(U, cfg_s)[0]
    assert np.array_equal(am[8], a_s[8])
    assert all(np.all(a_s[n] == 0.0) for n in (4, 2))
