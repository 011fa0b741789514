"""Pins of the oracle's Euler physics, HLL flux and exact Riemann solver."""
import os

import numpy as np

from oracle.euler import conserved, hll_flux, mirror, physical_flux, pressure, primitives
from oracle.exact_riemann import cell_averages, sample, star_state

GOLD = os.path.join(os.path.dirname(__file__), "golden")
G = 1.4


def _random_states(rng, d, n):
    w = np.empty((d + 2, n))
    w[0] = rng.uniform(0.1, 3.0, n)
    w[1:d + 1] = rng.uniform(-2.0, 2.0, (d, n))
    w[d + 1] = rng.uniform(0.05, 3.0, n)
    return conserved(w, G)


def test_eos_roundtrip_and_pressure():
    rng = np.random.default_rng(0)
    u = _random_states(rng, 3, 50)
    w = primitives(u, G)
    assert np.allclose(conserved(w, G), u, rtol=1e-14)
    # p = (gamma-1)(E - rho |v|^2/2) (eq. equation-of-state) on a hand case
    uu = np.array([[2.0], [2.0], [4.0], [10.0]])   # rho 2, v = (1, 2), E = 10
    assert np.isclose(pressure(uu, G)[0], 0.4 * (10.0 - 0.5 * 2.0 * 5.0))


def test_hll_consistency_and_upwinding():
    rng = np.random.default_rng(1)
    for d in (2, 3):
        u = _random_states(rng, d, 64)
        for a in range(d):
            assert np.allclose(hll_flux(u, u, a, G), physical_flux(u, a, G), rtol=1e-13, atol=1e-14)
    # both states supersonic to the right: the flux is f(u_L)
    uL = conserved(np.array([[1.0], [5.0], [0.3], [1.0]]), G)
    uR = conserved(np.array([[0.5], [4.0], [0.0], [0.8]]), G)
    assert np.allclose(hll_flux(uL, uR, 0, G), physical_flux(uL, 0, G))
    assert np.allclose(hll_flux(mirror(uR, 0), mirror(uL, 0), 0, G)[0], -physical_flux(uL, 0, G)[0])


def test_hll_wall_mirror_has_no_mass_or_energy_flux():
    rng = np.random.default_rng(2)
    u = _random_states(rng, 2, 40)
    for a in range(2):
        F = hll_flux(u, mirror(u, a), a, G)
        assert np.abs(F[0]).max() < 1e-14 and np.abs(F[3]).max() < 1e-13
        assert np.abs(F[1 + (1 - a)]).max() < 1e-14       # no tangential momentum flux


def test_hll_rotation_symmetry():
    rng = np.random.default_rng(3)
    uL, uR = _random_states(rng, 2, 30), _random_states(rng, 2, 30)
    sw = lambda u: u[[0, 2, 1, 3]]
    assert np.allclose(hll_flux(uL, uR, 1, G), sw(hll_flux(sw(uL), sw(uR), 0, G)), rtol=1e-13)


def test_exact_riemann_sod_star_state_matches_textbook():
    ps, us, rl, rr = np.loadtxt(os.path.join(GOLD, "sod_star_state.txt"))
    p, u = star_state((1.0, 0.0, 1.0), (0.125, 0.0, 0.1))
    assert abs(p - ps) < 1e-5 and abs(u - us) < 1e-5
    w = sample((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), [u - 1e-3, u + 1e-3])
    assert abs(w[0, 0] - rl) < 1e-5 and abs(w[0, 1] - rr) < 1e-5


def test_exact_riemann_rankine_hugoniot_and_symmetry():
    left, right = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)
    p, u = star_state(left, right)
    rR, uR, pR = right
    cR = np.sqrt(G * pR / rR)
    S = uR + cR * np.sqrt((G + 1) / (2 * G) * p / pR + (G - 1) / (2 * G))
    rs = sample(left, right, [u + 1e-9])[0, 0]
    # mass and momentum conservation across the right-moving shock
    assert np.isclose(rR * (uR - S), rs * (u - S), rtol=1e-12)
    assert np.isclose(rR * uR * (uR - S) + pR, rs * u * (u - S) + p, rtol=1e-12)
    # a symmetric double rarefaction has u* = 0
    p2, u2 = star_state((1.0, -1.0, 1.0), (1.0, 1.0, 1.0))
    assert abs(u2) < 1e-14 and p2 < 1.0
    # cell averages: total mass on [0,1] is conserved (walls far away)
    edges = np.linspace(0, 1, 101)
    avg = cell_averages(left, right, 0.5, 0.2, edges)
    assert np.isclose(avg[0].mean(), 0.5 * (1.0 + 0.125), rtol=1e-4)


# ---------------------------------------------------------------------------
# Einfeldt signal speeds (Sec. 3: HLL with Einfeldt's estimates) on state pairs
# whose Roe averages come out in closed form, gamma = 7/5. By hand:
#   L: rho = 1,   v = (1/2, 0),    p = 5/7:  c_L = sqrt(gamma p / rho) = 1,
#      E_L = p/(gamma-1) + rho |v|^2 / 2 = 25/14 + 1/8 = 107/56,
#      H_L = (E_L + p) / rho = 147/56 = 21/8
#   R: rho = 1/4, v = (-1/4, 1/2), p = 5/7:  c_R = 2,
#      E_R = 25/14 + (1/8)(5/16) = 1635/896,  H_R = 4 (1635 + 640)/896 = 325/32
#   Roe weights sqrt(rho): 1 and 1/2, sum 3/2:
#      v_hat = ((1/2 - 1/8), (1/4)) / (3/2) = (1/4, 1/6)
#      H_hat = (21/8 + 325/64) / (3/2) = 493/96
#      c_hat^2 = (2/5)(493/96 - (1/16 + 1/36)/2) = (2/5)(1466/288) = 733/360
# Direction x:  S_L = min(1/2 - 1, 1/4 - c_hat) = 1/4 - c_hat (Roe side, -1.177)
#               S_R = max(-1/4 + 2, 1/4 + c_hat) = 7/4       (right state, 1.677 < 1.75)
# Direction y:  S_L = min(0 - 1, 1/6 - c_hat) = 1/6 - c_hat, S_R = max(1/2 + 2, ...) = 5/2
# Pair swapped (L <-> R), direction x: S_L = min(-1/4 - 2, 1/4 - c_hat) = -9/4 (left
#               state), S_R = max(1/2 + 1, 1/4 + c_hat) = 1/4 + c_hat (Roe side)
# With a zero third velocity component in 3D, direction z: v_hat_z = 0,
#               S_L = min(-1, -c_hat) = -c_hat, S_R = max(2, c_hat) = 2.
# The four cases take each of the four branches of the min / max, so Davis'
# estimates (min(v_L - c_L, v_R - c_R), ...), arithmetic instead of Roe means, or
# swapped Roe weights all move at least one of them.
# ---------------------------------------------------------------------------
from fractions import Fraction as _Fr   # noqa: E402

_G75 = 1.4
_CHAT = (733.0 / 360.0) ** 0.5
_UA = (1.0, 0.5, 0.0, 107.0 / 56.0)                  # rho, m_x, m_y, E of state L
_UB = (0.25, -1.0 / 16.0, 1.0 / 8.0, 1635.0 / 896.0)  # state R
# physical fluxes by hand: f_x(L) = (1/2, 1/4 + 5/7, 0, (1/2)(147/56)),
# f_x(R) = (-1/16, 1/64 + 5/7, -1/32, (-1/4)(2275/896))
_FXA = (0.5, 27.0 / 28.0, 0.0, 21.0 / 16.0)
_FXB = (-1.0 / 16.0, 327.0 / 448.0, -1.0 / 32.0, -2275.0 / 3584.0)


def _col(x, d=2):
    u = np.array(x, dtype=np.float64)
    if d == 3:
        u = np.array([u[0], u[1], u[2], 0.0, u[3]])
    return u[:, None]


def _einfeldt_pin_failures():
    """Hand values of the speeds and of the flux; returns the failing checks."""
    import oracle.euler as eu
    bad = []
    cases = [  # (uL, uR, dim, direction, S_L, S_R)
        (_UA, _UB, 2, 0, 0.25 - _CHAT, 1.75),
        (_UA, _UB, 2, 1, 1.0 / 6.0 - _CHAT, 2.5),
        (_UB, _UA, 2, 0, -2.25, 0.25 + _CHAT),
        (_UA, _UB, 3, 2, -_CHAT, 2.0),
    ]
    for uL, uR, d, a, sl, sr in cases:
        SL, SR = eu.einfeldt_speeds(_col(uL, d), _col(uR, d), a, _G75)
        if not (abs(SL[0] - sl) < 1e-14 and abs(SR[0] - sr) < 1e-14):
            bad.append(("speeds", d, a, float(SL[0]), float(SR[0]), sl, sr))
    # the flux of the subsonic pair in x: the HLL average-state flux with these speeds
    sl, sr = 0.25 - _CHAT, 1.75
    want = [(sr * fa - sl * fb + sl * sr * (ub - ua)) / (sr - sl) for fa, fb, ua, ub in zip(_FXA, _FXB, _UA, _UB)]
    got = eu.hll_flux(_col(_UA), _col(_UB), 0, _G75)[:, 0]
    if not np.allclose(got, want, rtol=1e-14, atol=1e-15):
        bad.append(("flux", got.tolist(), want))
    return bad


def test_einfeldt_speeds_and_flux_against_hand_values():
    # the hand fractions behind the literals above
    g = _Fr(7, 5)
    EL = _Fr(5, 7) / (g - 1) + _Fr(1, 2) * _Fr(1, 4)
    ER = _Fr(5, 7) / (g - 1) + _Fr(1, 2) * _Fr(1, 4) * (_Fr(1, 16) + _Fr(1, 4))
    assert (EL, ER) == (_Fr(107, 56), _Fr(1635, 896))
    assert _einfeldt_pin_failures() == []


def test_einfeldt_pins_reject_planted_speed_mistakes(monkeypatch):
    """Plausible mistakes planted in the oracle's speed estimates fail the pins."""
    import oracle.euler as eu
    real = eu.einfeldt_speeds

    def parts(uL, uR, gamma):
        d = uL.shape[0] - 2
        pL, pR = eu.pressure(uL, gamma), eu.pressure(uR, gamma)
        vL = [uL[1 + k] / uL[0] for k in range(d)]
        vR = [uR[1 + k] / uR[0] for k in range(d)]
        cL, cR = np.sqrt(gamma * pL / uL[0]), np.sqrt(gamma * pR / uR[0])
        HL, HR = (uL[d + 1] + pL) / uL[0], (uR[d + 1] + pR) / uR[0]
        return d, vL, vR, cL, cR, HL, HR

    def davis(uL, uR, a, gamma):
        _, vL, vR, cL, cR, _, _ = parts(uL, uR, gamma)
        return np.minimum(vL[a] - cL, vR[a] - cR), np.maximum(vL[a] + cL, vR[a] + cR)

    def roe_with(wl, wr):
        def speeds(uL, uR, a, gamma):
            d, vL, vR, cL, cR, HL, HR = parts(uL, uR, gamma)
            sL, sR = wl(uL, uR), wr(uL, uR)
            vh = [(sL * vL[k] + sR * vR[k]) / (sL + sR) for k in range(d)]
            Hh = (sL * HL + sR * HR) / (sL + sR)
            ch = np.sqrt((gamma - 1.0) * (Hh - 0.5 * sum(v ** 2 for v in vh)))
            return np.minimum(vL[a] - cL, vh[a] - ch), np.maximum(vR[a] + cR, vh[a] + ch)
        return speeds

    swapped = roe_with(lambda uL, uR: np.sqrt(uR[0]), lambda uL, uR: np.sqrt(uL[0]))
    arithmetic = roe_with(lambda uL, uR: np.ones_like(uL[0]), lambda uL, uR: np.ones_like(uR[0]))
    faithful = roe_with(lambda uL, uR: np.sqrt(uL[0]), lambda uL, uR: np.sqrt(uR[0]))
    monkeypatch.setattr(eu, "einfeldt_speeds", faithful)      # a faithful restatement passes
    assert _einfeldt_pin_failures() == []
    for planted in (davis, swapped, arithmetic):
        monkeypatch.setattr(eu, "einfeldt_speeds", planted)
        assert _einfeldt_pin_failures() != [], planted
    monkeypatch.setattr(eu, "einfeldt_speeds", real)
