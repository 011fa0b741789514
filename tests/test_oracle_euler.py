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
