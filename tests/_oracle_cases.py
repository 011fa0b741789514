"""Small seeded cases for the oracle pins (grids built directly, no library)."""
import numpy as np

from oracle.blended import Config
from oracle.euler import conserved


def smooth_state(cfg, seed=0, noise=0.0):
    """Positive smooth state on the global subcell grid (cell-centre values are
    enough for pins that hold for any state)."""
    d = cfg.dim
    G = [cfg.nel[a] * cfg.M for a in range(d)][::-1]
    rng = np.random.default_rng(seed)
    axes = [np.linspace(0.0, 2 * np.pi, g, endpoint=False) + rng.uniform(0, 1) for g in G]
    grids = np.meshgrid(*axes, indexing="ij")
    w = np.empty((d + 2,) + tuple(G))
    w[0] = 1.0 + 0.3 * np.sin(grids[-1]) * np.cos(grids[0]) + noise * rng.uniform(-1, 1, G)
    for k in range(d):
        w[1 + k] = 0.4 * np.cos(grids[k] + k) + noise * rng.uniform(-1, 1, G)
    w[d + 1] = 1.0 + 0.2 * np.cos(grids[-1] + grids[0]) + noise * rng.uniform(-1, 1, G)
    return conserved(w, cfg.gamma)


def cfg2(M=4, nel=(3, 2), bc=(1, 1, 1, 1), **kw):
    return Config(dim=2, M=M, nel=nel, xlo=(-1.0, -0.5), xhi=(1.0, 0.5), bc=bc, **kw)


def cfg3(M=4, nel=(2, 2, 2), bc=(1, 1, 0, 0, 2, 2), **kw):
    return Config(dim=3, M=M, nel=nel, xlo=(0.0, 0.0, 0.0), xhi=(1.0, 1.2, 0.8), bc=bc, **kw)


def sub_grid_shape(cfg, n):
    return tuple(cfg.nel[a] * cfg.M // n for a in range(cfg.dim))[::-1]


def frozen(cfg, value_of_level, seed=None, beta=1.0):
    """alpha per level from value_of_level(n) (a number or 'random'); beta constant."""
    rng = np.random.default_rng(seed)
    al, be = {}, {}
    for n in cfg.levels:
        sh = sub_grid_shape(cfg, n)
        v = value_of_level(n)
        al[n] = rng.uniform(0, 1, sh) if isinstance(v, str) else np.full(sh, float(v))
        be[n] = np.full(sh, beta)
    return al, be
