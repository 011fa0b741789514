"""Seeded synthetic inputs: initial subcell mean values of the workloads.

This module holds no part of the scheme: it only builds initial states (and
their problem descriptions) that the library, its tests and the benchmark
consume. States are returned in the library's element-major layout
u[e][v][t] (e = ex + nx*(ey + ny*ez), t = ix + M*(iy + M*iz)), FP64.

Each initial mean value is the average of the pointwise conserved state over
its subcell, taken with an 8-point Gauss rule per direction (the paper
evaluates initial conditions on the mean values "via an appropriate quadrature
rule").

Workloads (configs are plain dicts with the fields of the library's config):
  sedov      Sedov blast on [-1,1]^d with reflecting walls: rho = 1 plus seeded
             uniform noise of amplitude 1e-3 per subcell, v = 0, p = 1e-5 and a
             Gaussian energy E/(2 pi sigma^2)^(d/2) exp(-|x|^2 / (2 sigma^2)),
             E = 1, sigma = 0.05 (the paper's Sedov setup, Sec. 3.6).
  kelvin_helmholtz  periodic [-1,1]^2: rho = 2 for |y| < 1/2 else 1, v_x = +-1/2,
             p = 2.5, v_y = 0.01 sin(2 pi x + phi) with a seeded phase.
  quadrants  four-quadrant 2D Riemann problem on [-1/2,1/2]^2 with outflow and
             seeded constant states (rho in [0.1, 2], p in [0.05, 2], |v| <= 1);
             stands in for the configurations of Lax & Liu the paper cites
             (their states are not given in the paper). Its means are exact:
             every subcell lies inside one quadrant.
  quadrant_ensemble  n four-quadrant problems of seeded sizes and M (the
             batched workload).
  density_wave  smooth periodic wave rho = 1 + A sin(pi (x + y)), constant v, p.
  sod        Sod shock tube along x on [0,1] (1D-in-2D, one element row, periodic in y).
  shock_tube any 1D-in-2D Riemann problem of that form (e.g. the Lax tube).
"""
import numpy as np
from numpy.polynomial import legendre as npleg

WALL, PERIODIC, OUTFLOW = 1, 0, 2


def make_config(dim, M, nel, xlo, xhi, bc, **kw):
    cfg = dict(dim=dim, M=M, nel=tuple(nel), xlo=tuple(xlo), xhi=tuple(xhi), bc=tuple(bc),
               gamma=1.4, tauA=100.0, tauS=0.05, alphaH=0.99, alphaL=0.01, betaL=0.95,
               cfl=0.5, family="gauss")
    cfg.update(kw)
    return cfg


def _subcell_quadrature(cfg, npts=8):
    """Gauss points/weights of every subcell along each axis: list over axes of
    (coords (G, npts), weights (npts,)) with weights summing to 1."""
    gx, gw = npleg.leggauss(npts)
    out = []
    for a in range(cfg["dim"]):
        G = cfg["nel"][a] * cfg["M"]
        h = (cfg["xhi"][a] - cfg["xlo"][a]) / G
        left = cfg["xlo"][a] + h * np.arange(G)
        xs = left[:, None] + 0.5 * h * (gx[None, :] + 1.0)
        out.append((xs, 0.5 * gw))
    return out


def _means(cfg, pointwise):
    """Subcell means of pointwise(coords...) -> (nv, G_{d-1}, ..., G_0) global grid."""
    d = cfg["dim"]
    q = _subcell_quadrature(cfg)
    if d == 2:
        (xs, wx), (ys, wy) = q
        Gx, Gy = xs.shape[0], ys.shape[0]
        nv = pointwise(xs[None, :1, None, :1], ys[:1, None, :1, None]).shape[0]
        out = np.empty((nv, Gy, Gx))
        rows = max(1, (1 << 22) // (Gx * xs.shape[1] * ys.shape[1]))   # bounded memory per slab
        for y0 in range(0, Gy, rows):
            X = xs[None, :, None, :]          # (1, Gx, 1, qx)
            Y = ys[y0:y0 + rows, None, :, None]
            vals = pointwise(X, Y)            # (nv, rows, Gx, qy, qx)
            out[:, y0:y0 + rows] = np.einsum("vyxjk,j,k->vyx", vals, wy, wx)
        return out
    (xs, wx), (ys, wy), (zs, wz) = q
    Gx, Gy, Gz = xs.shape[0], ys.shape[0], zs.shape[0]
    out = np.empty((5, Gz, Gy, Gx))
    for iz in range(Gz):                  # slab by slab to bound memory
        X = xs[None, :, None, :]
        Y = ys[:, None, :, None]
        acc = 0.0
        for kz in range(zs.shape[1]):
            vals = pointwise(X, Y, zs[iz, kz])
            acc = acc + wz[kz] * np.einsum("vyxjk,j,k->vyx", vals, wy, wx)
        out[:, iz] = acc
    return out


def _to_elements(U, cfg):
    d, M, nel = cfg["dim"], cfg["M"], cfg["nel"]
    nv = U.shape[0]
    if d == 2:
        nx, ny = nel[0], nel[1]
        x = U.reshape(nv, ny, M, nx, M).transpose(1, 3, 0, 2, 4)
        return np.ascontiguousarray(x.reshape(ny * nx, nv, M * M))
    nx, ny, nz = nel
    x = U.reshape(nv, nz, M, ny, M, nx, M).transpose(1, 3, 5, 0, 2, 4, 6)
    return np.ascontiguousarray(x.reshape(nz * ny * nx, nv, M ** 3))


def _conserved(rho, vel, p, gamma):
    kin = sum(v * v for v in vel)
    return np.stack(np.broadcast_arrays(rho, *[rho * v for v in vel], p / (gamma - 1.0) + 0.5 * rho * kin))


def sedov(dim, M, nel_per_dir, seed=0, sigma=0.05, energy=1.0, p0=1e-5, noise=1e-3, nel=None, xhi=None, **kw):
    """Sedov blast on [-1,1]^d (nel_per_dir elements per direction); nel / xhi give
    another mesh and box upper corner (the blast stays at the origin), e.g. the
    strip [-1,1] x [-1, 2N-1] of N stacked 256^2 blocks of a weak-scaling run."""
    nel = tuple(nel) if nel is not None else (nel_per_dir,) * dim
    xhi = tuple(xhi) if xhi is not None else (1.0,) * dim
    cfg = make_config(dim, M, nel, (-1.0,) * dim, xhi, (WALL,) * (2 * dim), **kw)
    g = cfg["gamma"]
    amp = energy / (2.0 * np.pi * sigma ** 2) ** (dim / 2.0)
    # the Gaussian is a product over the axes, so its subcell means under the tensor
    # Gauss rule are products of the per-axis 1D rule sums
    gauss = [np.exp(-0.5 * xs ** 2 / sigma ** 2) @ w for xs, w in _subcell_quadrature(cfg)]
    prod = gauss[0]
    for ga in gauss[1:]:
        prod = np.multiply.outer(ga, prod)                 # grid order (z,) y, x
    U = np.zeros((dim + 2,) + prod.shape)
    U[0] = 1.0
    U[dim + 1] = p0 / (g - 1.0) + amp * prod
    rng = np.random.default_rng(seed)
    U[0] += noise * rng.uniform(-1.0, 1.0, size=U[0].shape)
    return cfg, _to_elements(U, cfg)


def kelvin_helmholtz(M=8, nel_per_dir=128, seed=0, **kw):
    cfg = make_config(2, M, (nel_per_dir,) * 2, (-1.0, -1.0), (1.0, 1.0), (PERIODIC,) * 4, **kw)
    phi = np.random.default_rng(seed).uniform(0.0, 2.0 * np.pi)
    g = cfg["gamma"]

    def pw(X, Y):
        inside = np.abs(Y) < 0.5
        rho = np.where(inside, 2.0, 1.0) + 0.0 * X
        vx = np.where(inside, 0.5, -0.5) + 0.0 * X
        vy = 0.01 * np.sin(2.0 * np.pi * X + phi) + 0.0 * Y
        return _conserved(rho, (vx, vy), 2.5 + 0.0 * rho, g)
    return cfg, _to_elements(_means(cfg, pw), cfg)


def quadrants(M=8, nel_per_dir=64, seed=0, **kw):
    cfg = make_config(2, M, (nel_per_dir,) * 2, (-0.5, -0.5), (0.5, 0.5), (OUTFLOW,) * 4, **kw)
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.1, 2.0, 4)
    p = rng.uniform(0.05, 2.0, 4)
    ang = rng.uniform(0.0, 2.0 * np.pi, 4)
    speed = rng.uniform(0.0, 1.0, 4)
    vx, vy = speed * np.cos(ang), speed * np.sin(ang)
    g = cfg["gamma"]
    # M is even, so the lines x = 0 and y = 0 are subcell faces (index G/2) and
    # every subcell lies in one quadrant: its mean is that quadrant's state
    G = nel_per_dir * M
    side = (np.arange(G) >= G // 2).astype(int)
    q = side[None, :] + 2 * side[:, None]            # (Gy, Gx)
    U = _conserved(rho[q], (vx[q], vy[q]), p[q], g)
    return cfg, _to_elements(U, cfg)


def quadrant_ensemble(n=64, seed=0, nel_min=32, nel_max=256, Ms=(4, 8), **kw):
    """n independent four-quadrant problems with seeded states, mesh sizes drawn
    uniformly from nel_min^2 .. nel_max^2 elements and M drawn from Ms: a list of
    (cfg, u) pairs."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        nel = int(rng.integers(nel_min, nel_max + 1))
        M = int(Ms[int(rng.integers(0, len(Ms)))])
        out.append(quadrants(M=M, nel_per_dir=nel, seed=int(rng.integers(0, 2 ** 31)), **kw))
    return out


def density_wave(M=4, nel_per_dir=8, amp=0.2, vel=(1.0, 0.5), p=1.0, t=0.0, **kw):
    cfg = make_config(2, M, (nel_per_dir,) * 2, (-1.0, -1.0), (1.0, 1.0), (PERIODIC,) * 4, **kw)
    g = cfg["gamma"]

    def pw(X, Y):
        rho = 1.0 + amp * np.sin(np.pi * ((X - vel[0] * t) + (Y - vel[1] * t)))
        return _conserved(rho, (vel[0] + 0.0 * rho, vel[1] + 0.0 * rho), p + 0.0 * rho, g)
    return cfg, _to_elements(_means(cfg, pw), cfg)


def shock_tube(left, right, M=8, nel_x=32, nel_y=1, x0=0.5, **kw):
    """1D-in-2D Riemann problem along x on [0,1] (outflow in x, periodic in y);
    left / right = (rho, u, p)."""
    cfg = make_config(2, M, (nel_x, nel_y), (0.0, 0.0), (1.0, 1.0 * nel_y / nel_x),
                      (OUTFLOW, OUTFLOW, PERIODIC, PERIODIC), **kw)
    g = cfg["gamma"]

    def pw(X, Y):
        lft = (X < x0) + 0.0 * Y
        rho = np.where(lft, left[0], right[0])
        u = np.where(lft, left[1], right[1])
        p = np.where(lft, left[2], right[2])
        return _conserved(rho, (u, 0.0 * rho), p, g)
    return cfg, _to_elements(_means(cfg, pw), cfg)


def sod(M=8, nel_x=32, nel_y=1, **kw):
    cfg = make_config(2, M, (nel_x, nel_y), (0.0, 0.0), (1.0, 1.0 * nel_y / nel_x),
                      (OUTFLOW, OUTFLOW, PERIODIC, PERIODIC), **kw)
    g = cfg["gamma"]

    def pw(X, Y):
        left = (X < 0.5) + 0.0 * Y
        rho = np.where(left, 1.0, 0.125)
        p = np.where(left, 1.0, 0.1)
        return _conserved(rho, (0.0 * rho, 0.0 * rho), p, g)
    return cfg, _to_elements(_means(cfg, pw), cfg)


def random_coefficients(cfg, seed, lo=0.0, hi=1.0):
    """Seeded blending factors alpha and squeezing beta = 1 for every level and
    sub-element, in the library's coefficient layout (E, 2, S): [:,0,:] alpha and
    [:,1,:] beta, levels from M down to 2, sub-elements x fastest."""
    d, M = cfg["dim"], cfg["M"]
    E = int(np.prod(cfg["nel"]))
    S, n = 0, M
    while n >= 2:
        S += (M // n) ** d
        n //= 2
    rng = np.random.default_rng(seed)
    c = np.ones((E, 2, S))
    c[:, 0, :] = rng.uniform(lo, hi, size=(E, S))
    return c
