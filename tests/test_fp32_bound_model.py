"""A CPU model of the error bounds that the FP64 indicator's certified FP32 pass uses.

The kernel (level_sigma_f32 / factor_f32) forms the smoothness values of eq.
L1-norm-slope in FP32 and decides a blending factor of eq. calc-blending-factor
only where a forward error bound puts the ratio outside the transition band. This
file restates those bounds in numpy float32 (the same deviation form, nodal-value,
primitive, derivative and summation terms) and checks them against the oracle's
FP64 values on evolved states of the workloads: every FP32 sigma lies within its
bound of the oracle's sigma, every factor the model decides equals the oracle's
raw factor, and the bound is tight enough to decide most factors. A planted
mistake (reconstructing the means themselves while keeping the bound of the
deviation form) breaks the bound. The GPU test of the kernel itself compares its
coefficients with the FP64 evaluation bit for bit (tests/test_gpu_indicator_filter.py)."""
import numpy as np
import pytest

from oracle.blended import Config, block_reduce, blockwise, expand, indicator
from oracle.layout import to_grid
from oracle.ops import level_ops
from oracle.timestep import rk3_step
from paper_2011_03338_gb300 import inputs

U = 2.0 ** -24
F32 = np.float32


def _row_first(X, axis, n):
    """Each entry replaced by the first entry of its block of n along axis."""
    X = np.moveaxis(X, axis, -1)
    sh = X.shape
    B = X.reshape(sh[:-1] + (sh[-1] // n, n))
    return np.moveaxis(np.repeat(B[..., :1], n, axis=-1).reshape(sh), -1, axis)


def _prim_bound(q, e, g):
    """Primitives (rho, v, p) of FP32 nodal values q with bounds e of their errors,
    and bounds of the primitives' errors; ok where rho > 0, e_rho <= 1e-3 rho."""
    d = q.shape[0] - 2
    rho, er = q[0], e[0]
    ok = (rho > 0) & (er <= 1e-3 * rho)
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        inv = F32(1) / rho
        vel = [q[1 + k] * inv for k in range(d)]
        kin = sum(q[1 + k] * vel[k] for k in range(d))
        ev, ekin, mv = [], 0.0, 0.0
        for k in range(d):
            em = e[1 + k].astype(np.float64)
            evk = 1.003 * (em + np.abs(vel[k]) * er) * inv + 4 * U * np.abs(vel[k])
            ev.append(evk)
            ekin = ekin + np.abs(q[1 + k]) * evk + np.abs(vel[k]) * em + em * evk
            mv = mv + np.abs(q[1 + k] * vel[k])
        ekin = 1.001 * ekin + (d + 1) * U * mv
        gm1 = F32(g) - F32(1)
        p = gm1 * (q[-1] - F32(0.5) * kin)
        grel = 2.02 * U * F32(g) / gm1
        ep = 1.001 * gm1 * (e[-1] + 0.5 * ekin) + (2.01 * U + grel) * np.abs(p)
    w = np.stack([rho] + vel + [p]).astype(F32)
    b = np.stack([er] + ev + [ep]).astype(np.float64)
    ok &= np.all(np.isfinite(w), axis=0) & np.all(np.isfinite(b), axis=0)
    return w, b, ok


def fp32_sigma(Ug, cfg, deviations=True):
    """{n: (sigma in FP32, its bound)} per level on the global grid; the bound is inf
    in every element where the pass declines (a density the bound cannot resolve)."""
    d, M, g = cfg.dim, cfg.M, cfg.gamma
    vax = [d - a for a in range(d)]          # grid axes of the directions (variable axis first)
    sax = [a - 1 for a in vax]
    ref = block_reduce(Ug, M, vax, lambda X, axis: np.take(X, 0, axis=axis)).astype(F32)
    refg = expand(ref.astype(np.float64), M, vax)
    dev = (Ug - refg).astype(F32)
    qd = block_reduce(np.abs(dev.astype(np.float64)), M, vax, np.max)
    qm = np.abs(ref.astype(np.float64)) + 2 * qd
    qp = expand((qd + 2.0 ** -28 * qm) * (1 + 4 * U), M, vax)
    out = {}
    for n in cfg.levels:
        o = level_ops(n, cfg.family)
        R32 = o.R.astype(F32)
        lam = np.abs(R32.astype(np.float64)).sum(axis=1).max() * (1 + 1e-6)
        x = dev if deviations else Ug.astype(F32)
        for a in range(d):
            x = blockwise(x, R32, vax[a], n).astype(F32)
        q = (refg.astype(F32) + x).astype(F32) if deviations else x
        e = 1.01 * d * (n + 2) * U * lam ** d * qp + 1.01 * U * np.abs(q)
        w, b, ok = _prim_bound(q, e.astype(np.float64), g)
        Wn = np.ones(())
        for a in range(d - 1, -1, -1):
            Wn = np.multiply.outer(Wn, np.tile(o.w, cfg.nel[a] * M // n))
        D32 = o.Dnodal.astype(F32)
        Dabs = np.abs(o.Dnodal)
        cw, cw64 = (n + 3) * U, (n + 3) * 2.0 ** -53
        s = sb = 0.0
        for a in range(d):
            c = _row_first(w, vax[a], n)
            dw = blockwise((w - c).astype(F32), D32, vax[a], n)
            bj = b + cw * np.abs(w - c) + cw64 * np.abs(w)
            s = s + block_reduce(np.abs(dw).astype(np.float64) * Wn, n, vax, np.sum)
            sb = sb + block_reduce(blockwise(bj, Dabs, vax[a], n) * Wn, n, vax, np.sum)
        hd = (n / M) ** (d - 1)
        okel = block_reduce(ok.astype(float), M, sax, np.min) > 0
        bound = np.where(expand(okel, M // n, sax)[None], 1.01 * hd * sb, np.inf)
        out[n] = (hd * s, bound)
    return out


def decided_factors(sig, cfg):
    """Raw factors the pass decides (0 or 1) per level n >= 4, nan where open."""
    d, M = cfg.dim, cfg.M
    vax = [d - a for a in range(d)]
    kap = (d + M ** d + 8) * U
    out = {}
    for n in cfg.levels:
        if n < 4:
            continue
        sp, ep = sig[n]
        cs = block_reduce(sig[n // 2][0], 2, vax, np.sum)
        ce = block_reduce(sig[n // 2][1], 2, vax, np.sum)
        num, den = np.abs(sp - cs), np.maximum(np.maximum(sp, cs), 1.0)
        dl = 1.01 * (ep + ce + kap * (sp + cs))
        with np.errstate(invalid="ignore"):
            hi = (num + dl) / np.maximum(den - dl, 1.0) * (1 + 8 * U)
            lo = (num - dl) / (den + dl) * (1 - 8 * U)
        code = np.full(sp.shape, 2)
        code[hi < cfg.tauS * (1 - 1e-6)] = 1
        code[lo > (cfg.tauS + 1 / cfg.tauA) * (1 + 1e-6)] = 0
        code[~np.isfinite(dl)] = 2
        out[n] = np.where(np.any(code == 0, axis=0), 0.0, np.where(np.all(code == 1, axis=0), 1.0, np.nan))
    return out


def _evolved(cfg_d, u, steps):
    cfg = Config(**cfg_d)
    Ug = to_grid(u, cfg.dim, cfg.M, cfg_d["nel"])
    for _ in range(steps):
        Ug = rk3_step(Ug, cfg)
        if isinstance(Ug, tuple):
            Ug = Ug[0]
    return Ug, cfg


WORKLOADS = {
    "sedov2d_M8_20": (lambda: inputs.sedov(2, 8, 20), 6),
    "sedov2d_M8_20_lgl": (lambda: inputs.sedov(2, 8, 20, family="lgl"), 3),
    "kh_M8_16": (lambda: inputs.kelvin_helmholtz(8, 16, seed=3), 8),
    "quadrants_M4_24": (lambda: inputs.quadrants(4, 24, seed=11), 8),
    "sedov3d_M4_6": (lambda: inputs.sedov(3, 4, 6, sigma=0.2), 2),
}


@pytest.mark.parametrize("name", sorted(WORKLOADS))
def test_fp32_sigma_within_its_bound_and_decisions_exact(name):
    mk, steps = WORKLOADS[name]
    Ug, cfg = _evolved(*mk(), steps)
    _, beta, alpha_raw, sigma, _, _ = indicator(Ug, cfg)
    sig = fp32_sigma(Ug, cfg)
    for n in cfg.levels:
        s32, bnd = sig[n]
        fin = np.isfinite(bnd)
        assert fin.mean() > 0.5, f"level {n}: the pass declines most elements"
        err = np.abs(s32 - sigma[n])
        assert np.all(err[fin] <= bnd[fin]), f"level {n}: max err/bound {np.max(err[fin] / bnd[fin]):.3g}"
    decided = decided_factors(sig, cfg)
    total = hits = 0
    for n, a in decided.items():
        m = np.isfinite(a) & (beta[n] >= cfg.betaL)        # the kernel certifies beta = 1 itself
        assert np.array_equal(a[m], alpha_raw[n][m]), f"level {n}: a decided factor differs from the oracle's"
        total += a.size
        hits += int(np.isfinite(a).sum())
    assert hits > 0.5 * total, f"the bound decides only {hits} of {total} factors"


def test_bound_of_the_deviation_form_fails_without_deviations():
    """Reconstructing the means themselves makes the FP32 errors scale with their
    magnitude, which the deviation form's bound does not cover: planted, it fails."""
    Ug, cfg = _evolved(*inputs.sedov(2, 8, 12), 0)
    sig = fp32_sigma(Ug, cfg, deviations=False)
    _, _, _, sigma, _, _ = indicator(Ug, cfg)
    worst = 0.0
    for n in cfg.levels:
        s32, bnd = sig[n]
        fin = np.isfinite(bnd) & (bnd > 0)
        worst = max(worst, float(np.max(np.abs(s32 - sigma[n])[fin] / bnd[fin])))
    assert worst > 1.0
