"""Batched ensembles (sesc_batch_*): many problems of uneven sizes, dimensions, M
and precisions advanced by persistent launches per group, eagerly or by CUDA
graph replay, at grids chosen by the autotuner or set by hand.

Every problem of a batch runs the single-problem kernel bodies with its own
parameters and time step, so the bar is bit-identity with a standalone handle
of the same configuration (which the parity tests tie to the oracle), plus one
direct oracle comparison of a batched FP64 problem."""
import numpy as np
import pytest

from paper_2011_03338_gb300 import inputs
from tests._gpu_helpers import (density_squeezed_active, face_neighbours, levels_to_coeffs, near_threshold,
                                oracle_rhs, term_scale)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _mixed():
    """Five groups: (2D, M4, split), (2D, M8, split), (2D, M4, FP64), (3D, M4, FP64),
    (2D, M8, FP64), problems of each group interleaved with the others."""
    split = dict(precision="fp32_split")
    return [
        inputs.quadrants(4, 10, seed=1, **split),
        inputs.sedov(2, 4, 16),
        inputs.quadrants(8, 7, seed=2, **split),
        inputs.sedov(3, 4, 4),
        inputs.quadrants(4, 13, seed=3, **split),
        inputs.kelvin_helmholtz(8, 6),
        inputs.quadrants(8, 5, seed=4, **split),
        inputs.sedov(2, 4, 6, seed=7),
    ]


def _batch(probs):
    from paper_2011_03338_gb300 import Batch
    b = Batch([c for c, _ in probs])
    u = torch.empty(b.total, dtype=torch.float64, device="cuda")
    for k, (_, uk) in enumerate(probs):
        b.view(u, k).copy_(torch.from_numpy(uk))
    return b, u


def _bits(t):
    """Bit pattern of a float64 tensor (NaN-safe identity check)."""
    return t.contiguous().view(torch.int64)


def _standalone_steps(cfg, u0, steps):
    from paper_2011_03338_gb300 import Solver
    s = Solver(cfg)
    u = torch.from_numpy(u0).cuda()
    v = torch.empty_like(u)
    dts = []
    dt = torch.empty(1, dtype=torch.float64, device="cuda")
    for _ in range(steps):
        s.rk3_step(u, v, dt)
        dts.append(dt.item())
        u, v = v, u
    rc, counters = s.status()
    s.close()
    return u, dts, rc, counters


@pytest.fixture(scope="module")
def mixed():
    probs = _mixed()
    b, u = _batch(probs)
    yield probs, b, u
    b.close()


def test_groups(mixed):
    probs, b, _ = mixed
    assert b.ngroups == 5
    assert all(g > 0 for g in b.fused())      # by default a stage is one launch per group
    key = [(c["dim"], c["M"], c.get("precision", "fp64")) for c, _ in probs]
    for k in range(len(probs)):
        for j in range(len(probs)):
            assert (b.group_of[k] == b.group_of[j]) == (key[k] == key[j])


def test_batched_rhs_bit_identical_to_standalone(mixed):
    from paper_2011_03338_gb300 import Solver
    probs, b, u = mixed
    r = torch.empty_like(u)
    b.rhs(u, r)
    torch.cuda.synchronize()
    for k, (cfg, uk) in enumerate(probs):
        s = Solver(cfg)
        ud = torch.from_numpy(uk).cuda()
        rs = torch.empty_like(ud)
        s.rhs(ud, rs)
        assert torch.equal(_bits(b.view(r, k)), _bits(rs)), k
        s.close()


def test_batched_steps_bit_identical_to_standalone(mixed):
    probs, b, u0 = mixed
    b.reset_status()
    u = u0.clone()
    v = torch.empty_like(u)
    dt = torch.empty(len(probs), dtype=torch.float64, device="cuda")
    dts = []
    for _ in range(3):
        b.rk3_step(u, v, dt)
        dts.append(dt.cpu().numpy().copy())
        u, v = v, u
    rc, counters = b.status()
    clean = 0
    for k, (cfg, uk) in enumerate(probs):
        us, dts_k, rck, ck = _standalone_steps(cfg, uk, 3)
        assert torch.equal(_bits(b.view(u, k)), _bits(us)), k
        assert np.array_equal(np.array([d[k] for d in dts]).view(np.int64), np.array(dts_k).view(np.int64)), k
        assert counters[k] == ck, (k, counters[k], ck)      # same squeezing / fallback / error counts
        clean += rck == 0
    assert clean >= len(probs) - 2
    b.reset_status()


def test_graph_replay_bit_identical_to_eager(mixed):
    probs, b, u0 = mixed
    results = []
    for graph in (False, True):
        b.use_graph(graph)
        u = u0.clone()
        v = torch.empty_like(u)
        dt = torch.empty(len(probs), dtype=torch.float64, device="cuda")
        for _ in range(4):                     # ping-pong: two captured graphs, each replayed
            b.rk3_step(u, v, dt)
            u, v = v, u
        torch.cuda.synchronize()
        results.append((u.clone(), dt.clone()))
    b.use_graph(False)
    assert torch.equal(_bits(results[0][0]), _bits(results[1][0]))
    assert torch.equal(_bits(results[0][1]), _bits(results[1][1]))
    b.reset_status()


def test_results_do_not_depend_on_grid(mixed):
    probs, b, u0 = mixed
    ref = torch.empty_like(u0)
    b.rhs(u0, ref)
    default = b.grids()
    for g in (1, 3, 152 + 5):
        b.set_grids([[g] * 4 for _ in range(b.ngroups)])
        r = torch.empty_like(u0)
        b.rhs(u0, r)
        v = torch.empty_like(u0)
        dt = torch.empty(len(probs), dtype=torch.float64, device="cuda")
        b.rk3_step(u0, v, dt)
        torch.cuda.synchronize()
        assert torch.equal(_bits(r), _bits(ref)), g
        if g == 1:
            v1, dt1 = v.clone(), dt.clone()
        else:
            assert torch.equal(_bits(v), _bits(v1)) and torch.equal(_bits(dt), _bits(dt1)), g
    b.set_grids(default)
    from paper_2011_03338_gb300.sesc import SescError
    with pytest.raises(SescError):
        b.set_grids([[0, 1, 1, 1]] * b.ngroups)


def test_autotune(mixed):
    probs, b, u0 = mixed
    ref = torch.empty_like(u0)
    b.rhs(u0, ref)
    b.reset_status()
    grids = b.autotune(u0, reps=2)
    assert len(grids) == b.ngroups and all(len(g) == 4 and min(g) >= 1 for g in grids)
    rc, counters = b.status()
    assert rc == 0 and all(c[0] == 0 for c in counters)
    r = torch.empty_like(u0)
    b.rhs(u0, r)
    torch.cuda.synchronize()
    assert torch.equal(_bits(r), _bits(ref))


def test_batched_fp64_problem_matches_oracle(mixed):
    """Problem 1 (Sedov 2D, M = 4, 16^2, FP64) of the batch against the oracle with
    the parity bar of the standalone path (same exclusions)."""
    probs, b, u0 = mixed
    r = torch.empty_like(u0)
    b.rhs(u0, r)
    cfg, uk = probs[1]
    got = b.view(r, 1).cpu().numpy()
    ref, dg = oracle_rhs(cfg, uk)
    cref = levels_to_coeffs(cfg, dg.alpha, dg.beta)
    keep = ~(face_neighbours(cfg, near_threshold(cfg, dg)) | density_squeezed_active(cfg, dg, cref))
    err = np.abs(got - ref) / np.maximum(np.abs(ref), term_scale(cfg, uk))
    assert keep.sum() > 0.5 * len(keep)
    assert err[keep].max() <= 1e-12


def test_status_is_per_problem():
    probs = [inputs.sedov(2, 4, 4), inputs.quadrants(4, 6, seed=5), inputs.sedov(2, 4, 5)]
    bad = probs[1][1].copy()
    bad[7, 0, 2] = -1e-3                       # a negative density mean in problem 1 only
    probs[1] = (probs[1][0], bad)
    b, u = _batch(probs)
    r = torch.empty_like(u)
    b.rhs(u, r)
    rc, counters = b.status()
    assert rc == 4
    assert counters[1][0] & 1 and counters[0][0] == 0 and counters[2][0] == 0
    b.reset_status()
    rc, counters = b.status()
    assert rc == 0 and all(c[0] == 0 for c in counters)
    b.close()


def _permissible(u, cfg):
    d = cfg["dim"]
    x = u.view(-1, d + 2, cfg["M"] ** d)
    r, E = x[:, 0], x[:, d + 1]
    kin = 0.5 * (x[:, 1:1 + d] ** 2).sum(1) / r
    return bool(((r > 0) & ((cfg["gamma"] - 1) * (E - kin) > 0)).all())


def test_full_ensemble_graph_step():
    """The 64-problem four-quadrant ensemble (32^2 .. 256^2 elements, M in {4, 8},
    FP32-split) in the launch configuration the benchmark times (autotuned grids,
    graph replay): a few problems, including the smallest and the largest, are
    bit-identical to standalone handles after two steps with the same status
    counters, and every problem's state is permissible after each step. (The
    first, forward-Euler stage of some problems is not: with the seeded states of
    problem 40 it leaves negative pressures in 64 subcells per 32^2 elements, in
    the oracle as well, and the completed SSP-RK3 step is permissible again; the
    status word reports such stages.)"""
    probs = inputs.quadrant_ensemble(64, seed=0, precision="fp32_split")
    b, u0 = _batch(probs)
    b.autotune(u0, reps=1)
    b.use_graph(True)
    u = u0.clone()
    v = torch.empty_like(u)
    dt = torch.empty(len(probs), dtype=torch.float64, device="cuda")
    for _ in range(2):
        b.rk3_step(u, v, dt)
        u, v = v, u
        for k, (cfg, _) in enumerate(probs):
            assert _permissible(b.view(u, k), cfg), k
    rc, cs = b.status()
    assert rc in (0, 4)
    flagged = [k for k, c in enumerate(cs) if c[0]]
    assert len(flagged) <= len(probs) // 4, flagged
    sizes = [int(np.prod(c["nel"])) for c, _ in probs]
    pick = sorted({int(np.argmin(sizes)), int(np.argmax(sizes)), 17, 40})
    for k in pick:
        us, dts, rck, ck = _standalone_steps(probs[k][0], probs[k][1], 2)
        assert cs[k] == ck, k
        assert torch.equal(_bits(b.view(u, k)), _bits(us)), k
        assert dt[k].item() == dts[-1]
    b.close()


def test_one_launch_stage_bit_identical_to_three_launches(mixed):
    """A stage as one persistent launch (K1, grid barrier, K2, grid barrier, K3) at
    any grid up to all CTAs resident gives the same bits as the three separate
    launches, eagerly and replayed from a captured graph."""
    probs, b, u0 = mixed
    full = _full_grids(b)
    assert all(g >= 152 for g in full)
    results = []
    for modes in ([0] * b.ngroups, full, [min(152, g) for g in full], [1] * b.ngroups):
        b.set_fused(modes)
        for graph in (False, True):
            b.use_graph(graph)
            u = u0.clone()
            v = torch.empty_like(u)
            dt = torch.empty(len(probs), dtype=torch.float64, device="cuda")
            for _ in range(2):
                b.rk3_step(u, v, dt)
                u, v = v, u
            r = torch.empty_like(u0)
            b.rhs(u0, r)
            torch.cuda.synchronize()
            results.append((modes, graph, u.clone(), r))
    b.use_graph(False)
    b.set_fused(full)
    for modes, graph, u, r in results[1:]:
        assert torch.equal(_bits(u), _bits(results[0][2])), (modes, graph)
        assert torch.equal(_bits(r), _bits(results[0][3])), (modes, graph)
    from paper_2011_03338_gb300.sesc import SescError
    with pytest.raises(SescError):
        b.set_fused([g + 1 for g in full])
    b.reset_status()


def test_grid_barrier_timeout_is_reported_not_hung(mixed):
    """Every wait at a grid barrier of the one-launch stage is bounded: with the
    bound set to 0 polls a CTA that is not the last to arrive gives up at once, the
    stage ends early and the batch status reports SESC_ETIMEOUT; with the default
    bound back, the next stage runs normally."""
    from paper_2011_03338_gb300.sesc import SESC_ETIMEOUT
    probs, b, u0 = mixed
    _full_grids(b)
    b.reset_status()
    b.set_barrier_cap(0)
    r = torch.empty_like(u0)
    b.rhs(u0, r)
    rc, _ = b.status()
    assert rc == SESC_ETIMEOUT
    b.set_barrier_cap(1 << 24)
    b.reset_status()
    ref = torch.empty_like(u0)
    b.set_fused([0] * b.ngroups)
    b.rhs(u0, ref)
    _full_grids(b)
    b.rhs(u0, r)
    assert b.status()[0] == 0
    assert torch.equal(_bits(r), _bits(ref))


def _full_grids(b):
    """The largest grid of each group's one-launch stage (all CTAs resident)."""
    from paper_2011_03338_gb300.sesc import SescError
    out = []
    for gi in range(b.ngroups):
        lo, hi = 1, 152 * 64
        while lo < hi:                          # largest grid set_fused accepts
            mid = (lo + hi + 1) // 2
            trial = [0] * b.ngroups
            trial[gi] = mid
            try:
                b.set_fused(trial)
                lo = mid
            except SescError:
                hi = mid - 1
        out.append(lo)
    b.set_fused(out)
    return out
