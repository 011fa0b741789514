"""The partition of a mesh into slabs (paper_2011_03338_gb300.shard) on CPU: slab
bounds, the parts' configurations and neighbours, the message order of the halo
exchange, and a world-size-2 run over torch.distributed (gloo) whose parts compute
with the oracle: each rank evaluates its slab, exchanges the face-centred states
and level weights of its shared faces (the data the paper's parallel form
exchanges, appendix 3D extension) and the time step, and the gathered result must
equal the whole mesh's oracle right-hand side bit for bit."""
import os
import socket

import numpy as np
import pytest

from paper_2011_03338_gb300 import inputs
from paper_2011_03338_gb300.shard import element_range, messages, neighbours, part_config, slab_bounds


def test_slab_bounds_cover_the_layers():
    for n in (1, 5, 12, 64):
        for world in range(1, min(n, 9) + 1):
            b = [slab_bounds(n, world, r) for r in range(world)]
            assert b[0][0] == 0 and b[-1][1] == n
            assert all(b[i][1] == b[i + 1][0] for i in range(world - 1))
            sizes = [r1 - r0 for r0, r1 in b]
            assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 1
    with pytest.raises(ValueError):
        slab_bounds(3, 4, 0)


@pytest.mark.parametrize("periodic", [False, True])
@pytest.mark.parametrize("world", [2, 3, 4])
def test_part_configs_and_message_pairing(world, periodic):
    bc = (1, 2, 0, 0) if periodic else (1, 2, 1, 2)
    cfg = inputs.make_config(2, 4, (5, 9), (0.0, -1.0), (1.0, 2.0), bc)
    dx = 3.0 / 9
    for r in range(world):
        pc = part_config(cfg, world, r)
        r0, r1 = slab_bounds(9, world, r)
        assert pc["nel"] == (5, r1 - r0) and pc["bc"][:2] == (1, 2)
        assert abs(pc["xlo"][1] - (-1.0 + r0 * dx)) < 1e-15 and abs(pc["xhi"][1] - (-1.0 + r1 * dx)) < 1e-15
        assert pc["bc"][2] == (3 if (r > 0 or periodic) else 1)
        assert pc["bc"][3] == (3 if (r < world - 1 or periodic) else 2)
        e0, e1 = element_range(cfg, world, r)
        assert (e0, e1) == (5 * r0, 5 * r1)
    # every send has a matching receive, in the same position among the messages
    # between that pair of ranks
    for r in range(world):
        sends, _ = messages(cfg, world, r)
        for peer in {p for p, _ in sends}:
            out = [s for p, s in sends if p == peer]
            _, precv = messages(cfg, world, peer)
            inn = [s for p, s in precv if p == r]
            assert [s ^ 1 for s in out] == inn, (r, peer, out, inn)
    nb = [neighbours(cfg, world, r) for r in range(world)]
    assert (2 in nb[0]) == periodic and (3 in nb[-1]) == periodic


def _pack(states):
    """(U (nv, 1, G), {level: theta (1, G)}) -> flat float64 vector (levels sorted)."""
    U, th = states
    return np.concatenate([U.ravel()] + [th[n].ravel() for n in sorted(th)])


def _unpack(vec, like):
    U, th = like
    out, k = U.size, {}
    Ux = vec[:U.size].reshape(U.shape)
    for n in sorted(th):
        k[n] = vec[out:out + th[n].size].reshape(th[n].shape)
        out += th[n].size
    return Ux, k


def _rank_main(rank, world, port, periodic, result):
    import torch
    import torch.distributed as dist

    from oracle.blended import Config, blended_rhs
    from oracle.layout import to_elements, to_grid
    from oracle.timestep import cfl_dt
    from paper_2011_03338_gb300.shard import exchange_p2p
    from tests.test_gpu_parity import _shock_state
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bc = (1, 2, 0, 0) if periodic else (1, 2, 1, 2)
        cfg = inputs.make_config(2, 4, (3, 6), (0.0, 0.0), (0.9, 1.8), bc)
        u = _shock_state(cfg, seed=21)
        pc = part_config(cfg, world, rank)
        e0, e1 = element_range(cfg, world, rank)
        ul = u[e0:e1]
        U = to_grid(ul, 2, 4, pc["nel"])
        # phase 1: this part's face states (element-local; the halo sides' own
        # boundary conditions do not enter them)
        probe = dict(pc, bc=tuple(2 if b == 3 else b for b in pc["bc"]))
        _, dg = blended_rhs(U, Config(**probe), return_diag=True)
        nb = neighbours(cfg, world, rank)
        a = 1
        send = {s: torch.from_numpy(_pack(dg.boundary_states[(a, s % 2)])) for s in nb}
        recv = {s: torch.empty_like(send[s]) for s in nb}
        sends, recvs = messages(cfg, world, rank)
        exchange_p2p(send, recv, sends, recvs)
        ghost = {(a, s % 2): _unpack(recv[s].numpy(), dg.boundary_states[(a, s % 2)]) for s in nb}
        # phase 2: the part's right-hand side with the neighbours' states
        R = blended_rhs(U, Config(**pc), ghost=ghost)
        Rl = torch.from_numpy(to_elements(R, 2, 4, pc["nel"]).ravel())
        sizes = [element_range(cfg, world, r)[1] - element_range(cfg, world, r)[0] for r in range(world)]
        parts = [torch.empty(n * 4 * 16, dtype=torch.float64) for n in sizes]
        dist.all_gather(parts, Rl)
        dt = torch.tensor([cfl_dt(U, Config(**pc))], dtype=torch.float64)
        dist.all_reduce(dt, op=dist.ReduceOp.MIN)
        if rank == 0:
            whole = to_elements(blended_rhs(to_grid(u, 2, 4, cfg["nel"]), Config(**cfg)), 2, 4, cfg["nel"])
            got = torch.cat(parts).numpy().reshape(whole.shape)
            dref = cfl_dt(to_grid(u, 2, 4, cfg["nel"]), Config(**cfg))
            result.put((bool(np.array_equal(got, whole)), float(np.abs(got - whole).max()),
                        float(dt.item()) == dref))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("periodic", [False, True])
def test_two_rank_partition_reproduces_the_whole_mesh(periodic):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, periodic, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    equal, diff, dt_ok = q.get(timeout=5)
    assert equal, diff
    assert dt_ok
