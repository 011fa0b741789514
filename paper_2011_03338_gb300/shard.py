"""Partitioned meshes: one mesh split into Cartesian slabs of elements along its
last axis, one part per GPU (or several parts on one device), advanced together.

The parts exchange per RK stage exactly what the paper's parallel form exchanges
between processes (appendix: 3D extension and multi-level sketch, step IV): the
face-centred mean values and level weights of the element faces on the shared
sides, packed by the library (sesc_pack_halo) and handed to the neighbour
(sesc_set_halo); the time step of eq. cfl-condition is the minimum over the parts.
Both parts of a shared face evaluate its flux from the same two states, so a
partitioned run reproduces the unpartitioned one bit for bit.

This module holds the partition (slab bounds, the parts' configurations and
neighbours) and the exchange plumbing (torch.distributed point-to-point messages
between processes, or copies between parts that live in one process); every step
of the scheme runs in the library.
"""
import copy

BC_PERIODIC, BC_HALO = 0, 3


def slab_bounds(n, world, rank):
    """Element layers [r0, r1) of part `rank` when n layers are split into `world`
    contiguous slabs whose sizes differ by at most one."""
    if not (0 <= rank < world) or world > n:
        raise ValueError(f"cannot split {n} element layers into {world} parts (rank {rank})")
    base, extra = divmod(n, world)
    r0 = rank * base + min(rank, extra)
    return r0, r0 + base + (1 if rank < extra else 0)


def part_config(cfg, world, rank):
    """Configuration of part `rank`: the slab's layers along the last axis, its box,
    the whole mesh's element size, and SESC_BC_HALO on every side shared with
    another part (a periodic last axis becomes a ring of parts)."""
    d = int(cfg["dim"])
    a = d - 1
    n = int(cfg["nel"][a])
    r0, r1 = slab_bounds(n, world, rank)
    c = copy.deepcopy(dict(cfg))
    if world == 1:
        return c
    dx = (cfg["xhi"][a] - cfg["xlo"][a]) / n
    nel, xlo, xhi, bc = list(cfg["nel"]), list(cfg["xlo"]), list(cfg["xhi"]), list(cfg["bc"])
    nel[a] = r1 - r0
    xlo[a] = cfg["xlo"][a] + r0 * dx
    xhi[a] = cfg["xlo"][a] + r1 * dx
    periodic = cfg["bc"][2 * a] == BC_PERIODIC
    bc[2 * a] = BC_HALO if (r0 > 0 or periodic) else cfg["bc"][2 * a]
    bc[2 * a + 1] = BC_HALO if (r1 < n or periodic) else cfg["bc"][2 * a + 1]
    # the element size is given, not derived from the part's box: the part's factors
    # M / dx are then the whole mesh's to the last bit
    esz = [(cfg["xhi"][b] - cfg["xlo"][b]) / cfg["nel"][b] for b in range(d)]
    c.update(nel=tuple(nel), xlo=tuple(xlo), xhi=tuple(xhi), bc=tuple(bc), elem_size=tuple(esz))
    return c


def neighbours(cfg, world, rank):
    """{halo side: neighbour rank} of part `rank` (sides 2a and 2a + 1 of the last axis a)."""
    a = int(cfg["dim"]) - 1
    pc = part_config(cfg, world, rank)
    out = {}
    if pc["bc"][2 * a] == BC_HALO:
        out[2 * a] = (rank - 1) % world
    if pc["bc"][2 * a + 1] == BC_HALO:
        out[2 * a + 1] = (rank + 1) % world
    return out


def element_range(cfg, world, rank):
    """[e0, e1): part `rank`'s elements in the whole mesh's element order (the last
    axis is the slowest, so a slab is one contiguous range)."""
    d = int(cfg["dim"])
    ntr = 1
    for b in range(d - 1):
        ntr *= int(cfg["nel"][b])
    r0, r1 = slab_bounds(int(cfg["nel"][d - 1]), world, rank)
    return r0 * ntr, r1 * ntr


def messages(cfg, world, rank):
    """The point-to-point messages of one exchange for part `rank`, in the order
    both ends issue them: sends ordered by the sender's side, receives ordered by the
    side the sender packed (the side opposite to the receiving halo side), so that
    two messages between the same pair of parts (a ring of two) match in order.
    Returns (sends, recvs): lists of (peer, packed side) and (peer, halo side)."""
    nb = neighbours(cfg, world, rank)
    sends = [(nb[s], s) for s in sorted(nb)]
    recvs = sorted(((nb[s], s) for s in nb), key=lambda x: (x[0], x[1] ^ 1))
    sends.sort(key=lambda x: (x[0], x[1]))
    return sends, recvs


class Part:
    """One part: a handle of the library on its slab, with its send / receive
    buffers (uint8 device tensors of sesc_halo_bytes) registered as halos once."""

    def __init__(self, cfg, world, rank, device=None):
        import torch

        from .sesc import Solver
        self.cfg, self.world, self.rank = dict(cfg), world, rank
        self.local = part_config(cfg, world, rank)
        if device is not None:
            torch.cuda.set_device(device)
        self.solver = Solver(self.local)
        self.nb = neighbours(cfg, world, rank)
        dev = self.solver.device
        self.send = {s: torch.empty(self.solver.halo_bytes(s), dtype=torch.uint8, device=dev) for s in self.nb}
        self.recv = {s: torch.empty(self.solver.halo_bytes(s), dtype=torch.uint8, device=dev) for s in self.nb}
        for s, buf in self.recv.items():
            self.solver.set_halo(s, buf)
        self.e0, self.e1 = element_range(cfg, world, rank)

    def begin(self, us):
        """K1 on the part's state and the packed face states of its halo sides."""
        self.solver.indicator(us)
        for s, buf in self.send.items():
            self.solver.pack_halo(s, buf)

    def finish(self, us, out, u0=None, a=0.0, b=1.0, dt_dev=None, mode=1):
        self.solver.stage_finish(us, out, u0=u0, a=a, b=b, dt_dev=dt_dev, mode=mode)


class LocalGroup:
    """Several parts of one mesh in one process (on one or several devices): the
    exchange is a device copy from each part's send buffer to its neighbour's
    receive buffer on the current stream. For tests and single-GPU use."""

    def __init__(self, cfg, world):
        self.cfg, self.world = dict(cfg), world
        self.parts = [Part(cfg, world, r) for r in range(world)]

    def split(self, u):
        """The parts' states (views) of a whole-mesh state tensor [E][nv][M^d]."""
        return [u[p.e0:p.e1] for p in self.parts]

    def exchange(self):
        for p in self.parts:
            for s, peer in p.nb.items():
                # my halo side s holds the neighbour's packed opposite side
                p.recv[s].copy_(self.parts[peer].send[s ^ 1])

    def rhs(self, us, out):
        for p, x in zip(self.parts, us):
            p.begin(x)
        self.exchange()
        for p, x, o in zip(self.parts, us, out):
            p.finish(x, o, mode=0)

    def dt(self, u, dt_dev):
        import torch
        vals = []
        for p, x in zip(self.parts, u):
            t = torch.empty(1, dtype=torch.float64, device=x.device)
            p.solver.dt(x, t)
            vals.append(t)
        dt_dev.copy_(torch.stack(vals).min(dim=0).values)

    def rk3_step(self, u, uout, dt_dev, stage_bufs):
        """One SSP-RK3 step of every part; u, uout, stage_bufs[0..1]: lists of the
        parts' states."""
        self.dt(u, dt_dev)
        srcs = [u, stage_bufs[0], stage_bufs[1]]
        dsts = [stage_bufs[0], stage_bufs[1], uout]
        for (a, b), us, out in zip(((0.0, 1.0), (0.75, 0.25), (1.0 / 3.0, 2.0 / 3.0)), srcs, dsts):
            for p, x in zip(self.parts, us):
                p.begin(x)
            self.exchange()
            for p, x, o, x0 in zip(self.parts, us, out, u):
                p.finish(x, o, u0=x0, a=a, b=b, dt_dev=dt_dev, mode=1)


def exchange_p2p(send, recv, sends, recvs, group=None):
    """One halo exchange between ranks: send[side] (packed face states of this
    rank's side) to each neighbour, recv[side] (the neighbour's packed opposite side)
    from each, with the message order of `messages`. Works for CUDA tensors (NCCL)
    and CPU tensors (gloo)."""
    import torch.distributed as dist
    ops = [dist.P2POp(dist.isend, send[s], peer, group=group) for peer, s in sends]
    ops += [dist.P2POp(dist.irecv, recv[s], peer, group=group) for peer, s in recvs]
    if ops:
        for r in dist.batch_isend_irecv(ops):
            r.wait()


class DistPart:
    """This process's part of a mesh split over torch.distributed ranks (one part per
    rank, one GPU per rank): halo messages are point-to-point sends and receives
    between neighbouring ranks (NCCL on GPUs), the time step an all-reduce (MIN)."""

    def __init__(self, cfg, group=None):
        import torch.distributed as dist
        self.group = group
        self.world, self.rank = dist.get_world_size(group), dist.get_rank(group)
        self.part = Part(cfg, self.world, self.rank)
        self.sends, self.recvs = messages(cfg, self.world, self.rank)

    @property
    def solver(self):
        return self.part.solver

    def exchange(self):
        exchange_p2p(self.part.send, self.part.recv, self.sends, self.recvs, self.group)

    def dt(self, u, dt_dev):
        import torch.distributed as dist
        self.part.solver.dt(u, dt_dev)
        if self.world > 1:
            dist.all_reduce(dt_dev, op=dist.ReduceOp.MIN, group=self.group)

    def rhs(self, us, out):
        self.part.begin(us)
        self.exchange()
        self.part.finish(us, out, mode=0)

    def rk3_step(self, u, uout, dt_dev, stage_bufs):
        self.dt(u, dt_dev)
        srcs = [u, stage_bufs[0], stage_bufs[1]]
        dsts = [stage_bufs[0], stage_bufs[1], uout]
        for (a, b), us, out in zip(((0.0, 1.0), (0.75, 0.25), (1.0 / 3.0, 2.0 / 3.0)), srcs, dsts):
            self.part.begin(us)
            self.exchange()
            self.part.finish(us, out, u0=u, a=a, b=b, dt_dev=dt_dev, mode=1)
