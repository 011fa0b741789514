"""Partitioned meshes on the GPU: a mesh split into slabs along its last axis
(paper_2011_03338_gb300.shard), the parts exchanging only their boundary
face-centred states and level weights (sesc_pack_halo / sesc_set_halo) and the
minimum time step, must reproduce the unpartitioned handle bit for bit: the right-
hand side and several SSP-RK3 steps, walls and periodic rings, 2D and 3D, both
precisions. The parts run in one process on one GPU, one after the other between
exchanges (no kernel waits on another)."""
import numpy as np
import pytest

from paper_2011_03338_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _state(name):
    if name == "sedov2d_M8_12":
        return inputs.sedov(2, 8, 12)
    if name == "kh_M8_8":
        return inputs.kelvin_helmholtz(8, 8)
    if name == "sedov3d_M4_6":
        return inputs.sedov(3, 4, 6)
    if name == "quadrants_M4_10":
        return inputs.quadrants(4, 10, seed=3)
    if name == "sedov2d_M8_160":
        return inputs.sedov(2, 8, 160)
    raise KeyError(name)


CASES = [("sedov2d_M8_12", 2, "fp64"), ("sedov2d_M8_12", 3, "fp64"), ("kh_M8_8", 2, "fp64"), ("kh_M8_8", 4, "fp64"),
         ("sedov3d_M4_6", 3, "fp64"), ("quadrants_M4_10", 3, "fp64"), ("sedov2d_M8_12", 3, "fp32_split"),
         ("kh_M8_8", 2, "fp32_split"),
         # 25,600 elements: on a GB300 the whole mesh's update kernel takes its elements
         # class by class (at least 8 waves of resident CTAs), the parts' in mesh order
         ("sedov2d_M8_160", 2, "fp32_split"), ("sedov2d_M8_160", 4, "fp64")]


@pytest.mark.parametrize("name,parts,precision", CASES)
def test_partitioned_mesh_matches_the_whole_mesh_bit_for_bit(name, parts, precision):
    from paper_2011_03338_gb300 import Solver
    from paper_2011_03338_gb300.shard import LocalGroup
    cfg, u = _state(name)
    cfg = dict(cfg, precision=precision)
    whole = Solver(cfg)
    group = LocalGroup(cfg, parts)
    ud = torch.from_numpy(u).cuda()
    r = torch.empty_like(ud)
    whole.rhs(ud, r)
    rp = torch.full_like(ud, float("nan"))
    group.rhs(group.split(ud), group.split(rp))
    assert torch.equal(rp, r), (rp - r).abs().max().item()
    # SSP-RK3 steps: time step as the minimum over the parts
    a, b = ud.clone(), torch.empty_like(ud)
    pa, pb = ud.clone(), torch.empty_like(ud)
    s1, s2 = torch.empty_like(ud), torch.empty_like(ud)
    dt_w = torch.empty(1, dtype=torch.float64, device="cuda")
    dt_p = torch.empty(1, dtype=torch.float64, device="cuda")
    for _ in range(3):
        whole.rk3_step(a, b, dt_w)
        group.rk3_step(group.split(pa), group.split(pb), dt_p, (group.split(s1), group.split(s2)))
        assert torch.equal(dt_p, dt_w)
        a, b = b, a
        pa, pb = pb, pa
    assert whole.status()[0] == 0 and all(p.solver.status()[0] == 0 for p in group.parts)
    assert torch.equal(pa, a), (pa - a).abs().max().item()


def test_halo_side_without_a_halo_is_rejected():
    """A part whose halo side has no neighbour data set refuses to evaluate."""
    from paper_2011_03338_gb300 import Solver
    from paper_2011_03338_gb300.sesc import SESC_EINVAL, SescError
    from paper_2011_03338_gb300.shard import part_config
    cfg, u = inputs.sedov(2, 4, 6)
    s = Solver(part_config(cfg, 2, 0))
    x = torch.from_numpy(u[:18]).cuda()
    with pytest.raises(SescError) as ei:
        s.rhs(x, torch.empty_like(x))
    assert ei.value.code == SESC_EINVAL
    with pytest.raises(SescError):
        s.rhs_vjp(x, torch.ones_like(x), torch.empty_like(x))
