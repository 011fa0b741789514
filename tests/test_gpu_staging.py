"""Bulk-copy staging of an element's means (cp.async.bulk into shared memory,
completed on an mbarrier): the wait is bounded, a kernel that gives up reports it
through the status word and skips the element, and the context stays usable.

No GPU is faulted or hung here: a bound of 0 polls makes the kernels give up at
once, after a second bounded wait lets each copy land."""
import pytest

from paper_2011_03338_gb300 import Solver, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "fp32_split"])
def test_staging_wait_timeout_is_reported_not_hung(precision):
    from paper_2011_03338_gb300.sesc import SESC_ETIMEOUT
    cfg, u = inputs.sedov(2, 8, 12, precision=precision)
    s = Solver(cfg)
    ud = torch.from_numpy(u).cuda()
    ref = torch.empty_like(ud)
    s.rhs(ud, ref)
    assert s.status()[0] == 0
    # every element of the update kernel is staged: with 0 polls each one gives up
    # and its output is left as it was
    s.reset_status()
    s.set_stage_cap(0)
    r = torch.full_like(ud, 7.0)
    s.rhs(ud, r)
    rc, c = s.status()
    assert rc == SESC_ETIMEOUT and (c[0] & 4)
    assert bool((r == 7.0).all())
    # the default bound back: the same call is bit for bit the first one
    s.set_stage_cap(1 << 22)
    s.reset_status()
    s.rhs(ud, r)
    assert s.status()[0] == 0
    assert torch.equal(r, ref)
    with pytest.raises(Exception):
        s.set_stage_cap(-1)


def test_unaligned_state_takes_the_plain_loads():
    """A state whose elements are not 16-byte aligned (an odd offset into a larger
    buffer) cannot be bulk-copied; the kernels load it with plain loads and give the
    same result as an aligned copy."""
    cfg, u = inputs.sedov(2, 4, 10)
    s = Solver(cfg)
    ud = torch.from_numpy(u).cuda()
    big = torch.empty(ud.numel() + 1, dtype=torch.float64, device="cuda")
    mis = big[1:].view_as(ud)   # 8-byte offset from a 256-byte aligned allocation
    mis.copy_(ud)
    assert mis.data_ptr() % 16 == 8
    ref = torch.empty_like(ud)
    s.rhs(ud, ref)
    bigo = torch.empty(ud.numel() + 1, dtype=torch.float64, device="cuda")
    out = bigo[1:].view_as(ud)
    s.rhs(mis, out)
    assert s.status()[0] == 0
    assert torch.equal(out, ref)
