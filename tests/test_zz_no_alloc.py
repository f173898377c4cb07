"""cr_md_forces_noalloc (forces into caller-owned device memory, scratch in a
fixed device array of the library) against cr_md_forces through the C ABI,
on two calls in a row.  Kept in its own file, collected last, so that it runs
both alone in a fresh process and after every other GPU test."""
import numpy as np
import pytest

from paper_2109_07527_gb300 import workloads as W

pytestmark = pytest.mark.gpu

EMPTY = np.uint64(0xFFFFFFFFFFFFFFFF)
CR_NOALLOC_MAX_PARTICLES = 262144  # include/crmc.h
CR_ERR_CAPACITY = -4
CR_ERR_INVALID_ARG = -1


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_07527_gb300 import crmc
    crmc._lib()
    return torch, crmc


def _slots(ctx):
    i = ctx.info
    return i["nc"] ** 3 * i["cap"]


def _noalloc(torch, ctx, n_slots):
    force = torch.full((n_slots, 4), float("nan"), dtype=torch.float32, device="cuda")
    ids = torch.full((n_slots,), 7, dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    ctx.md_forces_noalloc(force.data_ptr(), ids.data_ptr(), n_slots)
    torch.cuda.synchronize()
    return force.cpu().numpy(), ids.cpu().numpy().view(np.uint64)


def _check(ref, force, ids):
    full = ids != EMPTY
    assert np.all(force[~full] == 0.0)
    order = np.argsort(ids[full], kind="stable")
    got_id = ids[full][order]
    got_f = force[full][order][:, :3].astype(np.float64)
    assert np.array_equal(got_id, ref["id"])
    # the same FP32 pair terms summed in the same exact 2^-24 fixed point:
    # equal to the bit, although this entry runs the lane-0 finishing variant
    # without the flat frame (the flat-frame differences are exact) and
    # evaluates every pair from both ends, where cr_md_forces evaluates each
    # pair once over half the stencil and adds the partner's share by atomics
    assert np.array_equal(got_f, ref["force"].astype(np.float64))
    assert np.all(force[full][:, 3] == 0.0)


@pytest.mark.parametrize("case", ["chain_after_sweeps", "polyelectrolyte_full"])
def test_noalloc_forces_match_cr_md_forces(env, case):
    torch, crmc = env
    if case == "chain_after_sweeps":
        w = W.config1(seed=5)
        ctx = crmc.Context(w)
        ctx.sweep(ctx.trials_per_sweep * 4, 3)  # inserted ions carry ids >= 2^32
    else:
        w = W.config2(seed=1)
        ctx = crmc.Context(w)
    ctx.md_forces()
    ref = ctx.state()
    assert np.abs(ref["force"]).max() > 1.0  # the comparison is not vacuous
    n_slots = _slots(ctx)
    for _ in range(2):  # two calls in a row
        force, ids = _noalloc(torch, ctx, n_slots)
        _check(ref, force, ids)
    # the context's own forces are untouched
    after = ctx.state()
    assert np.array_equal(after["force"], ref["force"])
    ctx.close()


def test_noalloc_rejects_capacity_beyond_the_scratch(env):
    torch, crmc = env
    w = W.config1(seed=2)
    w.capacity = CR_NOALLOC_MAX_PARTICLES + 1
    ctx = crmc.Context(w)
    n_slots = _slots(ctx)
    force = torch.zeros((n_slots, 4), dtype=torch.float32, device="cuda")
    ids = torch.zeros((n_slots,), dtype=torch.int64, device="cuda")
    with pytest.raises(crmc.CrError) as e:
        ctx.md_forces_noalloc(force.data_ptr(), ids.data_ptr(), n_slots)
    assert e.value.code == CR_ERR_CAPACITY
    with pytest.raises(crmc.CrError):  # output smaller than the slot count
        ctx.md_forces_noalloc(force.data_ptr(), ids.data_ptr(), n_slots - 1)
    ctx.close()


def test_noalloc_rejects_bad_pointers_before_any_launch(env):
    """A force array off its 16-byte alignment, an id array off its 8-byte
    alignment and NULL arrays are refused with CR_ERR_INVALID_ARG before
    anything is launched; a following valid call still works."""
    torch, crmc = env
    w = W.config1(seed=3)
    ctx = crmc.Context(w)
    ctx.md_forces()
    ref = ctx.state()
    n_slots = _slots(ctx)
    force = torch.zeros((n_slots + 1, 4), dtype=torch.float32, device="cuda")
    ids = torch.zeros((n_slots + 1,), dtype=torch.int64, device="cuda")
    f, i = force.data_ptr(), ids.data_ptr()
    for fp, ip in ((f + 4, i), (f + 8, i), (f, i + 4), (0, i), (f, 0)):
        with pytest.raises(crmc.CrError) as e:
            ctx.md_forces_noalloc(fp, ip, n_slots)
        assert e.value.code == CR_ERR_INVALID_ARG
    got_f, got_i = _noalloc(torch, ctx, n_slots)
    _check(ref, got_f, got_i)
    ctx.close()
