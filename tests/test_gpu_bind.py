"""Device memory owned by the caller (cr_bind_device_buffers): a context whose
configuration lives in torch tensors runs the same chain, bit for bit, as one
whose configuration lives in the library's own memory; the tensors hold the
cell-list layout the header describes after every synchronising call; the
library never frees them; bad arguments are refused before anything changes."""
import numpy as np
import pytest

from paper_2109_07527_gb300 import workloads as W

pytestmark = pytest.mark.gpu

DT, GAMMA = 0.005, 1.0


@pytest.fixture(scope="module")
def crmc():
    from paper_2109_07527_gb300 import crmc as m
    m._lib()
    return m


def _buffers(g):
    import torch
    i = g.info
    ncell, nslot = i["nc"] ** 3, i["nc"] ** 3 * i["cap"]
    t = dict(cnt=torch.zeros(ncell, dtype=torch.int32, device="cuda"),
             pos=torch.zeros(4 * nslot, dtype=torch.float32, device="cuda"),
             vel=torch.zeros(4 * nslot, dtype=torch.float32, device="cuda"),
             id=torch.zeros(nslot, dtype=torch.int64, device="cuda"),
             info=torch.zeros(nslot, dtype=torch.int32, device="cuda"))
    return t, ncell, nslot, i["cap"]


def _bind(g, t, ncell, nslot, pos_off=0):
    g.bind_device_buffers(t["cnt"].data_ptr(), t["pos"].data_ptr() + pos_off, t["vel"].data_ptr(),
                          t["id"].data_ptr(), t["info"].data_ptr(), ncell, nslot)


def _cycle(g, s):
    g.md_begin(DT, GAMMA, 700 + s)
    g.sweep(g.trials_per_sweep, 300 + s)
    g.md_end(DT, GAMMA, 700 + s)


def _same(a, b):
    for k in ("id", "xyz", "vel", "type", "state", "site_state"):
        assert np.array_equal(a[k], b[k]), k
    for k in ("n", "n_Am", "n_Xp", "n_Xm"):
        assert a[k] == b[k], k


def test_bound_context_runs_the_same_chain(crmc):
    w = W.config2(seed=6, scale=0.5)
    a = crmc.Context(w)  # library memory
    b = crmc.Context(w)  # bound after one cycle
    _cycle(a, 0)
    _cycle(b, 0)
    t, ncell, nslot, cap = _buffers(b)
    _bind(b, t, ncell, nslot)
    for s in range(1, 4):
        _cycle(a, s)
        _cycle(b, s)
    sa, sb = a.state(), b.state()
    _same(sa, sb)
    assert (sb["id"] >= 2 ** 32).any()  # ions inserted while bound
    # the tensors hold the configuration in the documented layout
    cnt = t["cnt"].cpu().numpy()
    assert int(cnt.sum()) == sb["n"]
    slots = (np.arange(ncell)[:, None] * cap + np.arange(cap)[None, :])[np.arange(cap)[None, :] < cnt[:, None]]
    ids = t["id"].cpu().numpy().view(np.uint64)[slots]
    order = np.argsort(ids)
    assert np.array_equal(ids[order], sb["id"])
    pos = t["pos"].cpu().numpy().reshape(-1, 4)[slots][order]
    assert np.array_equal(pos[:, :3], sb["xyz"])
    info = t["info"].cpu().numpy()[slots][order]
    assert np.array_equal(info & 15, sb["type"])
    a.close()
    b.close()
    # the library did not free the caller's memory: it is still readable and unchanged
    assert int(t["cnt"].sum().item()) == sb["n"]


def test_bound_contexts_form_a_batch(crmc):
    ws = [W.config2(seed=7, scale=0.5, pH=p) for p in (3.0, 4.5)]
    ref = [crmc.Context(w) for w in ws]
    bnd = [crmc.Context(w) for w in ws]
    keep = []
    for g in bnd:
        t, ncell, nslot, _ = _buffers(g)
        _bind(g, t, ncell, nslot)
        keep.append(t)
    ba, bb = crmc.Batch(ref), crmc.Batch(bnd)
    for s in range(2):
        ba.cycle(1, DT, GAMMA, 40 + s, 80 + s)
        bb.cycle(1, DT, GAMMA, 40 + s, 80 + s)
    for x, y in zip(ref, bnd):
        _same(x.state(), y.state())
    ba.close()
    bb.close()
    for g in ref + bnd:
        g.close()


def test_bind_refuses_bad_buffers(crmc):
    import torch
    w = W.config2(seed=8, scale=0.5)
    g = crmc.Context(w)
    before = g.state()
    t, ncell, nslot, _ = _buffers(g)
    cases = {
        "misaligned": lambda: _bind(g, t, ncell, nslot, pos_off=4),
        "too few slots": lambda: _bind(g, t, ncell, nslot - 1),
        "too few cells": lambda: _bind(g, t, ncell - 1, nslot),
        "host memory": lambda: g.bind_device_buffers(t["cnt"].data_ptr(),
                                                     torch.zeros(4 * nslot).pin_memory().data_ptr(),
                                                     t["vel"].data_ptr(), t["id"].data_ptr(), t["info"].data_ptr(),
                                                     ncell, nslot),
        "null": lambda: g.bind_device_buffers(0, t["pos"].data_ptr(), t["vel"].data_ptr(), t["id"].data_ptr(),
                                              t["info"].data_ptr(), ncell, nslot),
    }
    for name, f in cases.items():
        with pytest.raises(crmc.CrError) as e:
            f()
        assert e.value.code == -1, name
    _same(g.state(), before)  # nothing changed
    # a context in a batch cannot be bound; once the batch is gone it can, once
    b = crmc.Batch([g])
    with pytest.raises(crmc.CrError):
        _bind(g, t, ncell, nslot)
    b.close()
    _bind(g, t, ncell, nslot)
    with pytest.raises(crmc.CrError):
        _bind(g, t, ncell, nslot)
    _same(g.state(), before)
    g.close()
