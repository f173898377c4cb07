"""cr_state (id order established on the device) and cr_load round trips,
through the C ABI.

  * arrays come out ordered by id -- input ids ascending, then inserted ions
    (ids >= 2^32) ascending -- and equal the oracle's particles, with the
    interaction classes cr_load takes;
  * before any insertion (no ion to sort), after one sweep and after many;
  * cr_load of a read-back reproduces the configuration (ids become the
    indices) and its counts, and sweeps continue from it;
  * pinned host buffers (raw pointers) give the same arrays as numpy arrays;
  * a batch read (cr_batch_state) equals the contexts' own reads;
  * cr_load checks on the device: a non-neutral configuration, a moved site
    and a particle outside the box are reported at the next check.
"""
import numpy as np
import pytest

import oracle
from paper_2109_07527_gb300 import workloads as W
from parity_util import compare_states

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def crmc():
    from paper_2109_07527_gb300 import crmc as m
    m._lib()
    return m


def _expected_cls(w, s):
    ids, t = s["id"], s["type"]
    ion = (t == W.XP) | (t == W.XM)
    base = w.cls[np.minimum(ids, w.n - 1).astype(np.int64)]
    return np.where(ion, int(w.params["ion_cls"]), base).astype(np.int32)


@pytest.mark.parametrize("sweeps", [0, 1, 6])
def test_state_is_id_ordered_and_matches_oracle(crmc, sweeps):
    w = W.config2(seed=4, scale=0.5)
    g = crmc.Context(w)
    o = oracle.Oracle(w)
    if sweeps:
        g.sweep(g.trials_per_sweep * sweeps, 21)
        o.sweep(o.trials_per_sweep * sweeps, 21)
    sg, _ = compare_states(g, o, w.n_sites)
    ids = sg["id"]
    assert np.all(ids[1:] > ids[:-1])
    inserted = ids >= np.uint64(1 << 32)
    if inserted.any():  # inserted ions after every input particle
        assert np.all(inserted[int(np.argmax(inserted)):])
    if sweeps == 0:
        assert not inserted.any() and np.array_equal(ids, np.arange(w.n, dtype=np.uint64))
    else:
        assert inserted.sum() > 0
    assert np.array_equal(sg["cls"], _expected_cls(w, sg))


def test_load_round_trip(crmc):
    w = W.config2(seed=5, scale=0.5, pH=6.0)
    g = crmc.Context(w)
    g.sweep(g.trials_per_sweep * 4, 3)
    g.md_step(2, 0.005, 1.0, 9)
    s = g.state()
    n = int(s["n"])
    h = crmc.Context(w)
    h.load(n, np.ascontiguousarray(s["xyz"]), np.ascontiguousarray(s["vel"]), s["type"], s["cls"], s["state"])
    t = h.state()
    assert np.array_equal(t["id"], np.arange(n, dtype=np.uint64))
    for k in ("xyz", "vel", "type", "state", "cls", "site_state"):
        assert np.array_equal(t[k], s[k]), k
    for k in ("n", "n_A", "n_Am", "n_B", "n_Bp", "n_Xp", "n_Xm", "net_charge"):
        assert t[k] == s[k], k
    h.sweep(h.trials_per_sweep * 2, 4)
    h.check()
    u = h.state()
    assert u["net_charge"] == 0 and np.all(u["id"][1:] > u["id"][:-1])


def test_state_into_pinned_buffers(crmc):
    torch = pytest.importorskip("torch")
    w = W.config2(seed=6, scale=0.5)
    g = crmc.Context(w)
    g.sweep(g.trials_per_sweep * 3, 8)
    ref = g.state()
    cap = w.capacity
    b = dict(xyz=torch.empty((cap, 3), dtype=torch.float32).pin_memory(),
             vel=torch.empty((cap, 3), dtype=torch.float32).pin_memory(),
             id=torch.empty(cap, dtype=torch.int64).pin_memory(),
             type=torch.empty(cap, dtype=torch.int32).pin_memory(),
             state=torch.empty(cap, dtype=torch.int8).pin_memory(),
             cls=torch.empty(cap, dtype=torch.int32).pin_memory())
    c = g.state_into(**{k: v.data_ptr() for k, v in b.items()})
    n = int(c["n"])
    assert n == int(ref["n"])
    assert np.array_equal(b["xyz"].numpy()[:n], ref["xyz"])
    assert np.array_equal(b["vel"].numpy()[:n], ref["vel"])
    assert np.array_equal(b["id"].numpy()[:n].view(np.uint64), ref["id"])
    assert np.array_equal(b["type"].numpy()[:n], ref["type"])
    assert np.array_equal(b["state"].numpy()[:n], ref["state"])
    assert np.array_equal(b["cls"].numpy()[:n], ref["cls"])


def test_batch_state_equals_context_states(crmc):
    ws = [W.config2(seed=9, scale=0.5, pH=pH) for pH in (3.0, 5.0, 7.0)]
    ctxs = [crmc.Context(w) for w in ws]
    b = crmc.Batch(ctxs)
    b.sweep(3, 5)
    refs = [g.state() for g in ctxs]
    arrs = []
    for w in ws:
        cap = w.capacity
        arrs.append(dict(xyz=np.zeros((cap, 3), np.float32), vel=np.zeros((cap, 3), np.float32),
                         id=np.zeros(cap, np.uint64), type=np.zeros(cap, np.int32), state=np.zeros(cap, np.int8),
                         cls=np.zeros(cap, np.int32), site_state=np.zeros(max(w.n_sites, 1), np.int8)))
    counts = b.state_into(arrs)
    for ref, a, c, w in zip(refs, arrs, counts, ws):
        n = int(c["n"])
        assert n == int(ref["n"]) and c["n_Am"] == ref["n_Am"] and c["alpha"] == ref["alpha"]
        for k in ("xyz", "vel", "id", "type", "state", "cls"):
            assert np.array_equal(a[k][:n], ref[k]), k
        assert np.array_equal(a["site_state"][:w.n_sites], ref["site_state"])


@pytest.mark.parametrize("fault", ["not_neutral", "site_moved", "outside"])
def test_load_errors_reported_at_the_next_check(crmc, fault):
    w = W.config2(seed=10, scale=0.5)
    g = crmc.Context(w)
    s = g.state()
    n = int(s["n"])
    xyz, t, st = s["xyz"].copy(), s["type"].copy(), s["state"].copy()
    if fault == "not_neutral":
        k = int(np.flatnonzero(t == W.XP)[0])
        t[k] = W.XM
        code = "NOT_NEUTRAL"
    elif fault == "site_moved":
        k = int(np.flatnonzero(t == W.ACID)[0])
        t[k] = W.BEAD
        code = "INVALID_ARG"
    else:
        xyz[0, 0] = np.float32(w.params["box_L"]) * 2
        code = "INVALID_ARG"
    h = crmc.Context(w)
    h.load(n, xyz, s["vel"], t, s["cls"], st)  # checked on the device
    with pytest.raises(crmc.CrError) as e:
        h.check()
    assert crmc.ERRORS[e.value.code] == code


def test_state_with_more_ions_than_one_cta_sorts(crmc):
    """Past 16,384 inserted ions the ions are ordered by the device-wide radix
    sort instead of the one-CTA sort: ghost ions at high salt (pI_S = 0.5) fill
    an empty L = 120 box within three sweeps; the state still equals the
    oracle's."""
    import dataclasses
    w = dataclasses.replace(W.ideal(n_sites=10, L=120.0, pIS=0.5, n_pairs=20, seed=3), capacity=48000)
    g = crmc.Context(w)
    o = oracle.Oracle(w)
    g.sweep(g.trials_per_sweep * 3, 11)
    o.sweep(o.trials_per_sweep * 3, 11)
    sg, _ = compare_states(g, o, w.n_sites)
    assert int(np.sum(sg["id"] >= np.uint64(1 << 32))) > 16384
    assert np.all(sg["id"][1:] > sg["id"][:-1])


def test_batch_load_equals_context_loads(crmc):
    ws = [W.config2(seed=12, scale=0.5, pH=pH) for pH in (3.5, 6.5)]
    src = [crmc.Context(w) for w in ws]
    for r, g in enumerate(src):
        g.sweep(g.trials_per_sweep * 2, 30 + r)
    states = [g.state() for g in src]
    single = [crmc.Context(w) for w in ws]
    batched = [crmc.Context(w) for w in ws]
    b = crmc.Batch(batched)
    loads = [dict(n=int(s["n"]), xyz=np.ascontiguousarray(s["xyz"]), vel=np.ascontiguousarray(s["vel"]),
                  type=s["type"], cls=s["cls"], state=s["state"]) for s in states]
    for g, a in zip(single, loads):
        g.load(a["n"], a["xyz"], a["vel"], a["type"], a["cls"], a["state"])
    b.load(loads)
    for g1, g2 in zip(single, batched):
        s1, s2 = g1.state(), g2.state()
        for k in ("id", "xyz", "vel", "type", "state", "cls", "site_state"):
            assert np.array_equal(s1[k], s2[k]), k
    b.sweep(1, 7)
    for g in batched:
        g.check()


def test_packed_batch_state_and_load(crmc):
    """cr_batch_state_packed equals the contexts' own reads (replica r's
    block at r * stride); cr_batch_load_packed of those arrays equals the
    per-context loads; the batch then sweeps on."""
    ws = [W.config2(seed=13, scale=0.5, pH=pH) for pH in (3.0, 5.0, 7.0)]
    ctxs = [crmc.Context(w) for w in ws]
    b = crmc.Batch(ctxs)
    b.sweep(3, 21)
    refs = [g.state() for g in ctxs]
    R, S = len(ws), max(w.capacity for w in ws) + 5
    arr = dict(xyz=np.zeros((R * S, 3), np.float32), vel=np.zeros((R * S, 3), np.float32),
               id=np.zeros(R * S, np.uint64), type=np.zeros(R * S, np.int32), cls=np.zeros(R * S, np.int32),
               state=np.zeros(R * S, np.int8))
    n = np.zeros(R, np.int64)
    b.state_packed(S, arr, n)
    for r, ref in enumerate(refs):
        k = int(n[r])
        assert k == int(ref["n"])
        for key in ("xyz", "vel", "id", "type", "cls", "state"):
            assert np.array_equal(arr[key][r * S:r * S + k], ref[key]), (r, key)
    fresh = [crmc.Context(w) for w in ws]
    single = [crmc.Context(w) for w in ws]
    bf = crmc.Batch(fresh)
    bf.load_packed(S, {k: arr[k] for k in ("xyz", "vel", "type", "cls", "state")}, n)
    for r, g in enumerate(single):
        k = int(n[r])
        g.load(k, arr["xyz"][r * S:r * S + k].copy(), arr["vel"][r * S:r * S + k].copy(),
               arr["type"][r * S:r * S + k].copy(), arr["cls"][r * S:r * S + k].copy(),
               arr["state"][r * S:r * S + k].copy())
    for g1, g2 in zip(single, fresh):
        s1, s2 = g1.state(), g2.state()
        for key in ("id", "xyz", "vel", "type", "state", "cls", "site_state"):
            assert np.array_equal(s1[key], s2[key]), key
    bf.sweep(1, 8)
    for g in fresh:
        g.check()
    n2 = np.zeros(R, np.int64)
    bf.state_packed(S, {"id": np.zeros(R * S, np.uint64)}, n2)
    assert np.all(n2 > 0)


def test_packed_batch_state_with_a_replica_beyond_the_batched_ranking(crmc):
    """In a packed batch read a replica with more than 16,384 inserted ions
    (past the batched ranking) is read by itself, the others by the batched
    kernels; every block equals the context's own read."""
    import dataclasses
    ws = [dataclasses.replace(W.ideal(n_sites=10, L=120.0, pIS=pis, n_pairs=20, seed=3 + i), capacity=48000)
          for i, pis in enumerate((2.0, 0.5, 1.5))]
    ctxs = [crmc.Context(w) for w in ws]
    b = crmc.Batch(ctxs)
    b.sweep(3, 31)
    refs = [g.state() for g in ctxs]
    assert int(np.sum(refs[1]["id"] >= np.uint64(1 << 32))) > 16384
    assert int(np.sum(refs[0]["id"] >= np.uint64(1 << 32))) < 16384
    R, S = len(ws), 48000
    arr = dict(xyz=np.zeros((R * S, 3), np.float32), vel=np.zeros((R * S, 3), np.float32),
               id=np.zeros(R * S, np.uint64), type=np.zeros(R * S, np.int32), cls=np.zeros(R * S, np.int32),
               state=np.zeros(R * S, np.int8))
    n = np.zeros(R, np.int64)
    for _ in range(2):  # twice: the marks of the first read are cleared
        b.state_packed(S, arr, n)
        for r, ref in enumerate(refs):
            k = int(n[r])
            assert k == int(ref["n"])
            for key in ("xyz", "vel", "id", "type", "cls", "state"):
                assert np.array_equal(arr[key][r * S:r * S + k], ref[key]), (r, key)
    b.close()


def test_packed_batch_io_on_pinned_memory(crmc):
    """Pinned host arrays (read in place by the load kernels) give the same
    results as pageable arrays, both ways."""
    torch = pytest.importorskip("torch")
    ws = [W.config2(seed=14, scale=0.5, pH=pH) for pH in (4.0, 6.0)]
    ctxs = [crmc.Context(w) for w in ws]
    b = crmc.Batch(ctxs)
    b.sweep(2, 17)
    R, S = len(ws), max(w.capacity for w in ws)
    ref = dict(xyz=np.zeros((R * S, 3), np.float32), vel=np.zeros((R * S, 3), np.float32),
               id=np.zeros(R * S, np.uint64), type=np.zeros(R * S, np.int32), cls=np.zeros(R * S, np.int32),
               state=np.zeros(R * S, np.int8))
    nref = np.zeros(R, np.int64)
    b.state_packed(S, ref, nref)
    pk = dict(xyz=torch.zeros((R * S, 3), dtype=torch.float32).pin_memory(),
              vel=torch.zeros((R * S, 3), dtype=torch.float32).pin_memory(),
              id=torch.zeros(R * S, dtype=torch.int64).pin_memory(),
              type=torch.zeros(R * S, dtype=torch.int32).pin_memory(),
              cls=torch.zeros(R * S, dtype=torch.int32).pin_memory(),
              state=torch.zeros(R * S, dtype=torch.int8).pin_memory())
    n = torch.zeros(R, dtype=torch.int64).pin_memory()
    b.state_packed(S, {k: v.data_ptr() for k, v in pk.items()}, n.data_ptr())
    assert np.array_equal(n.numpy(), nref)
    for r in range(R):
        k = int(nref[r])
        for key in ref:
            got = pk[key].numpy()[r * S:r * S + k]
            if key == "id":
                got = got.view(np.uint64)
            assert np.array_equal(got, ref[key][r * S:r * S + k]), (r, key)
    # load in place from the pinned arrays into fresh contexts, read back again
    fresh = [crmc.Context(w) for w in ws]
    bf = crmc.Batch(fresh)
    bf.load_packed(S, {k: pk[k].data_ptr() for k in ("xyz", "vel", "type", "cls", "state")}, n.data_ptr())
    back = dict(xyz=np.zeros((R * S, 3), np.float32), type=np.zeros(R * S, np.int32), state=np.zeros(R * S, np.int8))
    nb = np.zeros(R, np.int64)
    bf.state_packed(S, back, nb)
    assert np.array_equal(nb, nref)
    for r in range(R):
        k = int(nref[r])
        for key in back:
            assert np.array_equal(back[key][r * S:r * S + k], ref[key][r * S:r * S + k]), (r, key)
