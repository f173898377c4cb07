"""The multi-rank host logic of bench.py on CPU: two gloo ranks.

Each rank runs an independent batch (different seeded structures, the same
pH grid and the same fixed work), the timed regions reduce to the slowest
rank's time, the whole-job rate counts every rank's units, and the reference
arm does its work on rank 0 only."""
import io
import multiprocessing as mp
import os
import socket
import sys
from contextlib import redirect_stdout

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    try:
        sys.path.insert(0, ROOT)
        os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                          MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        import torch.distributed as dist
        import bench
        dist.init_process_group("gloo", rank=rank, world_size=world)
        r, w, loc = bench.dist_env()
        out = {"env": (r, w, loc)}
        # each rank times a different duration; every rank gets the slowest
        out["ms"] = bench.max_over_ranks(10.0 * (rank + 1) + 0.25, "cpu")
        out["rate"] = bench.job_rate(1000, w, out["ms"] / 1e3)
        ws = bench.ph_sweep_workloads(r)
        out["pH"] = [x.params["pH"] for x in ws]
        out["n"] = [len(x.xyz) for x in ws]
        out["xyz0"] = np.asarray(ws[0].xyz[:64], dtype=np.float64)
        out["same_start"] = all(np.array_equal(ws[0].xyz, x.xyz) for x in ws)
        # the reference arm: rank 0 alone works and prints; the others return
        buf = io.StringIO()
        if r != 0:
            class A:
                steps, warmup, gpus = 1, 0, w
            with redirect_stdout(buf):
                ret = bench.run_reference(A)
            out["ref_ret"], out["ref_out"] = ret, buf.getvalue()
        dist.barrier()
        dist.destroy_process_group()
        q.put((rank, out))
    except BaseException as e:  # reported to the parent, which fails the test
        q.put((rank, {"error": repr(e)}))


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(2):
        assert "error" not in res[r], res[r]
        assert res[r]["env"] == (r, 2, r)
        # the slowest rank's time on both ranks
        assert res[r]["ms"] == 20.25
        # 1000 units on each of 2 ranks in 20.25 ms
        assert abs(res[r]["rate"] - 2000 / 0.02025) < 1e-6
        assert res[r]["pH"] == [2.0 + 0.5 * i for i in range(13)]
        assert res[r]["same_start"]
    # the same work per rank, different seeded structures
    assert res[0]["n"] == res[1]["n"]
    assert not np.array_equal(res[0]["xyz0"], res[1]["xyz0"])
    assert res[1]["ref_ret"] is None and res[1]["ref_out"] == ""


def test_single_process_reduction_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, "cpu") == 3.5
    assert bench.job_rate(10, 1, 2.0) == 5.0
