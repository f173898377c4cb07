"""bench.py's clock sampler on CPU, against a stand-in nvidia-smi that prints
one CSV row per GPU every period: rows are kept per GPU index, summarised over
the timed region only, and throttle reasons are picked up."""
import os
import stat
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

FAKE = """#!{py}
import sys, time
period = int(sys.argv[sys.argv.index("-lms") + 1]) / 1000.0
k = 0
while True:
    # GPU 0 at full clock, no reason; GPU 1 slowed with hw_slowdown active
    mhz = 2070 if k % 2 == 0 else 2040
    print(f"0, {{mhz}}, 2070, 900.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active", flush=True)
    print("1, 1200, 2070, 300.0, 0x0000000000000008, Active, Not Active, Not Active, Not Active", flush=True)
    k += 1
    time.sleep(period)
"""


def _fake_smi(tmp_path):
    p = tmp_path / "nvidia-smi"
    p.write_text(FAKE.format(py=sys.executable))
    p.chmod(p.stat().st_mode | stat.S_IXUSR)
    return str(p)


def test_samples_inside_the_region(tmp_path):
    cs = bench.ClockSampler(period_ms=20, smi=_fake_smi(tmp_path))
    cs.start()
    assert cs.rows, "start() returns once the first sample has arrived"
    time.sleep(0.2)
    t0 = time.perf_counter()
    time.sleep(0.3)
    t1 = time.perf_counter()
    time.sleep(0.1)
    c0 = cs.stop(0, t0, t1)
    assert c0["samples_in_region"] >= 5 and c0["samples"] == c0["samples_in_region"]
    n_all = sum(1 for _, r in cs.rows if r[0] == "0")
    assert c0["samples"] < n_all  # rows before and after the region are left out
    assert c0["sm_mhz"] in (2040.0, 2055.0, 2070.0) and c0["sm_max_mhz"] == 2070.0
    assert c0["reasons"] == [] and c0["period_ms"] == 20
    c1 = cs.stop(1, t0, t1)
    assert c1["reasons"] == ["hw_slowdown"] and c1["sm_mhz"] == 1200.0


def test_region_shorter_than_the_period(tmp_path):
    cs = bench.ClockSampler(period_ms=200, smi=_fake_smi(tmp_path))
    cs.start()
    time.sleep(0.05)
    t0 = time.perf_counter()
    t1 = t0 + 0.001
    time.sleep(0.5)
    c = cs.stop(0, t0, t1)
    assert c["samples_in_region"] == 0 and c["samples"] == 1
    assert c["sm_max_mhz"] == 2070.0


def test_missing_tool_gives_no_clocks():
    cs = bench.ClockSampler(smi="/nonexistent/nvidia-smi")
    cs.start()
    assert cs.stop(0, 0.0, 1.0) is None
