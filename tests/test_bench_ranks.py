"""The bench's multi-rank bookkeeping on CPU: two ranks joined over gloo
(127.0.0.1) read their rank from the environment, take the slowest rank's
step time as the job's, and report the units of both ranks over it."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import json, os, sys
sys.path.insert(0, sys.argv[1])
import torch.distributed as dist
import bench
world, rank, local = bench._dist()
dist.init_process_group("gloo", rank=rank, world_size=world)
ms = bench.max_over_ranks(1.0 + 2.0 * rank, "cpu")
print(json.dumps({"world": world, "rank": rank, "local": local, "ms": ms,
                  "value": bench.job_value(1000, world, ms)}))
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_ranks_take_the_slowest_step():
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                   LOCAL_RANK=str(rank), WORLD_SIZE="2")
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER, ROOT], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    assert sorted(o["rank"] for o in outs) == [0, 1]
    for o in outs:
        assert o["world"] == 2 and o["local"] == o["rank"]
        assert o["ms"] == 3.0                       # the slower rank's 3 ms
        assert abs(o["value"] - 2 * 1000 / 3e-3) < 1e-6


def test_captured_traffic_is_tied_to_workload_and_sources(monkeypatch):
    """A DRAM-traffic figure is reported only for the workload it was captured
    on and only while the digest of its kernel sources still matches."""
    sys.path.insert(0, ROOT)
    import bench
    for name, tr in list(bench.TRAFFIC.items()):
        current = dict(tr, sources=bench._sources_sha(tr["files"]))
        monkeypatch.setitem(bench.TRAFFIC, name, current)
        assert bench._traffic(name, bench.TRAFFIC_WORKLOAD) == tr["bytes_per_launch"], name
        other = ("clusters",) + tuple(bench.TRAFFIC_WORKLOAD[1:])
        assert bench._traffic(name, other) is None
        monkeypatch.setitem(bench.TRAFFIC, name, dict(tr, sources="0" * 16))
        assert bench._traffic(name, bench.TRAFFIC_WORKLOAD) is None
    assert bench._traffic("no_such_kernel", bench.TRAFFIC_WORKLOAD) is None


def test_clock_record_rejects_slowdowns_and_unexplained_low_clocks(tmp_path):
    """The bench's clock check: slowdown reasons or an SM clock stuck well
    below its maximum with no reason reject a timed window; a power cap
    alone does not.  The nvidia-smi CSV is parsed within the window only."""
    sys.path.insert(0, ROOT)
    import bench
    ok = {"sm_mhz": 2032.0, "sm_max_mhz": 2032.0, "reasons": []}
    assert bench.clocks_rejected(ok) == ""
    assert bench.clocks_rejected(dict(ok, reasons=["sw_power_cap"])) == ""
    assert bench.clocks_rejected(dict(ok, sm_mhz=1500.0, reasons=["sw_power_cap"])) == ""
    assert "hw_slowdown" in bench.clocks_rejected(dict(ok, reasons=["hw_slowdown"]))
    assert "sw_thermal_slowdown" in bench.clocks_rejected(
        dict(ok, reasons=["sw_power_cap", "sw_thermal_slowdown"]))
    assert "no reason" in bench.clocks_rejected(dict(ok, sm_mhz=1200.0))
    assert bench.clocks_rejected({"sm_mhz": None, "sm_max_mhz": None,
                                  "reasons": ["nvidia-smi unavailable"]}) == ""

    class _Done:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    path = tmp_path / "clocks.csv"
    c = bench.Clocks(0, str(path))
    c.f = open(path, "w")
    rows = [  # before, inside (two samples), after the window
        ("2026/01/01 00:00:00.000", 1000, "Not Active", "Not Active"),
        ("2026/01/01 00:00:10.100", 2032, "Not Active", "Active"),
        ("2026/01/01 00:00:10.300", 2010, "Not Active", "Not Active"),
        ("2026/01/01 00:00:20.000", 900, "Active", "Not Active"),
    ]
    for ts, mhz, hw, cap in rows:
        c.f.write(f"{ts}, 0, {mhz}, 2032, 700.0, 0x0, {hw}, Not Active, Not Active, {cap}\n")
    c.f.flush()
    c.proc = _Done()
    import time as _t
    c.t0 = _t.mktime(_t.strptime("2026/01/01 00:00:10", "%Y/%m/%d %H:%M:%S"))
    c.t1 = c.t0 + 0.5
    rec = c.stop()
    assert rec["samples"] == 2 and rec["sm_max_mhz"] == 2032.0
    assert rec["sm_mhz"] == 2021.0 and rec["reasons"] == ["sw_power_cap"]
    assert bench.clocks_rejected(rec) == ""
