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


def test_parity_check_selects_only_fully_sampled_sources():
    """The bench's per-run parity check: rows of A sources whose r-disc lies
    inside the oracle's RA band are compared.  With the full-sky oracle
    standing in for the library's rows, the band comparison must be equal
    (no selected source has a partner outside the band, also near the poles
    and the band's edges) and a single dropped or altered row must show."""
    sys.path.insert(0, ROOT)
    import numpy as np
    import torch

    import bench
    import oracle as O
    from paper_2301_07331_b300 import synth
    A, B = synth.fullsky_pair(seed=5, na=30000, nb=30000, device="cpu")
    # crowd the band's edges and the poles with close pairs
    ra_a, dec_a = A.ra.numpy().copy(), A.dec.numpy().copy()
    ra_a[:400] = np.linspace(-0.001, 0.001, 400) % 360.0
    ra_a[400:800] = 30.0 + np.linspace(-0.001, 0.001, 400)
    dec_a[800:1200] = np.linspace(89.95, 89.9999, 400)
    A = synth.Catalogue(torch.from_numpy(ra_a), torch.from_numpy(dec_a), A.id)
    ra_b, dec_b = B.ra.numpy().copy(), B.dec.numpy().copy()
    ra_b[:1200] = (ra_a[:1200] + 0.3 / 3600) % 360.0
    dec_b[:1200] = dec_a[:1200]
    B = synth.Catalogue(torch.from_numpy(ra_b), torch.from_numpy(dec_b), B.id)
    r, L = 50.0, 9
    full = O.match(*A.numpy(), *B.numpy(), r, L, O.COMPLETE)
    rows = (full["id_a"], full["id_b"], full["sep"])
    _, band = bench.cpu_baseline(A, B, r, L, False, 0.0, 30.0)
    rec = bench.oracle_parity(A, r, band, rows, 0.0, 30.0)
    assert rec["equal"] and rec["rows"] > 0 and rec["max_sep_err_arcsec"] == 0.0
    # one selected row dropped from the library's side
    sel = np.isin(rows[0], band["id_a"])
    k = int(np.flatnonzero(sel)[0])
    dropped = tuple(np.delete(x, k) for x in rows)
    assert not bench.oracle_parity(A, r, band, dropped, 0.0, 30.0)["equal"]
    # a separation off by more than the tolerance
    bad = (rows[0], rows[1], rows[2].copy())
    bad[2][k] += 2e-6
    rec = bench.oracle_parity(A, r, band, bad, 0.0, 30.0)
    assert rec["equal"] and not rec["sep_within_tolerance"]
    assert bench.rows_equal(rows, rows)["equal"]
    assert not bench.rows_equal(rows, dropped)["equal"]


def test_critical_path_adds_up_to_the_step():
    sys.path.insert(0, ROOT)
    import bench
    st = {"ms_plan_span": 1.5, "ms_plan_presort": 0.4, "ms_sort_passes": 0.45,
          "ms_candidates": 0.0, "ms_pair": 0.5, "ms_recheck": 0.05, "ms_output": 0.5}
    cp = bench.critical_path([st, st], 2.8)
    assert abs(sum(cp.values()) - 2.8) < 1e-9
    assert abs(cp["plan_payloads_table_dense_cells"] - 0.65) < 1e-9
    cp = bench.critical_path([dict(st, ms_plan_presort=0.0)], 2.8)
    assert "plan" in cp and abs(sum(cp.values()) - 2.8) < 1e-9
