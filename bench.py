"""Throughput of the cross-match hot path on one B300 (or N, one process each).

Workload (default): full sky, A = 10M and B = 10M float64 positions, 40%
uniform + 60% galactic disk exp(-|b|/10 deg), B = 60% jittered (0.5") copies
+ 40% fresh, r = 1.5", HEALPix fine order 12, coarse order 4, complete
8-neighbour mode; seeded synthetic data generated on the device.  A step is
one hlc_plan + hlc_match + hlc_free (prep/ang2pix, cell sort, cell table,
candidates, pair test, recheck, output rows sorted by (id_a, id_b)).

Metric: sources matched per second, (N_A + N_B) / step time, for the chosen
form (FP32 guard band) with the plain FP64 form timed beside it, plus pair
tests per second.  Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "sources matched/s and pair tests/s on 1 B300, chosen vs plain form, exact set"
MEASURED = os.path.join(ROOT, "MEASURED_PEAKS.json")


def _peaks():
    try:
        with open(MEASURED) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(ms: float, device) -> float:
    """The job's step time: the largest per-step time over the ranks (each
    rank runs its own independent instance; this is the only exchange)."""
    import torch
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size() == 1:
        return ms
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank: int, world: int, ms: float) -> float:
    """Whole-job throughput: the units all ranks processed over the job's
    step time (ms)."""
    return units_per_rank * world / (ms / 1e3)


class Clocks:
    """nvidia-smi sampling during the timed region."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, path: str = ""):
        self.idx = gpu_index
        self.proc = None
        self.path = path or os.path.join(tempfile.gettempdir(), "hlc_bench_clocks.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        # sampling live before the timed region starts (the first sample can
        # take most of a second); a short region then falls between samples
        # that stop() keeps by the margin around it
        t_end = time.time() + 5.0
        while time.time() < t_end and self.proc.poll() is None:
            self.f.flush()
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.02)

    def mark(self, which: str):
        setattr(self, which, time.time())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        t1 = getattr(self, "t1", None)
        if t1 is not None:  # a sample after the region's end, within the margin
            time.sleep(max(0.0, min(0.25, t1 + 0.12 - time.time())))
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        t0 = getattr(self, "t0", None)
        t1 = getattr(self, "t1", None)
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 10:
                continue
            try:
                ts = time.mktime(time.strptime(p[0].split(".")[0], "%Y/%m/%d %H:%M:%S"))
                ts += float("0." + p[0].split(".")[1]) if "." in p[0] else 0.0
                if t0 is not None and t1 is not None and not (t0 - 0.15 <= ts <= t1 + 0.15):
                    continue
                sm.append(float(p[2]))
                smax.append(float(p[3]))
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, p[6:10]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


REJECTING_REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown")


def clocks_rejected(clk: dict, floor: float = 0.85) -> str:
    """Why the clock record of a timed window rejects its number ('' when it
    stands): a hardware or thermal slowdown was active, or the median SM
    clock sat below `floor` x its maximum with no reason given (a clock
    lock left behind by another user).  A power cap alone is kept."""
    reasons = clk.get("reasons") or []
    bad = [r for r in reasons if r in REJECTING_REASONS]
    if bad:
        return ", ".join(bad)
    sm, smax = clk.get("sm_mhz"), clk.get("sm_max_mhz")
    if sm and smax and sm < floor * smax and "sw_power_cap" not in reasons:
        return "SM clock %.0f of %.0f MHz with no reason" % (sm, smax)
    return ""


def run_hlc(args):
    import torch
    import torch.distributed as dist

    import paper_2301_07331_b300 as hlc
    from paper_2301_07331_b300 import synth

    world, rank, local = _dist()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())
    A, B, r, L, Lc, wname = make_workload(args, rank, dev)
    # (captured DRAM traffic applies to the workload it was taken on)
    wkey = (args.workload, int(A.ra.numel()) if A.ra.numel() == B.ra.numel() else -1, args.mode)
    na, nb = A.ra.numel(), B.ra.numel()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    prec = hlc.HLC_FP32_GUARD if args.precision == "fp32" else hlc.HLC_FP64
    mode = hlc.HLC_QUAD if args.mode == "quad" else hlc.HLC_COMPLETE8

    def step(precision, A_, B_):
        plan = hlc.hlc_plan(A_, B_, r, L, coarse_level=Lc, boundary=mode, precision=precision,
                            stream=stream)
        res = hlc.hlc_match(plan, copy=False)
        st = res["stats"]
        n = res["n"]
        hlc.hlc_free(plan)
        return st, n

    def step_mode(precision, mode_):
        plan = hlc.hlc_plan(A, B, r, L, coarse_level=Lc, boundary=mode_, precision=precision,
                            stream=stream)
        res = hlc.hlc_match(plan, copy=False)
        st, n = res["stats"], res["n"]
        hlc.hlc_free(plan)
        return st, n

    def timed_mode(fn, precision, mode_, K, W):
        for _ in range(W):
            fn(precision, mode_)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        sts = []
        e0.record(stream)
        for _ in range(K):
            st, n = fn(precision, mode_)
            sts.append(st)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_ = e0.elapsed_time(e1) / K
        if world > 1:
            ms_ = max_over_ranks(ms_, dev)
        return ms_, sts, n

    def timed(precision, K, W, clk=None):
        for _ in range(W):
            step(precision, A, B)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        stats = []
        if clk is not None:
            clk.mark("t0")
        e0.record(stream)
        for _ in range(K):
            st, n = step(precision, A, B)
            stats.append(st)
        e1.record(stream)
        torch.cuda.synchronize()
        if clk is not None:
            clk.mark("t1")
        if world > 1:
            dist.barrier()
        ms = e0.elapsed_time(e1) / K
        if world > 1:
            ms = max_over_ranks(ms, dev)
        return ms, stats, n

    clocks = Clocks(local, args.clocks_out)
    clocks.start()
    ms, stats, nmatch = timed(prec, args.steps, args.warmup, clocks)
    clk = clocks.stop()
    # a window the clock record rejects is measured once more (every rank
    # takes the same decision, so that the barriers inside stay matched)
    why = clocks_rejected(clk)
    if max_over_ranks(1.0 if why else 0.0, dev) > 0.0:
        clocks.start()
        ms, stats, nmatch = timed(prec, args.steps, args.warmup, clocks)
        clk = clocks.stop()
        clk["remeasured_after"] = why or "another rank's clock record"
        # the second window is checked too: a throttled number is never
        # reported unflagged
        clk["still_rejected"] = clocks_rejected(clk)
    other = hlc.HLC_FP64 if prec == hlc.HLC_FP32_GUARD else hlc.HLC_FP32_GUARD
    ms_other, stats_other, _ = timed(other, max(2, args.steps // 2), 1)

    def rows_of(precision, mode_):
        """One untimed plan + match; the sorted rows on the host."""
        plan = hlc.hlc_plan(A, B, r, L, coarse_level=Lc, boundary=mode_, precision=precision,
                            stream=stream)
        res = hlc.hlc_match(plan, copy=False)
        out = (res["id_a"].cpu().numpy().view("u8"), res["id_b"].cpu().numpy().view("u8"),
               res["sep"].cpu().numpy())
        hlc.hlc_free(plan)
        return out

    # this run's rows in both forms: the plain form must return the same set
    rows = rows_of(prec, mode)
    rows_other = rows_of(other, mode)
    plain_equal = rows_equal(rows, rows_other)

    def mean(key, S):
        return sum(s[key] for s in S) / len(S)

    sources = (na + nb) * world
    value = job_value(na + nb, world, ms)
    tests = stats[-1]["pair_tests"]

    # roofline of the dominant kernel: the radix sort's digit passes
    # (k_onesweep, the largest share of the step), timed live by the library's
    # CUDA events on the launching stream; the pair test beside it
    peak, peak_kind = _peaks()
    stage_ms = {k: mean(k, stats) for k in ("ms_prep", "ms_sort", "ms_index", "ms_candidates",
                                            "ms_pair", "ms_recheck", "ms_output")}
    last = stats[-1]
    mA, mB = last["entries_a"], last["entries_b"]
    peak_src = ((peak_kind + " (MEASURED_PEAKS.json hbm_gbs)") if peak_kind == "measured"
                else "fallback 6.4 TB/s")
    quad = args.mode == "quad"
    roofline = None
    npass = last["sort_passes"]
    ms_passes = mean("ms_sort_passes", stats)
    if npass and ms_passes > 0:
        # each pass reads and writes a 4-byte key and a 4-byte value per entry,
        # the one-sort form's first makes its values (the library's sort_bytes;
        # a launch may cover both catalogues)
        per_pass = last["sort_bytes"] / npass
        gbs = per_pass * npass / (ms_passes / 1e3) / 1e9
        tr = _traffic("k_onesweep", wkey)
        roofline = {"kernel": "k_onesweep (cell-key radix sort digit pass)", "bound": "hbm",
                    "achieved": round(gbs, 1), "peak": peak, "unit": "GB/s",
                    "frac": round(gbs / peak, 4), "traffic": tr, "peak_source": peak_src,
                    "bytes_per_launch": int(per_pass),
                    "bytes_basis": "16 B per entry per pass (key and value read and "
                                   "written), 12 B in a first pass that makes its values "
                                   "from the positions; per launch: the mean over the passes",
                    "launches_per_step": npass, "ms_per_launch": ms_passes / npass,
                    "timing": "CUDA events around the digit passes; with device inputs "
                              "one launch per pass sorts both catalogues"}
    lt = 0
    while lt < L and 12 * 4 ** lt < mB:
        lt += 1
    # complete (table-cell) form: key + vector + source index per A entry, a B
    # vector per B entry, the offset table, a row and its B source index per
    # emitted row; quad form: key + vector per A entry, no index translation
    pair_bytes = (mA * (20 if quad else 24) + mB * 16 + (12 * 4 ** lt + 1) * 4
                  + (8 if quad else 12) * (last["matches"] + last["band_candidates"]))
    pair_gbs = pair_bytes / (stage_ms["ms_pair"] / 1e3) / 1e9
    kname = "k_pair<1,1,0,0>" if quad else "k_pair<1,0,0,1>"
    roofline_pair = {"kernel": kname + (" (FP32 quad form" if quad else " (FP32 complete form")
                     + ": candidates + pair test)",
                     "bound": "hbm", "achieved": round(pair_gbs, 1), "peak": peak,
                     "unit": "GB/s", "frac": round(pair_gbs / peak, 4),
                     "traffic": _traffic(kname, wkey) if prec == hlc.HLC_FP32_GUARD else None,
                     "peak_source": peak_src, "bytes_per_launch": int(pair_bytes),
                     "bytes_basis": ("20" if quad else "24") + " B per A entry (key + FP32 vector"
                                    + ("" if quad else " + source index") + "), 16 B per B entry, "
                                    "4 B per offset-table slot, " + ("8" if quad else "12")
                                    + " B per emitted row",
                     "ms_per_launch": stage_ms["ms_pair"]}
    if roofline is None:
        roofline = roofline_pair
    alg = alg_pair_tests(hlc, A, B, L) if args.mode == "complete" else None

    # end to end: pinned host inputs in, sorted rows back to host
    e2e = None
    if not args.no_e2e:
        Ah = synth.Catalogue(A.ra.cpu().pin_memory(), A.dec.cpu().pin_memory(),
                             A.id.cpu().pin_memory())
        Bh = synth.Catalogue(B.ra.cpu().pin_memory(), B.dec.cpu().pin_memory(),
                             B.id.cpu().pin_memory())
        times = []
        ke = min(args.steps, 30)
        cap = 2 * max(nmatch, 1)  # pinned result buffers, allocated once
        depth = max(1, min(args.e2e_depth, ke))  # (every worker runs at least one step)
        outs = [tuple(torch.empty(cap, dtype=dt).pin_memory()
                      for dt in (torch.int64, torch.int64, torch.float64)) for _ in range(depth)]

        def e2e_step(s, outb):
            plan = hlc.hlc_plan(Ah, Bh, r, L, coarse_level=Lc, boundary=mode, precision=prec,
                                stream=s)
            hlc.hlc_match(plan, copy=False)
            # (copies on the plan's stream; hlc_free synchronises it)
            ia_, ib_, sp_ = hlc.hlc_result_to_host(plan, out=outb, wait=False)
            hlc.hlc_free(plan)
            return ia_, ib_, sp_

        # (a) one step at a time: the latency of a step
        ks = min(ke, 10)
        for it in range(args.warmup + ks):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ia, ib, sp = e2e_step(stream, outs[0])
            t1 = time.perf_counter()
            if it >= args.warmup:
                times.append(t1 - t0)
        t_serial = sum(times) / len(times)
        # (b) the throughput: `depth` steps in flight, one per host thread and
        # stream (the library's calls release the interpreter lock), started a
        # fraction of a step apart, so that the link carries one step's copies
        # while the others build, match and order; each step still copies its
        # inputs in and its rows out
        import threading
        streams = [torch.cuda.Stream() for _ in range(depth)]
        counts = [ke // depth + (1 if w < ke % depth else 0) for w in range(depth)]
        errs, rows_out = [], [0] * depth
        go = threading.Barrier(depth + 1)

        def worker(w):
            try:
                e2e_step(streams[w], outs[w])  # (warm the stream)
                go.wait()
                time.sleep(w * t_serial / depth)  # (staggered: not all copying at once)
                for _ in range(counts[w]):
                    ia_, _, _ = e2e_step(streams[w], outs[w])
                    rows_out[w] = int(ia_.size)
            except Exception as e:  # noqa: BLE001 (re-raised below)
                errs.append(e)
                go.abort()
        ths = [threading.Thread(target=worker, args=(w,)) for w in range(depth)]
        for th in ths:
            th.start()
        torch.cuda.synchronize()
        try:
            go.wait()
        except threading.BrokenBarrierError:
            pass  # (a worker failed; raised below)
        t0 = time.perf_counter()
        for th in ths:
            th.join()
        torch.cuda.synchronize()
        t = (time.perf_counter() - t0) / ke
        if errs:
            raise errs[0]
        assert all(n_ == int(ia.size) for n_ in rows_out)
        e2e = {"value": sources / t, "unit": "sources/s", "ms_per_step": t * 1e3, "steps": ke,
               "h2d_bytes_per_step": (na + nb) * 24, "d2h_bytes_per_step": int(ia.size) * 24,
               "in_flight": depth, "serial_ms_per_step": t_serial * 1e3,
               "timing": "host wall clock over %d steps, %d at a time (one host thread and "
                         "stream each, started 1/%d step apart): pinned host catalogues in "
                         "through hlc_plan, rows copied to pinned host buffers by "
                         "hlc_result_to_host" % (ke, depth, depth)}

    # CPU oracle on a bounded sample of the same workload (rank 0 only), and
    # this run's rows against it
    cpu = parity = None
    if rank == 0 and not args.no_cpu and args.workload == "fullsky":
        cpu, ores = cpu_baseline(A, B, r, L, mode == hlc.HLC_QUAD)
        parity = oracle_parity(A, r, ores, rows, 0.0, 180.0)

    # the other boundary mode of the same workload (BASELINE config 2 names
    # both), timed and checked the same way on a narrower oracle sample
    other_mode = None
    if args.workload == "fullsky" and not args.no_other_mode:
        omode = hlc.HLC_COMPLETE8 if mode == hlc.HLC_QUAD else hlc.HLC_QUAD
        ko = max(3, args.steps // 4)
        ms_q, st_q, n_q = timed_mode(step_mode, prec, omode, ko, 2)
        ms_q64, _, _ = timed_mode(step_mode, other, omode, max(2, ko // 2), 1)
        rq, rq64 = rows_of(prec, omode), rows_of(other, omode)
        oq = None
        if rank == 0 and not args.no_cpu:
            _, oresq = cpu_baseline(A, B, r, L, omode == hlc.HLC_QUAD, 0.0, 30.0)
            oq = oracle_parity(A, r, oresq, rq, 0.0, 30.0)
        other_mode = {"boundary": "quad" if omode == hlc.HLC_QUAD else "complete",
                      "ms_per_step": ms_q, "value": sources / (ms_q / 1e3), "unit": "sources/s",
                      "steps": ko, "matches": n_q,
                      "quad_duplicates": st_q[-1]["quad_duplicates"],
                      "plain_form": {"ms_per_step": ms_q64, "value": sources / (ms_q64 / 1e3),
                                     **rows_equal(rq, rq64)},
                      "parity": oq}

    # per-source error radii (Eq. 4) on the same catalogues
    eq4 = None
    if args.workload == "fullsky" and not args.no_eq4 and mode == hlc.HLC_COMPLETE8:
        eq4 = eq4_line(args, hlc, synth, A, B, L, Lc, stream, rank, world, prec, other)

    # dense cells: the pair test where it is bound by the FP32 pipe
    dense = None
    if args.workload == "fullsky" and not args.no_dense:
        dense = dense_line(args, hlc, synth, dev, stream, rank, world)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "sources/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if prec == hlc.HLC_FP32_GUARD else "f64",
            "data": "synthetic (seeded, generated on device)",
            "config": {"workload": wname + ", " + args.mode + " mode",
                       "n_a": na, "n_b": nb, "radius_arcsec": r, "fine_level": L,
                       "coarse_level": Lc, "boundary": args.mode,
                       "form": args.precision + " (chosen)",
                       "l2": "inputs (%d MB) larger than L2 (126 MB)" % ((na + nb) * 24 // 10**6),
                       "parallelism": "independent instance per GPU" if world > 1 else "1 GPU"},
            "pair_tests_per_s": (alg / (stage_ms["ms_pair"] / 1e3)) if alg else None,
            "pair_tests_alg": alg, "pair_tests_executed": tests, "matches": nmatch,
            "band_candidates": stats[-1]["band_candidates"],
            "band_fp64": stats[-1]["band_fp64"],
            "dense_entries_b": stats[-1]["dense_entries_b"],
            "tile_items": stats[-1]["tile_items"], "tile_entries_a": stats[-1]["tile_entries_a"],
            "plain_form": {"precision": "fp64" if other == hlc.HLC_FP64 else "fp32",
                           "ms_per_step": ms_other, "value": sources / (ms_other / 1e3),
                           "stages_ms": {k: mean(k, stats_other) for k in stage_ms},
                           "equal_to_chosen": plain_equal["equal"],
                           "rows": plain_equal["rows"],
                           "max_sep_diff_arcsec": plain_equal["max_sep_diff_arcsec"]},
            "parity": parity,
            "critical_path_ms": critical_path(stats, ms),
            "stages_ms": stage_ms,
            "stages_note": "busy time per stage summed over both catalogues; stages of the "
                           "two catalogues overlap on two streams, so they do not add up to "
                           "ms_per_step (critical_path_ms does)",
            "roofline": roofline,
            "roofline_pair": roofline_pair,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(sum(s["kernel_launches"] for s in stats)),
            "clocks": clk,
        }
        if other_mode is not None:
            line["other_mode"] = other_mode
        if dense is not None:
            line["dense"] = dense
        if eq4 is not None:
            line["eq4"] = eq4
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


# DRAM bytes (read + write) per launch of a kernel from one ncu capture, with
# the digest of the kernel sources it was taken on; a changed source voids it.
TRAFFIC = {
    # captured on the default line's workload (full sky 10M x 10M, complete
    # mode, FP32 form) with ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum:
    # the three sort passes of a step (both catalogues per launch), read +
    # written: 80,645,376 + 121,016,576 (the first pass makes its values),
    # 160,946,432 + 120,703,488 and 160,590,336 + 119,894,016 B; their mean
    "k_onesweep": {"bytes_per_launch": 254598741, "sources": "baeb5a5edf527796",
                   "files": ("sort.cuh", "common.cuh")},
    # the pair test: 495,089,920 B read + 42,796,800 B written
    "k_pair<1,0,0,1>": {"bytes_per_launch": 537886720, "sources": "0f5305cd4a23c775",
                        "files": ("match.cuh", "canon.cuh", "index.cuh", "learned.cuh",
                                  "common.cuh", "fp32.cuh", "fastpix.cuh")},
}
TRAFFIC_WORKLOAD = ("fullsky", 10_000_000, "complete")


def _sources_sha(files) -> str:
    import hashlib
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2301_07331_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _traffic(name, workload):
    """Captured DRAM bytes per launch of `name`, or None when the bench runs
    another workload or the kernel's sources changed since the capture."""
    tr = TRAFFIC.get(name)
    if not tr or workload != TRAFFIC_WORKLOAD:
        return None
    return tr["bytes_per_launch"] if tr["sources"] == _sources_sha(tr["files"]) else None


def alg_pair_tests(hlc, A, B, L):
    """Algorithmic pair tests of complete mode: sum over A cells c of
    n_A(c) * sum of n_B over c and its neighbours (padded or superset tests
    not counted).  Computed outside the timed region."""
    import torch
    pa = hlc.hlc_ang2pix(A.ra, A.dec, L).to(torch.int64) & 0xFFFFFFFF
    pb = hlc.hlc_ang2pix(B.ra, B.dec, L).to(torch.int64) & 0xFFFFFFFF
    ua, ca = torch.unique(pa, return_counts=True)
    ub, cb = torch.unique(pb, return_counts=True)
    nb = hlc.hlc_neighbours(ua.to(torch.int32), L)
    cells = torch.cat([ua[:, None], nb], 1)
    idx = torch.searchsorted(ub, cells.clamp(min=0)).clamp(max=max(ub.numel() - 1, 0))
    present = (cells >= 0) & (ub[idx] == cells)
    nsum = torch.where(present, cb[idx], torch.zeros_like(cb[idx])).sum(1)
    return int((ca * nsum).sum())


def make_workload(args, rank, dev):
    """The synthetic catalogues of a workload, generated on the device."""
    from paper_2301_07331_b300 import synth
    w = args.workload
    if w == "fullsky":
        n = args.n or 10_000_000
        A, B = synth.fullsky_pair(seed=2301073311 + rank, na=n, nb=n, device=dev)
        name = "fullsky %s x %s (40%% uniform + 60%% galactic disk), r=1.5 arcsec, fine order 12" % (
            _mega(n), _mega(n))
        return A, B, 1.5, 12, 4, name
    if w == "clusters":
        n = args.n or 50_000_000
        ncl = max(1, n // 2_000_000)
        A, B = synth.clustered_pair(seed=2301073312 + rank, na=n, nb=n * 3 // 4,
                                    n_clusters=ncl, device=dev)
        name = ("clusters %s x %s (galactic mixture + %d Plummer clusters, a=2 arcmin, "
                "50k members), r=1 arcsec, fine order 13" % (_mega(n), _mega(n * 3 // 4), ncl))
        return A, B, 1.0, 13, 3, name
    if w == "bulge":
        n = args.n or 100_000_000
        A, B = synth.bulge_pair(seed=2301073314 + rank, na=n, nb=n, device=dev)
        name = ("bulge %s x %s (0.825%% uniform + 67.8%% disk + 31.4%% Gaussian bulge "
                "sigma 5 deg), r=1 arcsec, fine order 14" % (_mega(n), _mega(n)))
        return A, B, 1.0, 14, 4, name
    raise SystemExit("unknown workload " + w)


def _mega(n):
    return "%gM" % (n / 1e6) if n >= 1_000_000 else str(n)


def cpu_baseline(A, B, r, L, quad=False, lo=0.0, hi=180.0):
    """The oracle, as it stands, on the sources of both catalogues with RA in
    [lo, hi) deg (by default half of the same synthetic sky), single-threaded.
    Returns the baseline record and the oracle's rows."""
    import numpy as np

    import oracle as O
    ra_a, dec_a, id_a = (x.cpu().numpy() for x in (A.ra, A.dec, A.id))
    ra_b, dec_b, id_b = (x.cpu().numpy() for x in (B.ra, B.dec, B.id))
    sa = (ra_a >= lo) & (ra_a < hi)
    sb = (ra_b >= lo) & (ra_b < hi)
    t0 = time.perf_counter()
    res = O.match(ra_a[sa], dec_a[sa], id_a[sa].view(np.uint64), ra_b[sb], dec_b[sb],
                  id_b[sb].view(np.uint64), r, L, O.QUAD if quad else O.COMPLETE)
    t = time.perf_counter() - t0
    n = int(sa.sum() + sb.sum())
    rec = {"value": n / t, "unit": "sources/s", "cores": 1, "kind": "oracle",
           "sample": "sources with RA in [%g,%g) of both catalogues (%d sources, %d matches, "
                     "%s mode)" % (lo, hi, n, res["id_a"].size, "quad" if quad else "complete"),
           "seconds": t}
    return rec, res


def rows_equal(x, y) -> dict:
    """Equality of two sorted row sets (id_a, id_b, sep) from two forms of the
    library, and the largest separation difference."""
    import numpy as np
    eq = (x[0].size == y[0].size and bool(np.array_equal(x[0], y[0]))
          and bool(np.array_equal(x[1], y[1])))
    d = float(np.max(np.abs(x[2] - y[2]))) if eq and x[2].size else (0.0 if eq else None)
    return {"equal": eq, "rows": int(x[0].size), "max_sep_diff_arcsec": d}


def oracle_parity(A, r, ores, rows, lo, hi) -> dict:
    """This run's rows against the oracle's on its RA band [lo, hi): the A
    sources whose whole r-disc lies inside the band (RA at least twice the
    disc's RA half-width r / cos(dec) from either edge, |dec| < 89.9) have
    every partner in the oracle's sample, so their rows must be equal bit for
    bit and their separations within 1e-6 arcsec."""
    import numpy as np
    ra, dec, ida = (x.cpu().numpy() for x in (A.ra, A.dec, A.id))
    ida = ida.view(np.uint64)
    cosd = np.cos(np.radians(dec))
    w = 2.0 * (r / 3600.0) / np.maximum(cosd, 1e-12) + 1e-6
    inside = (ra >= lo + w) & (ra < hi - w) & (np.abs(dec) < 89.9)
    keep = np.sort(ida[inside])
    g = np.isin(rows[0], keep)
    o = np.isin(ores["id_a"], keep)
    ga, gb, gs = rows[0][g], rows[1][g], rows[2][g]
    oa, ob, os_ = ores["id_a"][o], ores["id_b"][o], ores["sep"][o]
    eq = ga.size == oa.size and bool(np.array_equal(ga, oa)) and bool(np.array_equal(gb, ob))
    err = float(np.max(np.abs(gs - os_))) if eq and ga.size else (0.0 if eq else None)
    return {"equal": eq, "rows": int(ga.size), "oracle_rows": int(oa.size),
            "a_sources": int(inside.sum()), "max_sep_err_arcsec": err,
            "sep_tolerance_arcsec": 1e-6, "sep_within_tolerance": bool(eq and err <= 1e-6),
            "sample": "A sources with RA in [%g,%g) deg whose r-disc lies inside the band" % (lo, hi)}


def critical_path(stats, ms_step) -> dict:
    """Consecutive intervals on the plan stream that add up to the step: the
    plan (its sort passes and, in the two-stream build, the part before them),
    the match's stages, and the rest of the step (host gaps, hlc_free)."""
    n = len(stats)

    def mean(k):
        return sum(s[k] for s in stats) / n
    plan = mean("ms_plan_span")
    pre = mean("ms_plan_presort")
    passes = mean("ms_sort_passes") if pre > 0 else 0.0
    out = {}
    if pre > 0:
        out["plan_preps_and_histograms"] = pre
        out["plan_sort_passes"] = passes
        out["plan_payloads_table_dense_cells"] = plan - pre - passes
    else:
        out["plan"] = plan
    for k in ("ms_candidates", "ms_pair", "ms_recheck", "ms_output"):
        out["match_" + k[3:]] = mean(k)
    out["host_gaps_and_free"] = ms_step - sum(out.values())
    return out


def eq4_line(args, hlc, synth, A, B, L, Lc, stream, rank, world, prec, other):
    """The same catalogues with per-source error radii (Eq. 4): e log-uniform
    in [0.05, 0.5] arcsec per source, so pair radii 3 sqrt(e_a^2 + e_b^2)
    span 0.2-2.1 arcsec.  Timed in both forms; the chosen form's rows must
    equal the plain form's and, for a sample of A sources, the oracle's."""
    import numpy as np
    import torch
    dev = A.ra.device
    ea = synth.error_radii(2301073315 + rank, 1, A.ra.numel(), 0.05, 0.5, device=dev)
    eb = synth.error_radii(2301073315 + rank, 2, B.ra.numel(), 0.05, 0.5, device=dev)

    def step(precision):
        plan = hlc.hlc_plan(A, B, 0.0, L, coarse_level=Lc, precision=precision, stream=stream,
                            err_a=ea, err_b=eb)
        res = hlc.hlc_match(plan, copy=False)
        st = res["stats"]
        hlc.hlc_free(plan)
        return st
    K = max(3, args.steps // 4)
    ms, sts = _timed_loop(lambda: step(prec), K, 2, stream, collect=True)
    ms64, _ = _timed_loop(lambda: step(other), max(2, K // 2), 1, stream)

    def rows(precision):
        plan = hlc.hlc_plan(A, B, 0.0, L, coarse_level=Lc, precision=precision, stream=stream,
                            err_a=ea, err_b=eb)
        res = hlc.hlc_match(plan, copy=False)
        out = (res["id_a"].cpu().numpy().view("u8"), res["id_b"].cpu().numpy().view("u8"),
               res["sep"].cpu().numpy())
        hlc.hlc_free(plan)
        return out
    r32, r64 = rows(prec), rows(other)
    parity = None
    if rank == 0 and not args.no_cpu:
        import oracle as O
        rng = np.random.default_rng(17)
        ra_a, dec_a, id_a = (x.cpu().numpy() for x in (A.ra, A.dec, A.id))
        id_a = id_a.view(np.uint64)
        pick = np.sort(rng.choice(ra_a.size, 20000, replace=False))
        t0 = time.perf_counter()
        want = O.match_eq4(ra_a[pick], dec_a[pick], id_a[pick], ea.cpu().numpy()[pick],
                           B.ra.cpu().numpy(), B.dec.cpu().numpy(),
                           B.id.cpu().numpy().view(np.uint64), eb.cpu().numpy(), L)
        t = time.perf_counter() - t0
        sel = np.isin(r32[0], id_a[pick])
        ga, gb, gs = r32[0][sel], r32[1][sel], r32[2][sel]
        eq = ga.size == want["id_a"].size and bool(np.array_equal(ga, want["id_a"])) and \
            bool(np.array_equal(gb, want["id_b"]))
        err = float(np.max(np.abs(gs - want["sep"]))) if eq and ga.size else (0.0 if eq else None)
        parity = {"equal": eq, "rows": int(ga.size), "a_sources": int(pick.size),
                  "max_sep_err_arcsec": err, "sep_within_tolerance": bool(eq and err <= 1e-6),
                  "oracle_seconds": t,
                  "sample": "20000 random A sources against all of B (oracle per-pair radii)"}
    n = A.ra.numel() + B.ra.numel()
    last = sts[-1]
    return {"radii": "e log-uniform in [0.05, 0.5] arcsec per source; r_ij = 3 sqrt(e_i^2 + "
                     "e_j^2) in [0.21, 2.12] arcsec",
            "ms_per_step": ms, "value": n / (ms / 1e3), "unit": "sources/s", "steps": K,
            "matches": last["matches"], "band_candidates": last["band_candidates"],
            "band_fp64": last["band_fp64"],
            "plain_form": {"ms_per_step": ms64, "value": n / (ms64 / 1e3), **rows_equal(r32, r64)},
            "parity": parity}


def dense_line(args, hlc, synth, dev, stream, rank, world):
    """Dense cells, where the pair test is bound by the FP32 pipe: the
    clustered workload at a reduced size (galactic mixture + Plummer clusters
    of 50k members, a = 2 arcmin, r = 1 arcsec, fine order 13).  Pair tests/s
    = algorithmic tests / pair-stage time, against SMs x 128 x f / 6 (six
    FP32 FMA-pipe instructions per test) at the median SM clock sampled in
    the timed window."""
    import torch
    n = args.dense_n
    ncl = max(1, n // 2_000_000)
    A, B = synth.clustered_pair(seed=2301073312 + rank, na=n, nb=n * 3 // 4, n_clusters=ncl,
                                device=dev)
    r, L, Lc = 1.0, 13, 3

    def step():
        plan = hlc.hlc_plan(A, B, r, L, coarse_level=Lc, stream=stream)
        res = hlc.hlc_match(plan, copy=False)
        st_ = res["stats"]
        hlc.hlc_free(plan)
        return st_
    K = max(3, args.steps // 10)
    clocks = Clocks(torch.cuda.current_device(), args.clocks_out + ".dense" if args.clocks_out
                    else "")
    clocks.start()
    ms, sts = _timed_loop(lambda: step(), K, 2, stream, collect=True)
    clk = clocks.stop()
    alg = alg_pair_tests(hlc, A, B, L)
    ms_pair = sum(s["ms_pair"] for s in sts) / len(sts)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    f_mhz = clk.get("sm_mhz") or 2032.0
    peak = sms * 128 * f_mhz * 1e6 / 6
    tps = alg / (ms_pair / 1e3)
    last = sts[-1]
    ms_tile = sum(s["ms_tile"] for s in sts) / len(sts)
    tile_tps = last["tile_tests"] / (ms_tile / 1e3) if ms_tile > 0 else None
    return {"workload": "clusters %s x %s (%d Plummer clusters), r=1 arcsec, fine order 13"
                        % (_mega(n), _mega(n * 3 // 4), ncl),
            "ms_per_step": ms, "value": (n + n * 3 // 4) / (ms / 1e3), "unit": "sources/s",
            "steps": K, "pair_tests_alg": alg, "pair_tests_executed": last["pair_tests"],
            "ms_pair": ms_pair, "pair_tests_per_s": tps,
            "fp32_bound": {"peak_tests_per_s": peak, "frac": tps / peak, "sms": sms,
                           "sm_mhz": f_mhz,
                           "basis": "SMs x 128 FP32 lanes x SM clock / 6 FP32 operations per "
                                    "test (3 differences, 1 square, 2 fused multiply-adds)"},
            "tile_kernel": {"kernel": "k_pair_tile (dense cells, A and B staged in shared "
                                      "memory by bulk copies; local-frame test, one add and "
                                      "three FMAs per pair on packed f32x2)",
                            "ms": ms_tile, "tests": last["tile_tests"],
                            "tests_per_s": tile_tps,
                            "frac_of_fp32_bound": (tile_tps / peak) if tile_tps else None,
                            "frac_of_own_form_bound": (tile_tps / (peak * 6 / 4))
                            if tile_tps else None,
                            "own_form_basis": "SMs x 128 FP32 lanes x SM clock / 4 FMA-pipe "
                                              "operations per test of the local form"},
            "tile_items": last["tile_items"], "tile_entries_a": last["tile_entries_a"],
            "matches": last["matches"], "clocks": clk}


def _timed_loop(fn, K, W, stream, collect=False, clocks=None):
    """W untimed steps, then K steps between CUDA events on `stream`; with
    `clocks` (a started Clocks), its samples are kept for the timed steps."""
    import torch
    for _ in range(W):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if clocks is not None:
        clocks.mark("t0")
    e0.record(stream)
    out = None
    outs = []
    for _ in range(K):
        out = fn()
        if collect:
            outs.append(out)
    e1.record(stream)
    torch.cuda.synchronize()
    if clocks is not None:
        clocks.mark("t1")
    return e0.elapsed_time(e1) / K, (outs if collect else out)


def _sampled_loop(args, fn, K, W, stream, tag):
    """_timed_loop with nvidia-smi clocks sampled over its timed steps."""
    import torch
    clocks = Clocks(torch.cuda.current_device(),
                    args.clocks_out + "." + tag if args.clocks_out else "")
    clocks.start()
    ms, out = _timed_loop(fn, K, W, stream, clocks=clocks)
    return ms, out, clocks.stop()


def _line(args, metric, value, unit, ms, config, higher_is_better=True, **extra):
    d = {"metric": metric, "value": value, "unit": unit, "n_gpus": 1, "steps": args.steps,
         "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": higher_is_better,
         "scaling": "weak",
         "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic (seeded, generated on device)",
         "config": config}
    d.update(extra)
    print(json.dumps(d))


def run_learned(args):
    """Learned offset index against the plain per-partition binary search on
    the bulge workload's B cells (order 14, partitions at order 4): lookups of
    every A cell, build time, hit rate and stored error bound; then the match
    through each index."""
    import torch

    import paper_2301_07331_b300 as hlc
    from paper_2301_07331_b300 import synth
    dev = torch.device("cuda", 0)
    n = args.n or 500_000_000
    L, Lc, r = 14, 4, 1.0
    A, B = synth.bulge_pair(na=n, nb=n, device=dev)
    stream = torch.cuda.current_stream()
    kb = hlc.hlc_ang2pix(B.ra, B.dec, L)
    vb = torch.arange(kb.numel(), dtype=torch.int32, device=dev)
    hlc.hlc_sort_pairs(kb, vb, 32)
    uniq, _start = hlc.hlc_cell_table(kb)
    del vb, _start
    qa = hlc.hlc_ang2pix(A.ra, A.dec, L)
    va = torch.arange(qa.numel(), dtype=torch.int32, device=dev)
    hlc.hlc_sort_pairs(qa, va, 32)
    del va
    shift = 2 * (L - Lc)
    res = {}
    ref = None
    clocks = Clocks(torch.cuda.current_device(),
                    args.clocks_out + ".learned" if args.clocks_out else "")
    clocks.start()
    torch.cuda.synchronize()
    clocks.mark("t0")
    for name, model in (("binary search", hlc.HLC_MODEL_NONE), ("pla", hlc.HLC_MODEL_PLA),
                        ("mlp", hlc.HLC_MODEL_MLP)):
        outs = []
        for it in range(args.warmup + args.steps):
            out, st = hlc.hlc_learned_lookup(uniq, shift, model, qa, stream=stream)
            if it >= args.warmup:
                outs.append(st)
        if ref is None:
            ref = out
        exact = bool(torch.equal(out, ref))
        ms_look = sum(s["ms_candidates"] for s in outs) / len(outs)
        ms_build = sum(s["ms_index"] for s in outs) / len(outs)
        res[name] = {"lookups_per_s": qa.numel() / (ms_look / 1e3), "ms_lookup": ms_look,
                     "ms_build": ms_build, "hit_rate": outs[-1]["learned_hit_rate"],
                     "max_err": outs[-1]["learned_max_err"], "models": outs[-1]["learned_models"],
                     "equal_to_binary_search": exact}
        del out
    torch.cuda.synchronize()
    clocks.mark("t1")
    clk = clocks.stop()
    base = res["binary search"]["ms_lookup"]
    for k in ("pla", "mlp"):
        res[k]["speedup_vs_binary_search"] = base / res[k]["ms_lookup"]
    # the whole match through each index on a slice of the same catalogues
    nm = min(n, args.n_match)
    Am = synth.Catalogue(A.ra[:nm], A.dec[:nm], A.id[:nm])
    Bm = synth.Catalogue(B.ra[:nm], B.dec[:nm], B.id[:nm])
    del qa, kb
    match = {}
    for name, index, model in (("binary search", hlc.HLC_INDEX_BSEARCH, hlc.HLC_MODEL_PLA),
                               ("pla", hlc.HLC_INDEX_LEARNED, hlc.HLC_MODEL_PLA),
                               ("mlp", hlc.HLC_INDEX_LEARNED, hlc.HLC_MODEL_MLP)):
        def step():
            plan = hlc.hlc_plan(Am, Bm, r, L, coarse_level=Lc, index=index, model=model,
                                stream=stream)
            out = hlc.hlc_match(plan, copy=False)
            n_ = out["n"]
            st_ = out["stats"]
            hlc.hlc_free(plan)
            return n_, st_
        ms, (nmatch, st) = _timed_loop(step, max(1, args.steps), 1, stream)
        match[name] = {"sources_per_s": 2 * nm / (ms / 1e3), "ms_per_step": ms,
                       "matches": nmatch, "ms_pair": st["ms_pair"],
                       "hit_rate": st["learned_hit_rate"]}
    best = max(("pla", "mlp"), key=lambda k: res[k]["lookups_per_s"])
    _line(args, "learned-index lookups/s (exact lower bounds of A cells in B's cells)",
          res[best]["lookups_per_s"], "lookups/s", res[best]["ms_lookup"],
          {"workload": "bulge %s x %s, fine order 14, partitions at order 4 (%d models), "
                       "%d unique B cells, %d queries" % (_mega(n), _mega(n),
                                                         res["pla"]["models"], uniq.numel(),
                                                         n),
           "best_model": best}, clocks=clk, lookups=res,
          match_slice={"n_a": nm, "n_b": nm, **match})


def _auto_order(nb, cone_deg, r_arcsec):
    """The batched plan's density rule (about two B sources per cell,
    capped by r <= theta_L / 8), for the one-plan-per-job comparison."""
    area = 2 * math.pi * max(1 - math.cos(math.radians(cone_deg)), 1e-12)
    cells = 4 * math.pi * max(nb, 1) / area / (12 * 2.0)
    L = int(math.floor(math.log(cells) / math.log(4) + 0.5)) if cells > 1 else 0
    lmax = 0
    while lmax < 14 and r_arcsec <= math.sqrt(math.pi / 3) / 2 ** (lmax + 1) * 648000 / math.pi / 8:
        lmax += 1
    return max(0, min(L, lmax))


def run_batched(args):
    """4096 cone-pair jobs in one batched plan (one persistent graph-captured
    pair launch, orders chosen per job by density) against one plan per job."""
    import torch

    import paper_2301_07331_b300 as hlc
    from paper_2301_07331_b300 import synth
    dev = torch.device("cuda", 0)
    njobs = args.jobs
    jobs = synth.cone_jobs(n_jobs=njobs, scale=args.scale, device=dev)
    stream = torch.cuda.current_stream()
    spec = [{"A": j.A, "B": j.B, "radius_arcsec": j.r_arcsec} for j in jobs]
    total = sum(j.A.ra.numel() + j.B.ra.numel() for j in jobs)
    # the autotuner (form 2) on a sample of these jobs, outside the timed region
    # (--tune-sample 0: not run; the library's rule is timed twice)
    if args.tune_sample > 0:
        t0 = time.perf_counter()
        tune, report = hlc.hlc_autotune(spec, sample_jobs=args.tune_sample, stream=stream)
        report["seconds"] = time.perf_counter() - t0
    else:
        tune, report = None, {"skipped": "--tune-sample 0"}

    # the C structs of the job list, built once as a C caller would (the
    # tuned list and the rule's)
    prepared = {id(tune): hlc.BatchedJobs(spec, stream=stream, tune=tune),
                id(None): hlc.BatchedJobs(spec, stream=stream)}

    def batched(tn=None):
        plan = hlc.hlc_plan_batched(prepared[id(tn)], stream=stream)
        out = hlc.hlc_match(plan, copy=False)
        n_, st_ = out["n"], out["stats"]
        hlc.hlc_free(plan)
        return n_, st_
    ms_b, (nb_, st_b), clk = _sampled_loop(args, lambda: batched(tune), args.steps, args.warmup,
                                           stream, "batched")
    ms_r, (nr_, st_r) = _timed_loop(lambda: batched(None), args.steps, args.warmup, stream)
    orders = [_auto_order(j.B.ra.numel(), j.cone_deg, j.r_arcsec) for j in jobs]

    def per_job():
        n_ = 0
        for j, L in zip(jobs, orders):
            plan = hlc.hlc_plan(j.A, j.B, j.r_arcsec, L, coarse_level=min(4, L), stream=stream)
            n_ += hlc.hlc_match(plan, copy=False)["n"]
            hlc.hlc_free(plan)
        return n_
    ms_j, nj_ = _timed_loop(per_job, 1, 1, stream) if not args.no_per_job else (float("nan"), 0)
    _line(args, "sources matched/s, batched cone jobs", total / (ms_b / 1e3), "sources/s", ms_b,
          {"workload": "%d cone-pair jobs (cone 0.1-2 deg, N log-uniform %g-%g per side, "
                       "r 0.5-5 arcsec), %d sources" % (njobs, 1e3 * args.scale, 1e6 * args.scale,
                                                       total)},
          matches=nb_, clocks=clk, per_job={"ms": ms_j, "sources_per_s": total / (ms_j / 1e3), "matches": nj_},
          speedup_vs_per_job=ms_j / ms_b, pair_tests=st_b["pair_tests"],
          autotune=report, rule={"ms": ms_r, "sources_per_s": total / (ms_r / 1e3),
                                 "matches": nr_, "ms_pair": st_r["ms_pair"]},
          tuned_vs_rule=ms_r / ms_b,
          gpu_launches=st_b["kernel_launches"], tile_items=st_b["tile_items"],
          tile_entries_a=st_b["tile_entries_a"], band_candidates=st_b["band_candidates"],
          stages_ms={k: st_b[k] for k in ("ms_prep", "ms_sort", "ms_index", "ms_pair",
                                          "ms_recheck", "ms_output")})


def run_streamed(args):
    """Host-resident catalogues larger than the device budget, streamed by
    coarse partition through pinned buffers, against the same catalogues
    matched in core from device memory."""
    import torch

    import paper_2301_07331_b300 as hlc
    from paper_2301_07331_b300 import synth
    dev = torch.device("cuda", 0)
    n = args.n or 400_000_000
    nb = n * 3 // 4
    ncl = max(1, n // 2_000_000)
    A, B = synth.clustered_pair(na=n, nb=nb, n_clusters=ncl, device=dev)
    stream = torch.cuda.current_stream()
    r, L, Lc = 1.0, 13, 3
    Ah = synth.Catalogue(A.ra.cpu().pin_memory(), A.dec.cpu().pin_memory(), A.id.cpu().pin_memory())
    Bh = synth.Catalogue(B.ra.cpu().pin_memory(), B.dec.cpu().pin_memory(), B.id.cpu().pin_memory())
    budget = args.budget_gb << 30
    fit = hlc.hlc_transfer_model()  # Eq. 5 on this machine (the plans reuse it)

    def streamed():
        plan = hlc.hlc_plan(Ah, Bh, r, L, coarse_level=Lc, device_mem_budget=budget,
                            stream=stream)
        out = hlc.hlc_match(plan, copy=False)
        n_, st_ = out["n"], out["stats"]
        hlc.hlc_free(plan)
        return n_, st_
    t0 = time.perf_counter()
    ms_s, (ns_, st_s), clk = _sampled_loop(args, streamed, args.steps, args.warmup, stream,
                                           "streamed")

    def in_core():
        plan = hlc.hlc_plan(A, B, r, L, coarse_level=Lc, stream=stream)
        out = hlc.hlc_match(plan, copy=False)
        n_ = out["n"]
        hlc.hlc_free(plan)
        return n_
    ms_c, nc_ = _timed_loop(in_core, args.steps, args.warmup, stream)
    # the two row sets, compared on the device (untimed)
    plan = hlc.hlc_plan(Ah, Bh, r, L, coarse_level=Lc, device_mem_budget=budget, stream=stream)
    so = hlc.hlc_match(plan, copy=False)
    sa, sb = so["id_a"].to(dev), so["id_b"].to(dev)
    hlc.hlc_free(plan)
    plan = hlc.hlc_plan(A, B, r, L, coarse_level=Lc, stream=stream)
    co = hlc.hlc_match(plan, copy=False)
    equal_rows = bool(sa.numel() == co["n"] and torch.equal(sa, co["id_a"])
                      and torch.equal(sb, co["id_b"]))
    hlc.hlc_free(plan)
    del sa, sb
    copy_ms = {"h2d": st_s["ms_h2d"], "d2h": st_s["ms_d2h"]}
    tmodel = {"alpha_us": {k: fit[k]["alpha_s"] * 1e6 for k in ("h2d", "d2h")},
              "beta_gbs": {k: fit[k]["gbs"] for k in ("h2d", "d2h")},
              "chunk_sources": st_s["stream_chunk"],
              "h2d": {"bytes": st_s["h2d_bytes"], "copies": st_s["h2d_copies"],
                      "model_ms": st_s["ms_model_h2d"], "measured_copy_ms": copy_ms["h2d"]},
              "d2h": {"bytes": st_s["d2h_bytes"], "copies": st_s["d2h_copies"],
                      "model_ms": st_s["ms_model_d2h"], "measured_copy_ms": copy_ms["d2h"]},
              "model_transfer_share_of_step": (st_s["ms_model_h2d"] + st_s["ms_model_d2h"])
              / ms_s,
              "basis": "Eq. 5 per copy, alpha from a one-byte copy and beta from a 256 MiB "
                       "copy (pinned); measured_copy_ms: the copies' own CUDA-event spans"}
    _line(args, "sources matched/s, streamed from pinned host memory", (n + nb) / (ms_s / 1e3),
          "sources/s", ms_s,
          {"workload": "clusters %s x %s (%d Plummer clusters), r=1 arcsec, fine order 13, "
                       "coarse order 3, device budget %d GiB" % (_mega(n), _mega(nb), ncl,
                                                               args.budget_gb)},
          matches=ns_, clocks=clk, partitions=st_s["partitions"], ms_h2d=st_s["ms_h2d"],
          phases_ms={k: st_s[k] for k in ("ms_stream_count", "ms_stream_bucket",
                                          "ms_stream_groups", "ms_stream_merge", "ms_d2h",
                                          "ms_prep", "ms_sort", "ms_index", "ms_pair",
                                          "ms_recheck", "ms_output")},
          h2d_gbs=st_s["h2d_bytes"] / (st_s["ms_h2d"] / 1e3) / 1e9 if st_s["ms_h2d"] else None,
          in_core={"ms": ms_c, "sources_per_s": (n + nb) / (ms_c / 1e3), "matches": nc_},
          equal_counts=ns_ == nc_, equal_rows=equal_rows, transfer_model=tmodel)


def run_completeness(args):
    """Completeness of the quad-direction strategy (the analogue of Table 4 and
    Sec. 5.3): for catalogues of growing size and several HEALPix orders, the
    pairs each quad reading (Algorithm 1 literal, and with the RA shift
    r / cos(dec)) loses against complete mode, whose set is the exact set of
    Eq. 1 (equal to the oracle's in the parity tests).  The paper's simulated
    data sets are not available; the full-sky recipe (40% uniform + 60%
    galactic disk, B = 60% jittered copies) and a clustered sky stand in."""
    import torch

    import paper_2301_07331_b300 as hlc
    from paper_2301_07331_b300 import synth
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    r = 1.5
    rows = []
    sizes = [int(x) for x in args.sizes.split(",")]
    levels = [int(x) for x in args.levels.split(",")]

    def run(A, B, L, mode):
        ms, (n, st) = _timed_loop(lambda: _one(A, B, L, mode), 2, 1, stream)
        return n, ms

    def _one(A, B, L, mode):
        plan = hlc.hlc_plan(A, B, r, L, coarse_level=min(4, L), boundary=mode, stream=stream)
        res = hlc.hlc_match(plan, copy=False)
        n, st = res["n"], res["stats"]
        hlc.hlc_free(plan)
        return n, st
    skies = [("fullsky", n, lambda n=n: synth.fullsky_pair(na=n, nb=n, device=dev)) for n in sizes]
    skies.append(("clusters", sizes[-1] // 2, lambda: synth.clustered_pair(
        na=sizes[-1] // 2, nb=sizes[-1] // 2, n_clusters=max(1, sizes[-1] // 4_000_000),
        device=dev)))
    for name, n, make in skies:
        A, B = make()
        for L in levels:
            if r > math.sqrt(math.pi / 3) / 2 ** L * 648000 / math.pi / 8:
                continue
            nc, msc = run(A, B, L, hlc.HLC_COMPLETE8)
            nq, msq = run(A, B, L, hlc.HLC_QUAD)
            nqc, msqc = run(A, B, L, hlc.HLC_QUAD_COSDEC)
            rows.append({"sky": name, "n_per_side": n, "order": L, "complete": nc,
                         "quad_lost": nc - nq, "quad_cosdec_lost": nc - nqc,
                         "ms_complete": msc, "ms_quad": msq, "ms_quad_cosdec": msqc})
        del A, B
        torch.cuda.empty_cache()
    total = sum(x["complete"] for x in rows)
    _line(args, "pairs lost by the quad-direction strategy against the exact set",
          sum(x["quad_cosdec_lost"] for x in rows), "pairs", sum(x["ms_quad_cosdec"] for x in rows),
          {"workload": "completeness study: full sky %s per side and a clustered sky, orders %s, "
                       "r = %g arcsec" % ("/".join(_mega(x) for x in sizes), args.levels, r)},
          higher_is_better=False, rows=rows, exact_pairs_total=total,
          quad_lost_total=sum(x["quad_lost"] for x in rows),
          quad_cosdec_lost_total=sum(x["quad_cosdec_lost"] for x in rows))


def run_reference(args):
    """Reference arm: the CPU oracle on a bounded sample per step."""
    import torch

    world, rank, local = _dist()
    if rank != 0:
        return
    import numpy as np

    import oracle as O
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    A, B, r, L, Lc, wname = make_workload(args, 0, dev)
    n_a, n_b = A.ra.numel(), B.ra.numel()
    ra_a, dec_a, id_a = (x.cpu().numpy() for x in (A.ra, A.dec, A.id))
    ra_b, dec_b, id_b = (x.cpu().numpy() for x in (B.ra, B.dec, B.id))
    width = 6.0  # deg of RA per step: about 1/60 of each catalogue
    mode = O.QUAD if args.mode == "quad" else O.COMPLETE
    times, counts = [], []
    for it in range(args.warmup + args.steps):
        lo = (it * width) % 360.0
        sa = (ra_a >= lo) & (ra_a < lo + width)
        sb = (ra_b >= lo) & (ra_b < lo + width)
        t0 = time.perf_counter()
        O.match(ra_a[sa], dec_a[sa], id_a[sa].view(np.uint64), ra_b[sb], dec_b[sb],
                id_b[sb].view(np.uint64), r, L, mode)
        t = time.perf_counter() - t0
        if it >= args.warmup:
            times.append(t)
            counts.append(int(sa.sum() + sb.sum()))
    v = sum(counts) / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "sources/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wname + ", " + args.mode + " mode", "n_a": n_a, "n_b": n_b,
                       "radius_arcsec": r, "fine_level": L, "coarse_level": Lc,
                       "boundary": args.mode},
            "cpu_baseline": {"value": v, "unit": "sources/s", "cores": 1, "kind": "oracle",
                             "sample": "one 6-deg RA strip of both catalogues per step "
                                       "(about 1/60 of the workload)"},
            "e2e": {"value": v, "unit": "sources/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="hlc", choices=["hlc", "reference"])
    ap.add_argument("--workload", default="fullsky",
                    choices=["fullsky", "clusters", "bulge", "learned", "batched", "streamed",
                             "completeness"])
    ap.add_argument("--n-match", type=int, default=100_000_000,
                    help="learned: sources per side of the match slice")
    ap.add_argument("--jobs", type=int, default=4096, help="batched: number of jobs")
    ap.add_argument("--scale", type=float, default=1.0, help="batched: source-count scale")
    ap.add_argument("--tune-sample", type=int, default=1024,
                    help="batched: jobs in the autotuner's calibration sample (0: skip it)")
    ap.add_argument("--budget-gb", type=int, default=16, help="streamed: device budget")
    ap.add_argument("--n", type=int, default=0, help="A sources (0: the workload's size)")
    ap.add_argument("--sizes", default="1000000,4000000,10000000,20000000",
                    help="completeness: sources per side of the full-sky catalogues")
    ap.add_argument("--levels", default="10,11,12,13", help="completeness: HEALPix orders")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--mode", default="complete", choices=["complete", "quad"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-depth", type=int, default=3,
                    help="steps in flight in the end-to-end throughput run")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-per-job", action="store_true",
                    help="batched: skip the one-plan-per-job comparison (profiling runs)")
    ap.add_argument("--no-other-mode", action="store_true",
                    help="skip the other boundary mode's sub-line")
    ap.add_argument("--no-dense", action="store_true", help="skip the dense-cell sub-line")
    ap.add_argument("--no-eq4", action="store_true",
                    help="skip the per-source radii (Eq. 4) sub-line")
    ap.add_argument("--dense-n", type=int, default=20_000_000,
                    help="A sources of the dense-cell sub-line (B = 3/4 of it)")
    ap.add_argument("--clocks-out", default="",
                    help="file for the nvidia-smi samples of the timed region "
                         "(default: one in the temporary directory)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "learned":
        run_learned(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "streamed":
        run_streamed(args)
    elif args.workload == "completeness":
        run_completeness(args)
    else:
        run_hlc(args)


if __name__ == "__main__":
    main()
