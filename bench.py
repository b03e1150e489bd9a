#!/usr/bin/env python
"""Benchmark of the transform-reduce-scan path on B300.

One step = one pass of the hot path over the headline workload: the segmented
transform-reduce of N = 2^28 f32 values x ~ N(0,1) through the rational map
P/Q of degree 6/6 (Q with positive even coefficients, no poles) into 65,536
segments (lengths U{1..8192} rescaled to N): per segment a compensated sum
(FP64 output), min and max -- load, map, accumulate, combine, all in one
tr_segmented_reduce launch.  Inputs (1 GiB) exceed the 126 MB L2, so no flush
is needed between steps.

Prints ONE JSON line (rank 0).  Besides the headline it reports, under
"configs", the other workloads of the path measured the same way (FP64 and
u32 reductions, u32/u64/f32 scans, FP16-storage reduction).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl tr|reference]

--impl reference times the CPU oracle (this project's reference arm: the plain
FP64 / exact-summation C implementation) on a bounded sample of the same
workload on the host cores.
"""
from __future__ import annotations

import argparse
import ctypes
import glob
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("elements/s and HBM GB/s (% of ~8 TB/s) for transform-reduce/scan; "
          "batched vs plain speedup at tol")
NOMINAL_HBM_GBS = 8000.0
N_HEAD = 1 << 28
NSEG_HEAD = 65536
WORKLOAD = ("segmented transform-reduce: N=2^28 f32 x~N(0,1), f = rational P/Q deg 6/6 (Q even, positive "
            "coefficients), 65536 segments with lengths U{1..8192} scaled to N; per segment compensated "
            "sum (f64 out), min, max")
SEG_SOURCES = ["paper_2309_03912_b300/csrc/" + f for f in (
    "k_segreduce.cu", "segreduce_kernel.cuh", "accum.cuh", "range.cuh", "dispatch.cuh", "internal.h",
    "common.cuh", "maps.h", "hd.h")]


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="tr", choices=["tr", "reference"])
    p.add_argument("--no-configs", action="store_true", help="headline only")
    p.add_argument("--no-cpu", action="store_true", help="skip the CPU baseline")
    p.add_argument("--only", default="", help="comma-separated names of the extra configurations to run "
                                              "(scan_u32, scan_f32, rational_reduce, map, reduce_f64, mixers_2^20, batched, vandermonde, f16); "
                                              "skips the headline")
    p.add_argument("--config-log2", type=int, default=28, help="log2 size of the 2^28 scan configurations")
    p.add_argument("--f16-log2", type=int, default=30, help="log2 size of the FP16-storage configuration")
    p.add_argument("--vander-log2-m", type=int, default=20,
                   help="log2 of the points of the Vandermonde configuration (smaller only for profiler captures)")
    p.add_argument("--head-n", type=int, default=N_HEAD,
                   help="elements of the headline workload (segments scale with it); smaller sizes are "
                        "for profiler captures only")
    return p.parse_args()


# ----------------------------------------------------------------------------- utilities

def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), "measured"
    except Exception:
        return 6400.0, 1800.0, "fallback"


class Clocks:
    """nvidia-smi samples (200 ms) while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = tempfile.mktemp(suffix=".csv")

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.3)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.proc:
            return None
        rows = [[s.strip() for s in line.split(",")] for line in open(self.path)]
        rows = [r for r in rows if len(r) >= 9]
        if not rows:
            return None

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for name, val in zip(names, r[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        pw = [num(r[3]) for r in rows if num(r[3]) is not None]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": num(rows[0][2]),
                "power_w_max": max(pw) if pw else None, "reasons": sorted(reasons), "samples": len(rows)}


def source_sha(sources):
    h = hashlib.sha256()
    for s in sources:
        with open(os.path.join(ROOT, s), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profile_traffic(kernel: str, sources: list[str]):
    """DRAM bytes per launch from an ncu capture summarised in profiles/, valid
    only while the kernel's sources are unchanged (their sha256 is stored there)."""
    sha = source_sha(sources)
    for p in glob.glob(os.path.join(ROOT, "profiles", f"{kernel}*.md")):
        txt = open(p).read()
        ms = re.search(r"source_sha:\s*([0-9a-f]+)", txt)
        mt = re.search(r"traffic_bytes_per_launch:\s*([0-9.e+]+)", txt)
        mn = re.search(r"traffic_n:\s*([0-9]+)", txt)
        if ms and mt and ms.group(1) == sha:
            return float(mt.group(1)), (int(mn.group(1)) if mn else None), sha
    return None, None, sha


def max_over_ranks(ms: float, world: int, device) -> float:
    """The slowest rank's time (every rank gets it); the job's throughput is
    the units all ranks processed divided by this."""
    if world == 1:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def time_launches(fn, steps, warmup, stream):
    """Device time per call (ms): CUDA events on `stream` between calls."""
    import torch
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        evs[0].record(stream)
        for i in range(steps):
            fn()
            evs[i + 1].record(stream)
        torch.cuda.synchronize()
    per = [evs[i].elapsed_time(evs[i + 1]) for i in range(steps)]
    return statistics.mean(per), min(per), per


def time_graph(fn, reps, stream, replays=10):
    """Device time per call (ms) of `fn` captured `reps` times into one CUDA
    graph (the C-ABI calls allocate and synchronise nothing, so they capture),
    replayed `replays` times between CUDA events.  Used for the small sizes,
    whose kernels are shorter than a host launch."""
    import torch
    with torch.cuda.stream(stream):
        fn()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            for _ in range(reps):
                fn()
        g.replay()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(replays):
            g.replay()
        b.record()
        torch.cuda.synchronize()
    return a.elapsed_time(b) / (replays * reps)


# ----------------------------------------------------------------------------- headline

def headline(args, rank, world, stream):
    import numpy as np
    import torch

    from paper_2309_03912_b300 import binding as B
    from paper_2309_03912_b300 import inputs as I

    nseg_req = max(1, round(NSEG_HEAD * args.head_n / N_HEAD))
    x, m, off = I.rational_segments(args.head_n, nseg_req, salt=rank)
    n, nseg = x.size, off.size - 1
    xd = torch.from_numpy(x).cuda()
    offd = torch.from_numpy(off).cuda()
    sums = torch.empty(nseg, dtype=torch.float64, device="cuda")
    mins = torch.empty(nseg, dtype=torch.float32, device="cuda")
    maxs = torch.empty(nseg, dtype=torch.float32, device="cuda")
    ws = B.workspace(B.tr_segmented_reduce_workspace_size(n, nseg, B.TR_F32))
    ex = B.make_exec(ws, stream=stream)
    ops = B.TR_SUM | B.TR_MIN | B.TR_MAX
    md = B.MapDesc(m)
    L = B.lib()
    exr = ctypes.byref(ex)

    def step():
        st = L.tr_segmented_reduce(md.ref(), xd.data_ptr(), B.TR_F32, n, offd.data_ptr(), nseg, ops,
                                   sums.data_ptr(), B.TR_F64, mins.data_ptr(), maxs.data_ptr(), exr)
        if st:
            raise B.TrError(st, L.tr_last_error().decode())

    with torch.cuda.stream(stream):
        clk = Clocks(torch.cuda.current_device())
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        with clk:
            # the warm-up steps run right before the timed ones (the sampler's start-up pause comes first,
            # so the GPU does not sit idle between warm-up and timing)
            for _ in range(args.warmup):
                step()
            B.tr_check(ex)
            if world > 1:
                torch.distributed.barrier()
            torch.cuda.synchronize()
            launches0 = B.tr_launch_count()
            evs[0].record(stream)
            for i in range(args.steps):
                step()
                evs[i + 1].record(stream)
            torch.cuda.synchronize()
            launches = B.tr_launch_count() - launches0
        if world > 1:
            torch.distributed.barrier()
        B.tr_check(ex)
        per = [evs[i].elapsed_time(evs[i + 1]) for i in range(args.steps)]
        total_ms = evs[0].elapsed_time(evs[-1])
        total_ms = max_over_ranks(total_ms, world, "cuda")
        results = (sums.cpu().numpy(), mins.cpu().numpy(), maxs.cpu().numpy())

        # end to end through the library's host-buffer entry point: every step copies x and the
        # offsets in from page-locked host memory and the results back out, inside the timed region
        xh = torch.from_numpy(x).pin_memory()
        offh = torch.from_numpy(off).pin_memory()
        sums_h = torch.empty(nseg, dtype=torch.float64).pin_memory()
        mins_h = torch.empty(nseg, dtype=torch.float32).pin_memory()
        maxs_h = torch.empty(nseg, dtype=torch.float32).pin_memory()

        def e2e_step():
            st = L.tr_segmented_reduce_host(md.ref(), xh.data_ptr(), B.TR_F32, n, offh.data_ptr(), nseg, ops,
                                            sums_h.data_ptr(), B.TR_F64, mins_h.data_ptr(), maxs_h.data_ptr(),
                                            xd.data_ptr(), offd.data_ptr(), sums.data_ptr(), mins.data_ptr(),
                                            maxs.data_ptr(), exr)
            if st:
                raise B.TrError(st, L.tr_last_error().decode())

        e2e_ms, _, _ = time_launches(e2e_step, max(3, min(args.steps, 10)), 2, stream)
        B.tr_check(ex)
        assert np.array_equal(sums_h.numpy(), results[0]), "host-buffer call differs from the device call"
    return {"n": n, "nseg": nseg, "per_ms": per, "total_ms": total_ms, "clocks": clk.summary(),
            "alg_bytes": n * 4 + (nseg + 1) * 8 + nseg * 16, "e2e_ms": e2e_ms,
            "h2d": n * 4 + (nseg + 1) * 8, "d2h": nseg * 16, "launches": launches,
            "x": x, "off": off, "map": m, "results": results}


# ----------------------------------------------------------------------------- other workloads

def other_configs(args, stream, hbm_peak, tensor_peak=1781.3):
    """The other workloads of the path, each timed with CUDA events.  Returns
    (records, checks): checks[name] holds the inputs and GPU outputs the CPU
    leg compares with the oracle (outside every timed region)."""
    import numpy as np
    import torch

    from paper_2309_03912_b300 import binding as B
    from paper_2309_03912_b300 import inputs as I

    out, checks = {}, {}
    steps, warm = max(5, min(args.steps, 20)), 3
    only = [o for o in args.only.split(",") if o]
    want = lambda name: not only or name in only
    big = 1 << args.config_log2

    def record(name, ms, n, nbytes, launches, extra=None):
        gbs = nbytes / (ms * 1e-3) / 1e9
        d = {"ms": round(ms, 5), "elements_per_s": n / (ms * 1e-3), "alg_bytes": nbytes, "hbm_gbs": round(gbs, 1),
             "frac_of_measured_hbm": round(gbs / hbm_peak, 4), "frac_of_8tbs": round(gbs / NOMINAL_HBM_GBS, 4),
             "launches_per_step": launches}
        d.update(extra or {})
        out[name] = d

    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # > L2, for the L2-resident sizes

    if want('reduce_f64'):
        # plain FP64 Horner reduce, N = 2^20 (L2-resident: timed as graph replays of 20 calls,
        # with and without an L2 flush before each call)
        x, m = I.horner_f64(1 << 20)
        xd = torch.from_numpy(x).cuda()
        ws = B.workspace(B.tr_reduce_workspace_size(x.size, B.TR_F64))
        s = torch.empty(3, dtype=torch.float64, device="cuda")
        f = lambda: B.tr_reduce(m, xd, 7, s[0:1], s[1:2], s[2:3], B.make_exec(ws))
        ms = time_graph(f, 20, stream)
        ms_flush = time_graph(lambda: (flush.zero_(), f()), 20, stream) - time_graph(lambda: flush.zero_(), 20, stream)
        name = "reduce_f64_horner8_2^20"
        record(name, ms, x.size, x.nbytes, 1,
               {"ms_after_l2_flush": round(ms_flush, 5), "timing": "cuda graph of 20 calls",
                "bound": "FP64 ALU (B300 FP64 is ~1/64 of FP32) and launch latency"})
        checks[name] = {"kind": "reduce_f64", "x": x, "map": m, "got": s.cpu().numpy()}

    if want('mixers_2^20'):
        # u32 xorshift32: exact u64 sum + u32 -> u64 inclusive scan, N = 2^20
        xu = I.mixer_u32(1 << 20)
        xud = torch.from_numpy(xu.view(np.int32)).cuda()
        wsr = B.workspace(B.tr_reduce_workspace_size(xu.size, B.TR_U32))
        wss = B.workspace(B.tr_scan_workspace_size(xu.size, B.TR_U32, B.TR_U64))
        s64 = torch.empty(1, dtype=torch.int64, device="cuda")
        y64 = torch.empty(xu.size, dtype=torch.int64, device="cuda")

        def c1b():
            B.tr_reduce({"kind": "xorshift32"}, xud, 1, s64, None, None, B.make_exec(wsr))
            B.tr_scan({"kind": "xorshift32"}, xud, y64, B.make_exec(wss))
        ms = time_graph(c1b, 20, stream)
        name = "sum_u64_and_scan_u64_xorshift32_2^20"
        record(name, ms, xu.size, xu.nbytes * 2 + y64.numel() * 8, 2, {"timing": "cuda graph of 20 calls"})
        checks[name] = {"kind": "mixers", "x": xu, "sum": int(s64.cpu().numpy().view(np.uint64)[0]),
                        "scan": y64.cpu().numpy().view(np.uint64)}
        del xud, y64

    if want('scan_u32'):
        # u32 splitmix32 inclusive scan mod 2^32, N = 2^28
        xu = I.mixer_u32(big, stream="mixer_u32_scan")
        xud = torch.from_numpy(xu.view(np.int32)).cuda()
        y = torch.empty_like(xud)
        wss = B.workspace(B.tr_scan_workspace_size(xud.numel(), B.TR_U32, B.TR_U32))
        exs = B.make_exec(wss, stream=stream)
        ms, _, _ = time_launches(lambda: B.tr_scan({"kind": "splitmix32"}, xud, y, exs), steps, warm, stream)
        B.tr_check(exs)
        name = f"scan_u32_splitmix32_2^{args.config_log2}"
        record(name, ms, xud.numel(), xud.numel() * 8, 1)
        checks[name] = {"kind": "scan_u32", "x": xu, "got": y.cpu().numpy().view(np.uint32)}
        # the same scan with sum / min / max of f from the same pass (one read of x, one write of y)
        sr = torch.zeros(3, dtype=torch.int32, device="cuda")
        ms_f, _, _ = time_launches(lambda: B.tr_scan_reduce({"kind": "splitmix32"}, xud, y, exs, ops=7,
                                                            out_sum=sr[0:1], out_min=sr[1:2], out_max=sr[2:3]),
                                   steps, warm, stream)
        B.tr_check(exs)
        name_f = f"scan_reduce_u32_splitmix32_2^{args.config_log2}"
        record(name_f, ms_f, xud.numel(), xud.numel() * 8, 1,
               {"fused": "inclusive scan + sum (mod 2^32) / min / max of f in one pass", "plain_scan_ms": round(ms, 5)})
        checks[name_f] = {"kind": "scan_reduce_u32", "x": xu, "got": y.cpu().numpy().view(np.uint32),
                          "red": sr.cpu().numpy().view(np.uint32).copy()}
        del xud, y

    if want('rational_reduce'):
        # the headline's map and inputs without segments: one sum / min / max over all 2^28 values (the
        # map's own ceiling for the segmented step)
        xr, mr, _ = I.rational_segments(N_HEAD, NSEG_HEAD)
        xrd = torch.from_numpy(xr).cuda()
        wsr = B.workspace(B.tr_reduce_workspace_size(xrd.numel(), B.TR_F32))
        exr = B.make_exec(wsr, stream=stream)
        sr = torch.empty(1, dtype=torch.float64, device="cuda")
        mmr = torch.empty(2, dtype=torch.float32, device="cuda")
        ms, _, _ = time_launches(lambda: B.tr_reduce(mr, xrd, 7, sr, mmr[0:1], mmr[1:2], exr), steps, warm, stream)
        B.tr_check(exr)
        name = "reduce_rational66_2^28_no_segments"
        record(name, ms, xrd.numel(), xrd.numel() * 4, 1,
               {"note": "the headline's map and input as one array: the cost of the map and the sum alone"})
        checks[name] = {"kind": "reduce_rational", "x": xr, "map": mr,
                        "got": (float(sr.item()), float(mmr[0].item()), float(mmr[1].item()))}
        del xrd

    if want('map'):
        # y = f(x) alone: the headline's map over its 2^28 inputs (read 1 GiB, write 1 GiB)
        xm_, mm_, _ = I.rational_segments(N_HEAD, NSEG_HEAD)
        xmd = torch.from_numpy(xm_).cuda()
        ym = torch.empty_like(xmd)
        exm = B.make_exec(None, stream=stream)
        ms, _, _ = time_launches(lambda: B.tr_map(mm_, xmd, ym, exm), steps, warm, stream)
        name = "map_rational66_2^28"
        record(name, ms, xmd.numel(), xmd.numel() * 8, 1)
        checks[name] = {"kind": "map_rational", "x": xm_, "map": mm_, "got": ym.cpu().numpy()}
        del xmd, ym

    if want('scan_f32'):
        # f32 compensated scan of x^2, N = 2^28
        xf = I.square_f32(big)
        xfd = torch.from_numpy(xf).cuda()
        y = torch.empty_like(xfd)
        wss = B.workspace(B.tr_scan_workspace_size(xfd.numel(), B.TR_F32, B.TR_F32))
        exs = B.make_exec(wss, stream=stream)
        ms, _, _ = time_launches(lambda: B.tr_scan(I.simple_map("square"), xfd, y, exs), steps, warm, stream)
        B.tr_check(exs)
        name = f"scan_f32_square_compensated_2^{args.config_log2}"
        record(name, ms, xfd.numel(), xfd.numel() * 8, 1)
        pos = np.unique(np.concatenate([np.random.default_rng(5).integers(0, xf.size, 4090),
                                        [0, 1, 8191, 8192, xf.size - 1]]))
        checks[name] = {"kind": "scan_f32", "x": xf, "pos": pos,
                        "got": y[torch.from_numpy(pos).cuda()].cpu().numpy()}
        del xfd, y

    if want('batched'):
        # batched: 10,000 f32 arrays (separate allocations), lengths log-uniform in [1, 2^20], map per array from
        # {Horner deg 4-16, rational 6/6, Newton 6}; one persistent launch in a CUDA graph, autotuned tiles,
        # against one tr_reduce launch per array (eager, and the same launches recorded in a graph)
        xs, lens, maps = I.batched(10000)
        total = int(np.sum(lens))
        dev = [torch.from_numpy(x).cuda() for x in xs]
        nb = len(dev)
        bs = torch.zeros(nb, dtype=torch.float64, device="cuda")
        bmn = torch.zeros(nb, dtype=torch.float32, device="cuda")
        bmx = torch.zeros(nb, dtype=torch.float32, device="cuda")
        with torch.cuda.stream(stream):
            plan = B.BatchPlan(dev, maps, bs, bmn, bmx, autotune=True, stream=stream)
        ms_b, _, _ = time_launches(lambda: plan.run(stream), steps, warm, stream)
        got = (bs.cpu().numpy(), bmn.cpu().numpy(), bmx.cpu().numpy())
        ms_eager, _, _ = time_launches(lambda: plan.run_unbatched(False, stream), 3, 1, stream)
        ms_graph, _, _ = time_launches(lambda: plan.run_unbatched(True, stream), 3, 1, stream)
        kinds = {}
        for m in maps:
            kinds[m["kind"]] = kinds.get(m["kind"], 0) + 1
        plan_desc = plan.describe()
        plan.close()
        del dev
        # the mix's roofline: the larger of the HBM time of its bytes and the FMA-pipe time of its
        # arithmetic, counted per element from each map's operation sequence (FP32 lane operations on
        # the FMA pipe: Horner degree d: d fmas + 1 for the compensated sum; rational dp/dq: dp + dq
        # fmas + 6 for the correctly rounded quotient + 1; Newton, I steps: 10 per step (the square, five for
        # the negated quotient, the step, three for the division by 3), one sign at the end, 1), and of its
        # reciprocals on the XU pipe (one per quotient)
        props = torch.cuda.get_device_properties(0)
        clock_hz = 2.032e9
        fma_ops, xu_ops, per_map = 0.0, 0.0, {}
        for m, L in zip(maps, lens):
            if m["kind"] == "horner":
                f_, x_, label = len(m["cp"]) - 1 + 1, 0, "horner"
            elif m["kind"] == "rational":
                f_, x_, label = (len(m["cp"]) - 1) + (len(m["cq"]) - 1) + 7, 1, "rational"
            else:
                f_, x_, label = 10 * m["iters"] + 2, m["iters"], "newton_cbrt"
            fma_ops += f_ * int(L)
            xu_ops += x_ * int(L)
            d = per_map.setdefault(label, {"elements": 0, "fma_lane_ops": 0})
            d["elements"] += int(L)
            d["fma_lane_ops"] += f_ * int(L)
        t_hbm = total * 4 / (hbm_peak * 1e9) * 1e3
        t_fma = fma_ops / (props.multi_processor_count * 128 * clock_hz) * 1e3
        t_xu = xu_ops / (props.multi_processor_count * 16 * clock_hz) * 1e3
        floor_ms = max(t_hbm, t_fma, t_xu)
        bound = {t_hbm: "hbm", t_fma: "fma pipe", t_xu: "xu pipe"}[floor_ms]
        name = "batched_10000_arrays_mixed_maps"
        record(name, ms_b, total, total * 4, 1,
               {"plan": plan_desc, "arrays": nb, "maps": kinds, "unbatched_eager_ms": round(ms_eager, 4),
                "unbatched_graph_ms": round(ms_graph, 4), "speedup_vs_eager": round(ms_eager / ms_b, 2),
                "speedup_vs_graph": round(ms_graph / ms_b, 2), "launches_unbatched": nb,
                "roofline": {"bound": bound, "floor_ms": round(floor_ms, 4), "frac": round(floor_ms / ms_b, 4),
                             "hbm_ms": round(t_hbm, 4), "fma_pipe_ms": round(t_fma, 4), "xu_pipe_ms": round(t_xu, 4),
                             "per_map": per_map,
                             "peaks": f"measured HBM {hbm_peak} GB/s; FMA pipe {props.multi_processor_count} SMs x "
                                      f"128 lanes x {clock_hz / 1e9} GHz; XU 16 lanes per SM"}})
        checks[name] = {"kind": "batched", "xs": xs, "maps": maps, "got": got}

    if want('vandermonde'):
        # 4096 polynomials of degree 31 at 2^20 points: Y = V(x) C (16 GiB of FP32 output), split-BF16 on
        # the tensor cores against plain FP32 Horner on the CUDA cores
        x, C = I.vandermonde(1 << args.vander_log2_m)
        xd, Cd = torch.from_numpy(x).cuda(), torch.from_numpy(C).cuda()
        m, npoly = x.size, C.shape[1]
        y = torch.empty((m, npoly), dtype=torch.float32, device="cuda")
        wsv = B.workspace(B.tr_vandermonde_workspace_size(m, npoly))
        exv = B.make_exec(wsv, stream=stream)
        vs = max(3, steps // 4)
        rows = np.arange(0, m, max(1, m // 512), dtype=np.int64)
        rows_d = torch.from_numpy(rows).cuda()
        ms_tc, _, _ = time_launches(lambda: B.tr_vandermonde(xd, Cd, y, B.TR_PREC_BF16X3, exv), vs, 2, stream)
        B.tr_check(exv)
        got_tc = y[rows_d].cpu().numpy()
        ms_32, _, _ = time_launches(lambda: B.tr_vandermonde(xd, Cd, y, B.TR_PREC_FP32, exv), vs, 2, stream)
        B.tr_check(exv)
        got_32 = y[rows_d].cpu().numpy()
        flops = 2.0 * m * 32 * npoly
        nbytes = m * npoly * 4 + m * 4 + C.nbytes
        vtag = f"2^{args.vander_log2_m}x32x4096"
        name_tc, name_32 = f"vandermonde_bf16x3_{vtag}", f"vandermonde_fp32_horner_{vtag}"
        record(name_tc, ms_tc, m * npoly, nbytes, 1,
               {"bound": "hbm (output write)", "tflops_algorithmic": round(flops / (ms_tc * 1e-3) / 1e12, 1),
                "tflops_tensor_executed": round(3 * flops / (ms_tc * 1e-3) / 1e12, 1),
                "fp32_horner_ms": round(ms_32, 4), "speedup_vs_fp32_horner": round(ms_32 / ms_tc, 3)})
        record(name_32, ms_32, m * npoly, nbytes, 1,
               {"bound": "fp32 fma pipe / hbm", "tflops": round(flops / (ms_32 * 1e-3) / 1e12, 1)})
        checks[name_tc] = {"kind": "vandermonde", "x": x, "C": C, "rows": rows, "got": got_tc, "bar": 1e-4}
        checks[name_32] = {"kind": "vandermonde", "x": x, "C": C, "rows": rows, "got": got_32,
                           "bar": 63 * 2.0 ** -24 / (1 - 63 * 2.0 ** -24)}
        # BF16 output (half the bytes written)
        yb = torch.empty((m, npoly), dtype=torch.bfloat16, device="cuda")
        del y
        ms_bf, _, _ = time_launches(lambda: B.tr_vandermonde(xd, Cd, yb, B.TR_PREC_BF16X3, exv), vs, 2, stream)
        B.tr_check(exv)
        name_bf = f"vandermonde_bf16x3_bf16out_{vtag}"
        record(name_bf, ms_bf, m * npoly, m * npoly * 2 + m * 4 + C.nbytes, 1,
               {"bound": "hbm (output write)", "tflops_algorithmic": round(flops / (ms_bf * 1e-3) / 1e12, 1)})
        checks[name_bf] = {"kind": "vandermonde", "x": x, "C": C, "rows": rows,
                           "got": yb[rows_d].float().cpu().numpy(), "bar": 1e-4 + 2.0 ** -8}
        del yb
        # the fused per-column sum / min / max without writing Y: tensor-bound
        cs = [torch.empty(npoly, dtype=torch.float32, device="cuda") for _ in range(3)]
        sub = 8192  # the error check: these points' column results against the oracle's full product
        for prec, tag, nprod in ((B.TR_PREC_BF16X3, "bf16x3", 3), (B.TR_PREC_BF16X6, "bf16x6", 6)):
            fn = lambda: B.tr_vandermonde(xd, Cd, None, prec, exv, colsum=cs[0], colmin=cs[1], colmax=cs[2])
            ms_c, _, _ = time_launches(fn, vs, 2, stream)
            B.tr_check(exv)
            tf_exec = nprod * flops / (ms_c * 1e-3) / 1e12
            name_c = f"vandermonde_{tag}_column_sum_min_max_{vtag}"
            record(name_c, ms_c, m * npoly, m * 4 + C.nbytes + 3 * npoly * 4, 2,
                   {"bound": "tensor", "tflops_algorithmic": round(flops / (ms_c * 1e-3) / 1e12, 1),
                    "tflops_tensor_executed": round(tf_exec, 1), "tensor_peak_tflops_bf16": tensor_peak,
                    "frac_of_tensor_peak": round(tf_exec / tensor_peak, 4),
                    "note": "frac_of_measured_hbm does not apply (no Y is written)"})
            B.tr_vandermonde(xd[:sub], Cd, None, prec, exv, colsum=cs[0], colmin=cs[1], colmax=cs[2])
            B.tr_check(exv)
            checks[name_c] = {"kind": "vandermonde_cols", "x": x[:sub], "C": C,
                              "got": [c.cpu().numpy().astype(np.float64) for c in cs],
                              "bar": 1e-4 if nprod == 3 else 1e-5}
        del xd, Cd

    if want('f16'):
        # FP16 storage, FP32 compute: Horner deg 8 sum/min/max, N = 2^30
        xh, m = I.horner_f16(1 << args.f16_log2)
        xhd = torch.from_numpy(xh).cuda()
        ws = B.workspace(B.tr_reduce_workspace_size(xhd.numel(), B.TR_F16))
        ex = B.make_exec(ws, stream=stream)
        s = torch.empty(1, dtype=torch.float64, device="cuda")
        mm = torch.empty(2, dtype=torch.float32, device="cuda")
        ms16, _, _ = time_launches(lambda: B.tr_reduce(m, xhd, 7, s, mm[0:1], mm[1:2], ex), steps, warm, stream)
        got16 = (float(s.item()), float(mm[0].item()), float(mm[1].item()))
        name16 = f"reduce_f16_storage_horner8_2^{args.f16_log2}"
        record(name16, ms16, xhd.numel(), xhd.numel() * 2, 1)
        # the same values in f32 storage: the plain FP32 comparison for the mixed-precision form
        xfd = xhd.float()
        del xhd
        ws = B.workspace(B.tr_reduce_workspace_size(xfd.numel(), B.TR_F32))
        ex = B.make_exec(ws, stream=stream)
        ms32, _, _ = time_launches(lambda: B.tr_reduce(m, xfd, 7, s, mm[0:1], mm[1:2], ex), steps, warm, stream)
        got32 = (float(s.item()), float(mm[0].item()), float(mm[1].item()))
        name32 = f"reduce_f32_storage_horner8_2^{args.f16_log2}"
        record(name32, ms32, xfd.numel(), xfd.numel() * 4, 1, {"f16_storage_speedup": round(ms32 / ms16, 3)})
        checks[name16] = {"kind": "reduce_f32c", "x": xh, "map": m, "got": got16}
        checks[name32] = {"kind": "reduce_f32c", "x": xh, "map": m, "got": got32, "same_values_as": name16}
        del xfd

    torch.cuda.synchronize()
    return out, checks


# ----------------------------------------------------------------------------- CPU leg: the oracle

def _err(max_err, bar, checked, ok=True, **extra):
    d = {"max_normwise": float(max_err), "bar": bar, "pass": bool(ok and max_err <= bar), "checked": checked}
    d.update(extra)
    return d


def _minmax_rel(lo, hi, rlo, rhi):
    """max |min - min_ref|, |max - max_ref| relative to max(|min_ref|, |max_ref|), non-empty results only."""
    import numpy as np
    lo, hi, rlo, rhi = (np.atleast_1d(np.asarray(v, dtype=np.float64)) for v in (lo, hi, rlo, rhi))
    ne = np.isfinite(rlo)
    if not ne.any():
        return 0.0
    scale = np.maximum(np.maximum(np.abs(rlo[ne]), np.abs(rhi[ne])), 1e-300)
    return float(np.max(np.maximum(np.abs(lo[ne] - rlo[ne]), np.abs(hi[ne] - rhi[ne])) / scale))


def _normwise(got, ref, scale):
    import numpy as np
    got, ref, scale = (np.atleast_1d(np.asarray(v, dtype=np.float64)) for v in (got, ref, scale))
    e = np.abs(got - ref) / np.maximum(scale, 1e-300)
    return float(np.max(e)) if e.size else 0.0


def check_configs(checks, threads):
    """The error of every result of the other workloads against the oracle
    (host cores, outside every timed region): normwise for float sums (|s -
    s_ref| / sum |f_ref|), relative to max |f_ref| for min / max, bit-exact
    mismatch counts for integer results."""
    import numpy as np

    import oracle
    errs = {}
    for name, c in checks.items():
        k = c["kind"]
        if k == "reduce_f64":
            spec = oracle.MapSpec("horner", c["map"]["cp"])
            rs, rlo, rhi, ra = oracle.reduce_float_mt(spec, c["x"], threads)
            s, lo, hi = c["got"]
            exact = lo == rlo and hi == rhi
            errs[name] = _err(abs(s - rs) / ra, 1e-13, "the sum, min and max", exact,
                              minmax="bit-exact" if exact else "differs")
        elif k == "mixers":
            spec = oracle.MapSpec("xorshift32")
            rs, _, _ = oracle.reduce_u32(spec, c["x"])
            bad = int(np.count_nonzero(c["scan"] != oracle.scan_u32_u64(spec, c["x"]))) + int(c["sum"] != rs)
            errs[name] = {"mismatches": bad, "bar": 0, "pass": bad == 0,
                          "checked": f"the u64 sum and all {c['x'].size} scan outputs, bit for bit"}
        elif k == "scan_u32":
            bad = int(np.count_nonzero(c["got"] != oracle.scan_u32(oracle.MapSpec("splitmix32"), c["x"])))
            errs[name] = {"mismatches": bad, "bar": 0, "pass": bad == 0,
                          "checked": f"all {c['x'].size} outputs, bit for bit"}
        elif k == "scan_reduce_u32":
            spec = oracle.MapSpec("splitmix32")
            rs, rlo, rhi = oracle.reduce_u32(spec, c["x"])
            bad = int(np.count_nonzero(c["got"] != oracle.scan_u32(spec, c["x"])))
            red_ok = [int(v) for v in c["red"]] == [rs % (1 << 32), rlo, rhi]
            errs[name] = {"mismatches": bad + (0 if red_ok else 1), "bar": 0, "pass": bad == 0 and red_ok,
                          "checked": f"all {c['x'].size} outputs and the sum, min, max, bit for bit"}
        elif k == "map_rational":
            m = c["map"]
            ref = oracle.map_values_f32(oracle.MapSpec(m["kind"], m["cp"], m["cq"]), c["x"])
            bad = int(np.count_nonzero(c["got"].astype(np.float64) != ref))
            errs[name] = {"mismatches": bad, "bar": 0, "pass": bad == 0,
                          "checked": f"all {c['x'].size} outputs against the map in binary32, bit for bit"}
        elif k == "reduce_rational":
            m = c["map"]
            spec = oracle.MapSpec(m["kind"], m["cp"], m["cq"])
            rs, rlo, rhi, ra = oracle.reduce_float_mt(spec, c["x"], threads)
            s, lo, hi = c["got"]
            em = _minmax_rel(lo, hi, rlo, rhi)
            errs[name] = _err(abs(s - rs) / ra, 1e-6, "the whole sum, min and max", em <= 1e-5,
                              minmax_rel_max_abs=em, minmax_bar=1e-5)
        elif k == "scan_f32":
            ref = oracle.scan_float_sampled(oracle.MapSpec("square"), c["x"], c["pos"])
            e = _normwise(c["got"], ref, np.abs(ref))
            errs[name] = _err(e, 1e-5, f"{c['pos'].size} of {c['x'].size} prefixes (exact, rounded once)",
                              metric="relative per output (all terms >= 0)")
        elif k == "batched":
            # the compensated sums against the exact sums of the binary32 map values (which the
            # device reproduces bit for bit; min / max must equal theirs), and, reported beside,
            # against FP64 evaluation of the maps (which adds the FP32 maps' own rounding)
            es, e64, em64, mm_exact = 0.0, 0.0, 0.0, True
            s, lo, hi = c["got"]
            for a, (x, m) in enumerate(zip(c["xs"], c["maps"])):
                spec = oracle.MapSpec(m["kind"], m.get("cp"), m.get("cq"), m.get("iters", 6))
                th = threads if x.size >= 65536 else 1
                rs, rlo, rhi, ra = oracle.reduce_float_mt(spec, x, th, f32=True)
                es = max(es, abs(s[a] - rs) / max(ra, 1e-300))
                mm_exact = mm_exact and lo[a] == rlo and hi[a] == rhi
                rs, rlo, rhi, ra = oracle.reduce_float_mt(spec, x, th)
                e64 = max(e64, abs(s[a] - rs) / max(ra, 1e-300))
                em64 = max(em64, _minmax_rel(lo[a], hi[a], rlo, rhi))
            errs[name] = _err(es, 1e-6, f"all {len(c['xs'])} arrays", mm_exact,
                              metric="|s - sum f32(x)| / sum |f32(x)|, f32 = the map in binary32 (bit-identical "
                                     "on the device)", minmax="bit-exact" if mm_exact else "differs",
                              vs_fp64={"max_normwise": e64, "minmax_rel_max_abs": em64,
                                       "note": "includes the FP32 evaluation error of the maps"})
        elif k == "vandermonde":
            y, S = oracle.vandermonde(c["x"], c["C"], c["rows"])
            e = _normwise(c["got"], y, S)
            errs[name] = _err(e, c["bar"], f"{c['rows'].size} of {c['x'].size} rows x {c['C'].shape[1]} polynomials",
                              metric="|y - y_ref| / sum_k |C_kj| |x_i|^k")
        elif k == "vandermonde_cols":
            y, S = oracle.vandermonde(c["x"], c["C"])
            s, lo, hi = c["got"]
            rs = np.array([math.fsum(y[:, j]) for j in range(y.shape[1])])
            es = _normwise(s, rs, S.sum(axis=0))
            em = max(_normwise(lo, y.min(axis=0), S.max(axis=0)), _normwise(hi, y.max(axis=0), S.max(axis=0)))
            errs[name] = _err(max(es, em), c["bar"], f"the column sum, min and max over the first {c['x'].size} "
                              f"points, all {y.shape[1]} polynomials (a run on those points)",
                              metric="sums: / sum_i S_ij; min, max: / max_i S_ij", sum_err=es, minmax_err=em)
        elif k == "reduce_f32c":
            spec = oracle.MapSpec("horner", c["map"]["cp"])
            rs, rlo, rhi, ra = oracle.reduce_float_mt(spec, c["x"], threads)
            s, lo, hi = c["got"]
            em = _minmax_rel(lo, hi, rlo, rhi)
            errs[name] = _err(abs(s - rs) / ra, 1e-6, "the whole sum, min and max", em <= 1e-5,
                              minmax_rel_max_abs=em, minmax_bar=1e-5)
    return errs


def cpu_leg(h, checks, threads):
    """The oracle on the host cores: timed on the whole headline workload with
    one thread and with every core it may use (both runs compute the same exact
    results), then the error of every GPU result against it."""
    import numpy as np

    import oracle
    oracle.build()
    m = h["map"]
    spec = oracle.MapSpec(m["kind"], m["cp"], m["cq"])
    x, off = h["x"], h["off"]
    t0 = time.perf_counter()
    oracle.segmented_reduce_float_mt(spec, x, off, 1)
    t1 = time.perf_counter() - t0
    t0 = time.perf_counter()
    rs, rlo, rhi, ra = oracle.segmented_reduce_float_mt(spec, x, off, threads)
    tn = time.perf_counter() - t0
    n = x.size
    cb = {"value": n / tn, "unit": "elements/s", "cores": threads, "kind": "oracle",
          "sample": f"the whole headline workload ({n} elements, {off.size - 1} segments; exact sums of f and "
                    f"|f|, min, max): {tn:.2f} s on {threads} threads, {t1:.2f} s on one",
          "single_thread": {"value": n / t1, "unit": "elements/s", "cores": 1, "seconds": round(t1, 3)},
          "host": {"os_cpu_count": os.cpu_count(), "affinity_cores": threads}}
    s, lo, hi = h["results"]
    em = _minmax_rel(lo, hi, rlo, rhi)
    r32 = oracle.segmented_reduce_float_mt(spec, x, off, threads, f32=True)
    ne = np.isfinite(r32[1])
    err = _err(_normwise(s, rs, ra), 1e-6, f"all {off.size - 1} segments", em <= 1e-5,
               minmax_rel_max_abs=em, minmax_bar=1e-5, metric="|s - s_ref| / sum |f_ref| per segment (FP64 f)",
               vs_binary32_values={"max_normwise": _normwise(s, r32[0], r32[3]),
                                   "minmax": "bit-exact" if (np.array_equal(lo[ne], r32[1][ne]) and
                                                             np.array_equal(hi[ne], r32[2][ne])) else "differs"})
    t0 = time.perf_counter()
    errs = check_configs(checks, threads) if checks else {}
    return cb, err, errs, time.perf_counter() - t0


def reference_arm(args):
    """--impl reference: the oracle as it stands on the host cores, each step
    the first segments of the headline workload holding about 2^25 elements."""
    import numpy as np

    import oracle
    from paper_2309_03912_b300 import inputs as I
    oracle.build()
    threads = oracle.host_threads()
    x, m, off = I.rational_segments(N_HEAD, NSEG_HEAD)
    k = max(1, min(int(np.searchsorted(off, 1 << 25)), off.size - 1))
    sub_off = np.ascontiguousarray(off[:k + 1])
    nel = int(sub_off[-1])
    xs = np.ascontiguousarray(x[:nel])
    del x
    spec = oracle.MapSpec(m["kind"], m["cp"], m["cq"])
    for _ in range(args.warmup):
        oracle.segmented_reduce_float_mt(spec, xs[:1 << 20], sub_off[sub_off <= (1 << 20)], threads)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.segmented_reduce_float_mt(spec, xs, sub_off, threads)
        times.append(time.perf_counter() - t0)
    value = nel / statistics.mean(times)
    cb = {"value": value, "unit": "elements/s", "cores": threads, "kind": "oracle",
          "sample": f"first {k} of {NSEG_HEAD} segments ({nel} of {N_HEAD} elements) per step, {threads} threads",
          "host": {"os_cpu_count": os.cpu_count(), "affinity_cores": threads}}
    return {"metric": METRIC, "value": value, "unit": "elements/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "n": N_HEAD, "n_seg": NSEG_HEAD, "step_sample_elements": nel,
                       "parallelism": f"host, {threads} threads"},
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": "elements/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


# ----------------------------------------------------------------------------- main

def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        if rank != 0:
            return 0
        print(json.dumps(reference_arm(args)))
        return 0

    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2309_03912_b300 import binding as B
    from paper_2309_03912_b300 import build as Bd
    if not os.path.exists(B.LIB_PATH):
        Bd.build()
    B.lib()
    hbm_peak, tensor_peak, peak_src = peaks()
    stream = torch.cuda.Stream()

    if args.only:
        recs, checks = other_configs(args, stream, hbm_peak, tensor_peak)
        if not args.no_cpu:
            import oracle
            oracle.build()
            for name, e in check_configs(checks, oracle.host_threads()).items():
                recs[name]["error"] = e
        print(json.dumps({"configs": recs}))
        return 0
    h = headline(args, rank, world, stream)
    configs, checks = (None, {}) if (args.no_configs or rank != 0) else other_configs(args, stream, hbm_peak, tensor_peak)
    cb, err, cfg_err, check_s = None, None, {}, None
    if rank == 0 and world == 1 and not args.no_cpu:
        import oracle
        cb, err, cfg_err, check_s = cpu_leg(h, checks, oracle.host_threads())
        for name, e in cfg_err.items():
            configs[name]["error"] = e
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    if rank != 0:
        return 0

    ms_step = h["total_ms"] / args.steps
    kern_ms = statistics.mean(h["per_ms"])
    achieved = h["alg_bytes"] / (kern_ms * 1e-3) / 1e9
    traffic, traffic_n, sha = profile_traffic("k_segreduce", SEG_SOURCES)
    if traffic is not None and traffic_n:
        traffic = traffic * h["n"] / traffic_n
    line = {
        "metric": METRIC, "value": world * h["n"] / (ms_step * 1e-3), "unit": "elements/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "step_ms": {"min": round(min(h["per_ms"]), 5), "median": round(statistics.median(h["per_ms"]), 5),
                    "max": round(max(h["per_ms"]), 5)},
        "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": h["n"], "n_seg": h["nseg"], "map": "rational 6/6",
                   "l2": "inputs (1 GiB) larger than L2 (126 MB); no flush", "parallelism": f"replicas x{world}"},
        "hbm_gbs": round(achieved, 1), "frac_of_8tbs": round(achieved / NOMINAL_HBM_GBS, 4),
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm_peak, "unit": "GB/s",
                     "frac": round(achieved / hbm_peak, 4), "traffic": traffic, "peak_source": peak_src,
                     "kernel": "k_segreduce_tma<float, Rational<float,6,6>> (timed with the small k_join_cut "
                               "launch that follows it: one tr_segmented_reduce call)",
                     "alg_bytes_per_launch": h["alg_bytes"],
                     "kernel_ms": round(kern_ms, 5), "source_sha": sha},
        "e2e": {"value": world * h["n"] / (h["e2e_ms"] * 1e-3), "unit": "elements/s",
                "h2d_bytes_per_step": h["h2d"], "d2h_bytes_per_step": h["d2h"],
                "call": "tr_segmented_reduce_host (page-locked host buffers; copies enqueued by the library call)"},
        "error": err,
        "gpu_launches": h["launches"],
        "clocks": h["clocks"],
        "cpu_baseline": cb,
        "oracle_check_seconds": round(check_s, 1) if check_s is not None else None,
        "configs": configs,
    }
    print(json.dumps(line))
    return 0


if __name__ == "__main__":
    sys.exit(main())
