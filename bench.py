"""Benchmark: fringe-fit trials/s of the cross-spectrum single-pulse search.

One step = the whole hot path (dedispersion shift table, FP64 channel
normalisation, calibration, dedispersion, delay FFT, window/rate FFTs, peak
search, FP64 series statistics + threshold, window match, host
cross-baseline match) over one EVN-scale scan segment: 15 baselines x
58,594 APs x 512 frequency points (3.6 GB complex64, larger than L2),
501 DM trials 0..1000, windows 1..32 AP, delay pad 4, rate pad 4, FP32.
A trial is one (baseline, DM trial, window, segment) fringe fit.

The default single-GPU run also times, on the same scan, the reduced-
precision forms (the rate transform of the 4..32-AP windows as a BF16,
FP16 or FP8 tensor-core DFT GEMM with FP32 re-evaluation), states their
error per candidate against the FP64 oracle for a sample of candidates, and
summarises the batched form (64 heterogeneous segments in one plan) and the
serving form (a Poisson request stream through the continuous-batching
server).

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Under torchrun each rank searches its own scan (weak scaling, no collective
on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fringe-fit trials/sec (baseline x DM x window x segment), EVN-scale scan"
UNIT = "trials/s"
FP32_LANES = 128  # FP32 FMA lanes per SM (sm_100 family)


def _evn_1bl_32dm(synth):
    import dataclasses
    return dataclasses.replace(synth.evn(), n_bl=1, n_dm=32)


def _band_1bl(n_chan):
    # one baseline of 20,000 APs with the EVN scan's 8 IFs widened to
    # n_chan channels each (1024 or 2048 points: folded delay transforms),
    # 16 DM trials over 0..937.5
    def make(synth):
        import dataclasses
        return dataclasses.replace(synth.evn(), n_bl=1, n_ap=20000, n_chan=n_chan, n_dm=16, dm_step=1000.0 / 16)
    return make


WORKLOADS = {
    # the EVN-scale scan the metric is quoted on
    "evn_fp32": lambda synth: synth.evn(),
    # the same scan with the rate transform of the 4..32-AP windows as a
    # tensor-core DFT GEMM (BF16 / FP16 / FP8 E4M3) + FP32 re-evaluation
    "evn_bf16": lambda synth: synth.evn(),
    "evn_fp16": lambda synth: synth.evn(),
    "evn_fp8": lambda synth: synth.evn(),
    # profiling cases: one baseline of the same scan (240 MB, larger than L2), 32 DM trials
    "evn_1bl_32dm": _evn_1bl_32dm,
    "evn_1bl_32dm_bf16": _evn_1bl_32dm,
    "evn_1bl_32dm_fp16": _evn_1bl_32dm,
    "evn_1bl_32dm_fp8": _evn_1bl_32dm,
    # profiling cases of the large band classes (FOLD 2 and 4)
    "band1024_1bl": _band_1bl(128),
    "band2048_1bl": _band_1bl(256),
}
# volks_params.precision of each workload (VOLKS_FP32 = 0, BF16 = 1, FP16 = 2, FP8 = 3)
PRECISION = {"evn_bf16": 1, "evn_fp16": 2, "evn_fp8": 3, "evn_1bl_32dm_bf16": 1, "evn_1bl_32dm_fp16": 2,
             "evn_1bl_32dm_fp8": 3}
PREC_NAMES = {"fp32": 0, "bf16": 1, "fp16": 2, "fp8": 3}
DTYPE = {0: "f32", 1: "bf16 rate GEMM + f32", 2: "f16 rate GEMM + f32", 3: "e4m3 rate GEMM + f32"}

# The batching recipe (64 heterogeneous segments) with durations and DM
# grids scaled so that one step takes ~10 s (the recipe's 5-120 s segments
# and 0-2000 DM ranges at step 2 would take minutes per step).
BATCH = dict(n_seg=64, dur_s=(2.0, 4.0), max_dm_trials=96)
# The serving recipe's request mix scaled the same way (1-3 s, <= 32 DM trials).
SERVING = dict(n=16, dur_s=(1.0, 3.0), max_dm_trials=32)


def workload(name="evn_fp32"):
    from paper_2108_05602_b300 import synth
    return WORKLOADS[name](synth)


def workload_config(name, wl, trials):
    """The `config` object both arms report for a scan workload."""
    return {"workload": name, "n_bl": wl.n_bl, "n_ap": wl.n_ap, "n_if": wl.n_if, "n_chan": wl.n_chan,
            "n_dm": wl.n_dm, "dm": [wl.dm_lo, wl.dm_lo + wl.dm_step * (wl.n_dm - 1)],
            "windows": list(wl.windows), "pad_delay": wl.pad_delay, "pad_rate": wl.pad_rate,
            "trials_per_step": trials, "input_bytes": wl.n_bl * wl.n_ap * wl.n_f * 8,
            "l2": f"inputs larger than L2 ({wl.n_bl * wl.n_ap * wl.n_f * 8 / 1e9:.2f} GB per step)"
            if wl.n_bl * wl.n_ap * wl.n_f * 8 > (126 << 20) else "inputs smaller than L2"}


def trial_count(wl, nvalid) -> int:
    n = 0
    for nv in nvalid:
        nv = max(int(nv), 0)
        n += sum(nv // w for w in wl.windows)
    return n * wl.n_bl


def algorithmic_flops(wl, nvalid) -> float:
    """Nominal flops of one search: 5 N log2 N per complex N-point FFT
    (delay transform of each dedispersed AP over M = 4 N_f points; rate
    transform of each segment's delay column over R = 4 w points), 3 per
    |Z|^2 cell, 2 (w - 1) per coherent sum when R = 1."""
    M = wl.pad_delay * wl.n_f
    tot = 0.0
    for nv in nvalid:
        nv = max(int(nv), 0)
        tot += nv * 5.0 * M * math.log2(M)
        for w in wl.windows:
            ns = nv // w
            R = 1 if (w == 1 or wl.pad_rate == 0) else wl.pad_rate * w
            if R > 1:
                tot += ns * M * 5.0 * R * math.log2(R)
            elif w > 1:
                tot += ns * M * 2.0 * (w - 1)
            tot += ns * R * M * 3.0
    return tot * wl.n_bl


def mma_flops(wl, nvalid, precision) -> float:
    """Executed tensor-core flops (2 per multiply-add, zero blocks of the
    block-diagonal operands included) of one reduced-precision search: per
    (baseline, DM trial, searched 32-AP tile, delay residue, 128-cell block)
    and window w in 4..32, M = 128 rows x N columns x K of the window's
    MMAs."""
    if precision == 0 or wl.pad_rate != 4 or wl.n_f < 256:
        return 0.0
    eb = 1 if precision == 3 else 2
    per_block = 0.0
    for w in wl.windows:
        if w < 4:
            continue
        seg_kb = 2 * w * eb
        if seg_kb >= 32:
            per_block += (32 // w) * 2.0 * 128 * (8 * w) * (2 * w)
        else:
            g = 32 // seg_kb
            per_block += (32 // w) // g * 2.0 * 128 * (8 * w * g) * (32 // eb)
    tiles = sum((max(int(v), 0) + 31) // 32 for v in nvalid)
    blocks_per_tile = wl.pad_delay * wl.n_f // 128   # residues x blocks = M / 128
    return per_block * tiles * blocks_per_tile * wl.n_bl


def cuda_core_flops_mma(wl, nvalid) -> float:
    """Nominal CUDA-core flops of one search on the tensor-core kernel: the
    FP32 delay transform and the 1- and 2-AP windows as in
    algorithmic_flops; for the GEMM windows (4..32 APs), 3 per coarse
    |Z|^2 cell (square, add, max) plus the FP32 refinement of at most 8
    delay cells per segment and delay-residue unit (5 R log2 R + 3 R each,
    counted at 8)."""
    M = wl.pad_delay * wl.n_f
    fold = max(1, wl.n_f // 512)
    units_per_seg = wl.pad_delay * fold
    tot = 0.0
    for nv in nvalid:
        nv = max(int(nv), 0)
        tot += nv * 5.0 * M * math.log2(M)
        for w in wl.windows:
            ns = nv // w
            R = 1 if w == 1 else 4 * w
            if w == 1:
                tot += ns * M * 3.0
            elif w == 2:
                tot += ns * M * (5.0 * R * math.log2(R) + 3.0 * R)
            else:
                tot += ns * (R * M * 3.0 + 8 * units_per_seg * (5.0 * R * math.log2(R) + 3.0 * R))
    return tot * wl.n_bl


TRAFFIC_FILE = "search_kernel_traffic.json"
# sources of the kernels whose committed DRAM capture bench.py scales
KERNEL_SOURCES = ("search_kernel.cuh", "search_common.cuh", "fft_regs.cuh", "twiddle_ce.h", "volks_internal.h")


def kernel_source_hash(files=KERNEL_SOURCES) -> str:
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2108_05602_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def fp32_peak_tflops(peaks, n_sm) -> tuple:
    """Derived FP32 FMA peak: SMs x 128 lanes x 2 flops x the measured
    maximum SM clock."""
    mhz = float(peaks.get("sm_max_mhz", 2032.0))
    return n_sm * FP32_LANES * 2 * mhz * 1e6 / 1e12, mhz


_bench_lib = None


def measured_fp32_tflops(stream: int = 0) -> float:
    """FP32 FMA throughput measured by the benchmark's probe kernel
    (libvolks_bench.so, a helper library only the benchmark loads)."""
    global _bench_lib
    if _bench_lib is None:
        from paper_2108_05602_b300 import build as B
        B.build()
        _bench_lib = ctypes.CDLL(B.BENCH_LIB)
        _bench_lib.bench_fp32_fma_tflops.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]
        _bench_lib.bench_fp32_fma_tflops.restype = ctypes.c_int
    t = ctypes.c_double()
    rc = _bench_lib.bench_fp32_fma_tflops(ctypes.c_void_p(stream), ctypes.byref(t))
    if rc != 0:
        raise RuntimeError(f"FP32 FMA probe failed (CUDA error {rc})")
    return t.value


def traffic_per_launch(wl, trials):
    """DRAM bytes (read + write) of one search-kernel launch, scaled from
    the committed capture of the one-baseline, 32-DM case: reads follow the
    input (each baseline's visibilities are read once, whatever the number
    of DM trials), writes follow the trials (one 8-byte key each).  None if
    there is no capture for the current kernel source."""
    try:
        with open(os.path.join(ROOT, "profiles", TRAFFIC_FILE)) as f:
            t = json.load(f)
    except OSError:
        return None
    if t.get("kernel_hash") != kernel_source_hash():
        return None
    if wl.n_ap * wl.n_f * 8 != t["input_bytes"] // t["n_bl"]:
        return None  # another baseline shape (band class): the capture does not apply
    reads = t["dram_read_bytes"] * wl.n_bl / t["n_bl"]
    writes = t["dram_write_bytes"] * trials / t["trials"]
    return {"bytes": reads + writes, "read": reads, "write": writes,
            "basis": f"ncu DRAM counters of one launch on {t['workload']} (1 pass), reads scaled by "
                     f"baselines ({wl.n_bl}/{t['n_bl']}), writes by trials"}


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        rows = []
        for line in (self.out or "").strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), smax=float(parts[2]), pw=float(parts[3]),
                                 hw=parts[5], hwt=parts[6], swt=parts[7], pcap=parts[8]))
            except ValueError:
                continue
        if not rows:
            return None
        load = [r for r in rows if r["pw"] > 300] or rows
        reasons = set()
        for r in rows:
            for k, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                            ("swt", "sw_thermal_slowdown"), ("pcap", "sw_power_cap")):
                if r[k].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in load),
                "sm_max_mhz": max(r["smax"] for r in rows), "samples": len(rows),
                "samples_under_load": len(load), "reasons": sorted(reasons)}


# ----------------------------------------------------------- oracle leg ----
def _oracle_one(args):
    wl, vis, cal, d = args
    from oracle import volks_oracle as O
    res = O.search(wl, vis, cal, with_second=False, dm_indices=[d])
    return sum(len(p.P) for p in res.peaks.values())


def oracle_sample(wl, vis_b, cal_b, n_ap, dm_indices, cores):
    """Time the FP64 oracle, as it stands, on one baseline x the given DM
    trials x the first n_ap APs, one process per DM trial (spawned)."""
    import dataclasses
    import multiprocessing as mp
    sub = dataclasses.replace(wl, n_bl=1, n_ap=n_ap)
    vis = np.ascontiguousarray(vis_b[None, :n_ap])
    cal = cal_b[None]
    ctx = mp.get_context("spawn")
    with ctx.Pool(processes=cores) as pool:
        pool.map(_oracle_one, [(sub, vis[:, :64], cal, 0)])  # start-up outside the clock
        t = time.perf_counter()
        n = sum(pool.map(_oracle_one, [(sub, vis, cal, d) for d in dm_indices]))
        dt = time.perf_counter() - t
    return n, dt


def error_vs_oracle(wl, vis_t, cal, forms_cands, baselines=(0, 1), max_list=32):
    """Part of the CPU leg: the FP64 oracle's peak for every candidate that
    each search form reports on the given baselines (the sample), against
    the reported peak power and cell.  Per form: the sample size, the
    largest and median relative power error, the number of identical peak
    cells, and the first max_list candidates one by one as [baseline, DM
    index, window, segment, relative power error, cell identical]."""
    from oracle import volks_oracle as O
    sh = O.shift_table(wl.f_lo_mhz, wl.chan_bw_mhz, wl.n_f, wl.dms(), wl.t_ap_s)
    M = wl.pad_delay * wl.n_f
    k = np.arange(wl.n_f)
    Xc = {}
    out = {}
    t0 = time.perf_counter()
    for name, cands in forms_cands.items():
        sample = sorted((c for c in cands if c["bl"] in baselines),
                        key=lambda c: (c["bl"], c["dm_idx"], c["win"], c["seg"]))
        rel, same, rows = [], 0, []
        for c in sample:
            b, d, w, sg = c["bl"], c["dm_idx"], c["win"], c["seg"]
            if b not in Xc:
                Xc[b] = O.calibrate(vis_t[b].cpu().numpy(), cal[b], wl.n_if, wl.n_chan, wl.chan_bw_mhz)
            t = np.arange(sg * w, (sg + 1) * w)
            Xd = Xc[b][t[:, None] + sh[d][None, :], k[None, :]]   # the segment's dedispersed APs
            pk = O.window_peaks(O.delay_transform(Xd, wl.pad_delay), w, wl.pad_rate)
            R = O.rate_len(w, wl.pad_rate)
            e = abs(c["peak_power"] - pk.P[0]) / pk.P[0]
            eq = (c["rate_idx"] % R, c["delay_idx"] % M) == (int(pk.q[0]), int(pk.m[0]))
            rel.append(e)
            same += int(eq)
            if len(rows) < max_list:
                rows.append([b, d, w, sg, e, bool(eq)])
        srt = sorted(rel)
        out[name] = {"candidates": len(sample), "max_rel_power_error": srt[-1] if srt else None,
                     "median_rel_power_error": srt[len(srt) // 2] if srt else None,
                     "peak_cell_equal": same, "per_candidate": rows}
    out["sample"] = (f"every candidate each form reports on baselines {list(baselines)} of the last step; "
                     "oracle: FP64 numpy on the segment's dedispersed APs")
    out["cpu_s"] = time.perf_counter() - t0
    return out


def batch_summary(steps, warmup, precisions=("fp32", "bf16")):
    """The batched form: 64 heterogeneous segments (the batching recipe,
    scaled as BATCH says) searched by one plan per precision (persistent
    launches per band class, one CUDA graph, autotuned work splits) against
    the plain path that searches the same segments one by one in FP32."""
    import torch
    from paper_2108_05602_b300 import synth
    from paper_2108_05602_b300 import volks as V
    wls = synth.batch_workloads(**BATCH)
    items, trials, flops_seg = [], 0, []
    for i, wl in enumerate(wls):
        vis, cal, _ = synth.gen_segment_torch(wl, seed=1000 + i)
        items.append((wl, vis, cal))
        _, nv = V.volks_shift_table(wl.f_lo_mhz, wl.chan_bw_mhz, wl.n_f, wl.t_ap_s, wl.n_ap,
                                    wl.dm_lo, wl.dm_step, wl.n_dm)
        trials += trial_count(wl, nv)
        flops_seg.append(algorithmic_flops(wl, nv))
    stream = torch.cuda.current_stream()
    sptr = stream.cuda_stream
    kms_seg = [0.0] * len(items)

    def plain_step():
        out = [V.Search(wl, vis, cal, stream=sptr) for wl, vis, cal in items]
        n = sum(len(s.candidates()) for s in out)
        for i, s in enumerate(out):
            kms_seg[i] = s.timing().ms_search
            s.close()
        return n, sum(kms_seg)

    def timed(fn):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = [fn() for _ in range(steps)]
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps, res

    peaks = measured_peaks()
    peak, _ = fp32_peak_tflops(peaks, torch.cuda.get_device_properties(0).multi_processor_count)
    t_plain, r_plain = timed(plain_step)
    classes = {}
    for i, (wl, _, _) in enumerate(items):
        c = classes.setdefault(wl.n_f, [0.0, 0.0, 0])
        c[0] += flops_seg[i]
        c[1] += kms_seg[i]
        c[2] += 1
    out = {"segments": len(items), "trials_per_step": trials,
           "input_bytes": sum(wl.n_bl * wl.n_ap * wl.n_f * 8 for wl in wls),
           "recipe": f"batching recipe with durations U{list(BATCH['dur_s'])} s and at most "
                     f"{BATCH['max_dm_trials']} DM trials per segment (DM ranges 0..U(200, 2000))",
           "n_f": sorted(classes), "steps": steps, "warmup": warmup,
           "plain_fp32": {"value": trials / (t_plain / 1e3), "unit": UNIT, "ms_per_step": t_plain,
                          "candidates": r_plain[-1][0]},
           "roofline_by_band_fp32": {str(nf): {"frac": c[0] / (c[1] / 1e3) / 1e12 / peak, "segments": c[2]}
                                     for nf, c in sorted(classes.items())}}
    for pname in precisions:
        prec = PREC_NAMES[pname]
        t0 = time.perf_counter()
        plan = V.Plan(items, autotune=True, graph=True, precision=prec)
        create_s = time.perf_counter() - t0

        def plan_step():
            plan.run(stream=sptr)
            n = sum(len(plan.result(i).candidates()) for i in range(len(items)))
            return n, plan.timing().ms_search

        t_plan, r_plan = timed(plan_step)
        info = plan.info()
        out["plan_" + pname] = {"value": trials / (t_plan / 1e3), "unit": UNIT, "ms_per_step": t_plan,
                                "vs_plain_fp32": t_plain / t_plan, "kernel_ms": statistics.mean(r[1] for r in r_plan),
                                "candidates": r_plan[-1][0], "search_launches_per_step": info["search_launches"],
                                "plan_create_s": create_s, "gpu_launches": plan.timing().n_launches}
        plan.close()
    del items
    torch.cuda.empty_cache()
    return out


def serving_summary(precisions=("fp32", "bf16"), rate_hz=20.0, duration_s=20.0, slo_ms=500.0):
    """The serving form: a Poisson stream (seeded) of search requests
    through the continuous-batching server; p50/p99 latency and completed
    trials/s at rate_hz for each precision, and for each precision the
    largest rate of a x1.25 sweep whose p99 stays within slo_ms with the
    trials/s completed at that rate."""
    import torch
    from paper_2108_05602_b300 import synth
    from paper_2108_05602_b300 import volks as V
    wls = synth.serving_workloads(**SERVING)
    pool = []
    for i, wl in enumerate(wls):
        vis, cal, _ = synth.gen_segment_torch(wl, seed=2000 + i)
        pool.append((wl, vis, cal))
    torch.cuda.synchronize()
    srv = V.Server(max_inflight=8, hbm_budget_bytes=120 << 30)
    out = {"requests_pool": len(pool), "rate_hz": rate_hz, "duration_s": duration_s,
           "recipe": f"serving recipe with durations U{list(SERVING['dur_s'])} s and at most "
                     f"{SERVING['max_dm_trials']} DM trials (DM ranges 0..U(200, 1500)), 3-15 baselines",
           "max_inflight": 8, "hbm_budget_bytes": 120 << 30, "p99_objective_ms": slo_ms}
    for pname in precisions:
        prec = PREC_NAMES[pname]
        for wl, vis, cal in pool[:2]:
            srv.wait(srv.submit(wl, vis, cal, precision=prec))
        trials, span, p50, p99, n = serve_once(V, srv, pool, rate_hz, duration_s, seed=5, prec=prec)
        out[pname] = {"p50_ms": p50, "p99_ms": p99, "trials_per_s": trials / span, "requests": n}
    for pname in precisions:
        prec = PREC_NAMES[pname]
        sweep, best = [], (rate_hz if out[pname]["p99_ms"] <= slo_ms else None)
        best_tps = out[pname]["trials_per_s"] if best else None
        rate = rate_hz
        for _ in range(5):
            rate *= 1.25
            tr, sp, a, b, m = serve_once(V, srv, pool, rate, 8.0, seed=int(rate), prec=prec)
            sweep.append({"rate_hz": rate, "p50_ms": a, "p99_ms": b, "trials_per_s": tr / sp, "requests": m})
            if b > slo_ms:
                break
            best, best_tps = rate, tr / sp
        out[pname]["sweep"] = sweep
        out[pname]["max_sustained_rate_hz"] = best
        out[pname]["max_sustained_trials_per_s"] = best_tps
    st = srv.stats()
    srv.close()
    if "fp32" in out and "bf16" in out and out["fp32"].get("max_sustained_trials_per_s"):
        out["bf16_vs_fp32_sustained"] = (out["bf16"]["max_sustained_trials_per_s"] or 0.0) / \
            out["fp32"]["max_sustained_trials_per_s"]
    out["server"] = {"peak_inflight": st.peak_inflight, "peak_bytes": st.peak_bytes, "completed": st.completed,
                     "failed": st.failed}
    del pool
    torch.cuda.empty_cache()
    return out


def run_reference(args):
    """The FP64 oracle, as it stands, on the host cores: each step is a
    bounded sample of the EVN-scale workload (1 baseline x 8 DM trials x
    5 s), the value is trials/s of that sample; the line carries the same
    config as the GPU arm."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle import volks_oracle as O
    from paper_2108_05602_b300 import synth
    wl = workload()
    sh = O.shift_table(wl.f_lo_mhz, wl.chan_bw_mhz, wl.n_f, wl.dms(), wl.t_ap_s)
    trials_full = trial_count(wl, [O.n_valid(wl.n_ap, r) for r in sh])
    cores = min(8, os.cpu_count() or 1)
    n_ap = 4883  # 5 s of the scan
    dms = list(range(0, wl.n_dm, wl.n_dm // cores))[:cores]
    wl_s, vis, cal, _ = synth.gen_evn_numpy(seed=2, wl=wl, n_ap=n_ap, n_pulses=1)
    for _ in range(args.warmup):
        oracle_sample(wl, vis[0], cal[0], n_ap, dms[:1], 1)
    times, n = [], 0
    for _ in range(args.steps):
        n, dt = oracle_sample(wl, vis[0], cal[0], n_ap, dms, cores)
        times.append(dt)
    value = n / statistics.mean(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.mean(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config("evn_fp32", wl, trials_full),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"each step: 1 baseline x {len(dms)} DM trials x {n_ap} APs "
                                       f"(5 s) of this workload, {n} trials, FP64 numpy, one spawned "
                                       "process per DM trial"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def serve_once(V, srv, pool, rate_hz, duration_s, seed, prec=0):
    """Submit pool requests at Poisson times; return (completed trials,
    span s, p50 ms, p99 ms, peak inflight, n requests)."""
    arr = None
    from paper_2108_05602_b300 import synth
    arr = synth.poisson_arrivals(rate_hz, duration_s, seed=seed)
    t0 = time.perf_counter()
    ids = []
    for i, ta in enumerate(arr):
        dt = ta - (time.perf_counter() - t0)
        if dt > 0:
            time.sleep(dt)
        wl, vis, cal = pool[i % len(pool)]
        ids.append(srv.submit(wl, vis, cal, precision=prec))
    lat, trials = [], 0
    for rid in ids:
        info, _ = srv.wait(rid)
        lat.append(info.latency_ms)
        trials += info.trials
    span = time.perf_counter() - t0
    lat.sort()
    pct = lambda p: lat[min(len(lat) - 1, int(round(p * (len(lat) - 1))))] if lat else 0.0
    return trials, span, pct(0.5), pct(0.99), len(ids)


# -------------------------------------------------------------- GPU leg ----
def run_volks(args):
    import torch
    import torch.distributed as dist
    from paper_2108_05602_b300 import build as B
    from paper_2108_05602_b300 import shard, synth
    from paper_2108_05602_b300 import volks as V

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    B.build()
    V.lib()
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    wl = workload(args.workload)
    prec = PRECISION.get(args.workload, 0)
    wl, vis, cal, pulses = synth.gen_evn_torch(seed=2 + rank, device="cuda", wl=wl)
    vis = vis.contiguous()
    stream = torch.cuda.current_stream()
    sptr = stream.cuda_stream
    _, nvalid = V.volks_shift_table(wl.f_lo_mhz, wl.chan_bw_mhz, wl.n_f, wl.t_ap_s, wl.n_ap,
                                    wl.dm_lo, wl.dm_step, wl.n_dm)
    trials = trial_count(wl, nvalid)
    flops = algorithmic_flops(wl, nvalid)

    def step(x, pv=prec):
        s = V.Search(wl, x, cal, stream=sptr, precision=pv)
        c = s.candidates()          # waits for the device, runs the host match
        t = s.timing()
        s.close()
        return c, t

    def barrier():
        if world > 1:
            dist.barrier()

    for _ in range(max(args.warmup, 0)):
        step(vis)
    torch.cuda.synchronize()
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    step_ms, search_ms, launches = [], [], 0
    cands = []
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        barrier()
        ev0.record(stream)
        for _ in range(args.steps):
            e_a, e_b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e_a.record(stream)
            cands, tm = step(vis)
            e_b.record(stream)
            e_b.synchronize()
            step_ms.append(e_a.elapsed_time(e_b))
            search_ms.append(tm.ms_search)
            launches += tm.n_launches
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
    total_ms = ev0.elapsed_time(ev1)
    n_all, t_max_s = shard.reduce_step(trials * args.steps, total_ms / 1e3, device="cuda")
    value = n_all / t_max_s

    # end to end through the public API with host (pinned) input: the 3.6 GB
    # host-to-device copy and the candidate read-back are inside the clock
    host = vis.cpu().pin_memory()
    e2e_steps = max(1, min(args.steps, 3))
    step(host)
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    n_c = 0
    for _ in range(e2e_steps):
        c, _ = step(host)
        n_c += len(c)
    torch.cuda.synchronize()
    barrier()
    e2e_s = time.perf_counter() - t0
    _, e2e_max = shard.reduce_step(0.0, e2e_s, device="cuda")
    e2e_value = n_all / args.steps * e2e_steps / e2e_max
    del host

    single = world == 1 and args.workload == "evn_fp32"
    # the reduced-precision forms of the same search on the same scan (N = 1
    # only): 1 warm-up + 2 timed steps each, CUDA events on the stream
    forms, forms_cands = None, {"fp32": cands}
    if prec == 0 and single and not args.no_forms:
        forms = {}
        ref_keys = {(c["bl"], c["dm_idx"], c["win"], c["seg"], c["g0_ap"], c["g1_ap"]) for c in cands}
        with ClockSampler(local) as fclk:
            for name in ("bf16", "fp16", "fp8"):
                pv = PREC_NAMES[name]
                step(vis, pv)
                torch.cuda.synchronize()
                fa, fb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                fa.record(stream)
                kms, fc = [], []
                for _ in range(2):
                    fc, tm = step(vis, pv)
                    kms.append(tm.ms_search)
                fb.record(stream)
                torch.cuda.synchronize()
                fms = fa.elapsed_time(fb) / 2
                keys = {(c["bl"], c["dm_idx"], c["win"], c["seg"], c["g0_ap"], c["g1_ap"]) for c in fc}
                mk = statistics.mean(kms)
                forms_cands[name] = fc
                forms[name] = {"value": trials / (fms / 1e3), "unit": UNIT, "ms_per_step": fms,
                               "kernel_ms": mk, "vs_fp32": (trials / (fms / 1e3)) / value,
                               "kernel_vs_fp32": statistics.mean(search_ms) / mk,
                               "tensor_tflops": mma_flops(wl, nvalid, pv) / (mk / 1e3) / 1e12,
                               "candidates": len(fc),
                               "candidates_differing_from_fp32": len(keys ^ ref_keys)}
        forms["clocks"] = fclk.summary()

    if rank == 0:
        peaks = measured_peaks()
        peak, mhz = fp32_peak_tflops(peaks, n_sm)
        try:
            fma_meas = measured_fp32_tflops(sptr)
        except Exception:
            fma_meas = None
        ms_k = statistics.mean(search_ms)
        achieved = flops / (ms_k / 1e3) / 1e12
        traffic = traffic_per_launch(wl, trials)
        cpu = None
        err = None
        if not args.no_cpu_baseline:
            err = error_vs_oracle(wl, vis, cal, forms_cands)
            cores = min(8, os.cpu_count() or 1)
            n_ap = 9766  # 10 s of the scan
            dms = list(range(0, wl.n_dm, wl.n_dm // cores))[:cores]
            vb = vis[0, :n_ap].cpu().numpy()
            n, dt = oracle_sample(wl, vb, cal[0], n_ap, dms, cores)
            cpu = {"value": n / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": f"1 baseline x {len(dms)} DM trials x {n_ap} APs (10 s) of this "
                             f"workload, FP64 numpy, {n} trials in {dt:.1f} s"}
        srt = sorted(step_ms)
        basis = (f"FP32 FMA: {n_sm} SMs (device) x {FP32_LANES} lanes x 2 x {mhz:.0f} MHz "
                 "(max SM clock, MEASURED_PEAKS.json)")
        if prec == 0:
            roofline = {"bound": "alu", "kernel": f"search_kernel<16,4,{max(1, wl.n_f // 512)}>"
                        if wl.n_f >= 512 else "search_kernel",
                        "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                        "frac": achieved / peak, "traffic": traffic["bytes"] if traffic else None,
                        "traffic_basis": traffic["basis"] if traffic else None,
                        "algorithmic_bytes": wl.n_bl * wl.n_ap * wl.n_f * 8 + 8 * trials,
                        "peak_basis": basis, "peak_measured_fma": fma_meas,
                        "frac_of_measured_fma": achieved / fma_meas if fma_meas else None,
                        "kernel_ms": ms_k, "algorithmic_flops": flops}
        else:
            alu = cuda_core_flops_mma(wl, nvalid)
            mma = mma_flops(wl, nvalid, prec)
            tpeak = float(peaks.get("bf16_tflops", 1817.4)) * (2.0 if prec == 3 else 1.0)
            roofline = {"bound": "alu", "kernel": f"search_mma_kernel<16,1,{prec}>",
                        "achieved": alu / (ms_k / 1e3) / 1e12, "peak": peak, "unit": "TFLOP/s",
                        "frac": alu / (ms_k / 1e3) / 1e12 / peak, "traffic": None,
                        "peak_basis": basis, "peak_measured_fma": fma_meas, "kernel_ms": ms_k,
                        "algorithmic_flops": alu, "fft_form_flops": flops, "fft_form_tflops": achieved,
                        "tensor": {"achieved": mma / (ms_k / 1e3) / 1e12, "peak": tpeak,
                                   "unit": "TFLOP/s", "frac": mma / (ms_k / 1e3) / 1e12 / tpeak,
                                   "executed_mma_flops": mma,
                                   "peak_basis": "measured bf16 burst (MEASURED_PEAKS.json)"
                                                 + (" x 2 (fp8/bf16 nominal ratio)" if prec == 3 else "")}}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t_max_s * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[prec],
            "data": "synthetic: complex64 N(0,1) noise + 20 dispersed pulses + station RFI",
            "config": dict(workload_config(args.workload, wl, trials),
                           step_ms_p50=srt[len(srt) // 2], step_ms_p99=srt[-1]),
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "steps": e2e_steps,
                    "h2d_bytes_per_step": wl.n_bl * wl.n_ap * wl.n_f * 8,
                    "d2h_bytes_per_step": 4 + n_c // e2e_steps * 96},
            "gpu_launches": launches,
            "clocks": clk.summary(),
            "candidates_per_step": len(cands),
        }
        if forms is not None:
            line["precision_forms"] = forms
        if err is not None:
            line["error_vs_oracle"] = err
        if single and not args.no_batch:
            del vis
            torch.cuda.empty_cache()
            with ClockSampler(local) as bclk:
                line["batch64"] = batch_summary(steps=1, warmup=1)
            line["batch64"]["clocks"] = bclk.summary()
        if single and not args.no_serving:
            with ClockSampler(local) as sclk:
                line["serving"] = serving_summary()
            line["serving"]["clocks"] = sclk.summary()
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_batch(args):
    """--workload batch64: the batched form alone, as its own JSON line."""
    import torch
    from paper_2108_05602_b300 import build as B
    from paper_2108_05602_b300 import volks as V
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    B.build()
    V.lib()
    precs = ("fp32", args.precision) if args.precision != "fp32" else ("fp32",)
    with ClockSampler(local) as clk:
        s = batch_summary(args.steps, args.warmup, precisions=precs)
    main = s["plan_" + args.precision]
    line = {"metric": METRIC.replace("EVN-scale scan", "64-segment heterogeneous batch"),
            "value": main["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": main["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": DTYPE[PREC_NAMES[args.precision]],
            "data": "synthetic: complex64 N(0,1) noise + 0-3 dispersed pulses per segment",
            "config": {"workload": "batch64", "l2": "inputs larger than L2"}, "batch64": s,
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    return 0


def run_serving(args):
    """--workload serving: the serving form alone, as its own JSON line."""
    import torch
    from paper_2108_05602_b300 import build as B
    from paper_2108_05602_b300 import volks as V
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    B.build()
    V.lib()
    precs = ("fp32", args.precision) if args.precision != "fp32" else ("fp32",)
    with ClockSampler(local) as clk:
        s = serving_summary(precisions=precs, duration_s=30.0)
    main = s[args.precision]
    line = {"metric": "fringe-fit trials/sec under a Poisson request stream; p50/p99 latency",
            "value": main["trials_per_s"], "unit": UNIT, "n_gpus": 1, "steps": 1, "warmup": args.warmup,
            "ms_per_step": 30.0e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE[PREC_NAMES[args.precision]],
            "data": "synthetic: 16 request shapes, complex64 noise + 0-3 pulses each",
            "config": {"workload": "serving"}, "latency_ms": {"p50": main["p50_ms"], "p99": main["p99_ms"]},
            "serving": s, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="volks", choices=["volks", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true",
                    help="skip the CPU legs (oracle timing and per-candidate oracle errors)")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the reduced-precision forms in the default EVN run")
    ap.add_argument("--no-batch", action="store_true", help="skip the batch64 summary in the default run")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving summary in the default run")
    ap.add_argument("--workload", default="evn_fp32", choices=sorted(WORKLOADS) + ["batch64", "serving"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16", "fp16", "fp8"],
                    help="rate-search arithmetic of the batch64 plan and the serving requests")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch64":
        return run_batch(args)
    if args.workload == "serving":
        return run_serving(args)
    return run_volks(args)


if __name__ == "__main__":
    sys.exit(main())
