"""Benchmark: fringe-fit trials/s of the cross-spectrum single-pulse search.

One step = the whole hot path (dedispersion shift table, FP64 channel
normalisation, calibration, dedispersion, delay FFT, window/rate FFTs, peak
search, FP64 series statistics + threshold, window match, host
cross-baseline match) over one EVN-scale scan segment: 15 baselines x
58,594 APs x 512 frequency points (3.6 GB complex64, larger than L2),
501 DM trials 0..1000, windows 1..32 AP, delay pad 4, rate pad 4, FP32.
A trial is one (baseline, DM trial, window, segment) fringe fit.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Under torchrun each rank searches its own scan (weak scaling, no collective
on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
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
SM_COUNT, FP32_LANES = 148, 128


WORKLOADS = {
    # the EVN-scale scan the metric is quoted on
    "evn_fp32": lambda synth: synth.evn(),
    # the same scan with the rate transform of the 4..32-AP windows as a
    # tensor-core DFT GEMM (BF16 / FP16 / FP8 E4M3) + FP32 top-8 refinement
    "evn_bf16": lambda synth: synth.evn(),
    "evn_fp16": lambda synth: synth.evn(),
    "evn_fp8": lambda synth: synth.evn(),
    # profiling cases: one baseline of the same scan (240 MB, larger than L2), 32 DM trials
    "evn_1bl_32dm": lambda synth: __import__("dataclasses").replace(synth.evn(), n_bl=1, n_dm=32),
    "evn_1bl_32dm_bf16": lambda synth: __import__("dataclasses").replace(synth.evn(), n_bl=1, n_dm=32),
    "evn_1bl_32dm_fp8": lambda synth: __import__("dataclasses").replace(synth.evn(), n_bl=1, n_dm=32),
}
# volks_params.precision of each workload (VOLKS_FP32 = 0, BF16 = 1, FP16 = 2, FP8 = 3)
PRECISION = {"evn_bf16": 1, "evn_fp16": 2, "evn_fp8": 3, "evn_1bl_32dm_bf16": 1, "evn_1bl_32dm_fp8": 3}
PREC_NAMES = {"fp32": 0, "bf16": 1, "fp16": 2, "fp8": 3}
DTYPE = {0: "f32", 1: "bf16 rate GEMM + f32", 2: "f16 rate GEMM + f32", 3: "e4m3 rate GEMM + f32"}


BATCH = dict(n_seg=64, dur_s=(3.0, 6.0), max_dm_trials=128)


def workload(name="evn_fp32"):
    from paper_2108_05602_b300 import synth
    return WORKLOADS[name](synth)


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


KERNEL_SOURCES = {
    # the FP32 search kernel and the tensor-core search kernel: sources whose
    # change invalidates a committed DRAM-traffic capture
    "search_kernel_traffic.json": ("search_kernel.cuh", "search_common.cuh", "fft_regs.cuh", "twiddle_ce.h",
                                   "volks_internal.h"),
    "search_mma_kernel_traffic.json": ("volks_mma.cu", "tcgen05.cuh", "search_common.cuh", "fft_regs.cuh",
                                       "twiddle_ce.h", "volks_internal.h"),
}


def kernel_source_hash(files) -> str:
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


def fp32_peak_tflops(peaks) -> tuple:
    mhz = float(peaks.get("sm_max_mhz", 2032.0))
    return SM_COUNT * FP32_LANES * 2 * mhz * 1e6 / 1e12, mhz


def traffic_per_launch(workload_name):
    """DRAM bytes (read + write) of one search-kernel launch from a committed
    full-size ncu capture, or None if there is none for this workload and
    the current kernel source."""
    for name, files in KERNEL_SOURCES.items():
        try:
            with open(os.path.join(ROOT, "profiles", name)) as f:
                t = json.load(f)
        except OSError:
            continue
        if t.get("workload") == workload_name and t.get("kernel_hash") == kernel_source_hash(files):
            return t["dram_bytes_per_launch"]
    return None


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


def oracle_error_sample(wl, vis_t, cal, cands, n=16):
    """Part of the CPU leg: the FP64 oracle's peak for the segments of the n
    highest-z candidates, against the reported peak power and cell (error
    of the reduced-precision search per candidate)."""
    from oracle import volks_oracle as O
    from paper_2108_05602_b300 import volks as V
    sh, _ = V.volks_shift_table(wl.f_lo_mhz, wl.chan_bw_mhz, wl.n_f, wl.t_ap_s, wl.n_ap,
                                wl.dm_lo, wl.dm_step, wl.n_dm)
    top = sorted(cands, key=lambda c: -c["z"])[:n]
    M = wl.pad_delay * wl.n_f
    rel, same, Xc = [], 0, {}
    for c in top:
        b, d, w, sg = c["bl"], c["dm_idx"], c["win"], c["seg"]
        if b not in Xc:
            Xc[b] = O.calibrate(vis_t[b].cpu().numpy(), cal[b], wl.n_if, wl.n_chan, wl.chan_bw_mhz)
        Xd = O.dedisperse(Xc[b], sh[d])[sg * w:(sg + 1) * w]
        pk = O.window_peaks(O.delay_transform(Xd, wl.pad_delay), w, wl.pad_rate)
        rel.append(abs(c["peak_power"] - pk.P[0]) / pk.P[0])
        R = 1 if (w == 1 or wl.pad_rate == 0) else wl.pad_rate * w
        q = c["rate_idx"] % R
        m = c["delay_idx"] % M
        same += int((q, m) == (int(pk.q[0]), int(pk.m[0])))
    rel.sort()
    return {"candidates": len(top), "max_rel_power_error": rel[-1] if rel else None,
            "median_rel_power_error": rel[len(rel) // 2] if rel else None,
            "peak_cell_equal": same, "sample": "the 16 highest-z candidates of the last step"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_2108_05602_b300 import synth
    wl = workload()
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
            "config": {"workload": "evn_sample", "n_bl": 1, "n_ap": n_ap, "n_dm": len(dms),
                       "n_f": wl.n_f, "windows": list(wl.windows)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"1 baseline x {len(dms)} DM trials x {n_ap} APs "
                                       "(5 s) of the EVN-scale workload, FP64 numpy"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


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
    units = int(sum(max(int(v), 0) for v in nvalid)) * wl.n_bl  # dedispersed APs x (b, d)

    def step(x):
        s = V.Search(wl, x, cal, stream=sptr, precision=prec)
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

    # end to end through the public API with host (pinned) input
    host = vis.cpu().pin_memory()
    e2e_steps = max(1, args.steps)
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

    # the reduced-precision forms of the same search on the same scan (N = 1
    # only): 1 warm-up + 2 timed steps each, CUDA events on the stream
    forms = None
    if prec == 0 and world == 1 and not args.no_forms and args.workload == "evn_fp32":
        forms = {}
        ref_keys = {(c["bl"], c["dm_idx"], c["win"], c["seg"], c["g0_ap"], c["g1_ap"]) for c in cands}
        for name, pv in (("bf16", 1), ("fp8", 3)):
            def fstep(x, pv=pv):
                s = V.Search(wl, x, cal, stream=sptr, precision=pv)
                c = s.candidates()
                t = s.timing()
                s.close()
                return c, t
            fstep(vis)
            torch.cuda.synchronize()
            fa, fb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            fa.record(stream)
            kms, fc = [], []
            for _ in range(2):
                fc, tm = fstep(vis)
                kms.append(tm.ms_search)
            fb.record(stream)
            torch.cuda.synchronize()
            fms = fa.elapsed_time(fb) / 2
            keys = {(c["bl"], c["dm_idx"], c["win"], c["seg"], c["g0_ap"], c["g1_ap"]) for c in fc}
            mk = statistics.mean(kms)
            forms[name] = {"value": trials / (fms / 1e3), "unit": UNIT, "ms_per_step": fms,
                           "kernel_ms": mk, "vs_fp32": (trials / (fms / 1e3)) / value,
                           "tensor_tflops": mma_flops(wl, nvalid, pv) / (mk / 1e3) / 1e12,
                           "candidates": len(fc),
                           "candidates_differing_from_fp32": len(keys ^ ref_keys)}

    if rank == 0:
        peaks = measured_peaks()
        peak, mhz = fp32_peak_tflops(peaks)
        ms_k = statistics.mean(search_ms)
        achieved = flops / (ms_k / 1e3) / 1e12
        traffic = traffic_per_launch(args.workload)
        cpu = None
        err = None
        if not args.no_cpu_baseline and prec != 0:
            err = oracle_error_sample(wl, vis, cal, cands, n=16)
        if not args.no_cpu_baseline:
            cores = min(8, os.cpu_count() or 1)
            n_ap = 9766  # 10 s of the scan
            dms = list(range(0, wl.n_dm, wl.n_dm // cores))[:cores]
            vb = vis[0, :n_ap].cpu().numpy()
            n, dt = oracle_sample(wl, vb, cal[0], n_ap, dms, cores)
            cpu = {"value": n / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": f"1 baseline x {len(dms)} DM trials x {n_ap} APs (10 s) of this "
                             f"workload, FP64 numpy, {n} trials in {dt:.1f} s"}
        srt = sorted(step_ms)
        basis = (f"FP32 FMA: {SM_COUNT} SMs x {FP32_LANES} lanes x 2 x {mhz:.0f} MHz "
                 "(max SM clock, MEASURED_PEAKS.json)")
        if prec == 0:
            roofline = {"bound": "alu", "kernel": "search_kernel<16,4>",
                        "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                        "frac": achieved / peak, "traffic": traffic, "peak_basis": basis,
                        "kernel_ms": ms_k, "algorithmic_flops": flops}
        else:
            alu = cuda_core_flops_mma(wl, nvalid)
            mma = mma_flops(wl, nvalid, prec)
            tpeak = float(peaks.get("bf16_tflops", 1817.4)) * (2.0 if prec == 3 else 1.0)
            roofline = {"bound": "alu", "kernel": f"search_mma_kernel<16,1,{prec}>",
                        "achieved": alu / (ms_k / 1e3) / 1e12, "peak": peak, "unit": "TFLOP/s",
                        "frac": alu / (ms_k / 1e3) / 1e12 / peak, "traffic": traffic,
                        "peak_basis": basis, "kernel_ms": ms_k, "algorithmic_flops": alu,
                        "fft_form_flops": flops, "fft_form_tflops": achieved,
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
            "config": {"workload": args.workload, "n_bl": wl.n_bl, "n_ap": wl.n_ap,
                       "n_if": wl.n_if, "n_chan": wl.n_chan, "n_dm": wl.n_dm,
                       "dm": [wl.dm_lo, wl.dm_lo + wl.dm_step * (wl.n_dm - 1)],
                       "windows": list(wl.windows), "pad_delay": wl.pad_delay,
                       "pad_rate": wl.pad_rate, "trials_per_step": trials,
                       "input_bytes": wl.n_bl * wl.n_ap * wl.n_f * 8,
                       "l2": "inputs larger than L2 (3.6 GB per step)",
                       "step_ms_p50": srt[len(srt) // 2], "step_ms_p99": srt[-1]},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT,
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
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_batch(args):
    """64 heterogeneous segments (the batching recipe) searched by one plan
    (persistent launches per band class, one CUDA graph, autotuned work
    splits) against the plain path that searches the same segments one by
    one with volks_search_segment."""
    import torch
    from paper_2108_05602_b300 import build as B
    from paper_2108_05602_b300 import synth
    from paper_2108_05602_b300 import volks as V

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    B.build()
    V.lib()
    wls = synth.batch_workloads(**BATCH)
    items, trials, flops = [], 0, 0.0
    for i, wl in enumerate(wls):
        vis, cal, _ = synth.gen_segment_torch(wl, seed=1000 + i)
        items.append((wl, vis, cal))
        _, nv = V.volks_shift_table(wl.f_lo_mhz, wl.chan_bw_mhz, wl.n_f, wl.t_ap_s, wl.n_ap,
                                    wl.dm_lo, wl.dm_step, wl.n_dm)
        trials += trial_count(wl, nv)
        flops += algorithmic_flops(wl, nv)
    stream = torch.cuda.current_stream()
    sptr = stream.cuda_stream

    def plain_step():
        out = []
        for wl, vis, cal in items:
            s = V.Search(wl, vis, cal, stream=sptr)
            out.append(s)
        n = sum(len(s.candidates()) for s in out)
        ms = sum(s.timing().ms_search for s in out)
        for s in out:
            s.close()
        return n, ms

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = [fn() for _ in range(steps)]
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps, res

    t_plain, r_plain = timed(plain_step, args.steps, args.warmup)
    prec = PREC_NAMES[args.precision]
    t0 = time.perf_counter()
    plan = V.Plan(items, autotune=True, graph=True, precision=prec)
    create_s = time.perf_counter() - t0

    def plan_step():
        plan.run(stream=sptr)
        n = sum(len(plan.result(i).candidates()) for i in range(len(items)))
        return n, plan.timing().ms_search

    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        t_plan, r_plan = timed(plan_step, args.steps, args.warmup)
    info = plan.info()
    tm = plan.timing()
    peaks = measured_peaks()
    peak, mhz = fp32_peak_tflops(peaks)
    ms_k = statistics.mean(r[1] for r in r_plan)
    line = {
        "metric": METRIC.replace("EVN-scale scan", "64-segment heterogeneous batch"),
        "value": trials / (t_plan / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_plan, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[prec],
        "data": "synthetic: complex64 N(0,1) noise + 0-3 dispersed pulses per segment",
        "config": {"workload": "batch64", "segments": len(items),
                   "n_f": sorted({wl.n_f for wl in wls}),
                   "n_bl": [min(wl.n_bl for wl in wls), max(wl.n_bl for wl in wls)],
                   "n_ap": [min(wl.n_ap for wl in wls), max(wl.n_ap for wl in wls)],
                   "n_dm": [min(wl.n_dm for wl in wls), max(wl.n_dm for wl in wls)],
                   "input_bytes": sum(wl.n_bl * wl.n_ap * wl.n_f * 8 for wl in wls),
                   "trials_per_step": trials, "plan_rounds": info["rounds"],
                   "search_launches_per_step": info["search_launches"],
                   "plan_create_s": create_s,
                   "l2": "inputs larger than L2"},
        "plain_fp32": {"value": trials / (t_plain / 1e3), "ms_per_step": t_plain,
                       "gpu_launches_per_step": 6 * len(items)},
        "speedup_vs_plain": t_plain / t_plan,
        "roofline": {"bound": "alu",
                     "kernel": "search_kernel (all band classes)" if prec == 0 else
                               "search_mma_kernel (n_f >= 256) + search_kernel (smaller bands)",
                     "achieved": flops / (ms_k / 1e3) / 1e12, "peak": peak, "unit": "TFLOP/s",
                     "frac": flops / (ms_k / 1e3) / 1e12 / peak, "traffic": None,
                     "kernel_ms": ms_k, "algorithmic_flops": flops,
                     "flops_basis": "nominal FFT-form flops of the search (same count for every precision)"},
        "gpu_launches": tm.n_launches,
        "clocks": clk.summary(),
        "candidates_per_step": r_plan[-1][0], "candidates_plain": r_plain[-1][0],
    }
    print(json.dumps(line), flush=True)
    plan.close()
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


def run_serving(args):
    """Poisson stream of search requests through the continuous-batching
    server: p50/p99 latency and throughput at 20 req/s, and the largest
    rate of a x1.25 sweep whose p99 stays within a 500 ms objective."""
    import torch
    from paper_2108_05602_b300 import build as B
    from paper_2108_05602_b300 import synth
    from paper_2108_05602_b300 import volks as V

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    B.build()
    V.lib()
    wls = synth.serving_workloads()
    pool = []
    for i, wl in enumerate(wls):
        vis, cal, _ = synth.gen_segment_torch(wl, seed=2000 + i)
        pool.append((wl, vis, cal))
    torch.cuda.synchronize()
    prec = PREC_NAMES[args.precision]
    srv = V.Server(max_inflight=8, hbm_budget_bytes=120 << 30)
    for wl, vis, cal in pool[: max(1, args.warmup)]:
        srv.wait(srv.submit(wl, vis, cal, precision=prec))
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        trials, span, p50, p99, n = serve_once(V, srv, pool, 20.0, 30.0, seed=5, prec=prec)
    sweep = []
    slo_ms = 500.0
    rate, best = 20.0, (20.0 if p99 <= slo_ms else None)
    for _ in range(4):
        rate *= 1.25
        tr, sp, a, b, m = serve_once(V, srv, pool, rate, 10.0, seed=int(rate), prec=prec)
        sweep.append({"rate_hz": rate, "p50_ms": a, "p99_ms": b, "trials_per_s": tr / sp, "requests": m})
        if b > slo_ms:
            break
        best = rate
    st = srv.stats()
    srv.close()
    line = {
        "metric": "fringe-fit trials/sec under a Poisson request stream; p50/p99 latency",
        "value": trials / span, "unit": UNIT, "n_gpus": 1, "steps": 1, "warmup": args.warmup,
        "ms_per_step": span * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPE[prec],
        "data": "synthetic: 16 request shapes, complex64 noise + 0-3 pulses each",
        "config": {"workload": "serving", "rate_hz": 20.0, "duration_s": 30.0, "requests": n,
                   "max_inflight": 8, "hbm_budget_bytes": 120 << 30,
                   "n_bl": [min(w.n_bl for w in wls), max(w.n_bl for w in wls)],
                   "n_f": sorted({w.n_f for w in wls}),
                   "n_ap": [min(w.n_ap for w in wls), max(w.n_ap for w in wls)],
                   "n_dm": [min(w.n_dm for w in wls), max(w.n_dm for w in wls)]},
        "latency_ms": {"p50": p50, "p99": p99},
        "sweep": sweep, "max_sustained_rate_hz": best, "p99_objective_ms": slo_ms,
        "server": {"peak_inflight": st.peak_inflight, "peak_bytes": st.peak_bytes,
                   "completed": st.completed, "failed": st.failed},
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="volks", choices=["volks", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the reduced-precision forms in the default EVN run")
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
