"""GPU parity of the reduced-precision search (tensor-core rate GEMM + FP32
refinement of the best coarse delay cells per segment) against the FP64 oracle.

* The rate GEMM itself (volks_check_rate_gemm): every accumulator column of
  one 128-cell block equals the DFT of Sec. 2.2's rate axis evaluated in
  FP64 from operands rounded to the operand type (BF16 / FP16 round to
  nearest even, E4M3 round to nearest even with saturation at 448), within
  the FP32 accumulation bound 1e-5 * sum |terms|.  This pins the operand
  layouts, descriptors and instruction shapes.
* Searches: the reported peak power is an FP32 evaluation of a real grid
  cell, so it must match the oracle's peak within the FP32 bound (relative
  1e-4) and sit at the oracle's cell, except (a) FP64 near-ties, as for the
  FP32 path, and (b) "coarse misses", where the oracle's peak delay cell was
  not among the 8 the coarse pass ranked highest: there the reported cell's
  FP64 power must equal the reported power (relative 1e-4) and lie within
  the coarse bound COARSE_REL of the oracle's peak.  Misses are counted and
  must stay rare (they need near-ties at the operand precision).
* The noise-free tests also use window 2 (a GEMM window) and window 1 (FP32).
"""
import math
import zlib

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import volks_oracle as O
from paper_2108_05602_b300 import build, synth
from paper_2108_05602_b300 import volks as V
from test_gpu_parity import P_REL, TIE_REL, Z_TOL, cell_power, exempt_pairs, gpu_search, make_data

pytestmark = pytest.mark.gpu

PRECS = {"bf16": V.VOLKS_BF16, "fp16": V.VOLKS_FP16, "fp8": V.VOLKS_FP8}
# bound on the relative error of a coarse |Z|^2 at a segment peak
COARSE_REL = {V.VOLKS_BF16: 3e-2, V.VOLKS_FP16: 5e-3, V.VOLKS_FP8: 0.3}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    V.lib()


# ---------------------------------------------------- operand rounding ----
def round_bf16(x):
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def round_fp16(x):
    return np.asarray(x, dtype=np.float32).astype(np.float16).astype(np.float64)


def round_e4m3(x):
    x = np.asarray(x, dtype=np.float32).astype(np.float64)
    a = np.abs(x)
    e = np.floor(np.log2(np.where(a > 0, a, 1.0)))
    spacing = np.exp2(np.maximum(e, -6.0) - 3.0)
    r = np.round(a / spacing) * spacing
    return np.sign(x) * np.minimum(r, 448.0)


ROUND = {V.VOLKS_BF16: round_bf16, V.VOLKS_FP16: round_fp16, V.VOLKS_FP8: round_e4m3}


def rate_gemm_reference(y, w, prec):
    """FP64 accumulator block from rounded operands: (value, sum |terms|)."""
    rnd = ROUND[prec]
    R = 4 * w
    a, b = rnd(y.real), rnd(y.imag)                    # [32][128]
    x = np.arange(R)[:, None] * np.arange(w)[None, :] % R     # [q][u]
    ang = 2.0 * np.pi * (x * (128 // R)) / 128.0
    c = rnd(np.cos(ang).astype(np.float32))
    sn = rnd(-(-np.sin(ang)).astype(np.float32))
    out = np.zeros((128, 256))
    mag = np.zeros((128, 256))
    for s in range(32 // w):
        A = a[s * w:(s + 1) * w].T                       # [128][w]
        B = b[s * w:(s + 1) * w].T
        re = A @ c.T + B @ sn.T                          # [128][R]
        im = -(A @ sn.T) + B @ c.T
        mre = np.abs(A) @ np.abs(c).T + np.abs(B) @ np.abs(sn).T
        mim = np.abs(A) @ np.abs(sn).T + np.abs(B) @ np.abs(c).T
        base = 8 * w * s
        out[:, base:base + 2 * R:2], out[:, base + 1:base + 2 * R:2] = re, im
        mag[:, base:base + 2 * R:2], mag[:, base + 1:base + 2 * R:2] = mre, mim
    return out, mag


@pytest.mark.parametrize("w", [2, 4, 8, 16, 32])
@pytest.mark.parametrize("pname", list(PRECS))
def test_rate_gemm_matches_rounded_operands(pname, w):
    prec = PRECS[pname]
    rng = np.random.default_rng(100 + w)
    scale = 2.0 if prec == V.VOLKS_FP8 else 8.0
    y = (rng.standard_normal((32, 128)) + 1j * rng.standard_normal((32, 128))) * scale
    y = y.astype(np.complex64)
    yd = torch.from_numpy(y).cuda()
    out = torch.full((128, 256), float("nan"), dtype=torch.float32, device="cuda")
    V.volks_check_rate_gemm(yd.data_ptr(), w, prec, out.data_ptr())
    got = out.cpu().numpy().astype(np.float64)
    want, mag = rate_gemm_reference(y.astype(np.complex128), w, prec)
    assert np.all(np.isfinite(got))
    err = np.abs(got - want)
    assert np.all(err <= 1e-5 * mag + 1e-30), float(np.max(err / np.maximum(mag, 1e-30)))


def test_bounded_wait_times_out_and_context_survives():
    """No MMA is issued, so the kernel's bounded wait on the tensor cores runs
    out: the call reports VOLKS_ETIMEOUT and the context still works."""
    y = torch.zeros((32, 128), dtype=torch.complex64, device="cuda")
    out = torch.zeros((128, 256), dtype=torch.float32, device="cuda")
    with pytest.raises(V.VolksError) as e:
        V.volks_check_rate_gemm(y.data_ptr(), 8, V.VOLKS_BF16, out.data_ptr(),
                                flags=V.VOLKS_CHECK_SKIP_MMA)
    assert e.value.code == V.VOLKS_ETIMEOUT
    y.normal_()
    V.volks_check_rate_gemm(y.data_ptr(), 8, V.VOLKS_BF16, out.data_ptr())
    assert torch.isfinite(out).all()
    torch.cuda.synchronize()


def test_unknown_check_arguments_rejected():
    y = torch.zeros((32, 128), dtype=torch.complex64, device="cuda")
    out = torch.zeros((128, 256), dtype=torch.float32, device="cuda")
    for w, p, f in [(1, V.VOLKS_BF16, 0), (64, V.VOLKS_BF16, 0), (8, V.VOLKS_FP32, 0), (8, V.VOLKS_BF16, 4)]:
        with pytest.raises(V.VolksError) as e:
            V.volks_check_rate_gemm(y.data_ptr(), w, p, out.data_ptr(), flags=f)
        assert e.value.code == V.VOLKS_EINVAL


# ------------------------------------------------------------- searches ----
def check_peaks_prec(wl, g, ref, vis, cal, prec):
    """Every segment of every series; returns (segments, FP64 ties, coarse misses)."""
    n = ties = misses = 0
    Ycache = {}

    def Y(b, d):
        if (b, d) not in Ycache:
            X = O.calibrate(vis[b], None if cal is None else cal[b], wl.n_if, wl.n_chan,
                            wl.chan_bw_mhz)
            Ycache[(b, d)] = O.delay_transform(O.dedisperse(X, ref.shifts[d]), wl.pad_delay)
        return Ycache[(b, d)]

    for (b, d, w), pk in ref.peaks.items():
        wi = list(wl.windows).index(w)
        P, q, m = g.peaks(b, d, wi)
        assert len(P) == len(pk.P), (b, d, w)
        n += len(P)
        for s in np.nonzero((q != pk.q) | (m != pk.m))[0]:
            gap = (pk.P[s] - pk.P2[s]) / max(pk.P[s], 1e-300)
            pc = cell_power(Y(b, d), w, wl.pad_rate, s, q[s], m[s])
            assert math.isclose(P[s], pc, rel_tol=P_REL), ((b, d, w, s), P[s], pc)
            if gap < TIE_REL:
                assert pc >= (1 - TIE_REL) * pk.P[s]
                ties += 1
            else:
                assert pc >= (1 - COARSE_REL[prec]) * pk.P[s], ((b, d, w, s), pc, pk.P[s])
                misses += 1
        same = (q == pk.q) & (m == pk.m)
        if np.any(same):
            np.testing.assert_allclose(P[same], pk.P[same], rtol=P_REL, atol=1e-30)
    return n, ties, misses


def check_candidates_prec(wl, g, ref):
    cg, co = g.candidates(), ref.matched
    ex = exempt_pairs(wl, ref)
    key = lambda c: (c["bl"], c["dm_idx"], c["win"], c["seg"], c.get("g0_ap", c.get("g0")),
                     c.get("g1_ap", c.get("g1")), c["n_windows"])
    kg = {key(c): c for c in cg if (c["bl"], c["dm_idx"]) not in ex}
    ko = {key(c): c for c in co if (c["bl"], c["dm_idx"]) not in ex}
    assert set(kg) == set(ko)
    for k, c in ko.items():
        assert math.isclose(kg[k]["peak_power"], c["peak_power"], rel_tol=P_REL)
        assert abs(kg[k]["z"] - c["z"]) <= Z_TOL * max(1.0, abs(c["z"]))
    return len(ko)


CONFIGS = [
    dict(name="nf256_w1-32", n_bl=1, n_ap=300, n_if=8, n_chan=32, n_dm=4, dm_step=15.0,
         windows=(1, 2, 4, 8, 16, 32)),
    dict(name="nf512_w1-32", n_bl=1, n_ap=161, n_if=8, n_chan=64, n_dm=4, dm_step=30.0,
         windows=(1, 2, 4, 8, 16, 32)),
    dict(name="nf512_w4", n_bl=2, n_ap=133, n_if=8, n_chan=64, n_dm=2, dm_step=30.0, windows=(4,)),
    dict(name="nf512_w8-32", n_bl=1, n_ap=150, n_if=8, n_chan=64, n_dm=3, dm_step=30.0, windows=(8, 32)),
    dict(name="nf512_w1-2", n_bl=1, n_ap=120, n_if=8, n_chan=64, n_dm=2, dm_step=30.0, windows=(1, 2)),
    dict(name="nf512_w1", n_bl=1, n_ap=90, n_if=8, n_chan=64, n_dm=2, dm_step=30.0, windows=(1,)),
    dict(name="nf256_w2-4", n_bl=2, n_ap=77, n_if=8, n_chan=32, n_dm=2, dm_step=30.0, windows=(2, 4)),
    dict(name="nf1024_w2-32", n_bl=1, n_ap=140, n_if=8, n_chan=128, n_dm=3, dm_step=40.0,
         windows=(2, 4, 8, 16, 32)),
    dict(name="nf2048_w2-32", n_bl=1, n_ap=100, n_if=16, n_chan=128, n_dm=2, dm_step=40.0,
         windows=(2, 8, 32)),
    # DM trials 400 and 800 shift the band by more than its 40 APs: no valid AP
    dict(name="nf256_nvalid0", n_bl=1, n_ap=40, n_if=8, n_chan=32, n_dm=3, dm_step=400.0,
         windows=(1, 4, 32)),
]


@pytest.mark.parametrize("pname", list(PRECS))
@pytest.mark.parametrize("cfg", CONFIGS, ids=[c["name"] for c in CONFIGS])
def test_search_matches_oracle(cfg, pname):
    prec = PRECS[pname]
    cfg = dict(cfg)
    name = cfg.pop("name")
    wl = synth.small(**cfg, name=name, min_baselines=1)
    vis, cal, _ = make_data(wl, seed=(zlib.crc32(name.encode()) + 17) % 1000)
    g = gpu_search(wl, vis, cal, precision=prec)
    ref = O.search(wl, vis, cal)
    n, ties, misses = check_peaks_prec(wl, g, ref, vis, cal, prec)
    assert n == sum(len(p.P) for p in ref.peaks.values())
    assert misses <= max(1, n // 20000), (misses, n)
    check_candidates_prec(wl, g, ref)
    g.close()


@pytest.mark.parametrize("pname", list(PRECS))
def test_pr1_reduced_precision(pname):
    prec = PRECS[pname]
    wl, vis, cal, pulses = synth.gen_pr1(seed=1)
    g = gpu_search(wl, vis, cal, precision=prec)
    ref = O.search(wl, vis, cal)
    n, ties, misses = check_peaks_prec(wl, g, ref, vis, cal, prec)
    assert n == 61090
    assert misses <= 3, misses
    check_candidates_prec(wl, g, ref)
    t0 = pulses[0].t0_ap
    hits = [c for c in g.candidates() if abs(c["dm"] - 50) <= 3 and c["g0_ap"] <= t0 + 2
            and c["g1_ap"] >= t0]
    assert hits and max(hits, key=lambda c: c["z"])["n_windows"] >= 2
    g.close()


def test_noise_free_on_grid_pulse_exact_cell():
    """Noise-free on-grid pulse: exact cell and the analytic power (a w N_f)^2,
    as for the FP32 path (n_f = 256, so the tensor-core kernel runs)."""
    wl = synth.small(n_bl=1, n_ap=64, n_if=8, n_chan=32, n_dm=1, windows=(8, 16, 32))
    M = 4 * wl.n_f
    for prec in PRECS.values():
        for w, wi in ((8, 0), (16, 1), (32, 2)):
            m0, q0 = 301, 3 * w // 2
            p = synth.Pulse(0.0, 32 - w if w < 32 else 0, w, 6.0,
                            np.array([m0 / (M * wl.chan_bw_mhz * 1e6)]),
                            np.array([q0 / (4 * w * wl.t_ap_s)]))
            vis = np.zeros((1, wl.n_ap, wl.n_f), dtype=np.complex64)
            synth.inject(vis, wl, np.zeros((1, wl.n_if, 2)), [p])
            g = gpu_search(wl, vis, None, normalize_chan=0, precision=prec)
            P, q, m = g.peaks(0, 0, wi)
            s = p.t0_ap // w
            a = 6.0 * math.sqrt(2.0 / (w * wl.n_f))
            assert (q[s], m[s]) == (q0, m0), (prec, w)
            assert math.isclose(P[s], (a * w * wl.n_f) ** 2, rel_tol=1e-5), (prec, w)
            g.close()


def test_all_zero_input_ties_to_cell_zero():
    wl = synth.small(n_bl=1, n_ap=100, n_if=8, n_chan=64, windows=(1, 2, 4, 8, 16, 32))
    vis = np.zeros((1, wl.n_ap, wl.n_f), dtype=np.complex64)
    g = gpu_search(wl, vis, None, precision=V.VOLKS_BF16)
    for d in range(wl.n_dm):
        for wi in range(len(wl.windows)):
            P, q, m = g.peaks(0, d, wi)
            assert np.all(P == 0) and np.all(q == 0) and np.all(m == 0)
    assert g.candidates() == []


def test_fp32_fallback_for_1d_and_small_bands():
    """1-D searches, bands under 256 points and sliding segments (stride 1)
    run the FP32 kernel whatever precision is asked: results equal the FP32
    search bit for bit."""
    for kw in (dict(n_if=4, n_chan=32, pad_rate=4, stride=0), dict(n_if=8, n_chan=32, pad_rate=0, stride=0),
               dict(n_if=8, n_chan=64, pad_rate=4, stride=1)):
        import dataclasses
        wl = synth.small(n_bl=1, n_ap=150, n_if=kw["n_if"], n_chan=kw["n_chan"], n_dm=2,
                         windows=(1, 4, 16))
        wl = dataclasses.replace(wl, pad_rate=kw["pad_rate"], stride=kw["stride"])
        vis, cal, _ = make_data(wl, seed=4)
        a = gpu_search(wl, vis, cal)
        b = gpu_search(wl, vis, cal, precision=V.VOLKS_BF16)
        for d in range(wl.n_dm):
            for wi in range(len(wl.windows)):
                for x, y in zip(a.peaks(0, d, wi), b.peaks(0, d, wi)):
                    assert np.array_equal(x, y)


@pytest.mark.parametrize("pname", ["fp32"] + list(PRECS))
def test_power_of_two_input_scale_commutes(pname):
    """Without channel normalisation, multiplying the input by 2^k scales
    every FP32 intermediate by 2^k exactly, so the FP32 search returns the
    same cells with powers scaled by 2^2k.  The FP16 / FP8 forms scale each
    tile's operands by a power of two chosen from its largest component, so
    their rounded operands, coarse passes and candidates are the same too;
    at 2^20 unscaled E4M3 operands (largest finite 448) would saturate."""
    prec = {"fp32": V.VOLKS_FP32, **PRECS}[pname]
    wl = synth.small(n_bl=1, n_ap=160, n_if=8, n_chan=64, n_dm=2, dm_step=30.0,
                     windows=(1, 2, 4, 8, 16, 32))
    vis, cal, _ = make_data(wl, seed=11)
    ref = gpu_search(wl, vis, cal, normalize_chan=0, precision=prec)
    for k in (20, -20):
        g = gpu_search(wl, (vis * np.float32(2.0 ** k)).astype(np.complex64), cal, normalize_chan=0,
                       precision=prec)
        for d in range(wl.n_dm):
            for wi in range(len(wl.windows)):
                P0, q0, m0 = ref.peaks(0, d, wi)
                P1, q1, m1 = g.peaks(0, d, wi)
                assert np.array_equal(q1, q0) and np.array_equal(m1, m0), (k, d, wi)
                assert np.array_equal(P1, (P0 * np.float32(2.0 ** (2 * k))).astype(np.float32)), (k, d, wi)
        c0, c1 = ref.candidates(), g.candidates()
        assert [(c["bl"], c["dm_idx"], c["win"], c["seg"]) for c in c1] == \
               [(c["bl"], c["dm_idx"], c["win"], c["seg"]) for c in c0]
        for a, b in zip(c0, c1):
            assert math.isclose(b["z"], a["z"], rel_tol=1e-12, abs_tol=1e-12)
        g.close()
    ref.close()


def test_deterministic_bitwise():
    wl = synth.small(n_bl=1, n_ap=200, n_if=8, n_chan=64, n_dm=3, dm_step=20.0,
                     windows=(1, 2, 4, 8, 16, 32))
    vis, cal, _ = make_data(wl, seed=9)
    runs = [gpu_search(wl, vis, cal, precision=V.VOLKS_BF16) for _ in range(2)]
    for d in range(wl.n_dm):
        for wi in range(len(wl.windows)):
            for x, y in zip(runs[0].peaks(0, d, wi), runs[1].peaks(0, d, wi)):
                assert np.array_equal(x, y)
    assert runs[0].candidates() == runs[1].candidates()


# ------------------------------------------------- plans, server, full size ----
def test_plan_with_reduced_precision_matches_oracle():
    """A batch plan whose band classes mix tensor-core (n_f >= 256, 2-D) and
    FP32 segments at precision BF16: every segment against the oracle."""
    shapes = [
        dict(n_bl=2, n_ap=190, n_if=8, n_chan=32, n_dm=3, dm_step=20.0, windows=(1, 2, 4, 8, 16, 32)),
        dict(n_bl=1, n_ap=170, n_if=8, n_chan=64, n_dm=3, dm_step=25.0, windows=(1, 4, 16)),
        dict(n_bl=1, n_ap=120, n_if=8, n_chan=128, n_dm=2, dm_step=30.0, windows=(2, 8, 32)),
        dict(n_bl=2, n_ap=210, n_if=4, n_chan=16, n_dm=4, dm_step=40.0, windows=(1, 2, 4, 8)),
    ]
    items = []
    for i, sh in enumerate(shapes):
        wl = synth.small(**sh, name=f"pmix{i}", min_baselines=1)
        vis, cal, _ = make_data(wl, seed=400 + i)
        items.append((wl, vis, cal))
    dev = [torch.from_numpy(v).cuda() for _, v, _ in items]
    plan = V.Plan([(wl, d, cal) for (wl, _, cal), d in zip(items, dev)], graph=True, autotune=True,
                  precision=V.VOLKS_BF16)
    plan.run(stream=torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    for i, (wl, vis, cal) in enumerate(items):
        ref = O.search(wl, vis, cal)
        r = plan.result(i)
        n, ties, misses = check_peaks_prec(wl, r, ref, vis, cal, V.VOLKS_BF16)
        assert misses <= 1
        check_candidates_prec(wl, r, ref)
    plan.close()


def test_server_reduced_precision_alone_equals_mix():
    """BF16 requests: each result in the continuous-batching mix equals the
    same search run alone, bit for bit (deterministic kernels)."""
    reqs = []
    for i in range(6):
        wl = synth.small(n_bl=1 + i % 2, n_ap=140 + 29 * i, n_if=8, n_chan=32 << (i % 2), n_dm=3,
                         dm_step=30.0, windows=(1, 2, 4, 8, 16, 32), min_baselines=1, name=f"preq{i}")
        vis, cal, _ = make_data(wl, seed=500 + i)
        reqs.append((wl, vis, cal))
    alone = []
    for wl, vis, cal in reqs:
        s = V.Search(wl, torch.from_numpy(vis).cuda(), cal, precision=V.VOLKS_BF16)
        alone.append(s.candidates())
        s.close()
    srv = V.Server(max_inflight=3, hbm_budget_bytes=8 << 30)
    devs = [torch.from_numpy(v).cuda() for _, v, _ in reqs]
    ids = [srv.submit(wl, d, cal, precision=V.VOLKS_BF16) for (wl, _, cal), d in zip(reqs, devs)]
    for i, rid in enumerate(ids):
        info, got = srv.wait_all(rid)
        assert info.status == 0
        assert got == alone[i]
    srv.close()


def test_evn_full_size_bf16_sampled_parity():
    """The EVN-scale scan (15 baselines x 58,594 APs x 512 points, 501 DM
    trials, windows 1..32) searched at BF16 in the benchmark's launch
    configuration: sampled segments against the oracle one by one, and the
    whole candidate list and sampled series against the FP32 search."""
    wl, vis_t, cal, pulses = synth.gen_evn_torch(seed=2)
    stream = torch.cuda.current_stream().cuda_stream
    g16 = V.Search(wl, vis_t, cal, stream=stream, precision=V.VOLKS_BF16)
    c16 = g16.candidates()
    g32 = V.Search(wl, vis_t, cal, stream=stream)
    c32 = g32.candidates()
    key = lambda c: (c["bl"], c["dm_idx"], c["win"], c["seg"], c["g0_ap"], c["g1_ap"], c["n_windows"])
    k16, k32 = {key(c): c for c in c16}, {key(c): c for c in c32}
    # a candidate can differ only through a coarse miss moving a series'
    # statistics across a decision boundary: allow a handful in ~5e4
    diff = set(k16) ^ set(k32)
    assert len(diff) <= max(2, len(k32) // 1000), (len(diff), len(k32))
    rng = np.random.default_rng(1)
    shifts, _ = g16.shifts()
    n_cmp = n_same = 0
    for _ in range(12):
        b, d = int(rng.integers(0, wl.n_bl)), int(rng.integers(0, wl.n_dm))
        for wi in range(len(wl.windows)):
            P16, q16, m16 = g16.peaks(b, d, wi)
            P32, q32, m32 = g32.peaks(b, d, wi)
            same = (q16 == q32) & (m16 == m32)
            n_cmp += len(P16)
            n_same += int(same.sum())
            np.testing.assert_allclose(P16[same], P32[same], rtol=1e-5)
    assert n_same >= n_cmp - max(3, n_cmp // 20000), (n_same, n_cmp)
    # sampled segments against the FP64 oracle
    for p in pulses[:3]:
        b = int(rng.integers(0, wl.n_bl))
        d = int(np.argmin(np.abs(wl.dms() - p.dm)))
        Sb = vis_t[b].cpu().numpy()
        X = O.calibrate(Sb, cal[b], wl.n_if, wl.n_chan, wl.chan_bw_mhz)
        lo = (p.t0_ap // 32) * 32
        Y = O.delay_transform(O.dedisperse(X, shifts[d])[lo:lo + 64], wl.pad_delay)
        for wi, w in enumerate(wl.windows):
            P, q, m = g16.peaks(b, d, wi)
            pk = O.window_peaks(Y, w, wl.pad_rate)
            s0 = lo // w
            for j in range(min(len(pk.P), len(P) - s0)):
                s = s0 + j
                assert math.isclose(P[s], pk.P[j], rel_tol=P_REL), (b, d, w, s)
                if (pk.P[j] - pk.P2[j]) / pk.P[j] >= TIE_REL:
                    assert (q[s], m[s]) == (pk.q[j], pk.m[j]), (b, d, w, s)
    g16.close()
    g32.close()
