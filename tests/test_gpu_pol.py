"""Polarisation combine and the HOPS auto-spectrum normalisation on the GPU
(Fig. 1: products combined after the initial calibration; Sec. 2.2:
|s_ij| / (mean a_i^2 mean a_j^2)^(1/4)) against the FP64 oracle, with the
tolerances of the plain search (tests/test_gpu_parity.py)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import volks_oracle as O
from paper_2108_05602_b300 import build, synth
from paper_2108_05602_b300 import volks as V

from test_gpu_parity import check_candidates, check_peaks

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    V.lib()


def pulses_for(wl, rng, n=3, snr=(9.0, 16.0)):
    M = wl.pad_delay * wl.n_f
    out = []
    for _ in range(n):
        dm = float(wl.dms()[rng.integers(0, wl.n_dm)])
        W = int(rng.integers(1, 9))
        hi = wl.n_ap - int(synth.arrival_offsets_ap(wl, dm).max()) - W - 1
        if hi <= 1:
            continue
        m0 = rng.integers(-M // 2, M // 2, size=wl.n_bl)
        out.append(synth.Pulse(dm, int(rng.integers(0, hi)), W, float(rng.uniform(*snr)),
                               m0 / (M * wl.chan_bw_mhz * 1e6), rng.uniform(-50, 50, size=wl.n_bl)))
    return out


def search(wl, vis, cal, autos=None, bl_st=None, device=True, **over):
    t = torch.from_numpy(vis).cuda() if device else vis
    a = None if autos is None else (torch.from_numpy(autos).cuda() if device else autos)
    s = V.Search(wl, t, cal, stream=torch.cuda.current_stream().cuda_stream, autos=a, bl_st=bl_st,
                 **over)
    s._tensors = (t, a)
    return s


SHAPES = [dict(n_bl=3, n_ap=400, n_if=4, n_chan=16, n_dm=4, dm_step=40.0, windows=(1, 2, 4, 8)),
          dict(n_bl=6, n_ap=700, n_if=8, n_chan=32, n_dm=3, dm_step=60.0, windows=(2, 4, 8, 16)),
          dict(n_bl=2, n_ap=333, n_if=2, n_chan=128, n_dm=2, dm_step=25.0, windows=(4, 32))]


@pytest.mark.parametrize("shape", SHAPES, ids=["64pt", "256pt", "256pt-ragged"])
@pytest.mark.parametrize("mode", ["dual+autos", "dual+rms", "single+autos"])
def test_search_matches_oracle(shape, mode):
    wl = synth.small(**shape, min_baselines=1)
    rng = np.random.default_rng(len(mode) * 7 + shape["n_chan"])
    n_pol = 1 if mode.startswith("single") else 2
    vis, cal, autos, bl_st, _ = synth.dual_pol_scan(wl, rng, pulses_for(wl, rng), n_pol=n_pol)
    kw = dict(autos=autos, bl_st=bl_st) if mode.endswith("autos") else {}
    if n_pol == 1:
        vis, cal = vis[0], cal[0]
    g = search(wl, vis, cal, **kw)
    ref = O.search(wl, vis, cal, **kw)
    gains = g.gains()
    vis_p = vis if vis.ndim == 4 else vis[None]
    cal_p = cal if cal.ndim == 4 else cal[None]
    gains_p = gains if gains.ndim == 3 else gains[None]
    for p in range(vis_p.shape[0]):
        for b in range(wl.n_bl):
            norm = (O.auto_norm(autos[p, bl_st[b, 0]], autos[p, bl_st[b, 1]]) if kw
                    else 1.0 / O.chan_rms(vis_p[p, b]))
            want = O.calib_phasor(cal_p[p, b], wl.n_if, wl.n_chan, wl.chan_bw_mhz) * norm
            np.testing.assert_allclose(gains_p[p, b], want, rtol=1e-6)
    n, _ = check_peaks(wl, g, ref, vis, cal, **kw)
    assert n == sum(len(p.P) for p in ref.peaks.values())
    check_candidates(wl, g, ref, matched=True)
    g.close()


def test_dual_polarisation_pulse_is_found():
    wl = synth.small(n_bl=6, n_ap=600, n_if=8, n_chan=32, n_dm=3, dm_step=50.0, windows=(2, 4, 8, 16),
                     min_baselines=3)
    rng = np.random.default_rng(5)
    M = 4 * wl.n_f
    p = synth.Pulse(50.0, 300, 4, 12.0, rng.integers(-M // 2, M // 2, size=wl.n_bl) / (M * wl.chan_bw_mhz * 1e6),
                    np.zeros(wl.n_bl))
    vis, cal, autos, bl_st, _ = synth.dual_pol_scan(wl, rng, [p])
    g = search(wl, vis, cal, autos=autos, bl_st=bl_st)
    cands = g.candidates()
    hit = [c for c in cands if c["dm_idx"] == 1 and c["g0_ap"] <= 304 and c["g1_ap"] >= 300]
    assert len({c["bl"] for c in hit}) == wl.n_bl
    g.close()


def test_host_input_equals_device_input_bitwise():
    wl = synth.small(n_bl=3, n_ap=300, n_if=4, n_chan=64, n_dm=3, dm_step=30.0, min_baselines=1)
    rng = np.random.default_rng(6)
    vis, cal, autos, bl_st, _ = synth.dual_pol_scan(wl, rng, pulses_for(wl, rng))
    a = search(wl, vis, cal, autos=autos, bl_st=bl_st)
    b = search(wl, vis, cal, autos=autos, bl_st=bl_st, device=False)
    for d in range(wl.n_dm):
        for wi in range(len(wl.windows)):
            for bl in range(wl.n_bl):
                pa, pb = a.peaks(bl, d, wi), b.peaks(bl, d, wi)
                for x, y in zip(pa, pb):
                    np.testing.assert_array_equal(x, y)
    assert a.candidates() == b.candidates()
    a.close()
    b.close()


def test_plan_and_server_equal_the_single_search():
    """A plan mixing a dual-polarisation, auto-normalised segment with a
    plain one, and the server running the same request, give the single
    search's peaks bit for bit."""
    wl = synth.small(n_bl=3, n_ap=400, n_if=4, n_chan=64, n_dm=3, dm_step=30.0, min_baselines=1)
    rng = np.random.default_rng(7)
    vis, cal, autos, bl_st, _ = synth.dual_pol_scan(wl, rng, pulses_for(wl, rng))
    wl2 = synth.small(n_bl=2, n_ap=500, n_if=8, n_chan=32, n_dm=2, dm_step=20.0, min_baselines=1)
    vis2 = synth.noise(wl2, rng)
    ref = search(wl, vis, cal, autos=autos, bl_st=bl_st)
    dv, da, dv2 = (torch.from_numpy(x).cuda() for x in (vis, autos, vis2))
    plan = V.Plan([(wl, dv, cal, dict(autos=da, bl_st=bl_st)), (wl2, dv2, None)], graph=True)
    plan.run(stream=torch.cuda.current_stream().cuda_stream)
    r = plan.result(0)
    for d in range(wl.n_dm):
        for wi in range(len(wl.windows)):
            for bl in range(wl.n_bl):
                for x, y in zip(ref.peaks(bl, d, wi), r.peaks(bl, d, wi)):
                    np.testing.assert_array_equal(x, y)
    assert ref.candidates() == r.candidates()
    plan.close()
    srv = V.Server(max_inflight=2)
    rid = srv.submit(wl, dv, cal, autos=da, bl_st=bl_st)
    info, cands = srv.wait_all(rid)
    assert info.status == 0
    assert cands == ref.candidates()
    with pytest.raises(V.VolksError) as e:
        srv.submit(wl, dv, cal, stream_id=3, autos=da, bl_st=bl_st)
    assert e.value.code == V.VOLKS_EINVAL
    srv.close()
    ref.close()


def test_calibrator_fit_per_polarisation():
    wl = synth.small(n_bl=3, n_ap=400, n_if=4, n_chan=32)
    rng = np.random.default_rng(8)
    cal = np.stack([synth.draw_calibration(wl, rng) for _ in range(2)])
    vis = np.stack([synth.calibrator_scan(wl, cal[p], 0.5, rng) for p in range(2)])
    got, amp = V.volks_fringe_fit_calibrator(wl, torch.from_numpy(vis).cuda())
    assert got.shape == (2, wl.n_bl, wl.n_if, 2)
    for p in range(2):
        for b in range(wl.n_bl):
            f = O.fringe_fit_calibrator(vis[p, b], wl.n_if, wl.n_chan, wl.chan_bw_mhz)
            np.testing.assert_array_equal(got[p, b, :, 0], f.tau_s)
            np.testing.assert_allclose(amp[p, b], f.amp, rtol=1e-9)


def test_noalloc_entry_point_refuses_two_products():
    wl = synth.small(n_bl=2, n_ap=100, n_if=4, n_chan=16)
    vis = torch.zeros((2, wl.n_bl, wl.n_ap, wl.n_f), dtype=torch.complex64, device="cuda")
    seg = V.volks_segment()
    keep = V.fill_segment(seg, wl, vis)
    prm = V.make_params(wl)
    pk = torch.zeros(1 << 16, dtype=torch.float32, device="cuda")
    cell = torch.zeros(1 << 16, dtype=torch.int32, device="cuda")
    with pytest.raises(V.VolksError) as e:
        V.volks_search_peaks_noalloc(seg, prm, torch.cuda.current_stream().cuda_stream, pk.data_ptr(),
                                     cell.data_ptr())
    assert e.value.code == V.VOLKS_EINVAL
    del keep
