"""Initial calibration on the GPU (volks_fringe_fit_calibrator, Sec. 2.1.1)
against the FP64 oracle: identical delay cells, phases and amplitudes to
FP64 rounding, exact recovery of on-grid instrumental terms, and a round
trip in which the fitted table calibrates a pulse search."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import volks_oracle as O
from paper_2108_05602_b300 import build, synth
from paper_2108_05602_b300 import volks as V

from test_gpu_parity import check_candidates, gpu_search

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    V.lib()


def _wrap(x):
    return np.angle(np.exp(1j * x))


@pytest.mark.parametrize("shape", [dict(n_if=4, n_chan=32, n_ap=300), dict(n_if=8, n_chan=64, n_ap=2500),
                                   dict(n_if=2, n_chan=128, n_ap=90), dict(n_if=16, n_chan=16, n_ap=4100)],
                         ids=["4x32", "8x64", "2x128", "16x16"])
@pytest.mark.parametrize("pad", [4, 2])
def test_calibrator_fit_matches_oracle(shape, pad):
    wl = synth.small(n_bl=3, **shape)
    rng = np.random.default_rng(shape["n_chan"] + pad)
    cal = synth.draw_calibration(wl, rng)               # off-grid delays
    vis = synth.calibrator_scan(wl, cal, 0.3, rng)
    got, amp = V.volks_fringe_fit_calibrator(wl, torch.from_numpy(vis).cuda(), pad=pad)
    for b in range(wl.n_bl):
        f = O.fringe_fit_calibrator(vis[b], wl.n_if, wl.n_chan, wl.chan_bw_mhz, pad=pad)
        np.testing.assert_array_equal(got[b, :, 0], f.tau_s)
        assert np.max(np.abs(_wrap(got[b, :, 1] - f.phi_rad))) < 1e-9
        np.testing.assert_allclose(amp[b], f.amp, rtol=1e-9)


def test_on_grid_terms_recovered_exactly_and_host_equals_device():
    wl = synth.small(n_bl=2, n_ap=500, n_if=8, n_chan=32)
    rng = np.random.default_rng(8)
    cal = synth.draw_calibration_on_grid(wl, rng)
    vis = synth.calibrator_scan(wl, cal, 1.0, None)
    got_d, amp_d = V.volks_fringe_fit_calibrator(wl, torch.from_numpy(vis).cuda())
    got_h, amp_h = V.volks_fringe_fit_calibrator(wl, vis)
    np.testing.assert_array_equal(got_d, got_h)
    np.testing.assert_array_equal(amp_d, amp_h)
    np.testing.assert_array_equal(got_d[..., 0], cal[..., 0])
    assert np.max(np.abs(_wrap(got_d[..., 1] - cal[..., 1]))) < 1e-6
    np.testing.assert_allclose(amp_d, 1.0, rtol=1e-6)


def test_fitted_table_calibrates_the_pulse_search():
    """Round trip: a calibrator scan and a pulse scan share the instrumental
    terms; the pulse search with the fitted table gives the candidates of the
    search with the true table, and both equal the oracle's."""
    wl = synth.small(n_bl=2, n_ap=260, n_if=8, n_chan=32, n_dm=3, dm_step=30.0,
                     windows=(1, 2, 4, 8, 16), min_baselines=1)
    rng = np.random.default_rng(9)
    cal = synth.draw_calibration_on_grid(wl, rng)
    cvis = synth.calibrator_scan(wl, cal, 0.8, rng, n_ap=1000)
    fitted, _ = V.volks_fringe_fit_calibrator(wl, cvis, n_ap=1000)
    np.testing.assert_array_equal(fitted[..., 0], cal[..., 0])
    vis = synth.noise(wl, rng)
    M = 4 * wl.n_f
    synth.inject(vis, wl, cal, [synth.Pulse(30.0, 100, 4, 25.0,
                                            np.array([40, -77]) / (M * wl.chan_bw_mhz * 1e6),
                                            np.array([2.0, -3.0]))])
    g_fit = gpu_search(wl, vis, fitted)
    g_true = gpu_search(wl, vis, cal)
    key = lambda c: (c["bl"], c["dm_idx"], c["win"], c["seg"], c["delay_idx"], c["rate_idx"])
    cf, ct = g_fit.candidates(), g_true.candidates()
    assert sorted(map(key, cf)) == sorted(map(key, ct))
    # the fitted phases carry the calibrator's radiometer error d_n per IF;
    # rotating IF n's share of a peak by d_n moves |Z|^2 by at most
    # 2 max|d_n| relative (plus the FP32 bound)
    dphi = np.max(np.abs(_wrap(fitted[..., 1] - cal[..., 1])))
    assert 0 < dphi < 0.05
    for a, b in zip(sorted(cf, key=key), sorted(ct, key=key)):
        assert math.isclose(a["peak_power"], b["peak_power"], rel_tol=2 * dphi + 1e-4)
    ref = O.search(wl, vis, fitted)
    check_candidates(wl, g_fit, ref)
    hits = [c for c in cf if c["dm_idx"] == 1 and c["g0_ap"] <= 104 and c["g1_ap"] >= 100]
    assert hits and max(hits, key=lambda c: c["z"])["n_windows"] >= 2


def test_rejects_bad_arguments():
    wl = synth.small(n_bl=1, n_ap=10, n_if=4, n_chan=16)
    vis = np.zeros((1, 10, wl.n_f), dtype=np.complex64)
    with pytest.raises(ValueError):
        V.volks_fine_calibration(wl, vis, n_ap=9)   # the binding checks the array's shape
    with pytest.raises(V.VolksError) as e:
        V.volks_fringe_fit_calibrator(wl, vis, pad=3)
    assert e.value.code == V.VOLKS_EINVAL
    cal, amp = V.volks_fringe_fit_calibrator(wl, vis, n_ap=0)
    assert np.all(cal == 0) and np.all(amp == 0)


# ------------------------------------------------------ fine calibration ----
@pytest.mark.parametrize("shape", [dict(n_if=8, n_chan=64, n_ap=700), dict(n_if=4, n_chan=32, n_ap=2100),
                                   dict(n_if=12, n_chan=32, n_ap=300)], ids=["512", "128", "384"])
@pytest.mark.parametrize("pad", [4, 2])
def test_fine_calibration_matches_oracle(shape, pad):
    wl = synth.small(n_bl=3, **shape)
    rng = np.random.default_rng(shape["n_chan"] * 3 + pad)
    cal = synth.draw_calibration(wl, rng)
    M = pad * wl.n_f
    tau = rng.uniform(-0.4, 0.4, size=wl.n_bl) * M / (M * wl.chan_bw_mhz * 1e6) / 2
    vis = synth.calibrator_scan(wl, cal, 0.2, rng, tau_s=tau)
    got, amp = V.volks_fine_calibration(wl, torch.from_numpy(vis).cuda(), cal, pad=pad)
    for b in range(wl.n_bl):
        f = O.fine_calibration(vis[b], cal[b], wl.n_if, wl.n_chan, wl.chan_bw_mhz, pad=pad)
        assert got[b] == f.tau_s
        assert abs(amp[b] - f.amp) <= 1e-9 * f.amp


def test_fine_calibration_on_grid_exact_and_host_equals_device():
    wl = synth.small(n_bl=4, n_ap=200, n_if=8, n_chan=32)
    rng = np.random.default_rng(12)
    cal = synth.draw_calibration(wl, rng)
    cells = np.array([5, -77, 300, -512])
    tau = cells / (4 * wl.n_f * wl.chan_bw_mhz * 1e6)
    vis = synth.calibrator_scan(wl, cal, 1.0, None, tau_s=tau)
    got_d, amp_d = V.volks_fine_calibration(wl, torch.from_numpy(vis).cuda(), cal)
    got_h, amp_h = V.volks_fine_calibration(wl, vis, cal)
    np.testing.assert_array_equal(got_d, got_h)
    np.testing.assert_array_equal(amp_d, amp_h)
    np.testing.assert_array_equal(got_d, tau)
    np.testing.assert_allclose(amp_d, 1.0, rtol=1e-6)


def test_fine_calibration_search_and_localisation_end_to_end():
    """Sec. 2.1.2 -> Sec. 2.2 -> Sec. 2.3 on synthetic geometry: instrumental
    delays common to a reference source and the target; the fine
    calibration's tau_cal, the pulse's per-baseline delays from the search
    and the geometric partials give the target's offset through Eq. 2 to
    the delay-grid resolution."""
    rng = np.random.default_rng(13)
    n_st = 5
    B, _ = synth.loc_geometry(n_st, rng)
    # min_baselines = 1: every baseline's window-matched group is returned
    wl = synth.small(n_bl=len(B), n_ap=300, n_if=8, n_chan=64, n_dm=3, dm_step=30.0,
                     windows=(1, 2, 4, 8, 16), min_baselines=1)
    ra0, dec0, gast = 0.9, 0.6, 1.3
    g = lambda ra, dec: synth.geometric_delay(B, ra, dec, gast)
    h = 1e-7
    pa = (g(ra0 + h, dec0) - g(ra0 - h, dec0)) / (2 * h)
    pd = (g(ra0, dec0 + h) - g(ra0, dec0 - h)) / (2 * h)
    off = np.array([1.5e-5, -1.0e-5])
    tau_geo = g(ra0 + off[0], dec0 + off[1]) - g(ra0, dec0)
    tau_inst = rng.uniform(-50e-9, 50e-9, size=wl.n_bl)
    cal = synth.draw_calibration(wl, rng)
    ref = synth.calibrator_scan(wl, cal, 0.3, rng, n_ap=400, tau_s=tau_inst)
    tau_cal, _ = V.volks_fine_calibration(wl, ref, cal, n_ap=400)
    cell = 1.0 / (4 * wl.n_f * wl.chan_bw_mhz * 1e6)
    assert np.all(np.abs(tau_cal - tau_inst) <= cell + 1e-15)
    vis = synth.noise(wl, rng)
    synth.inject(vis, wl, cal, [synth.Pulse(30.0, 120, 4, 40.0, tau_geo + tau_inst, np.zeros(wl.n_bl))])
    s2 = V.Search(wl, torch.from_numpy(vis).cuda(), cal, stream=torch.cuda.current_stream().cuda_stream)
    cands = [c for c in s2.candidates() if c["dm_idx"] == 1 and c["g0_ap"] <= 124 and c["g1_ap"] >= 120]
    best = {}
    for c in cands:
        if c["bl"] not in best or c["z"] > best[c["bl"]]["z"]:
            best[c["bl"]] = c
    assert len(best) == wl.n_bl
    tau_p = np.array([best[b]["delay_s"] for b in range(wl.n_bl)])
    assert np.all(np.abs(tau_p - (tau_geo + tau_inst)) <= cell + 1e-15)
    snr = np.array([best[b]["z"] for b in range(wl.n_bl)])
    loc = V.volks_localize(tau_p, tau_cal, pa, pd, snr, np.linalg.norm(B, axis=1))
    assert loc["status"] == 0 and loc["n_used"] == wl.n_bl
    assert np.hypot(*(loc["x"] - off)) < 0.05 * np.hypot(*off)
    # the re-fit of Sec. 3.1.2 on a 4x finer grid, with its SNR for the cut
    fits = s2.refit([best[b] for b in range(wl.n_bl)], pad=16)
    s2.close()
    tau_r = np.array([f["delay_s"] for f in fits])
    assert np.all(np.abs(tau_r - (tau_geo + tau_inst)) <= cell / 4 + 1e-15)
    snr_r = np.array([f["snr"] for f in fits])
    assert np.all(snr_r > 6)
    loc_r = V.volks_localize(tau_r, tau_cal, pa, pd, snr_r, np.linalg.norm(B, axis=1))
    assert loc_r["status"] == 0
    assert np.hypot(*(loc_r["x"] - off)) < 0.05 * np.hypot(*off)
