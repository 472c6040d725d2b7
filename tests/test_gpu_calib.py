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
    with pytest.raises(V.VolksError) as e:
        V.volks_fringe_fit_calibrator(wl, vis, pad=3)
    assert e.value.code == V.VOLKS_EINVAL
    cal, amp = V.volks_fringe_fit_calibrator(wl, vis, n_ap=0)
    assert np.all(cal == 0) and np.all(amp == 0)
