"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these re-call the oracle's own formula to produce an expected value:
expected values come from the paper's printed numbers (tests/golden), hand
arithmetic, brute force of Eq. 1 with physical frequencies, closed forms,
independent code (the data generator's own injection) or distributional facts.
"""
import math
import os

import numpy as np
import pytest

from oracle import volks_oracle as O
from paper_2108_05602_b300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def read_golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            kv = line.split(";")[0]
            k, v = [x.strip() for x in kv.split("=")]
            out[k] = v
    return out


# ------------------------------------------------------------ golden ----
def test_el060_shape_arithmetic():
    """The paper's printed EL060 numbers tie together with the oracle's
    padding: FFT size = 4 x freq points, ~4 M FFTs per DM, IF band edges."""
    g = read_golden("el060_params.txt")
    n_if, bw = int(g["n_if"]), float(g["if_bw_mhz"])
    assert abs(float(g["band_hi_mhz"]) - float(g["band_lo_mhz"]) - n_if * bw) < 1e-9
    n_f = int(g["freq_points"])
    x = np.zeros((1, n_f), dtype=np.complex128)
    assert O.delay_transform(x, int(g["pad_delay"])).shape[1] == int(g["fft_size"])
    n_ap = float(g["scan_s"]) / float(g["ap_s"])
    n_fft = n_ap * int(g["n_baselines"])
    assert round(n_fft / 1e6) == int(g["ffts_per_dm_millions"])
    n_st = int(g["n_stations"])
    assert n_st * (n_st - 1) // 2 == int(g["n_baselines"])


# ---------------------------------------------------------------- a1 ----
def test_shift_table_hand_values():
    """Hand arithmetic for the PR1 band (centres 1536.25 .. 1663.75 MHz,
    T_AP = 1.024 ms): 1/1536.25^2 - 1/1663.75^2 = 6.24447e-8 MHz^-2, so the
    bottom-channel delay is 4148.808 * DM * 6.24447e-8 s = 0.2590707 ms * DM
    = 0.2530 AP * DM.  DM 48 -> 12.14 -> 12; DM 50 -> 12.65 -> 13;
    DM 51 -> 12.90 -> 13; DM 96 -> 24.29 -> 24; the top channel never moves."""
    wl = synth.pr1()
    tab = O.shift_table(wl.f_lo_mhz, wl.chan_bw_mhz, wl.n_f, [0, 48, 50, 51, 96], wl.t_ap_s)
    assert tab.shape == (5, 256)
    assert np.all(tab[0] == 0)
    assert [int(r[0]) for r in tab[1:]] == [12, 13, 13, 24]
    assert np.all(tab[:, -1] == 0)
    # cold-plasma delay falls with frequency: shifts never increase with k
    assert np.all(np.diff(tab, axis=1) <= 0)


def test_shift_table_rounds_half_up_not_truncates():
    """DM 50 bottom channel is 12.65 AP: truncation would give 12."""
    wl = synth.pr1()
    tab = O.shift_table(wl.f_lo_mhz, wl.chan_bw_mhz, wl.n_f, [50.0], wl.t_ap_s)
    assert tab[0, 0] == 13


def test_dedispersion_realigns_generator_pulse():
    """A pulse the generator disperses with its own code at a trial DM lands
    in one AP column after the oracle's dedispersion at that DM, and nowhere
    at DM 0 (independent implementations of the sweep must agree)."""
    wl = synth.small(n_bl=1, n_ap=200, n_if=4, n_chan=16, n_dm=4, dm_step=60.0)
    dm = float(wl.dms()[3])
    cal = np.zeros((1, wl.n_if, 2))
    vis = np.zeros((1, wl.n_ap, wl.n_f), dtype=np.complex64)
    p = synth.Pulse(dm=dm, t0_ap=40, width_ap=1, snr=5.0,
                    tau_s=np.zeros(1), nu_hz=np.zeros(1))
    synth.inject(vis, wl, cal, [p])
    tab = O.shift_table(wl.f_lo_mhz, wl.chan_bw_mhz, wl.n_f, wl.dms(), wl.t_ap_s)
    assert tab[3].max() > 5
    Xd = O.dedisperse(vis[0].astype(np.complex128), tab[3])
    power = np.abs(Xd) ** 2
    assert np.all(power[40] > 0)
    assert np.count_nonzero(power.sum(axis=1)) == 1
    Xd0 = O.dedisperse(vis[0].astype(np.complex128), tab[0])
    assert np.count_nonzero(np.abs(Xd0).sum(axis=1)) > 5


def test_dm_zero_is_identity():
    rng = np.random.default_rng(0)
    X = rng.standard_normal((50, 64)) + 1j * rng.standard_normal((50, 64))
    Xd = O.dedisperse(X, np.zeros(64, dtype=np.int64))
    assert np.array_equal(Xd, X)


# ------------------------------------------------------------- a2-a3 ----
def test_normalised_noise_has_unit_power_and_dead_channel_is_zero():
    rng = np.random.default_rng(1)
    v = (rng.standard_normal((400, 64)) * 3.0 + 1j * rng.standard_normal((400, 64)) * 3.0)
    v[:, 5] = 0
    X = O.calibrate(v, None, 4, 16, 0.5, normalize=True)
    p = np.mean(np.abs(X) ** 2, axis=0)
    assert np.allclose(np.delete(p, 5), 1.0, rtol=1e-12, atol=0)
    assert np.all(X[:, 5] == 0)


def test_calibration_flattens_generator_phases():
    """The generator writes per-IF delays/phases into a noise-free pulse at
    DM 0, zero residual delay and rate.  After the oracle's calibration all
    frequency points share one phase, so the coherent sum reaches the sum of
    magnitudes."""
    wl = synth.small(n_bl=1, n_ap=8, n_if=4, n_chan=16, n_dm=1)
    rng = np.random.default_rng(3)
    cal = synth.draw_calibration(wl, rng)
    cal[..., 0] *= 50  # make the delay term large (+-1 us) so a slip shows
    vis = np.zeros((1, wl.n_ap, wl.n_f), dtype=np.complex64)
    synth.inject(vis, wl, cal, [synth.Pulse(0.0, 2, 1, 4.0, np.zeros(1), np.zeros(1))])
    X = O.calibrate(vis[0], cal[0], wl.n_if, wl.n_chan, wl.chan_bw_mhz, normalize=False)
    row = X[2]
    assert abs(abs(row.sum()) - np.abs(row).sum()) < 1e-5 * np.abs(row).sum()
    # wrong-sign calibration would double the phases instead
    Xbad = vis[0, 2].astype(np.complex128) * np.conj(
        O.calib_phasor(cal[0], wl.n_if, wl.n_chan, wl.chan_bw_mhz))
    assert abs(Xbad.sum()) < 0.9 * np.abs(Xbad).sum()


# ---------------------------------------------------------------- a5 ----
def _tiny_segment(rng, W, n_if, n_chan):
    n_f = n_if * n_chan
    return rng.standard_normal((W, n_f)) + 1j * rng.standard_normal((W, n_f))


@pytest.mark.parametrize("n_if,n_chan", [(2, 8), (3, 8), (12, 8)])
def test_delay_transform_equals_eq1_brute_force(n_if, n_chan):
    """Eq. 1 evaluated with physical frequencies (Hz) and delays (s) on every
    cell of the padded delay grid equals the oracle's FFT power, including
    the calibration term that Eq. 1 carries inside Phi; also for bands of
    3 x 2^a points (12 IFs), which take mixed-radix transforms."""
    rng = np.random.default_rng(4)
    bw, f_lo = 0.5, 1600.0
    S = _tiny_segment(rng, 1, n_if, n_chan)
    cal = np.stack([rng.uniform(-1e-7, 1e-7, n_if), rng.uniform(0, 6.28, n_if)], axis=1)
    M = 4 * n_if * n_chan
    m = np.arange(M)
    taus = np.where(m < M // 2, m, m - M) / (M * bw * 1e6)
    G = O.eq1_brute_force(S, cal, n_if, n_chan, f_lo, bw, 1.024e-3, taus, np.zeros(1))
    X = S * O.calib_phasor(cal, n_if, n_chan, bw)[None, :]
    Y = O.delay_transform(X, 4)
    assert np.allclose(np.abs(G[0]) ** 2, np.abs(Y[0]) ** 2, rtol=1e-10, atol=1e-9)


def test_delay_sign_positive_tau_peaks_at_positive_cell():
    """A tone exp(+2 pi i (f - f_lo) tau) with tau = +37 cells peaks at
    signed cell +37 (Eq. 1 uses exp(-i Phi))."""
    n_f, bw = 64, 0.5
    M = 4 * n_f
    tau = 37 / (M * bw * 1e6)
    f_rel = (np.arange(n_f) + 0.5) * bw * 1e6
    X = np.exp(2j * np.pi * f_rel * tau)[None, :]
    Y = O.delay_transform(X, 4)
    assert int(np.argmax(np.abs(Y[0]))) == 37


def test_parseval_delay():
    rng = np.random.default_rng(5)
    X = _tiny_segment(rng, 3, 4, 16)
    Y = O.delay_transform(X, 4)
    M = Y.shape[1]
    assert np.allclose((np.abs(Y) ** 2).sum(axis=1), M * (np.abs(X) ** 2).sum(axis=1),
                       rtol=1e-12)


# ---------------------------------------------------------------- a6 ----
def test_rate_grid_equals_brute_force_2d():
    """Every (rate, delay) cell of a 4-AP window equals the brute-force
    double sum over APs and frequency points."""
    rng = np.random.default_rng(6)
    n_if, n_chan, bw, f_lo, tap, W = 2, 4, 0.5, 1600.0, 1.024e-3, 4
    S = _tiny_segment(rng, W, n_if, n_chan)
    M, R = 4 * n_if * n_chan, 4 * W
    m, q = np.arange(M), np.arange(R)
    taus = np.where(m < M // 2, m, m - M) / (M * bw * 1e6)
    nus = np.where(q < R // 2, q, q - R) / (R * tap)
    G = O.eq1_brute_force(S, None, n_if, n_chan, f_lo, bw, tap, taus, nus)
    Y = O.delay_transform(S, 4)
    Z = np.fft.fft(Y, n=R, axis=0)  # reference grid for this check only
    assert np.allclose(np.abs(G) ** 2, np.abs(Z) ** 2, rtol=1e-10, atol=1e-9)
    pk = O.window_peaks(Y, W, 4)
    bf = np.abs(G) ** 2
    iq, im = np.unravel_index(np.argmax(bf), bf.shape)
    assert (pk.q[0], pk.m[0]) == (iq, im)
    assert math.isclose(pk.P[0], bf.max(), rel_tol=1e-10)


def test_one_d_mode_is_rate_zero_row():
    """pad_rate = 0 (the paper's 1-D search over a coherent window sum)
    gives the q = 0 row of the 2-D search."""
    rng = np.random.default_rng(7)
    Y = O.delay_transform(_tiny_segment(rng, 16, 2, 8), 4)
    one = O.window_peaks(Y, 4, 0)
    # coherent sum per segment, max over delay
    cs = Y.reshape(4, 4, -1).sum(axis=1)
    assert np.allclose(one.P, (np.abs(cs) ** 2).max(axis=1), rtol=1e-12)
    assert np.array_equal(one.m, np.argmax(np.abs(cs) ** 2, axis=1))
    assert np.all(one.q == 0)


def test_rate_parseval():
    rng = np.random.default_rng(8)
    Y = O.delay_transform(_tiny_segment(rng, 8, 2, 8), 4)
    Z = np.fft.fft(Y.reshape(1, 8, -1), n=32, axis=1)
    assert np.allclose((np.abs(Z) ** 2).sum(), 32 * (np.abs(Y) ** 2).sum(), rtol=1e-12)


# ---------------------------------------------------------------- a7 ----
@pytest.mark.parametrize("w,m0,q0", [(4, 37, 3), (8, -100, -5), (2, 255, 7), (1, -3, 0)])
def test_on_grid_pulse_found_at_exact_cell(w, m0, q0):
    """A noise-free pulse with on-grid delay m0 / (M df) and rate
    q0 / (R T_AP) filling one window exactly peaks at cell (q0, m0) with
    |Z| = a * w * N_f (a the generator's amplitude)."""
    wl = synth.small(n_bl=1, n_ap=64, n_if=4, n_chan=16, n_dm=1)
    M, R = 4 * wl.n_f, (1 if w == 1 else 4 * w)
    tau = m0 / (M * wl.chan_bw_mhz * 1e6)
    nu = q0 / (R * wl.t_ap_s)
    cal = np.zeros((1, wl.n_if, 2))
    vis = np.zeros((1, wl.n_ap, wl.n_f), dtype=np.complex128)
    t0 = 3 * w
    p = synth.Pulse(0.0, t0, w, 6.0, np.array([tau]), np.array([nu]))
    rows, val = synth.pulse_footprint(wl, cal, p)
    for k in range(wl.n_f):
        vis[0, rows[k], k] += val[0, k]
    X = O.calibrate(vis[0], cal[0], wl.n_if, wl.n_chan, wl.chan_bw_mhz, normalize=False)
    Y = O.delay_transform(O.dedisperse(X, np.zeros(wl.n_f, dtype=np.int64)), 4)
    pk = O.window_peaks(Y, w, 4)
    s = t0 // w
    a = 6.0 * math.sqrt(2.0 / (w * wl.n_f))
    assert (int(pk.q[s]), int(pk.m[s])) == (q0 % R, m0 % M)
    assert math.isclose(pk.P[s], (a * w * wl.n_f) ** 2, rel_tol=1e-9)


@pytest.mark.parametrize("n_if,n_chan", [(12, 16), (3, 32)])
def test_on_grid_pulse_in_a_twelve_if_band(n_if, n_chan):
    """Bands of 3 x 2^a points: an on-grid pulse peaks at its exact cell
    with |Z| = a w N_f (M = 4 N_f is not a power of two)."""
    wl = synth.small(n_bl=1, n_ap=64, n_if=n_if, n_chan=n_chan, n_dm=1)
    w, m0, q0 = 8, -221, 6
    M, R = 4 * wl.n_f, 4 * w
    p = synth.Pulse(0.0, 2 * w, w, 6.0, np.array([m0 / (M * wl.chan_bw_mhz * 1e6)]),
                    np.array([q0 / (R * wl.t_ap_s)]))
    cal = np.zeros((1, wl.n_if, 2))
    vis = np.zeros((1, wl.n_ap, wl.n_f), dtype=np.complex128)
    rows, val = synth.pulse_footprint(wl, cal, p)
    for k in range(wl.n_f):
        vis[0, rows[k], k] += val[0, k]
    X = O.calibrate(vis[0], cal[0], wl.n_if, wl.n_chan, wl.chan_bw_mhz, normalize=False)
    pk = O.window_peaks(O.delay_transform(O.dedisperse(X, np.zeros(wl.n_f, dtype=np.int64)), 4), w, 4)
    a = 6.0 * math.sqrt(2.0 / (w * wl.n_f))
    assert (int(pk.q[2]), int(pk.m[2])) == (q0, m0 % M)
    assert math.isclose(pk.P[2], (a * w * wl.n_f) ** 2, rel_tol=1e-9)


def test_argmax_ties_go_to_lowest_linear_index():
    Y = np.zeros((4, 32), dtype=np.complex128)
    pk = O.window_peaks(Y, 2, 4)
    assert np.all(pk.q == 0) and np.all(pk.m == 0) and np.all(pk.P == 0)
    Y = np.zeros((2, 32), dtype=np.complex128)
    Y[0, 5] = Y[0, 9] = 1.0      # two equal delay peaks, w = 1
    pk = O.window_peaks(Y, 1, 4)
    assert pk.m[0] == 5 and pk.P2[0] == pk.P[0]


# ---------------------------------------------------------------- a8 ----
def test_noise_cell_power_is_exponential():
    """For Gaussian noise normalised to unit power per point, a fixed cell
    of the delay transform has |Y|^2 / N_f ~ Exp(1): KS test, fixed seed."""
    from scipy import stats
    rng = np.random.default_rng(9)
    v = (rng.standard_normal((20000, 64)) + 1j * rng.standard_normal((20000, 64)))
    X = O.calibrate(v, None, 4, 16, 0.5, normalize=True)
    Y = O.delay_transform(X, 4)
    rho = np.abs(Y[:, 17]) ** 2 / 64
    assert abs(rho.mean() - 1.0) < 0.03
    assert stats.kstest(rho, "expon").pvalue > 0.01
    # a dropped normalisation (data variance 2) fails the same test
    rho_bad = np.abs(np.fft.fft(v, n=256, axis=1)[:, 17]) ** 2 / 64
    assert stats.kstest(rho_bad, "expon").pvalue < 1e-6


def test_series_stats_hand_example():
    """rho = [1, 2, 3, 10]: mean 4, population variance (9+4+1+36)/4 = 12.5."""
    mu, sd = O.series_stats(np.array([1.0, 2.0, 3.0, 10.0]))
    assert mu == 4.0 and math.isclose(sd, math.sqrt(12.5), rel_tol=1e-15)
    z = O.zscores(np.array([1.0, 2.0, 3.0, 10.0]), mu, sd)
    assert math.isclose(z[3], 6.0 / math.sqrt(12.5), rel_tol=1e-15)
    assert np.all(O.zscores(np.ones(5), *O.series_stats(np.ones(5))) == 0)


# ------------------------------------------------------------ a9 a10 ----
def _m(w, s, z):
    return O.Member(w=w, s=s, z=z, P=0.0, q=0, m=0)


def test_window_match_hand_cases():
    # w=1 s=5 -> [5,6); w=2 s=2 -> [4,6); w=4 s=1 -> [4,8): one group, 3 windows
    # w=1 s=20 -> [20,21) alone: dropped; touching intervals do not overlap
    mem = [_m(1, 5, 4.0), _m(2, 2, 5.0), _m(4, 1, 3.5), _m(1, 20, 9.0),
           _m(1, 30, 3.1), _m(2, 16, 3.2)]   # [30,31) and [32,34) touch? no gap 31..32
    out = O.window_match(mem, 2)
    assert len(out) == 1
    rep, nw, g0, g1 = out[0]
    assert (rep.w, rep.s, nw, g0, g1) == (2, 2, 3, 4, 8)
    # [6,8) (w=2,s=3) and [8,16) (w=8,s=1) only touch: separate groups
    out = O.window_match([_m(2, 3, 4.0), _m(8, 1, 4.0)], 2)
    assert out == []
    # equal z: the smaller window, then the earlier segment represents
    rep = O.window_match([_m(4, 1, 4.0), _m(2, 2, 4.0), _m(2, 3, 4.0)], 2)[0][0]
    assert (rep.w, rep.s) == (2, 2)


def test_overlap_components_match_brute_force_graph():
    rng = np.random.default_rng(11)
    for _ in range(200):
        n = int(rng.integers(1, 12))
        iv = []
        for _ in range(n):
            w = int(2 ** rng.integers(0, 4))
            s = int(rng.integers(0, 40 // w))
            iv.append((s * w, (s + 1) * w))
        iv = list(set(iv))
        comps = O.overlap_components(iv, lambda a: a[0], lambda a: a[1])
        # brute force: union-find over pairwise strict overlap
        parent = list(range(len(iv)))

        def find(i):
            while parent[i] != i:
                i = parent[i]
            return i
        for i in range(len(iv)):
            for j in range(len(iv)):
                if iv[i][0] < iv[j][1] and iv[j][0] < iv[i][1]:
                    parent[find(i)] = find(j)
        groups = {}
        for i, x in enumerate(iv):
            groups.setdefault(find(i), set()).add(x)
        assert sorted(map(sorted, groups.values())) == sorted(map(sorted, map(set, comps)))


def test_cross_baseline_hand_case():
    c = lambda bl, t0, t1: dict(bl=bl, t0=t0, t1=t1)
    cands = [c(0, 10, 12), c(1, 11, 13), c(2, 9, 11), c(3, 50, 52), c(4, 51, 52)]
    out = O.cross_baseline(cands, 3)
    assert sorted(x["bl"] for x in out) == [0, 1, 2]
    assert all(x["n_baselines"] == 3 for x in out)
    assert O.cross_baseline(cands, 2) and len(O.cross_baseline(cands, 2)) == 5


# ------------------------------------------------------------- whole ----
def test_pr1_pulse_recovered():
    """PR1 end to end: the DM 50, 3.2 us, 0.5 Hz pulse (SNR 10, 2 AP) is
    found at a DM trial next to 50 in >= 2 windows.  3.2 us aliases to
    -0.8 us in the 2 us delay window (1 / 0.5 MHz): cell -409.6 of 1024.
    0.5 Hz is far below one rate cell (>= 30 Hz), so rate cell 0."""
    wl, vis, cal, pulses = synth.gen_pr1(seed=1)
    res = O.search(wl, vis, cal, with_second=False)
    t0 = pulses[0].t0_ap
    hits = [c for c in res.candidates if abs(wl.dms()[c["dm_idx"]] - 50) <= 3
            and c["g0"] <= t0 + 2 and c["g1"] >= t0]
    assert hits, res.candidates
    best = max(hits, key=lambda c: c["z"])
    assert best["n_windows"] >= 2
    assert abs(best["delay_idx"] - (-410)) <= 1
    assert best["rate_idx"] == 0
    assert math.sqrt(best["rho"]) > 7
    # the generator's own sweep at DM 50 agrees with the DM 51 trial on most channels
    same = np.sum(synth.arrival_offsets_ap(wl, 50.0) ==
                  O.shift_table(wl.f_lo_mhz, wl.chan_bw_mhz, wl.n_f, [51.0], wl.t_ap_s)[0])
    assert same >= 200


# ------------------------------------------- initial calibration (Sec. 2.1.1) ----
def test_calibrator_fit_recovers_on_grid_delay_and_phase_exactly():
    """Noise-free calibrator with on-grid per-IF delays: the fit returns the
    injected (dtau0, dphi0) and a perfect fringe amplitude."""
    wl = synth.small(n_bl=2, n_ap=40, n_if=4, n_chan=32)
    rng = np.random.default_rng(3)
    cal = synth.draw_calibration_on_grid(wl, rng)
    vis = synth.calibrator_scan(wl, cal, 0.7, None)
    for b in range(wl.n_bl):
        f = O.fringe_fit_calibrator(vis[b], wl.n_if, wl.n_chan, wl.chan_bw_mhz)
        assert np.array_equal(f.tau_s, cal[b, :, 0])
        dphi = np.angle(np.exp(1j * (f.phi_rad - cal[b, :, 1])))
        assert np.max(np.abs(dphi)) < 1e-6
        np.testing.assert_allclose(f.amp, 1.0, rtol=1e-6)
        assert np.all((f.phi_rad > -np.pi) & (f.phi_rad <= np.pi))


def test_calibrator_fit_flattens_the_fringe_phase_with_the_search_phasor():
    """Applying the fitted table with the search's own calibration phasor
    (Eq. 1) makes the time-integrated phase zero in every channel: a wrong
    sign or channel-frequency reference in either would leave a slope."""
    wl = synth.small(n_bl=1, n_ap=25, n_if=8, n_chan=16)
    rng = np.random.default_rng(4)
    cal = synth.draw_calibration_on_grid(wl, rng)
    vis = synth.calibrator_scan(wl, cal, 1.3, None)
    f = O.fringe_fit_calibrator(vis[0], wl.n_if, wl.n_chan, wl.chan_bw_mhz)
    table = np.stack([f.tau_s, f.phi_rad], axis=1)
    X = O.calibrate(vis[0], table, wl.n_if, wl.n_chan, wl.chan_bw_mhz, normalize=False)
    ph = np.angle(X.sum(axis=0))
    assert np.max(np.abs(ph)) < 1e-5


def test_calibrator_fit_sign_offgrid_and_ambiguity():
    wl = synth.small(n_bl=1, n_ap=10, n_if=1, n_chan=64)
    bw = wl.chan_bw_mhz * 1e6
    Mc = 4 * wl.n_chan
    # a positive delay lands on a positive cell
    cal = np.array([[[7 / (Mc * bw), 0.4]]])
    f = O.fringe_fit_calibrator(synth.calibrator_scan(wl, cal, 1.0, None)[0], 1, 64, wl.chan_bw_mhz)
    assert f.cell[0] == 7
    # off grid: the nearest cell (within half a cell)
    cal = np.array([[[-12.3 / (Mc * bw), -1.1]]])
    f = O.fringe_fit_calibrator(synth.calibrator_scan(wl, cal, 1.0, None)[0], 1, 64, wl.chan_bw_mhz)
    assert f.cell[0] == -12
    # a delay one full period 1 / chan_bw away is the same fringe
    cal = np.array([[[5 / (Mc * bw) + 1.0 / bw, 2.0]]])
    f = O.fringe_fit_calibrator(synth.calibrator_scan(wl, cal, 1.0, None)[0], 1, 64, wl.chan_bw_mhz)
    assert f.cell[0] == 5


def test_calibrator_fit_in_noise_matches_expected_precision():
    """Calibrator at amplitude 0.5 in unit noise over 200 APs x 32 channels:
    delay on the right cell, phase error at the radiometer level."""
    wl = synth.small(n_bl=3, n_ap=200, n_if=4, n_chan=32)
    rng = np.random.default_rng(5)
    cal = synth.draw_calibration_on_grid(wl, rng)
    vis = synth.calibrator_scan(wl, cal, 0.5, rng)
    # per IF: signal |sum| = 0.5 * 200 * 32, noise std of the sum's phase
    sigma_phi = np.sqrt(2 * 200 * 32) / (0.5 * 200 * 32) / np.sqrt(2)
    for b in range(wl.n_bl):
        f = O.fringe_fit_calibrator(vis[b], wl.n_if, wl.n_chan, wl.chan_bw_mhz)
        assert np.array_equal(f.tau_s, cal[b, :, 0])
        dphi = np.angle(np.exp(1j * (f.phi_rad - cal[b, :, 1])))
        assert np.max(np.abs(dphi)) < 6 * sigma_phi


# --------------------------------------------- localisation (Sec. 2.3, Eq. 2) ----
def _loc_case(n_st=6, seed=0, noise_s=0.0, off=(2.0e-6, -1.5e-6)):
    """Delays of a point source offset by `off` (rad) from the a priori
    position, partials by central differences of the geometric delay."""
    rng = np.random.default_rng(seed)
    ra0, dec0, gast = 0.9, 0.6, 1.3
    B, _ = synth.loc_geometry(n_st, rng, ra0, dec0, gast)
    h = 1e-7
    pa = (synth.geometric_delay(B, ra0 + h, dec0, gast) - synth.geometric_delay(B, ra0 - h, dec0, gast)) / (2 * h)
    pd = (synth.geometric_delay(B, ra0, dec0 + h, gast) - synth.geometric_delay(B, ra0, dec0 - h, gast)) / (2 * h)
    tau_cal = rng.uniform(-5e-9, 5e-9, size=len(B))
    tau = (synth.geometric_delay(B, ra0 + off[0], dec0 + off[1], gast)
           - synth.geometric_delay(B, ra0, dec0, gast) + tau_cal + rng.normal(0, noise_s, size=len(B)))
    snr = np.full(len(B), 20.0)
    length = np.linalg.norm(B, axis=1)
    return tau, tau_cal, pa, pd, snr, length


def test_localize_recovers_offsets_of_a_linear_model_exactly():
    rng = np.random.default_rng(1)
    pa, pd = rng.normal(0, 5e-3, 10), rng.normal(0, 5e-3, 10)
    x_true = np.array([3e-6, -7e-6])
    tau_cal = rng.normal(0, 1e-8, 10)
    tau = tau_cal + pa * x_true[0] + pd * x_true[1]
    r = O.localize(tau, tau_cal, pa, pd, np.full(10, 9.0), np.full(10, 1e6))
    assert r.status == 0 and r.used.all() and r.outlier == -1
    np.testing.assert_allclose(r.x, x_true, rtol=1e-9)
    assert r.rms_s < 1e-20


def test_localize_recovers_a_geometric_offset_and_the_sign_of_eq2():
    """A source 0.4"/0.3" off the a priori position (geometric delays, not
    the linear model): recovered to the linearisation error; a flipped sign
    of tau - tau_cal would return the negated offset."""
    off = (2.0e-6, -1.5e-6)
    tau, tau_cal, pa, pd, snr, length = _loc_case(off=off)
    r = O.localize(tau, tau_cal, pa, pd, snr, length)
    assert r.status == 0
    np.testing.assert_allclose(r.x, off, rtol=1e-4)


def test_localize_applies_the_snr_and_length_cuts():
    tau, tau_cal, pa, pd, snr, length = _loc_case(n_st=7, seed=2)
    ref = O.localize(tau, tau_cal, pa, pd, snr, length)
    tau2, snr2, len2 = tau.copy(), snr.copy(), length.copy()
    tau2[0] += 1e-6; snr2[0] = 6.0          # SNR must exceed 6
    tau2[1] -= 1e-6; len2[1] = 3.2e6        # projected baseline over 3000 km
    r = O.localize(tau2, tau_cal, pa, pd, snr2, len2)
    assert not r.used[0] and not r.used[1] and r.used[2:].all()
    np.testing.assert_allclose(r.x, ref.x, rtol=1e-4)


def test_localize_needs_three_baselines():
    tau, tau_cal, pa, pd, snr, length = _loc_case(n_st=3, seed=3)
    assert O.localize(tau, tau_cal, pa, pd, snr, length).status == 0
    snr[2] = 2.0
    r = O.localize(tau, tau_cal, pa, pd, snr, length)
    assert r.status == 1


def test_localize_leave_one_out_flags_a_bad_baseline():
    """One baseline with a 30 ns fitting error (the RFI case of Sec. 3.1.2):
    the leave-one-out solution without it is the odd one out, it is flagged,
    and the clean solution recovers the offset; with no bad baseline nothing
    is flagged."""
    off = (2.0e-6, -1.5e-6)
    tau, tau_cal, pa, pd, snr, length = _loc_case(n_st=6, seed=4, noise_s=0.05e-9, off=off)
    r0 = O.localize(tau, tau_cal, pa, pd, snr, length)
    assert r0.outlier == -1
    tau[7] += 30e-9
    r = O.localize(tau, tau_cal, pa, pd, snr, length)
    assert r.outlier == 7
    assert np.hypot(*(r.x_clean - off)) < 0.05 * np.hypot(*off)
    assert np.hypot(*(r.x - off)) > 0.1 * np.hypot(*off)


def test_localize_reports_collinear_partials():
    """Eq. 2 has no unique solution when every baseline's partials are
    proportional (one direction of the sky is unconstrained)."""
    pa = np.array([1e-3, 2e-3, -3e-3, 4e-3])
    r = O.localize(np.zeros(4), np.zeros(4), pa, 0.5 * pa, np.full(4, 10.0), np.full(4, 1e6))
    assert r.status == 2
    # three of four collinear: solvable, but one leave-one-out system is not
    pd = 0.5 * pa
    pd[3] = -pa[3]
    x_true = np.array([1e-6, 2e-6])
    tau = pa * x_true[0] + pd * x_true[1]
    r = O.localize(tau, np.zeros(4), pa, pd, np.full(4, 10.0), np.full(4, 1e6))
    assert r.status == 0 and r.outlier == -1
    np.testing.assert_allclose(r.x, x_true, rtol=1e-9)
    assert np.isnan(r.loo[3]).all() and np.isfinite(r.loo[:3]).all()


# ------------------------- polarisation combine, HOPS normalisation ----
def test_auto_spectrum_normalisation_undoes_the_bandpass():
    """Cross spectrum sqrt(g_i g_j) Z with constant auto spectra g: the
    HOPS factor (mean a_i^2 mean a_j^2)^(-1/4) = 1/sqrt(g_i g_j) returns Z
    (a square-root instead of a fourth root, or a_i instead of a_i^2,
    leaves the bandpass in); a station without power zeroes its points."""
    rng = np.random.default_rng(41)
    n_ap, n_f = 50, 64
    g = synth.bandpass(1, 3, n_f, rng)[0]
    Z = rng.standard_normal((n_ap, n_f)) + 1j * rng.standard_normal((n_ap, n_f))
    autos = np.broadcast_to(g[:, None, :], (3, n_ap, n_f))
    i, j = 0, 2
    S = Z * np.sqrt(g[i] * g[j])[None, :]
    X = O.calibrate(S, None, 4, 16, 0.5, norm=O.auto_norm(autos[i], autos[j]))
    np.testing.assert_allclose(X, Z, rtol=1e-12)
    a0 = autos[i].copy()
    a0[:, 5] = 0.0
    f = O.auto_norm(a0, autos[j])
    assert f[5] == 0.0 and np.all(f[np.arange(n_f) != 5] > 0)


def test_polarisation_products_add_coherently_after_their_own_calibration():
    """An on-grid pulse in two products with different instrumental terms:
    each calibrated with its own table and summed, the peak is (2 a w N_f)^2
    at the pulse's cell; calibrating each with the other's table loses
    coherence."""
    wl = synth.small(n_bl=1, n_ap=64, n_if=4, n_chan=16, n_dm=1)
    rng = np.random.default_rng(42)
    w, m0, q0 = 8, 37, 5
    M, R = 4 * wl.n_f, 4 * w
    cal = np.stack([synth.draw_calibration_on_grid(wl, rng) for _ in range(2)])
    p = synth.Pulse(0.0, 3 * w, w, 6.0, np.array([m0 / (M * wl.chan_bw_mhz * 1e6)]),
                    np.array([q0 / (R * wl.t_ap_s)]))
    vis = np.zeros((2, 1, wl.n_ap, wl.n_f), dtype=np.complex128)
    for pol in range(2):
        rows, val = synth.pulse_footprint(wl, cal[pol], p)
        for k in range(wl.n_f):
            vis[pol, 0, rows[k], k] += val[0, k]
    a = 6.0 * math.sqrt(2.0 / (w * wl.n_f))

    def peak(c):
        X = O.prepare(vis, c, 0, wl.n_if, wl.n_chan, wl.chan_bw_mhz, normalize=False)
        Y = O.delay_transform(O.dedisperse(X, np.zeros(wl.n_f, dtype=np.int64)), 4)
        pk = O.window_peaks(Y, w, 4)
        return pk, 3

    pk, s = peak(cal)
    assert (int(pk.q[s]), int(pk.m[s])) == (q0, m0)
    assert math.isclose(pk.P[s], (2 * a * w * wl.n_f) ** 2, rel_tol=1e-9)
    pk_bad, _ = peak(cal[::-1])
    assert pk_bad.P[s] < 0.9 * pk.P[s]


def test_one_product_in_the_four_dimensional_layout_is_the_plain_search():
    wl = synth.small(n_bl=2, n_ap=96, n_if=4, n_chan=16, n_dm=3, dm_step=20.0)
    rng = np.random.default_rng(43)
    vis = synth.noise(wl, rng)
    cal = synth.draw_calibration(wl, rng)
    a = O.search(wl, vis, cal)
    b = O.search(wl, vis[None], cal[None])
    for key in a.peaks:
        np.testing.assert_array_equal(a.peaks[key].P, b.peaks[key].P)


def test_two_normalised_noise_products_double_the_cell_power():
    """Independent noise in two products adds incoherently: with the RMS
    normalisation each product has unit power per point, so a delay cell's
    mean power is 2 N_f; the HOPS normalisation removes the bandpass exactly
    (no auto-spectrum jitter) and leaves the generator's variance of 2 per
    point and product, so 4 N_f."""
    wl = synth.small(n_bl=3, n_ap=400, n_if=4, n_chan=16)
    rng = np.random.default_rng(44)
    vis, cal, autos, bl_st, g = synth.dual_pol_scan(wl, rng, [], auto_jitter=0.0)
    for kw in (dict(), dict(autos=autos, bl_st=bl_st)):
        X = O.prepare(vis, cal, 1, wl.n_if, wl.n_chan, wl.chan_bw_mhz, **kw)
        Y = O.delay_transform(X, 4)
        mean = np.mean(np.abs(Y) ** 2) / wl.n_f
        expect = 2.0 if not kw else 4.0
        assert abs(mean / expect - 1) < 0.03, (kw.keys(), mean)


# ------------------------------------------------- fine calibration ----
def test_fine_calibration_recovers_an_on_grid_band_delay_exactly():
    """A reference source with a residual delay on the band-wide grid and
    per-IF instrumental terms: with the initial calibration applied the
    residual delay is recovered exactly with amplitude 1 (positive delay,
    positive cell); without it the IFs add incoherently."""
    wl = synth.small(n_bl=3, n_ap=40, n_if=8, n_chan=32)
    rng = np.random.default_rng(51)
    cal = synth.draw_calibration(wl, rng)
    M = 4 * wl.n_f
    cells = np.array([37, -410, 511])
    tau = cells / (M * wl.chan_bw_mhz * 1e6)
    vis = synth.calibrator_scan(wl, cal, 1.0, None, tau_s=tau)
    for b in range(wl.n_bl):
        f = O.fine_calibration(vis[b], cal[b], wl.n_if, wl.n_chan, wl.chan_bw_mhz)
        assert f.cell == cells[b]
        assert f.tau_s == cells[b] / (M * wl.chan_bw_mhz * 1e6)
        assert math.isclose(f.amp, 1.0, rel_tol=1e-9)
        g = O.fine_calibration(vis[b], None, wl.n_if, wl.n_chan, wl.chan_bw_mhz)
        assert g.amp < 0.8


def test_fine_calibration_error_within_half_a_cell_off_grid():
    wl = synth.small(n_bl=4, n_ap=30, n_if=4, n_chan=32)
    rng = np.random.default_rng(52)
    cal = synth.draw_calibration(wl, rng)
    M = 4 * wl.n_f
    cell_s = 1.0 / (M * wl.chan_bw_mhz * 1e6)
    tau = rng.uniform(-200, 200, size=wl.n_bl) * cell_s
    vis = synth.calibrator_scan(wl, cal, 1.0, None, tau_s=tau)
    for b in range(wl.n_bl):
        f = O.fine_calibration(vis[b], cal[b], wl.n_if, wl.n_chan, wl.chan_bw_mhz)
        assert abs(f.tau_s - tau[b]) <= 0.5 * cell_s + 1e-18


# ----------------------------------------------------- pulse re-fit ----
def _pulse_only(wl, p, cal=None):
    cal = np.zeros((wl.n_bl, wl.n_if, 2)) if cal is None else cal
    vis = np.zeros((wl.n_bl, wl.n_ap, wl.n_f), dtype=np.complex128)
    rows, val = synth.pulse_footprint(wl, cal, p)
    for b in range(wl.n_bl):
        for k in range(wl.n_f):
            vis[b, rows[k], k] += val[b, k]
    return vis


def test_refit_finds_a_fine_grid_delay_exactly_and_its_snr():
    """A noise-free pulse with delay m0 on the 16-times padded grid (not on
    the search's 4-times grid) and a rate on the window's grid: the re-fit
    lands on m0 with |G| = a W N_f, SNR = a sqrt(W N_f), amplitude 1."""
    wl = synth.small(n_bl=1, n_ap=96, n_if=4, n_chan=16, n_dm=1)
    W, m0, q0 = 8, 157, 3
    R = 4 * W
    nu = q0 / (R * wl.t_ap_s)
    p = synth.Pulse(0.0, 40, W, 6.0, np.array([m0 / (16 * wl.n_f * wl.chan_bw_mhz * 1e6)]), np.array([nu]))
    vis = _pulse_only(wl, p)
    X = O.calibrate(vis[0], None, wl.n_if, wl.n_chan, wl.chan_bw_mhz, normalize=False)
    r = O.refit_pulse(X, np.zeros(wl.n_f, dtype=np.int64), 40, 40 + W, nu, wl.t_ap_s, wl.chan_bw_mhz, 16, wl.n_f)
    a = 6.0 * math.sqrt(2.0 / (W * wl.n_f))
    assert r.cell == m0
    assert math.isclose(r.snr, a * math.sqrt(W * wl.n_f), rel_tol=1e-9)
    assert math.isclose(r.amp, 1.0, rel_tol=1e-9)
    # removing the rate with the wrong sign loses coherence
    bad = O.refit_pulse(X, np.zeros(wl.n_f, dtype=np.int64), 40, 40 + W, -nu, wl.t_ap_s, wl.chan_bw_mhz, 16,
                        wl.n_f)
    assert bad.snr < 0.5 * r.snr


def test_refit_snr_of_a_pulse_in_noise_matches_the_injected_snr():
    """Unit-normalised noise plus pulses of SNR 20: the re-fit's SNR
    estimate is sqrt(snr^2 + noise) ~ 20 on average."""
    wl = synth.small(n_bl=8, n_ap=200, n_if=4, n_chan=32, n_dm=1)
    rng = np.random.default_rng(61)
    M16 = 16 * wl.n_f
    snrs = []
    for rep in range(3):
        vis = synth.noise(wl, rng)
        m0 = rng.integers(-M16 // 2, M16 // 2, size=wl.n_bl)
        p = synth.Pulse(0.0, 60, 4, 20.0, m0 / (M16 * wl.chan_bw_mhz * 1e6), np.zeros(wl.n_bl))
        synth.inject(vis, wl, np.zeros((wl.n_bl, wl.n_if, 2)), [p])
        for b in range(wl.n_bl):
            X = O.calibrate(vis[b], None, wl.n_if, wl.n_chan, wl.chan_bw_mhz)
            r = O.refit_pulse(X, np.zeros(wl.n_f, dtype=np.int64), 60, 64, 0.0, wl.t_ap_s, wl.chan_bw_mhz, 16,
                              wl.n_f)
            assert abs(r.cell - m0[b]) <= 1
            snrs.append(r.snr)
    assert abs(np.mean(snrs) / 20.0 - 1) < 0.1


# --------------------------------------------- sliding windows (stride 1) ----
def test_sliding_segments_are_phase_shifted_strided_segments():
    """Segment s of a sliding (stride 1) search of window w is segment
    (s - phi) / w of the back-to-back search of the series shifted by
    phi = s mod w; stride w is the default search; n - w + 1 segments."""
    rng = np.random.default_rng(71)
    Y = rng.standard_normal((70, 48)) + 1j * rng.standard_normal((70, 48))
    for w in (1, 2, 4, 8):
        sl = O.window_peaks(Y, w, 4, stride=1)
        assert len(sl.P) == 70 - w + 1
        np.testing.assert_array_equal(O.window_peaks(Y, w, 4, stride=w).P, O.window_peaks(Y, w, 4).P)
        for phi in range(w):
            ref = O.window_peaks(Y[phi:], w, 4)
            idx = np.arange(phi, len(sl.P), w)
            np.testing.assert_array_equal(sl.P[idx], ref.P[:len(idx)])
            np.testing.assert_array_equal(sl.q[idx], ref.q[:len(idx)])
            np.testing.assert_array_equal(sl.m[idx], ref.m[:len(idx)])


def test_sliding_window_finds_a_pulse_that_straddles_two_segments():
    """A noise-free on-grid pulse of 4 APs starting at AP 6: the
    back-to-back 4-AP segments [4, 8) and [8, 12) each hold half of it;
    the sliding segment starting at 6 holds all of it, at (a w N_f)^2."""
    wl = synth.small(n_bl=1, n_ap=40, n_if=4, n_chan=16, n_dm=1)
    w, m0 = 4, 21
    M = 4 * wl.n_f
    p = synth.Pulse(0.0, 6, w, 6.0, np.array([m0 / (M * wl.chan_bw_mhz * 1e6)]), np.zeros(1))
    vis = _pulse_only(wl, p)
    X = O.calibrate(vis[0], None, wl.n_if, wl.n_chan, wl.chan_bw_mhz, normalize=False)
    Y = O.delay_transform(X, 4)
    a = 6.0 * math.sqrt(2.0 / (w * wl.n_f))
    full = (a * w * wl.n_f) ** 2
    sl = O.window_peaks(Y, w, 4, stride=1)
    assert int(np.argmax(sl.P)) == 6 and math.isclose(sl.P[6], full, rel_tol=1e-9)
    assert (int(sl.q[6]), int(sl.m[6])) == (0, m0)
    bb = O.window_peaks(Y, w, 4)
    assert bb.P.max() < 0.5 * full
