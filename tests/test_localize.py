"""Single-pulse localisation (Sec. 2.3, Eq. 2; the baseline rules and the
leave-one-out check of Sec. 3.1.2) through the C ABI against the FP64
oracle.  Host code only: runs without a GPU."""
import math

import numpy as np
import pytest

from oracle import volks_oracle as O
from paper_2108_05602_b300 import synth
from paper_2108_05602_b300 import volks as V

C_LIGHT = synth.C_LIGHT


def geometry_case(n_st, seed, noise_s=0.0, off=(2.0e-6, -1.5e-6), snr_lo=7.0, snr_hi=40.0,
                  max_len_m=2.5e6):
    """Per-baseline inputs of Eq. 2 from synthetic station positions: the
    pulse's delays at the offset position (plus calibration delays and
    noise), partials by central differences at the a priori position."""
    rng = np.random.default_rng(seed)
    ra0, dec0, gast = 0.9, 0.6, 1.3
    B, _ = synth.loc_geometry(n_st, rng, ra0, dec0, gast, max_len_m=max_len_m)
    h = 1e-7
    g = lambda ra, dec: synth.geometric_delay(B, ra, dec, gast)
    pa = (g(ra0 + h, dec0) - g(ra0 - h, dec0)) / (2 * h)
    pd = (g(ra0, dec0 + h) - g(ra0, dec0 - h)) / (2 * h)
    tau_cal = rng.uniform(-5e-9, 5e-9, size=len(B))
    tau = g(ra0 + off[0], dec0 + off[1]) - g(ra0, dec0) + tau_cal + rng.normal(0, noise_s, len(B))
    snr = rng.uniform(snr_lo, snr_hi, size=len(B))
    length = np.linalg.norm(B, axis=1)
    return [tau, tau_cal, pa, pd, snr, length]


def params(**kw):
    p = V.volks_loc_default_params()
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def check_vs_oracle(cols, **kw):
    got = V.volks_localize(*cols, prm=params(**kw))
    ref = O.localize(*cols, **kw)
    assert got["status"] == ref.status
    np.testing.assert_array_equal(got["used"], ref.used)
    assert got["n_used"] == int(ref.used.sum())
    if ref.status != 0:
        return got, ref
    np.testing.assert_allclose(got["x"], ref.x, rtol=1e-9, atol=1e-18)
    np.testing.assert_allclose(got["cov"], ref.cov, rtol=1e-7, atol=1e-30)
    assert got["rms_s"] == pytest.approx(ref.rms_s, rel=1e-6, abs=1e-22)
    assert got["outlier"] == ref.outlier
    np.testing.assert_allclose(got["x_clean"], ref.x_clean, rtol=1e-9, atol=1e-18)
    idx = np.nonzero(ref.used)[0]
    loo = got["loo"]
    assert np.isnan(loo[~ref.used]).all()
    if len(ref.loo):
        np.testing.assert_allclose(loo[idx], ref.loo, rtol=1e-8, atol=1e-18, equal_nan=True)
    return got, ref


def test_default_params_follow_the_paper():
    p = V.volks_loc_default_params()
    assert (p.min_snr, p.max_proj_len_m, p.min_baselines, p.outlier_factor) == (6.0, 3.0e6, 3, 5.0)


@pytest.mark.parametrize("n_st", [3, 4, 6, 10])
@pytest.mark.parametrize("noise_s", [0.0, 0.05e-9])
def test_matches_oracle_on_synthetic_geometry(n_st, noise_s):
    for seed in range(4):
        cols = geometry_case(n_st, seed, noise_s=noise_s, snr_lo=4.0)
        check_vs_oracle(cols)


def test_noise_free_recovery_of_the_offset():
    off = (3.0e-6, 1.0e-6)
    got = V.volks_localize(*geometry_case(8, 11, off=off))
    assert got["status"] == 0 and got["outlier"] == -1
    np.testing.assert_allclose(got["x"], off, rtol=1e-4)


def test_noisy_recovery_within_the_formal_error():
    """Delay noise sigma: the error in each coordinate stays within a few
    formal sigmas over many pulses (chi^2 check of the covariance)."""
    off = np.array([1.0e-6, -2.0e-6])
    chi2 = []
    for seed in range(40):
        got = V.volks_localize(*geometry_case(7, 100 + seed, noise_s=0.1e-9, off=tuple(off)))
        e = got["x"] - off
        chi2.append(float(e @ np.linalg.solve(got["cov"], e)))
    # chi^2 with 2 degrees of freedom: mean 2; sigma is estimated from 19 residuals
    assert 1.0 < np.mean(chi2) < 3.5


def test_bad_baseline_is_flagged_and_removed():
    off = (2.0e-6, -1.5e-6)
    for seed, bad in [(4, 7), (5, 0), (6, 13)]:
        cols = geometry_case(6, seed, noise_s=0.05e-9, off=off)
        cols[0][bad] += 30e-9
        got, ref = check_vs_oracle(cols)
        assert got["outlier"] == bad
        assert np.hypot(*(got["x_clean"] - off)) < 0.05 * np.hypot(*off)


def test_cuts_and_too_few_baselines():
    cols = geometry_case(4, 21)
    cols[4][:] = 20.0
    cols[4][[0, 1]] = [6.0, 5.0]         # SNR must exceed 6
    cols[5][2] = 3.0e6 + 1.0              # longer than 3000 km
    got, ref = check_vs_oracle(cols)
    assert got["used"].tolist() == [False, False, False, True, True, True]
    assert got["status"] == 0
    cols[4][3] = 1.0
    cols[4][4] = 1.0
    got, _ = check_vs_oracle(cols)
    assert got["status"] == 1 and got["n_used"] == 1
    # two baselines are enough when asked for: exact solution, zero covariance
    cols = geometry_case(3, 22)
    got, _ = check_vs_oracle([c[:2] for c in cols], min_baselines=2)
    assert got["status"] == 0 and not got["cov"].any()


def test_collinear_partials():
    pa = np.array([1e-3, 2e-3, -3e-3, 4e-3])
    ones = np.full(4, 10.0)
    got, _ = check_vs_oracle([np.zeros(4), np.zeros(4), pa, 0.5 * pa, ones, np.full(4, 1e6)])
    assert got["status"] == 2
    pd = 0.5 * pa
    pd[3] = -pa[3]
    x_true = np.array([1e-6, 2e-6])
    got, _ = check_vs_oracle([pa * x_true[0] + pd * x_true[1], np.zeros(4), pa, pd, ones,
                              np.full(4, 1e6)])
    assert got["status"] == 0 and got["outlier"] == -1
    assert np.isnan(got["loo"][3]).all() and np.isfinite(got["loo"][:3]).all()


def test_empty_and_invalid_arguments():
    got = V.volks_localize([], [], [], [], [], [])
    assert got["status"] == 1 and got["n_used"] == 0
    cols = geometry_case(4, 31)
    with pytest.raises(V.VolksError):
        V.volks_localize(*cols, prm=params(min_baselines=1))
    cols[0][2] = math.nan
    with pytest.raises(V.VolksError):
        V.volks_localize(*cols)
    cols[4][2] = 1.0                      # a NaN on an unused baseline is ignored
    assert V.volks_localize(*cols)["status"] == 0


def test_matches_oracle_on_random_inputs():
    """300 random cases: baseline counts 0-15, random partials (some
    collinear), SNRs and lengths around the cuts, noise levels and one
    injected bad delay in a third of them; every output field against the
    oracle."""
    rng = np.random.default_rng(2024)
    for case in range(300):
        n = int(rng.integers(0, 16))
        pa = rng.normal(0, 5e-3, n)
        pd = rng.normal(0, 5e-3, n) if case % 7 else 0.5 * pa
        x = rng.normal(0, 3e-6, 2)
        tau_cal = rng.normal(0, 1e-8, n)
        tau = tau_cal + pa * x[0] + pd * x[1] + rng.normal(0, 10 ** rng.uniform(-12, -9), n)
        if n and case % 3 == 0:
            tau[int(rng.integers(0, n))] += 3e-8
        snr = rng.uniform(3, 12, n)
        length = rng.uniform(1e5, 3.5e6, n)
        kw = dict(min_baselines=int(rng.integers(2, 5)), outlier_factor=float(rng.uniform(3, 8)))
        check_vs_oracle([tau, tau_cal, pa, pd, snr, length], **kw)
