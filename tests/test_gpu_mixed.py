"""Bands of 3 x 2^a frequency points (e.g. 12 IFs): mixed-radix delay
transforms in the FP32 search kernel, every compiled work split, against
the FP64 oracle with the tolerances of tests/test_gpu_parity.py."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import volks_oracle as O
from paper_2108_05602_b300 import build, synth
from paper_2108_05602_b300 import volks as V

from test_gpu_parity import check_candidates, check_peaks, gpu_search, make_data

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    V.lib()


# one shape per compiled split (n1, fold): 96 (3,1), 192 (6,1), 384 (12,1),
# 768 (12,2), 1536 (12,4)
BANDS = [dict(n_if=12, n_chan=8, n_ap=333, n_bl=3, n_dm=5, dm_step=60.0),
         dict(n_if=12, n_chan=16, n_ap=301, n_bl=2, n_dm=4, dm_step=50.0),
         dict(n_if=12, n_chan=32, n_ap=270, n_bl=2, n_dm=3, dm_step=40.0),
         dict(n_if=12, n_chan=64, n_ap=200, n_bl=2, n_dm=2, dm_step=10.0),
         dict(n_if=12, n_chan=128, n_ap=150, n_bl=1, n_dm=2, dm_step=5.0)]


@pytest.mark.parametrize("band", BANDS, ids=["96", "192", "384", "768", "1536"])
@pytest.mark.parametrize("pad_rate", [4, 0])
def test_mixed_radix_band_matches_oracle(band, pad_rate):
    wl = synth.small(**band, windows=(1, 2, 4, 8, 32), pad_rate=pad_rate, min_baselines=1)
    vis, cal, _ = make_data(wl, seed=band["n_chan"] + pad_rate, n_pulses=2)
    g = gpu_search(wl, vis, cal)
    ref = O.search(wl, vis, cal)
    sh, nv = g.shifts()
    assert np.array_equal(sh, ref.shifts) and np.array_equal(nv, ref.nvalid)
    n, _ = check_peaks(wl, g, ref, vis, cal)
    assert n == sum(len(p.P) for p in ref.peaks.values())
    check_candidates(wl, g, ref, matched=True)
    g.close()


@pytest.mark.parametrize("pad_delay", [1, 2, 8])
def test_mixed_radix_pad_variants(pad_delay):
    wl = synth.small(n_if=12, n_chan=32, n_ap=200, n_bl=2, n_dm=2, dm_step=30.0, min_baselines=1)
    wl.pad_delay = pad_delay
    vis, cal, _ = make_data(wl, seed=11 + pad_delay, n_pulses=2)
    g = gpu_search(wl, vis, cal, pad_delay=pad_delay)
    ref = O.search(wl, vis, cal)
    check_peaks(wl, g, ref, vis, cal)
    check_candidates(wl, g, ref, matched=True)
    g.close()


def test_reduced_precision_request_runs_fp32_on_a_mixed_band():
    """The tensor-core path covers power-of-two bands only: a BF16 request
    on a 384-point band gives the FP32 search bit for bit."""
    wl = synth.small(n_if=12, n_chan=32, n_ap=260, n_bl=2, n_dm=3, dm_step=30.0, min_baselines=1)
    vis, cal, _ = make_data(wl, seed=21, n_pulses=2)
    a = gpu_search(wl, vis, cal)
    b = gpu_search(wl, vis, cal, precision=V.VOLKS_BF16)
    for d in range(wl.n_dm):
        for wi in range(len(wl.windows)):
            for bl in range(wl.n_bl):
                for x, y in zip(a.peaks(bl, d, wi), b.peaks(bl, d, wi)):
                    np.testing.assert_array_equal(x, y)
    a.close()
    b.close()


def test_plan_mixes_mixed_radix_and_power_of_two_bands():
    items = []
    rng_seed = 31
    for shape in (dict(n_if=12, n_chan=16, n_ap=240), dict(n_if=8, n_chan=16, n_ap=260),
                  dict(n_if=12, n_chan=64, n_ap=180)):
        wl = synth.small(**shape, n_bl=2, n_dm=3, dm_step=25.0, min_baselines=1)
        vis, cal, _ = make_data(wl, seed=rng_seed, n_pulses=1)
        rng_seed += 1
        items.append((wl, vis, cal))
    dev = [torch.from_numpy(v).cuda() for _, v, _ in items]
    plan = V.Plan([(wl, d, cal) for (wl, _, cal), d in zip(items, dev)], graph=True, autotune=True)
    plan.run(stream=torch.cuda.current_stream().cuda_stream)
    for i, (wl, vis, cal) in enumerate(items):
        ref = O.search(wl, vis, cal)
        r = plan.result(i)
        check_peaks(wl, r, ref, vis, cal)
        check_candidates(wl, r, ref, matched=True)
    plan.close()
