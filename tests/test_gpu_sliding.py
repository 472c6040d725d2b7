"""Sliding segments (volks_params.stride = 1: a segment starts at every
dedispersed AP) against the FP64 oracle, with the tolerances of
tests/test_gpu_parity.py."""
import dataclasses

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


SHAPES = [dict(n_bl=2, n_ap=150, n_if=4, n_chan=16, n_dm=3, dm_step=40.0, windows=(1, 2, 4, 8)),
          dict(n_bl=2, n_ap=133, n_if=8, n_chan=32, n_dm=2, dm_step=30.0, windows=(2, 8, 32)),
          dict(n_bl=1, n_ap=201, n_if=8, n_chan=64, n_dm=2, dm_step=20.0, windows=(1, 4, 16, 32)),
          dict(n_bl=2, n_ap=120, n_if=12, n_chan=16, n_dm=2, dm_step=30.0, windows=(2, 4, 8))]


@pytest.mark.parametrize("shape", SHAPES, ids=["64pt", "256pt-w32", "512pt", "192pt-mixed"])
@pytest.mark.parametrize("pad_rate", [4, 0])
def test_sliding_search_matches_oracle(shape, pad_rate):
    wl = synth.small(**shape, pad_rate=pad_rate, min_baselines=1)
    wl = dataclasses.replace(wl, stride=1)
    vis, cal, _ = make_data(wl, seed=shape["n_ap"] + pad_rate, n_pulses=2)
    g = gpu_search(wl, vis, cal)
    ref = O.search(wl, vis, cal)
    n, _ = check_peaks(wl, g, ref, vis, cal)
    assert n == sum(len(p.P) for p in ref.peaks.values())
    for (b, d, w), pk in ref.peaks.items():
        assert len(pk.P) == max(0, int(ref.nvalid[d]) - w + 1)
    check_candidates(wl, g, ref, matched=True)
    g.close()


def test_sliding_search_finds_a_pulse_between_back_to_back_segments():
    wl = dataclasses.replace(synth.small(n_bl=1, n_ap=200, n_if=8, n_chan=32, n_dm=1, windows=(4, 8),
                                         min_baselines=1), stride=1)
    rng = np.random.default_rng(81)
    vis = synth.noise(wl, rng)
    M = 4 * wl.n_f
    synth.inject(vis, wl, np.zeros((1, wl.n_if, 2)),
                 [synth.Pulse(0.0, 66, 4, 25.0, np.array([40 / (M * wl.chan_bw_mhz * 1e6)]), np.zeros(1))])
    g = gpu_search(wl, vis, None)
    hits = [c for c in g.candidates() if c["win"] == 4]
    assert any(c["t0_ap"] == 66 and c["delay_idx"] == 40 for c in hits)
    g.close()


def test_plan_mixes_sliding_and_back_to_back_segments():
    items = []
    for i, (shape, stride) in enumerate([(SHAPES[0], 1), (SHAPES[0], 0), (SHAPES[1], 1)]):
        wl = dataclasses.replace(synth.small(**shape, min_baselines=1, name=f"s{i}"), stride=stride)
        vis, cal, _ = make_data(wl, seed=90 + i, n_pulses=1)
        items.append((wl, vis, cal))
    dev = [torch.from_numpy(v).cuda() for _, v, _ in items]
    # each segment's parameters (and so its stride) come from its workload
    plan = V.Plan([(wl, d, cal) for (wl, _, cal), d in zip(items, dev)], graph=True, autotune=True)
    plan.run(stream=torch.cuda.current_stream().cuda_stream)
    for i, (wl, vis, cal) in enumerate(items):
        ref = O.search(wl, vis, cal)
        r = plan.result(i)
        check_peaks(wl, r, ref, vis, cal)
        check_candidates(wl, r, ref, matched=True)
    plan.close()


def test_reduced_precision_request_runs_fp32_when_sliding():
    wl = dataclasses.replace(synth.small(n_bl=2, n_ap=140, n_if=8, n_chan=32, n_dm=2, windows=(2, 4, 8, 16),
                                         min_baselines=1), stride=1)
    vis, cal, _ = make_data(wl, seed=95, n_pulses=1)
    a = gpu_search(wl, vis, cal)
    b = gpu_search(wl, vis, cal, precision=V.VOLKS_BF16)
    for d in range(wl.n_dm):
        for wi in range(len(wl.windows)):
            for bl in range(wl.n_bl):
                for x, y in zip(a.peaks(bl, d, wi), b.peaks(bl, d, wi)):
                    np.testing.assert_array_equal(x, y)
    a.close()
    b.close()


def test_noalloc_entry_point_refuses_sliding_segments():
    wl = synth.small(n_bl=1, n_ap=64, n_if=4, n_chan=16)
    vis = torch.zeros((1, wl.n_ap, wl.n_f), dtype=torch.complex64, device="cuda")
    seg = V.volks_segment()
    keep = V.fill_segment(seg, wl, vis)
    prm = V.make_params(wl, stride=1)
    pk = torch.zeros(1 << 16, dtype=torch.float32, device="cuda")
    cell = torch.zeros(1 << 16, dtype=torch.int32, device="cuda")
    with pytest.raises(V.VolksError) as e:
        V.volks_search_peaks_noalloc(seg, prm, torch.cuda.current_stream().cuda_stream, pk.data_ptr(),
                                     cell.data_ptr())
    assert e.value.code == V.VOLKS_EINVAL
    del keep
