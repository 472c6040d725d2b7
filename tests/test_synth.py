"""The seeded input generators that both the oracle and the CUDA path
consume: deterministic for a seed, the shapes and layouts the boundary
documents, and the statistics their models state (CPU)."""
import numpy as np
import pytest

from paper_2108_05602_b300 import synth


def test_generators_are_deterministic_for_a_seed():
    wl = synth.small(n_bl=3, n_ap=50, n_if=4, n_chan=16)
    a = synth.noise(wl, np.random.default_rng(7))
    b = synth.noise(wl, np.random.default_rng(7))
    np.testing.assert_array_equal(a, b)
    pa = synth.dual_pol_scan(wl, np.random.default_rng(8), [])
    pb = synth.dual_pol_scan(wl, np.random.default_rng(8), [])
    for x, y in zip(pa, pb):
        np.testing.assert_array_equal(x, y)


def test_shapes_and_layouts():
    wl = synth.small(n_bl=4, n_ap=30, n_if=8, n_chan=32)
    rng = np.random.default_rng(9)
    vis = synth.noise(wl, rng)
    assert vis.shape == (4, 30, 256) and vis.dtype == np.complex64 and vis.flags.c_contiguous
    cal = synth.draw_calibration(wl, rng)
    assert cal.shape == (4, 8, 2)
    v2, c2, autos, bl_st, g = synth.dual_pol_scan(wl, rng, [])
    assert v2.shape == (2, 4, 30, 256) and c2.shape == (2, 4, 8, 2)
    n_st = autos.shape[1]
    assert n_st * (n_st - 1) // 2 >= 4 and autos.shape == (2, n_st, 30, 256) and autos.dtype == np.float32
    assert bl_st.shape == (4, 2) and np.all(bl_st[:, 0] < bl_st[:, 1]) and bl_st.max() < n_st
    assert len({tuple(p) for p in bl_st}) == 4          # distinct station pairs


def test_noise_and_bandpass_statistics():
    """Unit-variance components; cross spectra scaled by sqrt(g_i g_j) and
    auto spectra g (1 + 0.01 N(0, 1))."""
    wl = synth.small(n_bl=3, n_ap=4000, n_if=4, n_chan=16)
    rng = np.random.default_rng(10)
    vis = synth.noise(wl, rng)
    assert abs(vis.real.var() - 1) < 0.02 and abs(vis.imag.var() - 1) < 0.02
    v2, _, autos, bl_st, g = synth.dual_pol_scan(wl, rng, [], auto_jitter=0.01)
    p, b = 1, 2
    i, j = bl_st[b]
    ratio = (np.abs(v2[p, b]) ** 2).mean(axis=0) / (2 * g[p, i] * g[p, j])
    assert abs(ratio.mean() - 1) < 0.02
    rel = autos[p, i] / g[p, i][None, :] - 1
    assert abs(rel.std() - 0.01) < 0.001


def test_calibration_on_grid_draws_grid_delays():
    wl = synth.small(n_bl=2, n_ap=10, n_if=4, n_chan=32)
    cal = synth.draw_calibration_on_grid(wl, np.random.default_rng(11))
    cells = cal[..., 0] * (4 * wl.n_chan * wl.chan_bw_mhz * 1e6)
    np.testing.assert_allclose(cells, np.round(cells), atol=1e-9)


def test_bench_flop_and_trial_counts_by_hand():
    """The nominal counts behind the reported roofline: 1 baseline, 64
    points (M = 256), windows 1 and 2, 10 dedispersed APs.
      delay FFTs   10 x 5 x 256 x log2 256          = 102,400
      w = 1        10 segments x 256 cells x 3       =   7,680
      w = 2        5 x 256 columns x 5 x 8 x log2 8  = 153,600
                   + 5 x 8 x 256 cells x 3           =  30,720
    total 294,400 flops; trials 10 + 5 = 15."""
    import bench
    wl = synth.small(n_bl=1, n_ap=10, n_if=4, n_chan=16, n_dm=1, windows=(1, 2))
    assert bench.algorithmic_flops(wl, [10]) == 294400.0
    assert bench.trial_count(wl, [10]) == 15


def test_bench_traffic_scaling_applies_only_to_the_captured_baseline_shape():
    """roofline.traffic scales the committed one-baseline DRAM capture:
    reads by baselines, writes by trials, and only for workloads whose
    baselines have the captured shape (58,594 APs x 512 points)."""
    import json
    import os
    import bench
    with open(os.path.join(bench.ROOT, "profiles", bench.TRAFFIC_FILE)) as f:
        cap = json.load(f)
    if cap.get("kernel_hash") != bench.kernel_source_hash():
        pytest.skip("the committed capture predates the current kernel sources")
    evn = bench.workload("evn_fp32")
    t = bench.traffic_per_launch(evn, 2 * cap["trials"])
    assert t["read"] == cap["dram_read_bytes"] * 15
    assert t["write"] == cap["dram_write_bytes"] * 2
    assert bench.traffic_per_launch(bench.workload("band1024_1bl"), cap["trials"]) is None
    assert bench.traffic_per_launch(bench.workload("band2048_1bl"), cap["trials"]) is None
