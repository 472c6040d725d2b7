"""Re-fit of detected pulses (Sec. 3.1.2, volks_refit_pulses) against the
FP64 oracle: the same fine delay cell (or a cell within the near-tie bound
on the oracle's own grid), SNR and amplitude to the FP32 bound."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import volks_oracle as O
from paper_2108_05602_b300 import build, synth
from paper_2108_05602_b300 import volks as V

from test_gpu_parity import P_REL, TIE_REL, gpu_search, make_data

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    V.lib()


def oracle_power_at(X, shifts_row, c, t_ap, pad, m):
    Xd = O.dedisperse(X, shifts_row)[c["t0_ap"]:c["t1_ap"]]
    u = np.arange(len(Xd))
    S = (Xd * np.exp(-2j * np.pi * c["rate_hz"] * u * t_ap)[:, None]).sum(axis=0)
    Mc = pad * X.shape[1]
    k = np.arange(X.shape[1])
    return abs(np.sum(S * np.exp(-2j * np.pi * k * (m % Mc) / Mc))) ** 2


def check_refits(wl, vis, cal, cands, fits, pad):
    sh = O.shift_table(wl.f_lo_mhz, wl.chan_bw_mhz, wl.n_f, wl.dms(), wl.t_ap_s)
    Xc = {}
    n_tie = 0
    for c, f in zip(cands, fits):
        b = c["bl"]
        if b not in Xc:
            Xc[b] = O.calibrate(vis[b], cal[b], wl.n_if, wl.n_chan, wl.chan_bw_mhz)
        r = O.refit_pulse(Xc[b], sh[c["dm_idx"]], c["t0_ap"], c["t1_ap"], c["rate_hz"], wl.t_ap_s,
                          wl.chan_bw_mhz, pad, wl.n_f)
        assert f["n_ap"] == c["t1_ap"] - c["t0_ap"]
        assert math.isclose(f["snr"], r.snr, rel_tol=P_REL)
        assert math.isclose(f["amp"], r.amp, rel_tol=P_REL)
        if f["delay_idx"] != r.cell:
            p_gpu = oracle_power_at(Xc[b], sh[c["dm_idx"]], c, wl.t_ap_s, pad, f["delay_idx"])
            p_best = (r.snr ** 2) * (c["t1_ap"] - c["t0_ap"]) * wl.n_f
            assert p_gpu >= (1 - TIE_REL) * p_best, (c, f, r)
            n_tie += 1
        else:
            assert f["delay_s"] == r.tau_s
    return n_tie


@pytest.mark.parametrize("shape,pad", [(dict(n_if=8, n_chan=32, n_ap=400), 16),
                                       (dict(n_if=4, n_chan=16, n_ap=300), 32),
                                       (dict(n_if=12, n_chan=32, n_ap=260), 8),
                                       (dict(n_if=8, n_chan=64, n_ap=330), 4)],
                         ids=["256x16", "64x32", "384x8", "512x4"])
def test_refit_matches_oracle(shape, pad):
    wl = synth.small(n_bl=3, n_dm=4, dm_step=30.0, windows=(1, 2, 4, 8, 16), min_baselines=1, **shape)
    vis, cal, _ = make_data(wl, seed=shape["n_chan"] + pad, n_pulses=3)
    g = gpu_search(wl, vis, cal)
    cands = g.candidates()
    assert cands
    fits = g.refit(cands, pad=pad)
    n_tie = check_refits(wl, vis, cal, cands, fits, pad)
    assert n_tie <= max(1, len(cands) // 20)
    g.close()


def test_refit_of_plan_results_equals_the_single_search():
    wl = synth.small(n_bl=2, n_ap=300, n_if=8, n_chan=32, n_dm=3, dm_step=30.0, min_baselines=1)
    vis, cal, _ = make_data(wl, seed=71, n_pulses=2)
    g = gpu_search(wl, vis, cal)
    cands = g.candidates()
    a = g.refit(cands)
    d = torch.from_numpy(vis).cuda()
    plan = V.Plan([(wl, d, cal)], graph=True)
    plan.run(stream=torch.cuda.current_stream().cuda_stream)
    b = plan.result(0).refit(cands)
    assert a == b
    plan.close()
    g.close()


def test_refit_rejects_candidates_outside_the_search():
    wl = synth.small(n_bl=2, n_ap=200, n_if=4, n_chan=16, n_dm=2, dm_step=30.0, min_baselines=1)
    vis, cal, _ = make_data(wl, seed=72, n_pulses=1)
    g = gpu_search(wl, vis, cal)
    nv = g.shifts()[1]
    base = dict(bl=0, dm_idx=1, win=4, seg=0, t0_ap=0, t1_ap=4, g0_ap=0, g1_ap=4, delay_idx=0, rate_idx=0,
                n_windows=1, n_baselines=1, peak_power=0.0, rho=0.0, z=0.0, dm=30.0, delay_s=0.0, rate_hz=0.0)
    assert g.refit([base])[0]["n_ap"] == 4
    for bad in (dict(bl=2), dict(dm_idx=2), dict(t1_ap=int(nv[1]) + 1, t0_ap=int(nv[1]) - 3),
                dict(t0_ap=5, t1_ap=5)):
        with pytest.raises(V.VolksError) as e:
            g.refit([dict(base, **bad)])
        assert e.value.code == V.VOLKS_EINVAL
    with pytest.raises(V.VolksError):
        g.refit([base], pad=64)
    g.close()
