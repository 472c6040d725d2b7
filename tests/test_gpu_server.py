"""The continuous-batching request server (volks_server_*): results alone
equal results in the mix, admission by device-memory budget, refusal of an
oversize request, host-side fault injection, bounded waits, and the
device-resident halo that carries a boundary-crossing pulse into the next
segment of a stream (checked against the FP64 oracle)."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import volks_oracle as O
from paper_2108_05602_b300 import build, synth
from paper_2108_05602_b300 import volks as V

from test_gpu_parity import check_candidates, make_data

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    V.lib()


def _requests(n=8):
    out = []
    for i in range(n):
        wl = synth.small(n_bl=1 + i % 3, n_ap=150 + 37 * i, n_if=4, n_chan=16 << (i % 4),
                         n_dm=3 + i % 3, dm_step=30.0, windows=(1, 2, 4, 8, 16, 32)[: 3 + i % 4],
                         min_baselines=1, name=f"req{i}")
        vis, cal, _ = make_data(wl, seed=300 + i)
        out.append((wl, vis, cal))
    return out


def _key(c):
    return (c["bl"], c["dm_idx"], c["win"], c["seg"], c["g0_ap"], c["g1_ap"], c["n_windows"],
            c["delay_idx"], c["rate_idx"])


class _Got:
    """Adapter: a collected server result seen as a search result."""

    def __init__(self, cands):
        self.cands = cands

    def candidates(self):
        return self.cands


def test_results_alone_equal_results_in_the_mix():
    reqs = _requests()
    alone = []
    for wl, vis, cal in reqs:
        s = V.Search(wl, torch.from_numpy(vis).cuda(), cal)
        alone.append(s.candidates())
        s.close()
    srv = V.Server(max_inflight=4, hbm_budget_bytes=8 << 30)
    devs = [torch.from_numpy(v).cuda() for _, v, _ in reqs]
    ids = [srv.submit(wl, d, cal) for (wl, _, cal), d in zip(reqs, devs)]
    for i, rid in enumerate(ids):
        info, got = srv.wait_all(rid)
        assert info.status == 0
        assert sorted(map(_key, got)) == sorted(map(_key, alone[i]))
        for a, b in zip(sorted(got, key=_key), sorted(alone[i], key=_key)):
            assert math.isclose(a["peak_power"], b["peak_power"], rel_tol=1e-4)
            assert abs(a["z"] - b["z"]) <= 1e-4 * max(1.0, abs(b["z"]))
    st = srv.stats()
    assert st.completed == len(reqs) and st.failed == 0 and st.peak_inflight >= 2
    assert st.p99_ms >= st.p50_ms > 0
    srv.close()


def test_budget_bounds_concurrency_and_oversize_is_refused():
    reqs = _requests(4)
    devs = [torch.from_numpy(v).cuda() for _, v, _ in reqs]
    srv = V.Server(max_inflight=4, hbm_budget_bytes=1)
    with pytest.raises(V.VolksError) as e:
        wl, _, cal = reqs[0]
        srv.submit(wl, devs[0], cal)
    assert e.value.code == V.VOLKS_ENOMEM
    srv.close()
    # learn each request's charge, then allow only the largest at a time
    srv = V.Server(max_inflight=4, hbm_budget_bytes=8 << 30)
    charge = []
    for (wl, _, cal), d in zip(reqs, devs):
        info, _ = srv.wait_all(srv.submit(wl, d, cal))
        charge.append(info.device_bytes)
    srv.close()
    budget = max(charge)
    assert sum(charge) > budget
    srv = V.Server(max_inflight=4, hbm_budget_bytes=budget)
    ids = [srv.submit(wl, d, cal) for (wl, _, cal), d in zip(reqs, devs)]
    for rid in ids:
        info, _ = srv.wait_all(rid)
        assert info.status == 0
    st = srv.stats()
    assert st.completed == 4 and st.peak_bytes <= budget and st.peak_inflight < 4
    srv.close()


def test_injected_allocation_failure_fails_one_request_only():
    reqs = _requests(6)
    devs = [torch.from_numpy(v).cuda() for _, v, _ in reqs]
    srv = V.Server(max_inflight=2, hbm_budget_bytes=8 << 30, fail_every=3)
    ids = [srv.submit(wl, d, cal) for (wl, _, cal), d in zip(reqs, devs)]
    ok = bad = 0
    for rid in ids:
        try:
            srv.wait_all(rid)
            ok += 1
        except V.VolksError as err:
            assert err.code == V.VOLKS_ENOMEM and "injected" in str(err)
            bad += 1
    assert bad == 2 and ok == 4
    assert srv.stats().failed == 2
    srv.close()


def test_wait_times_out_and_unknown_ids_are_rejected():
    wl = synth.small(n_bl=3, n_ap=2000, n_if=8, n_chan=64, n_dm=40, dm_step=10.0,
                     windows=(1, 2, 4, 8, 16, 32))
    vis, cal, _ = make_data(wl, seed=5, n_pulses=0)
    srv = V.Server(max_inflight=1, hbm_budget_bytes=8 << 30)
    rid = srv.submit(wl, torch.from_numpy(vis).cuda(), cal)
    with pytest.raises(V.VolksError) as e:
        srv.wait(rid, timeout_ms=0)
    assert e.value.code == V.VOLKS_ETIMEOUT
    srv.wait_all(rid)
    with pytest.raises(V.VolksError):
        srv.wait_all(rid)           # already collected
    srv.close()


def test_stream_halo_catches_a_pulse_across_the_boundary():
    """Three consecutive segments of one stream; a pulse arrives at the top
    of the band near the end of segment 0, its low-frequency part in
    segment 1.  Segment 0 alone cannot search it (its sweep runs past the
    end); segment 1, searched with the kept halo, finds it.  The server's
    answer for segment 1 equals the oracle on [halo | segment 1]."""
    wl_all = synth.small(n_bl=2, n_ap=3 * 240, n_if=4, n_chan=32, n_dm=4, dm_step=60.0,
                         windows=(1, 2, 4, 8), min_baselines=1)
    rng = np.random.default_rng(12)
    vis = synth.noise(wl_all, rng)
    cal = synth.draw_calibration(wl_all, rng)
    dm = float(wl_all.dms()[3])
    sweep = int(synth.arrival_offsets_ap(wl_all, dm).max())
    assert 10 < sweep < 200
    t0 = 240 - sweep // 2                      # straddles segments 0 and 1
    M = wl_all.pad_delay * wl_all.n_f
    synth.inject(vis, wl_all, cal, [synth.Pulse(dm, t0, 4, 30.0, np.full(2, 5 / (M * 0.5e6)),
                                                np.zeros(2))])
    import dataclasses
    wl = dataclasses.replace(wl_all, n_ap=240)
    segs = [np.ascontiguousarray(vis[:, 240 * k:240 * (k + 1)]) for k in range(3)]
    srv = V.Server(max_inflight=3, hbm_budget_bytes=8 << 30)
    devs = [torch.from_numpy(s).cuda() for s in segs]
    ids = [srv.submit(wl, d, cal, stream_id=7) for d in devs]
    res = [srv.wait_all(rid) for rid in ids]
    H = int(max(r.max() for r in O.shift_table(wl.f_lo_mhz, wl.chan_bw_mhz, wl.n_f, wl.dms(),
                                               wl.t_ap_s)))
    info1, c1 = res[1]
    assert info1.ap_offset == 240 - H
    # oracle on the extended input of segment 1
    ext = np.ascontiguousarray(vis[:, 240 - H:480])
    wl_ext = dataclasses.replace(wl, n_ap=ext.shape[1])
    ref = O.search(wl_ext, ext, cal)
    check_candidates(wl_ext, _Got(c1), ref, matched=False)
    hit = [c for c in c1 if c["dm_idx"] == 3 and c["g0_ap"] + info1.ap_offset <= t0 + 4
           and c["g1_ap"] + info1.ap_offset >= t0]
    assert hit, c1
    # segment 0 alone never reaches dedispersed AP t0 at this DM
    nv0 = 240 - sweep
    assert t0 >= nv0
    srv.close()
