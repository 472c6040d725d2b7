"""Batch plans (volks_plan_*): heterogeneous segments searched by shared
persistent launches, DM chunking, graph replay; every segment checked
against the FP64 oracle with the parity tolerances of test_gpu_parity."""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import volks_oracle as O
from paper_2108_05602_b300 import build, synth
from paper_2108_05602_b300 import volks as V

from test_gpu_parity import check_candidates, check_peaks, make_data

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    V.lib()


def _mixed():
    """Six segments of different bands, lengths, DM grids, windows, pads."""
    shapes = [
        dict(n_bl=2, n_ap=210, n_if=4, n_chan=16, n_dm=4, dm_step=40.0, windows=(1, 2, 4, 8)),
        dict(n_bl=1, n_ap=300, n_if=4, n_chan=32, n_dm=5, dm_step=30.0, windows=(2, 4, 8, 16)),
        dict(n_bl=3, n_ap=150, n_if=8, n_chan=32, n_dm=3, dm_step=20.0, windows=(1, 2, 4, 8, 16, 32)),
        dict(n_bl=1, n_ap=170, n_if=8, n_chan=64, n_dm=3, dm_step=25.0, windows=(1, 4, 16)),
        dict(n_bl=1, n_ap=120, n_if=8, n_chan=128, n_dm=2, dm_step=30.0, windows=(2, 8, 32)),
        dict(n_bl=2, n_ap=260, n_if=4, n_chan=16, n_dm=6, dm_step=35.0, windows=(1, 2, 4, 8),
             pad_rate=0),
    ]
    out = []
    for i, sh in enumerate(shapes):
        wl = synth.small(**sh, name=f"mix{i}", min_baselines=1)
        vis, cal, _ = make_data(wl, seed=100 + i)
        out.append((wl, vis, cal))
    return out


def _check_all(plan, items, refs):
    for i, (wl, vis, cal) in enumerate(items):
        r = plan.result(i)
        check_peaks(wl, r, refs[i], vis, cal)
        check_candidates(wl, r, refs[i])


@pytest.mark.parametrize("graph,autotune", [(True, True), (False, False)])
def test_plan_of_mixed_segments_matches_oracle(graph, autotune):
    items = _mixed()
    dev = [torch.from_numpy(v).cuda() for _, v, _ in items]
    plan = V.Plan([(wl, d, cal) for (wl, _, cal), d in zip(items, dev)], graph=graph,
                  autotune=autotune)
    plan.run(stream=torch.cuda.current_stream().cuda_stream)
    refs = [O.search(wl, vis, cal) for wl, vis, cal in items]
    _check_all(plan, items, refs)
    t = plan.timing()
    assert t.ms_search > 0 and t.n_search_launches >= 1
    # replay (same pointers) gives the same answers
    plan.run(stream=torch.cuda.current_stream().cuda_stream)
    _check_all(plan, items, refs)
    plan.close()


def test_one_shot_batch_matches_oracle():
    """volks_search_batch: create + one run in a single call."""
    items = _mixed()[:4]
    dev = [torch.from_numpy(v).cuda() for _, v, _ in items]
    plan = V.Plan([(wl, d, cal) for (wl, _, cal), d in zip(items, dev)],
                  one_shot_stream=torch.cuda.current_stream().cuda_stream)
    refs = [O.search(wl, vis, cal) for wl, vis, cal in items]
    _check_all(plan, items, refs)
    plan.close()


def test_plan_dm_chunks_match_oracle():
    items = _mixed()[:3]
    dev = [torch.from_numpy(v).cuda() for _, v, _ in items]
    # a peak budget far below one DM per segment forces one DM per round
    plan = V.Plan([(wl, d, cal) for (wl, _, cal), d in zip(items, dev)],
                  peak_budget_bytes=1, graph=True, autotune=False)
    info = plan.info()
    assert info["rounds"] == max(wl.n_dm for wl, _, _ in items)
    plan.run(stream=torch.cuda.current_stream().cuda_stream)
    refs = [O.search(wl, vis, cal) for wl, vis, cal in items]
    for i, (wl, vis, cal) in enumerate(items):
        r = plan.result(i)
        check_candidates(wl, r, refs[i])
        last = wl.n_dm - 1
        for wi, w in enumerate(wl.windows):
            P, q, m = r.peaks(0, last, wi)
            np.testing.assert_allclose(P, refs[i].peaks[(0, last, w)].P, rtol=1e-4)
            mu, sd = r.stats(0, 0, wi)
            assert abs(mu - refs[i].stats[(0, 0, w)][0]) <= 1e-4 * abs(mu)
        if wl.n_dm > 1:
            with pytest.raises(V.VolksError):
                r.peaks(0, 0, 0)
    plan.close()


def test_plan_new_visibilities_and_in_place_update():
    items = _mixed()[:2]
    dev = [torch.from_numpy(v).cuda() for _, v, _ in items]
    stream = torch.cuda.current_stream().cuda_stream
    plan = V.Plan([(wl, d, cal) for (wl, _, cal), d in zip(items, dev)], graph=True)
    plan.run(stream=stream)
    # new data in new buffers: the graph is re-captured
    items_b = []
    for i, (wl, _, cal) in enumerate(items):
        vis_b, _, _ = make_data(wl, seed=900 + i, with_cal=False)
        items_b.append((wl, vis_b, cal))
    dev_b = [torch.from_numpy(v).cuda() for _, v, _ in items_b]
    plan.run(vis=dev_b, stream=stream)
    _check_all(plan, items_b, [O.search(wl, v, c) for wl, v, c in items_b])
    # new data written into the same buffers: the captured graph is replayed
    items_c = []
    for i, (wl, _, cal) in enumerate(items):
        vis_c, _, _ = make_data(wl, seed=700 + i, with_cal=False)
        dev_b[i].copy_(torch.from_numpy(vis_c).cuda())
        items_c.append((wl, vis_c, cal))
    plan.run(stream=stream)
    _check_all(plan, items_c, [O.search(wl, v, c) for wl, v, c in items_c])
    plan.close()


def test_plan_rejects_host_visibilities():
    wl = synth.small()
    vis, cal, _ = make_data(wl, seed=1)
    with pytest.raises(V.VolksError) as e:
        V.Plan([(wl, vis, cal)])
    assert e.value.code == V.VOLKS_EINVAL
