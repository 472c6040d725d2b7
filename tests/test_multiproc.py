"""The N > 1 host path on CPU: sharding, the max/sum step reduction the
benchmark uses, and a scan whose baselines are split over two gloo ranks,
gathered to rank 0 and cross-matched once by the library (a10), against the
single-process oracle."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import volks_oracle as O
from paper_2108_05602_b300 import build, shard, synth
from paper_2108_05602_b300 import volks as V


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    V.lib()


def test_shard_range_partitions_exactly():
    for n in range(0, 40):
        for world in range(1, 9):
            parts = [shard.shard_range(n, world, r) for r in range(world)]
            assert parts[0][0] == 0 and parts[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(parts, parts[1:]))
            sizes = [hi - lo for lo, hi in parts]
            assert max(sizes) - min(sizes) <= 1


def _as_abi(c, dms):
    return dict(bl=c["bl"], dm_idx=c["dm_idx"], win=c["win"], seg=c["seg"], t0_ap=c["t0"],
                t1_ap=c["t1"], g0_ap=c["g0"], g1_ap=c["g1"], delay_idx=c["delay_idx"],
                rate_idx=c["rate_idx"], n_windows=c["n_windows"], n_baselines=0,
                peak_power=c["peak_power"], rho=c["rho"], z=c["z"], dm=float(dms[c["dm_idx"]]),
                delay_s=c["delay_s"], rate_hz=c["rate_hz"])


def _key(c):
    return (c["dm_idx"], c["t0_ap"] if "t0_ap" in c else c["t0"], c["bl"], c["win"], c["seg"],
            c["n_baselines"])


def _workload():
    wl = synth.small(n_bl=6, n_ap=260, n_if=4, n_chan=16, n_dm=3, dm_step=60.0,
                     windows=(1, 2, 4, 8), min_baselines=3)
    rng = np.random.default_rng(17)
    vis = synth.noise(wl, rng)
    cal = synth.draw_calibration(wl, rng)
    M = wl.pad_delay * wl.n_f
    synth.inject(vis, wl, cal, [synth.Pulse(float(wl.dms()[1]), 80, 3, 25.0,
                                            rng.integers(-20, 20, wl.n_bl) / (M * 0.5e6),
                                            rng.uniform(-20, 20, wl.n_bl))])
    return wl, vis, cal


def test_library_cross_match_equals_oracle():
    wl, vis, cal = _workload()
    ref = O.search(wl, vis, cal, with_second=False)
    got = V.volks_cross_match([_as_abi(c, wl.dms()) for c in ref.matched], wl.min_baselines)
    want = ref.candidates
    assert sorted(map(_key, got)) == sorted(map(_key, want))
    assert any(c["n_baselines"] >= 3 for c in got)


def _rank_main(rank, world, port, out_path):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        wl, vis, cal = _workload()
        lo, hi = shard.shard_range(wl.n_bl, world, rank)
        import dataclasses
        sub = dataclasses.replace(wl, n_bl=hi - lo)
        res = O.search(sub, vis[lo:hi], cal[lo:hi], with_second=False)
        mine = [_as_abi(c, wl.dms()) for c in res.matched]
        merged = shard.gather_candidates(mine, bl_offset=lo)
        trials = sum(len(p.P) for p in res.peaks.values())
        tot, tmax = shard.reduce_step(trials, 1.0 + rank)
        if rank == 0:
            final = shard.merge_shards(merged, wl.min_baselines)
            torch.save({"final": final, "tot": tot, "tmax": tmax}, out_path)
    finally:
        dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_two_rank_gloo_baseline_shards_match_single_process(tmp_path):
    out = str(tmp_path / "rank0.pt")
    mp.spawn(_rank_main, args=(2, _free_port(), out), nprocs=2, join=True)
    got = torch.load(out, weights_only=False)
    wl, vis, cal = _workload()
    ref = O.search(wl, vis, cal, with_second=False)
    assert sorted(map(_key, got["final"])) == sorted(map(_key, ref.candidates))
    assert got["tot"] == sum(len(p.P) for p in ref.peaks.values())
    assert got["tmax"] == 2.0


def test_library_cross_match_equals_oracle_on_random_lists():
    """400 random per-baseline candidate lists (1-6 DMs, 1-12 baselines,
    intervals that chain, nest, touch or stand apart): the C cross-baseline
    match keeps the same entries with the same baseline counts, in
    (dm, t0, bl) order."""
    from oracle import volks_oracle as O
    rng = np.random.default_rng(99)
    for case in range(400):
        n_dm, n_bl = int(rng.integers(1, 7)), int(rng.integers(1, 13))
        cands = []
        for _ in range(int(rng.integers(0, 40))):
            w = int(2 ** rng.integers(0, 6))
            t0 = int(rng.integers(0, 200))
            cands.append(dict(bl=int(rng.integers(0, n_bl)), dm_idx=int(rng.integers(0, n_dm)), win=w,
                              seg=t0 // w, t0=t0, t1=t0 + w, g0=t0, g1=t0 + w, delay_idx=0, rate_idx=0,
                              n_windows=2, peak_power=1.0, rho=1.0, z=float(rng.uniform(3, 9)),
                              delay_s=0.0, rate_hz=0.0))
        min_bl = int(rng.integers(1, 5))
        by_dm = {}
        for c in cands:
            by_dm.setdefault(c["dm_idx"], []).append(c)
        want = []
        for d in sorted(by_dm):
            want.extend(O.cross_baseline(by_dm[d], min_bl))
        want = sorted(want, key=lambda c: (c["dm_idx"], c["t0"], c["bl"]))
        got = V.volks_cross_match([_as_abi(c, np.arange(n_dm, dtype=float)) for c in cands], min_bl)
        assert sorted(map(_key, got)) == sorted(map(_key, want)), case
        assert [(c["dm_idx"], c["t0_ap"], c["bl"]) for c in got] == \
            [(c["dm_idx"], c["t0"], c["bl"]) for c in want], case
