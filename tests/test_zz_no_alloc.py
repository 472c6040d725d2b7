"""The no-allocation entry point, volks_search_peaks_noalloc.

It serves callers that cannot allocate device memory while they run (a
real-time correlator loop that reserved the GPU at start-up, or a host
framework whose allocator owns the device budget): they pass device buffers
for the input and outputs and the library takes its scratch from one static
device array.  Checked here through the C ABI against the FP64 oracle and
against the ordinary entry point, volks_search_segment, on a run of calls in
a row that change every size and option (a large call first, then smaller
ones), so that anything the shared scratch keeps from one call would show up
in the next.  The device-computed shift table of each call is read back and
compared with the oracle's bit for bit.  This file is collected last on
purpose.
"""
import ctypes as C
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import volks_oracle as O
from paper_2108_05602_b300 import build, synth
from paper_2108_05602_b300 import volks as V

pytestmark = pytest.mark.gpu

P_REL = 1e-4     # the FP32 tolerance the parity tests use
TIE_REL = 2e-5   # near-tied top-2 cells: either cell is a correct answer


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    V.lib()


def _data(wl, seed, with_cal=True):
    rng = np.random.default_rng(seed)
    vis = synth.noise(wl, rng)
    cal = synth.draw_calibration(wl, rng)
    M = wl.pad_delay * wl.n_f
    d = min(2, wl.n_dm - 1)
    synth.inject(vis, wl, cal, [synth.Pulse(float(wl.dms()[d]), 40 + seed % 20, 3, 15.0,
                                            np.full(wl.n_bl, 21 / (M * wl.chan_bw_mhz * 1e6)),
                                            np.full(wl.n_bl, 4.0))])
    return vis, (cal if with_cal else None)


def _offsets(wl):
    off, spb = [], 0
    for w in wl.windows:
        off.append(spb)
        spb += wl.n_ap // w
    return off, spb


def _segment(wl, dev, cal):
    calc = None if cal is None else np.ascontiguousarray(cal, dtype=np.float64)
    seg = V.volks_segment(wl.n_bl, wl.n_ap, wl.n_if, wl.n_chan, wl.t_ap_s, wl.f_lo_mhz,
                          wl.chan_bw_mhz, dev.data_ptr(),
                          None if calc is None else calc.ctypes.data_as(C.POINTER(C.c_double)))
    return seg, calc


def _noalloc(wl, dev, cal, stream, **over):
    """One no-allocation call: (power, cell) on the host, plus the device
    shift table and n_valid read back from the scratch."""
    _, spb = _offsets(wl)
    prm = V.make_params(wl, **over)
    power = torch.full((wl.n_bl, wl.n_dm, spb), -7.0, device="cuda")
    cell = torch.full((wl.n_bl, wl.n_dm, spb), -7, dtype=torch.int32, device="cuda")
    seg, _keep = _segment(wl, dev, cal)
    V.volks_search_peaks_noalloc(seg, prm, stream, power.data_ptr(), cell.data_ptr())
    sh = torch.full((wl.n_dm, wl.n_f), -7, dtype=torch.int32, device="cuda")
    nv = torch.full((wl.n_dm,), -7, dtype=torch.int32, device="cuda")
    V.volks_noalloc_tables(stream, sh.data_ptr(), nv.data_ptr(), wl.n_dm, wl.n_f)
    return power.cpu().numpy(), cell.cpu().numpy(), sh.cpu().numpy(), nv.cpu().numpy()


def _check_call(wl, vis, cal, stream, normalize=1, skip=0):
    dev = torch.from_numpy(vis).cuda()
    pw, cl, sh, nv = _noalloc(wl, dev, cal, stream, normalize_chan=normalize, skip_first_chan=skip)
    orc = O.search(wl, vis, cal, normalize=bool(normalize), skip_first_chan=bool(skip))
    # the device-computed tables equal the oracle's bit for bit
    assert np.array_equal(sh, orc.shifts) and np.array_equal(nv, orc.nvalid)
    ref = V.Search(wl, dev, cal, stream=stream, normalize_chan=normalize, skip_first_chan=skip)
    off, _ = _offsets(wl)
    M = wl.pad_delay * wl.n_f
    for b in range(wl.n_bl):
        for d in range(wl.n_dm):
            for wi, w in enumerate(wl.windows):
                pk = orc.peaks[(b, d, w)]
                n = len(pk.P)
                assert n == max(0, int(orc.nvalid[d])) // w
                got_p = pw[b, d, off[wi]:off[wi] + n]
                got_c = cl[b, d, off[wi]:off[wi] + n].astype(np.int64)
                # against the oracle
                np.testing.assert_allclose(got_p, pk.P, rtol=P_REL, atol=0)
                tie = (pk.P - pk.P2) / np.maximum(pk.P, 1e-300) < TIE_REL
                assert np.all((got_c == pk.q.astype(np.int64) * M + pk.m) | tie), (b, d, w)
                # against the ordinary entry point
                P, q, m = ref.peaks(b, d, wi)
                assert len(P) == n
                np.testing.assert_allclose(got_p, P, rtol=P_REL, atol=0)
                assert np.all((got_c == q.astype(np.int64) * M + m) | tie), (b, d, w)
                # entries past the last segment are marked empty
                rest = slice(off[wi] + n, off[wi] + wl.n_ap // w)
                assert np.all(pw[b, d, rest] == 0) and np.all(cl[b, d, rest] == -1)
    ref.close()
    return orc


def test_noalloc_matches_search_segment_on_two_calls_in_a_row():
    wl = synth.small(n_bl=2, n_ap=233, n_if=4, n_chan=32, n_dm=5, dm_step=50.0,
                     windows=(1, 2, 4, 8, 16, 32), min_baselines=1)
    stream = torch.cuda.current_stream().cuda_stream
    for seed in (1, 2):                      # two calls in a row, different data
        vis, cal = _data(wl, seed)
        _check_call(wl, vis, cal, stream)


# a large call first, then smaller ones that change every size and option
SEQUENCE = [
    dict(shape=dict(n_bl=3, n_ap=400, n_if=8, n_chan=64, n_dm=6, dm_step=40.0,
                    windows=(1, 2, 4, 8, 16, 32)), cal=True),
    dict(shape=dict(n_bl=1, n_ap=150, n_if=4, n_chan=16, n_dm=4, dm_step=60.0, windows=(2, 8),
                    pad_rate=0), cal=False),
    dict(shape=dict(n_bl=2, n_ap=233, n_if=4, n_chan=32, n_dm=5, dm_step=50.0,
                    windows=(1, 4, 16)), pad_delay=2, skip=1, cal=True),
    dict(shape=dict(n_bl=1, n_ap=200, n_if=8, n_chan=32, n_dm=3, dm_step=30.0,
                    windows=(1, 2, 4, 8, 16, 32)), pad_delay=8, normalize=0, cal=True),
    # the largest DM trials sweep past the end of the scan: no valid AP
    dict(shape=dict(n_bl=1, n_ap=120, n_if=4, n_chan=16, n_dm=6, dm_step=400.0,
                    windows=(1, 2, 4)), cal=False, runs_out=True),
]


def test_noalloc_sequence_of_shapes_and_options():
    stream = torch.cuda.current_stream().cuda_stream
    for i, case in enumerate(SEQUENCE):
        wl = synth.small(**case["shape"], min_baselines=1, name=f"seq{i}")
        if "pad_delay" in case:
            wl = dataclasses.replace(wl, pad_delay=case["pad_delay"])
        vis, cal = _data(wl, 10 + i, with_cal=case["cal"])
        orc = _check_call(wl, vis, cal, stream, normalize=case.get("normalize", 1),
                          skip=case.get("skip", 0))
        if case.get("runs_out"):
            assert (orc.nvalid <= 0).any() and (orc.nvalid > 0).any()


@pytest.mark.parametrize("n_if,n_chan,t_ap_s,f_lo", [(8, 64, 1.024e-3, 1472.0), (4, 16, 5.12e-4, 1600.0),
                                                      (8, 32, 2.048e-3, 4990.25), (4, 32, 1.024e-3, 327.5)])
def test_noalloc_device_shift_table_bit_exact_on_a_wide_dm_grid(n_if, n_chan, t_ap_s, f_lo):
    """The no-allocation call computes its shift table on the GPU; the
    ordinary path computes it on the host.  Over a wide DM grid (0..2000 in
    steps of 0.37) both must equal the oracle's table exactly, ties of
    x + 0.5 included."""
    wl = synth.small(n_bl=1, n_ap=64, n_if=n_if, n_chan=n_chan, n_dm=5406, dm_step=0.37,
                     windows=(1, 2), min_baselines=1)
    wl = dataclasses.replace(wl, t_ap_s=t_ap_s, f_lo_mhz=f_lo)
    stream = torch.cuda.current_stream().cuda_stream
    dev = torch.zeros((1, wl.n_ap, wl.n_f), dtype=torch.complex64, device="cuda")
    _, _, sh, nv = _noalloc(wl, dev, None, stream)
    want = O.shift_table(wl.f_lo_mhz, wl.chan_bw_mhz, wl.n_f, wl.dms(), wl.t_ap_s)
    want_nv = np.array([O.n_valid(wl.n_ap, r) for r in want])
    assert np.array_equal(sh, want) and np.array_equal(nv, want_nv)
    host_sh, host_nv = V.volks_shift_table(wl.f_lo_mhz, wl.chan_bw_mhz, wl.n_f, wl.t_ap_s, wl.n_ap,
                                           wl.dm_lo, wl.dm_step, wl.n_dm)
    assert np.array_equal(host_sh, sh) and np.array_equal(host_nv, nv)


def test_noalloc_rejects_host_outputs_and_other_buffers():
    wl = synth.small(n_bl=1, n_ap=64, n_if=4, n_chan=16, n_dm=2, windows=(1, 2))
    _, spb = _offsets(wl)
    prm = V.make_params(wl)
    dev = torch.zeros((1, wl.n_ap, wl.n_f), dtype=torch.complex64, device="cuda")
    seg, _keep = _segment(wl, dev, None)
    host_p = np.zeros((wl.n_bl, wl.n_dm, spb), dtype=np.float32)
    host_c = np.zeros((wl.n_bl, wl.n_dm, spb), dtype=np.int32)
    good_p = torch.zeros((wl.n_bl, wl.n_dm, spb), device="cuda")
    good_c = torch.zeros((wl.n_bl, wl.n_dm, spb), dtype=torch.int32, device="cuda")
    for pp, cc, name in [(host_p.ctypes.data, good_c.data_ptr(), "peak_power"),
                         (good_p.data_ptr(), host_c.ctypes.data, "peak_cell")]:
        with pytest.raises(V.VolksError) as e:
            V.volks_search_peaks_noalloc(seg, prm, 0, pp, cc)
        assert e.value.code == V.VOLKS_EINVAL and name in str(e.value)
    # a host visibility buffer is refused as well
    hv = np.zeros((1, wl.n_ap, wl.n_f), dtype=np.complex64)
    hseg = V.volks_segment(wl.n_bl, wl.n_ap, wl.n_if, wl.n_chan, wl.t_ap_s, wl.f_lo_mhz,
                           wl.chan_bw_mhz, hv.ctypes.data, None)
    with pytest.raises(V.VolksError) as e:
        V.volks_search_peaks_noalloc(hseg, prm, 0, good_p.data_ptr(), good_c.data_ptr())
    assert e.value.code == V.VOLKS_EINVAL and "vis" in str(e.value)
    # the context is still usable
    torch.cuda.synchronize()


def test_noalloc_rejects_a_segment_larger_than_its_scratch():
    wl = synth.small(n_bl=4, n_ap=30000, n_if=8, n_chan=64, n_dm=2)   # ~500 MB of scratch
    prm = V.make_params(wl)
    seg = V.volks_segment(wl.n_bl, wl.n_ap, wl.n_if, wl.n_chan, wl.t_ap_s, wl.f_lo_mhz,
                          wl.chan_bw_mhz, 1, None)   # never dereferenced
    with pytest.raises(V.VolksError) as e:
        V.volks_search_peaks_noalloc(seg, prm, 0, 1, 1)
    assert e.value.code == V.VOLKS_EINVAL
    assert "scratch" in str(e.value)
