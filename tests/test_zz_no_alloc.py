"""The no-allocation entry point, volks_search_peaks_noalloc.

It serves callers that cannot allocate device memory while they run (a
real-time correlator loop that reserved the GPU at start-up, or a host
framework whose allocator owns the device budget): they pass device buffers
for the input and outputs and the library takes its scratch from one static
device array.  Checked here through the C ABI against the ordinary entry
point, volks_search_segment, on two calls in a row with different data, so
that anything left in the shared scratch by the first call would show up in
the second.  This file is collected last on purpose.
"""
import ctypes as C

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


def _data(wl, seed):
    rng = np.random.default_rng(seed)
    vis = synth.noise(wl, rng)
    cal = synth.draw_calibration(wl, rng)
    M = wl.pad_delay * wl.n_f
    synth.inject(vis, wl, cal, [synth.Pulse(float(wl.dms()[2]), 40 + seed, 3, 15.0,
                                            np.full(wl.n_bl, 21 / (M * wl.chan_bw_mhz * 1e6)),
                                            np.full(wl.n_bl, 4.0))])
    return vis, cal


def _layout(wl, nvalid):
    off, seg_per_bd = [], 0
    for w in wl.windows:
        off.append(seg_per_bd)
        seg_per_bd += wl.n_ap // w
    return off, seg_per_bd


def test_noalloc_matches_search_segment_on_two_calls_in_a_row():
    wl = synth.small(n_bl=2, n_ap=233, n_if=4, n_chan=32, n_dm=5, dm_step=50.0,
                     windows=(1, 2, 4, 8, 16, 32), min_baselines=1)
    stream = torch.cuda.current_stream().cuda_stream
    prm = V.make_params(wl)
    _, nvalid = V.volks_shift_table(wl.f_lo_mhz, wl.chan_bw_mhz, wl.n_f, wl.t_ap_s, wl.n_ap,
                                    wl.dm_lo, wl.dm_step, wl.n_dm)
    off, spb = _layout(wl, nvalid)
    M = wl.pad_delay * wl.n_f
    for seed in (1, 2):                      # two calls in a row, different data
        vis, cal = _data(wl, seed)
        dev = torch.from_numpy(vis).cuda()
        power = torch.full((wl.n_bl, wl.n_dm, spb), -7.0, device="cuda")
        cell = torch.full((wl.n_bl, wl.n_dm, spb), -7, dtype=torch.int32, device="cuda")
        calc = np.ascontiguousarray(cal)
        seg = V.volks_segment(wl.n_bl, wl.n_ap, wl.n_if, wl.n_chan, wl.t_ap_s, wl.f_lo_mhz,
                              wl.chan_bw_mhz, dev.data_ptr(),
                              calc.ctypes.data_as(C.POINTER(C.c_double)))
        V.volks_search_peaks_noalloc(seg, prm, stream, power.data_ptr(), cell.data_ptr())
        ref = V.Search(wl, dev, cal, stream=stream)           # the ordinary entry point
        orc = O.search(wl, vis, cal)                          # only to tell near-ties apart
        pw, cl = power.cpu().numpy(), cell.cpu().numpy()
        for b in range(wl.n_bl):
            for d in range(wl.n_dm):
                for wi, w in enumerate(wl.windows):
                    P, q, m = ref.peaks(b, d, wi)
                    n = len(P)
                    got_p = pw[b, d, off[wi]:off[wi] + n]
                    got_c = cl[b, d, off[wi]:off[wi] + n]
                    np.testing.assert_allclose(got_p, P, rtol=P_REL, atol=0)
                    want_c = q.astype(np.int64) * M + m
                    pk = orc.peaks[(b, d, w)]
                    tie = (pk.P - pk.P2) / np.maximum(pk.P, 1e-300) < TIE_REL
                    assert np.all((got_c == want_c) | tie), (seed, b, d, w)
                    # entries past the last segment are marked empty
                    rest = slice(off[wi] + n, off[wi] + wl.n_ap // w)
                    assert np.all(pw[b, d, rest] == 0) and np.all(cl[b, d, rest] == -1)
        ref.close()


def test_noalloc_rejects_a_segment_larger_than_its_scratch():
    wl = synth.small(n_bl=4, n_ap=30000, n_if=8, n_chan=64, n_dm=2)   # ~500 MB of scratch
    prm = V.make_params(wl)
    seg = V.volks_segment(wl.n_bl, wl.n_ap, wl.n_if, wl.n_chan, wl.t_ap_s, wl.f_lo_mhz,
                          wl.chan_bw_mhz, 1, None)   # never dereferenced
    with pytest.raises(V.VolksError) as e:
        V.volks_search_peaks_noalloc(seg, prm, 0, 1, 1)
    assert e.value.code == V.VOLKS_EINVAL
    assert "scratch" in str(e.value)
