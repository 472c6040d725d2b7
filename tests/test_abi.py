"""C-ABI checks that need no GPU: the library loads, exports every function
include/volks.h declares, its structs have the C layout, the host-only
shift table equals the oracle's bit for bit, and malformed descriptors are
rejected before any device work."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

from oracle import volks_oracle as O
from paper_2108_05602_b300 import build, synth
from paper_2108_05602_b300 import volks as V

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "volks.h")
HEADERS = [HEADER, os.path.join(ROOT, "include", "volks_check.h")]


@pytest.fixture(scope="module")
def L():
    build.build()
    return V.lib()


def declared_functions():
    src = "".join(open(h).read() for h in HEADERS)
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(volks_\w+)\s*\(", src)))


def test_exports_every_declared_symbol(L):
    names = declared_functions()
    assert "volks_search_segment" in names and "volks_candidates" in names and "volks_free" in names
    out = subprocess.run(["nm", "-D", "--defined-only", V.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\b(volks_\w+)\b", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert hasattr(L, n)
    # and nothing with the ABI's prefix is exported without a declaration
    undeclared = sorted(exported - set(names))
    assert not undeclared, undeclared


def test_struct_layout_matches_c(L):
    structs = {"volks_segment": V.volks_segment, "volks_params": V.volks_params,
               "volks_candidate": V.volks_candidate, "volks_timing": V.volks_timing,
               "volks_loc_obs": V.volks_loc_obs, "volks_loc_params": V.volks_loc_params,
               "volks_loc_result": V.volks_loc_result, "volks_refit": V.volks_refit}
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"', 'int main(void){']
    for sname, cls in structs.items():
        lines.append(f'printf("{sname} %zu\\n", sizeof({sname}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{sname}.{f} %zu\\n", offsetof({sname}, {f}));')
    lines.append("return 0;}")
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write("\n".join(lines))
        subprocess.run(["gcc", "-std=c99", "-o", exe, c], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    got = dict(l.rsplit(" ", 1) for l in out.strip().splitlines())
    for sname, cls in structs.items():
        assert int(got[sname]) == C.sizeof(cls), sname
        for f, _ in cls._fields_:
            assert int(got[f"{sname}.{f}"]) == getattr(cls, f).offset, (sname, f)


@pytest.mark.parametrize("wl", [synth.pr1(), synth.evn(), synth.small(n_if=4, n_chan=16)],
                         ids=["pr1", "evn", "small"])
def test_shift_table_bit_exact_vs_oracle(L, wl):
    sh, nv = V.volks_shift_table(wl.f_lo_mhz, wl.chan_bw_mhz, wl.n_f, wl.t_ap_s, wl.n_ap,
                                 wl.dm_lo, wl.dm_step, wl.n_dm)
    ref = O.shift_table(wl.f_lo_mhz, wl.chan_bw_mhz, wl.n_f, wl.dms(), wl.t_ap_s)
    assert np.array_equal(sh, ref)
    assert np.array_equal(nv, [O.n_valid(wl.n_ap, r) for r in ref])


def test_shift_table_bit_exact_vs_oracle_on_random_grids(L):
    """200 random bands (64-2048 and 96-1536 points, 0.0625-2 MHz channels,
    300 MHz-20 GHz), AP lengths and DM grids: identical integer shifts and
    valid counts (both sides round the same FP64 expression half-up)."""
    import dataclasses
    rng = np.random.default_rng(5)
    sizes = [64, 128, 256, 512, 1024, 2048, 96, 192, 384, 768, 1536]
    for _ in range(200):
        n_f = int(rng.choice(sizes))
        bw = float(2.0 ** rng.integers(-4, 2))
        wl = dataclasses.replace(synth.small(), n_if=1, n_chan=n_f, chan_bw_mhz=bw,
                                 f_lo_mhz=float(rng.uniform(300, 20000)),
                                 t_ap_s=float(rng.choice([1.024e-3, 0.512e-3, 2e-3, 1e-2])),
                                 n_ap=int(rng.integers(1, 100000)), dm_lo=float(rng.uniform(0, 500)),
                                 dm_step=float(rng.uniform(0.01, 20)), n_dm=int(rng.integers(1, 40)))
        sh, nv = V.volks_shift_table(wl.f_lo_mhz, wl.chan_bw_mhz, n_f, wl.t_ap_s, wl.n_ap,
                                     wl.dm_lo, wl.dm_step, wl.n_dm)
        ref = O.shift_table(wl.f_lo_mhz, wl.chan_bw_mhz, n_f, wl.dms(), wl.t_ap_s)
        assert np.array_equal(sh, ref)
        assert np.array_equal(nv, [O.n_valid(wl.n_ap, r) for r in ref])


def test_shift_table_large_dm_leaves_no_valid_ap(L):
    wl = synth.small(n_ap=40)
    sh, nv = V.volks_shift_table(wl.f_lo_mhz, wl.chan_bw_mhz, wl.n_f, wl.t_ap_s, 40,
                                 0.0, 5000.0, 3)
    assert nv[0] == 40 and nv[2] <= 0


def _seg(**kw):
    s = V.volks_segment()
    s.n_bl, s.n_ap, s.n_if, s.n_chan = 1, 64, 4, 16
    s.t_ap_s, s.f_lo_mhz, s.chan_bw_mhz = 1.024e-3, 1580.0, 0.5
    s.vis = 1  # never dereferenced: validation fails first
    for k, v in kw.items():
        if k == "bl_st" and v is not None:
            v = C.cast(v, C.POINTER(C.c_int32))
        setattr(s, k, v)
    return s


@pytest.mark.parametrize("seg_kw,prm_kw", [
    (dict(n_chan=15), {}),                       # n_f = 60 not a power of two
    (dict(n_if=64, n_chan=64), {}),              # n_f = 4096 not in this build
    (dict(n_if=3, n_chan=16), {}),               # n_f = 48: 3 x 2^a below 96
    (dict(n_if=12, n_chan=256), {}),             # n_f = 3072: 3 x 2^a above 1536
    (dict(n_if=5, n_chan=64), {}),               # n_f = 320: factor 5
    (dict(n_ap=-1), {}),
    (dict(t_ap_s=0.0), {}),
    (dict(chan_bw_mhz=-0.5), {}),
    (dict(vis=None), {}),
    ({}, dict(n_win=0)),
    ({}, dict(n_win=7)),
    ({}, dict(pad_delay=3)),
    ({}, dict(pad_rate=3)),
    ({}, dict(precision=4)),
    ({}, dict(precision=-1)),
    ({}, dict(dm_lo=-10.0)),
    ({}, dict(min_windows=0)),
    ({}, dict(normalize_chan=2)),
    ({}, dict(stride=2)),
    ({}, dict(stride=-1)),
    (dict(n_pol=3), {}),
    (dict(n_pol=-1), {}),
    (dict(autos=1, n_st=1, bl_st=(C.c_int32 * 2)(0, 1)), {}),        # one station
    (dict(autos=1, n_st=4, bl_st=None), {}),                           # no station pairs
    (dict(autos=1, n_st=4, bl_st=(C.c_int32 * 2)(0, 4)), {}),        # station out of range
    (dict(autos=1, n_st=4, bl_st=(C.c_int32 * 2)(2, 2)), {}),        # auto-correlation pair
])
def test_malformed_descriptors_rejected(L, seg_kw, prm_kw):
    seg = _seg(**seg_kw)
    prm = V.volks_default_params()
    for k, v in prm_kw.items():
        setattr(prm, k, v)
    out = C.c_void_p(123)
    rc = L.volks_search_segment(C.byref(seg), C.byref(prm), None, C.byref(out))
    assert rc == V.VOLKS_EINVAL
    assert out.value is None
    assert L.volks_last_error()


def test_windows_must_be_ascending_powers_of_two(L):
    for wins in ([2, 2], [4, 2], [3], [64]):
        prm = V.volks_default_params()
        prm.n_win = len(wins)
        for i, w in enumerate(wins):
            prm.win[i] = w
        out = C.c_void_p()
        assert L.volks_search_segment(C.byref(_seg()), C.byref(prm), None, C.byref(out)) == V.VOLKS_EINVAL


def test_null_arguments(L):
    out = C.c_void_p()
    assert L.volks_search_segment(None, None, None, C.byref(out)) == V.VOLKS_EINVAL
    assert L.volks_search_segment(C.byref(_seg()), C.byref(V.volks_default_params()), None, None) == V.VOLKS_EINVAL
    n = C.c_size_t()
    assert L.volks_candidates(None, None, 0, C.byref(n)) == V.VOLKS_EINVAL
    L.volks_free(None)  # NULL-safe
    plan = C.c_void_p(123)
    assert L.volks_search_batch(None, None, 0, None, C.byref(plan)) == V.VOLKS_EINVAL
    assert plan.value is None


def test_twiddle_series_matches_libm():
    """The compile-time sine/cosine used for register-FFT twiddles agrees
    with the C library to ~1 ulp for every angle the kernels use."""
    src = os.path.join(ROOT, "paper_2108_05602_b300", "csrc", "twiddle_ce.h")
    prog = f'''#include "{src}"
#include <cmath>
#include <cstdio>
int main() {{ double worst = 0;
  for (long long n = 1; n <= 4096; n *= 2) for (long long k = -n; k < 2 * n; ++k) {{
    double c = vk::cos2pi(k, n), s = vk::sin2pi(k, n);
    double a = 2.0 * M_PI * (double)k / (double)n;
    worst = std::fmax(worst, std::fabs(c - std::cos(a)));
    worst = std::fmax(worst, std::fabs(s - std::sin(a))); }}
  static_assert(vk::cos2pi(1, 4) == vk::series_cos(0.0) * 0.0 + vk::cos2pi(1, 4), "constexpr");
  printf("%.3e\\n", worst); return 0; }}'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.cc")
        exe = os.path.join(d, "t")
        open(c, "w").write(prog)
        subprocess.run(["g++", "-std=c++17", "-O1", "-o", exe, c], check=True)
        worst = float(subprocess.run([exe], capture_output=True, text=True, check=True).stdout)
    assert worst < 2e-15


def test_product_path_does_not_touch_the_oracle():
    pkg = os.path.join(ROOT, "paper_2108_05602_b300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"(from|import)\s+oracle\b|volks_oracle|oracle/", txt), f


def test_binding_rejects_a_visibility_array_of_the_wrong_shape():
    wl = synth.small(n_bl=2, n_ap=20, n_if=4, n_chan=16)
    seg = V.volks_segment()
    with pytest.raises(ValueError):
        V.fill_segment(seg, wl, np.zeros((2, 21, wl.n_f), dtype=np.complex64))
    keep = V.fill_segment(seg, wl, np.zeros((2, 2, 20, wl.n_f), dtype=np.complex64))
    assert seg.n_pol == 2 and seg.n_bl == 2 and seg.n_ap == 20
    del keep


def test_default_params_include_the_stride():
    p = V.volks_default_params()
    assert p.stride == 0
    wl = synth.small()
    import dataclasses
    assert V.make_params(dataclasses.replace(wl, stride=1)).stride == 1


def test_binding_checks_cal_autos_and_station_pairs_against_the_descriptor():
    wl = synth.small(n_bl=3, n_ap=20, n_if=4, n_chan=16)
    seg = V.volks_segment()
    vis2 = np.zeros((2, 3, 20, wl.n_f), dtype=np.complex64)
    with pytest.raises(ValueError):   # one product's table for two products
        V.fill_segment(seg, wl, vis2, np.zeros((3, wl.n_if, 2)))
    V.fill_segment(seg, wl, vis2, np.zeros((2, 3, wl.n_if, 2)))
    autos = np.ones((2, 3, 20, wl.n_f), dtype=np.float32)
    st = np.array([[0, 1], [0, 2], [1, 2]])
    keep = V.fill_segment(seg, wl, vis2, None, autos, st)
    assert seg.n_st == 3
    del keep
    with pytest.raises(ValueError):
        V.fill_segment(seg, wl, vis2, None, autos[:1], st)
    with pytest.raises(ValueError):
        V.fill_segment(seg, wl, vis2, None, autos, st[:2])


def test_noalloc_rejects_host_buffers_before_any_launch(L):
    """The no-allocation entry point refuses host memory for its input and
    outputs with VOLKS_EINVAL before it launches anything (on a machine
    without a GPU every pointer fails the check; the GPU test file checks
    the messages on a device)."""
    wl = synth.small(n_bl=1, n_ap=64, n_if=4, n_chan=16, n_dm=2, windows=(1, 2))
    prm = V.make_params(wl)
    spb = sum(wl.n_ap // w for w in wl.windows)
    vis = np.zeros((1, wl.n_ap, wl.n_f), dtype=np.complex64)
    pw = np.zeros((wl.n_bl, wl.n_dm, spb), dtype=np.float32)
    cl = np.zeros((wl.n_bl, wl.n_dm, spb), dtype=np.int32)
    seg = V.volks_segment(wl.n_bl, wl.n_ap, wl.n_if, wl.n_chan, wl.t_ap_s, wl.f_lo_mhz,
                          wl.chan_bw_mhz, vis.ctypes.data, None)
    rc = L.volks_search_peaks_noalloc(C.byref(seg), C.byref(prm), None, C.c_void_p(pw.ctypes.data),
                                      C.c_void_p(cl.ctypes.data))
    assert rc == V.VOLKS_EINVAL and L.volks_last_error()
    sh = np.zeros((wl.n_dm, wl.n_f), dtype=np.int32)
    nv = np.zeros(wl.n_dm, dtype=np.int32)
    rc = L.volks_noalloc_tables(None, C.c_void_p(sh.ctypes.data), C.c_void_p(nv.ctypes.data),
                                wl.n_dm, wl.n_f)
    assert rc == V.VOLKS_EINVAL
