"""ctypes binding of libvolks.so (include/volks.h), names as in the C ABI.

Argument marshalling only: every step of the search runs in the library's
CUDA kernels (and its host driver for the shift table and the
cross-baseline match).  Loading fails loudly if the library is missing;
there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvolks.so")

VOLKS_OK, VOLKS_EINVAL, VOLKS_ENOMEM, VOLKS_ETIMEOUT, VOLKS_ECUDA = 0, -1, -2, -3, -4
VOLKS_FP32, VOLKS_BF16, VOLKS_FP16, VOLKS_FP8 = 0, 1, 2, 3
VOLKS_PLAN_AUTOTUNE, VOLKS_PLAN_GRAPH = 1, 2


class volks_segment(C.Structure):
    _fields_ = [("n_bl", C.c_int32), ("n_ap", C.c_int32), ("n_if", C.c_int32),
                ("n_chan", C.c_int32), ("t_ap_s", C.c_double), ("f_lo_mhz", C.c_double),
                ("chan_bw_mhz", C.c_double), ("vis", C.c_void_p),
                ("cal", C.POINTER(C.c_double)), ("n_pol", C.c_int32), ("n_st", C.c_int32),
                ("bl_st", C.POINTER(C.c_int32)), ("autos", C.c_void_p)]


class volks_params(C.Structure):
    _fields_ = [("dm_lo", C.c_double), ("dm_step", C.c_double), ("n_dm", C.c_int32),
                ("n_win", C.c_int32), ("win", C.c_int32 * 8), ("pad_delay", C.c_int32),
                ("pad_rate", C.c_int32), ("thresh", C.c_double),
                ("min_windows", C.c_int32), ("min_baselines", C.c_int32),
                ("precision", C.c_int32), ("normalize_chan", C.c_int32),
                ("skip_first_chan", C.c_int32), ("stride", C.c_int32)]


class volks_candidate(C.Structure):
    _fields_ = [("bl", C.c_int32), ("dm_idx", C.c_int32), ("win", C.c_int32),
                ("seg", C.c_int32), ("t0_ap", C.c_int32), ("t1_ap", C.c_int32),
                ("g0_ap", C.c_int32), ("g1_ap", C.c_int32), ("delay_idx", C.c_int32),
                ("rate_idx", C.c_int32), ("n_windows", C.c_int32),
                ("n_baselines", C.c_int32), ("peak_power", C.c_float), ("_pad", C.c_float),
                ("rho", C.c_double), ("z", C.c_double), ("dm", C.c_double),
                ("delay_s", C.c_double), ("rate_hz", C.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "_pad"}


class volks_timing(C.Structure):
    _fields_ = [("ms_h2d", C.c_float), ("ms_prep", C.c_float), ("ms_search", C.c_float),
                ("ms_select", C.c_float), ("ms_match", C.c_float),
                ("n_launches", C.c_int32), ("n_search_launches", C.c_int32)]


class volks_server_config(C.Structure):
    _fields_ = [("max_inflight", C.c_int32), ("fail_every", C.c_int32),
                ("hbm_budget_bytes", C.c_int64)]


class volks_request_info(C.Structure):
    _fields_ = [("status", C.c_int32), ("_pad", C.c_int32), ("queue_ms", C.c_double),
                ("latency_ms", C.c_double), ("device_bytes", C.c_int64),
                ("ap_offset", C.c_int64), ("trials", C.c_int64)]


class volks_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("failed", C.c_int64),
                ("queued", C.c_int32), ("inflight", C.c_int32), ("peak_inflight", C.c_int32),
                ("_pad", C.c_int32), ("bytes_in_use", C.c_int64), ("peak_bytes", C.c_int64),
                ("p50_ms", C.c_double), ("p99_ms", C.c_double), ("mean_ms", C.c_double),
                ("trials", C.c_int64), ("trials_per_s", C.c_double)]


class volks_refit(C.Structure):
    _fields_ = [("delay_s", C.c_double), ("snr", C.c_double), ("amp", C.c_double),
                ("delay_idx", C.c_int32), ("n_ap", C.c_int32)]


class volks_loc_obs(C.Structure):
    _fields_ = [("tau_s", C.c_double), ("tau_cal_s", C.c_double), ("dtau_dalpha", C.c_double),
                ("dtau_ddelta", C.c_double), ("snr", C.c_double), ("proj_len_m", C.c_double)]


class volks_loc_params(C.Structure):
    _fields_ = [("min_snr", C.c_double), ("max_proj_len_m", C.c_double),
                ("min_baselines", C.c_int32), ("outlier_factor", C.c_double)]


class volks_loc_result(C.Structure):
    _fields_ = [("status", C.c_int32), ("n_used", C.c_int32), ("outlier", C.c_int32),
                ("x", C.c_double * 2), ("cov", C.c_double * 4), ("rms_s", C.c_double),
                ("x_clean", C.c_double * 2)]


_lib: Optional[C.CDLL] = None


def lib() -> C.CDLL:
    """Load libvolks.so from the package directory (built by build.py)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libvolks.so not built at {LIB_PATH}; run "
                          "python -m paper_2108_05602_b300.build")
    L = C.CDLL(LIB_PATH)
    P, I32, SZ = C.c_void_p, C.c_int32, C.c_size_t
    L.volks_default_params.argtypes = [C.POINTER(volks_params)]
    L.volks_default_params.restype = None
    L.volks_search_segment.argtypes = [C.POINTER(volks_segment), C.POINTER(volks_params), P,
                                       C.POINTER(P)]
    L.volks_search_segment.restype = C.c_int
    L.volks_candidates.argtypes = [P, C.POINTER(volks_candidate), SZ, C.POINTER(SZ)]
    L.volks_candidates.restype = C.c_int
    L.volks_free.argtypes = [P]
    L.volks_free.restype = None
    L.volks_last_error.argtypes = []
    L.volks_last_error.restype = C.c_char_p
    L.volks_shift_table.argtypes = [C.c_double, C.c_double, I32, C.c_double, I32, C.c_double,
                                    C.c_double, I32, C.POINTER(I32), C.POINTER(I32)]
    L.volks_shift_table.restype = C.c_int
    L.volks_result_timing.argtypes = [P, C.POINTER(volks_timing)]
    L.volks_result_timing.restype = C.c_int
    L.volks_result_shifts.argtypes = [P, C.POINTER(I32), C.POINTER(I32)]
    L.volks_result_shifts.restype = C.c_int
    L.volks_result_peaks.argtypes = [P, I32, I32, I32, C.POINTER(C.c_float), C.POINTER(I32),
                                     C.POINTER(I32), SZ, C.POINTER(SZ)]
    L.volks_result_peaks.restype = C.c_int
    L.volks_result_stats.argtypes = [P, I32, I32, I32, C.POINTER(C.c_double),
                                     C.POINTER(C.c_double)]
    L.volks_result_stats.restype = C.c_int
    L.volks_result_gains.argtypes = [P, C.POINTER(C.c_float), SZ]
    L.volks_result_gains.restype = C.c_int
    L.volks_plan_create.argtypes = [C.POINTER(volks_segment), C.POINTER(volks_params), I32,
                                    C.c_int64, I32, C.POINTER(P)]
    L.volks_plan_create.restype = C.c_int
    L.volks_plan_run.argtypes = [P, C.POINTER(P), P]
    L.volks_plan_run.restype = C.c_int
    L.volks_plan_result.argtypes = [P, I32, C.POINTER(P)]
    L.volks_plan_result.restype = C.c_int
    L.volks_plan_timing.argtypes = [P, C.POINTER(volks_timing)]
    L.volks_plan_timing.restype = C.c_int
    L.volks_plan_info.argtypes = [P, C.POINTER(I32), C.POINTER(C.c_int64), C.POINTER(I32)]
    L.volks_plan_info.restype = C.c_int
    L.volks_plan_free.argtypes = [P]
    L.volks_plan_free.restype = None
    L.volks_server_create.argtypes = [C.POINTER(volks_server_config), C.POINTER(P)]
    L.volks_server_create.restype = C.c_int
    L.volks_server_submit.argtypes = [P, C.POINTER(volks_segment), C.POINTER(volks_params),
                                      C.c_int64, C.POINTER(C.c_uint64)]
    L.volks_server_submit.restype = C.c_int
    L.volks_server_wait.argtypes = [P, C.c_uint64, I32, C.POINTER(volks_candidate), SZ,
                                    C.POINTER(SZ), C.POINTER(volks_request_info)]
    L.volks_server_wait.restype = C.c_int
    L.volks_server_get_stats.argtypes = [P, C.POINTER(volks_server_stats)]
    L.volks_server_get_stats.restype = C.c_int
    L.volks_server_drain.argtypes = [P, I32]
    L.volks_server_drain.restype = C.c_int
    L.volks_server_free.argtypes = [P]
    L.volks_server_free.restype = None
    L.volks_cross_match.argtypes = [C.POINTER(volks_candidate), SZ, I32,
                                    C.POINTER(volks_candidate), SZ, C.POINTER(SZ)]
    L.volks_cross_match.restype = C.c_int
    L.volks_search_peaks_noalloc.argtypes = [C.POINTER(volks_segment), C.POINTER(volks_params),
                                             P, P, P]
    L.volks_search_peaks_noalloc.restype = C.c_int
    L.volks_noalloc_tables.argtypes = [P, P, P, I32, I32]
    L.volks_noalloc_tables.restype = C.c_int
    L.volks_fringe_fit_calibrator.argtypes = [C.POINTER(volks_segment), I32, P, C.POINTER(C.c_double),
                                              C.POINTER(C.c_double)]
    L.volks_fringe_fit_calibrator.restype = C.c_int
    L.volks_fine_calibration.argtypes = [C.POINTER(volks_segment), I32, P, C.POINTER(C.c_double),
                                         C.POINTER(C.c_double)]
    L.volks_fine_calibration.restype = C.c_int
    L.volks_check_rate_gemm.argtypes = [P, I32, I32, I32, P]
    L.volks_check_rate_gemm.restype = C.c_int
    L.volks_search_batch.argtypes = [C.POINTER(volks_segment), C.POINTER(volks_params), I32, P,
                                     C.POINTER(P)]
    L.volks_search_batch.restype = C.c_int
    L.volks_refit_pulses.argtypes = [P, C.POINTER(volks_candidate), I32, I32, C.POINTER(volks_refit)]
    L.volks_refit_pulses.restype = C.c_int
    L.volks_loc_default_params.argtypes = [C.POINTER(volks_loc_params)]
    L.volks_loc_default_params.restype = C.c_int
    L.volks_localize.argtypes = [C.POINTER(volks_loc_obs), I32, C.POINTER(volks_loc_params),
                                 C.POINTER(volks_loc_result), P, P]
    L.volks_localize.restype = C.c_int
    _lib = L
    return L


class VolksError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = lib().volks_last_error().decode(errors="replace")
        super().__init__(f"{where} failed ({code}): {msg}")
        self.code = code


def _check(rc: int, where: str):
    if rc != VOLKS_OK:
        raise VolksError(rc, where)


# ---- thin wrappers with the C names ----------------------------------------
def volks_default_params() -> volks_params:
    p = volks_params()
    lib().volks_default_params(C.byref(p))
    return p


def volks_search_segment(seg: volks_segment, prm: volks_params, stream: int = 0) -> int:
    out = C.c_void_p()
    _check(lib().volks_search_segment(C.byref(seg), C.byref(prm), C.c_void_p(stream),
                                      C.byref(out)), "volks_search_segment")
    return out.value


def volks_candidates(res: int) -> List[volks_candidate]:
    n = C.c_size_t()
    _check(lib().volks_candidates(C.c_void_p(res), None, 0, C.byref(n)), "volks_candidates")
    buf = (volks_candidate * max(1, n.value))()
    _check(lib().volks_candidates(C.c_void_p(res), buf, n.value, C.byref(n)), "volks_candidates")
    return list(buf[:n.value])


def volks_free(res: Optional[int]):
    if res:
        lib().volks_free(C.c_void_p(res))


def volks_search_peaks_noalloc(seg: volks_segment, prm: volks_params, stream: int,
                               peak_power_ptr: int, peak_cell_ptr: int):
    """Peak search into caller-owned device buffers with no device
    allocation (see include/volks.h for the layout and the rules)."""
    _check(lib().volks_search_peaks_noalloc(C.byref(seg), C.byref(prm), C.c_void_p(stream),
                                            C.c_void_p(peak_power_ptr),
                                            C.c_void_p(peak_cell_ptr)),
           "volks_search_peaks_noalloc")


def volks_noalloc_tables(stream: int, shifts_ptr: int, nvalid_ptr: int, n_dm: int, n_f: int):
    """Copy the last no-allocation call's device shift table and n_valid
    into caller device buffers (a checking accessor)."""
    _check(lib().volks_noalloc_tables(C.c_void_p(stream), C.c_void_p(shifts_ptr),
                                      C.c_void_p(nvalid_ptr), n_dm, n_f), "volks_noalloc_tables")


def volks_fringe_fit_calibrator(wl, vis, pad: int = 4, stream: int = 0, n_bl=None, n_ap=None):
    """Initial calibration from a calibrator scan (see include/volks.h):
    returns (cal [n_bl][n_if][2] = (delay s, phase rad), amp [n_bl][n_if])."""
    seg = volks_segment()
    keep = fill_segment(seg, wl, vis, None, None, None, n_bl, n_ap)
    lead = (seg.n_pol,) if seg.n_pol == 2 else ()
    cal = np.zeros(lead + (seg.n_bl, wl.n_if, 2), dtype=np.float64)
    amp = np.zeros(lead + (seg.n_bl, wl.n_if), dtype=np.float64)
    DP = C.POINTER(C.c_double)
    _check(lib().volks_fringe_fit_calibrator(C.byref(seg), pad, C.c_void_p(stream),
                                             cal.ctypes.data_as(DP), amp.ctypes.data_as(DP)),
           "volks_fringe_fit_calibrator")
    del keep
    return cal, amp


def volks_fine_calibration(wl, vis, cal=None, pad: int = 4, stream: int = 0, n_ap=None):
    """Residual band-wide delay of a reference scan per baseline (see
    include/volks.h): returns (tau_cal [n_bl] s, amp [n_bl]), with a leading
    polarisation axis for two products."""
    seg = volks_segment()
    keep = fill_segment(seg, wl, vis, cal, n_ap=n_ap)
    lead = (seg.n_pol,) if seg.n_pol == 2 else ()
    tau = np.zeros(lead + (seg.n_bl,), dtype=np.float64)
    amp = np.zeros(lead + (seg.n_bl,), dtype=np.float64)
    DP = C.POINTER(C.c_double)
    _check(lib().volks_fine_calibration(C.byref(seg), pad, C.c_void_p(stream), tau.ctypes.data_as(DP),
                                        amp.ctypes.data_as(DP)), "volks_fine_calibration")
    del keep
    return tau, amp


VOLKS_CHECK_SKIP_MMA = 1


def volks_check_rate_gemm(y_ptr: int, win: int, precision: int, out_ptr: int, flags: int = 0):
    """One 128-delay-cell block of the tensor-core rate GEMM (checking aid,
    see include/volks.h): y device complex64 [32][128] -> out device float
    [128][256]."""
    _check(lib().volks_check_rate_gemm(C.c_void_p(y_ptr), win, precision, flags,
                                       C.c_void_p(out_ptr)), "volks_check_rate_gemm")


def volks_loc_default_params() -> volks_loc_params:
    p = volks_loc_params()
    _check(lib().volks_loc_default_params(C.byref(p)), "volks_loc_default_params")
    return p


def volks_localize(tau_s, tau_cal_s, dtau_dalpha, dtau_ddelta, snr, proj_len_m,
                   prm: Optional[volks_loc_params] = None) -> dict:
    """Single-pulse position offset from per-baseline delays (Eq. 2; see
    include/volks.h).  Returns status, n_used, used [n] bool, x (dalpha,
    ddelta) rad, cov 2x2, rms_s, loo [n][2], outlier (index or -1), x_clean."""
    cols = [np.ascontiguousarray(a, dtype=np.float64).ravel()
            for a in (tau_s, tau_cal_s, dtau_dalpha, dtau_ddelta, snr, proj_len_m)]
    n = len(cols[0])
    if any(len(c) != n for c in cols):
        raise ValueError("per-baseline arrays differ in length")
    obs = (volks_loc_obs * max(1, n))()
    for i in range(n):
        obs[i] = volks_loc_obs(*(float(c[i]) for c in cols))
    prm = prm if prm is not None else volks_loc_default_params()
    res = volks_loc_result()
    used = np.zeros(max(1, n), dtype=np.uint8)
    loo = np.zeros((max(1, n), 2), dtype=np.float64)
    _check(lib().volks_localize(obs, n, C.byref(prm), C.byref(res), used.ctypes.data,
                                loo.ctypes.data), "volks_localize")
    return dict(status=res.status, n_used=res.n_used, used=used[:n].astype(bool),
                x=np.array(res.x[:]), cov=np.array(res.cov[:]).reshape(2, 2), rms_s=res.rms_s,
                loo=loo[:n], outlier=res.outlier, x_clean=np.array(res.x_clean[:]))


def volks_cross_match(cands: Sequence[dict], min_baselines: int) -> List[dict]:
    """Cross-baseline match (a10) of candidate dicts gathered from several
    searches of one scan; returns the kept entries as dicts."""
    n = len(cands)
    arr = (volks_candidate * max(1, n))()
    names = [k for k, _ in volks_candidate._fields_ if k != "_pad"]
    for i, c in enumerate(cands):
        for k in names:
            setattr(arr[i], k, c[k])
    out = (volks_candidate * max(1, n))()
    n_out = C.c_size_t()
    _check(lib().volks_cross_match(arr, n, min_baselines, out, n, C.byref(n_out)),
           "volks_cross_match")
    return [out[i].as_dict() for i in range(n_out.value)]


def volks_shift_table(f_lo_mhz, chan_bw_mhz, n_f, t_ap_s, n_ap, dm_lo, dm_step, n_dm):
    sh = np.zeros((max(n_dm, 0), n_f), dtype=np.int32)
    nv = np.zeros(max(n_dm, 0), dtype=np.int32)
    I32P = C.POINTER(C.c_int32)
    _check(lib().volks_shift_table(f_lo_mhz, chan_bw_mhz, n_f, t_ap_s, n_ap, dm_lo, dm_step,
                                   n_dm, sh.ctypes.data_as(I32P), nv.ctypes.data_as(I32P)),
           "volks_shift_table")
    return sh, nv


# ---- convenience: marshal a workload description + array -----------------
def make_params(wl, **over) -> volks_params:
    p = volks_default_params()
    p.dm_lo, p.dm_step, p.n_dm = wl.dm_lo, wl.dm_step, wl.n_dm
    win = list(wl.windows)
    p.n_win = len(win)
    for i, w in enumerate(win):
        p.win[i] = w
    p.pad_delay, p.pad_rate = wl.pad_delay, wl.pad_rate
    p.thresh, p.min_windows, p.min_baselines = wl.thresh, wl.min_windows, wl.min_baselines
    p.stride = getattr(wl, "stride", 0)
    for k, v in over.items():
        setattr(p, k, v)
    return p


def _vis_pointer(vis):
    """(pointer, keepalive) of a contiguous complex64 array or tensor."""
    try:
        import torch
        if isinstance(vis, torch.Tensor):
            if vis.dtype != torch.complex64 or not vis.is_contiguous():
                raise ValueError("vis must be a contiguous complex64 tensor")
            return vis.data_ptr(), vis
    except ImportError:
        pass
    arr = np.ascontiguousarray(vis, dtype=np.complex64)
    return arr.ctypes.data, arr


def _autos_pointer(autos):
    """(pointer, keepalive) of a contiguous float32 array or tensor."""
    try:
        import torch
        if isinstance(autos, torch.Tensor):
            if autos.dtype != torch.float32 or not autos.is_contiguous():
                raise ValueError("autos must be a contiguous float32 tensor")
            return autos.data_ptr(), autos
    except ImportError:
        pass
    arr = np.ascontiguousarray(autos, dtype=np.float32)
    return arr.ctypes.data, arr


def fill_segment(seg: volks_segment, wl, vis, cal=None, autos=None, bl_st=None,
                 n_bl: Optional[int] = None, n_ap: Optional[int] = None) -> list:
    """Fill a segment descriptor; returns the objects that must outlive it.
    vis [n_bl][n_ap][n_f] is one polarisation product, [n_pol][n_bl][n_ap][n_f]
    two; cal [n_pol][n_bl][n_if][2] likewise; autos [n_pol][n_st][n_ap][n_f]
    float32 with bl_st [n_bl][2] station indices, or None."""
    ptr, keep_vis = _vis_pointer(vis)
    seg.n_bl = wl.n_bl if n_bl is None else n_bl
    seg.n_ap = wl.n_ap if n_ap is None else n_ap
    seg.n_if, seg.n_chan = wl.n_if, wl.n_chan
    seg.t_ap_s, seg.f_lo_mhz, seg.chan_bw_mhz = wl.t_ap_s, wl.f_lo_mhz, wl.chan_bw_mhz
    seg.vis = ptr
    seg.n_pol = int(vis.shape[0]) if len(vis.shape) == 4 else 1
    if seg.n_bl * seg.n_ap > 0 and tuple(vis.shape[-3:]) != (seg.n_bl, seg.n_ap, wl.n_if * wl.n_chan):
        raise ValueError(f"vis shape {tuple(vis.shape)} does not hold [n_bl={seg.n_bl}][n_ap={seg.n_ap}]"
                         f"[n_f={wl.n_if * wl.n_chan}]")
    calc = None if cal is None else np.ascontiguousarray(cal, dtype=np.float64)
    if calc is not None and calc.size != seg.n_pol * seg.n_bl * wl.n_if * 2:
        raise ValueError(f"cal shape {calc.shape} does not hold [n_pol={seg.n_pol}][n_bl={seg.n_bl}]"
                         f"[n_if={wl.n_if}][2]")
    seg.cal = None if calc is None else calc.ctypes.data_as(C.POINTER(C.c_double))
    keep = [keep_vis, calc]
    if autos is not None:
        if len(autos.shape) != 4 or autos.shape[0] != seg.n_pol or \
                tuple(autos.shape[2:]) != (seg.n_ap, wl.n_if * wl.n_chan):
            raise ValueError(f"autos shape {tuple(autos.shape)} does not hold [n_pol={seg.n_pol}][n_st]"
                             f"[n_ap={seg.n_ap}][n_f={wl.n_if * wl.n_chan}]")
        aptr, keep_a = _autos_pointer(autos)
        st = np.ascontiguousarray(bl_st, dtype=np.int32)
        if st.shape != (seg.n_bl, 2):
            raise ValueError(f"bl_st shape {st.shape} is not [n_bl={seg.n_bl}][2]")
        seg.autos = aptr
        seg.n_st = int(autos.shape[-3])
        seg.bl_st = st.ctypes.data_as(C.POINTER(C.c_int32))
        keep += [keep_a, st]
    return keep


class Search:
    """One search handle; frees its device scratch on close()/__del__."""

    def __init__(self, wl, vis, cal: Optional[np.ndarray] = None, stream: int = 0,
                 n_bl: Optional[int] = None, n_ap: Optional[int] = None, autos=None, bl_st=None,
                 **over):
        seg = volks_segment()
        self._keep_vis = fill_segment(seg, wl, vis, cal, autos, bl_st, n_bl, n_ap)
        self.seg, self.prm = seg, make_params(wl, **over)
        self.n_f = wl.n_if * wl.n_chan
        self.n_bl = seg.n_bl
        self.handle = volks_search_segment(seg, self.prm, stream)

    def candidates(self) -> List[dict]:
        return [c.as_dict() for c in volks_candidates(self.handle)]

    def timing(self) -> volks_timing:
        t = volks_timing()
        _check(lib().volks_result_timing(C.c_void_p(self.handle), C.byref(t)), "timing")
        return t

    def refit(self, cands: Sequence[dict], pad: int = 16) -> List[dict]:
        """volks_refit_pulses on candidate dicts: delay_s, snr, amp, delay_idx, n_ap each."""
        n = len(cands)
        arr = (volks_candidate * max(1, n))()
        names = [k for k, _ in volks_candidate._fields_ if k != "_pad"]
        for i, c in enumerate(cands):
            for k in names:
                setattr(arr[i], k, c[k])
        out = (volks_refit * max(1, n))()
        _check(lib().volks_refit_pulses(C.c_void_p(self.handle), arr, n, pad, out), "volks_refit_pulses")
        return [{k: getattr(out[i], k) for k, _ in volks_refit._fields_} for i in range(n)]

    def shifts(self):
        sh = np.zeros((self.prm.n_dm, self.n_f), dtype=np.int32)
        nv = np.zeros(self.prm.n_dm, dtype=np.int32)
        I32P = C.POINTER(C.c_int32)
        _check(lib().volks_result_shifts(C.c_void_p(self.handle), sh.ctypes.data_as(I32P),
                                         nv.ctypes.data_as(I32P)), "shifts")
        return sh, nv

    def peaks(self, b: int, d: int, wi: int):
        n = C.c_size_t()
        _check(lib().volks_result_peaks(C.c_void_p(self.handle), b, d, wi, None, None, None, 0,
                                        C.byref(n)), "peaks")
        P = np.zeros(n.value, dtype=np.float32)
        q = np.zeros(n.value, dtype=np.int32)
        m = np.zeros(n.value, dtype=np.int32)
        _check(lib().volks_result_peaks(
            C.c_void_p(self.handle), b, d, wi, P.ctypes.data_as(C.POINTER(C.c_float)),
            q.ctypes.data_as(C.POINTER(C.c_int32)), m.ctypes.data_as(C.POINTER(C.c_int32)),
            n.value, C.byref(n)), "peaks")
        return P, q, m

    def stats(self, b: int, d: int, wi: int):
        mu, sd = C.c_double(), C.c_double()
        _check(lib().volks_result_stats(C.c_void_p(self.handle), b, d, wi, C.byref(mu),
                                        C.byref(sd)), "stats")
        return mu.value, sd.value

    def gains(self) -> np.ndarray:
        """[n_bl][n_f] complex gains, or [n_pol][n_bl][n_f] for two products."""
        n_pol = self.seg.n_pol if getattr(self, "seg", None) is not None else 1
        lead = (n_pol,) if n_pol == 2 else ()
        g = np.zeros(lead + (self.n_bl, self.n_f, 2), dtype=np.float32)
        _check(lib().volks_result_gains(C.c_void_p(self.handle),
                                        g.ctypes.data_as(C.POINTER(C.c_float)), g.size), "gains")
        return g[..., 0] + 1j * g[..., 1]

    def close(self):
        if getattr(self, "handle", None) and not getattr(self, "borrowed", False):
            volks_free(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Plan:
    """Batch plan over many segments (volks_plan_* in include/volks.h).

    `items` is a list of (workload, vis device tensor, cal) triples; keyword
    overrides apply to every segment's parameters."""

    def __init__(self, items, peak_budget_bytes: int = 0, autotune: bool = True,
                 graph: bool = True, one_shot_stream: Optional[int] = None, **over):
        """one_shot_stream: create and run at once through volks_search_batch
        on that stream (no budget, autotuning or graph)."""
        n = len(items)
        self._keep = []
        segs = (volks_segment * n)()
        prms = (volks_params * n)()
        for i, item in enumerate(items):
            wl, vis, cal = item[:3]
            extra = item[3] if len(item) > 3 else {}
            self._keep += fill_segment(segs[i], wl, vis, cal, extra.get("autos"), extra.get("bl_st"))
            prms[i] = make_params(wl, **over)
        self.n = n
        self._segs = segs
        self.n_f = [it[0].n_if * it[0].n_chan for it in items]
        self.n_bl = [it[0].n_bl for it in items]
        self.prms = prms
        flags = (VOLKS_PLAN_AUTOTUNE if autotune else 0) | (VOLKS_PLAN_GRAPH if graph else 0)
        out = C.c_void_p()
        if one_shot_stream is not None:
            _check(lib().volks_search_batch(segs, prms, n, C.c_void_p(one_shot_stream), C.byref(out)),
                   "volks_search_batch")
        else:
            _check(lib().volks_plan_create(segs, prms, n, int(peak_budget_bytes), flags,
                                           C.byref(out)), "volks_plan_create")
        self.handle = out.value

    def run(self, vis=None, stream: int = 0):
        arr = None
        if vis is not None:
            ptrs = []
            for v in vis:
                p, keep = _vis_pointer(v)
                self._keep.append(keep)
                ptrs.append(p)
            arr = (C.c_void_p * self.n)(*ptrs)
        _check(lib().volks_plan_run(C.c_void_p(self.handle), arr, C.c_void_p(stream)),
               "volks_plan_run")

    def result(self, i: int) -> "Search":
        h = C.c_void_p()
        _check(lib().volks_plan_result(C.c_void_p(self.handle), i, C.byref(h)),
               "volks_plan_result")
        r = Search.__new__(Search)
        r.handle, r.prm, r.n_f, r.borrowed = h.value, self.prms[i], self.n_f[i], True
        r.seg, r.n_bl = self._segs[i], self.n_bl[i]
        return r

    def timing(self) -> volks_timing:
        t = volks_timing()
        _check(lib().volks_plan_timing(C.c_void_p(self.handle), C.byref(t)), "plan timing")
        return t

    def info(self):
        r, b, s = C.c_int32(), C.c_int64(), C.c_int32()
        _check(lib().volks_plan_info(C.c_void_p(self.handle), C.byref(r), C.byref(b),
                                     C.byref(s)), "plan info")
        return {"rounds": r.value, "device_bytes": b.value, "search_launches": s.value}

    def close(self):
        if getattr(self, "handle", None):
            lib().volks_plan_free(C.c_void_p(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching request server (volks_server_* in include/volks.h)."""

    def __init__(self, max_inflight: int = 4, hbm_budget_bytes: int = 64 << 30,
                 fail_every: int = 0):
        cfg = volks_server_config(max_inflight, fail_every, int(hbm_budget_bytes))
        out = C.c_void_p()
        _check(lib().volks_server_create(C.byref(cfg), C.byref(out)), "volks_server_create")
        self.handle = out.value
        self._keep = {}

    def submit(self, wl, vis, cal=None, stream_id: int = -1, autos=None, bl_st=None, **over) -> int:
        seg = volks_segment()
        keep = fill_segment(seg, wl, vis, cal, autos, bl_st)
        prm = make_params(wl, **over)
        rid = C.c_uint64()
        _check(lib().volks_server_submit(C.c_void_p(self.handle), C.byref(seg), C.byref(prm),
                                         int(stream_id), C.byref(rid)), "volks_server_submit")
        self._keep[rid.value] = keep
        return rid.value

    def wait(self, rid: int, timeout_ms: int = 600000):
        n = C.c_size_t()
        info = volks_request_info()
        L = lib()
        # first call sizes the buffer; the request is collected by the second
        buf = (volks_candidate * 1)()
        rc = L.volks_server_wait(C.c_void_p(self.handle), rid, timeout_ms, buf, 0, C.byref(n),
                                 C.byref(info))
        self._keep.pop(rid, None)
        if rc != VOLKS_OK:
            raise VolksError(rc, "volks_server_wait")
        return info, n.value

    def wait_all(self, rid: int, timeout_ms: int = 600000):
        """Collect a request: (info, list of candidate dicts)."""
        L = lib()
        cap = 1 << 16
        while True:
            buf = (volks_candidate * cap)()
            n = C.c_size_t()
            info = volks_request_info()
            rc = L.volks_server_wait(C.c_void_p(self.handle), rid, timeout_ms, buf, cap,
                                     C.byref(n), C.byref(info))
            if rc != VOLKS_OK:
                self._keep.pop(rid, None)
                raise VolksError(rc, "volks_server_wait")
            self._keep.pop(rid, None)
            if n.value <= cap:
                return info, [buf[i].as_dict() for i in range(n.value)]
            raise RuntimeError(f"request {rid}: {n.value} candidates exceed {cap}")

    def stats(self) -> volks_server_stats:
        st = volks_server_stats()
        _check(lib().volks_server_get_stats(C.c_void_p(self.handle), C.byref(st)), "stats")
        return st

    def drain(self, timeout_ms: int = 600000):
        _check(lib().volks_server_drain(C.c_void_p(self.handle), timeout_ms), "drain")

    def close(self):
        if getattr(self, "handle", None):
            lib().volks_server_free(C.c_void_p(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
