"""FP64 CPU oracle for the VOLKS2 cross-spectrum single-pulse search.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and
its Python binding) may import or call this module; only the tests, the
smoke check and the benchmark's CPU-baseline leg do.  It shares no code,
tables or constants with the CUDA path.

It computes, plainly and slowly, what the fringe-fitting search of the paper
computes, in the order the paper gives (Sec. 2.4.2 "Code optimization",
steps 3-6, then the detection criteria of Sec. 3.1.1):

  a1 dedispersion shift table (per-frequency integer AP shift, Sec. 2.4.2)
  a2 amplitude normalisation (HOPS/Mk4 style with the stations' auto spectra,
     else the cross-spectrum RMS, Sec. 2.2), per polarisation product
  a3 initial calibration phasor (Eq. 1, second line; Sec. 2.1.1), per
     polarisation product, then the products summed (Fig. 1)
  a4 dedispersion (step 4)
  a5 delay transform: FFT along frequency, zero-padded by 4 (step 5, Sec. 2.2)
  a6 window combine and fringe-rate transform (step 6; the 2-D "geodetic"
     form of Sec. 2.2 over the APs of each window)
  a7 peak search (step 6 "find max")
  a8 normalised power, series statistics and threshold (Sec. 3.1.1, item 1)
  a9 window match (Sec. 3.1.1, item 2)
  a10 cross-baseline match (Sec. 3.1.1, item 3)

and, around the search:

  initial calibration: fringe fit of a calibrator scan per baseline and IF
     (Sec. 2.1.1), giving the table a3 removes
  fine calibration: residual band-wide delay of a reference source per
     baseline (Sec. 2.1.2), the tau_cal of Eq. 2
  pulse re-fit: the detected pulse's visibilities summed coherently and
     fitted on a finer delay grid with its SNR (Sec. 3.1.2)
  localisation: least-squares position offset from the single pulse's
     delays (Sec. 2.3, Eq. 2) with the baseline cuts and the leave-one-out
     check of Sec. 3.1.2

Library primitives used as steps: numpy's FFT (a5, a6), argmax, sort.

Readings of points the paper leaves open: dispersion constant 4.148808e3
s MHz^2 pc^-1 cm^3 referenced to the top channel centre and rounded
half-up; frequency points at channel centres; Eq. 1's inner sum taken over
all channels; normalisation by the HOPS auto-spectrum factor, or by the
per-channel RMS over the segment without auto spectra; polarisation
products summed after their own calibration; f_ref = lower band edge;
segments of w APs at stride w by default, sliding (stride 1) when asked;
normalised power rho = P / (w * N_eff) thresholded as a z-score over the
(baseline, DM, window) series; matching by interval overlap; the calibrator
delay on the padded delay grid and its phase at the IF's first channel
centre; the leave-one-out outlier flagged when its solution lies more than
5x the median distance from the median solution (offsets compared in
radians of RA and Dec as given).

Every function is pinned by tests against closed forms, brute force or
invariants (see tests/test_oracle_pins.py); none is "parity unpinned".
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

K_DM = 4.148808e3  # s MHz^2 pc^-1 cm^3


# ---------------------------------------------------------------- a1 ----
def chan_centres_mhz(f_lo_mhz: float, chan_bw_mhz: float, n_f: int) -> np.ndarray:
    """Sky frequency of each frequency point: IFs are contiguous (Sec. 2.2,
    Tab. 1), point k = n*J + j sits at the centre of its channel."""
    return f_lo_mhz + (np.arange(n_f, dtype=np.float64) + 0.5) * chan_bw_mhz


def shift_table(f_lo_mhz: float, chan_bw_mhz: float, n_f: int,
                dms: Sequence[float], t_ap_s: float) -> np.ndarray:
    """a1: integer AP shift per (DM, frequency point) (Sec. 2.4.2 step 4: a
    specific time shift per frequency point).  Cold-plasma delay relative to
    the highest channel centre, in APs, rounded half-up."""
    f = chan_centres_mhz(f_lo_mhz, chan_bw_mhz, n_f)
    ftop = f[-1]
    dms = np.asarray(dms, dtype=np.float64)
    out = np.empty((len(dms), n_f), dtype=np.int64)
    for i, dm in enumerate(dms):
        x = (K_DM * dm / t_ap_s) * (1.0 / (f * f) - 1.0 / (ftop * ftop))
        out[i] = np.floor(x + 0.5).astype(np.int64)
    return out


def n_valid(n_ap: int, shifts_row: np.ndarray) -> int:
    """Dedispersed APs available at one DM: the series ends when the lowest
    channel runs out of data."""
    return int(n_ap - int(shifts_row.max()))


# ------------------------------------------------------------- a2, a3 ----
def chan_rms(vis_b: np.ndarray) -> np.ndarray:
    """a2: per-frequency-point RMS over the segment's APs (FP64).  Stands in
    for the auto-spectrum dispersion of the HOPS normalisation (Sec. 2.2)."""
    v = vis_b.astype(np.complex128)
    return np.sqrt(np.mean(v.real ** 2 + v.imag ** 2, axis=0))


def calib_phasor(cal_b: Optional[np.ndarray], n_if: int, n_chan: int,
                 chan_bw_mhz: float) -> np.ndarray:
    """a3: exp(-i (2 pi f_j dtau0^n + dphi0^n)) per point (Eq. 1 second line).
    f_j is the channel-centre frequency within IF n."""
    n_f = n_if * n_chan
    if cal_b is None:
        return np.ones(n_f, dtype=np.complex128)
    k = np.arange(n_f)
    n = k // n_chan
    j = k % n_chan
    f_j = (j + 0.5) * chan_bw_mhz * 1e6
    return np.exp(-1j * (2 * np.pi * f_j * cal_b[n, 0] + cal_b[n, 1]))


def auto_norm(autos_i: np.ndarray, autos_j: np.ndarray) -> np.ndarray:
    """a2 with auto spectra, the HOPS amplitude normalisation (Sec. 2.2):
    |s~_ij| = |s_ij| / (mean a_i^2  mean a_j^2)^(1/4) per frequency point,
    means over the segment's APs (FP64).  Returns the factor
    (mean a_i^2 mean a_j^2)^(-1/4); 0 where either station has no power."""
    Ai = np.mean(autos_i.astype(np.float64) ** 2, axis=0)
    Aj = np.mean(autos_j.astype(np.float64) ** 2, axis=0)
    prod = Ai * Aj
    return np.where(prod > 0, np.where(prod > 0, prod, 1.0) ** -0.25, 0.0)


def calibrate(vis_b: np.ndarray, cal_b: Optional[np.ndarray], n_if: int, n_chan: int,
              chan_bw_mhz: float, normalize: bool = True,
              skip_first_chan: bool = False, norm: Optional[np.ndarray] = None) -> np.ndarray:
    """Steps a2+a3 applied to one baseline: X = S * norm_k * phasor_k, with
    norm_k = 1 / rms_k of the cross spectrum, or the given factors (e.g.
    auto_norm).  A channel with zero power contributes zero."""
    X = vis_b.astype(np.complex128)
    if normalize:
        if norm is None:
            rms = chan_rms(vis_b)
            norm = np.where(rms > 0, 1.0 / np.where(rms > 0, rms, 1.0), 0.0)
        X = X * np.asarray(norm, dtype=np.float64)[None, :]
    X = X * calib_phasor(cal_b, n_if, n_chan, chan_bw_mhz)[None, :]
    if skip_first_chan:
        X[:, (np.arange(n_if * n_chan) % n_chan) == 0] = 0
    return X


# ------------------------------------------------ initial calibration ----
@dataclass
class CalFit:
    tau_s: np.ndarray    # [n_if] delay dtau0^n
    phi_rad: np.ndarray  # [n_if] phase dphi0^n in (-pi, pi]
    cell: np.ndarray     # [n_if] signed delay cell of the peak
    amp: np.ndarray      # [n_if] |G(peak)| / sum_j |S(j)| (1 for a perfect fringe)


def fringe_fit_calibrator(vis_b: np.ndarray, n_if: int, n_chan: int, chan_bw_mhz: float,
                          pad: int = 4) -> CalFit:
    """Initial calibration (Sec. 2.1.1): fringe fit of a strong calibrator,
    per IF n of one baseline, giving the (dtau0^n, dphi0^n) that the search
    removes with exp(-i (2 pi f_j dtau0^n + dphi0^n)) (Eq. 1).

      1. coherent integration over the scan: S(j) = sum_t vis[t, n J + j];
      2. delay transform over the IF's J channels, zero-padded by `pad` (the
         factor of Sec. 2.2): G(m) = sum_j S(j) exp(-2 pi i j m / (pad J));
      3. peak m* = argmax |G|^2 (lowest cell on ties), signed in
         [-pad J / 2, pad J / 2): dtau0 = m* / (pad J chan_bw);
      4. phase at the peak, referenced to the channel centres f_j = (j + 1/2)
         chan_bw: dphi0 = arg G(m*) - pi chan_bw dtau0, wrapped to (-pi, pi].
    The delay is found on the transform grid (resolution 1 / (pad J chan_bw))
    and is ambiguous modulo 1 / chan_bw."""
    J = n_chan
    Mc = pad * J
    bw = chan_bw_mhz * 1e6
    tau = np.zeros(n_if)
    phi = np.zeros(n_if)
    cell = np.zeros(n_if, dtype=np.int64)
    amp = np.zeros(n_if)
    for n in range(n_if):
        S = vis_b[:, n * J:(n + 1) * J].astype(np.complex128).sum(axis=0)
        G = np.fft.fft(S, n=Mc)
        pw = G.real ** 2 + G.imag ** 2
        m = int(np.argmax(pw))
        ms = m - Mc if m >= Mc // 2 else m
        tau[n] = ms / (Mc * bw)
        ph = np.angle(G[m]) - np.pi * bw * tau[n]
        phi[n] = math.remainder(ph, 2 * np.pi)
        if phi[n] <= -np.pi:
            phi[n] += 2 * np.pi
        cell[n] = ms
        tot = np.abs(S).sum()
        amp[n] = abs(G[m]) / tot if tot > 0 else 0.0
    return CalFit(tau, phi, cell, amp)


# --------------------------------------------------- fine calibration ----
@dataclass
class FineCal:
    tau_s: float         # residual band-wide delay tau_cal
    cell: int            # signed delay cell of the peak
    amp: float           # |G(peak)| / sum_k |S(k)|


def fine_calibration(vis_b: np.ndarray, cal_b: Optional[np.ndarray], n_if: int, n_chan: int,
                     chan_bw_mhz: float, pad: int = 4) -> FineCal:
    """Fine calibration (Sec. 2.1.2): the residual delay of a reference
    source near the target, fitted per baseline with the target's scheme
    (Sec. 2.2), delay only:

      1. a2 + a3: per-point normalisation and the initial calibration;
      2. coherent integration over the scan: S(k) = sum_t X[t, k];
      3. one delay across all IFs: G(m) = sum_k S(k) exp(-2 pi i k m / (pad N_f));
      4. peak m* (lowest on ties), signed: tau_cal = m* / (pad N_f chan_bw)."""
    X = calibrate(vis_b, cal_b, n_if, n_chan, chan_bw_mhz, normalize=True)
    S = X.sum(axis=0)
    Mc = pad * n_if * n_chan
    G = np.fft.fft(S, n=Mc)
    m = int(np.argmax(G.real ** 2 + G.imag ** 2))
    ms = m - Mc if m >= Mc // 2 else m
    tot = np.abs(S).sum()
    return FineCal(ms / (Mc * chan_bw_mhz * 1e6), ms, abs(G[m]) / tot if tot > 0 else 0.0)


# ------------------------------------------------------ pulse re-fit ----
@dataclass
class Refit:
    tau_s: float         # delay of the peak on the pad * N_f grid
    cell: int            # signed cell
    snr: float           # |G(peak)| / sqrt(W N_eff)
    amp: float           # |G(peak)| / sum_k |S(k)|


def refit_pulse(X: np.ndarray, shifts_row: np.ndarray, t0: int, t1: int, rate_hz: float, t_ap_s: float,
                chan_bw_mhz: float, pad: int, n_eff: int) -> Refit:
    """Re-fit of one detected pulse on one baseline for localisation (Sec.
    3.1.2): the visibilities that hold the pulse (dedispersed APs t0..t1-1
    of the normalised, calibrated X) are summed coherently after removing
    the found fringe rate, S(k) = sum_u Xd[t0 + u, k] exp(-2 pi i rate u
    T_AP), and fitted again on a finer delay grid, G(m) = sum_k S(k)
    exp(-2 pi i k m / (pad N_f)); peak m* (lowest on ties), its delay, and
    the SNR |G(m*)| / sqrt(W N_eff) of a coherent sum of W N_eff
    unit-variance points."""
    Xd = dedisperse(X, shifts_row)[t0:t1]
    W = t1 - t0
    u = np.arange(W)
    S = (Xd * np.exp(-2j * np.pi * rate_hz * u * t_ap_s)[:, None]).sum(axis=0)
    n_f = X.shape[1]
    Mc = pad * n_f
    G = np.fft.fft(S, n=Mc)
    m = int(np.argmax(G.real ** 2 + G.imag ** 2))
    ms = m - Mc if m >= Mc // 2 else m
    tot = np.abs(S).sum()
    return Refit(ms / (Mc * chan_bw_mhz * 1e6), ms, abs(G[m]) / math.sqrt(W * n_eff),
                 abs(G[m]) / tot if tot > 0 else 0.0)


# ------------------------------------------------------- localisation ----
@dataclass
class LocResult:
    status: int                 # 0 solved, 1 fewer than min_baselines usable baselines,
                                # 2 partials of the used baselines collinear (no unique solution)
    used: np.ndarray            # bool [n] baselines passing the SNR and length cuts
    x: np.ndarray               # (dalpha, ddelta) rad from all used baselines
    cov: np.ndarray             # 2x2: sigma^2 (A^T A)^-1, sigma^2 = RSS / (n - 2) (0 when n = 2)
    rms_s: float                # rms delay residual
    loo: np.ndarray             # [n_used][2]: solution without each used baseline (n_used >= 3)
    outlier: int                # index into the input of the flagged baseline, or -1
    x_clean: np.ndarray         # solution without the flagged baseline (= x when none)


def localize(tau_s, tau_cal_s, dtau_dalpha, dtau_ddelta, snr, proj_len_m, min_snr=6.0,
             max_proj_len_m=3.0e6, min_baselines=3, outlier_factor=5.0) -> LocResult:
    """Single-pulse position offset from delays (Sec. 2.3, Eq. 2, with the
    rules of Sec. 3.1.2).

      1. keep baselines with SNR > min_snr and projected length
         <= max_proj_len_m (longer ones have an ambiguous delay); at least
         min_baselines must remain;
      2. least squares for (dalpha, ddelta) in
         tau - tau_cal = dtau/dalpha dalpha + dtau/ddelta ddelta;
         (status 2 when the used baselines' partials have numerical rank
         < 2: smallest singular value <= 1e-12 x the largest);
      3. leave-one-out: the solution without each baseline in turn; a bad
         baseline makes every solution that includes it deviate, so the one
         solution without it is the odd one out: with d_i the distance of the
         i-th leave-one-out solution from their median, the baseline with the
         largest d_i is flagged when d_i > outlier_factor * median(d) and at
         least 4 baselines are used and every leave-one-out system has rank
         2 (a rank-deficient one gets NaN rows and no baseline is flagged);
         the flagged baseline is dropped from x_clean."""
    tau_s, tau_cal_s = np.asarray(tau_s, float), np.asarray(tau_cal_s, float)
    pa, pd = np.asarray(dtau_dalpha, float), np.asarray(dtau_ddelta, float)
    used = (np.asarray(snr, float) > min_snr) & (np.abs(np.asarray(proj_len_m, float)) <= max_proj_len_m)
    idx = np.nonzero(used)[0]
    empty = np.zeros(2)
    if len(idx) < max(min_baselines, 2):
        return LocResult(1, used, empty, np.zeros((2, 2)), 0.0, np.zeros((0, 2)), -1, empty)
    A = np.stack([pa[idx], pd[idx]], axis=1)
    y = tau_s[idx] - tau_cal_s[idx]
    x, _, rank, _ = np.linalg.lstsq(A, y, rcond=1e-12)
    if rank < 2:
        return LocResult(2, used, empty, np.zeros((2, 2)), 0.0, np.zeros((0, 2)), -1, empty)
    r = y - A @ x
    n = len(idx)
    s2 = float(r @ r) / (n - 2) if n > 2 else 0.0
    cov = s2 * np.linalg.inv(A.T @ A)
    loo = np.zeros((0, 2))
    outlier, x_clean = -1, x.copy()
    if n >= 3:
        loo = np.full((n, 2), np.nan)
        for i in range(n):
            xi, _, rk, _ = np.linalg.lstsq(np.delete(A, i, 0), np.delete(y, i), rcond=1e-12)
            if rk == 2:
                loo[i] = xi
        if n >= 4 and np.isfinite(loo).all():
            med = np.median(loo, axis=0)
            d = np.hypot(loo[:, 0] - med[0], loo[:, 1] - med[1])
            i = int(np.argmax(d))
            if d[i] > outlier_factor * np.median(d):
                outlier = int(idx[i])
                x_clean = loo[i]
    return LocResult(0, used, x, cov, float(np.sqrt(np.mean(r ** 2))), loo, outlier, x_clean)


# ---------------------------------------------------------------- a4 ----
def dedisperse(X: np.ndarray, shifts_row: np.ndarray) -> np.ndarray:
    """a4: Xd[t, k] = X[t + shift_k, k] for t < n_valid."""
    nv = n_valid(X.shape[0], shifts_row)
    if nv <= 0:
        return np.zeros((0, X.shape[1]), dtype=X.dtype)
    t = np.arange(nv)[:, None] + shifts_row[None, :]
    return X[t, np.arange(X.shape[1])[None, :]]


# ---------------------------------------------------------------- a5 ----
def delay_transform(Xd: np.ndarray, pad_delay: int = 4) -> np.ndarray:
    """a5: FFT along frequency of every AP, zero-padded to pad_delay * N_f
    points (Sec. 2.2: padding factor 4 against cyclic effects).  Output
    cell m is the delay m / (M * chan_bw), Eq. 1 with f_ref at the band's
    lower edge."""
    M = pad_delay * Xd.shape[1]
    return np.fft.fft(Xd, n=M, axis=1)


# ------------------------------------------------------------ a6, a7 ----
def rate_len(w: int, pad_rate: int) -> int:
    """Fringe-rate cells of a window of w APs: pad_rate*w (w >= 2); one cell
    for w = 1 or in the paper's 1-D mode (pad_rate = 0)."""
    return 1 if (w == 1 or pad_rate == 0) else pad_rate * w


@dataclass
class Peaks:
    P: np.ndarray      # peak power |Z|^2 per segment
    q: np.ndarray      # rate cell of the peak (0..R-1)
    m: np.ndarray      # delay cell of the peak (0..M-1)
    P2: np.ndarray     # best power over all other cells (near-tie check)


def window_peaks(Y: np.ndarray, w: int, pad_rate: int,
                 with_second: bool = True, chunk_bytes: int = 1 << 28,
                 stride: Optional[int] = None) -> Peaks:
    """a6+a7 for one window size: segments s cover dedispersed APs
    [s*stride, s*stride + w) (stride w: back to back; 1: sliding); the FFTed
    APs of a segment are combined by a zero-padded DFT along time (rate cell
    q is nu = q / (R * T_AP); q = 0 is the paper's coherent sum), then the
    maximum |Z|^2 over (q, m) is found, ties going to the lowest q*M + m."""
    n_t, M = Y.shape
    R = rate_len(w, pad_rate)
    st = w if stride is None else stride
    n_seg = (n_t - w) // st + 1 if n_t >= w else 0
    P = np.zeros(n_seg)
    q = np.zeros(n_seg, dtype=np.int64)
    m = np.zeros(n_seg, dtype=np.int64)
    P2 = np.zeros(n_seg)
    per = max(1, chunk_bytes // (16 * R * M))
    for s0 in range(0, n_seg, per):
        s1 = min(n_seg, s0 + per)
        if st == w:
            Ys = Y[s0 * w:s1 * w].reshape(s1 - s0, w, M)
        else:
            Ys = np.stack([Y[i * st:i * st + w] for i in range(s0, s1)])
        Z = np.fft.fft(Ys, n=R, axis=1) if R > 1 else Ys.sum(axis=1, keepdims=True)
        pw = (Z.real ** 2 + Z.imag ** 2).reshape(s1 - s0, R * M)
        idx = np.argmax(pw, axis=1)            # first (lowest) index on ties
        rows = np.arange(s1 - s0)
        P[s0:s1] = pw[rows, idx]
        q[s0:s1] = idx // M
        m[s0:s1] = idx % M
        if with_second:
            pw[rows, idx] = -np.inf
            P2[s0:s1] = pw.max(axis=1) if R * M > 1 else -np.inf
    return Peaks(P, q, m, P2)


# ---------------------------------------------------------------- a8 ----
def series_stats(rho: np.ndarray) -> Tuple[float, float]:
    """Mean and (population) standard deviation of a normalised-power series."""
    if rho.size == 0:
        return 0.0, 0.0
    mu = float(np.mean(rho))
    sd = float(np.sqrt(np.mean((rho - mu) ** 2)))
    return mu, sd


def zscores(rho: np.ndarray, mu: float, sd: float) -> np.ndarray:
    """z = (rho - mean) / std; an all-equal series has no outliers (z = 0)."""
    if sd <= 0.0:
        return np.zeros_like(rho)
    return (rho - mu) / sd


# ---------------------------------------------------------------- a9 ----
@dataclass
class Member:
    w: int
    s: int
    z: float
    P: float
    q: int
    m: int
    stride: int = 0      # segment start = s * stride (0: stride w)

    @property
    def t0(self):
        return self.s * (self.stride or self.w)

    @property
    def t1(self):
        return self.t0 + self.w


def overlap_components(items: List, start, end) -> List[List]:
    """Connected components of the 'intervals overlap' graph, by a sweep over
    intervals sorted by start: an interval joins the running component when
    it starts before the component's current end."""
    order = sorted(items, key=lambda it: (start(it), end(it)))
    comps, cur, cur_end = [], [], None
    for it in order:
        if cur and start(it) < cur_end:
            cur.append(it)
            cur_end = max(cur_end, end(it))
        else:
            if cur:
                comps.append(cur)
            cur, cur_end = [it], end(it)
    if cur:
        comps.append(cur)
    return comps


def representative(members: List[Member]) -> Member:
    """Highest z; ties to the smaller window, then the earlier segment."""
    return sorted(members, key=lambda a: (-a.z, a.w, a.s))[0]


def window_match(members: List[Member], min_windows: int):
    """a9: on one baseline and DM, group selected segments of all windows
    whose AP intervals overlap; keep a group seen in >= min_windows distinct
    window sizes (Sec. 3.1.1: 'appears in at least 2 windows')."""
    out = []
    for comp in overlap_components(members, lambda a: a.t0, lambda a: a.t1):
        nw = len({a.w for a in comp})
        if nw >= min_windows:
            out.append((representative(comp), nw,
                        min(a.t0 for a in comp), max(a.t1 for a in comp)))
    return out


# --------------------------------------------------------------- a10 ----
def cross_baseline(cands: List[dict], min_baselines: int) -> List[dict]:
    """a10: at one DM, candidates of different baselines whose representative
    intervals overlap belong to one pulse; keep a pulse seen on
    >= min_baselines distinct baselines (Sec. 3.1.1 item 3)."""
    out = []
    for comp in overlap_components(cands, lambda c: c["t0"], lambda c: c["t1"]):
        nb = len({c["bl"] for c in comp})
        if nb >= min_baselines:
            for c in comp:
                c = dict(c)
                c["n_baselines"] = nb
                out.append(c)
    return out


# ---------------------------------------------------------- pipeline ----
@dataclass
class SearchResult:
    shifts: np.ndarray                          # [D][N_f]
    nvalid: np.ndarray                          # [D]
    peaks: Dict[Tuple[int, int, int], Peaks] = field(default_factory=dict)  # (b, d, w)
    stats: Dict[Tuple[int, int, int], Tuple[float, float]] = field(default_factory=dict)
    rho: Dict[Tuple[int, int, int], np.ndarray] = field(default_factory=dict)
    z: Dict[Tuple[int, int, int], np.ndarray] = field(default_factory=dict)
    matched: List[dict] = field(default_factory=list)      # after a9
    candidates: List[dict] = field(default_factory=list)   # after a10


def signed(i: int, n: int) -> int:
    return i - n if i >= (n + 1) // 2 and n > 1 else i


def prepare(vis_pols: np.ndarray, cal_pols: Optional[np.ndarray], b: int, n_if: int, n_chan: int,
            chan_bw_mhz: float, normalize: bool = True, skip_first_chan: bool = False,
            autos: Optional[np.ndarray] = None, bl_st: Optional[np.ndarray] = None) -> np.ndarray:
    """a2+a3 for baseline b with its polarisation products combined: each
    product vis_pols[p, b] normalised (auto spectra autos[p, station] when
    given, else the cross-spectrum RMS) and calibrated with its own table
    cal_pols[p, b], then summed coherently (Fig. 1: the products are combined
    after the initial calibration)."""
    X = 0
    for p in range(vis_pols.shape[0]):
        norm = None
        if autos is not None and normalize:
            i, j = int(bl_st[b][0]), int(bl_st[b][1])
            norm = auto_norm(autos[p, i], autos[p, j])
        X = X + calibrate(vis_pols[p, b], None if cal_pols is None else cal_pols[p, b], n_if, n_chan,
                          chan_bw_mhz, normalize, skip_first_chan, norm)
    return X


def search(wl, vis: np.ndarray, cal: Optional[np.ndarray], *,
           normalize: bool = True, skip_first_chan: bool = False,
           with_second: bool = True, baselines: Optional[Sequence[int]] = None,
           dm_indices: Optional[Sequence[int]] = None, autos: Optional[np.ndarray] = None,
           bl_st: Optional[np.ndarray] = None) -> SearchResult:
    """The whole search (a1..a10) on one scan segment vis[b, t, k] (one
    polarisation product, cal[b, n, 2]) or vis[p, b, t, k] (several,
    cal[p, b, n, 2]); autos[p, station, t, k] with bl_st[b] = (i, j) select
    the HOPS normalisation.

    ``wl`` carries n_if, n_chan, n_ap, t_ap_s, f_lo_mhz, chan_bw_mhz, dms(),
    windows, pad_delay, pad_rate, thresh, min_windows, min_baselines."""
    vis_pols = vis if vis.ndim == 4 else vis[None]
    cal_pols = None if cal is None else (cal if np.ndim(cal) == 4 else np.asarray(cal)[None])
    n_f = wl.n_if * wl.n_chan
    dms = wl.dms()
    shifts = shift_table(wl.f_lo_mhz, wl.chan_bw_mhz, n_f, dms, wl.t_ap_s)
    nval = np.array([n_valid(vis_pols.shape[2], r) for r in shifts])
    res = SearchResult(shifts=shifts, nvalid=nval)
    n_eff = n_f - (wl.n_if if skip_first_chan else 0)
    M = wl.pad_delay * n_f
    bls = range(vis_pols.shape[1]) if baselines is None else baselines
    dis = range(len(dms)) if dm_indices is None else dm_indices
    for b in bls:
        X = prepare(vis_pols, cal_pols, b, wl.n_if, wl.n_chan, wl.chan_bw_mhz, normalize,
                    skip_first_chan, autos, bl_st)
        for d in dis:
            Xd = dedisperse(X, shifts[d])
            Y = delay_transform(Xd, wl.pad_delay)
            members = []
            for w in wl.windows:
                st = getattr(wl, "stride", 0) or w
                pk = window_peaks(Y, w, wl.pad_rate, with_second, stride=st)
                rho = pk.P / (w * n_eff)
                mu, sd = series_stats(rho)
                z = zscores(rho, mu, sd)
                key = (b, d, w)
                res.peaks[key], res.stats[key], res.rho[key], res.z[key] = pk, (mu, sd), rho, z
                for s in np.nonzero(z >= wl.thresh)[0]:
                    members.append(Member(w, int(s), float(z[s]), float(pk.P[s]),
                                          int(pk.q[s]), int(pk.m[s]), st))
            for rep, nw, g0, g1 in window_match(members, wl.min_windows):
                R = rate_len(rep.w, wl.pad_rate)
                di, ri = signed(rep.m, M), signed(rep.q, R)
                res.matched.append(dict(
                    bl=b, dm_idx=d, win=rep.w, seg=rep.s, t0=rep.t0, t1=rep.t1,
                    g0=g0, g1=g1, delay_idx=di, rate_idx=ri, n_windows=nw,
                    peak_power=rep.P, rho=rep.P / (rep.w * n_eff), z=rep.z,
                    delay_s=di / (M * wl.chan_bw_mhz * 1e6),
                    rate_hz=ri / (R * wl.t_ap_s)))
    by_dm: Dict[int, List[dict]] = {}
    for c in res.matched:
        by_dm.setdefault(c["dm_idx"], []).append(c)
    out = []
    for d in sorted(by_dm):
        out.extend(cross_baseline(by_dm[d], wl.min_baselines))
    res.candidates = sorted(out, key=lambda c: (c["dm_idx"], c["t0"], c["bl"]))
    return res


# ------------------------------------------------------- brute force ----
def eq1_brute_force(S_seg: np.ndarray, cal_b: Optional[np.ndarray], n_if: int,
                    n_chan: int, f_lo_mhz: float, chan_bw_mhz: float,
                    t_ap_s: float, delays_s: np.ndarray,
                    rates_hz: np.ndarray) -> np.ndarray:
    """Eq. 1 evaluated term by term, extended over the APs of a window by the
    fringe-rate phase: G(tau, nu) = sum_u sum_n sum_j S_u(n, j)
    exp(-i Phi(n, j)) exp(-2 pi i nu u T_AP), with Phi = 2 pi (f_0^n + f_j -
    f_ref) tau + 2 pi f_j dtau0^n + dphi0^n.  S_seg[u, k] are the (normalised,
    dedispersed) spectra of the window's APs.  O(W N_f |tau| |nu|)."""
    n_f = n_if * n_chan
    out = np.zeros((len(rates_hz), len(delays_s)), dtype=np.complex128)
    f_ref = f_lo_mhz * 1e6
    for u in range(S_seg.shape[0]):
        for n in range(n_if):
            f0n = (f_lo_mhz + n * n_chan * chan_bw_mhz) * 1e6
            dt0, dp0 = (0.0, 0.0) if cal_b is None else (cal_b[n, 0], cal_b[n, 1])
            for j in range(n_chan):
                fj = (j + 0.5) * chan_bw_mhz * 1e6
                s = S_seg[u, n * n_chan + j]
                for iq, nu in enumerate(rates_hz):
                    for im, tau in enumerate(delays_s):
                        phi = (2 * math.pi * (f0n + fj - f_ref) * tau
                               + 2 * math.pi * fj * dt0 + dp0)
                        out[iq, im] += s * complex(math.cos(-phi), math.sin(-phi)) * \
                            complex(math.cos(-2 * math.pi * nu * u * t_ap_s),
                                    math.sin(-2 * math.pi * nu * u * t_ap_s))
    return out
