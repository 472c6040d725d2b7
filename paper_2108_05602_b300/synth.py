"""Seeded synthetic VLBI cross-spectra shaped like the paper's EVN data.

This module is the only code shared between the FP64 oracle's tests and the
CUDA path's tests/benchmark: it draws inputs and holds none of the search's
arithmetic (no dedispersion table, no transforms, no peak search).

Data model (the paper gives none; these are the stated synthetic readings):

* Visibilities ``vis[b, t, k]`` are complex64, baseline ``b``, accumulation
  period (AP) ``t``, frequency point ``k = n * n_chan + j`` (IF ``n``, channel
  ``j``).  IFs are contiguous (Sec. 2.2 treats the band as one fringe; Tab. 1
  lists 8 contiguous 16 MHz IFs).  Noise is N(0, 1) per real component.
* A single pulse is a dispersed, band-limited burst seen on every baseline.
  At frequency point ``k`` (channel centre ``f_k``) it arrives at AP
  ``t0 + d_k`` where ``d_k`` is the cold-plasma delay relative to the top
  channel, rounded half-up to whole APs, and lasts ``width_ap`` APs.  Its
  phase carries the baseline's residual delay ``tau`` (Eq. 1's delay term,
  measured from the band's lower edge), a fringe rate ``nu`` against absolute
  time, and the per-IF instrumental delay/phase that initial calibration
  (Sec. 2.1.1) removes.  Amplitude ``a = snr * sqrt(2 / (width_ap * n_f))``
  makes the matched coherent sum reach amplitude SNR ``snr`` after the data
  are normalised to unit noise power.
* Narrowband RFI (EVN-scale workload only) is excess noise on a few contiguous
  channels for a few tens of APs at one station, so it appears on every
  baseline that contains that station.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

# Cold-plasma dispersion constant in s MHz^2 pc^-1 cm^3 (the paper does not
# print one; this is the standard value).
K_DM = 4.148808e3


@dataclasses.dataclass
class Pulse:
    dm: float
    t0_ap: int            # arrival AP at the top channel
    width_ap: int
    snr: float
    tau_s: np.ndarray     # [n_bl] residual delay per baseline
    nu_hz: np.ndarray     # [n_bl] fringe rate per baseline


@dataclasses.dataclass
class Workload:
    """Shape of one scan segment plus the search parameters run on it."""
    name: str
    n_bl: int
    n_ap: int
    n_if: int
    n_chan: int
    t_ap_s: float
    f_lo_mhz: float
    chan_bw_mhz: float
    dm_lo: float
    dm_step: float
    n_dm: int
    windows: Sequence[int]
    pad_delay: int = 4
    pad_rate: int = 4
    thresh: float = 3.0
    min_windows: int = 2
    min_baselines: int = 5
    stride: int = 0          # segment stride: 0 = w (back to back), 1 = sliding

    @property
    def n_f(self) -> int:
        return self.n_if * self.n_chan

    def dms(self) -> np.ndarray:
        return self.dm_lo + self.dm_step * np.arange(self.n_dm, dtype=np.float64)

    def n_trials_upper(self) -> int:
        """Trials if no AP were lost to dedispersion (an upper bound)."""
        return self.n_bl * self.n_dm * sum(self.n_ap // w for w in self.windows)


def pr1() -> Workload:
    """1 baseline, 8 IFs x 32 channels of 0.5 MHz centred on 1600 MHz,
    1000 APs of 1.024 ms; DM 0..96 step 3; windows 1, 2, 4, 8 AP."""
    return Workload("pr1", n_bl=1, n_ap=1000, n_if=8, n_chan=32,
                    t_ap_s=1.024e-3, f_lo_mhz=1536.0, chan_bw_mhz=0.5,
                    dm_lo=0.0, dm_step=3.0, n_dm=33, windows=(1, 2, 4, 8),
                    min_baselines=1)


def evn() -> Workload:
    """6 stations (15 baselines), 8 IFs x 64 channels of 0.5 MHz over
    1472-1728 MHz, a 60 s scan of 1.024 ms APs (58,594 APs); DM 0..1000
    step 2 (501 trials); windows 1..32 AP in powers of two."""
    return Workload("evn", n_bl=15, n_ap=58594, n_if=8, n_chan=64,
                    t_ap_s=1.024e-3, f_lo_mhz=1472.0, chan_bw_mhz=0.5,
                    dm_lo=0.0, dm_step=2.0, n_dm=501,
                    windows=(1, 2, 4, 8, 16, 32))


def small(n_bl=2, n_ap=300, n_if=4, n_chan=16, n_dm=6, dm_step=40.0,
          windows=(1, 2, 4, 8), pad_rate=4, min_baselines=1,
          name="small") -> Workload:
    """A small shape that spans several AP tiles and a ragged tail."""
    return Workload(name, n_bl=n_bl, n_ap=n_ap, n_if=n_if, n_chan=n_chan,
                    t_ap_s=1.024e-3, f_lo_mhz=1600.0 - 0.5 * n_if * n_chan / 2,
                    chan_bw_mhz=0.5, dm_lo=0.0, dm_step=dm_step, n_dm=n_dm,
                    windows=windows, pad_rate=pad_rate,
                    min_baselines=min_baselines)


def chan_centres_mhz(wl: Workload) -> np.ndarray:
    return wl.f_lo_mhz + (np.arange(wl.n_f) + 0.5) * wl.chan_bw_mhz


def arrival_offsets_ap(wl: Workload, dm: float) -> np.ndarray:
    """Physical arrival AP of a pulse at each frequency point, relative to
    the top channel, rounded half-up to whole APs."""
    f = chan_centres_mhz(wl)
    ftop = f[-1]
    sec = K_DM * dm * (1.0 / (f * f) - 1.0 / (ftop * ftop))
    return np.floor(sec / wl.t_ap_s + 0.5).astype(np.int64)


def draw_calibration(wl: Workload, rng: np.random.Generator) -> np.ndarray:
    """Per-baseline, per-IF instrumental (delay s, phase rad)."""
    cal = np.empty((wl.n_bl, wl.n_if, 2), dtype=np.float64)
    cal[..., 0] = rng.uniform(-20e-9, 20e-9, size=(wl.n_bl, wl.n_if))
    cal[..., 1] = rng.uniform(0.0, 2 * np.pi, size=(wl.n_bl, wl.n_if))
    return cal


def calibrator_scan(wl: Workload, cal: np.ndarray, amp: float, rng: Optional[np.random.Generator],
                    n_ap: Optional[int] = None, tau_s: Optional[np.ndarray] = None) -> np.ndarray:
    """A strong continuum source: every AP carries amp * exp(i (2 pi f_j
    dtau^n + dphi^n)) at channel j of IF n (f_j the channel-centre frequency
    within the IF; (dtau, dphi) = cal[b, n]), times exp(2 pi i f tau_s[b])
    with f the frequency above the band's lower edge when a residual
    band-wide delay is given (a reference source for fine calibration),
    plus unit noise when rng is given.  complex64 [n_bl][n_ap][n_f]."""
    n_ap = wl.n_ap if n_ap is None else n_ap
    k = np.arange(wl.n_f)
    n = k // wl.n_chan
    j = k % wl.n_chan
    f_j_hz = (j + 0.5) * wl.chan_bw_mhz * 1e6
    ph = 2 * np.pi * f_j_hz[None, :] * cal[:, n, 0] + cal[:, n, 1]       # [n_bl][n_f]
    if tau_s is not None:
        f_rel_hz = (k + 0.5) * wl.chan_bw_mhz * 1e6
        ph = ph + 2 * np.pi * f_rel_hz[None, :] * np.asarray(tau_s, dtype=np.float64)[:, None]
    sig = (amp * np.exp(1j * ph)).astype(np.complex64)
    vis = np.broadcast_to(sig[:, None, :], (wl.n_bl, n_ap, wl.n_f)).copy()
    if rng is not None:
        vis += noise(wl, rng, n_ap)
    return vis


def draw_calibration_on_grid(wl: Workload, rng: np.random.Generator, pad: int = 4) -> np.ndarray:
    """Per-baseline, per-IF (delay, phase) with the delay on the grid of a
    pad-times zero-padded transform over one IF's channels, within
    +-1 / (4 chan_bw)."""
    Mc = pad * wl.n_chan
    cells = rng.integers(-Mc // 4, Mc // 4, size=(wl.n_bl, wl.n_if))
    cal = np.empty((wl.n_bl, wl.n_if, 2), dtype=np.float64)
    cal[..., 0] = cells / (Mc * wl.chan_bw_mhz * 1e6)
    cal[..., 1] = rng.uniform(-np.pi, np.pi, size=(wl.n_bl, wl.n_if))
    return cal


C_LIGHT = 299792458.0


def loc_geometry(n_st: int, rng: np.random.Generator, ra0: float = 0.9, dec0: float = 0.6,
                 gast: float = 1.3, max_len_m: float = 2.5e6):
    """Synthetic VLBI geometry for localisation tests: n_st stations at
    Earth-fixed positions (m) within max_len_m of each other, a priori
    source direction (ra0, dec0) rad, Greenwich sidereal angle gast rad.
    Returns (baseline vectors [n_bl][3], station index pairs)."""
    pos = rng.uniform(-0.5, 0.5, size=(n_st, 3)) * (max_len_m / math.sqrt(3.0))
    pairs = [(i, j) for i in range(n_st) for j in range(i + 1, n_st)]
    B = np.array([pos[j] - pos[i] for i, j in pairs])
    return B, pairs


def geometric_delay(B: np.ndarray, ra: float, dec: float, gast: float) -> np.ndarray:
    """tau = -B . s / c for the source unit vector s in the Earth-fixed frame
    (hour angle gast - ra)."""
    h = gast - ra
    s = np.array([math.cos(dec) * math.cos(h), -math.cos(dec) * math.sin(h), math.sin(dec)])
    return -(B @ s) / C_LIGHT


def pulse_footprint(wl: Workload, cal: np.ndarray, p: Pulse):
    """Return (rows [n_f, W], values [n_bl, n_f, W]) of one pulse.

    rows[k, u] is the AP index the pulse occupies at frequency point k."""
    W = p.width_ap
    off = arrival_offsets_ap(wl, p.dm)
    rows = p.t0_ap + off[:, None] + np.arange(W)[None, :]
    k = np.arange(wl.n_f)
    n = k // wl.n_chan
    j = k % wl.n_chan
    f_rel_hz = (k + 0.5) * wl.chan_bw_mhz * 1e6      # from the band's lower edge
    f_j_hz = (j + 0.5) * wl.chan_bw_mhz * 1e6        # within the IF
    a = p.snr * math.sqrt(2.0 / (W * wl.n_f))
    t_s = rows * wl.t_ap_s                            # absolute time
    ph = (2 * np.pi * f_rel_hz[None, :, None] * p.tau_s[:, None, None]
          + 2 * np.pi * p.nu_hz[:, None, None] * t_s[None, :, :]
          + 2 * np.pi * f_j_hz[None, :, None] * cal[:, n, 0][:, :, None]
          + cal[:, n, 1][:, :, None])
    return rows, a * np.exp(1j * ph)


def inject(vis: np.ndarray, wl: Workload, cal: np.ndarray, pulses: List[Pulse]):
    """Add pulses in place into a numpy array vis[b, t, k]."""
    k = np.arange(wl.n_f)
    for p in pulses:
        rows, val = pulse_footprint(wl, cal, p)
        for b in range(wl.n_bl):
            np.add.at(vis[b], (rows, np.broadcast_to(k[:, None], rows.shape)),
                      val[b].astype(np.complex64))


def noise(wl: Workload, rng: np.random.Generator, n_ap: Optional[int] = None):
    n_ap = wl.n_ap if n_ap is None else n_ap
    re = rng.standard_normal((wl.n_bl, n_ap, wl.n_f, 2), dtype=np.float32)
    return re.view(np.complex64)[..., 0]


def station_pairs(n_bl: int):
    """The smallest station count whose baselines cover n_bl, and the first
    n_bl station pairs (i < j) in order: (n_st, bl_st int32 [n_bl][2])."""
    n_st = 2
    while n_st * (n_st - 1) // 2 < n_bl:
        n_st += 1
    pairs = [(i, j) for i in range(n_st) for j in range(i + 1, n_st)][:n_bl]
    return n_st, np.array(pairs, dtype=np.int32).reshape(-1, 2)


def bandpass(n_pol: int, n_st: int, n_f: int, rng: np.random.Generator) -> np.ndarray:
    """Station power gain per polarisation and frequency point
    [n_pol][n_st][n_f]: a level U[0.3, 3] times a smooth ripple of 1-4
    cycles across the band, +-40 %."""
    k = np.arange(n_f) / n_f
    lvl = rng.uniform(0.3, 3.0, size=(n_pol, n_st, 1))
    cyc = rng.uniform(1.0, 4.0, size=(n_pol, n_st, 1))
    ph = rng.uniform(0.0, 2 * np.pi, size=(n_pol, n_st, 1))
    return lvl * (1.0 + 0.4 * np.sin(2 * np.pi * cyc * k[None, None, :] + ph))


def dual_pol_scan(wl: Workload, rng: np.random.Generator, pulses: List[Pulse], n_pol: int = 2,
                  auto_jitter: float = 0.01, cal: Optional[np.ndarray] = None):
    """A scan with n_pol polarisation products (e.g. LL, RR) seen through
    the stations' bandpasses: product p of baseline (i, j) is
    sqrt(g_pi g_pj) x (unit noise + the pulses with product p's instrumental
    terms cal[p]); the stations' auto spectra are g_pi (1 + auto_jitter
    N(0, 1)) per AP.  An unpolarised source: every product carries the same
    pulses.  Returns (vis complex64 [n_pol][n_bl][n_ap][n_f], cal
    [n_pol][n_bl][n_if][2], autos float32 [n_pol][n_st][n_ap][n_f], bl_st
    [n_bl][2], g)."""
    n_st, bl_st = station_pairs(wl.n_bl)
    g = bandpass(n_pol, n_st, wl.n_f, rng)
    if cal is None:
        cal = np.stack([draw_calibration(wl, rng) for _ in range(n_pol)])
    vis = np.empty((n_pol, wl.n_bl, wl.n_ap, wl.n_f), dtype=np.complex64)
    for p in range(n_pol):
        v = noise(wl, rng)
        inject(v, wl, cal[p], pulses)
        scale = np.sqrt(g[p, bl_st[:, 0]] * g[p, bl_st[:, 1]]).astype(np.float32)
        vis[p] = v * scale[:, None, :]
    jit = rng.standard_normal((n_pol, n_st, wl.n_ap, wl.n_f), dtype=np.float32)
    autos = (g[:, :, None, :] * (1.0 + auto_jitter * jit)).astype(np.float32)
    return vis, cal, autos, bl_st, g


def pr1_pulse(wl: Workload, rng: np.random.Generator) -> Pulse:
    """The single PR1 pulse: DM 50, 2 ms (2 AP), SNR 10, 3.2 us, 0.5 Hz."""
    W = 2
    last = wl.n_ap - int(arrival_offsets_ap(wl, 50.0).max()) - W
    t0 = int(rng.integers(0, last))
    return Pulse(dm=50.0, t0_ap=t0, width_ap=W, snr=10.0,
                 tau_s=np.full(wl.n_bl, 3.2e-6), nu_hz=np.full(wl.n_bl, 0.5))


def gen_pr1(seed: int = 1):
    """PR1 workload: noise + one injected pulse.  Returns (wl, vis, cal, pulses)."""
    wl = pr1()
    rng = np.random.default_rng(seed)
    vis = noise(wl, rng)
    cal = draw_calibration(wl, rng)
    pulses = [pr1_pulse(wl, rng)]
    inject(vis, wl, cal, pulses)
    return wl, vis, cal, pulses


def evn_pulses(wl: Workload, rng: np.random.Generator, n_pulses: int = 20,
               n_ap: Optional[int] = None) -> List[Pulse]:
    """Pulses of DM U[100,900], width U{1..16} AP, SNR U[7,30], on-grid delay
    within +-1 us, rate U[-5,5] Hz, separated by at least 32 APs plus the
    largest dispersion sweep so no two overlap."""
    n_ap = wl.n_ap if n_ap is None else n_ap
    M = wl.pad_delay * wl.n_f
    cell_s = 1.0 / (M * wl.chan_bw_mhz * 1e6)
    max_sweep = int(arrival_offsets_ap(wl, 900.0).max())
    slot = 32 + max_sweep + 16
    n_slots = n_ap // slot
    n_pulses = min(n_pulses, n_slots)
    slots = np.sort(rng.choice(n_slots, size=n_pulses, replace=False))
    out = []
    for s in slots:
        dm = float(rng.uniform(100.0, 900.0))
        W = int(rng.integers(1, 17))
        snr = float(rng.uniform(7.0, 30.0))
        m0 = rng.integers(-int(1e-6 / cell_s), int(1e-6 / cell_s) + 1, size=wl.n_bl)
        nu = rng.uniform(-5.0, 5.0, size=wl.n_bl)
        out.append(Pulse(dm=dm, t0_ap=int(s * slot + 16), width_ap=W, snr=snr,
                         tau_s=m0 * cell_s, nu_hz=nu))
    return out


def evn_rfi(wl: Workload, rng: np.random.Generator, n_ap: Optional[int] = None):
    """(baselines, channel slice, AP slice, extra sigma) of narrowband RFI:
    2 stations x 3 bursts of 4 channels x 50 APs at 10x the noise variance."""
    n_ap = wl.n_ap if n_ap is None else n_ap
    n_st = int(round((1 + math.sqrt(1 + 8 * wl.n_bl)) / 2))
    pairs = [(i, j) for i in range(n_st) for j in range(i + 1, n_st)]
    bursts = []
    for st in rng.choice(n_st, size=min(2, n_st), replace=False):
        bls = [b for b, (i, j) in enumerate(pairs) if st in (i, j)]
        for _ in range(3):
            k0 = int(rng.integers(0, wl.n_f - 4))
            t0 = int(rng.integers(0, max(1, n_ap - 50)))
            bursts.append((bls, slice(k0, k0 + 4), slice(t0, t0 + 50), 3.0))
    return bursts


def gen_evn_numpy(seed: int = 2, wl: Optional[Workload] = None,
                  n_ap: Optional[int] = None, n_pulses: int = 20):
    """EVN-shaped workload on the host (use a reduced wl for tests)."""
    wl = evn() if wl is None else wl
    if n_ap is not None:
        wl = dataclasses.replace(wl, n_ap=n_ap)
    rng = np.random.default_rng(seed)
    vis = noise(wl, rng)
    cal = draw_calibration(wl, rng)
    pulses = evn_pulses(wl, rng, n_pulses=n_pulses)
    inject(vis, wl, cal, pulses)
    for bls, ks, ts, sig in evn_rfi(wl, rng):
        for b in bls:
            shp = vis[b, ts, ks].shape
            extra = rng.standard_normal(shp + (2,), dtype=np.float32) * sig
            vis[b, ts, ks] += extra.view(np.complex64)[..., 0]
    return wl, vis, cal, pulses


def gen_evn_torch(seed: int = 2, device: str = "cuda", wl: Optional[Workload] = None,
                  n_pulses: int = 20):
    """EVN-shaped workload drawn straight into device memory with torch's
    seeded generator (the full 3.6 GB scan takes minutes with numpy).

    Pulses and RFI use the same model as ``gen_evn_numpy``; the noise stream
    differs (torch Philox instead of numpy PCG64)."""
    import torch
    wl = evn() if wl is None else wl
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    vis = torch.randn((wl.n_bl, wl.n_ap, wl.n_f, 2), generator=g,
                      device=device, dtype=torch.float32)
    vis = torch.view_as_complex(vis)
    rng = np.random.default_rng(seed)
    cal = draw_calibration(wl, rng)
    pulses = evn_pulses(wl, rng, n_pulses=n_pulses)
    k = np.arange(wl.n_f)
    for p in pulses:
        rows, val = pulse_footprint(wl, cal, p)
        r = torch.as_tensor(rows.reshape(-1), device=device)
        kk = torch.as_tensor(np.broadcast_to(k[:, None], rows.shape).reshape(-1),
                             device=device)
        for b in range(wl.n_bl):
            v = torch.as_tensor(val[b].reshape(-1).astype(np.complex64), device=device)
            vis[b].index_put_((r, kk), v, accumulate=True)
    for bls, ks, ts, sig in evn_rfi(wl, rng):
        for b in bls:
            shp = vis[b, ts, ks].shape
            extra = torch.randn(shp + (2,), generator=g, device=device) * sig
            vis[b, ts, ks] += torch.view_as_complex(extra)
    return wl, vis, cal, pulses


def batch_workloads(seed: int = 3, n_seg: int = 64, dur_s=(5.0, 10.0), max_dm_trials: int = 200):
    """Heterogeneous segments for batched searches: stations U{3..10}
    (3-45 baselines), IFs {4, 8, 16} x channels {16, 32, 64, 128} per IF of
    16 or 32 MHz centred on 1.6 GHz, duration U[dur_s] s of 1.024 ms APs,
    DM range [0, U(200, 2000)] sampled with at most max_dm_trials trials
    (step >= 2), windows 1..32."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_seg):
        n_st = int(rng.integers(3, 11))
        n_if = int(rng.choice([4, 8, 16]))
        n_chan = int(rng.choice([16, 32, 64, 128]))
        if_bw = float(rng.choice([16.0, 32.0]))
        bw = if_bw / n_chan
        n_ap = int(rng.uniform(*dur_s) / 1.024e-3)
        dm_hi = float(rng.uniform(200.0, 2000.0))
        step = max(2.0, dm_hi / max_dm_trials)
        out.append(Workload(f"seg{i}", n_bl=n_st * (n_st - 1) // 2, n_ap=n_ap, n_if=n_if,
                            n_chan=n_chan, t_ap_s=1.024e-3,
                            f_lo_mhz=1600.0 - n_if * if_bw / 2, chan_bw_mhz=bw,
                            dm_lo=0.0, dm_step=step, n_dm=int(dm_hi // step) + 1,
                            windows=(1, 2, 4, 8, 16, 32)))
    return out


def gen_segment_torch(wl: Workload, seed: int, device: str = "cuda", n_pulses: int = 3):
    """One segment drawn into device memory: torch Philox noise, the
    calibration table and a few pulses (DM within the segment's grid, width
    1..16 AP, SNR 8..25) at random arrival APs."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    vis = torch.view_as_complex(torch.randn((wl.n_bl, wl.n_ap, wl.n_f, 2), generator=g,
                                            device=device, dtype=torch.float32))
    rng = np.random.default_rng(seed)
    cal = draw_calibration(wl, rng)
    M = wl.pad_delay * wl.n_f
    cell = 1.0 / (M * wl.chan_bw_mhz * 1e6)
    pulses = []
    k = np.arange(wl.n_f)
    for _ in range(n_pulses):
        dm = float(rng.uniform(wl.dm_lo, wl.dm_lo + wl.dm_step * (wl.n_dm - 1)))
        W = int(rng.integers(1, 17))
        sweep = int(arrival_offsets_ap(wl, dm).max())
        if wl.n_ap - sweep - W - 1 <= 1:
            continue
        p = Pulse(dm=dm, t0_ap=int(rng.integers(0, wl.n_ap - sweep - W - 1)), width_ap=W,
                  snr=float(rng.uniform(8.0, 25.0)),
                  tau_s=rng.integers(-M // 8, M // 8, size=wl.n_bl) * cell,
                  nu_hz=rng.uniform(-5.0, 5.0, size=wl.n_bl))
        rows, val = pulse_footprint(wl, cal, p)
        r = torch.as_tensor(rows.reshape(-1), device=device)
        kk = torch.as_tensor(np.broadcast_to(k[:, None], rows.shape).reshape(-1), device=device)
        for b in range(wl.n_bl):
            vis[b].index_put_((r, kk), torch.as_tensor(val[b].reshape(-1).astype(np.complex64),
                                                       device=device), accumulate=True)
        pulses.append(p)
    return vis, cal, pulses


def serving_workloads(seed: int = 4, n: int = 16, dur_s=(1.0, 3.0), max_dm_trials: int = 32):
    """Request shapes for a serving stream: stations U{3..6} (3-15
    baselines), IFs {8, 16} x channels {32, 64, 128} of 16 MHz IFs centred
    on 1.6 GHz, duration U[dur_s] s of 1.024 ms APs, DM range
    [0, U(200, 1500)] with at most max_dm_trials trials (step >= 2),
    windows 1..32."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        n_st = int(rng.integers(3, 7))
        n_if = int(rng.choice([8, 16]))
        n_chan = int(rng.choice([32, 64, 128]))
        bw = 16.0 / n_chan
        dm_hi = float(rng.uniform(200.0, 1500.0))
        step = max(2.0, dm_hi / max_dm_trials)
        out.append(Workload(f"req{i}", n_bl=n_st * (n_st - 1) // 2,
                            n_ap=int(rng.uniform(*dur_s) / 1.024e-3), n_if=n_if, n_chan=n_chan,
                            t_ap_s=1.024e-3, f_lo_mhz=1600.0 - n_if * 8.0, chan_bw_mhz=bw,
                            dm_lo=0.0, dm_step=step, n_dm=int(dm_hi // step) + 1,
                            windows=(1, 2, 4, 8, 16, 32)))
    return out


def poisson_arrivals(rate_hz: float, duration_s: float, seed: int = 5) -> np.ndarray:
    """Arrival times (s) of a Poisson process of the given rate."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += float(rng.exponential(1.0 / rate_hz))
        if t >= duration_s:
            return np.array(out)
        out.append(t)
