/*
 * volks.h -- C ABI of the B300 (sm_103a) cross-spectrum single-pulse search.
 *
 * The search is the fringe-fitting hot path of VOLKS2 (Liu et al. 2021,
 * arXiv 2108.05602): for every baseline, dispersion-measure (DM) trial and
 * window size, the complex visibility spectra are normalised and calibrated
 * (Sec. 2.2 HOPS normalisation; Eq. 1 second line, Sec. 2.1.1), dedispersed
 * by a per-frequency integer shift in accumulation periods (Sec. 2.4.2 step
 * 4), transformed along frequency with zero padding 4 (Sec. 2.2, step 5),
 * combined over windows of w APs and transformed along time to fringe rate
 * (step 6; the 2-D geodetic form of Sec. 2.2), searched for the peak (step
 * 6 "find max"), and filtered by normalised-power threshold, window match
 * and cross-baseline match (Sec. 3.1.1).
 *
 * Plain C: pointers and sizes only.  Every call returns 0 or a negative
 * VOLKS_E* code; nothing throws across the ABI; volks_last_error() gives a
 * thread-local message for the last failure on the calling thread.
 */
#ifndef VOLKS_H
#define VOLKS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define VOLKS_OK 0
#define VOLKS_EINVAL (-1)   /* malformed descriptor or parameter */
#define VOLKS_ENOMEM (-2)   /* device or host allocation failed */
#define VOLKS_ETIMEOUT (-3) /* a bounded device wait gave up */
#define VOLKS_ECUDA (-4)    /* a CUDA runtime call failed */

/*
 * Arithmetic of the delay/rate search (volks_params.precision).
 *
 * VOLKS_FP32: every delay and rate cell is evaluated in FP32 on the CUDA
 * cores (register FFTs).
 * VOLKS_BF16, VOLKS_FP16, VOLKS_FP8: the delay transform stays FP32; the
 * fringe-rate transform of the 4..32-AP windows of a 2-D search
 * (pad_rate 4, Sec. 2.2) is a coarse DFT-matrix GEMM on the tensor cores
 * with operands in BF16, FP16 or FP8 E4M3 (a power-of-two scale per 32-AP
 * tile for FP16 and FP8) and FP32 accumulation.  Per segment and delay
 * residue class, the delay cells whose coarse power is within a margin of
 * the coarse maximum (1/16 for BF16, 1/64 for FP16, 1/4 for FP8; halved
 * while more than 8 pass), at most 8, are then re-evaluated in FP32 over
 * all their rate cells, and the peak is the largest FP32 value among
 * them; 1- and 2-AP windows are always FP32.  A peak therefore differs
 * from the FP32 search only when the FP32 peak's delay cell is not among
 * those retained, which needs a near-tie at the coarse precision.  1-D
 * searches (pad_rate 0) and bands under 256 points run FP32 whatever is
 * asked.
 */
#define VOLKS_FP32 0
#define VOLKS_BF16 1
#define VOLKS_FP16 2
#define VOLKS_FP8 3

#define VOLKS_MAX_WIN 6     /* windows are distinct powers of two, 1..32 AP */

/*
 * One scan segment: n_bl baselines x n_ap accumulation periods (APs) x
 * n_f = n_if * n_chan frequency points.  IFs are contiguous and searched as
 * one band (Sec. 2.2); frequency point k = n * n_chan + j of IF n, channel j
 * sits at f_lo_mhz + (k + 1/2) * chan_bw_mhz.  n_f is a power of two in
 * 64..2048 or three times one in 96..1536 (e.g. 12 IFs x 32 channels;
 * mixed-radix delay transforms; those bands always search in FP32);
 * volks_search_peaks_noalloc takes powers of two 64..512 only.
 *
 * vis: complex64 (interleaved float re, im), row-major
 *      [n_pol][n_bl][n_ap][n_f].  Device memory, or host memory (pageable
 *      or pinned; the library then copies it to the device on the call's
 *      stream).  Borrowed: it must stay valid and unchanged until
 *      volks_candidates() returns.
 * cal: host memory, float64 [n_pol][n_bl][n_if][2] = {delay s, phase rad}
 *      of the initial calibration of each polarisation product (Eq. 1:
 *      2 pi f_j dtau0^n + dphi0^n, f_j the channel-centre frequency within
 *      the IF; Sec. 2.1.1 fits it per polarisation, baseline and IF), or
 *      NULL for none.  Read during the call only.
 * n_pol: polarisation products in vis, 1 (0 means 1) or 2 (e.g. LL and RR).
 *      Each product is normalised and calibrated on its own, then the
 *      products are summed coherently (Fig. 1: polarisations are combined
 *      after the initial calibration), so the noise of a normalised cell
 *      is n_pol times that of one product.
 * autos, n_st, bl_st: the stations' auto spectra for the HOPS amplitude
 *      normalisation (Sec. 2.2): |s_ij| / (mean a_i^2  mean a_j^2)^(1/4)
 *      per frequency point and polarisation, the means over the segment's
 *      APs in FP64.  autos: float32 [n_pol][n_st][n_ap][n_f] auto-spectrum
 *      power, device or host memory, borrowed like vis; bl_st: host
 *      int32 [n_bl][2], the two stations (i != j, < n_st) of each
 *      baseline, read during the call only.  With autos NULL (n_st, bl_st
 *      ignored) each frequency point is divided by the RMS of its cross
 *      spectrum over the segment instead.  Only read when
 *      volks_params.normalize_chan is 1.  A station whose auto power is 0
 *      at a point zeroes that point on its baselines.
 * Zero-initialise the struct: n_pol, n_st, bl_st and autos = 0 give one
 * product and the cross-spectrum RMS normalisation.
 */
typedef struct {
  int32_t n_bl, n_ap, n_if, n_chan;
  double t_ap_s;        /* AP length, e.g. 1.024e-3 (Sec. 2.2) */
  double f_lo_mhz;      /* lower edge of IF 0, channel 0 */
  double chan_bw_mhz;   /* channel width */
  const void *vis;
  const double *cal;
  int32_t n_pol;        /* 0/1: one polarisation product; 2: two, combined */
  int32_t n_st;         /* stations in autos */
  const int32_t *bl_st; /* host [n_bl][2] station pair of each baseline */
  const void *autos;    /* float32 [n_pol][n_st][n_ap][n_f], or NULL */
} volks_segment;

/*
 * Search parameters.  DM trials are dm_lo + i * dm_step, i < n_dm (pc cm^-3).
 * win: n_win distinct window sizes in APs, each a power of two in 1..32,
 *      ascending (Sec. 3.1.1 uses 2, 4, 8, 16).
 * pad_delay: zero-padding factor of the delay transform (Sec. 2.2: 4);
 *      1, 2, 4 or 8.
 * pad_rate: fringe-rate cells per window AP for w >= 2 (R = pad_rate * w);
 *      4 gives the 2-D delay x rate search, 0 the paper's 1-D search over the
 *      coherent window sum (R = 1).  w = 1 always has R = 1.
 * thresh: z-score threshold on normalised power (Sec. 3.1.1: 3).
 * min_windows / min_baselines: detection needs that many distinct windows on
 *      one baseline / distinct baselines (Sec. 3.1.1: 2 and 5).
 * normalize_chan: 1 applies the HOPS amplitude normalisation (Sec. 2.2)
 *      with the segment's auto spectra, or, without them, divides each
 *      frequency point by its cross-spectrum RMS over the segment (FP64);
 *      0 leaves the amplitudes as they are.
 * stride: 0 (default) places the segments of window w back to back, at
 *      dedispersed APs s w; 1 slides them by one AP (segment s starts at AP
 *      s: n_valid - w + 1 segments per series, w times the trials).  Sliding
 *      searches run the FP32 search kernel whatever precision asks.
 * skip_first_chan: 1 drops channel 0 of every IF (Eq. 1's inner sum read
 *      literally as j = 1 .. J-1).
 */
typedef struct {
  double dm_lo, dm_step;
  int32_t n_dm;
  int32_t n_win;
  int32_t win[8];
  int32_t pad_delay;
  int32_t pad_rate;
  double thresh;
  int32_t min_windows, min_baselines;
  int32_t precision;
  int32_t normalize_chan, skip_first_chan;
  int32_t stride;       /* segment stride: 0 = w (back to back), 1 = sliding */
} volks_params;

/*
 * One detected single pulse on one baseline at one DM trial (the paper's
 * "SP list per DM", Fig. 1).  The representative is the window-matched
 * group member with the highest z (ties: smaller window, then earlier
 * segment); [t0_ap, t1_ap) is its interval and [g0_ap, g1_ap) the group's,
 * in dedispersed APs (arrival time at the top channel).
 */
typedef struct {
  int32_t bl, dm_idx, win, seg;
  int32_t t0_ap, t1_ap, g0_ap, g1_ap;
  int32_t delay_idx;    /* signed delay cell, -M/2 .. M/2-1, M = pad_delay*n_f */
  int32_t rate_idx;     /* signed rate cell, -R/2 .. R/2-1 */
  int32_t n_windows, n_baselines;
  float peak_power;     /* max |Z|^2 */
  float _pad;
  double rho;           /* peak_power / (win * n_eff) */
  double z;             /* (rho - mean) / std over the (bl, DM, win) series */
  double dm;            /* pc cm^-3 */
  double delay_s;       /* delay_idx / (M * chan_bw) */
  double rate_hz;       /* rate_idx / (R * t_ap) */
} volks_candidate;

/* Per-stage device times of one search, from CUDA events on its stream. */
typedef struct {
  float ms_h2d;         /* host -> device copy of vis (0 for device input) */
  float ms_prep;        /* a2-a3: channel power (FP64) + normalise/transpose */
  float ms_search;      /* a4-a7: fused dedisperse/delay/rate/peak kernel */
  float ms_select;      /* a8: FP64 series statistics + threshold */
  float ms_match;       /* a9: window match */
  int32_t n_launches;   /* kernels this library launched for the search */
  int32_t n_search_launches;
} volks_timing;

typedef struct volks_result volks_result;   /* opaque, library-owned */

/* Fill *p with the paper's defaults: DM 0, step 1, 1 trial; windows 2,4,8,16;
 * pad_delay 4; pad_rate 4; thresh 3; min_windows 2; min_baselines 5; FP32;
 * normalize_chan 1; skip_first_chan 0; stride 0. */
void volks_default_params(volks_params *p);

/*
 * Enqueue the whole search (steps a1-a9) of one segment on `cuda_stream`
 * (a cudaStream_t; NULL = legacy default stream) and return a result handle.
 * The call validates everything before enqueuing, builds the shift table
 * (FP64 on the host, rounded half-up; Sec. 2.4.2 step 4) and returns
 * without waiting for the device.  Device scratch (about 8 bytes per
 * trial plus one normalised copy of vis) is allocated stream-ordered and
 * owned by *out.
 * Errors: VOLKS_EINVAL (bad sizes, windows, pads, NULL vis with n_bl*n_ap
 * > 0, unknown precision), VOLKS_ENOMEM, VOLKS_ECUDA.  On error *out
 * is NULL and nothing stays enqueued that touches caller memory.  The
 * tensor-core kernel bounds its waits on the tensor cores (about 2 s);
 * if one gives up, the calls that wait for the search (volks_candidates,
 * volks_result_*) return VOLKS_ETIMEOUT.
 */
int volks_search_segment(const volks_segment *seg, const volks_params *prm,
                         void *cuda_stream, volks_result **out);

/*
 * Wait for the search, run the cross-baseline match on the host (a10,
 * Sec. 3.1.1 item 3) and copy up to `cap` candidates, sorted by (dm_idx,
 * t0_ap, bl), into `buf` (host; may be NULL when cap == 0).  *n_total
 * (required) receives the number of candidates, which may exceed cap.
 * Calling it again returns the same list.
 */
int volks_candidates(volks_result *res, volks_candidate *buf, size_t cap,
                     size_t *n_total);

/* Release the handle and its device scratch (stream-ordered).  NULL-safe. */
void volks_free(volks_result *res);

/* Thread-local message of the last failing call on this thread. */
const char *volks_last_error(void);

/*
 * Host only, no device work: the dedispersion shift table of step a1
 * (Sec. 2.4.2 step 4: one integer AP shift per frequency point and DM).
 * shift[d][k] = floor(x + 1/2), x = (K_DM DM_d / t_ap) (f_k^-2 - f_top^-2),
 * K_DM = 4.148808e3 s MHz^2 pc^-1 cm^3, f_k = f_lo + (k + 1/2) chan_bw,
 * f_top = f_{n_f-1}; computed in FP64.  nvalid[d] = n_ap - max_k shift[d][k]
 * (may be <= 0: no dedispersed AP is left).  shifts holds n_dm * n_f int32,
 * nvalid n_dm int32 (either may be NULL).  Same validation as the search.
 */
int volks_shift_table(double f_lo_mhz, double chan_bw_mhz, int32_t n_f, double t_ap_s,
                      int32_t n_ap, double dm_lo, double dm_step, int32_t n_dm,
                      int32_t *shifts, int32_t *nvalid);

/*
 * Host only, no device work: the cross-baseline match of step a10 (Sec.
 * 3.1.1 item 3) over window-matched candidates gathered from several
 * searches of one scan (e.g. baselines split over GPUs, each searched with
 * min_baselines = 1).  Entries at one dm_idx whose [t0_ap, t1_ap) overlap
 * form one pulse; pulses on >= min_baselines distinct `bl` values are kept,
 * with n_baselines set, sorted by (dm_idx, t0_ap, bl).  `in` (n entries)
 * and `out` (cap entries) are host arrays; *n_out receives the full count.
 * volks_candidates applies the same rule to one search's own list.
 */
int volks_cross_match(const volks_candidate *in, size_t n, int32_t min_baselines,
                      volks_candidate *out, size_t cap, size_t *n_out);

/*
 * Initial calibration (Sec. 2.1.1): fringe fit of a strong calibrator scan
 * giving, per baseline and IF, the (delay, phase) that volks_segment.cal
 * takes (the search removes exp(-i (2 pi f_j dtau0^n + dphi0^n)), Eq. 1).
 * seg: the calibrator scan, as for the search (vis device or host memory;
 *      cal ignored).  Per (baseline b, IF n): the spectrum is integrated
 *      coherently over the scan in FP64, transformed to delay over the IF's
 *      n_chan channels zero-padded by `pad` (1, 2, 4 or 8; Sec. 2.2 uses 4),
 *      and the largest |G| cell m* (lowest on ties, signed) gives
 *      dtau0 = m* / (pad n_chan chan_bw) and dphi0 = arg G(m*) - pi chan_bw
 *      dtau0 in (-pi, pi] (channel-centre frequencies).  The delay is on the
 *      transform grid and ambiguous modulo 1 / chan_bw.
 * cal_out: host, float64 [n_pol][n_bl][n_if][2] = {dtau0 s, dphi0 rad}
 *      (each polarisation product fitted on its own, Sec. 2.1.1), the
 *      layout volks_segment.cal takes.
 * amp_out: host, float64 [n_pol][n_bl][n_if] = |G(m*)| / sum_j |S(j)| (1
 *      for a perfect fringe), or NULL.
 * Runs on cuda_stream (device scratch stream-ordered) and waits for it.
 * Errors: VOLKS_EINVAL (sizes as for the search, pad, pad * n_chan > 16384,
 * n_pol * n_bl > 65535),
 * VOLKS_ENOMEM, VOLKS_ECUDA.
 */
int volks_fringe_fit_calibrator(const volks_segment *seg, int32_t pad, void *cuda_stream,
                                double *cal_out, double *amp_out);

/*
 * Fine calibration (Sec. 2.1.2): the residual delay tau_cal of a reference
 * source near the target, per baseline (and polarisation product), fitted
 * with the target's scheme (Sec. 2.2), delay only -- the tau_cal of Eq. 2
 * (volks_localize).  seg: the reference scan as for the search, with
 * seg->cal the initial calibration.  Per row: each point normalised by its
 * RMS over the scan and multiplied by the calibration phasor (steps a2,
 * a3), integrated coherently over the scan in FP64, transformed to delay
 * over all n_f points zero-padded by `pad` (one delay across the IFs, Eq.
 * 1), and the largest |G| cell m* (lowest on ties, signed) gives
 * tau_cal = m* / (pad n_f chan_bw), on the transform grid and ambiguous
 * modulo 1 / chan_bw.
 * tau_out: host, float64 [n_pol][n_bl].  amp_out: host, float64
 * [n_pol][n_bl] = |G(m*)| / sum_k |S(k)|, or NULL.
 * Runs on cuda_stream and waits for it.  Errors: VOLKS_EINVAL (sizes as
 * for the search, pad 1/2/4/8, pad * n_f > 16384), VOLKS_ENOMEM,
 * VOLKS_ECUDA.
 */
int volks_fine_calibration(const volks_segment *seg, int32_t pad, void *cuda_stream,
                           double *tau_out, double *amp_out);

/* ---- introspection, for checking each step against a reference ---- */

/* Waits for the search.  Stage times and launch counts. */
int volks_result_timing(volks_result *res, volks_timing *t);

/* Copy the shift table int32 [n_dm][n_f] and n_valid int32 [n_dm] (the
 * dedispersed APs left at each DM) to host buffers of >= that many items. */
int volks_result_shifts(volks_result *res, int32_t *shifts, int32_t *nvalid);

/* Waits for the search.  Per-segment peaks of one (baseline, DM trial,
 * window index) series: P[s] = max |Z|^2, q[s] / m[s] = its unsigned rate /
 * delay cell, for s < *n_seg = n_valid / win; buffers hold >= cap items. */
int volks_result_peaks(volks_result *res, int32_t bl, int32_t dm_idx,
                       int32_t win_idx, float *P, int32_t *q, int32_t *m,
                       size_t cap, size_t *n_seg);

/* Waits for the search.  FP64 mean and population standard deviation of
 * the normalised power of one series. */
int volks_result_stats(volks_result *res, int32_t bl, int32_t dm_idx,
                       int32_t win_idx, double *mean, double *std);

/* Waits for the search.  Complex64 gains [n_pol][n_bl][n_f] (calibration
 * phasor times the amplitude normalisation: 1 / channel RMS, or the HOPS
 * factor with auto spectra) applied before dedispersion. */
int volks_result_gains(volks_result *res, float *gains, size_t cap_floats);

/* The checking entry points (tensor-core GEMM layout and fault path, the
 * no-allocation variant's device tables) are declared in volks_check.h. */

/* ---- batch plans --------------------------------------------------------
 *
 * A plan searches many segments of different shapes (baselines, APs, IFs,
 * channels, DM grids, windows) together: the per-(baseline, DM, tile)
 * work of all segments of one band class (n_f, pad_rate) is done
 * by one persistent search launch whose CTAs pull work from a shared
 * counter, followed by one select and one match launch over all segments.
 * Results are those of volks_search_segment on each segment.
 *
 * volks_plan_create: validates every (segment, params) pair; visibilities
 *   and auto spectra must be device memory (every run reads the auto
 *   spectra at the pointer given here).  peak_budget_bytes > 0 bounds the per-trial peak
 *   buffers (8 bytes per trial) of the whole plan: segments whose peaks do
 *   not fit are processed in DM chunks (rounds), reusing their buffers;
 *   <= 0 keeps all DMs resident.  flags: VOLKS_PLAN_AUTOTUNE times the
 *   compiled work splits of each band class on the plan's own data and
 *   keeps the fastest (cached per process); VOLKS_PLAN_GRAPH captures a run
 *   into one CUDA graph, replayed by every volks_plan_run with the same
 *   visibility pointers.  Allocates all device memory (cudaMalloc) here.
 * volks_plan_run: enqueue one run on `cuda_stream`; vis = n device pointers
 *   of new visibilities of the same shapes, or NULL to reuse the previous
 *   ones.  A changed pointer re-captures the graph.  Waits for the plan's
 *   previous run if it was on another stream.
 * volks_plan_result: borrowed handle of segment i (valid until
 *   volks_plan_free; volks_free on it does nothing).  volks_candidates,
 *   volks_result_peaks/_stats/_gains/_shifts/_timing work on it and refer
 *   to the last run.  Peaks are readable only for the DMs of a segment's
 *   last chunk.
 * volks_plan_timing: device time of the last run: ms_search = the search
 *   launches, ms_select = everything else (prep, select, match, clears).
 */
#define VOLKS_PLAN_AUTOTUNE 1
#define VOLKS_PLAN_GRAPH 2

typedef struct volks_plan volks_plan;

int volks_plan_create(const volks_segment *segs, const volks_params *prms, int32_t n,
                      int64_t peak_budget_bytes, int32_t flags, volks_plan **out);
int volks_plan_run(volks_plan *plan, const void *const *vis, void *cuda_stream);
int volks_plan_result(volks_plan *plan, int32_t i, volks_result **res);
int volks_plan_timing(volks_plan *plan, volks_timing *t);
/* Rounds (DM chunks) per run, device bytes held, search launches per run. */
int volks_plan_info(volks_plan *plan, int32_t *n_rounds, int64_t *device_bytes,
                    int32_t *n_search_launches_per_run);
void volks_plan_free(volks_plan *plan);

/*
 * One-shot batch search of n segments (the batching form of
 * volks_search_segment): volks_plan_create with no peak budget, no
 * autotuning and no graph, then one volks_plan_run on cuda_stream.
 * Returns the plan in *out (free it with volks_plan_free); per-segment
 * results come from volks_plan_result.  Same rules and errors as those two
 * calls (visibilities and auto spectra in device memory).
 */
int volks_search_batch(const volks_segment *segs, const volks_params *prms, int32_t n,
                       void *cuda_stream, volks_plan **out);

/* ---- request server (continuous batching) --------------------------------
 *
 * volks_server_submit queues a scan segment and returns at once.  A
 * scheduler thread admits queued requests in arrival order while one of
 * max_inflight slots (CUDA streams) is free and the request's device bytes
 * fit the remaining hbm_budget_bytes; each admitted search runs on its own
 * stream, so requests that arrive while others run share the device.  A
 * request that does not fit the budget waits at the head of the queue; one
 * whose stream's previous segment is still running is passed over.
 *
 * stream_id >= 0 chains segments of one observation: the server keeps, in
 * device memory, the last H APs of the stream's previous segment (H = the
 * largest dispersion shift of the stream's DM grid) and searches [halo |
 * segment], so pulses crossing a segment boundary are searched whole; the
 * candidates' AP indices then count from the start of that extended input,
 * which begins at stream AP volks_request_info.ap_offset.  All segments of
 * a stream need the same n_bl and n_f, at least H APs and no larger sweep,
 * one polarisation product and no auto spectra (VOLKS_EINVAL otherwise).
 * stream_id < 0: the segment is searched alone.
 *
 * vis and autos (host or device) must stay valid until the request is
 * collected; cal and bl_st are copied at submission.  volks_server_wait blocks up to timeout_ms
 * (VOLKS_ETIMEOUT after that), then returns the candidates and removes the
 * request.  A request larger than the whole budget is refused at
 * submission (VOLKS_ENOMEM); a request whose search fails is reported by
 * volks_server_wait with its error.  fail_every > 0 makes every
 * fail_every-th admission fail with VOLKS_ENOMEM before it touches the
 * device (host-side fault injection for tests).
 */
typedef struct {
  int32_t max_inflight;       /* concurrent requests on the device, 1..64 */
  int32_t fail_every;         /* 0: off */
  int64_t hbm_budget_bytes;   /* admission budget for request scratch */
} volks_server_config;

typedef struct {
  int32_t status;             /* 0 done, < 0 VOLKS_E* */
  int32_t _pad;
  double queue_ms;            /* submit -> admission */
  double latency_ms;          /* submit -> candidates ready on the host */
  int64_t device_bytes;       /* budget charged */
  int64_t ap_offset;          /* stream AP index of the searched input's AP 0 */
  int64_t trials;
} volks_request_info;

typedef struct {
  int64_t submitted, completed, failed;
  int32_t queued, inflight, peak_inflight, _pad;
  int64_t bytes_in_use, peak_bytes;
  double p50_ms, p99_ms, mean_ms;   /* latency of completed requests */
  int64_t trials;                   /* trials of completed requests */
  double trials_per_s;              /* over first submission .. last completion */
} volks_server_stats;

typedef struct volks_server volks_server;

int volks_server_create(const volks_server_config *cfg, volks_server **out);
int volks_server_submit(volks_server *srv, const volks_segment *seg, const volks_params *prm,
                        int64_t stream_id, uint64_t *request_id);
int volks_server_wait(volks_server *srv, uint64_t request_id, int32_t timeout_ms,
                      volks_candidate *buf, size_t cap, size_t *n_total,
                      volks_request_info *info);
int volks_server_get_stats(volks_server *srv, volks_server_stats *stats);
/* Wait (up to timeout_ms) until no request is queued or running. */
int volks_server_drain(volks_server *srv, int32_t timeout_ms);
/* Stops admitting, waits for running requests, frees everything. */
void volks_server_free(volks_server *srv);

/*
 * Re-fit of detected pulses for localisation (Sec. 3.1.2: the pulse's
 * visibilities are extracted and fitted again, and an SNR derived).  Per
 * candidate (its bl, dm_idx, [t0_ap, t1_ap) and rate_hz, e.g. from
 * volks_candidates of the same result): the search's normalised,
 * calibrated, polarisation-combined visibilities of baseline bl,
 * dedispersed at DM dm_idx, over APs t0_ap .. t1_ap - 1, summed coherently
 * after removing the fringe rate, S(k) = sum_u X[t0 + u, k] exp(-2 pi i
 * rate_hz u t_ap); delay transform over all n_f points zero-padded by pad
 * (a power of two 1..32, pad * n_f <= 16384), peak cell m* (lowest on
 * ties, signed), delay m* / (pad n_f chan_bw), SNR |G(m*)| / sqrt(W
 * N_eff) (W = t1_ap - t0_ap; for unit-normalised noise a pulse of
 * amplitude a per point gives a sqrt(W N_eff)), amplitude |G(m*)| /
 * sum_k |S(k)|.  FP32 on the device; waits for the search first.
 * res: a volks_search_segment or volks_plan_result handle (its data stay
 * on the device until volks_free / volks_plan_free).  cands, out: host,
 * n entries.  Errors: VOLKS_EINVAL (bad pad, a candidate outside the
 * search's baselines, DMs or dedispersed APs, or longer than 1024 APs).
 */
typedef struct {
  double delay_s;       /* delay of the peak on the pad * n_f grid */
  double snr;           /* |G| / sqrt(W N_eff) */
  double amp;           /* |G| / sum_k |S(k)| */
  int32_t delay_idx;    /* signed cell, -pad n_f / 2 .. pad n_f / 2 - 1 */
  int32_t n_ap;         /* W */
} volks_refit;

int volks_refit_pulses(volks_result *res, const volks_candidate *cands, int32_t n, int32_t pad,
                       volks_refit *out);

/*
 * Single-pulse localisation (Sec. 2.3, Eq. 2, with the rules of Sec.
 * 3.1.2).  Host only, no device work.  One volks_loc_obs per baseline on
 * which the pulse was fitted:
 *   tau_s        residual delay of the pulse's fringe fit (s)
 *   tau_cal_s    fine-calibration delay: the fringe-fit delay of a nearby
 *                reference source on the same baseline (s)
 *   dtau_dalpha, dtau_ddelta
 *                partial derivatives of the geometric delay with respect to
 *                right ascension and declination at the a priori position
 *                (s/rad), supplied by the caller's geometry model
 *   snr          the fit's SNR;  proj_len_m  the projected baseline length
 * Baselines with snr > min_snr and |proj_len_m| <= max_proj_len_m are used
 * (longer ones have an ambiguous delay); with fewer than min_baselines
 * (>= 2) left, status = 1.  The offset x = (dalpha, ddelta) rad is the
 * least-squares solution of tau - tau_cal = dtau/dalpha dalpha +
 * dtau/ddelta ddelta over the used baselines (QR by modified Gram-Schmidt
 * in FP64); status = 2 when their partials have numerical rank < 2
 * (R22 <= 1e-12 max(R11, |column 2|)).  cov = sigma^2 (A^T A)^-1 with sigma^2 = RSS /
 * (n - 2) (0 for n = 2), rms_s the rms residual.  Leave-one-out (n >= 3):
 * the solution without each used baseline in turn; with n >= 4 and every
 * such system of rank 2, d_i = distance of solution i from the
 * coordinate-wise median of all of them, and the baseline with the largest
 * d_i (first on ties) is flagged when d_i > outlier_factor * median(d)
 * (a bad baseline perturbs every solution that includes it, so the one
 * that excludes it stands out); x_clean is the solution without it (= x
 * when none is flagged).
 * obs: host, n entries.  used_out: host, n bytes (1 = used), or NULL.
 * loo_out: host, float64 [n][2], row i = solution without baseline i for
 * used baselines (NaN for unused ones or rank-deficient systems), or NULL.
 * Errors: VOLKS_EINVAL (NULL obs/out with n > 0, n < 0, min_baselines < 2,
 * a non-finite input on a used baseline).
 */
typedef struct {
  double tau_s, tau_cal_s, dtau_dalpha, dtau_ddelta, snr, proj_len_m;
} volks_loc_obs;

typedef struct {
  double min_snr;         /* 6 (Sec. 3.1.2) */
  double max_proj_len_m;  /* 3.0e6 (Sec. 3.1.2) */
  int32_t min_baselines;  /* 3 (Sec. 3.1.2) */
  double outlier_factor;  /* 5 */
} volks_loc_params;

typedef struct {
  int32_t status;         /* 0 solved, 1 too few baselines, 2 collinear partials */
  int32_t n_used;
  int32_t outlier;        /* index into obs of the flagged baseline, or -1 */
  double x[2];            /* (dalpha, ddelta) rad, all used baselines */
  double cov[4];          /* row-major 2x2 */
  double rms_s;
  double x_clean[2];
} volks_loc_result;

int volks_loc_default_params(volks_loc_params *p);
int volks_localize(const volks_loc_obs *obs, int32_t n, const volks_loc_params *p,
                   volks_loc_result *out, uint8_t *used_out, double *loo_out);

/* ---- no-allocation variant ---------------------------------------------
 *
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory while they run: for example a
 * real-time correlator or streaming service that reserves the whole GPU at
 * start-up and cannot afford allocator latency or an out-of-memory failure
 * in the middle of an observation, or a host framework whose own allocator
 * owns the device-memory budget.
 *
 * volks_search_peaks_noalloc runs the per-segment peak search of
 * volks_search_segment (steps a1-a7: shift table, FP64 channel
 * normalisation, calibration, dedispersion, delay and rate transforms,
 * peak search) on `cuda_stream` and writes, for every (baseline, DM trial,
 * segment), its peak power and peak cell.  It calls no cudaMalloc,
 * cudaFree or other allocating routine: all scratch lives in one static
 * device array of VOLKS_NOALLOC_SCRATCH_BYTES that every device which loads
 * this library holds until the process exits.
 *
 *   seg->vis      device memory of the current device (host pointers and
 *                 other devices' memory are rejected), as for
 *                 volks_search_segment; seg->cal host memory or NULL, at
 *                 most 256 (n_bl * n_if) entries.
 *   peak_power    device memory of the current device, float
 *                 [n_bl][n_dm][S]: max |Z|^2 of the segment.
 *   peak_cell     device memory of the current device, int32
 *                 [n_bl][n_dm][S]: q * M + m of that cell (unsigned rate
 *                 cell q, delay cell m, M = pad_delay*n_f).
 *   S = sum_i floor(n_ap / win[i]); window i's segments start at
 *   sum_{j<i} floor(n_ap / win[j]); segment s of window i exists while
 *   s < max(0, n_valid) / win[i] (n_valid as in volks_shift_table); the
 *   entries past that hold power 0 and cell -1.
 *
 * Returns VOLKS_EINVAL (nothing launched) for a segment whose scratch
 * (about 8 bytes per visibility + 8 bytes per output entry + tables)
 * exceeds VOLKS_NOALLOC_SCRATCH_BYTES, for two polarisation products or
 * auto spectra (one product, cross-spectrum normalisation only), or for
 * the descriptors volks_search_segment rejects; VOLKS_ECUDA if a launch
 * fails.  Returns without waiting for the device.
 *
 * All calls on a device share the one scratch array, which keeps the
 * previous call's contents; every part of it that a call reads is first
 * written by that call on its own stream (no part needs to start at zero,
 * so nothing is cleared).  Calls that overlap on the GPU (different streams or
 * host threads) race on the array and must be serialised by the caller.
 * The first call on each device looks up the array's device address with
 * that device current; make that first call before any stream capture.
 */
#define VOLKS_NOALLOC_SCRATCH_BYTES (64u << 20)

int volks_search_peaks_noalloc(const volks_segment *seg, const volks_params *prm,
                               void *cuda_stream, float *peak_power, int32_t *peak_cell);


#ifdef __cplusplus
}
#endif
#endif /* VOLKS_H */
