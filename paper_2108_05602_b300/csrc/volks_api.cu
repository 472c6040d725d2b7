// Host side of the C ABI declared in include/volks.h: validation, the FP64
// shift table, stream-ordered scratch, kernel launches, the cross-baseline
// match (a10) and result accessors.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <set>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/volks.h"
#include "volks_internal.h"

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  const int code = (e == cudaErrorMemoryAllocation) ? VOLKS_ENOMEM : VOLKS_ECUDA;
  return fail(code, "%s: %s", what, cudaGetErrorString(e));
}

// Cold-plasma dispersion constant, s MHz^2 pc^-1 cm^3.
constexpr double kDispersion = 4.148808e3;
constexpr double kTwoPi = 6.283185307179586476925286766559;

bool is_pow2(long long x) { return x > 0 && (x & (x - 1)) == 0; }
int ilog2i(int x) {
  int l = 0;
  while ((1 << l) < x) ++l;
  return l;
}

}  // namespace

void vk::set_last_error(const char* msg) { g_err = msg; }

struct volks_result {
  cudaStream_t stream = nullptr;
  volks_segment seg{};
  volks_params prm{};
  int n_f = 0, M = 0, n_eff = 0, n_tiles = 0;
  int win_log[vk::kMaxWinLog + 1] = {};
  int win_off[vk::kMaxWinLog + 1] = {};   // segment offset, by window index
  int word_off[vk::kMaxWinLog + 1] = {};  // bit-word offset, by window index
  long long seg_per_bd = 0, word_per_bd = 0;
  std::vector<int32_t> shifts, nvalid;
  const float2* d_vis = nullptr;          // caller's device buffer or our copy
  void* d_vis_copy = nullptr;
  float2* d_xn = nullptr;
  double* d_part = nullptr;
  double2* d_phasor = nullptr;
  float2* d_gain = nullptr;
  int32_t* d_shifts = nullptr;
  int32_t* d_nvalid = nullptr;
  float2* d_tw_n = nullptr;
  float2* d_tw_m = nullptr;
  unsigned long long* d_keys = nullptr;
  double* d_stats = nullptr;
  uint32_t* d_bits = nullptr;
  vk::DevCand* d_cand = nullptr;
  unsigned int* d_count = nullptr;
  unsigned int cap = 0;
  cudaEvent_t ev[6] = {};
  int n_launch = 0, n_search_launch = 0;
  bool empty = true, synced = false, have_cands = false;
  std::vector<volks_candidate> cands;
  // host staging that must outlive the asynchronous copies
  std::vector<double2> h_phasor;
  std::vector<float2> h_tw_n, h_tw_m;
  vk::MatchArgs match_args{};
};

namespace {

template <class T>
cudaError_t dalloc(T** p, size_t n, cudaStream_t s) {
  *p = nullptr;
  if (n == 0) return cudaSuccess;
  return cudaMallocAsync(reinterpret_cast<void**>(p), n * sizeof(T), s);
}

void release(volks_result* r) {
  if (!r) return;
  void* ptrs[] = {r->d_vis_copy, r->d_xn, r->d_part, r->d_phasor, r->d_gain, r->d_shifts,
                  r->d_nvalid, r->d_tw_n, r->d_tw_m, r->d_keys, r->d_stats, r->d_bits,
                  r->d_cand, r->d_count};
  for (void* p : ptrs)
    if (p) cudaFreeAsync(p, r->stream);
  // the host staging vectors may still feed in-flight copies
  if (!r->synced) cudaStreamSynchronize(r->stream);
  for (auto& e : r->ev)
    if (e) cudaEventDestroy(e);
  delete r;
}

int validate(const volks_segment* s, const volks_params* p) {
  if (!s || !p) return fail(VOLKS_EINVAL, "NULL segment or params");
  if (s->n_bl < 0 || s->n_ap < 0) return fail(VOLKS_EINVAL, "negative n_bl or n_ap");
  if (s->n_if < 1 || s->n_chan < 1) return fail(VOLKS_EINVAL, "n_if and n_chan must be >= 1");
  const long long n_f = (long long)s->n_if * s->n_chan;
  if (!is_pow2(n_f) || n_f < 64 || n_f > 2048)
    return fail(VOLKS_EINVAL, "n_if*n_chan = %lld: this build supports powers of two 64..2048", n_f);
  if (!(std::isfinite(s->t_ap_s) && s->t_ap_s > 0)) return fail(VOLKS_EINVAL, "t_ap_s must be > 0");
  if (!(std::isfinite(s->chan_bw_mhz) && s->chan_bw_mhz > 0))
    return fail(VOLKS_EINVAL, "chan_bw_mhz must be > 0");
  if (!(std::isfinite(s->f_lo_mhz) && s->f_lo_mhz > 0)) return fail(VOLKS_EINVAL, "f_lo_mhz must be > 0");
  if ((long long)s->n_bl * s->n_ap > 0 && !s->vis) return fail(VOLKS_EINVAL, "vis is NULL");
  if (p->n_dm < 0) return fail(VOLKS_EINVAL, "n_dm < 0");
  if (!std::isfinite(p->dm_lo) || !std::isfinite(p->dm_step)) return fail(VOLKS_EINVAL, "DM grid not finite");
  if (p->n_dm > 0 && (p->dm_lo < 0 || p->dm_lo + p->dm_step * (p->n_dm - 1) < 0))
    return fail(VOLKS_EINVAL, "negative DM trial");
  if (p->n_win < 1 || p->n_win > VOLKS_MAX_WIN) return fail(VOLKS_EINVAL, "n_win must be 1..%d", VOLKS_MAX_WIN);
  for (int i = 0; i < p->n_win; ++i) {
    if (!is_pow2(p->win[i]) || p->win[i] > 32) return fail(VOLKS_EINVAL, "win[%d] = %d: powers of two 1..32 only", i, p->win[i]);
    if (i > 0 && p->win[i] <= p->win[i - 1]) return fail(VOLKS_EINVAL, "windows must be strictly ascending");
  }
  if (!(p->pad_delay == 1 || p->pad_delay == 2 || p->pad_delay == 4 || p->pad_delay == 8))
    return fail(VOLKS_EINVAL, "pad_delay must be 1, 2, 4 or 8");
  if (!(p->pad_rate == 0 || p->pad_rate == 4)) return fail(VOLKS_EINVAL, "pad_rate must be 0 or 4");
  if (p->precision != VOLKS_FP32) return fail(VOLKS_EINVAL, "precision %d not available", p->precision);
  if (!std::isfinite(p->thresh)) return fail(VOLKS_EINVAL, "thresh not finite");
  if (p->min_windows < 1 || p->min_baselines < 1) return fail(VOLKS_EINVAL, "min_windows and min_baselines must be >= 1");
  if ((p->normalize_chan & ~1) || (p->skip_first_chan & ~1)) return fail(VOLKS_EINVAL, "flags must be 0 or 1");
  return 0;
}

int sync_result(volks_result* r) {
  if (r->synced) return 0;
  cudaError_t e = cudaStreamSynchronize(r->stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  r->synced = true;
  return 0;
}

#define VK_TRY(expr, what)                              \
  do {                                                  \
    cudaError_t e_ = (expr);                            \
    if (e_ != cudaSuccess) {                            \
      int rc_ = cuda_fail(e_, what);                    \
      release(r);                                       \
      return rc_;                                       \
    }                                                   \
  } while (0)

// a1 (see volks_shift_table in volks.h).
int shift_table(double f_lo_mhz, double chan_bw_mhz, int n_f, double t_ap_s, int n_ap, double dm_lo,
                double dm_step, int n_dm, int32_t* shifts, int32_t* nvalid) {
  std::vector<double> f(n_f);
  for (int k = 0; k < n_f; ++k) f[k] = f_lo_mhz + (k + 0.5) * chan_bw_mhz;
  const double ftop = f[n_f - 1];
  for (int d = 0; d < n_dm; ++d) {
    const double dm = dm_lo + dm_step * d;
    int mx = 0;
    for (int k = 0; k < n_f; ++k) {
      const double x = (kDispersion * dm / t_ap_s) * (1.0 / (f[k] * f[k]) - 1.0 / (ftop * ftop));
      const double sh = std::floor(x + 0.5);
      if (!(sh < 2.0e9 && sh > -2.0e9)) return fail(VOLKS_EINVAL, "dispersion shift overflows at DM %g", dm);
      if (shifts) shifts[(size_t)d * n_f + k] = (int32_t)sh;
      mx = std::max(mx, (int)sh);
    }
    if (nvalid) nvalid[d] = n_ap - mx;
  }
  return 0;
}

// a10 (Sec. 3.1.1 item 3): at one DM, entries of different baselines whose
// representative intervals [t0_ap, t1_ap) overlap are one pulse; keep the
// pulses seen on >= min_baselines distinct baselines, each entry carrying
// n_baselines; output sorted by (dm_idx, t0_ap, bl).
std::vector<volks_candidate> cross_match(std::vector<volks_candidate> all, int min_baselines) {
  std::sort(all.begin(), all.end(), [](const volks_candidate& a, const volks_candidate& b) {
    if (a.dm_idx != b.dm_idx) return a.dm_idx < b.dm_idx;
    if (a.t0_ap != b.t0_ap) return a.t0_ap < b.t0_ap;
    if (a.t1_ap != b.t1_ap) return a.t1_ap < b.t1_ap;
    return a.bl < b.bl;
  });
  std::vector<volks_candidate> out;
  size_t i = 0;
  while (i < all.size()) {
    size_t j = i + 1;
    int end = all[i].t1_ap;
    while (j < all.size() && all[j].dm_idx == all[i].dm_idx && all[j].t0_ap < end) {
      end = std::max(end, all[j].t1_ap);
      ++j;
    }
    std::set<int> bls;
    for (size_t k = i; k < j; ++k) bls.insert(all[k].bl);
    if ((int)bls.size() >= min_baselines)
      for (size_t k = i; k < j; ++k) {
        all[k].n_baselines = (int)bls.size();
        out.push_back(all[k]);
      }
    i = j;
  }
  std::stable_sort(out.begin(), out.end(), [](const volks_candidate& a, const volks_candidate& b) {
    if (a.dm_idx != b.dm_idx) return a.dm_idx < b.dm_idx;
    if (a.t0_ap != b.t0_ap) return a.t0_ap < b.t0_ap;
    return a.bl < b.bl;
  });
  return out;
}

int launch_match_into(volks_result* r) {
  r->match_args.out = r->d_cand;
  r->match_args.cap = r->cap;
  cudaError_t e = cudaMemsetAsync(r->d_count, 0, sizeof(unsigned int), r->stream);
  if (e != cudaSuccess) return cuda_fail(e, "memset count");
  e = vk::launch_match(r->match_args, r->stream, &r->n_launch);
  if (e != cudaSuccess) return cuda_fail(e, "match kernel");
  return 0;
}

}  // namespace

extern "C" {

const char* volks_last_error(void) { return g_err.c_str(); }

void volks_default_params(volks_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof *p);
  p->dm_lo = 0.0;
  p->dm_step = 1.0;
  p->n_dm = 1;
  p->n_win = 4;
  p->win[0] = 2;
  p->win[1] = 4;
  p->win[2] = 8;
  p->win[3] = 16;
  p->pad_delay = 4;
  p->pad_rate = 4;
  p->thresh = 3.0;
  p->min_windows = 2;
  p->min_baselines = 5;
  p->precision = VOLKS_FP32;
  p->normalize_chan = 1;
  p->skip_first_chan = 0;
}

int volks_search_segment(const volks_segment* seg, const volks_params* prm, void* cuda_stream,
                         volks_result** out) {
  if (!out) return fail(VOLKS_EINVAL, "out is NULL");
  *out = nullptr;
  int rc = validate(seg, prm);
  if (rc) return rc;

  volks_result* r = new (std::nothrow) volks_result();
  if (!r) return fail(VOLKS_ENOMEM, "host allocation");
  r->stream = static_cast<cudaStream_t>(cuda_stream);
  r->seg = *seg;
  r->prm = *prm;
  const int n_bl = seg->n_bl, n_ap = seg->n_ap, n_f = seg->n_if * seg->n_chan;
  const int n_dm = prm->n_dm, n_win = prm->n_win;
  r->n_f = n_f;
  r->M = prm->pad_delay * n_f;
  r->n_eff = n_f - (prm->skip_first_chan ? seg->n_if : 0);
  r->n_tiles = (n_ap + vk::kTile - 1) / vk::kTile;
  int win_mask = 0;
  long long so = 0, wo = 0;
  for (int i = 0; i < n_win; ++i) {
    r->win_log[i] = ilog2i(prm->win[i]);
    r->win_off[i] = (int)so;
    r->word_off[i] = (int)wo;
    const long long ns = n_ap / prm->win[i];
    so += ns;
    wo += (ns + 31) / 32;
    win_mask |= 1 << r->win_log[i];
  }
  r->seg_per_bd = so;
  r->word_per_bd = wo;

  // a1: shift table, FP64 on the host, rounded half-up (Sec. 2.4.2 step 4).
  r->shifts.resize((size_t)n_dm * n_f);
  r->nvalid.resize(n_dm);
  rc = shift_table(seg->f_lo_mhz, seg->chan_bw_mhz, n_f, seg->t_ap_s, n_ap, prm->dm_lo, prm->dm_step,
                   n_dm, r->shifts.data(), r->nvalid.data());
  if (rc) {
    release(r);
    return rc;
  }
  r->empty = ((long long)n_bl * n_ap * n_dm == 0);

  for (auto& e : r->ev) VK_TRY(cudaEventCreate(&e), "cudaEventCreate");
  cudaStream_t st = r->stream;
  VK_TRY(cudaEventRecord(r->ev[0], st), "event");

  // candidates buffer exists even for an empty search
  r->cap = (unsigned)std::max<long long>(4096, std::min<long long>(1LL << 24, (long long)n_bl * n_dm * 64));
  VK_TRY(dalloc(&r->d_cand, r->cap, st), "alloc candidates");
  VK_TRY(dalloc(&r->d_count, 1, st), "alloc count");
  VK_TRY(cudaMemsetAsync(r->d_count, 0, sizeof(unsigned int), st), "memset count");

  if (r->empty) {
    for (int i = 1; i < 6; ++i) VK_TRY(cudaEventRecord(r->ev[i], st), "event");
    *out = r;
    return 0;
  }

  // input: the caller's device buffer, or a stream-ordered copy of host memory
  const size_t vis_n = (size_t)n_bl * n_ap * n_f;
  cudaPointerAttributes attr{};
  cudaError_t pe = cudaPointerGetAttributes(&attr, seg->vis);
  if (pe != cudaSuccess) {
    cudaGetLastError();
    attr.type = cudaMemoryTypeUnregistered;
  }
  if (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged) {
    r->d_vis = static_cast<const float2*>(seg->vis);
  } else {
    VK_TRY(cudaMallocAsync(&r->d_vis_copy, vis_n * sizeof(float2), st), "alloc vis copy");
    VK_TRY(cudaMemcpyAsync(r->d_vis_copy, seg->vis, vis_n * sizeof(float2), cudaMemcpyHostToDevice, st),
           "copy vis to device");
    r->d_vis = static_cast<const float2*>(r->d_vis_copy);
  }
  VK_TRY(cudaEventRecord(r->ev[1], st), "event");

  // calibration phasor (FP64) and FFT twiddles, computed on the host
  r->h_phasor.resize((size_t)n_bl * n_f);
  for (int b = 0; b < n_bl; ++b)
    for (int k = 0; k < n_f; ++k) {
      const int n = k / seg->n_chan, j = k % seg->n_chan;
      double ph = 0.0;
      if (seg->cal) {
        const double fj = (j + 0.5) * seg->chan_bw_mhz * 1e6;
        ph = kTwoPi * fj * seg->cal[((size_t)b * seg->n_if + n) * 2 + 0] + seg->cal[((size_t)b * seg->n_if + n) * 2 + 1];
      }
      r->h_phasor[(size_t)b * n_f + k] = make_double2(std::cos(ph), -std::sin(ph));
    }
  r->h_tw_n.resize(n_f);
  for (int i = 0; i < n_f; ++i)
    r->h_tw_n[i] = make_float2((float)std::cos(kTwoPi * i / n_f), (float)-std::sin(kTwoPi * i / n_f));
  r->h_tw_m.resize(r->M);
  for (int i = 0; i < r->M; ++i)
    r->h_tw_m[i] = make_float2((float)std::cos(kTwoPi * i / r->M), (float)-std::sin(kTwoPi * i / r->M));

  const int tchunk = 1024;
  const int n_tchunk = (n_ap + tchunk - 1) / tchunk;
  VK_TRY(dalloc(&r->d_xn, vis_n, st), "alloc normalised copy");
  VK_TRY(dalloc(&r->d_part, (size_t)n_bl * n_tchunk * n_f, st), "alloc partial sums");
  VK_TRY(dalloc(&r->d_phasor, (size_t)n_bl * n_f, st), "alloc phasor");
  VK_TRY(dalloc(&r->d_gain, (size_t)n_bl * n_f, st), "alloc gains");
  VK_TRY(dalloc(&r->d_shifts, (size_t)n_dm * n_f, st), "alloc shifts");
  VK_TRY(dalloc(&r->d_nvalid, (size_t)n_dm, st), "alloc nvalid");
  VK_TRY(dalloc(&r->d_tw_n, (size_t)n_f, st), "alloc twiddles");
  VK_TRY(dalloc(&r->d_tw_m, (size_t)r->M, st), "alloc twiddles");
  const size_t n_keys = (size_t)n_bl * n_dm * r->seg_per_bd;
  VK_TRY(dalloc(&r->d_keys, n_keys, st), "alloc peaks");
  VK_TRY(dalloc(&r->d_stats, (size_t)n_bl * n_dm * n_win * 2, st), "alloc stats");
  VK_TRY(dalloc(&r->d_bits, (size_t)n_bl * n_dm * r->word_per_bd, st), "alloc bitmaps");
  VK_TRY(cudaMemcpyAsync(r->d_phasor, r->h_phasor.data(), r->h_phasor.size() * sizeof(double2),
                         cudaMemcpyHostToDevice, st), "copy phasor");
  VK_TRY(cudaMemcpyAsync(r->d_shifts, r->shifts.data(), r->shifts.size() * sizeof(int32_t),
                         cudaMemcpyHostToDevice, st), "copy shifts");
  VK_TRY(cudaMemcpyAsync(r->d_nvalid, r->nvalid.data(), r->nvalid.size() * sizeof(int32_t),
                         cudaMemcpyHostToDevice, st), "copy nvalid");
  VK_TRY(cudaMemcpyAsync(r->d_tw_n, r->h_tw_n.data(), r->h_tw_n.size() * sizeof(float2),
                         cudaMemcpyHostToDevice, st), "copy twiddles");
  VK_TRY(cudaMemcpyAsync(r->d_tw_m, r->h_tw_m.data(), r->h_tw_m.size() * sizeof(float2),
                         cudaMemcpyHostToDevice, st), "copy twiddles");
  VK_TRY(cudaMemsetAsync(r->d_keys, 0, n_keys * sizeof(unsigned long long), st), "memset peaks");

  // a2-a3
  vk::PrepArgs pa{};
  pa.vis = r->d_vis;
  pa.xn = r->d_xn;
  pa.part = r->d_part;
  pa.phasor = r->d_phasor;
  pa.gain = r->d_gain;
  pa.n_bl = n_bl;
  pa.n_ap = n_ap;
  pa.n_f = n_f;
  pa.n_chan = seg->n_chan;
  pa.n_tchunk = n_tchunk;
  pa.tchunk = tchunk;
  pa.normalize = prm->normalize_chan;
  pa.skip_first_chan = prm->skip_first_chan;
  VK_TRY(vk::launch_prep(pa, st, &r->n_launch), "prep kernels");
  VK_TRY(cudaEventRecord(r->ev[2], st), "event");

  // a4-a7
  vk::SearchArgs sa{};
  sa.xn = r->d_xn;
  sa.shifts = r->d_shifts;
  sa.nvalid = r->d_nvalid;
  sa.tw_n = r->d_tw_n;
  sa.tw_m = r->d_tw_m;
  sa.keys = r->d_keys;
  sa.n_bl = n_bl;
  sa.n_ap = n_ap;
  sa.n_f = n_f;
  sa.n_dm = n_dm;
  sa.pad_delay = prm->pad_delay;
  sa.M = r->M;
  sa.win_mask = win_mask;
  for (int i = 0; i < n_win; ++i) sa.win_off[r->win_log[i]] = r->win_off[i];
  sa.seg_per_bd = r->seg_per_bd;
  sa.n_tiles = r->n_tiles;
  sa.fold = 1;  // measured: one 512-thread CTA beats two folded 256-thread CTAs at n_f = 512
  if (const char* f = std::getenv("VOLKS_SEARCH_FOLD")) sa.fold = std::atoi(f);
  const int before = r->n_launch;
  VK_TRY(vk::launch_search(sa, prm->pad_rate, st, &r->n_launch), "search kernel");
  r->n_search_launch = r->n_launch - before;
  VK_TRY(cudaEventRecord(r->ev[3], st), "event");

  // a8
  vk::SelectArgs ea{};
  ea.keys = r->d_keys;
  ea.nvalid = r->d_nvalid;
  ea.stats = r->d_stats;
  ea.bits = r->d_bits;
  ea.n_bl = n_bl;
  ea.n_dm = n_dm;
  ea.n_win = n_win;
  ea.n_eff = r->n_eff;
  for (int i = 0; i < n_win; ++i) {
    ea.win_log[i] = r->win_log[i];
    ea.win_off[i] = r->win_off[i];
    ea.word_off[i] = r->word_off[i];
  }
  ea.seg_per_bd = r->seg_per_bd;
  ea.word_per_bd = r->word_per_bd;
  ea.thresh = prm->thresh;
  VK_TRY(vk::launch_select(ea, st, &r->n_launch), "select kernel");
  VK_TRY(cudaEventRecord(r->ev[4], st), "event");

  // a9
  vk::MatchArgs& ma = r->match_args;
  ma.keys = r->d_keys;
  ma.stats = r->d_stats;
  ma.bits = r->d_bits;
  ma.nvalid = r->d_nvalid;
  ma.count = r->d_count;
  ma.n_bl = n_bl;
  ma.n_dm = n_dm;
  ma.n_win = n_win;
  ma.n_eff = r->n_eff;
  ma.min_windows = prm->min_windows;
  for (int i = 0; i < n_win; ++i) {
    ma.win_log[i] = r->win_log[i];
    ma.win_off[i] = r->win_off[i];
    ma.word_off[i] = r->word_off[i];
  }
  ma.seg_per_bd = r->seg_per_bd;
  ma.word_per_bd = r->word_per_bd;
  rc = launch_match_into(r);
  if (rc) {
    release(r);
    return rc;
  }
  VK_TRY(cudaEventRecord(r->ev[5], st), "event");
  *out = r;
  return 0;
}

int volks_candidates(volks_result* r, volks_candidate* buf, size_t cap, size_t* n_total) {
  if (!r || !n_total) return fail(VOLKS_EINVAL, "NULL result or n_total");
  if (cap > 0 && !buf) return fail(VOLKS_EINVAL, "NULL buffer with cap > 0");
  if (!r->have_cands) {
    int rc = sync_result(r);
    if (rc) return rc;
    unsigned int count = 0;
    cudaError_t e = cudaMemcpy(&count, r->d_count, sizeof count, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "read candidate count");
    if (count > r->cap) {  // grow and re-run the window match only
      cudaFreeAsync(r->d_cand, r->stream);
      r->cap = count;
      e = dalloc(&r->d_cand, r->cap, r->stream);
      if (e != cudaSuccess) return cuda_fail(e, "grow candidates");
      r->synced = false;
      rc = launch_match_into(r);
      if (rc) return rc;
      rc = sync_result(r);
      if (rc) return rc;
      e = cudaMemcpy(&count, r->d_count, sizeof count, cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) return cuda_fail(e, "read candidate count");
    }
    std::vector<vk::DevCand> dc(count);
    if (count) {
      e = cudaMemcpy(dc.data(), r->d_cand, count * sizeof(vk::DevCand), cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) return cuda_fail(e, "read candidates");
    }
    const volks_segment& s = r->seg;
    const volks_params& p = r->prm;
    std::vector<volks_candidate> all(count);
    for (unsigned i = 0; i < count; ++i) {
      const vk::DevCand& c = dc[i];
      volks_candidate& o = all[i];
      std::memset(&o, 0, sizeof o);
      const int W = 1 << c.win_log;
      const int R = (W == 1 || p.pad_rate == 0) ? 1 : p.pad_rate * W;
      const int q = (int)(c.lin / (uint32_t)r->M), m = (int)(c.lin % (uint32_t)r->M);
      o.bl = c.bl;
      o.dm_idx = c.dm_idx;
      o.win = W;
      o.seg = c.seg;
      o.t0_ap = c.seg * W;
      o.t1_ap = o.t0_ap + W;
      o.g0_ap = c.g0;
      o.g1_ap = c.g1;
      o.delay_idx = m >= r->M / 2 ? m - r->M : m;
      o.rate_idx = (R > 1 && q >= R / 2) ? q - R : q;
      o.n_windows = c.n_windows;
      o.peak_power = c.P;
      o.rho = c.rho;
      o.z = c.z;
      o.dm = p.dm_lo + p.dm_step * c.dm_idx;
      o.delay_s = o.delay_idx / (r->M * s.chan_bw_mhz * 1e6);
      o.rate_hz = o.rate_idx / (R * s.t_ap_s);
    }
    // a10: cross-baseline match per DM over representative intervals
    r->cands = cross_match(all, p.min_baselines);
    r->have_cands = true;
  }
  *n_total = r->cands.size();
  const size_t n = std::min(cap, r->cands.size());
  if (n) std::memcpy(buf, r->cands.data(), n * sizeof(volks_candidate));
  return 0;
}

void volks_free(volks_result* r) { release(r); }

int volks_cross_match(const volks_candidate* in, size_t n, int32_t min_baselines, volks_candidate* out,
                      size_t cap, size_t* n_out) {
  if (!n_out || (n > 0 && !in) || (cap > 0 && !out)) return fail(VOLKS_EINVAL, "NULL argument");
  if (min_baselines < 1) return fail(VOLKS_EINVAL, "min_baselines must be >= 1");
  std::vector<volks_candidate> v(in, in + n);
  v = cross_match(std::move(v), min_baselines);
  *n_out = v.size();
  const size_t k = std::min(cap, v.size());
  if (k) std::memcpy(out, v.data(), k * sizeof(volks_candidate));
  return 0;
}

int volks_shift_table(double f_lo_mhz, double chan_bw_mhz, int32_t n_f, double t_ap_s, int32_t n_ap,
                      double dm_lo, double dm_step, int32_t n_dm, int32_t* shifts, int32_t* nvalid) {
  volks_segment s{};
  s.n_bl = 0;
  s.n_ap = n_ap;
  s.n_if = 1;
  s.n_chan = n_f;
  s.t_ap_s = t_ap_s;
  s.f_lo_mhz = f_lo_mhz;
  s.chan_bw_mhz = chan_bw_mhz;
  volks_params p;
  volks_default_params(&p);
  p.dm_lo = dm_lo;
  p.dm_step = dm_step;
  p.n_dm = n_dm;
  int rc = validate(&s, &p);
  if (rc) return rc;
  return shift_table(f_lo_mhz, chan_bw_mhz, n_f, t_ap_s, n_ap, dm_lo, dm_step, n_dm, shifts, nvalid);
}

int volks_result_timing(volks_result* r, volks_timing* t) {
  if (!r || !t) return fail(VOLKS_EINVAL, "NULL argument");
  int rc = sync_result(r);
  if (rc) return rc;
  std::memset(t, 0, sizeof *t);
  float* dst[5] = {&t->ms_h2d, &t->ms_prep, &t->ms_search, &t->ms_select, &t->ms_match};
  for (int i = 0; i < 5; ++i) {
    cudaError_t e = cudaEventElapsedTime(dst[i], r->ev[i], r->ev[i + 1]);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventElapsedTime");
  }
  t->n_launches = r->n_launch;
  t->n_search_launches = r->n_search_launch;
  return 0;
}

int volks_result_shifts(volks_result* r, int32_t* shifts, int32_t* nvalid) {
  if (!r) return fail(VOLKS_EINVAL, "NULL result");
  if (shifts && !r->shifts.empty()) std::memcpy(shifts, r->shifts.data(), r->shifts.size() * sizeof(int32_t));
  if (nvalid && !r->nvalid.empty()) std::memcpy(nvalid, r->nvalid.data(), r->nvalid.size() * sizeof(int32_t));
  return 0;
}

int volks_result_peaks(volks_result* r, int32_t bl, int32_t dm_idx, int32_t win_idx, float* P, int32_t* q,
                       int32_t* m, size_t cap, size_t* n_seg) {
  if (!r || !n_seg) return fail(VOLKS_EINVAL, "NULL argument");
  if (bl < 0 || bl >= r->seg.n_bl || dm_idx < 0 || dm_idx >= r->prm.n_dm || win_idx < 0 ||
      win_idx >= r->prm.n_win)
    return fail(VOLKS_EINVAL, "series index out of range");
  int rc = sync_result(r);
  if (rc) return rc;
  const int W = 1 << r->win_log[win_idx];
  const size_t ns = (size_t)std::max(0, r->nvalid[dm_idx]) / W;
  *n_seg = ns;
  const size_t n = std::min(ns, cap);
  if (n == 0 || r->empty) return 0;
  std::vector<unsigned long long> k(n);
  const size_t off = ((size_t)bl * r->prm.n_dm + dm_idx) * r->seg_per_bd + r->win_off[win_idx];
  cudaError_t e = cudaMemcpy(k.data(), r->d_keys + off, n * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "read peaks");
  for (size_t i = 0; i < n; ++i) {
    const uint32_t hi = (uint32_t)(k[i] >> 32), lin = 0xffffffffu - (uint32_t)(k[i] & 0xffffffffu);
    float f;
    std::memcpy(&f, &hi, 4);
    if (P) P[i] = f;
    if (q) q[i] = (int32_t)(lin / (uint32_t)r->M);
    if (m) m[i] = (int32_t)(lin % (uint32_t)r->M);
  }
  return 0;
}

int volks_result_stats(volks_result* r, int32_t bl, int32_t dm_idx, int32_t win_idx, double* mean, double* sd) {
  if (!r || !mean || !sd) return fail(VOLKS_EINVAL, "NULL argument");
  if (bl < 0 || bl >= r->seg.n_bl || dm_idx < 0 || dm_idx >= r->prm.n_dm || win_idx < 0 ||
      win_idx >= r->prm.n_win)
    return fail(VOLKS_EINVAL, "series index out of range");
  int rc = sync_result(r);
  if (rc) return rc;
  if (r->empty) {
    *mean = *sd = 0.0;
    return 0;
  }
  double v[2];
  const size_t off = (((size_t)bl * r->prm.n_dm + dm_idx) * r->prm.n_win + win_idx) * 2;
  cudaError_t e = cudaMemcpy(v, r->d_stats + off, sizeof v, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "read stats");
  *mean = v[0];
  *sd = v[1];
  return 0;
}

int volks_result_gains(volks_result* r, float* gains, size_t cap_floats) {
  if (!r || !gains) return fail(VOLKS_EINVAL, "NULL argument");
  const size_t n = (size_t)r->seg.n_bl * r->n_f * 2;
  if (cap_floats < n) return fail(VOLKS_EINVAL, "gains buffer holds %zu floats, need %zu", cap_floats, n);
  int rc = sync_result(r);
  if (rc) return rc;
  if (r->empty || !r->d_gain) {
    std::memset(gains, 0, n * sizeof(float));
    return 0;
  }
  cudaError_t e = cudaMemcpy(gains, r->d_gain, n * sizeof(float), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "read gains");
  return 0;
}

}  // extern "C"
