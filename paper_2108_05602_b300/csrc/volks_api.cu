// Host side of the single-segment C ABI declared in include/volks.h:
// validation, the FP64 shift table, stream-ordered scratch, kernel
// launches, the cross-baseline match (a10) and result accessors.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <set>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/volks.h"
#include "../../include/volks_check.h"
#include "volks_internal.h"
#include "volks_job.h"
#include "volks_result.h"

namespace {

thread_local std::string g_err;

// Cold-plasma dispersion constant, s MHz^2 pc^-1 cm^3.
constexpr double kDispersion = 4.148808e3;
constexpr double kTwoPi = 6.283185307179586476925286766559;

bool is_pow2(long long x) { return x > 0 && (x & (x - 1)) == 0; }
int ilog2i(int x) {
  int l = 0;
  while ((1 << l) < x) ++l;
  return l;
}

template <class T>
cudaError_t dalloc(T** p, size_t n, cudaStream_t s, bool ordered) {
  *p = nullptr;
  if (n == 0) return cudaSuccess;
  return ordered ? cudaMallocAsync(reinterpret_cast<void**>(p), n * sizeof(T), s)
                 : cudaMalloc(reinterpret_cast<void**>(p), n * sizeof(T));
}

}  // namespace

namespace vk {

void set_last_error(const char* msg) { g_err = msg; }

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

int sm_count() {
  static std::mutex mu;
  static int cache[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
  std::lock_guard<std::mutex> lk(mu);
  if (!cache[dev]) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
    cache[dev] = n;
  }
  return cache[dev];
}

int validate(const volks_segment* s, const volks_params* p) {
  if (!s || !p) return fail(VOLKS_EINVAL, "NULL segment or params");
  if (s->n_bl < 0 || s->n_ap < 0) return fail(VOLKS_EINVAL, "negative n_bl or n_ap");
  if (s->n_if < 1 || s->n_chan < 1) return fail(VOLKS_EINVAL, "n_if and n_chan must be >= 1");
  const long long n_f = (long long)s->n_if * s->n_chan;
  const bool pow2_band = is_pow2(n_f) && n_f >= 64 && n_f <= 2048;
  const bool mixed_band = n_f % 3 == 0 && is_pow2(n_f / 3) && n_f >= 96 && n_f <= 1536;
  if (!pow2_band && !mixed_band)
    return fail(VOLKS_EINVAL,
                "n_if*n_chan = %lld: this build supports powers of two 64..2048 and 3 x powers of two 96..1536",
                n_f);
  if (!(std::isfinite(s->t_ap_s) && s->t_ap_s > 0)) return fail(VOLKS_EINVAL, "t_ap_s must be > 0");
  if (!(std::isfinite(s->chan_bw_mhz) && s->chan_bw_mhz > 0))
    return fail(VOLKS_EINVAL, "chan_bw_mhz must be > 0");
  if (!(std::isfinite(s->f_lo_mhz) && s->f_lo_mhz > 0)) return fail(VOLKS_EINVAL, "f_lo_mhz must be > 0");
  if ((long long)s->n_bl * s->n_ap > 0 && !s->vis) return fail(VOLKS_EINVAL, "vis is NULL");
  if (s->n_pol < 0 || s->n_pol > 2) return fail(VOLKS_EINVAL, "n_pol = %d: 1 or 2 products (0 means 1)", s->n_pol);
  if (s->autos && p && p->normalize_chan == 1 && (long long)s->n_bl * s->n_ap > 0) {
    if (s->n_st < 2 || !s->bl_st) return fail(VOLKS_EINVAL, "auto spectra need n_st >= 2 and bl_st");
    for (int b = 0; b < s->n_bl; ++b) {
      const int i = s->bl_st[2 * b], j = s->bl_st[2 * b + 1];
      if (i < 0 || j < 0 || i >= s->n_st || j >= s->n_st || i == j)
        return fail(VOLKS_EINVAL, "bl_st[%d] = (%d, %d): two different stations < n_st = %d", b, i, j, s->n_st);
    }
  }
  if (p->n_dm < 0) return fail(VOLKS_EINVAL, "n_dm < 0");
  if (!std::isfinite(p->dm_lo) || !std::isfinite(p->dm_step)) return fail(VOLKS_EINVAL, "DM grid not finite");
  if (p->n_dm > 0 && (p->dm_lo < 0 || p->dm_lo + p->dm_step * (p->n_dm - 1) < 0))
    return fail(VOLKS_EINVAL, "negative DM trial");
  if (p->n_win < 1 || p->n_win > VOLKS_MAX_WIN) return fail(VOLKS_EINVAL, "n_win must be 1..%d", VOLKS_MAX_WIN);
  for (int i = 0; i < p->n_win; ++i) {
    if (!is_pow2(p->win[i]) || p->win[i] > 32)
      return fail(VOLKS_EINVAL, "win[%d] = %d: powers of two 1..32 only", i, p->win[i]);
    if (i > 0 && p->win[i] <= p->win[i - 1]) return fail(VOLKS_EINVAL, "windows must be strictly ascending");
  }
  if (!(p->pad_delay == 1 || p->pad_delay == 2 || p->pad_delay == 4 || p->pad_delay == 8))
    return fail(VOLKS_EINVAL, "pad_delay must be 1, 2, 4 or 8");
  if (!(p->pad_rate == 0 || p->pad_rate == 4)) return fail(VOLKS_EINVAL, "pad_rate must be 0 or 4");
  if (p->precision < VOLKS_FP32 || p->precision > VOLKS_FP8)
    return fail(VOLKS_EINVAL, "precision %d unknown", p->precision);
  if (!std::isfinite(p->thresh)) return fail(VOLKS_EINVAL, "thresh not finite");
  if (p->min_windows < 1 || p->min_baselines < 1)
    return fail(VOLKS_EINVAL, "min_windows and min_baselines must be >= 1");
  if ((p->normalize_chan & ~1) || (p->skip_first_chan & ~1)) return fail(VOLKS_EINVAL, "flags must be 0 or 1");
  if (p->stride != 0 && p->stride != 1) return fail(VOLKS_EINVAL, "stride must be 0 (window) or 1 (sliding)");
  return 0;
}

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

// ------------------------------------------------------------- SegJob ----
int SegJob::init(const volks_segment& s, const volks_params& p, int chunk) {
  seg = s;
  prm = p;
  n_f = s.n_if * s.n_chan;
  M = p.pad_delay * n_f;
  n_eff = n_f - (p.skip_first_chan ? s.n_if : 0);
  n_tiles = (s.n_ap + kTile - 1) / kTile;
  n_tchunk = (s.n_ap + tchunk - 1) / tchunk;
  slide = p.stride == 1;
  prec = slide ? VOLKS_FP32 : effective_precision(n_f, p.pad_rate, p.precision);
  win_mask = 0;
  long long so = 0, wo = 0;
  for (int l = 0; l <= kMaxWinLog; ++l) win_off_l[l] = 0;
  for (int i = 0; i < p.n_win; ++i) {
    win_log[i] = ilog2i(p.win[i]);
    win_off[i] = (int)so;
    word_off[i] = (int)wo;
    win_off_l[win_log[i]] = (int)so;
    const long long ns = seg_count(s.n_ap, win_log[i], slide ? 1 : 0);
    so += ns;
    wo += (ns + 31) / 32;
    win_mask |= 1 << win_log[i];
  }
  seg_per_bd = so;
  word_per_bd = wo;
  dm_chunk = (chunk <= 0 || chunk > p.n_dm) ? std::max(1, p.n_dm) : chunk;
  empty = ((long long)s.n_bl * s.n_ap * p.n_dm == 0);
  shifts.assign((size_t)p.n_dm * n_f, 0);
  nvalid.assign(p.n_dm, 0);
  int rc = shift_table(s.f_lo_mhz, s.chan_bw_mhz, n_f, s.t_ap_s, s.n_ap, p.dm_lo, p.dm_step, p.n_dm,
                       shifts.data(), nvalid.data());
  if (rc) return rc;
  n_pol = s.n_pol == 2 ? 2 : 1;
  use_autos = s.autos != nullptr && p.normalize_chan == 1 && !empty;
  n_rows = n_pol * (use_autos ? s.n_st : s.n_bl);
  const size_t n_pb = (size_t)n_pol * s.n_bl;
  h_phasor.resize(n_pb * n_f);
  for (size_t pb = 0; pb < n_pb; ++pb)
    for (int k = 0; k < n_f; ++k) {
      const int n = k / s.n_chan, j = k % s.n_chan;
      double ph = 0.0;
      if (s.cal) {
        const double fj = (j + 0.5) * s.chan_bw_mhz * 1e6;
        ph = kTwoPi * fj * s.cal[(pb * s.n_if + n) * 2 + 0] + s.cal[(pb * s.n_if + n) * 2 + 1];
      }
      h_phasor[pb * n_f + k] = make_double2(std::cos(ph), -std::sin(ph));
    }
  h_blst.clear();
  if (use_autos)
    for (int b = 0; b < s.n_bl; ++b) h_blst.push_back(make_int2(s.bl_st[2 * b], s.bl_st[2 * b + 1]));
  // the calibration table and station pairs are read during the creating call only
  seg.cal = nullptr;
  seg.bl_st = nullptr;
  h_tw_n.resize(n_f);
  for (int i = 0; i < n_f; ++i)
    h_tw_n[i] = make_float2((float)std::cos(kTwoPi * i / n_f), (float)-std::sin(kTwoPi * i / n_f));
  h_tw_m.resize(M);
  for (int i = 0; i < M; ++i)
    h_tw_m[i] = make_float2((float)std::cos(kTwoPi * i / M), (float)-std::sin(kTwoPi * i / M));
  cap = (unsigned)std::max<long long>(4096, std::min<long long>(1LL << 24, (long long)s.n_bl * p.n_dm * 64));
  return 0;
}

size_t SegJob::input_bytes() const {
  size_t b = (size_t)n_pol * seg.n_bl * seg.n_ap * n_f * sizeof(float2);
  if (use_autos) b += (size_t)n_pol * seg.n_st * seg.n_ap * n_f * sizeof(float);
  return b;
}

size_t SegJob::device_bytes() const {
  const size_t vis_n = (size_t)seg.n_bl * seg.n_ap * n_f;
  return vis_n * 8 + (size_t)n_rows * n_tchunk * n_f * 8 + (size_t)n_pol * seg.n_bl * n_f * 24 +
         (size_t)seg.n_bl * 8 +
         (size_t)prm.n_dm * (n_f + 1) * 4 + (size_t)(n_f + M) * 8 + keys_bytes_per_dm() * dm_chunk +
         (size_t)seg.n_bl * prm.n_dm * prm.n_win * 16 + (size_t)seg.n_bl * dm_chunk * word_per_bd * 4 +
         (size_t)cap * sizeof(DevCand) + 4;
}

int SegJob::alloc(cudaStream_t s, bool ordered) {
  stream_ordered = ordered;
  cudaError_t e;
#define VK_A(ptr, n, what)                                 \
  if ((e = dalloc(&ptr, (n), s, ordered)) != cudaSuccess) \
    return cuda_fail(e, what);
  VK_A(d_cand, cap, "alloc candidates");
  VK_A(d_count, 1, "alloc count");
  if (empty) return 0;
  const size_t vis_n = (size_t)seg.n_bl * seg.n_ap * n_f;
  VK_A(d_xn, vis_n, "alloc normalised copy");
  VK_A(d_part, (size_t)n_rows * n_tchunk * n_f, "alloc partial sums");
  VK_A(d_phasor, (size_t)n_pol * seg.n_bl * n_f, "alloc phasor");
  VK_A(d_gain, (size_t)n_pol * seg.n_bl * n_f, "alloc gains");
  if (use_autos) VK_A(d_blst, (size_t)seg.n_bl, "alloc station pairs");
  VK_A(d_shifts, (size_t)prm.n_dm * n_f, "alloc shifts");
  VK_A(d_nvalid, (size_t)prm.n_dm, "alloc nvalid");
  VK_A(d_tw_n, (size_t)n_f, "alloc twiddles");
  VK_A(d_tw_m, (size_t)M, "alloc twiddles");
  VK_A(d_keys, (size_t)seg.n_bl * dm_chunk * seg_per_bd, "alloc peaks");
  VK_A(d_stats, (size_t)seg.n_bl * prm.n_dm * prm.n_win * 2, "alloc stats");
  VK_A(d_bits, (size_t)seg.n_bl * dm_chunk * word_per_bd, "alloc bitmaps");
#undef VK_A
  return 0;
}

bool is_device_pointer(const void* p) {
  cudaPointerAttributes attr{};
  if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

// Device pointer of a borrowed input: itself, or a stream-ordered copy of
// host memory into *copy.
static int stage_one(const void* src, size_t bytes, cudaStream_t s, bool ordered, void** copy, const void** dev,
                     const char* what) {
  if (is_device_pointer(src)) {
    *dev = src;
    return 0;
  }
  cudaError_t e = ordered ? cudaMallocAsync(copy, bytes, s) : cudaMalloc(copy, bytes);
  if (e != cudaSuccess) return cuda_fail(e, what);
  e = cudaMemcpyAsync(*copy, src, bytes, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_fail(e, what);
  *dev = *copy;
  return 0;
}

int SegJob::stage_input(cudaStream_t s) {
  if (empty) return 0;
  const void* dv = nullptr;
  int rc = stage_one(seg.vis, (size_t)n_pol * seg.n_bl * seg.n_ap * n_f * sizeof(float2), s, stream_ordered,
                     &d_vis_copy, &dv, "copy vis to device");
  if (rc) return rc;
  d_vis = static_cast<const float2*>(dv);
  if (use_autos) {
    const void* da = nullptr;
    rc = stage_one(seg.autos, (size_t)n_pol * seg.n_st * seg.n_ap * n_f * sizeof(float), s, stream_ordered,
                   &d_autos_copy, &da, "copy auto spectra to device");
    if (rc) return rc;
    d_autos = static_cast<const float*>(da);
  }
  return 0;
}

int SegJob::upload(cudaStream_t s) {
  if (empty) return 0;
  cudaError_t e;
#define VK_C(dst, src, what)                                                                  \
  if ((e = cudaMemcpyAsync(dst, (src).data(), (src).size() * sizeof((src)[0]),                \
                           cudaMemcpyHostToDevice, s)) != cudaSuccess)                        \
    return cuda_fail(e, what);
  VK_C(d_phasor, h_phasor, "copy phasor");
  if (use_autos) VK_C(d_blst, h_blst, "copy station pairs");
  VK_C(d_shifts, shifts, "copy shifts");
  VK_C(d_nvalid, nvalid, "copy nvalid");
  VK_C(d_tw_n, h_tw_n, "copy twiddles");
  VK_C(d_tw_m, h_tw_m, "copy twiddles");
#undef VK_C
  return 0;
}

void SegJob::release(cudaStream_t s) {
  void* ptrs[] = {d_vis_copy, d_autos_copy, d_blst, d_xn,    d_part,  d_phasor, d_gain, d_shifts,
                  d_nvalid,   d_tw_n,       d_tw_m, d_keys,  d_stats, d_bits,   d_cand, d_count};
  for (void* p : ptrs)
    if (p) {
      if (stream_ordered) cudaFreeAsync(p, s);
      else cudaFree(p);
    }
  d_vis_copy = nullptr;
  d_autos_copy = nullptr;
  d_blst = nullptr;
  d_xn = nullptr;
  d_part = nullptr;
  d_phasor = nullptr;
  d_gain = nullptr;
  d_shifts = nullptr;
  d_nvalid = nullptr;
  d_tw_n = d_tw_m = nullptr;
  d_keys = nullptr;
  d_stats = nullptr;
  d_bits = nullptr;
  d_cand = nullptr;
  d_count = nullptr;
}

SegDesc SegJob::desc(int c) const {
  SegDesc d;
  std::memset(&d, 0, sizeof d);
  const int d0 = c * dm_chunk;
  d.xn = d_xn;
  d.shifts = d_shifts + (size_t)d0 * n_f;
  d.nvalid = d_nvalid + d0;
  d.tw_n = d_tw_n;
  d.tw_m = d_tw_m;
  d.keys = d_keys;
  d.stats = d_stats;
  d.bits = d_bits;
  d.cand = d_cand;
  d.count = d_count;
  d.cap = cap;
  d.seg_id = seg_id;
  d.seg_per_bd = seg_per_bd;
  d.word_per_bd = word_per_bd;
  d.n_bl = seg.n_bl;
  d.n_ap = seg.n_ap;
  d.n_f = n_f;
  d.n_dm = std::min(dm_chunk, prm.n_dm - d0);
  d.n_dm_total = prm.n_dm;
  d.d0 = d0;
  d.pad_delay = prm.pad_delay;
  d.M = M;
  d.n_tiles = n_tiles;
  d.n_win = prm.n_win;
  d.n_eff = n_eff;
  d.min_windows = prm.min_windows;
  d.win_mask = win_mask | (slide ? kSlideBit | (prm.win[prm.n_win - 1] << 8) : 0);
  for (int i = 0; i <= kMaxWinLog; ++i) {
    d.win_log[i] = win_log[i];
    d.win_off[i] = win_off[i];
    d.word_off[i] = word_off[i];
    d.win_off_l[i] = win_off_l[i];
  }
  d.thresh = prm.thresh;
  return d;
}

cudaError_t SegJob::enqueue_prep(cudaStream_t s, int* n_launch) const {
  PrepArgs pa{};
  pa.vis = d_vis;
  pa.autos = use_autos ? d_autos : nullptr;
  pa.bl_st = d_blst;
  pa.n_pol = n_pol;
  pa.n_st = seg.n_st;
  pa.xn = d_xn;
  pa.part = d_part;
  pa.phasor = d_phasor;
  pa.gain = d_gain;
  pa.n_bl = seg.n_bl;
  pa.n_ap = seg.n_ap;
  pa.n_f = n_f;
  pa.n_chan = seg.n_chan;
  pa.n_tchunk = n_tchunk;
  pa.tchunk = tchunk;
  pa.normalize = prm.normalize_chan;
  pa.skip_first_chan = prm.skip_first_chan;
  return launch_prep(pa, s, n_launch);
}

}  // namespace vk

// ============================================================ results ====
namespace {

using vk::cuda_fail;
using vk::fail;

void release(volks_result* r) {
  if (!r || r->borrowed) return;
  if (r->own_job) {
    r->own_job->release(r->stream);
    // the job's host vectors may still feed in-flight copies
    if (!r->synced) cudaStreamSynchronize(r->stream);
    delete r->own_job;
  }
  if (r->counter) cudaFreeAsync(r->counter, r->stream);
  for (auto& e : r->ev)
    if (e) cudaEventDestroy(e);
  delete r;
}

int sync_result(volks_result* r) {
  if (r->synced) return 0;
  cudaError_t e = cudaStreamSynchronize(r->stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  if (r->d_err) {
    unsigned int flag = 0;
    e = cudaMemcpy(&flag, r->d_err, sizeof flag, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "read error flag");
    if (flag) return fail(VOLKS_ETIMEOUT, "the tensor-core search gave up waiting for its MMAs");
  }
  r->synced = true;
  return 0;
}

#define VK_TRY(expr, what)           \
  do {                               \
    cudaError_t e_ = (expr);         \
    if (e_ != cudaSuccess) {         \
      int rc_ = cuda_fail(e_, what); \
      release(r);                    \
      return rc_;                    \
    }                                \
  } while (0)

}  // namespace

int vk_sync_result(volks_result* r) { return sync_result(r); }

int vk_rerun_match(volks_result* r) {
  vk::SegJob* j = r->job;
  cudaError_t e = cudaMemsetAsync(j->d_count, 0, sizeof(unsigned int), r->stream);
  if (e != cudaSuccess) return cuda_fail(e, "memset count");
  vk::Batch b;
  std::memset(&b, 0, sizeof b);
  b.d[0] = j->desc(0);
  b.n_desc = 1;
  b.total = (long long)j->seg.n_bl * b.d[0].n_dm;
  int n = 0;
  e = vk::launch_match_batch(b, r->stream, &n);
  if (e != cudaSuccess) return cuda_fail(e, "match kernel");
  r->synced = false;
  return 0;
}

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
  p->stride = 0;
}

int volks_search_segment(const volks_segment* seg, const volks_params* prm, void* cuda_stream,
                         volks_result** out) {
  if (!out) return fail(VOLKS_EINVAL, "out is NULL");
  *out = nullptr;
  int rc = vk::validate(seg, prm);
  if (rc) return rc;
  volks_result* r = new (std::nothrow) volks_result();
  if (!r) return fail(VOLKS_ENOMEM, "host allocation");
  r->own_job = new (std::nothrow) vk::SegJob();
  if (!r->own_job) {
    delete r;
    return fail(VOLKS_ENOMEM, "host allocation");
  }
  r->job = r->own_job;
  r->stream = static_cast<cudaStream_t>(cuda_stream);
  vk::SegJob& j = *r->job;
  rc = j.init(*seg, *prm, 0);
  if (rc) {
    release(r);
    return rc;
  }
  for (auto& e : r->ev) VK_TRY(cudaEventCreate(&e), "cudaEventCreate");
  cudaStream_t st = r->stream;
  VK_TRY(cudaEventRecord(r->ev[0], st), "event");
  rc = j.alloc(st, true);
  if (!rc) rc = j.stage_input(st);
  if (rc) {
    release(r);
    return rc;
  }
  VK_TRY(cudaMemsetAsync(j.d_count, 0, sizeof(unsigned int), st), "memset count");
  if (j.empty) {
    for (int i = 1; i < 6; ++i) VK_TRY(cudaEventRecord(r->ev[i], st), "event");
    *out = r;
    return 0;
  }
  VK_TRY(cudaEventRecord(r->ev[1], st), "event");
  rc = j.upload(st);
  if (rc) {
    release(r);
    return rc;
  }
  VK_TRY(j.enqueue_prep(st, &r->n_launch), "prep kernels");
  VK_TRY(cudaEventRecord(r->ev[2], st), "event");

  // a4-a7: persistent CTAs over the segment's (baseline, DM, tile) units; every
  // valid segment's key is stored once, so the key buffer needs no clearing
  int fold = 0;
  if (const char* f = std::getenv("VOLKS_SEARCH_FOLD")) fold = std::atoi(f);
  const vk::SearchVariant v = vk::default_variant(j.n_f, j.prec, fold);
  vk::Batch b;
  std::memset(&b, 0, sizeof b);
  b.d[0] = j.desc(0);
  b.n_desc = 1;
  b.total = vk::search_units(b.d[0], v);
  const char* pe = std::getenv("VOLKS_SEARCH_PERSISTENT");
  // the tensor-core kernel is always persistent
  const bool persistent = !(pe && pe[0] == '0') || j.prec != VOLKS_FP32;
  int grid = 0;
  if (persistent) {
    // [0] work counter, [1] error flag of the bounded waits
    VK_TRY(cudaMallocAsync(reinterpret_cast<void**>(&r->counter), 2 * sizeof(unsigned long long), st),
           "alloc work counter");
    VK_TRY(cudaMemsetAsync(r->counter, 0, 2 * sizeof(unsigned long long), st), "memset counter");
    b.counter = r->counter;
    b.err = reinterpret_cast<unsigned int*>(r->counter + 1);
    if (j.prec != VOLKS_FP32) r->d_err = b.err;
    grid = std::max(1, vk::search_occupancy(v, prm->pad_rate, j.prec)) * vk::sm_count();
  }
  const int before = r->n_launch;
  VK_TRY(vk::launch_search_batch(b, v, prm->pad_rate, j.prec, grid, st, &r->n_launch), "search kernel");
  r->n_search_launch = r->n_launch - before;
  VK_TRY(cudaEventRecord(r->ev[3], st), "event");

  // a8
  b.counter = nullptr;
  b.total = (long long)seg->n_bl * prm->n_dm * prm->n_win;
  VK_TRY(vk::launch_select_batch(b, st, &r->n_launch), "select kernel");
  VK_TRY(cudaEventRecord(r->ev[4], st), "event");
  // a9
  b.total = (long long)seg->n_bl * prm->n_dm;
  VK_TRY(vk::launch_match_batch(b, st, &r->n_launch), "match kernel");
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
    vk::SegJob& j = *r->job;
    unsigned int count = 0;
    cudaError_t e = cudaMemcpy(&count, j.d_count, sizeof count, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "read candidate count");
    if (count > j.cap) {  // grow and re-run the window match only
      if (j.n_chunks() > 1)
        return fail(VOLKS_ENOMEM,
                    "segment %d: %u window-matched groups exceed the buffer of %u and its earlier DM "
                    "chunks are gone; search it again with a larger peak budget",
                    j.seg_id, count, j.cap);
      if (j.stream_ordered) cudaFreeAsync(j.d_cand, r->stream);
      else cudaFree(j.d_cand);
      j.cap = count;
      e = j.stream_ordered
              ? cudaMallocAsync(reinterpret_cast<void**>(&j.d_cand), j.cap * sizeof(vk::DevCand), r->stream)
              : cudaMalloc(reinterpret_cast<void**>(&j.d_cand), j.cap * sizeof(vk::DevCand));
      if (e != cudaSuccess) return cuda_fail(e, "grow candidates");
      rc = vk_rerun_match(r);
      if (!rc) rc = sync_result(r);
      if (rc) return rc;
      e = cudaMemcpy(&count, j.d_count, sizeof count, cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) return cuda_fail(e, "read candidate count");
    }
    std::vector<vk::DevCand> dc(count);
    if (count) {
      e = cudaMemcpy(dc.data(), j.d_cand, count * sizeof(vk::DevCand), cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) return cuda_fail(e, "read candidates");
    }
    const volks_segment& s = j.seg;
    const volks_params& p = j.prm;
    std::vector<volks_candidate> all(count);
    for (unsigned i = 0; i < count; ++i) {
      const vk::DevCand& c = dc[i];
      volks_candidate& o = all[i];
      std::memset(&o, 0, sizeof o);
      const int W = 1 << c.win_log;
      const int R = (W == 1 || p.pad_rate == 0) ? 1 : p.pad_rate * W;
      const int q = (int)(c.lin / (uint32_t)j.M), m = (int)(c.lin % (uint32_t)j.M);
      o.bl = c.bl;
      o.dm_idx = c.dm_idx;
      o.win = W;
      o.seg = c.seg;
      o.t0_ap = vk::seg_start(c.seg, c.win_log, j.slide ? 1 : 0);
      o.t1_ap = o.t0_ap + W;
      o.g0_ap = c.g0;
      o.g1_ap = c.g1;
      o.delay_idx = m >= j.M / 2 ? m - j.M : m;
      o.rate_idx = (R > 1 && q >= R / 2) ? q - R : q;
      o.n_windows = c.n_windows;
      o.peak_power = c.P;
      o.rho = c.rho;
      o.z = c.z;
      o.dm = p.dm_lo + p.dm_step * c.dm_idx;
      o.delay_s = o.delay_idx / (j.M * s.chan_bw_mhz * 1e6);
      o.rate_hz = o.rate_idx / (R * s.t_ap_s);
    }
    // a10: cross-baseline match per DM over representative intervals
    r->cands = vk::cross_match(std::move(all), p.min_baselines);
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
  v = vk::cross_match(std::move(v), min_baselines);
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
  int rc = vk::validate(&s, &p);
  if (rc) return rc;
  return vk::shift_table(f_lo_mhz, chan_bw_mhz, n_f, t_ap_s, n_ap, dm_lo, dm_step, n_dm, shifts, nvalid);
}

int volks_result_timing(volks_result* r, volks_timing* t) {
  if (!r || !t) return fail(VOLKS_EINVAL, "NULL argument");
  int rc = sync_result(r);
  if (rc) return rc;
  std::memset(t, 0, sizeof *t);
  if (r->plan) return vk_plan_timing(r->plan, t);
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
  const vk::SegJob& j = *r->job;
  if (shifts && !j.shifts.empty()) std::memcpy(shifts, j.shifts.data(), j.shifts.size() * sizeof(int32_t));
  if (nvalid && !j.nvalid.empty()) std::memcpy(nvalid, j.nvalid.data(), j.nvalid.size() * sizeof(int32_t));
  return 0;
}

int volks_result_peaks(volks_result* r, int32_t bl, int32_t dm_idx, int32_t win_idx, float* P, int32_t* q,
                       int32_t* m, size_t cap, size_t* n_seg) {
  if (!r || !n_seg) return fail(VOLKS_EINVAL, "NULL argument");
  const vk::SegJob& j = *r->job;
  if (bl < 0 || bl >= j.seg.n_bl || dm_idx < 0 || dm_idx >= j.prm.n_dm || win_idx < 0 || win_idx >= j.prm.n_win)
    return fail(VOLKS_EINVAL, "series index out of range");
  const int last = j.n_chunks() - 1;
  const int d0 = last > 0 ? last * j.dm_chunk : 0;
  if (dm_idx < d0) return fail(VOLKS_EINVAL, "peaks of DM %d were overwritten by a later DM chunk", dm_idx);
  int rc = sync_result(r);
  if (rc) return rc;
  const int W = 1 << j.win_log[win_idx];
  const size_t ns = (size_t)vk::seg_count(j.nvalid[dm_idx], j.win_log[win_idx], j.slide ? 1 : 0);
  *n_seg = ns;
  const size_t n = std::min(ns, cap);
  if (n == 0 || j.empty) return 0;
  std::vector<unsigned long long> k(n);
  const int n_dm_c = std::min(j.dm_chunk, j.prm.n_dm - d0);
  const size_t off = ((size_t)bl * n_dm_c + (dm_idx - d0)) * j.seg_per_bd + j.win_off[win_idx];
  cudaError_t e = cudaMemcpy(k.data(), j.d_keys + off, n * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "read peaks");
  for (size_t i = 0; i < n; ++i) {
    const uint32_t hi = (uint32_t)(k[i] >> 32), lin = 0xffffffffu - (uint32_t)(k[i] & 0xffffffffu);
    float f;
    std::memcpy(&f, &hi, 4);
    if (P) P[i] = f;
    if (q) q[i] = (int32_t)(lin / (uint32_t)j.M);
    if (m) m[i] = (int32_t)(lin % (uint32_t)j.M);
  }
  return 0;
}

int volks_result_stats(volks_result* r, int32_t bl, int32_t dm_idx, int32_t win_idx, double* mean, double* sd) {
  if (!r || !mean || !sd) return fail(VOLKS_EINVAL, "NULL argument");
  const vk::SegJob& j = *r->job;
  if (bl < 0 || bl >= j.seg.n_bl || dm_idx < 0 || dm_idx >= j.prm.n_dm || win_idx < 0 || win_idx >= j.prm.n_win)
    return fail(VOLKS_EINVAL, "series index out of range");
  int rc = sync_result(r);
  if (rc) return rc;
  if (j.empty) {
    *mean = *sd = 0.0;
    return 0;
  }
  double v[2];
  const size_t off = (((size_t)bl * j.prm.n_dm + dm_idx) * j.prm.n_win + win_idx) * 2;
  cudaError_t e = cudaMemcpy(v, j.d_stats + off, sizeof v, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "read stats");
  *mean = v[0];
  *sd = v[1];
  return 0;
}

int volks_result_gains(volks_result* r, float* gains, size_t cap_floats) {
  if (!r || !gains) return fail(VOLKS_EINVAL, "NULL argument");
  const vk::SegJob& j = *r->job;
  const size_t n = (size_t)j.n_pol * j.seg.n_bl * j.n_f * 2;
  if (cap_floats < n) return fail(VOLKS_EINVAL, "gains buffer holds %zu floats, need %zu", cap_floats, n);
  int rc = sync_result(r);
  if (rc) return rc;
  if (j.empty || !j.d_gain) {
    std::memset(gains, 0, n * sizeof(float));
    return 0;
  }
  cudaError_t e = cudaMemcpy(gains, j.d_gain, n * sizeof(float), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "read gains");
  return 0;
}

int volks_check_rate_gemm(const void* y, int32_t win, int32_t precision, int32_t flags, float* out) {
  if (!y || !out) return fail(VOLKS_EINVAL, "NULL argument");
  if (flags & ~VOLKS_CHECK_SKIP_MMA) return fail(VOLKS_EINVAL, "unknown flags");
  int l = -1;
  for (int i = 1; i <= 5; ++i)
    if (win == (1 << i)) l = i;
  if (l < 0) return fail(VOLKS_EINVAL, "win = %d: 2, 4, 8, 16 or 32 only", win);
  if (!(precision == VOLKS_BF16 || precision == VOLKS_FP16 || precision == VOLKS_FP8))
    return fail(VOLKS_EINVAL, "precision %d has no tensor-core form", precision);
  const int M = 128;  // W_R^x = W_128^{x 128 / R} for every R = 4 win <= 128
  std::vector<float2> tw(M);
  for (int i = 0; i < M; ++i) tw[i] = make_float2((float)std::cos(kTwoPi * i / M), (float)-std::sin(kTwoPi * i / M));
  float2* d_tw = nullptr;
  unsigned int* d_err = nullptr;
  cudaError_t e = cudaMalloc(&d_tw, M * sizeof(float2));
  if (e == cudaSuccess) e = cudaMalloc(&d_err, sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMemcpy(d_tw, tw.data(), M * sizeof(float2), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(d_err, 0, sizeof(unsigned int));
  if (e == cudaSuccess)
    e = vk::launch_rate_gemm_probe(static_cast<const float2*>(y), d_tw, M, l, precision,
                                   (flags & VOLKS_CHECK_SKIP_MMA) ? 1 : 0, out, d_err, nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  unsigned int flag = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&flag, d_err, sizeof flag, cudaMemcpyDeviceToHost);
  if (d_tw) cudaFree(d_tw);
  if (d_err) cudaFree(d_err);
  if (e != cudaSuccess) return cuda_fail(e, "rate GEMM check");
  if (flag) return fail(VOLKS_ETIMEOUT, "the tensor cores did not complete the MMAs");
  return 0;
}

}  // extern "C"
