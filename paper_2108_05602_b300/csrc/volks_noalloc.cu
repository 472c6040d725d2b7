// volks_search_peaks_noalloc: the per-segment peak search (steps a1-a7)
// with every piece of device scratch taken from one file-scope static
// device array instead of cudaMalloc.
//
// Who needs this: callers that must not allocate device memory while they
// run, e.g. a real-time correlator or streaming service that reserves the
// whole GPU at start-up and cannot afford allocator latency or an
// out-of-memory failure in the middle of an observation, or a host
// framework whose own allocator owns the device-memory budget.  Such a
// caller passes device buffers for the input and the outputs; everything
// else lives in g_noalloc_scratch below.
//
// Rules of use (also in include/volks.h):
//  * scratch is VOLKS_NOALLOC_SCRATCH_BYTES per device, held by every
//    device that loads this library until the process exits;
//  * larger problems are rejected with VOLKS_EINVAL (nothing is launched);
//  * all calls on a device share the array and it keeps the previous
//    call's contents; every part a call reads is first written by that
//    call on its stream, so nothing needs clearing.  Calls that overlap on
//    the GPU (other streams, other host threads) race on the array:
//    serialise them;
//  * the first call on each device looks up the array's device address
//    with cudaGetSymbolAddress (with that device current); make that first
//    call before any stream capture.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/volks.h"
#include "../../include/volks_check.h"
#include "volks_internal.h"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[VOLKS_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
constexpr int kMaxCal = 256;             // n_bl * n_if calibration entries
constexpr double kDispersionNA = 4.148808e3;  // s MHz^2 pc^-1 cm^3
constexpr double kTwoPiNA = 6.283185307179586476925286766559;

std::mutex g_mu;
void* g_dev_ptr[kMaxDevices] = {};

// Where the last call on each device left its shift table in the scratch
// (read back by volks_noalloc_tables).
struct LastTables {
  size_t o_shifts, o_nvalid;
  int n_dm, n_f;
  bool set;
};
LastTables g_last[kMaxDevices] = {};

// Errors go to the library's thread-local message (volks_last_error()).
int na_fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  vk::set_last_error(buf);
  return code;
}

// Device address of the static scratch on the current device (looked up
// once per device; cudaGetSymbolAddress needs that device current).
int scratch_ptr(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return na_fail(VOLKS_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return na_fail(VOLKS_EINVAL, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_dev_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return na_fail(VOLKS_ECUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
    g_dev_ptr[dev] = p;
  }
  *out = g_dev_ptr[dev];
  return 0;
}

bool pow2(long long x) { return x > 0 && (x & (x - 1)) == 0; }

// A caller buffer must be device (or managed) memory of the current device:
// a host pointer would fault in the kernels that write it, and another
// device's memory would be reached through peer access that may not be on.
int device_buffer(const void* p, int dev, const char* name) {
  cudaPointerAttributes attr{};
  if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
    cudaGetLastError();
    return na_fail(VOLKS_EINVAL, "%s: not a CUDA allocation", name);
  }
  if (!(attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged))
    return na_fail(VOLKS_EINVAL, "%s must be device memory for the no-allocation entry point", name);
  if (attr.device != dev)
    return na_fail(VOLKS_EINVAL, "%s is on device %d; the current device is %d", name, attr.device, dev);
  return 0;
}

struct TableArgs {
  double f_lo_mhz, chan_bw_mhz, t_ap_s, dm_lo, dm_step;
  int n_bl, n_if, n_chan, n_f, n_dm, n_ap, M, has_cal;
  int32_t* shifts;
  int32_t* nvalid;
  double2* phasor;
  float2* tw_n;
  float2* tw_m;
  double cal[kMaxCal][2];
};
// TableArgs is passed by value as a kernel parameter (about 4.2 KB): above
// the classic 4 KB limit, within the 32,764-byte limit that CUDA 12.1+
// toolkits allow on Volta and later GPUs.
static_assert(sizeof(TableArgs) <= 32764, "kernel parameter block too large");

// Shift table with the same FP64 operation order as the host's table
// (round-to-nearest intrinsics, no contraction), one block per DM trial.
__global__ void na_shift_kernel(const TableArgs a) {
  __shared__ int red[256];
  const int d = blockIdx.x;
  const double dm = __dadd_rn(a.dm_lo, __dmul_rn(a.dm_step, (double)d));
  const double ftop = __dadd_rn(a.f_lo_mhz, __dmul_rn((double)(a.n_f - 1) + 0.5, a.chan_bw_mhz));
  const double c = __ddiv_rn(__dmul_rn(kDispersionNA, dm), a.t_ap_s);
  const double itop = __ddiv_rn(1.0, __dmul_rn(ftop, ftop));
  int mx = 0;
  for (int k = threadIdx.x; k < a.n_f; k += blockDim.x) {
    const double f = __dadd_rn(a.f_lo_mhz, __dmul_rn((double)k + 0.5, a.chan_bw_mhz));
    const double x = __dmul_rn(c, __dsub_rn(__ddiv_rn(1.0, __dmul_rn(f, f)), itop));
    const int sh = (int)floor(__dadd_rn(x, 0.5));
    a.shifts[(size_t)d * a.n_f + k] = sh;
    mx = max(mx, sh);
  }
  red[threadIdx.x] = mx;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) red[threadIdx.x] = max(red[threadIdx.x], red[threadIdx.x + h]);
    __syncthreads();
  }
  if (threadIdx.x == 0) a.nvalid[d] = a.n_ap - red[0];
}

// Calibration phasor (FP64) and FFT twiddle tables.
__global__ void na_tables_kernel(const TableArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < a.n_bl * a.n_f) {
    const int b = i / a.n_f, k = i % a.n_f;
    const int n = k / a.n_chan, j = k % a.n_chan;
    double ph = 0.0;
    if (a.has_cal) {
      const double fj = ((double)j + 0.5) * a.chan_bw_mhz * 1e6;
      ph = kTwoPiNA * fj * a.cal[b * a.n_if + n][0] + a.cal[b * a.n_if + n][1];
    }
    a.phasor[i] = make_double2(cos(ph), -sin(ph));
  }
  if (i < a.n_f)
    a.tw_n[i] = make_float2((float)cos(kTwoPiNA * i / a.n_f), (float)-sin(kTwoPiNA * i / a.n_f));
  if (i < a.M)
    a.tw_m[i] = make_float2((float)cos(kTwoPiNA * i / a.M), (float)-sin(kTwoPiNA * i / a.M));
}

struct UnpackArgs {
  const unsigned long long* keys;
  const int32_t* nvalid;
  float* peak_power;
  int32_t* peak_cell;
  int n_dm, n_win;
  long long seg_per_bd, total;
  int win[VOLKS_MAX_WIN];
  int win_off[VOLKS_MAX_WIN];
};

// keys -> caller's (power, cell); segments past n_valid get (0, -1).
__global__ void na_unpack_kernel(const UnpackArgs a) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.total) return;
  const long long bd = i / a.seg_per_bd;
  const int o = (int)(i % a.seg_per_bd);
  const int d = (int)(bd % a.n_dm);
  int wi = 0;
  for (int w = 1; w < a.n_win; ++w)
    if (o >= a.win_off[w]) wi = w;
  const int s = o - a.win_off[wi];
  const int nseg = max(a.nvalid[d], 0) / a.win[wi];
  if (s < nseg) {
    const unsigned long long k = a.keys[i];
    a.peak_power[i] = __uint_as_float((uint32_t)(k >> 32));
    a.peak_cell[i] = (int32_t)(0xffffffffu - (uint32_t)(k & 0xffffffffu));
  } else {
    a.peak_power[i] = 0.f;
    a.peak_cell[i] = -1;
  }
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

extern "C" int volks_search_peaks_noalloc(const volks_segment* seg, const volks_params* prm,
                                          void* cuda_stream, float* peak_power,
                                          int32_t* peak_cell) {
  if (!seg || !prm) return na_fail(VOLKS_EINVAL, "NULL segment or params");
  const int n_bl = seg->n_bl, n_ap = seg->n_ap, n_if = seg->n_if, n_chan = seg->n_chan;
  if (n_bl < 0 || n_ap < 0 || n_if < 1 || n_chan < 1) return na_fail(VOLKS_EINVAL, "bad segment sizes");
  const long long n_f = (long long)n_if * n_chan;
  if (!pow2(n_f) || n_f < 64 || n_f > 512)
    return na_fail(VOLKS_EINVAL, "n_if*n_chan = %lld: powers of two 64..512 only", n_f);
  if (!(seg->t_ap_s > 0 && std::isfinite(seg->t_ap_s)) || !(seg->chan_bw_mhz > 0 && std::isfinite(seg->chan_bw_mhz)) ||
      !(seg->f_lo_mhz > 0 && std::isfinite(seg->f_lo_mhz)))
    return na_fail(VOLKS_EINVAL, "t_ap_s, chan_bw_mhz and f_lo_mhz must be finite and > 0");
  if (prm->n_dm < 0 || !std::isfinite(prm->dm_lo) || !std::isfinite(prm->dm_step))
    return na_fail(VOLKS_EINVAL, "bad DM grid");
  if (prm->n_dm > 0 && (prm->dm_lo < 0 || prm->dm_lo + prm->dm_step * (prm->n_dm - 1) < 0))
    return na_fail(VOLKS_EINVAL, "negative DM trial");
  if (prm->n_win < 1 || prm->n_win > VOLKS_MAX_WIN) return na_fail(VOLKS_EINVAL, "n_win must be 1..%d", VOLKS_MAX_WIN);
  int win_mask = 0;
  for (int i = 0; i < prm->n_win; ++i) {
    if (!pow2(prm->win[i]) || prm->win[i] > 32 || (i > 0 && prm->win[i] <= prm->win[i - 1]))
      return na_fail(VOLKS_EINVAL, "windows must be ascending powers of two 1..32");
    int l = 0;
    while ((1 << l) < prm->win[i]) ++l;
    win_mask |= 1 << l;
  }
  if (!(prm->pad_delay == 1 || prm->pad_delay == 2 || prm->pad_delay == 4 || prm->pad_delay == 8))
    return na_fail(VOLKS_EINVAL, "pad_delay must be 1, 2, 4 or 8");
  if (!(prm->pad_rate == 0 || prm->pad_rate == 4)) return na_fail(VOLKS_EINVAL, "pad_rate must be 0 or 4");
  if (prm->precision != VOLKS_FP32) return na_fail(VOLKS_EINVAL, "precision %d not available", prm->precision);
  if ((prm->normalize_chan & ~1) || (prm->skip_first_chan & ~1)) return na_fail(VOLKS_EINVAL, "flags must be 0 or 1");
  if (prm->stride != 0) return na_fail(VOLKS_EINVAL, "this entry point searches back-to-back segments only");
  if (seg->n_pol > 1 || seg->n_pol < 0 || seg->autos)
    return na_fail(VOLKS_EINVAL, "this entry point takes one polarisation product and no auto spectra");
  if (seg->cal && (long long)n_bl * n_if > kMaxCal)
    return na_fail(VOLKS_EINVAL, "n_bl*n_if = %lld calibration entries; this entry point takes at most %d",
                   (long long)n_bl * n_if, kMaxCal);
  // largest shift (lowest channel, largest DM) must fit an int
  if (prm->n_dm > 0) {
    const double f0 = seg->f_lo_mhz + 0.5 * seg->chan_bw_mhz, f1 = seg->f_lo_mhz + (n_f - 0.5) * seg->chan_bw_mhz;
    const double dmax = std::max(prm->dm_lo, prm->dm_lo + prm->dm_step * (prm->n_dm - 1));
    const double x = kDispersionNA * dmax / seg->t_ap_s * (1.0 / (f0 * f0) - 1.0 / (f1 * f1));
    if (!(x < 2.0e9)) return na_fail(VOLKS_EINVAL, "dispersion shift overflows");
  }

  const int n_dm = prm->n_dm, n_win = prm->n_win, M = prm->pad_delay * (int)n_f;
  long long seg_per_bd = 0;
  int win_off_i[VOLKS_MAX_WIN] = {};
  int win_off_l[vk::kMaxWinLog + 1] = {};
  for (int i = 0; i < n_win; ++i) {
    int l = 0;
    while ((1 << l) < prm->win[i]) ++l;
    win_off_i[i] = (int)seg_per_bd;
    win_off_l[l] = (int)seg_per_bd;
    seg_per_bd += n_ap / prm->win[i];
  }
  const long long total = (long long)n_bl * n_dm * seg_per_bd;
  if (total > 0 && (!peak_power || !peak_cell)) return na_fail(VOLKS_EINVAL, "NULL output buffer");
  if ((long long)n_bl * n_ap * n_dm == 0) return 0;  // nothing to search, nothing written

  // scratch layout, each piece 256-byte aligned
  const int tchunk = 1024, n_tchunk = (n_ap + tchunk - 1) / tchunk;
  const size_t vis_n = (size_t)n_bl * n_ap * n_f;
  size_t off = 0;
  auto take = [&](size_t bytes) { const size_t o = off; off = align256(off + bytes); return o; };
  const size_t o_xn = take(vis_n * sizeof(float2));
  const size_t o_part = take((size_t)n_bl * n_tchunk * n_f * sizeof(double));
  const size_t o_phasor = take((size_t)n_bl * n_f * sizeof(double2));
  const size_t o_gain = take((size_t)n_bl * n_f * sizeof(float2));
  const size_t o_shifts = take((size_t)n_dm * n_f * sizeof(int32_t));
  const size_t o_nvalid = take((size_t)n_dm * sizeof(int32_t));
  const size_t o_twn = take((size_t)n_f * sizeof(float2));
  const size_t o_twm = take((size_t)M * sizeof(float2));
  const size_t o_keys = take((size_t)total * sizeof(unsigned long long));
  if (off > (size_t)VOLKS_NOALLOC_SCRATCH_BYTES)
    return na_fail(VOLKS_EINVAL,
                   "segment needs %zu bytes of scratch; the no-allocation entry point has %zu "
                   "(use volks_search_segment)", off, (size_t)VOLKS_NOALLOC_SCRATCH_BYTES);
  if (!seg->vis) return na_fail(VOLKS_EINVAL, "vis is NULL");
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return na_fail(VOLKS_EINVAL, "no current CUDA device");
  }
  int rc = device_buffer(seg->vis, dev, "vis");
  if (!rc) rc = device_buffer(peak_power, dev, "peak_power");
  if (!rc) rc = device_buffer(peak_cell, dev, "peak_cell");
  if (rc) return rc;

  void* base = nullptr;
  rc = scratch_ptr(&base);
  if (rc) return rc;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    g_last[dev] = LastTables{o_shifts, o_nvalid, n_dm, (int)n_f, true};
  }
  unsigned char* sp = static_cast<unsigned char*>(base);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  int n_launch = 0;
  auto cu = [&](cudaError_t e, const char* what) {
    return e == cudaSuccess ? 0 : na_fail(VOLKS_ECUDA, "%s: %s", what, cudaGetErrorString(e));
  };

  TableArgs ta;
  std::memset(&ta, 0, sizeof ta);
  ta.f_lo_mhz = seg->f_lo_mhz;
  ta.chan_bw_mhz = seg->chan_bw_mhz;
  ta.t_ap_s = seg->t_ap_s;
  ta.dm_lo = prm->dm_lo;
  ta.dm_step = prm->dm_step;
  ta.n_bl = n_bl;
  ta.n_if = n_if;
  ta.n_chan = n_chan;
  ta.n_f = (int)n_f;
  ta.n_dm = n_dm;
  ta.n_ap = n_ap;
  ta.M = M;
  ta.has_cal = seg->cal != nullptr;
  if (seg->cal)
    for (int i = 0; i < n_bl * n_if; ++i) {
      ta.cal[i][0] = seg->cal[2 * i];
      ta.cal[i][1] = seg->cal[2 * i + 1];
    }
  ta.shifts = reinterpret_cast<int32_t*>(sp + o_shifts);
  ta.nvalid = reinterpret_cast<int32_t*>(sp + o_nvalid);
  ta.phasor = reinterpret_cast<double2*>(sp + o_phasor);
  ta.tw_n = reinterpret_cast<float2*>(sp + o_twn);
  ta.tw_m = reinterpret_cast<float2*>(sp + o_twm);
  na_shift_kernel<<<n_dm, 256, 0, st>>>(ta);
  if ((rc = cu(cudaGetLastError(), "shift table kernel"))) return rc;
  const int nt = std::max<int>(n_bl * (int)n_f, M);
  na_tables_kernel<<<(nt + 255) / 256, 256, 0, st>>>(ta);
  if ((rc = cu(cudaGetLastError(), "table kernel"))) return rc;

  vk::PrepArgs pa{};
  pa.vis = static_cast<const float2*>(seg->vis);
  pa.xn = reinterpret_cast<float2*>(sp + o_xn);
  pa.part = reinterpret_cast<double*>(sp + o_part);
  pa.phasor = ta.phasor;
  pa.gain = reinterpret_cast<float2*>(sp + o_gain);
  pa.n_bl = n_bl;
  pa.n_ap = n_ap;
  pa.n_f = (int)n_f;
  pa.n_chan = n_chan;
  pa.n_tchunk = n_tchunk;
  pa.tchunk = tchunk;
  pa.n_pol = 1;
  pa.normalize = prm->normalize_chan;
  pa.skip_first_chan = prm->skip_first_chan;
  if ((rc = cu(vk::launch_prep(pa, st, &n_launch), "prep kernels"))) return rc;

  // every valid segment's key is stored once by the search (the unpack
  // kernel reads only those), so the keys need no clearing
  unsigned long long* keys = reinterpret_cast<unsigned long long*>(sp + o_keys);
  vk::SearchArgs sa{};
  sa.xn = pa.xn;
  sa.shifts = ta.shifts;
  sa.nvalid = ta.nvalid;
  sa.tw_n = ta.tw_n;
  sa.tw_m = ta.tw_m;
  sa.keys = keys;
  sa.n_bl = n_bl;
  sa.n_ap = n_ap;
  sa.n_f = (int)n_f;
  sa.n_dm = n_dm;
  sa.pad_delay = prm->pad_delay;
  sa.M = M;
  sa.win_mask = win_mask;
  for (int l = 0; l <= vk::kMaxWinLog; ++l) sa.win_off[l] = win_off_l[l];
  sa.seg_per_bd = seg_per_bd;
  sa.n_tiles = (n_ap + vk::kTile - 1) / vk::kTile;
  if ((rc = cu(vk::launch_search(sa, prm->pad_rate, st, &n_launch), "search kernel"))) return rc;

  UnpackArgs ua{};
  ua.keys = keys;
  ua.nvalid = ta.nvalid;
  ua.peak_power = peak_power;
  ua.peak_cell = peak_cell;
  ua.n_dm = n_dm;
  ua.n_win = n_win;
  ua.seg_per_bd = seg_per_bd;
  ua.total = total;
  for (int i = 0; i < n_win; ++i) {
    ua.win[i] = prm->win[i];
    ua.win_off[i] = win_off_i[i];
  }
  na_unpack_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(ua);
  return cu(cudaGetLastError(), "unpack kernel");
}

extern "C" int volks_noalloc_tables(void* cuda_stream, int32_t* shifts, int32_t* nvalid, int32_t n_dm,
                                    int32_t n_f) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return na_fail(VOLKS_EINVAL, "no current CUDA device");
  }
  if (dev < 0 || dev >= kMaxDevices) return na_fail(VOLKS_EINVAL, "device ordinal %d out of range", dev);
  LastTables lt;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    lt = g_last[dev];
  }
  if (!lt.set) return na_fail(VOLKS_EINVAL, "no no-allocation search has run on device %d", dev);
  if (n_dm != lt.n_dm || n_f != lt.n_f)
    return na_fail(VOLKS_EINVAL, "last call had n_dm %d, n_f %d (asked %d, %d)", lt.n_dm, lt.n_f, n_dm, n_f);
  if (lt.n_dm == 0) return 0;
  int rc = device_buffer(shifts, dev, "shifts");
  if (!rc) rc = device_buffer(nvalid, dev, "nvalid");
  if (rc) return rc;
  void* base = nullptr;
  if ((rc = scratch_ptr(&base))) return rc;
  const unsigned char* sp = static_cast<const unsigned char*>(base);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  cudaError_t e = cudaMemcpyAsync(shifts, sp + lt.o_shifts, (size_t)lt.n_dm * lt.n_f * sizeof(int32_t),
                                  cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(nvalid, sp + lt.o_nvalid, (size_t)lt.n_dm * sizeof(int32_t), cudaMemcpyDeviceToDevice, st);
  return e == cudaSuccess ? 0 : na_fail(VOLKS_ECUDA, "copy tables: %s", cudaGetErrorString(e));
}
