// sm_103a kernels of the cross-spectrum single-pulse search.
//
//   prep     a2-a3  per-channel power (FP64 accumulation), gains, normalise + calibrate +
//                   transpose the visibilities to channel-major [b][k][t]
//   search   a4-a7  fused: dedispersed gather of a 32-AP tile, delay FFT
//                   (pad 4, one residue class of delay cells per pass, every
//                   residue of the tile in one unit), rate FFTs of every
//                   window, |Z|^2 and arg-max, all on chip; one key store
//                   per segment to global memory
//   select   a8     FP64 series mean / std, z-score threshold -> bitmaps
//   match    a9     per (baseline, DM) sweep over selected segments of all
//                   windows in start order: overlap groups -> candidates
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <cuda_runtime.h>

#include "../../include/volks.h"
#include "fft_regs.cuh"
#include "search_common.cuh"
#include "search_kernel.cuh"
#include "volks_internal.h"

namespace vk {

// ============================================================== prep ====
// Partial sums over a chunk of APs.  Row r of the grid's z axis is
// (polarisation, baseline) summing |S|^2 of the cross spectrum, or, with
// auto spectra, (polarisation, station) summing a^2.  Each thread owns two
// adjacent frequency points (one 16-byte load of two complex values, or 8
// bytes of two auto powers) and one AP phase of 8; four APs are loaded at
// once, their squares summed in FP32 (a few terms, one rounding each) and
// that sum accumulated in FP64 over the chunk, so the per-point power over
// the segment is an FP64 accumulation.  VEC = false takes the same path
// with 8-byte loads when the caller's buffer is not 16-byte aligned.
template <bool AUTO, bool VEC>
__global__ void __launch_bounds__(256) chan_power_kernel(const PrepArgs a) {
  __shared__ double red[8][2][33];
  const int k = 2 * (blockIdx.x * 32 + threadIdx.x);
  const int tc = blockIdx.y, row = blockIdx.z;
  const int t_beg = tc * a.tchunk;
  const int t_end = min(a.n_ap, t_beg + a.tchunk);
  double s0 = 0.0, s1 = 0.0;
  if (k < a.n_f) {  // n_f is even
    // (power of point k, power of point k + 1) of AP t
    auto pw = [&](int t) -> float2 {
      if constexpr (AUTO) {
        const float* v = a.autos + ((size_t)row * a.n_ap + t) * a.n_f + k;
        float2 x;
        if constexpr (VEC) {
          x = __ldg(reinterpret_cast<const float2*>(v));
        } else {
          x = make_float2(__ldg(v), __ldg(v + 1));
        }
        return make_float2(x.x * x.x, x.y * x.y);
      } else {
        const float2* v = a.vis + ((size_t)row * a.n_ap + t) * a.n_f + k;
        float4 x;
        if constexpr (VEC) {
          x = __ldg(reinterpret_cast<const float4*>(v));
        } else {
          const float2 u = __ldg(v), w = __ldg(v + 1);
          x = make_float4(u.x, u.y, w.x, w.y);
        }
        return make_float2(fmaf(x.y, x.y, x.x * x.x), fmaf(x.w, x.w, x.z * x.z));
      }
    };
    int t = t_beg + (int)threadIdx.y;
    for (; t + 24 < t_end; t += 32) {
      const float2 p0 = pw(t), p1 = pw(t + 8), p2 = pw(t + 16), p3 = pw(t + 24);
      s0 += (double)((p0.x + p1.x) + (p2.x + p3.x));
      s1 += (double)((p0.y + p1.y) + (p2.y + p3.y));
    }
    for (; t < t_end; t += 8) {
      const float2 p0 = pw(t);
      s0 += (double)p0.x;
      s1 += (double)p0.y;
    }
  }
  red[threadIdx.y][0][threadIdx.x] = s0;
  red[threadIdx.y][1][threadIdx.x] = s1;
  __syncthreads();
  if (threadIdx.y < 2 && k < a.n_f) {
    const int j = threadIdx.y;
    double v = 0.0;
#pragma unroll
    for (int i = 0; i < 8; ++i) v += red[i][j][threadIdx.x];
    a.part[((size_t)row * a.n_tchunk + tc) * a.n_f + k + j] = v;
  }
}

__device__ __forceinline__ double mean_power(const PrepArgs& a, int row, int k) {
  double s = 0.0;
  for (int tc = 0; tc < a.n_tchunk; ++tc) s += a.part[((size_t)row * a.n_tchunk + tc) * a.n_f + k];
  return s / (double)a.n_ap;
}

// gain[p][b][k] = phasor * normalisation (FP64, then rounded once to FP32):
// 1 / RMS of the cross spectrum, or (mean a_i^2 mean a_j^2)^(-1/4) with the
// stations' auto spectra (HOPS, Sec. 2.2).
__global__ void gain_kernel(const PrepArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n_pol * a.n_bl * a.n_f) return;
  const int pb = i / a.n_f, k = i % a.n_f;
  const double2 ph = a.phasor[i];
  double gr = ph.x, gi = ph.y;
  if (a.normalize) {
    double norm;
    if (a.autos) {
      const int p = pb / a.n_bl, b = pb % a.n_bl;
      const int2 st = a.bl_st[b];
      const double pij = mean_power(a, p * a.n_st + st.x, k) * mean_power(a, p * a.n_st + st.y, k);
      norm = pij > 0.0 ? 1.0 / sqrt(sqrt(pij)) : 0.0;
    } else {
      const double rms = sqrt(mean_power(a, pb, k));
      norm = rms > 0.0 ? 1.0 / rms : 0.0;
    }
    gr *= norm;
    gi *= norm;
  }
  if (a.skip_first_chan && (k % a.n_chan) == 0) gr = gi = 0.0;
  a.gain[i] = make_float2((float)gr, (float)gi);
}

// xn[b][k][t] = sum_p vis[p][b][t][k] * gain[p][b][k]: 32x32 tiles through
// shared memory.
template <int NPOL>
__global__ void __launch_bounds__(256) normalize_transpose_kernel(const PrepArgs a) {
  __shared__ float2 tile[32][33];
  const int t0 = blockIdx.x * 32, k0 = blockIdx.y * 32, b = blockIdx.z;
  const int k = k0 + threadIdx.x;
  const size_t plane = (size_t)a.n_bl * a.n_ap * a.n_f;
  float2 g[NPOL];
#pragma unroll
  for (int p = 0; p < NPOL; ++p) g[p] = a.gain[((size_t)p * a.n_bl + b) * a.n_f + k];
  const float2* v = a.vis + (size_t)b * a.n_ap * a.n_f;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int tl = threadIdx.y + 8 * i;
    const int t = t0 + tl;
    float2 x = make_float2(0.f, 0.f);
    if (t < a.n_ap) {
      x = cmul(v[(size_t)t * a.n_f + k], g[0]);
#pragma unroll
      for (int p = 1; p < NPOL; ++p) {
        const float2 y = cmul(v[p * plane + (size_t)t * a.n_f + k], g[p]);
        x.x += y.x;
        x.y += y.y;
      }
    }
    tile[tl][threadIdx.x] = x;
  }
  __syncthreads();
  float2* o = a.xn + (size_t)b * a.n_f * a.n_ap;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int kl = threadIdx.y + 8 * i;
    const int t = t0 + threadIdx.x;
    if (t < a.n_ap) o[(size_t)(k0 + kl) * a.n_ap + t] = tile[threadIdx.x][kl];
  }
}

cudaError_t launch_prep(const PrepArgs& a, cudaStream_t s, int* n_launch) {
  dim3 blk(32, 8);
  const bool autos = a.normalize && a.autos;
  const int rows = a.n_pol * (autos ? a.n_st : a.n_bl);
  if (a.normalize) {
    // two frequency points per thread: bands have an even number of points
    if (a.n_f & 1) return cudaErrorInvalidValue;
    const dim3 g((a.n_f + 63) / 64, a.n_tchunk, rows);
    if (autos) {
      if ((reinterpret_cast<uintptr_t>(a.autos) & 7) == 0)
        chan_power_kernel<true, true><<<g, blk, 0, s>>>(a);
      else
        chan_power_kernel<true, false><<<g, blk, 0, s>>>(a);
    } else {
      if ((reinterpret_cast<uintptr_t>(a.vis) & 15) == 0)
        chan_power_kernel<false, true><<<g, blk, 0, s>>>(a);
      else
        chan_power_kernel<false, false><<<g, blk, 0, s>>>(a);
    }
    *n_launch += 1;
  }
  gain_kernel<<<(a.n_pol * a.n_bl * a.n_f + 255) / 256, 256, 0, s>>>(a);
  const dim3 grid((a.n_ap + 31) / 32, a.n_f / 32, a.n_bl);
  if (a.n_pol == 2)
    normalize_transpose_kernel<2><<<grid, blk, 0, s>>>(a);
  else
    normalize_transpose_kernel<1><<<grid, blk, 0, s>>>(a);
  *n_launch += 2;
  return cudaGetLastError();
}

// ============================================================ search ====
VK_MIXED_VARIANTS(VK_SEARCH_EXTERN, 0)
VK_MIXED_VARIANTS(VK_SEARCH_EXTERN, 4)
VK_POW2_VARIANTS(VK_SEARCH_EXTERN_SLIDE, 0)
VK_POW2_VARIANTS(VK_SEARCH_EXTERN_SLIDE, 4)

// Compiled work splits: (n1, fold) with 32 * n1 * fold = n_f; n1 = 3, 6, 12
// serve the bands of 3 * 2^a points (96 .. 1536) with mixed-radix FFTs.
#define VK_VARIANTS(X, PADR) VK_POW2_VARIANTS(X, PADR) VK_MIXED_VARIANTS(X, PADR)

int effective_precision(int n_f, int pad_rate, int precision) {
  if (precision == VOLKS_FP32 || pad_rate != 4) return VOLKS_FP32;
  SearchVariant v[4];
  int n = 0;
#define VK_LIST(N1, PADR, FOLD) \
  if (32 * N1 * FOLD == n_f && n < 4) v[n++] = SearchVariant{N1, FOLD};
  VK_VARIANTS(VK_LIST, 0)
#undef VK_LIST
  for (int i = 0; i < n; ++i)
    if (mma_supported(v[i], pad_rate, precision)) return precision;
  return VOLKS_FP32;
}

int search_variants(int n_f, int precision, SearchVariant* out) {
  int n = 0;
#define VK_LIST(N1, PADR, FOLD)                                                         \
  if (32 * N1 * FOLD == n_f && n < 4 &&                                                 \
      (precision == VOLKS_FP32 || mma_supported(SearchVariant{N1, FOLD}, 4, precision))) \
    out[n++] = SearchVariant{N1, FOLD};
  VK_VARIANTS(VK_LIST, 0)
#undef VK_LIST
  return n;
}

SearchVariant default_variant(int n_f, int precision, int fold_override) {
  SearchVariant v[4];
  const int n = search_variants(n_f, precision, v);
  if (fold_override > 0)
    for (int i = 0; i < n; ++i)
      if (v[i].fold == fold_override) return v[i];
  // fewest folds (fewest gathered inputs per thread), then the most threads
  SearchVariant best = n > 0 ? v[0] : SearchVariant{0, 0};
  for (int i = 1; i < n; ++i)
    if (v[i].fold < best.fold) best = v[i];
  return best;
}

// Work units of a range: (baseline, DM trial, 32-AP tile[, AP phase]); a
// unit runs all pad_delay x fold delay residues of its tile.
long long search_units(const SegDesc& d, SearchVariant v) {
  (void)v;
  return (long long)d.n_bl * d.n_tiles * d.n_dm * desc_phases(d.win_mask);
}

int search_occupancy(SearchVariant v, int pad_rate, int precision) {
  if (precision != VOLKS_FP32) return mma_supported(v, pad_rate, precision) ? 1 : 0;
#define VK_OCC(N1, PADR, FOLD) \
  if (v.n1 == N1 && v.fold == FOLD && pad_rate == PADR) return occupancy_t<N1, PADR, FOLD, false>();
  VK_VARIANTS(VK_OCC, 0)
  VK_VARIANTS(VK_OCC, 4)
#undef VK_OCC
  return 0;
}

cudaError_t launch_search_batch(Batch& b, SearchVariant v, int pad_rate, int precision, int grid_ctas,
                                cudaStream_t s, int* n_launch) {
  if (precision != VOLKS_FP32) {
    if (!mma_supported(v, pad_rate, precision)) return cudaErrorInvalidValue;
    return launch_search_mma(b, v, precision, grid_ctas, s, n_launch);
  }
  // a launch with any sliding range takes the sliding form (which also
  // serves back-to-back ranges)
  bool slide = false;
  for (int i = 0; i < b.n_desc; ++i) slide = slide || desc_slide(b.d[i].win_mask);
#define VK_LAUNCH(N1, PADR, FOLD)                                                   \
  if (v.n1 == N1 && v.fold == FOLD && pad_rate == PADR)                              \
    return slide ? launch_search_t<N1, PADR, FOLD, true>(b, grid_ctas, s, n_launch) \
                 : launch_search_t<N1, PADR, FOLD, false>(b, grid_ctas, s, n_launch);
  VK_VARIANTS(VK_LAUNCH, 0)
  VK_VARIANTS(VK_LAUNCH, 4)
#undef VK_LAUNCH
  return cudaErrorInvalidValue;
}

cudaError_t launch_search(const SearchArgs& a, int pad_rate, cudaStream_t s, int* n_launch) {
  Batch b;
  memset(&b, 0, sizeof b);
  SegDesc& d = b.d[0];
  d.xn = a.xn;
  d.shifts = a.shifts;
  d.nvalid = a.nvalid;
  d.tw_n = a.tw_n;
  d.tw_m = a.tw_m;
  d.keys = a.keys;
  d.seg_per_bd = a.seg_per_bd;
  d.n_bl = a.n_bl;
  d.n_ap = a.n_ap;
  d.n_f = a.n_f;
  d.n_dm = a.n_dm;
  d.n_dm_total = a.n_dm;
  d.pad_delay = a.pad_delay;
  d.M = a.M;
  d.n_tiles = a.n_tiles;
  d.win_mask = a.win_mask;
  for (int l = 0; l <= kMaxWinLog; ++l) d.win_off_l[l] = a.win_off[l];
  b.n_desc = 1;
  const SearchVariant v = default_variant(a.n_f, VOLKS_FP32, a.fold);
  if (v.n1 == 0) return cudaErrorInvalidValue;
  b.total = search_units(d, v);
  return launch_search_batch(b, v, pad_rate, VOLKS_FP32, 0, s, n_launch);
}

// ============================================================ select ====
// Normalised power rho = P / (W N_eff) and z = (rho - mu) / sd of one
// segment, each as a product with a reciprocal formed once per series (FP64
// division is costly on this part), with round-to-nearest intrinsics so
// that the select and match kernels compute bit-identical values.  sd = 0
// (an all-equal series) gives inv_sd = 0 and so z = 0.
__device__ __forceinline__ double seg_inv_wn(int W, int n_eff) { return __ddiv_rn(1.0, (double)(W * n_eff)); }
__device__ __forceinline__ double seg_inv_sd(double sd) { return sd > 0.0 ? __ddiv_rn(1.0, sd) : 0.0; }
__device__ __forceinline__ double seg_rho(unsigned long long key, double inv_wn) {
  const float P = __uint_as_float((uint32_t)(key >> 32));
  return __dmul_rn((double)P, inv_wn);
}
__device__ __forceinline__ double seg_z(double rho, double mu, double inv_sd) {
  return __dmul_rn(__dsub_rn(rho, mu), inv_sd);
}

template <int NT>
__device__ __forceinline__ double2 block_sum2(double a, double b, double2* red) {
  red[threadIdx.x] = make_double2(a, b);
  __syncthreads();
#pragma unroll
  for (int h = NT / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) {
      const double2 x = red[threadIdx.x], y = red[threadIdx.x + h];
      red[threadIdx.x] = make_double2(x.x + y.x, x.y + y.y);
    }
    __syncthreads();
  }
  const double2 r = red[0];
  __syncthreads();
  return r;
}

// One CTA per (range, baseline, DM trial, window) series: FP64 mean and
// population standard deviation of rho (one read of the keys), then the
// z >= thresh bitmap (a second read).
__global__ void __launch_bounds__(256) select_kernel(const __grid_constant__ Batch p) {
  constexpr int NT = 256;
  __shared__ double2 red2[NT];
  const long long u = (long long)blockIdx.x + p.unit0;
  if (u >= p.total) return;
  const SegDesc& a = p.d[find_desc(p, u)];
  long long ls = u - a.base;
  const int wi = (int)(ls % a.n_win);
  ls /= a.n_win;
  const int d = (int)(ls % a.n_dm);
  const int b = (int)(ls / a.n_dm);
  const int W = 1 << a.win_log[wi];
  const int nseg = seg_count(a.nvalid[d], a.win_log[wi], desc_slide(a.win_mask));
  const double inv_wn = seg_inv_wn(W, a.n_eff);
  const size_t bd = (size_t)b * a.n_dm + d;
  const unsigned long long* k = a.keys + bd * a.seg_per_bd + a.win_off[wi];
  // one pass over the keys: sums of (rho - K) and (rho - K)^2 about the
  // series' first value K (the shift keeps the variance free of
  // cancellation), combined in a fixed tree
  const double K = nseg > 0 ? seg_rho(k[0], inv_wn) : 0.0;
  double s1 = 0.0, s2 = 0.0;
  for (int i = threadIdx.x; i < nseg; i += NT) {
    const double dv = seg_rho(k[i], inv_wn) - K;
    s1 += dv;
    s2 = fma(dv, dv, s2);
  }
  double mu = 0.0, sd = 0.0;
  if (nseg > 0) {
    const double2 t = block_sum2<NT>(s1, s2, red2);
    const double n = (double)nseg, m1 = t.x / n;
    mu = K + m1;
    sd = sqrt(fmax(t.y / n - m1 * m1, 0.0));
  }
  if (threadIdx.x == 0) {
    double* st = a.stats + (((size_t)b * a.n_dm_total + a.d0 + d) * a.n_win + wi) * 2;
    st[0] = mu;
    st[1] = sd;
  }
  uint32_t* bits = a.bits + bd * a.word_per_bd + a.word_off[wi];
  const double thresh = a.thresh, inv_sd = seg_inv_sd(sd);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int base = warp * 32; base < nseg; base += NT) {
    const int i = base + lane;
    const bool sel = i < nseg && seg_z(seg_rho(k[i], inv_wn), mu, inv_sd) >= thresh;
    const uint32_t w = __ballot_sync(0xffffffffu, sel);
    if (lane == 0) bits[base / 32] = w;
  }
}

cudaError_t launch_select_batch(Batch& b, cudaStream_t s, int* n_launch) {
  const long long max_grid = 2147483647LL;
  for (long long u0 = 0; u0 < b.total; u0 += max_grid) {
    b.unit0 = u0;
    select_kernel<<<(unsigned)std::min(max_grid, b.total - u0), 256, 0, s>>>(b);
    ++*n_launch;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// ============================================================= match ====
// One thread per (range, baseline, DM trial): merge the selected segments
// of all windows in order of start AP and sweep overlap groups.
__global__ void __launch_bounds__(128) match_kernel(const __grid_constant__ Batch p) {
  const long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x + p.unit0;
  if (u >= p.total) return;
  const SegDesc& a = p.d[find_desc(p, u)];
  const long long lu = u - a.base;
  const int d = (int)(lu % a.n_dm), b = (int)(lu / a.n_dm);
  const int nv = max(a.nvalid[d], 0);
  const size_t bd = (size_t)b * a.n_dm + d;
  const uint32_t* bits = a.bits + bd * a.word_per_bd;
  const unsigned long long* keys = a.keys + bd * a.seg_per_bd;
  const int n_win = a.n_win, n_eff = a.n_eff;
  int wlog[kMaxWinLog + 1], woff[kMaxWinLog + 1], wdoff[kMaxWinLog + 1];
  uint32_t cur[kMaxWinLog + 1];
  int wordi[kMaxWinLog + 1], nwords[kMaxWinLog + 1];
  for (int wi = 0; wi < n_win; ++wi) {
    wlog[wi] = a.win_log[wi];
    woff[wi] = a.win_off[wi];
    wdoff[wi] = a.word_off[wi];
    const int nseg = seg_count(nv, wlog[wi], desc_slide(a.win_mask));
    nwords[wi] = (nseg + 31) / 32;
    wordi[wi] = 0;
    cur[wi] = nwords[wi] > 0 ? bits[wdoff[wi]] : 0u;
  }
  const double* stats = a.stats + ((size_t)b * a.n_dm_total + a.d0 + d) * n_win * 2;
  int g0 = 0, g1 = 0, mask = 0;
  int rw = 0, rs = 0;
  double rz = 0.0, rrho = 0.0;
  unsigned long long rkey = 0;
  auto flush = [&]() {
    if (mask != 0 && __popc(mask) >= a.min_windows) {
      const unsigned int o = atomicAdd(a.count, 1u);
      if (o < a.cap) {
        DevCand c;
        c.bl = b;
        c.dm_idx = a.d0 + d;
        c.win_log = wlog[rw];
        c.seg = rs;
        c.g0 = g0;
        c.g1 = g1;
        c.n_windows = __popc(mask);
        c.lin = 0xffffffffu - (uint32_t)(rkey & 0xffffffffu);
        c.P = __uint_as_float((uint32_t)(rkey >> 32));
        c._pad = 0.f;
        c.rho = rrho;
        c.z = rz;
        a.cand[o] = c;
      }
    }
  };
  for (;;) {
    int bw = -1, bstart = 0x7fffffff, bsg = 0;
    for (int wi = 0; wi < n_win; ++wi) {
      while (cur[wi] == 0u && wordi[wi] + 1 < nwords[wi]) {
        ++wordi[wi];
        cur[wi] = bits[wdoff[wi] + wordi[wi]];
      }
      if (cur[wi] != 0u) {
        const int sg = wordi[wi] * 32 + __ffs(cur[wi]) - 1;
        const int st = seg_start(sg, wlog[wi], desc_slide(a.win_mask));
        if (st < bstart) {
          bstart = st;
          bw = wi;
          bsg = sg;
        }
      }
    }
    if (bw < 0) break;
    cur[bw] &= cur[bw] - 1u;
    const int W = 1 << wlog[bw];
    const int end = bstart + W;
    const unsigned long long key = keys[woff[bw] + bsg];
    const double rho = seg_rho(key, seg_inv_wn(W, n_eff));
    const double z = seg_z(rho, stats[bw * 2], seg_inv_sd(stats[bw * 2 + 1]));
    if (mask != 0 && bstart < g1) {
      g1 = max(g1, end);
      mask |= 1 << bw;
      const int RW = 1 << wlog[rw];
      if (z > rz || (z == rz && (W < RW || (W == RW && bsg < rs)))) {
        rz = z; rrho = rho; rw = bw; rs = bsg; rkey = key;
      }
    } else {
      flush();
      g0 = bstart;
      g1 = end;
      mask = 1 << bw;
      rz = z; rrho = rho; rw = bw; rs = bsg; rkey = key;
    }
  }
  flush();
}

cudaError_t launch_match_batch(Batch& b, cudaStream_t s, int* n_launch) {
  const long long per = 2147483647LL * 128;
  for (long long u0 = 0; u0 < b.total; u0 += per) {
    b.unit0 = u0;
    const long long n = std::min(per, b.total - u0);
    match_kernel<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(b);
    ++*n_launch;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace vk
