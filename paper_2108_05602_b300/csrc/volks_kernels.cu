// sm_103a kernels of the cross-spectrum single-pulse search.
//
//   prep     a2-a3  FP64 per-channel power, gains, normalise + calibrate +
//                   transpose the visibilities to channel-major [b][k][t]
//   search   a4-a7  fused: dedispersed gather of a 32-AP tile, delay FFT
//                   (pad 4, one residue class of delay cells per CTA), rate
//                   FFTs of every window, |Z|^2 and arg-max, all on chip;
//                   one 64-bit atomicMax per (segment, CTA) to global memory
//   select   a8     FP64 series mean / std, z-score threshold -> bitmaps
//   match    a9     per (baseline, DM) sweep over selected segments of all
//                   windows in start order: overlap groups -> candidates
#include <algorithm>
#include <cstdint>
#include <cuda_runtime.h>

#include "fft_regs.cuh"
#include "volks_internal.h"

namespace vk {

// ============================================================== prep ====
// Partial sums of |S|^2 in FP64 over a chunk of APs, one thread per
// (frequency point, AP phase); coalesced along frequency.
__global__ void __launch_bounds__(256) chan_power_kernel(const PrepArgs a) {
  __shared__ double red[8][33];
  const int k = blockIdx.x * 32 + threadIdx.x;
  const int tc = blockIdx.y, b = blockIdx.z;
  const int t_beg = tc * a.tchunk;
  const int t_end = min(a.n_ap, t_beg + a.tchunk);
  double s = 0.0;
  if (k < a.n_f) {
    const float2* v = a.vis + (size_t)b * a.n_ap * a.n_f + k;
    for (int t = t_beg + (int)threadIdx.y; t < t_end; t += 8) {
      const float2 x = v[(size_t)t * a.n_f];
      s = fma((double)x.x, (double)x.x, s);
      s = fma((double)x.y, (double)x.y, s);
    }
  }
  red[threadIdx.y][threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.y == 0 && k < a.n_f) {
    double t = 0.0;
#pragma unroll
    for (int i = 0; i < 8; ++i) t += red[i][threadIdx.x];
    a.part[((size_t)b * a.n_tchunk + tc) * a.n_f + k] = t;
  }
}

// gain = phasor / rms (FP64, then rounded once to FP32).
__global__ void gain_kernel(const PrepArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n_bl * a.n_f) return;
  const int b = i / a.n_f, k = i % a.n_f;
  double s = 0.0;
  for (int tc = 0; tc < a.n_tchunk; ++tc) s += a.part[((size_t)b * a.n_tchunk + tc) * a.n_f + k];
  const double2 ph = a.phasor[i];
  double gr = ph.x, gi = ph.y;
  if (a.normalize) {
    const double rms = sqrt(s / (double)a.n_ap);
    if (rms > 0.0) {
      gr /= rms;
      gi /= rms;
    } else {
      gr = gi = 0.0;
    }
  }
  if (a.skip_first_chan && (k % a.n_chan) == 0) gr = gi = 0.0;
  a.gain[i] = make_float2((float)gr, (float)gi);
}

// xn[b][k][t] = vis[b][t][k] * gain[b][k]: 32x32 tiles through shared memory.
__global__ void __launch_bounds__(256) normalize_transpose_kernel(const PrepArgs a) {
  __shared__ float2 tile[32][33];
  const int t0 = blockIdx.x * 32, k0 = blockIdx.y * 32, b = blockIdx.z;
  const int k = k0 + threadIdx.x;
  const float2 g = a.gain[(size_t)b * a.n_f + k];
  const float2* v = a.vis + (size_t)b * a.n_ap * a.n_f;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int tl = threadIdx.y + 8 * i;
    const int t = t0 + tl;
    float2 x = make_float2(0.f, 0.f);
    if (t < a.n_ap) x = cmul(v[(size_t)t * a.n_f + k], g);
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
  chan_power_kernel<<<dim3((a.n_f + 31) / 32, a.n_tchunk, a.n_bl), blk, 0, s>>>(a);
  gain_kernel<<<(a.n_bl * a.n_f + 255) / 256, 256, 0, s>>>(a);
  normalize_transpose_kernel<<<dim3((a.n_ap + 31) / 32, a.n_f / 32, a.n_bl), blk, 0, s>>>(a);
  *n_launch += 3;
  return cudaGetLastError();
}

// ============================================================ search ====
// Arg-max over cells LO .. LO+LEN-1 by a balanced tree (depth log2 LEN, so
// the compare/select chain does not serialise): the right half wins only if
// strictly larger, which keeps the lowest index on exact ties.
template <int LO, int LEN, class F>
__device__ __forceinline__ void argmax_tree(const F& pw, float& v, uint32_t& q) {
  if constexpr (LEN == 1) {
    v = pw(std::integral_constant<int, LO>{});
    q = LO;
  } else {
    float v1, v2;
    uint32_t q1, q2;
    argmax_tree<LO, LEN / 2>(pw, v1, q1);
    argmax_tree<LO + LEN / 2, LEN / 2>(pw, v2, q2);
    const bool right = v2 > v1;
    v = right ? v2 : v1;
    q = right ? q2 : q1;
  }
}

// Rate transform, |Z|^2 and arg-max of every window-W segment of the tile
// for the delay column this thread owns.  Per segment the warp's best
// (power, lowest linear cell) goes to slot[(slot0 + s) * N1 + warp].
template <int W, int PADR, int N1>
__device__ __forceinline__ void rate_window(const float2* __restrict__ S, int c, uint32_t m,
                                            uint32_t M, int t0, int nv, int slot0,
                                            uint2* slot, int warp, int lane) {
  constexpr int N = 32 * N1, LD = N + 1;
  constexpr int NSEG = kTile / W;
  constexpr int R = (W == 1 || PADR == 0) ? 1 : PADR * W;
  const int nseg = min(NSEG, max(0, nv / W - t0 / W));
#pragma unroll 1
  for (int s = 0; s < nseg; ++s) {
    const float2* col = S + (s * W) * LD + c;
    float best;
    uint32_t bq;
    if constexpr (R == 1) {
      float2 z = col[0];
      static_for<1, W>([&](auto u) { z = cadd(z, col[decltype(u)::value * LD]); });
      best = cabs2(z);
      bq = 0;
    } else if constexpr (W == 2 && R == 8) {
      // |y0 + y1 W_8^q|^2 = r0 + 2 Re(r1 W_8^q), r0 = |y0|^2 + |y1|^2,
      // r1 = y1 conj(y0): the power spectrum is the DFT of the lag products.
      const float2 y0 = col[0], y1 = col[LD];
      const float r0 = fmaf(y1.y, y1.y, fmaf(y1.x, y1.x, cabs2(y0)));
      const float rx = fmaf(y1.y, y0.y, y1.x * y0.x);
      const float ry = fmaf(y1.y, y0.x, -(y1.x * y0.y));
      constexpr float kS2 = Tw<8, 1>::re * 2.0f;   // sqrt(2)
      const float a = rx + rx, bb = ry + ry;
      const float cc = kS2 * (rx + ry), dd = kS2 * (ry - rx);
      const float P[8] = {r0 + a, r0 + cc, r0 + bb, r0 + dd, r0 - a, r0 - cc, r0 - bb, r0 - dd};
      argmax_tree<0, 8>([&](auto qq) { return P[decltype(qq)::value]; }, best, bq);
    } else {
      best = -1.f;
      bq = 0;
      static_for<0, PADR>([&](auto rho) {
        constexpr int RHO = decltype(rho)::value;
        // reload the column for every residue rather than keep 2W registers live
        asm volatile("" ::: "memory");
        float2 y[W];
        static_for<0, W>([&](auto u) {
          constexpr int U = decltype(u)::value;
          y[U] = twiddle<R, U * RHO>(col[U * LD]);
        });
        fft_dif<W>(y);
        float vb;
        uint32_t vq;
        argmax_tree<0, W>([&](auto qq) { return cabs2(y[bitrev(decltype(qq)::value, ilog2(W))]); },
                          vb, vq);
        const uint32_t q = PADR * vq + RHO;
        if (vb > best || (vb == best && q < bq)) {
          best = vb;
          bq = q;
        }
      });
    }
    const uint32_t lin = bq * M + m;
    const uint32_t pb = __float_as_uint(best);
    const uint32_t wmax = __reduce_max_sync(0xffffffffu, pb);
    const uint32_t wlin = __reduce_min_sync(0xffffffffu, pb == wmax ? lin : 0xffffffffu);
    if (lane == 0) slot[(slot0 + s) * N1 + warp] = make_uint2(wmax, wlin);
  }
}

// One CTA = (baseline b, DM trial d, 32-AP tile, delay residue r).  Zero
// padding by pad_delay, with the band folded FOLD times, splits the M-point
// delay transform (M = pad_delay * n_f) into P = pad_delay * FOLD
// independent N-point FFTs, N = n_f / FOLD:
//   Y[P c + r] = sum_{k<N} W_M^{k r} (sum_{f<FOLD} X[k + N f] W_P^{f r}) W_N^{k c},
// so a CTA computes the delay cells m = P c + r (c < N) of its residue r.
// N = 32 * N1; the CTA has N threads.
//   stage 0  lane = AP, warp owns k0 = warp*KPW + j: gather xn[k][t + shift_k],
//            fold and pre-twiddle
//   stage 1  N1-point FFTs over k1 (k = k0 + 32 k1), twiddle W_N^{k0 m1}
//   stage 2  lane = AP, warp = m1: 32-point FFT over k0 -> Y[m1 + N1 m2]
//   stage 3  thread = delay column c: rate FFTs over the tile's APs
template <int N1, int PADR, int FOLD>
__global__ void __launch_bounds__(32 * N1, 16 / N1) search_kernel(const SearchArgs a, int b_base) {
  constexpr int N = 32 * N1;
  constexpr int KPW = 32 / N1;
  constexpr int LD = N + 1;
  extern __shared__ __align__(16) float2 sm[];
  float2* S = sm;
  uint2* slot = reinterpret_cast<uint2*>(sm + 32 * LD);

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int P = a.pad_delay * FOLD;
  long long bid = blockIdx.x;
  const int r = (int)(bid % P);
  bid /= P;
  const int d = (int)(bid % a.n_dm);
  bid /= a.n_dm;
  const int tile = (int)(bid % a.n_tiles);
  const int b = b_base + (int)(bid / a.n_tiles);
  const int t0 = tile * kTile;
  const int nv = a.nvalid[d];
  if (t0 >= nv) return;

  // ---- stage 0 + 1 ----
  {
    const float2* xb = a.xn + (size_t)b * a.n_f * a.n_ap;
    const int32_t* sh = a.shifts + (size_t)d * a.n_f;
    const int t = t0 + lane;
    const bool tin = t < nv;
    float2 wf[FOLD];  // W_P^{f r} = W_M^{N f r}
    static_for<0, FOLD>([&](auto ff) {
      constexpr int F = decltype(ff)::value;
      wf[F] = F == 0 ? make_float2(1.f, 0.f) : __ldg(a.tw_m + (N * F * r) % a.M);
    });
    static_for<0, KPW>([&](auto jj) {
      constexpr int J = decltype(jj)::value;
      const int k0 = warp * KPW + J;
      float2 x[N1];
      static_for<0, N1>([&](auto kk1) {
        constexpr int K1 = decltype(kk1)::value;
        const int k = k0 + 32 * K1;
        float2 v = make_float2(0.f, 0.f);
        static_for<0, FOLD>([&](auto ff) {
          constexpr int F = decltype(ff)::value;
          const int kf = k + N * F;
          float2 u = make_float2(0.f, 0.f);
          if (tin) u = __ldg(xb + (size_t)kf * a.n_ap + t + __ldg(sh + kf));
          if constexpr (F == 0) {
            v = u;
          } else {
            v = cadd(v, cmul(u, wf[F]));
          }
        });
        if (r != 0) v = cmul(v, __ldg(a.tw_m + (k * r) % a.M));
        x[K1] = v;
      });
      fft_dif<N1>(x);
      static_for<0, N1>([&](auto mm1) {
        constexpr int M1 = decltype(mm1)::value;
        float2 v = x[bitrev(M1, ilog2(N1))];
        // W_N^{k0 m1} = W_{n_f}^{k0 m1 FOLD}
        if constexpr (M1 != 0) v = cmul(v, __ldg(a.tw_n + (k0 * M1 * FOLD) % a.n_f));
        S[lane * LD + k0 * N1 + M1] = v;
      });
    });
  }
  __syncthreads();
  // ---- stage 2 ----
  {
    float2 y[32];
    static_for<0, 32>([&](auto kk0) {
      constexpr int K0 = decltype(kk0)::value;
      y[K0] = S[lane * LD + K0 * N1 + warp];
    });
    fft_dif<32>(y);
    __syncthreads();
    static_for<0, 32>([&](auto mm2) {
      constexpr int M2 = decltype(mm2)::value;
      S[lane * LD + warp + N1 * M2] = y[bitrev(M2, 5)];
    });
  }
  __syncthreads();
  // ---- stage 3 ----
  const int c = threadIdx.x;
  const uint32_t m = (uint32_t)(c * P + r);
  const uint32_t M = (uint32_t)a.M;
  // slot base of window 2^l: segments of the searched smaller windows first
  auto slot_base = [&](int l) {
    int o = 0;
    for (int i = 0; i < l; ++i)
      if (a.win_mask & (1 << i)) o += kTile >> i;
    return o;
  };
  if (a.win_mask & 1) rate_window<1, PADR, N1>(S, c, m, M, t0, nv, slot_base(0), slot, warp, lane);
  if (a.win_mask & 2) rate_window<2, PADR, N1>(S, c, m, M, t0, nv, slot_base(1), slot, warp, lane);
  if (a.win_mask & 4) rate_window<4, PADR, N1>(S, c, m, M, t0, nv, slot_base(2), slot, warp, lane);
  if (a.win_mask & 8) rate_window<8, PADR, N1>(S, c, m, M, t0, nv, slot_base(3), slot, warp, lane);
  if (a.win_mask & 16) rate_window<16, PADR, N1>(S, c, m, M, t0, nv, slot_base(4), slot, warp, lane);
  if (a.win_mask & 32) rate_window<32, PADR, N1>(S, c, m, M, t0, nv, slot_base(5), slot, warp, lane);
  __syncthreads();
  // ---- merge the warps' bests and publish one key per segment ----
  const int ns = slot_base(kMaxWinLog + 1);
  for (int i = threadIdx.x; i < ns; i += N) {
    int l = 0, base = 0;
    for (;; ++l) {
      if (!(a.win_mask & (1 << l))) continue;
      if (i < base + (kTile >> l)) break;
      base += kTile >> l;
    }
    const int s = i - base;
    const int W = 1 << l;
    const int sg = t0 / W + s;
    if ((sg + 1) * W > nv) continue;
    uint32_t bp = 0, bl = 0xffffffffu;
#pragma unroll 4
    for (int w = 0; w < N1; ++w) {
      const uint2 e = slot[i * N1 + w];
      if (e.x > bp || (e.x == bp && e.y < bl)) {
        bp = e.x;
        bl = e.y;
      }
    }
    const unsigned long long key = ((unsigned long long)bp << 32) | (unsigned long long)(0xffffffffu - bl);
    int woff = 0;  // a.win_off[l] without a dynamic index into the parameter block
#pragma unroll
    for (int i = 0; i <= kMaxWinLog; ++i)
      if (i == l) woff = a.win_off[i];
    atomicMax(a.keys + ((size_t)b * a.n_dm + d) * a.seg_per_bd + woff + sg, key);
  }
}

template <int N1, int PADR, int FOLD>
static cudaError_t launch_search_t(const SearchArgs& a, cudaStream_t s, int* n_launch) {
  constexpr int N = 32 * N1;
  const size_t smem = (size_t)32 * (N + 1) * sizeof(float2) + (size_t)kMaxSegPerTile * N1 * sizeof(uint2);
  cudaError_t e = cudaFuncSetAttribute(search_kernel<N1, PADR, FOLD>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long per_b = (long long)a.n_tiles * a.n_dm * a.pad_delay * FOLD;
  const long long max_grid = 2147483647LL;
  const int b_chunk = (int)std::max(1LL, std::min((long long)a.n_bl, max_grid / std::max(1LL, per_b)));
  for (int b0 = 0; b0 < a.n_bl; b0 += b_chunk) {
    const int nb = std::min(b_chunk, a.n_bl - b0);
    search_kernel<N1, PADR, FOLD><<<(unsigned)(per_b * nb), N, smem, s>>>(a, b0);
    ++*n_launch;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Work split of the delay transform by band size: N = n_f / FOLD points
// per residue FFT, one thread per point.  n_f = 512 runs as one 512-thread
// CTA per SM (a.fold = 1); a.fold = 2 selects two folded 256-thread CTAs
// (each gathers twice the input per thread; slower on B300).
template <int PADR>
static cudaError_t launch_search_p(const SearchArgs& a, cudaStream_t s, int* n_launch) {
  switch (a.n_f) {
    case 64: return launch_search_t<2, PADR, 1>(a, s, n_launch);
    case 128: return launch_search_t<4, PADR, 1>(a, s, n_launch);
    case 256: return launch_search_t<8, PADR, 1>(a, s, n_launch);
    case 512:
      return a.fold == 2 ? launch_search_t<8, PADR, 2>(a, s, n_launch)
                         : launch_search_t<16, PADR, 1>(a, s, n_launch);
    case 1024: return launch_search_t<8, PADR, 4>(a, s, n_launch);
    case 2048: return launch_search_t<8, PADR, 8>(a, s, n_launch);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_search(const SearchArgs& a, int pad_rate, cudaStream_t s, int* n_launch) {
  switch (pad_rate) {
    case 0: return launch_search_p<0>(a, s, n_launch);
    case 4: return launch_search_p<4>(a, s, n_launch);
    default: return cudaErrorInvalidValue;
  }
}

// ============================================================ select ====
// z-score of one segment, with round-to-nearest intrinsics so that the
// select and match kernels compute bit-identical values.
__device__ __forceinline__ double seg_rho(unsigned long long key, int W, int n_eff) {
  const float P = __uint_as_float((uint32_t)(key >> 32));
  return __ddiv_rn((double)P, (double)(W * n_eff));
}
__device__ __forceinline__ double seg_z(double rho, double mu, double sd) {
  return sd > 0.0 ? __ddiv_rn(__dsub_rn(rho, mu), sd) : 0.0;
}

template <int NT>
__device__ __forceinline__ double block_sum(double v, double* red) {
  red[threadIdx.x] = v;
  __syncthreads();
#pragma unroll
  for (int h = NT / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  const double r = red[0];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(256) select_kernel(const SelectArgs a) {
  constexpr int NT = 256;
  __shared__ double red[NT];
  long long bid = blockIdx.x;
  const int wi = (int)(bid % a.n_win);
  bid /= a.n_win;
  const int d = (int)(bid % a.n_dm);
  const int b = (int)(bid / a.n_dm);
  const int W = 1 << a.win_log[wi];
  const int nseg = max(a.nvalid[d], 0) / W;
  const size_t bd = (size_t)b * a.n_dm + d;
  const unsigned long long* k = a.keys + bd * a.seg_per_bd + a.win_off[wi];
  double s = 0.0;
  for (int i = threadIdx.x; i < nseg; i += NT) s += seg_rho(k[i], W, a.n_eff);
  const double mu = nseg > 0 ? block_sum<NT>(s, red) / (double)nseg : 0.0;
  double ss = 0.0;
  for (int i = threadIdx.x; i < nseg; i += NT) {
    const double dv = seg_rho(k[i], W, a.n_eff) - mu;
    ss = fma(dv, dv, ss);
  }
  const double sd = nseg > 0 ? sqrt(block_sum<NT>(ss, red) / (double)nseg) : 0.0;
  if (threadIdx.x == 0) {
    a.stats[(bd * a.n_win + wi) * 2 + 0] = mu;
    a.stats[(bd * a.n_win + wi) * 2 + 1] = sd;
  }
  uint32_t* bits = a.bits + bd * a.word_per_bd + a.word_off[wi];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int base = warp * 32; base < nseg; base += NT) {
    const int i = base + lane;
    const bool sel = i < nseg && seg_z(seg_rho(k[i], W, a.n_eff), mu, sd) >= a.thresh;
    const uint32_t w = __ballot_sync(0xffffffffu, sel);
    if (lane == 0) bits[base / 32] = w;
  }
}

cudaError_t launch_select(const SelectArgs& a, cudaStream_t s, int* n_launch) {
  const long long n = (long long)a.n_bl * a.n_dm * a.n_win;
  if (n == 0) return cudaSuccess;
  select_kernel<<<(unsigned)n, 256, 0, s>>>(a);
  ++*n_launch;
  return cudaGetLastError();
}

// ============================================================= match ====
// One thread per (baseline, DM): merge the selected segments of all windows
// in order of start AP and sweep overlap groups.
__global__ void __launch_bounds__(128) match_kernel(const MatchArgs a) {
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (long long)a.n_bl * a.n_dm) return;
  const int d = (int)(id % a.n_dm), b = (int)(id / a.n_dm);
  const int nv = max(a.nvalid[d], 0);
  const size_t bd = (size_t)b * a.n_dm + d;
  const uint32_t* bits = a.bits + bd * a.word_per_bd;
  const unsigned long long* keys = a.keys + bd * a.seg_per_bd;
  uint32_t cur[kMaxWinLog + 1];
  int wordi[kMaxWinLog + 1], nwords[kMaxWinLog + 1];
  for (int wi = 0; wi < a.n_win; ++wi) {
    const int nseg = nv >> a.win_log[wi];
    nwords[wi] = (nseg + 31) / 32;
    wordi[wi] = 0;
    cur[wi] = nwords[wi] > 0 ? bits[a.word_off[wi]] : 0u;
  }
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
        c.dm_idx = d;
        c.win_log = a.win_log[rw];
        c.seg = rs;
        c.g0 = g0;
        c.g1 = g1;
        c.n_windows = __popc(mask);
        c.lin = 0xffffffffu - (uint32_t)(rkey & 0xffffffffu);
        c.P = __uint_as_float((uint32_t)(rkey >> 32));
        c._pad = 0.f;
        c.rho = rrho;
        c.z = rz;
        a.out[o] = c;
      }
    }
  };
  for (;;) {
    int bw = -1, bstart = 0x7fffffff, bsg = 0;
    for (int wi = 0; wi < a.n_win; ++wi) {
      while (cur[wi] == 0u && wordi[wi] + 1 < nwords[wi]) {
        ++wordi[wi];
        cur[wi] = bits[a.word_off[wi] + wordi[wi]];
      }
      if (cur[wi] != 0u) {
        const int sg = wordi[wi] * 32 + __ffs(cur[wi]) - 1;
        const int st = sg << a.win_log[wi];
        if (st < bstart) {
          bstart = st;
          bw = wi;
          bsg = sg;
        }
      }
    }
    if (bw < 0) break;
    cur[bw] &= cur[bw] - 1u;
    const int W = 1 << a.win_log[bw];
    const int end = bstart + W;
    const unsigned long long key = keys[a.win_off[bw] + bsg];
    const double rho = seg_rho(key, W, a.n_eff);
    const double* st = a.stats + (bd * a.n_win + bw) * 2;
    const double z = seg_z(rho, st[0], st[1]);
    if (mask != 0 && bstart < g1) {
      g1 = max(g1, end);
      mask |= 1 << bw;
      const int RW = 1 << a.win_log[rw];
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

cudaError_t launch_match(const MatchArgs& a, cudaStream_t s, int* n_launch) {
  const long long n = (long long)a.n_bl * a.n_dm;
  if (n == 0) return cudaSuccess;
  match_kernel<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(a);
  ++*n_launch;
  return cudaGetLastError();
}

}  // namespace vk
