// Device code shared by the FP32 search kernel (volks_kernels.cu) and the
// tensor-core search kernel (volks_mma.cu): work-unit decoding, the fused
// dedispersed gather + zero-padded delay FFT of one 32-AP tile (stages 0-2),
// the FP32 rate transform of one window and the arg-max helpers.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "fft_regs.cuh"
#include "volks_internal.h"

namespace vk {

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

// |Z_q|^2 of the 8 rate cells of a 2-AP segment (R = 8) in closed form:
// |y0 + y1 W_8^q|^2 = r0 + 2 Re(r1 W_8^q), r0 = |y0|^2 + |y1|^2,
// r1 = y1 conj(y0): the power spectrum is the DFT of the lag products.
__device__ __forceinline__ void rate_cells_w2(float2 y0, float2 y1, float (&P)[8]) {
  const float r0 = fmaf(y1.y, y1.y, fmaf(y1.x, y1.x, cabs2(y0)));
  const float rx = fmaf(y1.y, y0.y, y1.x * y0.x);
  const float ry = fmaf(y1.y, y0.x, -(y1.x * y0.y));
  constexpr float kS2 = Tw<8, 1>::re * 2.0f;   // sqrt(2)
  const float a = rx + rx, bb = ry + ry;
  const float cc = kS2 * (rx + ry), dd = kS2 * (ry - rx);
  P[0] = r0 + a;
  P[1] = r0 + cc;
  P[2] = r0 + bb;
  P[3] = r0 + dd;
  P[4] = r0 - a;
  P[5] = r0 - cc;
  P[6] = r0 - bb;
  P[7] = r0 - dd;
}

// Rate transform, |Z|^2 and arg-max of every window-W segment of the tile
// for the delay column this thread owns.  Per segment the warp's best
// (power, lowest linear cell) goes to slot[(slot0 + s) * N1 + warp].
template <int W, int PADR, int N1, bool SLIDE = false>
__device__ __forceinline__ void rate_window(const float2* __restrict__ S, int c, uint32_t m,
                                            uint32_t M, int t0, int nv, int slot0,
                                            uint2* slot, int warp, int lane) {
  constexpr int N = 32 * N1, LD = N + 1;
  constexpr int NSEG = kTile / W;
  constexpr int R = (W == 1 || PADR == 0) ? 1 : PADR * W;
  // the tile's segments that end within the nv valid APs (a sliding unit's
  // t0 need not be a multiple of W)
  const int nseg = SLIDE ? min(NSEG, max(0, nv - t0) / W) : min(NSEG, max(0, nv / W - t0 / W));
#pragma unroll 1
  for (int s = 0; s < nseg; ++s) {
    const float2* col = S + (s * W) * LD + c;
    float best;
    uint32_t bq;
    if constexpr (R == 1) {
      float2 z = col[0];
      static_for<1, W>([&](auto u) { z = cadd_t<true>(z, col[decltype(u)::value * LD]); });
      best = cabs2(z);
      bq = 0;
    } else if constexpr (W == 2 && R == 8) {
      float P[8];
      rate_cells_w2(col[0], col[LD], P);
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

// The 2-AP window of the 2-D search (R = 8) with one warp per segment:
// each lane walks N1 delay columns (c = lane + 32 j) keeping the column with
// the largest cell, whose power is r0 + max(|2 rx|, |2 ry|, |sqrt2 (rx +
// ry)|, |sqrt2 (ry - rx)|) -- the same FP32 expressions as rate_cells_w2, so
// by monotonic rounding it equals the largest of the column's eight cells --
// and resolves that column's rate cell once (lowest q on ties; equal powers
// in one lane keep the lower column).  The warp's best goes to the
// segment's first slot, the other N1 - 1 slots get an entry that never wins.
template <int N1, bool SLIDE>
__device__ __forceinline__ void rate_window_w2_seg(const float2* __restrict__ S, uint32_t M, int Pd, int r,
                                                   int t0, int nv, int slot0, uint2* slot, int warp, int lane) {
  constexpr int N = 32 * N1, LD = N + 1, W = 2, NSEG = kTile / W;
  const int nseg = SLIDE ? min(NSEG, max(0, nv - t0) / W) : min(NSEG, max(0, nv / W - t0 / W));
#pragma unroll 1
  for (int s = warp; s < nseg; s += N1) {
    const float2* y0p = S + (2 * s) * LD;
    const float2* y1p = y0p + LD;
    float bp = -1.f;
    int bc = lane;
#pragma unroll 4
    for (int jj = 0; jj < N1; ++jj) {
      const int c = lane + 32 * jj;
      const float2 y0 = y0p[c], y1 = y1p[c];
      const float r0 = fmaf(y1.y, y1.y, fmaf(y1.x, y1.x, cabs2(y0)));
      const float rx = fmaf(y1.y, y0.y, y1.x * y0.x);
      const float ry = fmaf(y1.y, y0.x, -(y1.x * y0.y));
      constexpr float kS2 = Tw<8, 1>::re * 2.0f;
      const float a = rx + rx, bb = ry + ry;
      const float cc = kS2 * (rx + ry), dd = kS2 * (ry - rx);
      const float pm = r0 + fmaxf(fmaxf(fabsf(a), fabsf(bb)), fmaxf(fabsf(cc), fabsf(dd)));
      if (pm > bp) {
        bp = pm;
        bc = c;
      }
    }
    float P8[8];
    rate_cells_w2(y0p[bc], y1p[bc], P8);
    float pv;
    uint32_t qv;
    argmax_tree<0, 8>([&](auto qq) { return P8[decltype(qq)::value]; }, pv, qv);
    const uint32_t lin = qv * M + (uint32_t)(bc * Pd + r);
    const uint32_t pb = __float_as_uint(pv);
    const uint32_t wmax = __reduce_max_sync(0xffffffffu, pb);
    const uint32_t wlin = __reduce_min_sync(0xffffffffu, pb == wmax ? lin : 0xffffffffu);
    if (lane < N1) slot[(slot0 + s) * N1 + lane] = lane == 0 ? make_uint2(wmax, wlin) : make_uint2(0u, 0xffffffffu);
  }
}

// Range holding work unit u (ranges are in increasing `base` order).
__device__ __forceinline__ int find_desc(const Batch& p, long long u) {
  int lo = 0, hi = p.n_desc - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (p.d[mid].base <= u) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Per-unit state in shared memory: the range descriptor and the decoded
// unit.  Fields are re-read from here after each barrier instead of being
// kept live in registers through the FFT stages.
struct UnitState {
  SegDesc a;
  int b, d, r, t0, nv, valid;
};

// Segment of slot i of a tile (slots of the searched windows in ascending
// window order): its window log2 l and its index sg in the (b, DM, window)
// series, or false if the segment is not complete within the nv valid APs.
template <bool SLIDE>
__device__ __forceinline__ bool slot_segment(int i, int win_mask, int desc_mask, int t0, int nv, int& l, int& sg) {
  int base = 0;
  for (l = 0;; ++l) {
    if (!(win_mask & (1 << l))) continue;
    if (i < base + (kTile >> l)) break;
    base += kTile >> l;
  }
  const int s = i - base;
  const int W = 1 << l;
  if constexpr (SLIDE) {
    const int start = t0 + s * W;
    if (start + W > nv) return false;
    sg = desc_slide(desc_mask) ? start : start >> l;
  } else {
    sg = t0 / W + s;
    if ((sg + 1) * W > nv) return false;
  }
  return true;
}

// Store the tile's final keys (largest over its delay residues) once.
template <bool SLIDE>
__device__ __forceinline__ void store_keys(const UnitState& us, const unsigned long long* run, int win_mask) {
  int ns = 0;
  for (int l = 0; l <= kMaxWinLog; ++l)
    if (win_mask & (1 << l)) ns += kTile >> l;
  unsigned long long* keys = us.a.keys + ((size_t)us.b * us.a.n_dm + us.d) * us.a.seg_per_bd;
  for (int i = threadIdx.x; i < ns; i += blockDim.x) {
    int l, sg;
    if (slot_segment<SLIDE>(i, win_mask, us.a.win_mask, us.t0, us.nv, l, sg)) keys[us.a.win_off_l[l] + sg] = run[i];
  }
}


// max of three floats in one instruction (NaN operands are ignored, as by
// fmaxf)
__device__ __forceinline__ float fmax3_f(float a, float b, float c) {
  float d;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}

// 8-byte asynchronous copy global -> shared (L1-cached); src_bytes 0
// fills the destination with zeros and reads nothing.
__device__ __forceinline__ void cp_async8(void* dst, const void* src, int src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
               "l"(__cvta_generic_to_global(src)), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// One pass of a work unit (baseline b, DM trial d, 32-AP tile) per delay
// residue r.
// Zero padding by pad_delay, with the band folded FOLD times, splits the
// M-point delay transform (M = pad_delay * n_f) into P = pad_delay * FOLD
// independent N-point FFTs, N = n_f / FOLD:
//   Y[P c + r] = sum_{k<N} W_M^{k r} (sum_{f<FOLD} X[k + N f] W_P^{f r}) W_N^{k c},
// so a unit computes the delay cells m = P c + r (c < N) of its residue r.
// N = 32 * N1 (N1 a power of two, or 3 times one for bands of 3 * 2^a
// points); the CTA has N threads.
//   stage 0  lane = AP, warp owns k0 = warp*KPW + j: gather xn[k][t + shift_k],
//            fold and pre-twiddle
//   stage 1  N1-point FFTs over k1 (k = k0 + 32 k1), twiddle W_N^{k0 m1}
//   stage 2  lane = AP, warp = m1: 32-point FFT over k0 -> Y[m1 + N1 m2]
// delay_stage runs stages 0-2 and leaves Y[t][m1 + N1 m2] (row pitch N + 1)
// in S; the rate stage (FP32 register FFTs or the tensor-core GEMM) follows.
// Called by every thread of the CTA after `us` has been filled and
// synchronised; returns after a barrier, with Y complete in S.  With AMAX,
// the largest |Re| or |Im| of Y is also folded into *amax (an FP32 bit
// pattern; non-negative floats order like their bits).
template <int N1, int FOLD, bool PK = true, bool PK2 = PK, bool AMAX = false>
__device__ __forceinline__ void delay_stage(const UnitState& us, float2* S, unsigned int* amax = nullptr) {
  constexpr int N = 32 * N1;
  // N1 a power of two (radix-2 register FFTs, each warp owns 32 / N1
  // consecutive k0) or 3 times one (mixed-radix FFTs, k0 = warp + N1 j)
  constexpr bool kPow2 = (N1 & (N1 - 1)) == 0;
  constexpr int KPW = (32 + N1 - 1) / N1;
  constexpr int LD = N + 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // ---- stage 0 + 1 ----
  {
    const SegDesc& a = us.a;
    const int b = us.b, d = us.d, r = us.r, nv = us.nv;
    const int n_ap = a.n_ap, n_f = a.n_f, Mm = a.M;
    const float2* xb = a.xn + (size_t)b * n_f * n_ap;
    const int32_t* sh = a.shifts + (size_t)d * n_f;
    const float2* tw_m = a.tw_m;
    const float2* tw_n = a.tw_n;
    const int t = us.t0 + lane;
    const bool tin = t < nv;
    float2 wf[FOLD];  // W_P^{f r} = W_M^{N f r}
    static_for<0, FOLD>([&](auto ff) {
      constexpr int F = decltype(ff)::value;
      wf[F] = F == 0 ? make_float2(1.f, 0.f) : __ldg(tw_m + (N * F * r) % Mm);
    });
    // Folded bands (FOLD > 1) read FOLD N-point sections per residue, more
    // than the L1 keeps between residues: the first section of every k0
    // this warp owns goes to S by asynchronous copies, all in flight at
    // once and into the very slots S[t][k0 N1 + m1] that this thread later
    // overwrites with its stage-1 outputs, so no other thread touches them
    // (one copy group per k0); for FOLD = 2 section 1 is loaded while they
    // land (with more sections that measured slower).
    // Unfolded bands load directly: the copies measured slower there.
    if constexpr (FOLD > 1) static_for<0, KPW>([&](auto jj) {
      constexpr int J = decltype(jj)::value;
      const int k0 = kPow2 ? warp * KPW + J : warp + N1 * J;
      if (kPow2 || k0 < 32) {
        static_for<0, N1>([&](auto kk1) {
          constexpr int K1 = decltype(kk1)::value;
          const int kf = k0 + 32 * K1;
          const float2* src = tin ? xb + (size_t)kf * n_ap + t + __ldg(sh + kf) : xb;
          cp_async8(S + lane * LD + k0 * N1 + K1, src, tin ? 8 : 0);
        });
      }
      cp_async_commit();
    });
    static_for<0, KPW>([&](auto jj) {
      constexpr int J = decltype(jj)::value;
      const int k0 = kPow2 ? warp * KPW + J : warp + N1 * J;
      if (!kPow2 && k0 >= 32) return;
      // fold passes F >= 1 add the band's F-th N-point section (N1
      // independent loads per pass), summed in the order F = 1, 2, ..
      float2 x[N1];
      if constexpr (FOLD == 2) {
        // section 1 is loaded before waiting for the copies of section 0
        float2 u1[N1];
        static_for<0, N1>([&](auto kk1) {
          constexpr int K1 = decltype(kk1)::value;
          const int kf = k0 + 32 * K1 + N;
          u1[K1] = make_float2(0.f, 0.f);
          if (tin) u1[K1] = __ldg(xb + (size_t)kf * n_ap + t + __ldg(sh + kf));
        });
        cp_async_wait<KPW - 1 - J>();
        static_for<0, N1>([&](auto kk1) {
          constexpr int K1 = decltype(kk1)::value;
          x[K1] = cadd_t<PK>(S[lane * LD + k0 * N1 + K1], cmul(u1[K1], wf[1]));
        });
      } else if constexpr (FOLD > 2) {
        cp_async_wait<KPW - 1 - J>();
        static_for<0, N1>([&](auto kk1) {
          constexpr int K1 = decltype(kk1)::value;
          x[K1] = S[lane * LD + k0 * N1 + K1];
        });
      } else {
        static_for<0, N1>([&](auto kk1) {
          constexpr int K1 = decltype(kk1)::value;
          const int kf = k0 + 32 * K1;
          x[K1] = make_float2(0.f, 0.f);
          if (tin) x[K1] = __ldg(xb + (size_t)kf * n_ap + t + __ldg(sh + kf));
        });
      }
      static_for<FOLD == 2 ? 2 : 1, FOLD>([&](auto ff) {
        constexpr int F = decltype(ff)::value;
        static_for<0, N1>([&](auto kk1) {
          constexpr int K1 = decltype(kk1)::value;
          const int kf = k0 + 32 * K1 + N * F;
          float2 u = make_float2(0.f, 0.f);
          if (tin) u = __ldg(xb + (size_t)kf * n_ap + t + __ldg(sh + kf));
          x[K1] = cadd_t<PK>(x[K1], cmul(u, wf[F]));
        });
      });
      if (r != 0) {
        static_for<0, N1>([&](auto kk1) {
          constexpr int K1 = decltype(kk1)::value;
          x[K1] = cmul(x[K1], __ldg(tw_m + (k0 + 32 * K1) * r));  // k < N, r < P: k r < M
        });
      }
      if constexpr (kPow2) {
        fft_dif<N1, PK>(x);
      } else {
        fft3_nat<N1>(x);
      }
      static_for<0, N1>([&](auto mm1) {
        constexpr int M1 = decltype(mm1)::value;
        float2 v = x[kPow2 ? bitrev(M1, ilog2(N1)) : M1];
        // W_N^{k0 m1} = W_{n_f}^{k0 m1 FOLD}
        if constexpr (M1 != 0) v = cmul(v, __ldg(tw_n + k0 * M1 * FOLD));  // < 32 N1 FOLD = n_f
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
    fft_dif<32, PK2>(y);
    __syncthreads();
    static_for<0, 32>([&](auto mm2) {
      constexpr int M2 = decltype(mm2)::value;
      S[lane * LD + warp + N1 * M2] = y[bitrev(M2, 5)];
    });
    if constexpr (AMAX) {
      // four independent chains of 3-input maxima (one serial chain of 64
      // maxima measured ~4 % of the tensor-core kernel's time)
      float m[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int i = 0; i < 32; ++i) m[i & 3] = fmax3_f(m[i & 3], fabsf(y[i].x), fabsf(y[i].y));
      const float mm = fmaxf(fmaxf(m[0], m[1]), fmaxf(m[2], m[3]));
      const uint32_t wm = __reduce_max_sync(0xffffffffu, __float_as_uint(mm));
      if (lane == 0) atomicMax(amax, wm);
    }
  }
  __syncthreads();
}

}  // namespace vk
