// Reduced-precision search kernel (a4-a7) for sm_103a: the fringe-rate
// transform of the 4..32-AP windows runs as a DFT-matrix GEMM on the
// tcgen05 tensor cores (BF16, FP16 or FP8 E4M3 operands, FP32 accumulation
// in tensor memory), followed by an FP32 re-evaluation of the best delay
// columns of every segment.
//
// Per work unit (baseline, DM trial, 32-AP tile, delay residue r):
//   delay   stages 0-2 of the FP32 kernel (shared code): FP32 delay
//           spectrum Y[t][c] of the tile's 32 APs x N = 32 N1 delay cells
//           in shared memory S.
//   w=1,2   exact FP32 windows on the CUDA cores, one warp per segment,
//           while the first GEMMs run.
//   GEMM    per M-block of 128 delay cells: A = Y^T rounded to the operand
//           type (rows = delay cells, K = 32 APs x (re, im)); per window w,
//           B = the real embedding of the R = 4w point rate DFT of each
//           segment, so D[c][2q + {0,1}] = (Re, Im) Z_w[s, q, c]
//           (Sec. 2.2 2-D search; Sec. 2.4.2 step 6 window combine).  Two
//           256-column TMEM buffers: the epilogue of one (M-block, window)
//           job overlaps the MMAs of the next.
//   coarse  epilogue: per (segment, delay cell) the largest coarse |Z|^2
//           over the segment's rate cells; a warp per segment keeps the
//           8 delay cells with the largest coarse values (ties: lower cell).
//   refine  the 8 retained delay cells of every segment are re-evaluated in
//           FP32 from S (all R rate cells of each: pre-twiddled w-point
//           register FFTs, as the FP32 kernel computes them); the segment's
//           peak is the largest refined power, ties to the lowest q M + m.
//   publish one 64-bit atomicMax per segment, as the FP32 kernel.
//
// Reported peaks are therefore FP32 evaluations of real grid cells; they
// equal the FP32 search whenever its peak cell lies in one of the 8 delay
// cells the coarse pass ranks highest for that segment.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "../../include/volks.h"
#include "fft_regs.cuh"
#include "search_common.cuh"
#include "tcgen05.cuh"
#include "volks_internal.h"

namespace vk {

namespace {

constexpr int kMRows = 128;          // MMA M: delay cells per M-block
constexpr int kJobCols = 256;        // TMEM columns of one (M-block, window) job
constexpr int kTmemCols = 512;       // two job buffers
constexpr int kGemmSegs = 15;        // segments of windows 4, 8, 16, 32 in a tile
constexpr int kTopK = 8;             // delay cells refined per segment
constexpr long long kWaitCycles = 4000000000LL;  // ~2 s at 2 GHz

template <int PREC>
struct Op {
  static constexpr int EB = PREC == VOLKS_FP8 ? 1 : 2;      // bytes per element
  static constexpr uint32_t SBO_A = 512u * EB;              // 8-row group of A
  static constexpr uint32_t A_BYTES = 16u * SBO_A;          // 128 rows x 64 K
  // per window l = 2..5: segments per MMA, rows (MMA N), K bytes per row
  static constexpr int seg_per_mma(int l) { return (2 << l) * EB >= 32 ? 1 : 32 / ((2 << l) * EB); }
  static constexpr int b_rows(int l) { return (8 << l) * seg_per_mma(l); }
  static constexpr int b_row_bytes(int l) { return (2 << l) * EB >= 32 ? (2 << l) * EB : 32; }
  static constexpr int b_bytes(int l) { return b_rows(l) * b_row_bytes(l); }
  static constexpr int b_off(int l) {
    int o = 0;
    for (int i = 2; i < l; ++i) o += b_bytes(i);
    return o;
  }
  static constexpr int B_BYTES = b_off(6);
  // operand scale target for the per-tile power-of-two scaling
  static constexpr int SCALE_EXP = PREC == VOLKS_FP8 ? 8 : 14;
};

template <int N1, int PREC>
struct MmaSmem {
  static constexpr int N = 32 * N1;
  static constexpr size_t S_BYTES = (size_t)32 * (N + 1) * sizeof(float2);
  static constexpr size_t OFF_A = (S_BYTES + 1023) & ~(size_t)1023;
  static constexpr size_t OFF_B = OFF_A + 2 * Op<PREC>::A_BYTES;
  static constexpr size_t OFF_COL = OFF_B + Op<PREC>::B_BYTES;                // u32 [15][128]
  static constexpr size_t OFF_TOP = OFF_COL + (size_t)kGemmSegs * kMRows * 4;  // uint2 [15][8]
  static constexpr size_t OFF_BEST = OFF_TOP + (size_t)kGemmSegs * kTopK * 8;  // u64 [63]
  static constexpr size_t USED = OFF_BEST + (size_t)kMaxSegPerTile * 8;
  // more than half an SM's shared memory: one CTA per SM, so the 512-column
  // TMEM allocation never waits on another CTA
  static constexpr size_t BYTES = USED > 120 * 1024 ? USED : 120 * 1024;
};

__device__ __forceinline__ uint32_t pack2(float a, float b, std::integral_constant<int, VOLKS_BF16>) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}
__device__ __forceinline__ uint32_t pack2(float a, float b, std::integral_constant<int, VOLKS_FP16>) {
  __half2 h = __floats2half2_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}
// two E4M3 values, a in the low byte
__device__ __forceinline__ uint32_t e4m3x2(float a, float b) {
  uint16_t r;
  asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(r) : "f"(b), "f"(a));
  return r;
}

// Rate-DFT operand B of window 2^l (rows n = MMA N, K-major, interleaved
// layout), from the FP32 twiddle table W_M^i: row 2q of a segment block
// holds (cos, sin) and row 2q + 1 (-sin, cos) of 2 pi q u / R against
// (Re, Im) of AP u, so that D = A B^T gives (Re, Im) of
// Z_q = sum_u Y_u exp(-2 pi i q u / R), R = 4w.  Segments sharing one MMA
// (K of a segment shorter than one MMA) get a block-diagonal B.
template <int PREC>
__device__ void build_rate_dft(uint8_t* B, const float2* __restrict__ tw_m, int M, int tid, int nt) {
  using O = Op<PREC>;
  constexpr int EB = O::EB;
#pragma unroll 1
  for (int l = 2; l <= 5; ++l) {
    const int w = 1 << l, R = 4 * w;
    const int rows = O::b_rows(l), kel = O::b_row_bytes(l) / EB;
    const uint32_t sbo = 8u * O::b_row_bytes(l);
    uint8_t* base = B + O::b_off(l);
#pragma unroll 1
    for (int i = tid; i < rows * kel; i += nt) {
      const int n = i / kel, k = i % kel;
      const int hn = n / (8 * w), nn = n % (8 * w), hk = k / (2 * w), kk = k % (2 * w);
      float v = 0.f;
      if (hn == hk) {
        const int q = nn >> 1, comp = nn & 1, u = kk >> 1, part = kk & 1;
        const float2 t = __ldg(tw_m + ((q * u) % R) * (M / R));  // (cos, -sin)
        v = comp == 0 ? (part == 0 ? t.x : -t.y) : (part == 0 ? t.y : t.x);
      }
      const uint32_t off = (uint32_t)(n >> 3) * sbo + (uint32_t)((k * EB) >> 4) * 128u +
                           (uint32_t)(n & 7) * 16u + (uint32_t)((k * EB) & 15);
      if constexpr (PREC == VOLKS_FP8) {
        base[off] = (uint8_t)(e4m3x2(v, 0.f) & 0xffu);
      } else if constexpr (PREC == VOLKS_BF16) {
        *reinterpret_cast<__nv_bfloat16*>(base + off) = __float2bfloat16_rn(v);
      } else {
        *reinterpret_cast<__half*>(base + off) = __float2half_rn(v);
      }
    }
  }
}

// A operand of M-block b: rows = delay cells 128 b + row, K = (Re, Im) of
// the 32 APs, scaled by `scale` and rounded to the operand type.
template <int LD, int PREC>
__device__ __forceinline__ void pack_a(const float2* __restrict__ S, uint8_t* A, int b, float scale, int tid,
                                       int nt) {
  using O = Op<PREC>;
  constexpr int APC = 8 / O::EB;  // APs per 16-byte chunk
  constexpr int CH = 32 / APC;    // chunks per row
#pragma unroll 1
  for (int i = tid; i < kMRows * CH; i += nt) {
    const int row = i & (kMRows - 1), ch = i >> 7;
    const float2* src = S + (ch * APC) * LD + b * kMRows + row;
    uint32_t wv[4];
    if constexpr (PREC == VOLKS_FP8) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float2 v0 = src[(2 * j) * LD], v1 = src[(2 * j + 1) * LD];
        wv[j] = e4m3x2(v0.x * scale, v0.y * scale) | (e4m3x2(v1.x * scale, v1.y * scale) << 16);
      }
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float2 v = src[j * LD];
        wv[j] = pack2(v.x * scale, v.y * scale, std::integral_constant<int, PREC>{});
      }
    }
    const uint32_t off = (uint32_t)(row >> 3) * O::SBO_A + (uint32_t)ch * 128u + (uint32_t)(row & 7) * 16u;
    *reinterpret_cast<uint4*>(A + off) = make_uint4(wv[0], wv[1], wv[2], wv[3]);
  }
}

// Issue the MMAs of window 2^l for one M-block into TMEM columns d .. d+255
// (column 8 w s + 2 q + {0,1} = (Re, Im) of rate cell q of segment s).
template <int PREC>
__device__ __forceinline__ void issue_window(int l, uint32_t a_base, uint32_t b_base, uint32_t d) {
  using O = Op<PREC>;
  constexpr int EB = O::EB;
  const int w = 1 << l;
  const int seg_kb = 2 * w * EB;  // K bytes of one segment; one MMA consumes 32
  const uint32_t sbo_b = 8u * (uint32_t)O::b_row_bytes(l);
  if (seg_kb >= 32) {
    const int nseg = 32 / w, n = 8 * w, ks = seg_kb / 32;
    const uint32_t idesc = PREC == VOLKS_FP8 ? tc::idesc_e4m3(n) : tc::idesc_f16(n, PREC == VOLKS_BF16);
    for (int s = 0; s < nseg; ++s)
      for (int k = 0; k < ks; ++k) {
        const uint64_t ad = tc::sdesc(a_base + (uint32_t)(16 * w * EB * s + 256 * k), 128u, O::SBO_A);
        const uint64_t bd = tc::sdesc(b_base + (uint32_t)(256 * k), 128u, sbo_b);
        if constexpr (PREC == VOLKS_FP8) tc::mma_f8(d + (uint32_t)(n * s), ad, bd, idesc, k > 0);
        else tc::mma_f16(d + (uint32_t)(n * s), ad, bd, idesc, k > 0);
      }
  } else {
    const int g = 32 / seg_kb, n = 8 * w * g, ngrp = (32 / w) / g;
    const uint32_t idesc = PREC == VOLKS_FP8 ? tc::idesc_e4m3(n) : tc::idesc_f16(n, PREC == VOLKS_BF16);
    for (int p = 0; p < ngrp; ++p) {
      const uint64_t ad = tc::sdesc(a_base + (uint32_t)(256 * p), 128u, O::SBO_A);
      const uint64_t bd = tc::sdesc(b_base, 128u, sbo_b);
      if constexpr (PREC == VOLKS_FP8) tc::mma_f8(d + (uint32_t)(n * p), ad, bd, idesc, false);
      else tc::mma_f16(d + (uint32_t)(n * p), ad, bd, idesc, false);
    }
  }
}

// FP32 evaluation of all R = 4W rate cells of delay column c for the
// residue class rho of q (q = 4 j + rho): pre-twiddle by W_R^{u rho},
// W-point FFT, largest |Z|^2 (ties: lowest j).
template <int W, int LD>
__device__ __forceinline__ void refine_column(const float2* __restrict__ S, int c, int u0, int rho,
                                              const float2* __restrict__ tw_m, int M, float& best,
                                              uint32_t& bq) {
  const int step = M / (4 * W);
  float2 y[W];
  static_for<0, W>([&](auto uu) {
    constexpr int U = decltype(uu)::value;
    const float2 v = S[(u0 + U) * LD + c];
    y[U] = U == 0 ? v : cmul(v, __ldg(tw_m + U * rho * step));
  });
  fft_dif<W>(y);
  uint32_t vq;
  argmax_tree<0, W>([&](auto qq) { return cabs2(y[bitrev(decltype(qq)::value, ilog2(W))]); }, best, vq);
  bq = 4u * vq + (uint32_t)rho;
}

__device__ __forceinline__ unsigned long long seg_key(uint32_t pbits, uint32_t lin) {
  return ((unsigned long long)pbits << 32) | (unsigned long long)(0xffffffffu - lin);
}

// Warp-wide (max power, lowest linear cell) -> key (all lanes).
__device__ __forceinline__ unsigned long long warp_key(float p, uint32_t lin) {
  const uint32_t pb = __float_as_uint(p);
  const uint32_t wmax = __reduce_max_sync(0xffffffffu, pb);
  const uint32_t wlin = __reduce_min_sync(0xffffffffu, pb == wmax ? lin : 0xffffffffu);
  return seg_key(wmax, wlin);
}

struct MmaCtx {
  uint32_t tmem;        // TMEM base address (512 columns)
  uint32_t phase[2];    // parity of the next completion of each job buffer
};

// One unit on the tensor-core path.  Returns false if a wait for the MMAs
// timed out (the error flag is set; the caller stops).
template <int N1, int FOLD, int PREC>
__device__ __forceinline__ bool mma_tile(const UnitState& us, uint8_t* smem, MmaCtx& cx, uint64_t* bar,
                                         float* s_amax, unsigned int* err) {
  using O = Op<PREC>;
  using L = MmaSmem<N1, PREC>;
  constexpr int N = 32 * N1, LD = N + 1, NT = N, NW = N1, NMB = N / kMRows;
  constexpr int G = NW / 4;             // warps sharing one TMEM lane quarter
  constexpr int CPT = 8 / G;            // 32-column chunks per thread per job
  float2* S = reinterpret_cast<float2*>(smem);
  uint8_t* A = smem + L::OFF_A;
  uint8_t* Bm = smem + L::OFF_B;
  uint32_t* colmax = reinterpret_cast<uint32_t*>(smem + L::OFF_COL);
  uint2* top = reinterpret_cast<uint2*>(smem + L::OFF_TOP);
  unsigned long long* best = reinterpret_cast<unsigned long long*>(smem + L::OFF_BEST);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  delay_stage<N1, FOLD>(us, S);

  const int win_mask = us.a.win_mask;
  const int t0 = us.t0, nv = us.nv, r = us.r;
  const int P = us.a.pad_delay * FOLD;
  const uint32_t M = (uint32_t)us.a.M;
  const float2* tw_m = us.a.tw_m;
  auto slot_base = [&](int l) {
    int o = 0;
    for (int i = 0; i < l; ++i)
      if (win_mask & (1 << i)) o += kTile >> i;
    return o;
  };
  auto seg_valid = [&](int l, int s) { return ((t0 >> l) + s + 1) << l <= nv; };
  // GEMM windows (4..32) present; sigma numbers their segments in
  // ascending window order
  const uint32_t gmask = (uint32_t)win_mask & 0x3cu;
  const int nG = __popc(gmask);
  auto gwin = [&](int i) { return __fns(gmask, 0, i + 1); };  // log2 of the i-th GEMM window
  auto sig_base = [&](int l) {
    int o = 0;
    for (int i = 2; i < l; ++i)
      if (gmask & (1u << i)) o += kTile >> i;
    return o;
  };
  const int nsig = sig_base(6);
  const int njobs = NMB * nG;

  float scale = 1.f;
  if (nG > 0) {
    if constexpr (PREC != VOLKS_BF16) {
      // per-tile power-of-two operand scale: largest |component| -> < 2^SCALE_EXP
      float mx = 0.f;
      for (int i = tid; i < 32 * N; i += NT) {
        const float2 v = S[(i / N) * LD + (i % N)];
        mx = tc::fmax3(mx, fabsf(v.x), fabsf(v.y));
      }
      const uint32_t wm = __reduce_max_sync(0xffffffffu, __float_as_uint(mx));
      if (lane == 0) atomicMax(reinterpret_cast<unsigned int*>(s_amax), wm);
      __syncthreads();
      const float amax = *s_amax;
      if (amax > 0.f && amax < 3.0e38f) {
        int e;
        frexpf(amax, &e);
        scale = ldexpf(1.f, max(-120, min(120, O::SCALE_EXP - e)));
      }
    }
    pack_a<LD, PREC>(S, A, 0, scale, tid, NT);
    if (NMB > 1) pack_a<LD, PREC>(S, A + O::A_BYTES, 1, scale, tid, NT);
    for (int i = tid; i < nsig * kMRows; i += NT) colmax[i] = 0u;
    for (int i = tid; i < nsig * kTopK; i += NT) top[i] = make_uint2(0u, 0xffffffffu);
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (tid == 0) {
      for (int j = 0; j < 2 && j < njobs; ++j) {
        const int b = j / nG, l = gwin(j % nG);
        issue_window<PREC>(l, tc::smem_u32(A + (b & 1) * O::A_BYTES), tc::smem_u32(Bm + O::b_off(l)),
                           cx.tmem + (uint32_t)(j & 1) * kJobCols);
        tc::mma_commit(&bar[j & 1]);
      }
    }
  }

  // ---- exact windows on the CUDA cores (overlap the first MMAs) ----
  if (win_mask & 1) {
    for (int s = warp; s < kTile; s += NW) {
      if (!seg_valid(0, s)) continue;
      float bp = -1.f;
      int bc = 0;
#pragma unroll 4
      for (int j = 0; j < N1; ++j) {
        const int c = lane + 32 * j;
        const float p = cabs2(S[s * LD + c]);
        if (p > bp) {
          bp = p;
          bc = c;
        }
      }
      const unsigned long long key = warp_key(bp, (uint32_t)(bc * P + r));
      if (lane == 0) best[slot_base(0) + s] = key;
    }
  }
  if (win_mask & 2) {
    for (int s = warp; s < kTile / 2; s += NW) {
      if (!seg_valid(1, s)) continue;
      float bp = -1.f;
      uint32_t bl = 0xffffffffu;
#pragma unroll 2
      for (int j = 0; j < N1; ++j) {
        const int c = lane + 32 * j;
        float P8[8];
        rate_cells_w2(S[(2 * s) * LD + c], S[(2 * s + 1) * LD + c], P8);
        float pv;
        uint32_t qv;
        argmax_tree<0, 8>([&](auto qq) { return P8[decltype(qq)::value]; }, pv, qv);
        const uint32_t lin = qv * M + (uint32_t)(c * P + r);
        if (pv > bp || (pv == bp && lin < bl)) {
          bp = pv;
          bl = lin;
        }
      }
      const unsigned long long key = warp_key(bp, bl);
      if (lane == 0) best[slot_base(1) + s] = key;
    }
  }

  if (nG > 0) {
    const int quarter = warp & 3, g = warp >> 2;
    const int row = quarter * 32 + lane;
#pragma unroll 1
    for (int j = 0; j < njobs; ++j) {
      const int buf = j & 1, b = j / nG, l = gwin(j % nG);
      const bool ok = tc::mbar_wait_bounded(&bar[buf], cx.phase[buf], kWaitCycles);
      cx.phase[buf] ^= 1u;
      if (__syncthreads_or(!ok)) {
        if (tid == 0) atomicOr(err, 1u);
        return false;
      }
      tc::fence_after_sync();
      // epilogue: coarse |Z|^2, max over each segment's rate cells
      const uint32_t tb = cx.tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)buf * kJobCols;
#pragma unroll 1
      for (int ch = g * CPT; ch < (g + 1) * CPT; ch += 2) {
        uint32_t v0[32], v1[32];
        tc::tmem_ld32(tb + (uint32_t)ch * 32u, v0);
        tc::tmem_ld32(tb + (uint32_t)(ch + 1) * 32u, v1);
        tc::tmem_wait_ld();
        float m0 = 0.f, m1 = 0.f;
#pragma unroll
        for (int i = 0; i < 32; i += 4) {
          const float a0 = __uint_as_float(v0[i]), a1 = __uint_as_float(v0[i + 1]);
          const float a2 = __uint_as_float(v0[i + 2]), a3 = __uint_as_float(v0[i + 3]);
          m0 = tc::fmax3(m0, fmaf(a0, a0, a1 * a1), fmaf(a2, a2, a3 * a3));
          const float c0 = __uint_as_float(v1[i]), c1 = __uint_as_float(v1[i + 1]);
          const float c2 = __uint_as_float(v1[i + 2]), c3 = __uint_as_float(v1[i + 3]);
          m1 = tc::fmax3(m1, fmaf(c0, c0, c1 * c1), fmaf(c2, c2, c3 * c3));
        }
        const int s0 = (ch * 32) >> (l + 3), s1 = ((ch + 1) * 32) >> (l + 3);
        uint32_t* cm = colmax + sig_base(l) * kMRows + row;
        if (s0 == s1) {
          atomicMax(cm + s0 * kMRows, __float_as_uint(fmaxf(m0, m1)));
        } else {
          atomicMax(cm + s0 * kMRows, __float_as_uint(m0));
          atomicMax(cm + s1 * kMRows, __float_as_uint(m1));
        }
      }
      tc::fence_before_sync();
      __syncthreads();
      if (j % nG == nG - 1) {
        // M-block b done: merge its 128 delay cells into each segment's top 8
        for (int sg = warp; sg < nsig; sg += NW) {
          uint32_t v[4], cidx[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            v[i] = colmax[sg * kMRows + lane + 32 * i];
            cidx[i] = (uint32_t)(b * kMRows + lane + 32 * i);
            colmax[sg * kMRows + lane + 32 * i] = 0u;
          }
          uint32_t v4 = 0u, c4 = 0xffffffffu;
          if (lane < kTopK) {
            const uint2 t = top[sg * kTopK + lane];
            v4 = t.x;
            c4 = t.y;
          }
          uint2 out = make_uint2(0u, 0xffffffffu);
#pragma unroll 1
          for (int rr = 0; rr < kTopK; ++rr) {
            uint32_t bv = v4, bc = c4;
            int bi = 4;
#pragma unroll
            for (int i = 0; i < 4; ++i)
              if (v[i] > bv || (v[i] == bv && cidx[i] < bc)) {
                bv = v[i];
                bc = cidx[i];
                bi = i;
              }
            const uint32_t wv = __reduce_max_sync(0xffffffffu, bv);
            const uint32_t wc = __reduce_min_sync(0xffffffffu, bv == wv ? bc : 0xffffffffu);
            if (lane == rr) out = make_uint2(wv, wc);
            if (bv == wv && bc == wc) {
#pragma unroll
              for (int i = 0; i < 4; ++i)
                if (bi == i) {
                  v[i] = 0u;
                  cidx[i] = 0xffffffffu;
                }
              if (bi == 4) {
                v4 = 0u;
                c4 = 0xffffffffu;
              }
            }
          }
          if (lane < kTopK) top[sg * kTopK + lane] = out;
        }
        if (b + 2 < NMB) {
          pack_a<LD, PREC>(S, A + (b & 1) * O::A_BYTES, b + 2, scale, tid, NT);
          tc::fence_async_smem();
        }
        __syncthreads();
      }
      tc::fence_after_sync();
      if (tid == 0 && j + 2 < njobs) {
        const int j2 = j + 2, b2 = j2 / nG, l2 = gwin(j2 % nG);
        issue_window<PREC>(l2, tc::smem_u32(A + (b2 & 1) * O::A_BYTES), tc::smem_u32(Bm + O::b_off(l2)),
                           cx.tmem + (uint32_t)buf * kJobCols);
        tc::mma_commit(&bar[buf]);
      }
    }
    // ---- FP32 refinement of the retained delay cells ----
    for (int sg = warp; sg < nsig; sg += NW) {
      int l = gwin(0);
      for (int i = 1; i < nG; ++i)
        if (sg >= sig_base(gwin(i))) l = gwin(i);
      const int s = sg - sig_base(l);
      if (!seg_valid(l, s)) continue;
      const uint2 t = top[sg * kTopK + (lane >> 2)];
      const int c = (int)t.y;
      const int rho = lane & 3;
      float pw;
      uint32_t q;
      const int u0 = s << l;
      switch (l) {
        case 2: refine_column<4, LD>(S, c, u0, rho, tw_m, (int)M, pw, q); break;
        case 3: refine_column<8, LD>(S, c, u0, rho, tw_m, (int)M, pw, q); break;
        case 4: refine_column<16, LD>(S, c, u0, rho, tw_m, (int)M, pw, q); break;
        default: refine_column<32, LD>(S, c, u0, rho, tw_m, (int)M, pw, q); break;
      }
      const unsigned long long key = warp_key(pw, q * M + (uint32_t)(c * P + r));
      if (lane == 0) best[slot_base(l) + s] = key;
    }
  }
  __syncthreads();
  // ---- publish one key per valid segment ----
  const int ns = slot_base(kMaxWinLog + 1);
  unsigned long long* keys = us.a.keys + ((size_t)us.b * us.a.n_dm + us.d) * us.a.seg_per_bd;
  for (int i = tid; i < ns; i += NT) {
    int l = 0, base = 0;
    for (;; ++l) {
      if (!(win_mask & (1 << l))) continue;
      if (i < base + (kTile >> l)) break;
      base += kTile >> l;
    }
    const int s = i - base;
    const int sg = (t0 >> l) + s;
    if ((sg + 1) << l > nv) continue;
    atomicMax(keys + us.a.win_off_l[l] + sg, best[i]);
  }
  return true;
}

// Persistent tensor-core search kernel: one CTA per SM pulls units from
// p.counter; the rate-DFT operands are built once per CTA.
template <int N1, int FOLD, int PREC>
__global__ void __launch_bounds__(32 * N1, 1) search_mma_kernel(const __grid_constant__ Batch p) {
  constexpr int N = 32 * N1;
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ UnitState us;
  __shared__ int s_desc;
  __shared__ long long s_unit;
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ uint32_t s_tmem;
  __shared__ float s_amax;
  const int tid = threadIdx.x;
  using L = MmaSmem<N1, PREC>;
  build_rate_dft<PREC>(smem + L::OFF_B, p.d[0].tw_m, p.d[0].M, tid, N);
  if (tid == 0) {
    tc::mbar_init(&bar[0], 1);
    tc::mbar_init(&bar[1], 1);
    tc::mbar_init_fence();
  }
  if ((tid >> 5) == 0) {
    tc::tmem_alloc(&s_tmem, kTmemCols);
    tc::tmem_relinquish();
  }
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  MmaCtx cx;
  cx.tmem = s_tmem;
  cx.phase[0] = cx.phase[1] = 0u;
  for (;;) {
    if (tid == 0) {
      const long long u = (long long)atomicAdd(p.counter, 1ULL);
      s_unit = u;
      s_desc = u < p.total ? find_desc(p, u) : -1;
      s_amax = 0.f;
    }
    __syncthreads();
    const int di = s_desc;
    if (di < 0) break;
    {
      const unsigned long long* src = reinterpret_cast<const unsigned long long*>(&p.d[di]);
      unsigned long long* dst = reinterpret_cast<unsigned long long*>(&us.a);
      for (int i = tid; i < (int)(sizeof(SegDesc) / 8); i += N) dst[i] = src[i];
    }
    if (tid == 0) {
      const SegDesc& a = p.d[di];
      long long unit = s_unit - a.base;
      const int P = a.pad_delay * FOLD;
      us.r = (int)(unit % P);
      unit /= P;
      us.d = (int)(unit % a.n_dm);
      unit /= a.n_dm;
      const int tile = (int)(unit % a.n_tiles);
      us.b = (int)(unit / a.n_tiles);
      us.t0 = tile * kTile;
      us.nv = a.nvalid[us.d];
      us.valid = us.t0 < us.nv;
    }
    __syncthreads();
    if (us.valid && !mma_tile<N1, FOLD, PREC>(us, smem, cx, bar, &s_amax, p.err)) break;
    __syncthreads();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if ((tid >> 5) == 0) tc::tmem_dealloc(cx.tmem, kTmemCols);
}

template <int N1, int FOLD, int PREC>
cudaError_t launch_mma_t(Batch& b, int grid_ctas, cudaStream_t s, int* n_launch) {
  const size_t smem = MmaSmem<N1, PREC>::BYTES;
  static_assert(MmaSmem<N1, PREC>::BYTES <= 227 * 1024, "shared memory");
  cudaError_t e = cudaFuncSetAttribute(search_mma_kernel<N1, FOLD, PREC>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (b.total <= 0) return cudaSuccess;
  if (!b.counter || !b.err) return cudaErrorInvalidValue;
  b.unit0 = 0;
  search_mma_kernel<N1, FOLD, PREC><<<(unsigned)std::max(1, grid_ctas), 32 * N1, smem, s>>>(b);
  ++*n_launch;
  return cudaGetLastError();
}

// ------------------------------------------------------------- checking --
// One M-block of one window through the same operand builders and MMA
// issue as the search kernel; dumps the job's 256 TMEM columns.
template <int PREC>
__global__ void __launch_bounds__(128, 1) rate_gemm_probe_kernel(const float2* __restrict__ y,
                                                                  const float2* __restrict__ tw_m, int M,
                                                                  int l, int skip_mma, long long wait_cycles,
                                                                  float* __restrict__ out, unsigned int* err) {
  constexpr int LD = kMRows + 1;
  extern __shared__ __align__(1024) uint8_t smem[];
  using O = Op<PREC>;
  constexpr size_t OFF_A = ((size_t)32 * LD * sizeof(float2) + 1023) & ~(size_t)1023;
  constexpr size_t OFF_B = OFF_A + O::A_BYTES;
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t s_tmem;
  float2* S = reinterpret_cast<float2*>(smem);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int i = tid; i < 32 * kMRows; i += 128) S[(i / kMRows) * LD + (i % kMRows)] = y[i];
  __syncthreads();
  build_rate_dft<PREC>(smem + OFF_B, tw_m, M, tid, 128);
  pack_a<LD, PREC>(S, smem + OFF_A, 0, 1.f, tid, 128);
  if (tid == 0) {
    tc::mbar_init(&bar, 1);
    tc::mbar_init_fence();
  }
  if (warp == 0) {
    tc::tmem_alloc(&s_tmem, 256);
    tc::tmem_relinquish();
  }
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = s_tmem;
  if (tid == 0 && !skip_mma) {
    issue_window<PREC>(l, tc::smem_u32(smem + OFF_A), tc::smem_u32(smem + OFF_B + O::b_off(l)), tmem);
    tc::mma_commit(&bar);
  }
  // skip_mma: nothing arrives on the barrier, so the bounded wait runs out
  const bool ok = tc::mbar_wait_bounded(&bar, 0u, wait_cycles);
  if (__syncthreads_or(!ok)) {
    if (tid == 0) atomicOr(err, 1u);
  } else {
    tc::fence_after_sync();
    const int row = warp * 32 + lane;
    for (int ch = 0; ch < 8; ++ch) {
      uint32_t v[32];
      tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)ch * 32u, v);
      tc::tmem_wait_ld();
      for (int i = 0; i < 32; ++i) out[(size_t)row * kJobCols + ch * 32 + i] = __uint_as_float(v[i]);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, 256);
}

template <int PREC>
cudaError_t launch_probe_t(const float2* y, const float2* tw_m, int M, int l, int skip_mma, float* out,
                           unsigned int* err, cudaStream_t s) {
  using O = Op<PREC>;
  const size_t off_a = ((size_t)32 * (kMRows + 1) * sizeof(float2) + 1023) & ~(size_t)1023;
  size_t smem = off_a + O::A_BYTES + O::B_BYTES;
  smem = std::max(smem, (size_t)120 * 1024);
  cudaError_t e = cudaFuncSetAttribute(rate_gemm_probe_kernel<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  // a skipped MMA gives up after ~0.1 s; a real one has ~2 s
  const long long wait = skip_mma ? kWaitCycles / 20 : kWaitCycles;
  rate_gemm_probe_kernel<PREC><<<1, 128, smem, s>>>(y, tw_m, M, l, skip_mma, wait, out, err);
  return cudaGetLastError();
}

}  // namespace

// Compiled tensor-core work splits: (n1, fold) with 32 * n1 * fold = n_f.
#define VK_MMA_VARIANTS(X, PREC) X(8, 1, PREC) X(16, 1, PREC) X(16, 2, PREC) X(16, 4, PREC)

bool mma_supported(SearchVariant v, int pad_rate, int precision) {
  if (pad_rate != 4) return false;
  if (!(precision == VOLKS_BF16 || precision == VOLKS_FP16 || precision == VOLKS_FP8)) return false;
#define VK_SUP(N1, FOLD, PREC) \
  if (v.n1 == N1 && v.fold == FOLD) return true;
  VK_MMA_VARIANTS(VK_SUP, 0)
#undef VK_SUP
  return false;
}

cudaError_t launch_search_mma(Batch& b, SearchVariant v, int precision, int grid_ctas, cudaStream_t s,
                              int* n_launch) {
#define VK_MLAUNCH(N1, FOLD, PREC) \
  if (v.n1 == N1 && v.fold == FOLD && precision == PREC) return launch_mma_t<N1, FOLD, PREC>(b, grid_ctas, s, n_launch);
  VK_MMA_VARIANTS(VK_MLAUNCH, VOLKS_BF16)
  VK_MMA_VARIANTS(VK_MLAUNCH, VOLKS_FP16)
  VK_MMA_VARIANTS(VK_MLAUNCH, VOLKS_FP8)
#undef VK_MLAUNCH
  return cudaErrorInvalidValue;
}

cudaError_t launch_rate_gemm_probe(const float2* y, const float2* tw_m, int M, int l, int precision, int skip_mma,
                                   float* out, unsigned int* err, cudaStream_t s) {
  if (l < 2 || l > 5) return cudaErrorInvalidValue;
  switch (precision) {
    case VOLKS_BF16: return launch_probe_t<VOLKS_BF16>(y, tw_m, M, l, skip_mma, out, err, s);
    case VOLKS_FP16: return launch_probe_t<VOLKS_FP16>(y, tw_m, M, l, skip_mma, out, err, s);
    case VOLKS_FP8: return launch_probe_t<VOLKS_FP8>(y, tw_m, M, l, skip_mma, out, err, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace vk
