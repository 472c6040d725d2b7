// Reduced-precision search kernel (a4-a7) for sm_103a: the fringe-rate
// transform of the 4..32-AP windows runs as a DFT-matrix GEMM on the
// tcgen05 tensor cores (BF16, FP16 or FP8 E4M3 operands, FP32 accumulation
// in tensor memory), followed by an FP32 re-evaluation of the best delay
// columns of every segment.
//
// Per work unit (baseline, DM trial, 32-AP tile), for each delay residue r
// in turn:
//   delay   stages 0-2 of the FP32 kernel (shared code): FP32 delay
//           spectrum Y[t][c] of the tile's 32 APs x N = 32 N1 delay cells
//           in shared memory S.
//   GEMM    per M-block of 128 delay cells: A = Y^T rounded to the operand
//           type (rows = delay cells, K = 32 APs x (re, im)); per window w,
//           B = the real embedding of the R = 4w point rate DFT of each
//           segment, so D[c][2q + {0,1}] = (Re, Im) Z_w[s, q, c]
//           (Sec. 2.2 2-D search; Sec. 2.4.2 step 6 window combine).  One
//           thread issues the MMAs; two 256-column TMEM buffers let a
//           warpgroup drain one (M-block, window) job while the next runs.
//   coarse  the drain warps store per (segment, delay cell) the largest
//           coarse |Z|^2 over the segment's rate cells; helper warps merge
//           each block's cells within delta of the segment's running
//           maximum into a candidate list (the last block is merged by the
//           warp that refines the segment; at most 8 are kept).
//   w=1,2   exact FP32 windows on the CUDA cores, taken in pieces (one
//           segment each) by the helper warps while they wait, the rest by
//           every warp after its refinement.
//   refine  the retained delay cells of every segment are re-evaluated in
//           FP32 from S (all R rate cells of each: pre-twiddled w-point
//           register FFTs, as the FP32 kernel computes them); the segment's
//           peak is the largest refined power, ties to the lowest q M + m.
//   publish the residue's keys fold into the tile's running keys; each
//           key is stored once after the tile's last residue.
//
// Reported peaks are therefore FP32 evaluations of real grid cells; they
// equal the FP32 search whenever its peak cell lies in one of the delay
// cells the coarse pass retains for that segment.
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
constexpr uint32_t kGemmMask = 0x3cu;  // windows on the tensor cores: 4, 8, 16, 32 (log2 2..5)
constexpr int kGemmSegs = 15;        // their segments in a tile
constexpr int kTopK = 8;             // most delay cells refined per segment and unit
constexpr int kPerBlk = 6;           // most delay cells a 128-cell block adds to a segment's list
constexpr int kList = 24;            // candidate list length per segment (>= 4 blocks x kPerBlk)
constexpr long long kWaitCycles = 4000000000LL;  // ~2 s at 2 GHz

// Helper warps during the GEMM phase.  With two drain warpgroups the
// issuing warp's scheduler (warps 0, 4, 8, 12: warp % 4 picks it, and the
// drain warps' TMEM lane quarters fix theirs) also runs two drain warps;
// for BF16 / FP16 (four MMAs per job) warp 12 sits the phase out so the
// issuing thread waits less for issue slots (BF16 measured 1.7 % faster,
// FP16 the same); for FP8 (two MMAs per job) the seventh helper is worth
// more (0.9 %).
template <int NW, int NWG, int PREC>
struct Helpers {
  static constexpr bool kSpare = NWG == 2 && PREC != VOLKS_FP8;
  static constexpr int count = NW - 1 - 4 * NWG - (kSpare ? 1 : 0);
};

template <int PREC>
struct Op {
  static constexpr int EB = PREC == VOLKS_FP8 ? 1 : 2;      // bytes per element
  static constexpr uint32_t A_ROW = 64u * EB;               // K bytes of an A row (32 APs x re, im)
  static constexpr uint32_t A_BYTES = 128u * A_ROW;         // 128 rows
  // per window l = 1..5: segments per MMA, rows (MMA N), K bytes per row
  static constexpr int seg_per_mma(int l) { return (2 << l) * EB >= 32 ? 1 : 32 / ((2 << l) * EB); }
  static constexpr int b_rows(int l) { return (8 << l) * seg_per_mma(l); }
  static constexpr int b_row_bytes(int l) { return (2 << l) * EB >= 32 ? (2 << l) * EB : 32; }
  static constexpr int b_bytes(int l) { return b_rows(l) * b_row_bytes(l); }
  static constexpr int b_off(int l) {
    int o = 0;
    for (int i = 1; i < l; ++i) o += b_bytes(i);
    return o;
  }
  static constexpr int B_BYTES = b_off(6);
  // the search keeps only windows 4..32 (log2 2..5) on the tensor cores
  static constexpr int B_SEARCH = b_off(6) - b_off(2);
  // operand scale target for the per-tile power-of-two scaling
  static constexpr int SCALE_EXP = PREC == VOLKS_FP8 ? 8 : 14;
};

template <int N1, int PREC>
struct MmaSmem {
  static constexpr int N = 32 * N1;
  static constexpr size_t S_BYTES = (size_t)32 * (N + 1) * sizeof(float2);
  static constexpr size_t OFF_A = (S_BYTES + 1023) & ~(size_t)1023;
  static constexpr size_t OFF_B = OFF_A + 2 * Op<PREC>::A_BYTES;
  static constexpr size_t OFF_COL = OFF_B + Op<PREC>::B_SEARCH;                    // u32 [2][15][128]
  static constexpr size_t OFF_LIST = OFF_COL + (size_t)2 * kGemmSegs * kMRows * 4;  // uint2 [15][kList]
  static constexpr size_t OFF_LCOUNT = OFF_LIST + (size_t)kGemmSegs * kList * 8;    // int [15]
  static constexpr size_t OFF_RUNMAX = OFF_LCOUNT + 64;                             // u32 [15]
  static constexpr size_t OFF_BEST = OFF_RUNMAX + 64;                               // u64 [63]
  static constexpr size_t OFF_PIECE = OFF_BEST + (size_t)kMaxSegPerTile * 8;        // int
  static constexpr size_t USED = OFF_PIECE + 8;
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

// Rate-DFT operand B of window 2^l (rows n = MMA N, K-major, swizzled
// layout of b_row_bytes(l)), from the FP32 twiddle table W_M^i: row 2q of a segment block
// holds (cos, sin) and row 2q + 1 (-sin, cos) of 2 pi q u / R against
// (Re, Im) of AP u, so that D = A B^T gives (Re, Im) of
// Z_q = sum_u Y_u exp(-2 pi i q u / R), R = 4w.  Segments sharing one MMA
// (K of a segment shorter than one MMA) get a block-diagonal B.
template <int PREC, int L0 = 1>
__device__ void build_rate_dft(uint8_t* B, const float2* __restrict__ tw_m, int M, int tid, int nt) {
  using O = Op<PREC>;
  constexpr int EB = O::EB;
#pragma unroll 1
  for (int l = L0; l <= 5; ++l) {
    const int w = 1 << l, R = 4 * w;
    const int rows = O::b_rows(l), kel = O::b_row_bytes(l) / EB;
    const uint32_t rb = (uint32_t)O::b_row_bytes(l);
    uint8_t* base = B + O::b_off(l) - O::b_off(L0);
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
      const uint32_t off = tc::sw_offset((uint32_t)n, (uint32_t)(k * EB), rb);
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
    const uint32_t off = tc::sw_offset((uint32_t)row, (uint32_t)ch * 16u, O::A_ROW);
    *reinterpret_cast<uint4*>(A + off) = make_uint4(wv[0], wv[1], wv[2], wv[3]);
  }
}

// Issue the MMAs of window 2^L for one M-block into TMEM columns d .. d+255
// (column 8 w s + 2 q + {0,1} = (Re, Im) of rate cell q of segment s).
// ad / bd: descriptors of the A block and of the window's B at K byte 0;
// every other operand offset is a compile-time constant added to the
// descriptors' start-address field (bytes >> 4), so the issuing thread
// does almost no scalar work between MMAs.
template <int PREC, int L>
__device__ __forceinline__ void issue_window_t(uint64_t ad, uint64_t bd, uint32_t d) {
  using O = Op<PREC>;
  constexpr int EB = O::EB;
  constexpr int w = 1 << L;
  constexpr int seg_kb = 2 * w * EB;  // K bytes of one segment; one MMA consumes 32
  if constexpr (seg_kb >= 32) {
    constexpr int nseg = 32 / w, n = 8 * w, ks = seg_kb / 32;
    constexpr uint32_t idesc = PREC == VOLKS_FP8 ? tc::idesc_e4m3(n) : tc::idesc_f16(n, PREC == VOLKS_BF16);
    static_for<0, nseg>([&](auto ss) {
      constexpr int s = decltype(ss)::value;
      static_for<0, ks>([&](auto kk) {
        constexpr int k = decltype(kk)::value;
        const uint64_t a = ad + (uint64_t)((seg_kb * s + 32 * k) >> 4);
        const uint64_t b = bd + (uint64_t)((32 * k) >> 4);
        if constexpr (PREC == VOLKS_FP8) tc::mma_f8_c<(k > 0)>(d + (uint32_t)(n * s), a, b, idesc);
        else tc::mma_f16_c<(k > 0)>(d + (uint32_t)(n * s), a, b, idesc);
      });
    });
  } else {
    constexpr int g = 32 / seg_kb, n = 8 * w * g, ngrp = (32 / w) / g;
    constexpr uint32_t idesc = PREC == VOLKS_FP8 ? tc::idesc_e4m3(n) : tc::idesc_f16(n, PREC == VOLKS_BF16);
    static_for<0, ngrp>([&](auto pp) {
      constexpr int p = decltype(pp)::value;
      const uint64_t a = ad + (uint64_t)((32 * p) >> 4);
      if constexpr (PREC == VOLKS_FP8) tc::mma_f8_c<false>(d + (uint32_t)(n * p), a, bd, idesc);
      else tc::mma_f16_c<false>(d + (uint32_t)(n * p), a, bd, idesc);
    });
  }
}

template <int PREC>
__device__ __forceinline__ void issue_window(int l, uint32_t a_base, uint32_t b_base, uint32_t d) {
  using O = Op<PREC>;
  const uint64_t ad = tc::sdesc_sw(a_base, O::A_ROW);
  const uint64_t bd = tc::sdesc_sw(b_base, (uint32_t)O::b_row_bytes(l));
  switch (l) {
    case 1: issue_window_t<PREC, 1>(ad, bd, d); break;
    case 2: issue_window_t<PREC, 2>(ad, bd, d); break;
    case 3: issue_window_t<PREC, 3>(ad, bd, d); break;
    case 4: issue_window_t<PREC, 4>(ad, bd, d); break;
    default: issue_window_t<PREC, 5>(ad, bd, d); break;
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
  fft_dif<W, true>(y);
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

// Per-thread pipeline state that persists across work units: the TMEM base,
// the jobs issued into each buffer (issuing thread) and one phase-parity bit
// per barrier this thread waits on (bit PB_*: + buffer index).
struct MmaCtx {
  uint32_t tmem;        // TMEM base address (512 columns)
  uint32_t par;         // parity bits, see PB_*
  uint32_t n_use0, n_use1;
};
constexpr int PB_FULL = 0, PB_AFULL = 2, PB_CFREE = 4, PB_ADONE = 6, PB_CDONE = 8;
__device__ __forceinline__ uint32_t pbit(uint32_t par, int b) { return (par >> b) & 1u; }

// Operand descriptors, built once per CTA.
struct JobTable {
  uint64_t bd[6];               // B descriptor of each GEMM window (log2 2..5)
  uint64_t ad[2];               // A descriptor of each A buffer
};

struct MmaBars {
  uint64_t full[2];     // the MMAs of the job in TMEM buffer i completed (tcgen05.commit)
  uint64_t empty[2];    // the drain warpgroup of buffer i has read it
  uint64_t afull[2];    // the helper warps packed A buffer i
  uint64_t adone[2];    // every MMA reading A buffer i completed (commit after a block's last job)
  uint64_t cdone[2];    // every drain warp wrote its rows of column-maxima buffer i
  uint64_t cfree[2];    // the helper warps merged column-maxima buffer i (it may be rewritten)
};

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(bar)) : "memory");
}

// One warp-wide bounded wait (lane 0 polls, the result is broadcast).
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, int lane) {
  bool w = true;
  if (lane == 0) w = tc::mbar_wait_bounded(bar, parity, kWaitCycles);
  return __shfl_sync(0xffffffffu, w, 0) != 0;
}

// Warp-wide wait that does other work meanwhile: while the phase is not
// complete, run work pieces (`piece()` returns false when none is left),
// then fall back to the bounded wait.
template <class F>
__device__ __forceinline__ bool warp_wait_busy(uint64_t* bar, uint32_t parity, int lane, F&& piece) {
  for (;;) {
    bool done = false;
    if (lane == 0) done = tc::mbar_test(bar, parity);
    if (__shfl_sync(0xffffffffu, done, 0)) return true;
    if (!piece()) return warp_wait(bar, parity, lane);
  }
}

// max |Z|^2 over the 16 cells of a 32-column chunk ((Re, Im) column pairs)
__device__ __forceinline__ float fold32(const uint32_t (&v)[32]) {
  float ma = 0.f, mb = 0.f;
#pragma unroll
  for (int i = 0; i < 32; i += 8) {
    const float a0 = __uint_as_float(v[i]), a1 = __uint_as_float(v[i + 1]);
    const float a2 = __uint_as_float(v[i + 2]), a3 = __uint_as_float(v[i + 3]);
    const float b0 = __uint_as_float(v[i + 4]), b1 = __uint_as_float(v[i + 5]);
    const float b2 = __uint_as_float(v[i + 6]), b3 = __uint_as_float(v[i + 7]);
    ma = tc::fmax3(ma, fmaf(a0, a0, a1 * a1), fmaf(a2, a2, a3 * a3));
    mb = tc::fmax3(mb, fmaf(b0, b0, b1 * b1), fmaf(b2, b2, b3 * b3));
  }
  return fmaxf(ma, mb);
}

// Drain one job (window 2^L, 256 TMEM columns) for this warp's 32 rows: the
// eight 32-column chunks are loaded two at a time (the next load in flight
// while the previous chunk is folded), the buffer is handed back to the
// issuing thread after the last load, and the largest coarse |Z|^2 of each
// segment (8 w columns) is stored for this row at cm[s * kMRows].
template <int L>
__device__ __forceinline__ void drain_job(uint32_t tb, uint32_t* cm, uint64_t* empty, int lane) {
  constexpr int SEGC = 8 << L;  // columns per segment
  constexpr int CPS = SEGC / 32;  // chunks per segment
  static_assert(SEGC >= 32, "a chunk lies within one segment");
  uint32_t va[32], vb[32];
  float m = 0.f;
  tc::tmem_ld32(tb, va);
  tc::tmem_wait_ld_dep(va);
#pragma unroll
  for (int ch = 0; ch < 8; ch += 2) {
    tc::tmem_ld32(tb + (uint32_t)(ch + 1) * 32u, vb);
    m = fmaxf(m, fold32(va));
    if ((ch + 1) % CPS == 0) {
      cm[(ch / CPS) * kMRows] = __float_as_uint(m);
      m = 0.f;
    }
    tc::tmem_wait_ld_dep(vb);
    if (ch + 2 < 8) {
      tc::tmem_ld32(tb + (uint32_t)(ch + 2) * 32u, va);
    } else {
      // every load of the job is complete: hand the buffer back
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) mbar_arrive(empty);
    }
    m = fmaxf(m, fold32(vb));
    if ((ch + 2) % CPS == 0) {
      cm[((ch + 1) / CPS) * kMRows] = __float_as_uint(m);
      m = 0.f;
    }
    if (ch + 2 < 8) tc::tmem_wait_ld_dep(va);
  }
}

// Candidate delay cells of a segment (per work unit): the cells whose coarse
// power is at least Keep<PREC> times the segment's coarse maximum, at most
// kTopK of them.  Keep = 1 - delta, delta ~4x the coarse relative error of
// |Z|^2 at a peak for the operand type, so the FP32 peak's cell is retained
// unless more than kTopK cells lie within delta of the coarse maximum (then
// delta is halved, a few times at most, and the lowest cells are kept).
template <int PREC>
struct Keep {
  static constexpr float value = PREC == VOLKS_FP8 ? 1.0f - 1.0f / 4 : PREC == VOLKS_FP16 ? 1.0f - 1.0f / 64 : 1.0f - 1.0f / 16;
};

// Append the cells of one 128-cell block (column maxima cm[cell]) that lie
// within delta of the segment's running maximum (this block included) to the
// segment's list, at most kPerBlk of them (delta halved while more pass, then
// the lowest cells).  The running maximum only grows, so the list holds
// every cell that the final threshold (`finish_list`) can keep.  One warp.
template <int PREC>
__device__ __forceinline__ void merge_block(const uint32_t* __restrict__ cm, int b, uint2* lst, int* lcount,
                                            uint32_t* runmax, int sg, int lane) {
  uint32_t v[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) v[i] = cm[lane + 32 * i];
  const uint32_t bm = __reduce_max_sync(0xffffffffu, max(max(v[0], v[1]), max(v[2], v[3])));
  const uint32_t mx = max(runmax[sg], bm);
  float keep = Keep<PREC>::value;
  bool kn[4];
  uint32_t bn[4];
  int total;
#pragma unroll 1
  for (int it = 0;; ++it) {
    const uint32_t thr = __float_as_uint(__uint_as_float(mx) * keep);
    total = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      kn[i] = v[i] >= thr;
      bn[i] = __ballot_sync(0xffffffffu, kn[i]);
      total += __popc(bn[i]);
    }
    if (total <= kPerBlk || it == 6) break;
    keep = 0.5f * (1.0f + keep);
  }
  // cell = 128 b + lane + 32 i: ballot order (i, then lane) is cell order
  const int base = lcount[sg];
  const uint32_t lt = (1u << lane) - 1u;
  int pos = base;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int p = pos + __popc(bn[i] & lt);
    if (kn[i] && p < base + kPerBlk) lst[sg * kList + p] = make_uint2(v[i], (uint32_t)(b * kMRows + lane + 32 * i));
    pos += __popc(bn[i]);
  }
  __syncwarp();
  if (lane == 0) {
    lcount[sg] = base + min(total, kPerBlk);
    runmax[sg] = mx;
  }
  __syncwarp();
}

// Final candidates of a segment from its list: the entries within delta of
// the segment's coarse maximum (delta halved while more than kTopK pass,
// then the lowest cells), compacted to the front of the list; returns their
// number.  One warp.
template <int PREC>
__device__ __forceinline__ int finish_list(uint2* lst, const int* lcount, const uint32_t* runmax, int sg, int lane) {
  const int n = lcount[sg];
  const uint2 e = lane < n ? lst[sg * kList + lane] : make_uint2(0u, 0xffffffffu);
  const uint32_t mx = runmax[sg];
  float keep = Keep<PREC>::value;
  bool k;
  uint32_t bal;
  int total;
#pragma unroll 1
  for (int it = 0;; ++it) {
    const uint32_t thr = __float_as_uint(__uint_as_float(mx) * keep);
    k = lane < n && e.x >= thr;
    bal = __ballot_sync(0xffffffffu, k);
    total = __popc(bal);
    if (total <= kTopK || it == 6) break;
    keep = 0.5f * (1.0f + keep);
  }
  const int p = __popc(bal & ((1u << lane) - 1u));
  __syncwarp();
  if (k && p < kTopK) lst[sg * kList + p] = e;
  __syncwarp();
  return min(total, kTopK);
}

// One unit on the tensor-core path.  Returns false if a bounded wait gave
// up (the error flag is set; the caller stops).
//
// Warp roles during the GEMM phase (NW warps):
//   warp 0, lane 0   issues every job's MMAs once its TMEM buffer is free and
//                    its A block packed, then commits to the job's `full`
//                    barrier (and, after a block's last job, to `adone`);
//   drain warps      warps 4 .. 4 + 4 NWG - 1: one warpgroup per TMEM buffer
//                    (two when NW = 16, so jobs alternate between them; one
//                    that takes every job when NW = 8); each warp reads the
//                    whole job for its 32 TMEM lanes (lane quarter = warp % 4)
//                    and stores per-(segment, delay cell) coarse maxima into
//                    one of two column-maxima buffers (by block parity);
//   helper warps     the others (but warp 12 for BF16 / FP16, see Helpers):
//                    the exact 1- and 2-AP windows, the A blocks
//                    from the third on (once `adone` says the MMAs reading the
//                    buffer are complete), and the candidate merges of each
//                    block but the last (once every drain warp passed
//                    `cdone`); after the phase every warp merges the last
//                    block of the segment it then refines.
template <int N1, int FOLD, int PREC>
__device__ __forceinline__ bool mma_tile(const UnitState& us, uint8_t* smem, MmaCtx& cx, MmaBars& bars,
                                         const JobTable& jt, float* s_amax, unsigned int* err,
                                         unsigned long long* run) {
  using O = Op<PREC>;
  using L = MmaSmem<N1, PREC>;
  constexpr int N = 32 * N1, LD = N + 1, NT = N, NW = N1, NMB = N / kMRows;
  constexpr int NWG = NW >= 16 ? 2 : 1;      // drain warpgroups
  constexpr int NHELP = Helpers<NW, NWG, PREC>::count;
  static_assert(NHELP >= 1 && NMB >= 2, "work split");
  float2* S = reinterpret_cast<float2*>(smem);
  uint8_t* A = smem + L::OFF_A;
  uint32_t* colmax = reinterpret_cast<uint32_t*>(smem + L::OFF_COL);
  uint2* lst = reinterpret_cast<uint2*>(smem + L::OFF_LIST);
  int* lcount = reinterpret_cast<int*>(smem + L::OFF_LCOUNT);
  uint32_t* runmax = reinterpret_cast<uint32_t*>(smem + L::OFF_RUNMAX);
  unsigned long long* best = reinterpret_cast<unsigned long long*>(smem + L::OFF_BEST);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  // FP16 / FP8: the delay stage also folds max |Re|, |Im| of Y into s_amax
  delay_stage<N1, FOLD, false, false, PREC != VOLKS_BF16>(us, S, reinterpret_cast<unsigned int*>(s_amax));

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
  const uint32_t gmask = (uint32_t)win_mask & kGemmMask;
  const int nG = __popc(gmask);
  // gl: log2 of the i-th GEMM window in bits 3i..3i+2; sb: first sigma of
  // window 2^l in bits 5l..5l+4
  uint32_t gl = 0u, sb = 0u;
  int nsig = 0;
  for (int l = 1, i = 0; l <= 5; ++l)
    if (gmask & (1u << l)) {
      gl |= (uint32_t)l << (3 * i++);
      sb |= (uint32_t)nsig << (5 * l);
      nsig += kTile >> l;
    }
  auto gwin = [&](int i) { return (int)((gl >> (3 * i)) & 7u); };
  auto sig_base = [&](int l) { return (int)((sb >> (5 * l)) & 31u); };

  int* piece_next = reinterpret_cast<int*>(smem + L::OFF_PIECE);
  for (int i = tid; i < kMaxSegPerTile; i += NT) best[i] = 0ull;
  if (tid == 0) *piece_next = 0;
  float scale = 1.f;
  if (nG == 0) __syncthreads();
  if (nG > 0) {
    if constexpr (PREC != VOLKS_BF16) {
      // per-tile power-of-two operand scale: largest |component| -> < 2^SCALE_EXP
      const float amax = *s_amax;
      if (amax > 0.f && amax < 3.0e38f) {
        int e;
        frexpf(amax, &e);
        scale = ldexpf(1.f, max(-120, min(120, O::SCALE_EXP - e)));
      }
    }
    pack_a<LD, PREC>(S, A, 0, scale, tid, NT);
    pack_a<LD, PREC>(S, A + O::A_BYTES, 1, scale, tid, NT);
    for (int i = tid; i < nsig; i += NT) {
      lcount[i] = 0;
      runmax[i] = 0u;
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
  }

  // ---- the exact 1- and 2-AP windows as a pool of work pieces ----
  // The helper warps take pieces while the barrier they wait on is not yet
  // complete, and after their own work: piece p < n1p is a 1-AP segment, the
  // next n2p are 2-AP segments (halves and quarters of segments measured
  // slower: each piece pays a counter atomic and a warp reduction); each
  // ends in one 64-bit atomicMax into the segment's key, so the order of
  // the pieces does not matter.
  const int n1p = (win_mask & 1) ? kTile : 0;
  const int n2p = (win_mask & 2) ? kTile / 2 : 0;
  auto piece = [&]() -> bool {
    int pc = 0;
    if (lane == 0) pc = atomicAdd(piece_next, 1);
    pc = __shfl_sync(0xffffffffu, pc, 0);
    if (pc >= n1p + n2p) return false;
    if (pc < n1p) {
      const int s = pc;
      if (!seg_valid(0, s)) return true;
      float bp = -1.f;
      int bc = 0;
#pragma unroll 4
      for (int jj = 0; jj < N1; ++jj) {
        const int c = lane + 32 * jj;
        const float pw = cabs2(S[s * LD + c]);
        if (pw > bp) {
          bp = pw;
          bc = c;
        }
      }
      const unsigned long long key = warp_key(bp, (uint32_t)(bc * P + r));
      if (lane == 0) atomicMax(best + slot_base(0) + s, key);
    } else {
      // 2-AP segment s: each column's largest rate cell
      // is r0 + max(|2 rx|, |2 ry|, |sqrt2 (rx + ry)|, |sqrt2 (ry - rx)|),
      // which equals the largest of the eight cells rate_cells_w2 gives
      // (rounding is monotonic); the lane's best column (the first on equal
      // powers) is then resolved to its cell once.
      const int s = pc - n1p;
      if (!seg_valid(1, s)) return true;
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
        const float pm = r0 + tc::fmax3(fabsf(a), fabsf(bb), fmaxf(fabsf(cc), fabsf(dd)));
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
      const unsigned long long key = warp_key(pv, qv * M + (uint32_t)(bc * P + r));
      if (lane == 0) atomicMax(best + slot_base(1) + s, key);
    }
    return true;
  };

  bool ok = true;
  const bool drain = warp >= 4 && warp < 4 + 4 * NWG;
  if (warp == 0) {
    // ---- issuing thread ----
    if (lane == 0 && nG > 0) {
      int j = 0;
      for (int b = 0; ok && b < NMB; ++b) {
        if (b >= 2) {
          ok = tc::mbar_wait_bounded(&bars.afull[b & 1], pbit(cx.par, PB_AFULL + (b & 1)), kWaitCycles);
          cx.par ^= 1u << (PB_AFULL + (b & 1));
        }
        for (int gi = 0; ok && gi < nG; ++gi, ++j) {
          const int buf = j & 1, l = gwin(gi);
          const uint32_t nu = buf ? cx.n_use1 : cx.n_use0;
          if (nu > 0) ok = tc::mbar_wait_bounded(&bars.empty[buf], (nu - 1u) & 1u, kWaitCycles);
          if (!ok) break;
          tc::fence_after_sync();
          const uint64_t ad = jt.ad[b & 1], bd = jt.bd[l];
          const uint32_t d = cx.tmem + (uint32_t)buf * kJobCols;
          // straight-line MMAs with compile-time operand offsets
          switch (l) {
            case 2: issue_window_t<PREC, 2>(ad, bd, d); break;
            case 3: issue_window_t<PREC, 3>(ad, bd, d); break;
            case 4: issue_window_t<PREC, 4>(ad, bd, d); break;
            default: issue_window_t<PREC, 5>(ad, bd, d); break;
          }
          tc::mma_commit(&bars.full[buf]);
          if (buf) ++cx.n_use1; else ++cx.n_use0;
        }
        // A buffer b & 1 is free once these MMAs complete
        if (ok && b + 2 < NMB) tc::mma_commit(&bars.adone[b & 1]);
      }
    }
    __syncwarp();
    if (nG == 0)
      while (piece()) {
      }
  } else if (drain) {
    // ---- drain warpgroups: whole jobs, 32 TMEM lanes per warp ----
    if (nG > 0) {
      const int q = warp & 3, wg = (warp - 4) >> 2;
      const int row = q * 32 + lane;
      int j = 0;
#pragma unroll 1
      for (int b = 0; b < NMB; ++b) {
        uint32_t* cmb = colmax + (size_t)(b & 1) * kGemmSegs * kMRows + row;
        if (b >= 2) {
          // the helpers have merged block b - 2 out of this buffer
          if (ok) ok = warp_wait(&bars.cfree[b & 1], pbit(cx.par, PB_CFREE + (b & 1)), lane);
          cx.par ^= 1u << (PB_CFREE + (b & 1));
        }
#pragma unroll 1
        for (int gi = 0; gi < nG; ++gi, ++j) {
          const int buf = j & 1, l = gwin(gi);
          if (NWG == 2 && buf != wg) continue;
          if (ok) ok = warp_wait(&bars.full[buf], pbit(cx.par, PB_FULL + buf), lane);
          cx.par ^= 1u << (PB_FULL + buf);
          tc::fence_after_sync();
          const uint32_t tb = cx.tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)buf * kJobCols;
          uint32_t* cm = cmb + sig_base(l) * kMRows;
          if (ok) {
            switch (l) {
              case 2: drain_job<2>(tb, cm, &bars.empty[buf], lane); break;
              case 3: drain_job<3>(tb, cm, &bars.empty[buf], lane); break;
              case 4: drain_job<4>(tb, cm, &bars.empty[buf], lane); break;
              default: drain_job<5>(tb, cm, &bars.empty[buf], lane); break;
            }
          } else {
            // after a failed wait: no TMEM reads, but every arrival still happens
            __syncwarp();
            if (lane == 0) mbar_arrive(&bars.empty[buf]);
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&bars.cdone[b & 1]);
      }
    }
  } else {
    // ---- helper warps ----
    constexpr bool kSpare = Helpers<NW, NWG, PREC>::kSpare;
    const int hw = warp < 4 ? warp - 1 : warp - 4 - 4 * NWG + 3 - (kSpare ? 1 : 0);
    if (nG > 0 && !(kSpare && warp == 12)) {
#pragma unroll 1
      for (int b = 0; b < NMB; ++b) {
        if (b + 2 < NMB) {
          // refill A buffer b & 1 with block b + 2 once its MMAs are done
          if (ok) ok = warp_wait_busy(&bars.adone[b & 1], pbit(cx.par, PB_ADONE + (b & 1)), lane, piece);
          cx.par ^= 1u << (PB_ADONE + (b & 1));
          if (ok) {
            pack_a<LD, PREC>(S, A + (b & 1) * O::A_BYTES, b + 2, scale, hw * 32 + lane, NHELP * 32);
            tc::fence_async_smem();
          }
          __syncwarp();
          if (lane == 0) mbar_arrive(&bars.afull[b & 1]);
        }
        if (b == NMB - 1) {
          // the last block is merged after the GEMM phase by every warp (one
          // segment each, fused with its refinement); the drain warps have
          // arrived on cdone by then, so only the parity advances here
          cx.par ^= 1u << (PB_CDONE + (b & 1));
          break;
        }
        if (ok) ok = warp_wait_busy(&bars.cdone[b & 1], pbit(cx.par, PB_CDONE + (b & 1)), lane, piece);
        cx.par ^= 1u << (PB_CDONE + (b & 1));
        if (ok) {
          // the same warp merges a segment in every block, so blocks stay in order
          const uint32_t* cmb = colmax + (size_t)(b & 1) * kGemmSegs * kMRows;
          for (int sg = hw; sg < nsig; sg += NHELP)
            merge_block<PREC>(cmb + sg * kMRows, b, lst, lcount, runmax, sg, lane);
        }
        if (b + 2 < NMB) {
          __syncwarp();
          if (lane == 0) mbar_arrive(&bars.cfree[b & 1]);
        }
      }
    }
    // pieces still left go to every warp after the refinement
    if (ok && nG == 0)
      while (piece()) {
      }
  }
  if (__syncthreads_or(!ok)) {
    if (tid == 0) atomicOr(err, 1u);
    return false;
  }
  if (nG > 0) {
    // ---- last block's merge and FP32 refinement of the candidate delay
    // cells (all warps, one segment at a time) ----
    // descending sigma: the largest windows (longest refinements) go first
    const uint32_t* cml = colmax + (size_t)((NMB - 1) & 1) * kGemmSegs * kMRows;
    for (int sg = nsig - 1 - warp; sg >= 0; sg -= NW) {
      int l = gwin(0);
      for (int i = 1; i < nG; ++i)
        if (sg >= sig_base(gwin(i))) l = gwin(i);
      const int s = sg - sig_base(l);
      if (!seg_valid(l, s)) continue;
      merge_block<PREC>(cml + sg * kMRows, NMB - 1, lst, lcount, runmax, sg, lane);
      const int nc = finish_list<PREC>(lst, lcount, runmax, sg, lane);
      int ci = lane >> 2;
      if (ci >= nc) ci = 0;
      const int c = (int)lst[sg * kList + ci].y;
      const int rho = lane & 3;
      float pw;
      uint32_t qq;
      const int u0 = s << l;
      switch (l) {
        case 1: refine_column<2, LD>(S, c, u0, rho, tw_m, (int)M, pw, qq); break;
        case 2: refine_column<4, LD>(S, c, u0, rho, tw_m, (int)M, pw, qq); break;
        case 3: refine_column<8, LD>(S, c, u0, rho, tw_m, (int)M, pw, qq); break;
        case 4: refine_column<16, LD>(S, c, u0, rho, tw_m, (int)M, pw, qq); break;
        default: refine_column<32, LD>(S, c, u0, rho, tw_m, (int)M, pw, qq); break;
      }
      const unsigned long long key = warp_key(pw, qq * M + (uint32_t)(c * P + r));
      if (lane == 0) best[slot_base(l) + s] = key;
    }
    // the exact 1- and 2-AP pieces the helper warps left: the warps with
    // short refinements take them
    while (piece()) {
    }
  }
  __syncthreads();
  // ---- fold this residue's keys into the tile's running keys ----
  const int ns = slot_base(kMaxWinLog + 1);
  for (int i = tid; i < ns; i += NT) run[i] = max(run[i], best[i]);
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
  __shared__ __align__(8) MmaBars bars;
  __shared__ __align__(8) JobTable jt;
  __shared__ uint32_t s_tmem;
  __shared__ float s_amax;
  __shared__ unsigned long long run[kMaxSegPerTile];
  const int tid = threadIdx.x;
  using L = MmaSmem<N1, PREC>;
  build_rate_dft<PREC, 2>(smem + L::OFF_B, p.d[0].tw_m, p.d[0].M, tid, N);
  if (tid == 0) {
    constexpr int NWG = N1 >= 16 ? 2 : 1, NHELP = Helpers<N1, NWG, PREC>::count;
    for (int l = 2; l <= 5; ++l) {
      jt.bd[l] = tc::sdesc_sw(tc::smem_u32(smem + L::OFF_B + Op<PREC>::b_off(l) - Op<PREC>::b_off(2)),
                              (uint32_t)Op<PREC>::b_row_bytes(l));
    }
    for (int i = 0; i < 2; ++i) {
      jt.ad[i] = tc::sdesc_sw(tc::smem_u32(smem + L::OFF_A + i * Op<PREC>::A_BYTES), Op<PREC>::A_ROW);
      tc::mbar_init(&bars.full[i], 1);
      tc::mbar_init(&bars.empty[i], 4);
      tc::mbar_init(&bars.afull[i], NHELP);
      tc::mbar_init(&bars.adone[i], 1);
      tc::mbar_init(&bars.cdone[i], 4 * NWG);
      tc::mbar_init(&bars.cfree[i], NHELP);
    }
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
  cx.par = 0u;
  cx.n_use0 = cx.n_use1 = 0u;
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
      us.d = (int)(unit % a.n_dm);
      unit /= a.n_dm;
      const int tile = (int)(unit % a.n_tiles);
      us.b = (int)(unit / a.n_tiles);
      us.t0 = tile * kTile;
      us.nv = a.nvalid[us.d];
      us.valid = us.t0 < us.nv;
    }
    __syncthreads();
    if (us.valid) {
      // every delay residue of the tile in turn; each key is stored once
      const int P = us.a.pad_delay * FOLD;
      for (int i = tid; i < kMaxSegPerTile; i += N) run[i] = 0ull;
      bool failed = false;
      for (int r = 0; r < P && !failed; ++r) {
        if (tid == 0) {
          us.r = r;
          s_amax = 0.f;
        }
        __syncthreads();
        failed = !mma_tile<N1, FOLD, PREC>(us, smem, cx, bars, jt, &s_amax, p.err, run);
        __syncthreads();
      }
      if (failed) break;
      store_keys<false>(us, run, us.a.win_mask);
    }
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
  if (l < 1 || l > 5) return cudaErrorInvalidValue;
  switch (precision) {
    case VOLKS_BF16: return launch_probe_t<VOLKS_BF16>(y, tw_m, M, l, skip_mma, out, err, s);
    case VOLKS_FP16: return launch_probe_t<VOLKS_FP16>(y, tw_m, M, l, skip_mma, out, err, s);
    case VOLKS_FP8: return launch_probe_t<VOLKS_FP8>(y, tw_m, M, l, skip_mma, out, err, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace vk
