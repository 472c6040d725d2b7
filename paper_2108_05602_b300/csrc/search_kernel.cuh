// The FP32 search kernel (a4-a7) and its host launch wrappers, as
// templates over the work split (N1, FOLD) and the rate padding PADR.
// Included by volks_kernels.cu (dispatch, power-of-two bands) and by the
// translation units that instantiate the mixed-radix bands, so the
// instantiations compile in parallel.
#pragma once
#include <algorithm>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/volks.h"
#include "fft_regs.cuh"
#include "search_common.cuh"
#include "volks_internal.h"

namespace vk {

// ============================================================ search ====
// Stage 3 of one residue pass on CUDA cores after the delay stage: thread =
// delay column c, FP32 rate FFTs of every window, |Z|^2 and arg-max, merged
// over the warps into the tile's running key of each segment.
// Windows searched by a sliding-form unit whose tile starts at AP t0 (phase
// phi = t0 mod 32): those wider than phi.
__device__ __forceinline__ int sliding_windows(int win_mask, int t0) {
  const int phi = t0 & (kTile - 1);
  const int w = win_mask & kWinBits;
  return phi > 0 ? w & ~((1 << (32 - __clz(phi))) - 1) : w;
}

template <int N1, int PADR, int FOLD, bool SLIDE>
__device__ __forceinline__ void search_tile(const UnitState& us, float2* S, uint2* slot, unsigned long long* run) {
  constexpr int N = 32 * N1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  delay_stage<N1, FOLD>(us, S);
  // ---- stage 3 ----
  // a sliding unit of AP phase phi = t0 mod 32 searches the windows wider than phi
  const int win_mask = SLIDE ? sliding_windows(us.a.win_mask, us.t0) : us.a.win_mask;
  // slot base of window 2^l: segments of the searched smaller windows first
  auto slot_base = [&](int l) {
    int o = 0;
    for (int i = 0; i < l; ++i)
      if (win_mask & (1 << i)) o += kTile >> i;
    return o;
  };
  {
    const int c = threadIdx.x;
    const int P = us.a.pad_delay * FOLD;
    const uint32_t m = (uint32_t)(c * P + us.r);
    const uint32_t M = (uint32_t)us.a.M;
    const int t0 = us.t0, nv = us.nv;
    if (win_mask & 1) rate_window<1, PADR, N1, SLIDE>(S, c, m, M, t0, nv, slot_base(0), slot, warp, lane);
    if (win_mask & 2) {
      if constexpr (PADR == 4)
        rate_window_w2_seg<N1, SLIDE>(S, M, P, us.r, t0, nv, slot_base(1), slot, warp, lane);
      else
        rate_window<2, PADR, N1, SLIDE>(S, c, m, M, t0, nv, slot_base(1), slot, warp, lane);
    }
    if (win_mask & 4) rate_window<4, PADR, N1, SLIDE>(S, c, m, M, t0, nv, slot_base(2), slot, warp, lane);
    if (win_mask & 8) rate_window<8, PADR, N1, SLIDE>(S, c, m, M, t0, nv, slot_base(3), slot, warp, lane);
    if (win_mask & 16) rate_window<16, PADR, N1, SLIDE>(S, c, m, M, t0, nv, slot_base(4), slot, warp, lane);
    if (win_mask & 32) rate_window<32, PADR, N1, SLIDE>(S, c, m, M, t0, nv, slot_base(5), slot, warp, lane);
  }
  __syncthreads();
  // ---- merge the warps' bests into the tile's running key of each segment ----
  const int ns = slot_base(kMaxWinLog + 1);
  for (int i = threadIdx.x; i < ns; i += N) {
    int l, sg;
    if (!slot_segment<SLIDE>(i, win_mask, us.a.win_mask, us.t0, us.nv, l, sg)) continue;
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
    run[i] = max(run[i], key);
  }
}

// Search kernel over the ranges of a Batch: one unit (baseline, DM trial,
// 32-AP tile) per CTA, or persistent CTAs pulling units from an atomic
// counter (dynamic load balancing across ranges of different sizes).  A
// unit runs every delay residue of its tile in turn and keeps each
// segment's best key in shared memory, so each key is stored once.
template <int N1, int PADR, int FOLD, bool SLIDE>
__global__ void __launch_bounds__(32 * N1, 16 / N1) search_kernel(const __grid_constant__ Batch p) {
  constexpr int N = 32 * N1;
  extern __shared__ __align__(16) float2 sm[];
  float2* S = sm;
  uint2* slot = reinterpret_cast<uint2*>(sm + 32 * (N + 1));
  __shared__ UnitState us;
  __shared__ int s_desc;
  __shared__ long long s_unit;
  __shared__ unsigned long long run[kMaxSegPerTile];
  const bool persistent = p.counter != nullptr;
  long long next = (long long)blockIdx.x + p.unit0;
  for (;;) {
    if (threadIdx.x == 0) {
      const long long u = persistent ? (long long)atomicAdd(p.counter, 1ULL) : next;
      s_unit = u;
      s_desc = u < p.total ? find_desc(p, u) : -1;
    }
    __syncthreads();
    const int di = s_desc;
    if (di < 0) return;
    // copy the range descriptor to shared memory (8-byte words)
    {
      const unsigned long long* src = reinterpret_cast<const unsigned long long*>(&p.d[di]);
      unsigned long long* dst = reinterpret_cast<unsigned long long*>(&us.a);
      for (int i = threadIdx.x; i < (int)(sizeof(SegDesc) / 8); i += N) dst[i] = src[i];
    }
    if (threadIdx.x == 0) {
      const SegDesc& a = p.d[di];
      long long unit = s_unit - a.base;
      // sliding segments: a search of every window w back to back from AP
      // phase phi < w, for each phase (the unit searches the windows wider
      // than its phase)
      int phi = 0;
      if (SLIDE && desc_phases(a.win_mask) > 1) {
        phi = (int)(unit % desc_phases(a.win_mask));
        unit /= desc_phases(a.win_mask);
      }
      us.d = (int)(unit % a.n_dm);
      unit /= a.n_dm;
      const int tile = (int)(unit % a.n_tiles);
      us.b = (int)(unit / a.n_tiles);
      us.t0 = phi + tile * kTile;
      us.nv = a.nvalid[us.d];
      us.valid = us.t0 < us.nv && (!SLIDE || sliding_windows(a.win_mask, us.t0) != 0);
    }
    __syncthreads();
    if (us.valid) {
      const int P = us.a.pad_delay * FOLD;
      const int win_mask = SLIDE ? sliding_windows(us.a.win_mask, us.t0) : us.a.win_mask;
      for (int i = threadIdx.x; i < kMaxSegPerTile; i += N) run[i] = 0ull;
      for (int r = 0; r < P; ++r) {
        if (threadIdx.x == 0) us.r = r;
        __syncthreads();
        search_tile<N1, PADR, FOLD, SLIDE>(us, S, slot, run);
        __syncthreads();
      }
      store_keys<SLIDE>(us, run, win_mask);
    }
    if (!persistent) return;
    __syncthreads();
  }
}

template <int N1, int PADR, int FOLD>
size_t search_smem() {
  return (size_t)32 * (32 * N1 + 1) * sizeof(float2) + (size_t)kMaxSegPerTile * N1 * sizeof(uint2);
}

template <int N1, int PADR, int FOLD, bool SLIDE>
cudaError_t launch_search_t(Batch& b, int grid_ctas, cudaStream_t s, int* n_launch) {
  constexpr int N = 32 * N1;
  const size_t smem = search_smem<N1, PADR, FOLD>();
  cudaError_t e = cudaFuncSetAttribute(search_kernel<N1, PADR, FOLD, SLIDE>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (b.total <= 0) return cudaSuccess;
  if (b.counter) {
    b.unit0 = 0;
    search_kernel<N1, PADR, FOLD, SLIDE><<<(unsigned)std::max(1, grid_ctas), N, smem, s>>>(b);
    ++*n_launch;
    return cudaGetLastError();
  }
  const long long max_grid = 2147483647LL;
  for (long long u0 = 0; u0 < b.total; u0 += max_grid) {
    b.unit0 = u0;
    search_kernel<N1, PADR, FOLD, SLIDE><<<(unsigned)std::min(max_grid, b.total - u0), N, smem, s>>>(b);
    ++*n_launch;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <int N1, int PADR, int FOLD, bool SLIDE>
int occupancy_t() {
  int n = 0;
  if (cudaFuncSetAttribute(search_kernel<N1, PADR, FOLD, SLIDE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)search_smem<N1, PADR, FOLD>()) != cudaSuccess)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, search_kernel<N1, PADR, FOLD, SLIDE>, 32 * N1,
                                                    search_smem<N1, PADR, FOLD>()) != cudaSuccess)
    return 0;
  return n;
}

// Work splits of the bands of 3 * 2^a points (96 .. 1536): mixed-radix
// N1-point FFTs, instantiated in volks_search_mixed{0,4}.cu.
#define VK_MIXED_VARIANTS(X, PADR) \
  X(3, PADR, 1) X(6, PADR, 1) X(12, PADR, 1) X(12, PADR, 2) X(12, PADR, 4)
// Power-of-two work splits; their sliding forms are instantiated in
// volks_search_slide{0,4}.cu.
#define VK_POW2_VARIANTS(X, PADR)                                                      \
  X(2, PADR, 1) X(4, PADR, 1) X(8, PADR, 1) X(16, PADR, 1) X(8, PADR, 2) X(16, PADR, 2) \
  X(8, PADR, 4) X(16, PADR, 4)

#define VK_SEARCH_INST_S(N1, PADR, FOLD, SL)                                                \
  template cudaError_t launch_search_t<N1, PADR, FOLD, SL>(Batch&, int, cudaStream_t, int*); \
  template int occupancy_t<N1, PADR, FOLD, SL>();
#define VK_SEARCH_EXTERN_S(N1, PADR, FOLD, SL)                                                     \
  extern template cudaError_t launch_search_t<N1, PADR, FOLD, SL>(Batch&, int, cudaStream_t, int*); \
  extern template int occupancy_t<N1, PADR, FOLD, SL>();
#define VK_SEARCH_INST(N1, PADR, FOLD) VK_SEARCH_INST_S(N1, PADR, FOLD, false) VK_SEARCH_INST_S(N1, PADR, FOLD, true)
#define VK_SEARCH_EXTERN(N1, PADR, FOLD) \
  VK_SEARCH_EXTERN_S(N1, PADR, FOLD, false) VK_SEARCH_EXTERN_S(N1, PADR, FOLD, true)
#define VK_SEARCH_INST_SLIDE(N1, PADR, FOLD) VK_SEARCH_INST_S(N1, PADR, FOLD, true)
#define VK_SEARCH_EXTERN_SLIDE(N1, PADR, FOLD) VK_SEARCH_EXTERN_S(N1, PADR, FOLD, true)

}  // namespace vk
