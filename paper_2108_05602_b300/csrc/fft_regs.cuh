// Register-resident complex FFTs with compile-time twiddles.
//
// Twiddles W_N^K = exp(-2 pi i K / N) are evaluated at compile time by a
// constexpr power series (after an exact octant reduction of the rational
// angle K / N), so unrolled butterflies multiply by immediates and the
// trivial twiddles (+-1, +-i) cost nothing.
#pragma once
#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

#include "twiddle_ce.h"

namespace vk {

template <int N, int K>
struct Tw {  // W_N^K = exp(-2 pi i K / N)
  static constexpr float re = float(cos2pi(K, N));
  static constexpr float im = float(-sin2pi(K, N));
};

// ---- compile-time loops --------------------------------------------------
template <int B, int E, class F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    static_for<B + 1, E>(f);
  }
}

constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n / 2); }
constexpr int bitrev(int x, int bits) {
  int r = 0;
  for (int i = 0; i < bits; ++i) r |= ((x >> i) & 1) << (bits - 1 - i);
  return r;
}

// ---- complex helpers -----------------------------------------------------
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float cabs2(float2 a) { return fmaf(a.x, a.x, a.y * a.y); }

// v * W_N^K with the trivial and eighth-turn cases specialised.
template <int N, int K>
__device__ __forceinline__ float2 twiddle(float2 v) {
  constexpr int k = ((K % N) + N) % N;
  if constexpr (k == 0) {
    return v;
  } else if constexpr (4 * k == N) {          // -i
    return make_float2(v.y, -v.x);
  } else if constexpr (2 * k == N) {          // -1
    return make_float2(-v.x, -v.y);
  } else if constexpr (4 * k == 3 * N) {      // +i
    return make_float2(-v.y, v.x);
  } else if constexpr (8 * k == N) {          // (1 - i) / sqrt2
    constexpr float c = Tw<8, 1>::re;
    return make_float2((v.x + v.y) * c, (v.y - v.x) * c);
  } else if constexpr (8 * k == 3 * N) {      // (-1 - i) / sqrt2
    constexpr float c = Tw<8, 1>::re;
    return make_float2((v.y - v.x) * c, -(v.x + v.y) * c);
  } else if constexpr (8 * k == 5 * N) {      // (-1 + i) / sqrt2
    constexpr float c = Tw<8, 1>::re;
    return make_float2(-(v.x + v.y) * c, (v.x - v.y) * c);
  } else if constexpr (8 * k == 7 * N) {      // (1 + i) / sqrt2
    constexpr float c = Tw<8, 1>::re;
    return make_float2((v.x - v.y) * c, (v.x + v.y) * c);
  } else {
    constexpr float cr = Tw<N, k>::re, ci = Tw<N, k>::im;
    return make_float2(fmaf(v.x, cr, -v.y * ci), fmaf(v.x, ci, v.y * cr));
  }
}

// In-place radix-2 decimation-in-frequency FFT of N points held in
// registers: natural-order input, output X[k] left at position bitrev(k).
template <int N>
__device__ __forceinline__ void fft_dif(float2 (&x)[N]) {
  constexpr int L = ilog2(N);
  static_for<0, L>([&](auto st) {
    constexpr int half = N >> (decltype(st)::value + 1);
    static_for<0, N / (2 * half)>([&](auto blk) {
      static_for<0, half>([&](auto j) {
        constexpr int i0 = decltype(blk)::value * 2 * half + decltype(j)::value;
        constexpr int i1 = i0 + half;
        const float2 a = x[i0], b = x[i1];
        x[i0] = cadd(a, b);
        x[i1] = twiddle<2 * half, decltype(j)::value>(csub(a, b));
      });
    });
  });
}

template <int N>
__device__ __forceinline__ float2 fft_out(const float2 (&x)[N], int k) { return x[bitrev(k, ilog2(N))]; }

}  // namespace vk
