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

// Complex add and subtract as one packed FP32x2 instruction each (sm_100
// family) when PK: the same IEEE round-to-nearest result per component as
// two scalar operations, in half the issue slots.  The FP32 search kernel
// is issue-bound and takes the packed form throughout; the tensor-core
// kernel measured faster with scalar adds in its delay stage (either half
// packed was 2-5 % slower) and with packed adds in its re-evaluation FFTs.
template <bool PK>
__device__ __forceinline__ float2 cadd_t(float2 a, float2 b) {
  if constexpr (PK) {
    unsigned long long ra, rb, rd;
    asm("mov.b64 %0, {%1, %2};" : "=l"(ra) : "f"(a.x), "f"(a.y));
    asm("mov.b64 %0, {%1, %2};" : "=l"(rb) : "f"(b.x), "f"(b.y));
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(rd) : "l"(ra), "l"(rb));
    float2 d;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(d.x), "=f"(d.y) : "l"(rd));
    return d;
  } else {
    return cadd(a, b);
  }
}
template <bool PK>
__device__ __forceinline__ float2 csub_t(float2 a, float2 b) {
  if constexpr (PK) {
    unsigned long long ra, rb, rd;
    asm("mov.b64 %0, {%1, %2};" : "=l"(ra) : "f"(a.x), "f"(a.y));
    asm("mov.b64 %0, {%1, %2};" : "=l"(rb) : "f"(b.x), "f"(b.y));
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(rd) : "l"(ra), "l"(rb));
    float2 d;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(d.x), "=f"(d.y) : "l"(rd));
    return d;
  } else {
    return csub(a, b);
  }
}
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
template <int N, bool PK = true>
__device__ __forceinline__ void fft_dif(float2 (&x)[N]) {
  constexpr int L = ilog2(N);
  static_for<0, L>([&](auto st) {
    constexpr int half = N >> (decltype(st)::value + 1);
    static_for<0, N / (2 * half)>([&](auto blk) {
      static_for<0, half>([&](auto j) {
        constexpr int i0 = decltype(blk)::value * 2 * half + decltype(j)::value;
        constexpr int i1 = i0 + half;
        const float2 a = x[i0], b = x[i1];
        x[i0] = cadd_t<PK>(a, b);
        x[i1] = twiddle<2 * half, decltype(j)::value>(csub_t<PK>(a, b));
      });
    });
  });
}

template <int N>
__device__ __forceinline__ float2 fft_out(const float2 (&x)[N], int k) { return x[bitrev(k, ilog2(N))]; }

// In-place FFT of N = 3 Q points (Q a power of two) held in registers,
// natural-order output.  Cooley-Tukey with the factor 3 outermost:
//   F_n1[k2]      = sum_{n2<Q} x[3 n2 + n1] W_Q^{n2 k2}          (3 Q-point FFTs)
//   X[k2 + Q k1]  = sum_{n1<3} W_3^{n1 k1} (W_N^{n1 k2} F_n1[k2])  (Q 3-point DFTs)
// with the 3-point DFT of (a, b, c): X0 = a + (b + c),
// X1,2 = a - (b + c)/2 -+ i sin(2 pi/3) (b - c).
template <int N>
__device__ __forceinline__ void fft3_nat(float2 (&x)[N]) {
  static_assert(N % 3 == 0 && ((N / 3) & (N / 3 - 1)) == 0, "N = 3 * 2^a");
  constexpr int Q = N / 3;
  constexpr float h = float(sin2pi(1, 3));
  float2 f[3][Q];
  static_for<0, 3>([&](auto a1) {
    static_for<0, Q>([&](auto a2) {
      f[decltype(a1)::value][decltype(a2)::value] = x[3 * decltype(a2)::value + decltype(a1)::value];
    });
    if constexpr (Q > 1) fft_dif<Q>(f[decltype(a1)::value]);
  });
  static_for<0, Q>([&](auto kk) {
    constexpr int K2 = decltype(kk)::value;
    constexpr int P = bitrev(K2, ilog2(Q));
    const float2 a = f[0][P];
    const float2 b = twiddle<N, K2>(f[1][P]);
    const float2 c = twiddle<N, 2 * K2>(f[2][P]);
    const float2 sum = cadd_t<true>(b, c), dif = csub_t<true>(b, c);
    const float2 t = make_float2(fmaf(-0.5f, sum.x, a.x), fmaf(-0.5f, sum.y, a.y));
    x[K2] = cadd_t<true>(a, sum);
    x[K2 + Q] = make_float2(fmaf(h, dif.y, t.x), fmaf(-h, dif.x, t.y));      // t - i h dif
    x[K2 + 2 * Q] = make_float2(fmaf(-h, dif.y, t.x), fmaf(h, dif.x, t.y));  // t + i h dif
  });
}

}  // namespace vk
