// Compile-time sine / cosine of the rational angle 2 pi k / n, used to build
// FFT twiddles as immediates.  Plain C++17 (also compiled by the host tests).
#pragma once

namespace vk {

constexpr double kPi = 3.141592653589793238462643383279502884;

// Maclaurin series of sin and cos, for |x| <= pi/4 (truncation < 1e-25).
constexpr double series_sin(double x) {
  double t = x, s = x;
  for (int i = 1; i < 16; ++i) {
    t *= -x * x / double((2 * i) * (2 * i + 1));
    s += t;
  }
  return s;
}
constexpr double series_cos(double x) {
  double t = 1.0, s = 1.0;
  for (int i = 1; i < 16; ++i) {
    t *= -x * x / double((2 * i - 1) * (2 * i));
    s += t;
  }
  return s;
}

// Exact reduction of k/n (mod 1) to the nearest quarter turn qraw/4
// (qraw in 0..4) plus a residual angle 2 pi (k/n - qraw/4) in [-pi/4, pi/4].
constexpr long long mod_pos(long long a, long long n) { return ((a % n) + n) % n; }
constexpr long long quarter_turns(long long k, long long n) {
  return (8 * mod_pos(k, n) + n) / (2 * n);
}
constexpr double residual(long long k, long long n) {
  return kPi * double(4 * mod_pos(k, n) - quarter_turns(k, n) * n) / double(2 * n);
}
constexpr double cos2pi(long long k, long long n) {
  const double x = residual(k, n);
  switch (quarter_turns(k, n) % 4) {
    case 0: return series_cos(x);
    case 1: return -series_sin(x);
    case 2: return -series_cos(x);
    default: return series_sin(x);
  }
}
constexpr double sin2pi(long long k, long long n) {
  const double x = residual(k, n);
  switch (quarter_turns(k, n) % 4) {
    case 0: return series_sin(x);
    case 1: return series_cos(x);
    case 2: return -series_sin(x);
    default: return -series_cos(x);
  }
}

}  // namespace vk
