// Single-pulse localisation (Sec. 2.3, Eq. 2; baseline rules of Sec. 3.1.2).
// Host code: a pulse has a handful of baselines, so the 2-unknown least
// squares and its leave-one-out repeats are microseconds of CPU work.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "../../include/volks.h"
#include "volks_job.h"

namespace vk {
namespace {

// Least squares of y = [a1 a2] x by modified Gram-Schmidt QR, skipping row
// `skip` (-1: none).  Returns false when the two columns have numerical
// rank < 2.  R (r11, r12, r22) is returned for the covariance.
bool lsq2(const std::vector<double>& a1, const std::vector<double>& a2, const std::vector<double>& y, int skip,
          double x[2], double r[3]) {
  const int n = (int)y.size();
  double n1 = 0.0, n2 = 0.0;
  for (int i = 0; i < n; ++i)
    if (i != skip) {
      n1 += a1[i] * a1[i];
      n2 += a2[i] * a2[i];
    }
  const double r11 = std::sqrt(n1), na2 = std::sqrt(n2);
  if (!(r11 > 0.0)) return false;
  std::vector<double> q1(n, 0.0), v(n, 0.0), yr(n, 0.0);
  double r12 = 0.0, b1 = 0.0;
  for (int i = 0; i < n; ++i)
    if (i != skip) {
      q1[i] = a1[i] / r11;
      r12 += q1[i] * a2[i];
      b1 += q1[i] * y[i];
    }
  double n22 = 0.0;
  for (int i = 0; i < n; ++i)
    if (i != skip) {
      v[i] = a2[i] - r12 * q1[i];
      yr[i] = y[i] - b1 * q1[i];
      n22 += v[i] * v[i];
    }
  const double r22 = std::sqrt(n22);
  if (r22 <= 1e-12 * std::max(r11, na2)) return false;
  double b2 = 0.0;
  for (int i = 0; i < n; ++i)
    if (i != skip) b2 += v[i] / r22 * yr[i];
  x[1] = b2 / r22;
  x[0] = (b1 - r12 * x[1]) / r11;
  r[0] = r11;
  r[1] = r12;
  r[2] = r22;
  return true;
}

// Median as the mean of the two middle values for an even count.
double median(std::vector<double> v) {
  std::sort(v.begin(), v.end());
  const size_t k = v.size();
  return k % 2 ? v[k / 2] : 0.5 * (v[k / 2 - 1] + v[k / 2]);
}

}  // namespace
}  // namespace vk

extern "C" int volks_loc_default_params(volks_loc_params* p) {
  if (!p) return vk::fail(VOLKS_EINVAL, "NULL params");
  p->min_snr = 6.0;
  p->max_proj_len_m = 3.0e6;
  p->min_baselines = 3;
  p->outlier_factor = 5.0;
  return 0;
}

extern "C" int volks_localize(const volks_loc_obs* obs, int32_t n, const volks_loc_params* p,
                              volks_loc_result* out, uint8_t* used_out, double* loo_out) {
  using vk::fail;
  if (!out || !p || n < 0 || (n > 0 && !obs)) return fail(VOLKS_EINVAL, "NULL argument or n < 0");
  if (p->min_baselines < 2) return fail(VOLKS_EINVAL, "min_baselines must be >= 2");
  const double nan = std::nan("");
  std::vector<int> idx;
  for (int i = 0; i < n; ++i) {
    const volks_loc_obs& o = obs[i];
    const bool u = o.snr > p->min_snr && std::fabs(o.proj_len_m) <= p->max_proj_len_m;
    if (u) {
      if (!std::isfinite(o.tau_s) || !std::isfinite(o.tau_cal_s) || !std::isfinite(o.dtau_dalpha) ||
          !std::isfinite(o.dtau_ddelta))
        return fail(VOLKS_EINVAL, "baseline %d: non-finite delay or partial", i);
      idx.push_back(i);
    }
    if (used_out) used_out[i] = u ? 1 : 0;
  }
  if (loo_out)
    for (int i = 0; i < 2 * n; ++i) loo_out[i] = nan;
  *out = volks_loc_result{};
  out->outlier = -1;
  const int m = (int)idx.size();
  out->n_used = m;
  if (m < p->min_baselines) {
    out->status = 1;
    return 0;
  }
  std::vector<double> a1(m), a2(m), y(m);
  for (int k = 0; k < m; ++k) {
    const volks_loc_obs& o = obs[idx[k]];
    a1[k] = o.dtau_dalpha;
    a2[k] = o.dtau_ddelta;
    y[k] = o.tau_s - o.tau_cal_s;
  }
  double x[2], r[3];
  if (!vk::lsq2(a1, a2, y, -1, x, r)) {
    out->status = 2;
    return 0;
  }
  double rss = 0.0;
  for (int k = 0; k < m; ++k) {
    const double e = y[k] - a1[k] * x[0] - a2[k] * x[1];
    rss += e * e;
  }
  const double s2 = m > 2 ? rss / (m - 2) : 0.0;
  // (A^T A)^-1 = R^-1 R^-T
  const double r11 = r[0], r12 = r[1], r22 = r[2];
  const double c01 = -r12 / (r11 * r22 * r22);
  out->cov[0] = s2 * (1.0 / (r11 * r11) + r12 * r12 / (r11 * r11 * r22 * r22));
  out->cov[1] = out->cov[2] = s2 * c01;
  out->cov[3] = s2 / (r22 * r22);
  out->x[0] = out->x_clean[0] = x[0];
  out->x[1] = out->x_clean[1] = x[1];
  out->rms_s = std::sqrt(rss / m);
  if (m >= 3) {
    std::vector<double> l0(m), l1(m);
    bool all_ok = true;
    for (int k = 0; k < m; ++k) {
      double xk[2], rk[3];
      if (vk::lsq2(a1, a2, y, k, xk, rk)) {
        l0[k] = xk[0];
        l1[k] = xk[1];
        if (loo_out) {
          loo_out[2 * idx[k]] = xk[0];
          loo_out[2 * idx[k] + 1] = xk[1];
        }
      } else {
        all_ok = false;
      }
    }
    if (m >= 4 && all_ok) {
      const double m0 = vk::median(l0), m1 = vk::median(l1);
      std::vector<double> d(m);
      int worst = 0;
      for (int k = 0; k < m; ++k) {
        d[k] = std::hypot(l0[k] - m0, l1[k] - m1);
        if (d[k] > d[worst]) worst = k;
      }
      if (d[worst] > p->outlier_factor * vk::median(d)) {
        out->outlier = idx[worst];
        out->x_clean[0] = l0[worst];
        out->x_clean[1] = l1[worst];
      }
    }
  }
  return 0;
}
