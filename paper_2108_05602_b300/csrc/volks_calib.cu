// Calibration fits (Sec. 2.1): per baseline a coherent integration of a
// strong source's scan and a peak search of its zero-padded delay
// transform.
//
//   initial calibration (Sec. 2.1.1, volks_fringe_fit_calibrator): a
//   calibrator scan, one fit per IF over its J channels, giving the
//   (dtau0^n, dphi0^n) table that the search removes with
//   exp(-i (2 pi f_j dtau0^n + dphi0^n)) (Eq. 1, second line);
//   fine calibration (Sec. 2.1.2, volks_fine_calibration): a reference
//   source near the target, normalised and initially calibrated as the
//   search does (a2, a3), one fit over all n_f points of the band (Eq. 1's
//   single delay across the IFs), giving the residual delay tau_cal.
//
//   calib_sum_kernel  FP64 partial sums over 2048-AP chunks:
//                     part[r][c][k] = sum_t vis[r][t][k] (and sum |vis|^2)
//   calib_fit_kernel  one CTA per (fit, row): S(j) = sum_c part (times the
//                     calibration phasor / RMS for fine calibration), the
//                     delay transform G(m) = sum_j S(j) exp(-2 pi i j m /
//                     (pad J)) evaluated directly in FP64, the peak cell
//                     (lowest on ties), its delay m* / (pad J chan_bw) and
//                     phase arg G(m*) - pi chan_bw dtau (channel centres).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/volks.h"
#include "volks_internal.h"
#include "volks_job.h"

namespace vk {
namespace {

constexpr int kCalChunk = 2048;  // APs per partial sum

__global__ void __launch_bounds__(256) calib_sum_kernel(const float2* __restrict__ vis, double2* __restrict__ part,
                                                        double* __restrict__ pw, int n_ap, int n_f, int n_chunk) {
  const int c = blockIdx.x, b = blockIdx.y;
  const int t0 = c * kCalChunk, t1 = min(n_ap, t0 + kCalChunk);
  const float2* v = vis + (size_t)b * n_ap * n_f;
  for (int k = threadIdx.x; k < n_f; k += blockDim.x) {
    double re = 0.0, im = 0.0, p = 0.0;
    for (int t = t0; t < t1; ++t) {
      const float2 x = v[(size_t)t * n_f + k];
      re += (double)x.x;
      im += (double)x.y;
      if (pw) p = fma((double)x.x, (double)x.x, fma((double)x.y, (double)x.y, p));
    }
    part[((size_t)b * n_chunk + c) * n_f + k] = make_double2(re, im);
    if (pw) pw[((size_t)b * n_chunk + c) * n_f + k] = p;
  }
}

// grid (n_fit, rows); fit n covers points n J .. n J + J - 1.  phasor / pw
// (both or neither): [rows][n_f] calibration phasor, and power partial sums
// [rows][n_chunk][n_f] for the 1 / RMS normalisation.
__global__ void __launch_bounds__(256) calib_fit_kernel(const double2* __restrict__ part,
                                                        const double* __restrict__ pw,
                                                        const double2* __restrict__ phasor, int n_chunk,
                                                        int n_f, int n_ap, int J, int pad, double chan_bw_hz,
                                                        double* __restrict__ out) {
  extern __shared__ double2 sS[];               // [J]
  __shared__ double s_abs[256];
  __shared__ double s_best[256];
  __shared__ int s_cell[256];
  const int n = blockIdx.x, b = blockIdx.y, n_fit = gridDim.x;
  const int Mc = pad * J;
  double abs_sum = 0.0;
  for (int j = threadIdx.x; j < J; j += blockDim.x) {
    const int k = n * J + j;
    double re = 0.0, im = 0.0;
    for (int c = 0; c < n_chunk; ++c) {
      const double2 p = part[((size_t)b * n_chunk + c) * n_f + k];
      re += p.x;
      im += p.y;
    }
    if (phasor) {
      double e = 0.0;
      for (int c = 0; c < n_chunk; ++c) e += pw[((size_t)b * n_chunk + c) * n_f + k];
      const double rms = sqrt(e / (double)n_ap);
      const double g = rms > 0.0 ? 1.0 / rms : 0.0;
      const double2 ph = phasor[(size_t)b * n_f + k];
      const double xr = re * ph.x - im * ph.y, xi = re * ph.y + im * ph.x;
      re = xr * g;
      im = xi * g;
    }
    sS[j] = make_double2(re, im);
    abs_sum += hypot(re, im);
  }
  s_abs[threadIdx.x] = abs_sum;
  __syncthreads();
  // padded delay transform: every thread a set of cells, FP64
  double best = -1.0;
  int bcell = 0;
  for (int m = threadIdx.x; m < Mc; m += blockDim.x) {
    double gr = 0.0, gi = 0.0;
    for (int j = 0; j < J; ++j) {
      double sn, cs;
      sincospi(-2.0 * (double)((long long)j * m % Mc) / (double)Mc, &sn, &cs);
      const double2 s = sS[j];
      gr = fma(s.x, cs, fma(-s.y, sn, gr));
      gi = fma(s.x, sn, fma(s.y, cs, gi));
    }
    const double p = gr * gr + gi * gi;
    if (p > best) {  // m increases within a thread: keeps the lowest cell on ties
      best = p;
      bcell = m;
    }
  }
  s_best[threadIdx.x] = best;
  s_cell[threadIdx.x] = bcell;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0, bp = -1.0;
    int bm = 0;
    for (int i = 0; i < (int)blockDim.x; ++i) {
      tot += s_abs[i];
      if (s_best[i] > bp || (s_best[i] == bp && s_cell[i] < bm)) {
        bp = s_best[i];
        bm = s_cell[i];
      }
    }
    // the peak cell's value, re-evaluated in one fixed order
    double gr = 0.0, gi = 0.0;
    for (int j = 0; j < J; ++j) {
      double sn, cs;
      sincospi(-2.0 * (double)((long long)j * bm % Mc) / (double)Mc, &sn, &cs);
      const double2 s = sS[j];
      gr = fma(s.x, cs, fma(-s.y, sn, gr));
      gi = fma(s.x, sn, fma(s.y, cs, gi));
    }
    const int ms = bm >= Mc / 2 ? bm - Mc : bm;
    const double tau = (double)ms / ((double)Mc * chan_bw_hz);
    double phi = remainder(atan2(gi, gr) - 3.14159265358979323846 * chan_bw_hz * tau, 6.28318530717958647692);
    if (phi <= -3.14159265358979323846) phi += 6.28318530717958647692;
    double* o = out + ((size_t)b * n_fit + n) * 3;
    o[0] = tau;
    o[1] = phi;
    o[2] = tot > 0.0 ? sqrt(gr * gr + gi * gi) / tot : 0.0;
  }
}

// Both entry points: validate, stage the scan, sum, fit; h receives
// [rows][n_fit][3] = {delay, phase, amplitude}.  band: one fit over all
// n_f points with the search's normalisation and initial calibration.
int calib_run(const volks_segment* seg, int32_t pad, void* cuda_stream, bool band, std::vector<double>& h,
              int* rows_out, int* n_fit_out) {
  if (!seg) return fail(VOLKS_EINVAL, "NULL segment");
  if (!(pad == 1 || pad == 2 || pad == 4 || pad == 8)) return fail(VOLKS_EINVAL, "pad must be 1, 2, 4 or 8");
  volks_params prm;
  volks_default_params(&prm);
  int rc = validate(seg, &prm);
  if (rc) return rc;
  const int n_pol = seg->n_pol == 2 ? 2 : 1;
  // the polarisation products are fitted independently: rows = (pol, baseline)
  const int rows = n_pol * seg->n_bl;
  const int n_ap = seg->n_ap, n_if = seg->n_if, n_f = n_if * seg->n_chan;
  const int J = band ? n_f : seg->n_chan, n_fit = n_f / J;
  if (rows > 65535) return fail(VOLKS_EINVAL, "n_pol * n_bl = %d: at most 65535 rows per call", rows);
  if ((long long)pad * J > 16384)
    return fail(VOLKS_EINVAL, "pad * %d points = %lld cells: at most 16384", J, (long long)pad * J);
  *rows_out = rows;
  *n_fit_out = n_fit;
  h.assign((size_t)rows * n_fit * 3, 0.0);
  if ((long long)rows * n_ap == 0) return 0;
  std::vector<double2> hph;
  if (band) {
    hph.resize((size_t)rows * n_f);
    for (int r = 0; r < rows; ++r)
      for (int k = 0; k < n_f; ++k) {
        const int in = k / seg->n_chan, j = k % seg->n_chan;
        double ph = 0.0;
        if (seg->cal) {
          const double fj = (j + 0.5) * seg->chan_bw_mhz * 1e6;
          ph = 2.0 * 3.14159265358979323846 * fj * seg->cal[((size_t)r * n_if + in) * 2] +
               seg->cal[((size_t)r * n_if + in) * 2 + 1];
        }
        hph[(size_t)r * n_f + k] = make_double2(std::cos(ph), -std::sin(ph));
      }
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const bool dev = is_device_pointer(seg->vis);
  const size_t vis_bytes = (size_t)rows * n_ap * n_f * sizeof(float2);
  const int n_chunk = (n_ap + kCalChunk - 1) / kCalChunk;
  void* d_vis = nullptr;
  double2* d_part = nullptr;
  double* d_pw = nullptr;
  double2* d_ph = nullptr;
  double* d_out = nullptr;
  const size_t n_part = (size_t)rows * n_chunk * n_f;
  cudaError_t e = cudaSuccess;
  if (!dev) e = cudaMallocAsync(&d_vis, vis_bytes, st);
  if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void**>(&d_part), n_part * sizeof(double2), st);
  if (e == cudaSuccess && band) e = cudaMallocAsync(reinterpret_cast<void**>(&d_pw), n_part * sizeof(double), st);
  if (e == cudaSuccess && band)
    e = cudaMallocAsync(reinterpret_cast<void**>(&d_ph), hph.size() * sizeof(double2), st);
  if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void**>(&d_out), h.size() * sizeof(double), st);
  if (e == cudaSuccess && !dev) e = cudaMemcpyAsync(d_vis, seg->vis, vis_bytes, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && band)
    e = cudaMemcpyAsync(d_ph, hph.data(), hph.size() * sizeof(double2), cudaMemcpyHostToDevice, st);
  const float2* vis = dev ? static_cast<const float2*>(seg->vis) : static_cast<const float2*>(d_vis);
  if (e == cudaSuccess) {
    calib_sum_kernel<<<dim3(n_chunk, rows), 256, 0, st>>>(vis, d_part, d_pw, n_ap, n_f, n_chunk);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    calib_fit_kernel<<<dim3(n_fit, rows), 256, (size_t)J * sizeof(double2), st>>>(
        d_part, d_pw, d_ph, n_chunk, n_f, n_ap, J, pad, seg->chan_bw_mhz * 1e6, d_out);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), d_out, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (d_vis) cudaFreeAsync(d_vis, st);
  if (d_part) cudaFreeAsync(d_part, st);
  if (d_pw) cudaFreeAsync(d_pw, st);
  if (d_ph) cudaFreeAsync(d_ph, st);
  if (d_out) cudaFreeAsync(d_out, st);
  const cudaError_t e2 = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) return cuda_fail(e, band ? "fine calibration" : "calibrator fringe fit");
  return 0;
}

}  // namespace
}  // namespace vk

extern "C" int volks_fringe_fit_calibrator(const volks_segment* seg, int32_t pad, void* cuda_stream,
                                           double* cal_out, double* amp_out) {
  if (!cal_out) return vk::fail(VOLKS_EINVAL, "NULL output");
  std::vector<double> h;
  int rows = 0, n_fit = 0;
  const int rc = vk::calib_run(seg, pad, cuda_stream, false, h, &rows, &n_fit);
  if (rc) return rc;
  for (size_t i = 0; i < (size_t)rows * n_fit; ++i) {
    cal_out[2 * i] = h[3 * i];
    cal_out[2 * i + 1] = h[3 * i + 1];
    if (amp_out) amp_out[i] = h[3 * i + 2];
  }
  return 0;
}

extern "C" int volks_fine_calibration(const volks_segment* seg, int32_t pad, void* cuda_stream, double* tau_out,
                                      double* amp_out) {
  if (!tau_out) return vk::fail(VOLKS_EINVAL, "NULL output");
  std::vector<double> h;
  int rows = 0, n_fit = 0;
  const int rc = vk::calib_run(seg, pad, cuda_stream, true, h, &rows, &n_fit);
  if (rc) return rc;
  for (int r = 0; r < rows; ++r) {
    tau_out[r] = h[3 * (size_t)r];
    if (amp_out) amp_out[r] = h[3 * (size_t)r + 2];
  }
  return 0;
}
