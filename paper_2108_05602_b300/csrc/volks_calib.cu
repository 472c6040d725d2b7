// Initial calibration (Sec. 2.1.1): fringe fit of a strong calibrator scan,
// per baseline and IF, giving the (dtau0^n, dphi0^n) table that the search
// removes with exp(-i (2 pi f_j dtau0^n + dphi0^n)) (Eq. 1, second line).
//
//   calib_sum_kernel  coherent integration over the scan in FP64:
//                     part[b][c][k] = sum_{t in chunk c} vis[b][t][k]
//   calib_fit_kernel  one CTA per (IF, baseline): S(j) = sum_c part, the
//                     delay transform over the IF's J channels zero-padded by
//                     `pad` (Sec. 2.2), G(m) = sum_j S(j) exp(-2 pi i j m /
//                     (pad J)), the peak cell (lowest on ties), the delay
//                     m* / (pad J chan_bw) and the phase arg G(m*) - pi
//                     chan_bw dtau0 (channel-centre frequencies), FP64.
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
                                                        int n_ap, int n_f, int n_chunk) {
  const int c = blockIdx.x, b = blockIdx.y;
  const int t0 = c * kCalChunk, t1 = min(n_ap, t0 + kCalChunk);
  const float2* v = vis + (size_t)b * n_ap * n_f;
  for (int k = threadIdx.x; k < n_f; k += blockDim.x) {
    double re = 0.0, im = 0.0;
    for (int t = t0; t < t1; ++t) {
      const float2 x = v[(size_t)t * n_f + k];
      re += (double)x.x;
      im += (double)x.y;
    }
    part[((size_t)b * n_chunk + c) * n_f + k] = make_double2(re, im);
  }
}

__global__ void __launch_bounds__(256) calib_fit_kernel(const double2* __restrict__ part, int n_chunk, int n_f,
                                                        int n_chan, int pad, double chan_bw_hz,
                                                        double* __restrict__ out) {
  extern __shared__ double2 sS[];               // [n_chan]
  __shared__ double s_abs[256];
  __shared__ double s_best[256];
  __shared__ int s_cell[256];
  const int n = blockIdx.x, b = blockIdx.y, n_if = gridDim.x;
  const int J = n_chan, Mc = pad * J;
  double abs_sum = 0.0;
  for (int j = threadIdx.x; j < J; j += blockDim.x) {
    double re = 0.0, im = 0.0;
    for (int c = 0; c < n_chunk; ++c) {
      const double2 p = part[((size_t)b * n_chunk + c) * n_f + n * J + j];
      re += p.x;
      im += p.y;
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
    double* o = out + ((size_t)b * n_if + n) * 3;
    o[0] = tau;
    o[1] = phi;
    o[2] = tot > 0.0 ? sqrt(gr * gr + gi * gi) / tot : 0.0;
  }
}

}  // namespace
}  // namespace vk

extern "C" int volks_fringe_fit_calibrator(const volks_segment* seg, int32_t pad, void* cuda_stream,
                                           double* cal_out, double* amp_out) {
  using vk::cuda_fail;
  using vk::fail;
  if (!seg || !cal_out) return fail(VOLKS_EINVAL, "NULL segment or output");
  if (!(pad == 1 || pad == 2 || pad == 4 || pad == 8)) return fail(VOLKS_EINVAL, "pad must be 1, 2, 4 or 8");
  volks_params prm;
  volks_default_params(&prm);
  int rc = vk::validate(seg, &prm);
  if (rc) return rc;
  // the polarisation products are fitted independently: rows = (pol, baseline)
  const int n_bl = (seg->n_pol == 2 ? 2 : 1) * seg->n_bl;
  const int n_ap = seg->n_ap, n_if = seg->n_if, J = seg->n_chan, n_f = n_if * J;
  if (n_bl > 65535) return fail(VOLKS_EINVAL, "n_pol * n_bl = %d: at most 65535 rows per call", n_bl);
  if ((long long)pad * J > 16384) return fail(VOLKS_EINVAL, "pad * n_chan = %lld cells: at most 16384", (long long)pad * J);
  const size_t n_out = (size_t)n_bl * n_if;
  if ((long long)n_bl * n_ap == 0) {
    for (size_t i = 0; i < n_out; ++i) {
      cal_out[2 * i] = cal_out[2 * i + 1] = 0.0;
      if (amp_out) amp_out[i] = 0.0;
    }
    return 0;
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  cudaPointerAttributes attr{};
  if (cudaPointerGetAttributes(&attr, seg->vis) != cudaSuccess) {
    cudaGetLastError();
    attr.type = cudaMemoryTypeUnregistered;
  }
  const bool dev = attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
  const size_t vis_bytes = (size_t)n_bl * n_ap * n_f * sizeof(float2);
  const int n_chunk = (n_ap + vk::kCalChunk - 1) / vk::kCalChunk;
  void* d_vis = nullptr;
  double2* d_part = nullptr;
  double* d_out = nullptr;
  cudaError_t e = cudaSuccess;
  if (!dev) e = cudaMallocAsync(&d_vis, vis_bytes, st);
  if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void**>(&d_part), (size_t)n_bl * n_chunk * n_f * sizeof(double2), st);
  if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void**>(&d_out), n_out * 3 * sizeof(double), st);
  if (e == cudaSuccess && !dev) e = cudaMemcpyAsync(d_vis, seg->vis, vis_bytes, cudaMemcpyHostToDevice, st);
  const float2* vis = dev ? static_cast<const float2*>(seg->vis) : static_cast<const float2*>(d_vis);
  if (e == cudaSuccess) {
    vk::calib_sum_kernel<<<dim3(n_chunk, n_bl), 256, 0, st>>>(vis, d_part, n_ap, n_f, n_chunk);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    vk::calib_fit_kernel<<<dim3(n_if, n_bl), 256, (size_t)J * sizeof(double2), st>>>(
        d_part, n_chunk, n_f, J, pad, seg->chan_bw_mhz * 1e6, d_out);
    e = cudaGetLastError();
  }
  std::vector<double> h(n_out * 3);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), d_out, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (d_vis) cudaFreeAsync(d_vis, st);
  if (d_part) cudaFreeAsync(d_part, st);
  if (d_out) cudaFreeAsync(d_out, st);
  const cudaError_t e2 = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) return cuda_fail(e, "calibrator fringe fit");
  for (size_t i = 0; i < n_out; ++i) {
    cal_out[2 * i] = h[3 * i];
    cal_out[2 * i + 1] = h[3 * i + 1];
    if (amp_out) amp_out[i] = h[3 * i + 2];
  }
  return 0;
}
