// Re-fit of detected pulses for localisation (Sec. 3.1.2): the
// visibilities that hold a pulse are taken again from the search's
// normalised, calibrated, channel-major copy, summed coherently over the
// pulse's window after removing its fringe rate, and fitted on a finer
// delay grid; the SNR of that coherent sum is what the localisation cuts
// on (SNR > 6).
//
//   refit_kernel  one CTA per candidate: S(k) = sum_u xn[b][k][t0 + u +
//                 shift_d(k)] exp(-2 pi i rate u T_AP) (FP32), then every
//                 cell of G(m) = sum_k S(k) W_Mc^{k m}, Mc = pad n_f, from a
//                 shared-memory twiddle table; peak (lowest cell on ties).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/volks.h"
#include "fft_regs.cuh"
#include "volks_job.h"
#include "volks_result.h"

namespace vk {
namespace {

constexpr int kRefitThreads = 256;

struct RefitJob {
  int b, d, t0, w;
  float rate_cyc_per_ap;   // rate * T_AP
};

__global__ void __launch_bounds__(kRefitThreads) refit_kernel(const float2* __restrict__ xn,
                                                              const int32_t* __restrict__ shifts,
                                                              const RefitJob* __restrict__ jobs,
                                                              const float2* __restrict__ tw, int n_ap, int n_f,
                                                              int Mc, float4* __restrict__ out) {
  extern __shared__ float2 sm[];
  float2* S = sm;          // [n_f]
  float2* T = sm + n_f;    // [Mc]
  __shared__ float s_abs[kRefitThreads];
  __shared__ float s_best[kRefitThreads];
  __shared__ int s_cell[kRefitThreads];
  const RefitJob jb = jobs[blockIdx.x];
  for (int i = threadIdx.x; i < Mc; i += blockDim.x) T[i] = tw[i];
  float abs_sum = 0.f;
  const int32_t* sh = shifts + (size_t)jb.d * n_f;
  for (int k = threadIdx.x; k < n_f; k += blockDim.x) {
    const float2* row = xn + ((size_t)jb.b * n_f + k) * n_ap + jb.t0 + sh[k];
    float2 acc = make_float2(0.f, 0.f);
    for (int u = 0; u < jb.w; ++u) {
      float sn, cs;
      sincospif(-2.f * jb.rate_cyc_per_ap * (float)u, &sn, &cs);
      acc = cadd(acc, cmul(row[u], make_float2(cs, sn)));
    }
    S[k] = acc;
    abs_sum += sqrtf(cabs2(acc));
  }
  s_abs[threadIdx.x] = abs_sum;
  __syncthreads();
  float best = -1.f;
  int bcell = 0;
  for (int m = threadIdx.x; m < Mc; m += blockDim.x) {
    float2 g = make_float2(0.f, 0.f);
    int idx = 0;  // k m mod Mc, advanced by m per point
    for (int k = 0; k < n_f; ++k) {
      g = cadd(g, cmul(S[k], T[idx]));
      idx += m;
      if (idx >= Mc) idx -= Mc;
    }
    const float p = cabs2(g);
    if (p > best) {  // m increases within a thread: keeps the lowest cell on ties
      best = p;
      bcell = m;
    }
  }
  s_best[threadIdx.x] = best;
  s_cell[threadIdx.x] = bcell;
  __syncthreads();
  if (threadIdx.x == 0) {
    float tot = 0.f, bp = -1.f;
    int bm = 0;
    for (int i = 0; i < (int)blockDim.x; ++i) {
      tot += s_abs[i];
      if (s_best[i] > bp || (s_best[i] == bp && s_cell[i] < bm)) {
        bp = s_best[i];
        bm = s_cell[i];
      }
    }
    out[blockIdx.x] = make_float4(bp, __int_as_float(bm), sqrtf(bp), tot);
  }
}

}  // namespace
}  // namespace vk

extern "C" int volks_refit_pulses(volks_result* r, const volks_candidate* cands, int32_t n, int32_t pad,
                                  volks_refit* out) {
  using vk::cuda_fail;
  using vk::fail;
  if (!r || n < 0 || (n > 0 && (!cands || !out))) return fail(VOLKS_EINVAL, "NULL argument or n < 0");
  if (!(pad == 1 || pad == 2 || pad == 4 || pad == 8 || pad == 16 || pad == 32))
    return fail(VOLKS_EINVAL, "pad must be a power of two 1..32");
  const vk::SegJob& j = *r->job;
  const int n_f = j.n_f, Mc = pad * n_f;
  if (Mc > 16384) return fail(VOLKS_EINVAL, "pad * n_f = %d cells: at most 16384", Mc);
  if (n == 0) return 0;
  if (j.empty || !j.d_xn) return fail(VOLKS_EINVAL, "the search holds no data");
  std::vector<vk::RefitJob> jobs(n);
  for (int i = 0; i < n; ++i) {
    const volks_candidate& c = cands[i];
    if (c.bl < 0 || c.bl >= j.seg.n_bl || c.dm_idx < 0 || c.dm_idx >= j.prm.n_dm)
      return fail(VOLKS_EINVAL, "candidate %d: baseline or DM index out of range", i);
    if (c.t0_ap < 0 || c.t1_ap <= c.t0_ap || c.t1_ap > j.nvalid[c.dm_idx] || c.t1_ap - c.t0_ap > 1024)
      return fail(VOLKS_EINVAL, "candidate %d: AP interval [%d, %d) outside the %d dedispersed APs", i, c.t0_ap,
                  c.t1_ap, j.nvalid[c.dm_idx]);
    if (!std::isfinite(c.rate_hz)) return fail(VOLKS_EINVAL, "candidate %d: rate not finite", i);
    jobs[i] = vk::RefitJob{c.bl, c.dm_idx, c.t0_ap, c.t1_ap - c.t0_ap, (float)(c.rate_hz * j.seg.t_ap_s)};
  }
  int rc = vk_sync_result(r);
  if (rc) return rc;
  std::vector<float2> htw(Mc);
  for (int i = 0; i < Mc; ++i)
    htw[i] = make_float2((float)std::cos(2.0 * M_PI * i / Mc), (float)-std::sin(2.0 * M_PI * i / Mc));
  cudaStream_t st = r->stream;
  const size_t smem = (size_t)(n_f + Mc) * sizeof(float2);
  vk::RefitJob* d_jobs = nullptr;
  float2* d_tw = nullptr;
  float4* d_out = nullptr;
  std::vector<float4> h(n);
  cudaError_t e = cudaFuncSetAttribute(vk::refit_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void**>(&d_jobs), n * sizeof(vk::RefitJob), st);
  if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void**>(&d_tw), Mc * sizeof(float2), st);
  if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void**>(&d_out), n * sizeof(float4), st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_jobs, jobs.data(), n * sizeof(vk::RefitJob), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_tw, htw.data(), Mc * sizeof(float2), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    vk::refit_kernel<<<n, vk::kRefitThreads, smem, st>>>(j.d_xn, j.d_shifts, d_jobs, d_tw, j.seg.n_ap, n_f, Mc,
                                                         d_out);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), d_out, n * sizeof(float4), cudaMemcpyDeviceToHost, st);
  if (d_jobs) cudaFreeAsync(d_jobs, st);
  if (d_tw) cudaFreeAsync(d_tw, st);
  if (d_out) cudaFreeAsync(d_out, st);
  const cudaError_t e2 = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) return cuda_fail(e, "pulse re-fit");
  const double bw_hz = j.seg.chan_bw_mhz * 1e6;
  for (int i = 0; i < n; ++i) {
    int m = 0;
    std::memcpy(&m, &h[i].y, sizeof m);
    const int ms = m >= Mc / 2 ? m - Mc : m;
    const int w = jobs[i].w;
    out[i].delay_idx = ms;
    out[i].n_ap = w;
    out[i].delay_s = (double)ms / ((double)Mc * bw_hz);
    out[i].snr = (double)h[i].z / std::sqrt((double)w * j.n_eff);
    out[i].amp = h[i].w > 0.f ? (double)h[i].z / (double)h[i].w : 0.0;
  }
  return 0;
}
