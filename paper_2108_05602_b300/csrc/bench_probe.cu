// Benchmark helper, built into its own library (libvolks_bench.so) and
// loaded by the benchmark only; not part of the search library's C ABI.
//
// FP32 FMA throughput of the device: the denominator of the FP32 search
// kernel's roofline, measured rather than derived from the lane count and
// clock.  Every thread runs 8 independent FMA chains (enough to cover the
// FMA latency with 16 warps per SM); one launch covers every SM.
//
//   int bench_fp32_fma_tflops(void *cuda_stream, double *tflops);
//
// times two launches (the first warms up) with CUDA events on cuda_stream
// and returns 0, or a CUDA error code (nonzero) on failure.
#include <cstdint>

#include <cuda_runtime.h>


namespace vk {
namespace {

constexpr int kProbeThreads = 512;
constexpr int kProbeUnroll = 16;

__global__ void __launch_bounds__(kProbeThreads) fma_probe_kernel(float* out, int iters, float a, float b) {
  float x[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) x[c] = 1e-6f * (float)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kProbeUnroll; ++k) {
#pragma unroll
      for (int c = 0; c < 8; ++c) x[c] = fmaf(x[c], a, b);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < 8; ++c) s += x[c];
  if (s == 1234.5f) out[blockIdx.x] = s;  // keeps the chains live; never true for a = 0.999, b = 1e-4
}

}  // namespace
}  // namespace vk

extern "C" int bench_fp32_fma_tflops(void* cuda_stream, double* tflops) {
  if (!tflops) return (int)cudaErrorInvalidValue;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0, n_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return (int)e;
  const int blocks = 2 * n_sm, iters = 4096;
  float* d_out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if ((e = cudaMallocAsync(reinterpret_cast<void**>(&d_out), blocks * sizeof(float), st)) != cudaSuccess)
    return (int)e;
  e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float ms = 0.f;
  for (int rep = 0; e == cudaSuccess && rep < 2; ++rep) {  // the first launch warms up
    e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) {
      vk::fma_probe_kernel<<<blocks, vk::kProbeThreads, 0, st>>>(d_out, iters, 0.999f, 1e-4f);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  }
  cudaFreeAsync(d_out, st);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return (int)e;
  const double flops = 2.0 * 8 * vk::kProbeUnroll * (double)iters * vk::kProbeThreads * blocks;
  *tflops = ms > 0.f ? flops / (ms * 1e-3) / 1e12 : 0.0;
  return 0;
}
