// Measurement helper: the FP32 FMA throughput of the device, against which the
// plain-FP32 stages (SIMT MLP, the nearest-neighbour search arithmetic) are
// placed. Every thread runs 16 independent FMA chains; the grid fills every
// SM with 2048 threads, so the FMA pipes, not latency, bound the kernel.
#include "npg_internal.cuh"

namespace npg {

constexpr int PROBE_CHAINS = 16;

__global__ void __launch_bounds__(256) fma_probe_kernel(float* __restrict__ out, int iters,
                                                        float b, float c) {
  float a[PROBE_CHAINS];
#pragma unroll
  for (int j = 0; j < PROBE_CHAINS; ++j) a[j] = (float)(threadIdx.x + j) * 1e-3f;
  for (int k = 0; k < iters; ++k) {
#pragma unroll
    for (int j = 0; j < PROBE_CHAINS; ++j) a[j] = fmaf(a[j], b, c);
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < PROBE_CHAINS; ++j) s += a[j];
  out[(long long)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace npg

extern "C" int npg_fp32_fma_rate(double* tflops, double* ms_out, void* stream) {
  if (!tflops) return npg::set_error_message(NPG_EINVAL, "npg_fp32_fma_rate: tflops is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = sms * 8, threads = 256;
  const int iters = 1 << 19;  // ~65 ms at 80 TFLOP/s
  float* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaMallocAsync(&out, sizeof(float) * (size_t)blocks * threads, s);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float ms = 0.f;
  if (e == cudaSuccess) {
    // b, c keep every chain bounded (a -> c / (1 - b))
    npg::fma_probe_kernel<<<blocks, threads, 0, s>>>(out, iters / 16, 0.999999f, 1e-6f);
    cudaEventRecord(e0, s);
    npg::fma_probe_kernel<<<blocks, threads, 0, s>>>(out, iters, 0.999999f, 1e-6f);
    cudaEventRecord(e1, s);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  }
  if (out) cudaFreeAsync(out, s);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess)
    return npg::set_error_message(NPG_ECUDA, "npg_fp32_fma_rate: %s", cudaGetErrorString(e));
  const double flop = 2.0 * npg::PROBE_CHAINS * (double)iters * blocks * threads;
  *tflops = flop / (ms * 1e-3) / 1e12;
  if (ms_out) *ms_out = ms;
  return cudaStreamSynchronize(s) == cudaSuccess ? NPG_OK
                                                   : npg::set_error_message(NPG_ECUDA, "sync");
}
