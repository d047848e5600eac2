// Allocation-free variant of the standalone Sobolev preconditioner.
//
// Some callers cannot allocate device memory at the point where they need the
// preconditioner: a process whose GPU memory is already owned by another
// allocator (a framework's caching pool that reserved the device), a loop with
// a fixed memory budget, or code that must not risk the implicit device
// synchronisation of cudaMalloc / cudaFree. npg_precondition_static serves them
// from one file-scope device array of fixed size instead of per-call scratch.
#include <mutex>

#include "npg_internal.cuh"

#define NPG_PC_STATIC_MAX_ELEMS (1 << 20)
// r^3 * F <= 2^20 with F >= 1 caps r at floor(cbrt(2^20)) = 101
#define NPG_PC_STATIC_MAX_R 101
#define NPG_PC_STATIC_TABLE (2 * NPG_PC_STATIC_MAX_R * NPG_PC_STATIC_MAX_R + NPG_PC_STATIC_MAX_R)

// Two transform buffers of NPG_PC_STATIC_MAX_ELEMS floats, then the DCT
// tables of one level (C, C^T, mu). Every GPU that loads this library holds
// this array (about 8.5 MB) until the process exits.
static __device__ __align__(256) float g_pc_scratch[2 * NPG_PC_STATIC_MAX_ELEMS +
                                                     NPG_PC_STATIC_TABLE];

namespace npg {

// C[k][n] = a_k cos(pi k (2n+1) / 2r), C^T, mu_k = 2 - 2 cos(pi k / r), in FP64.
__global__ void dct_tables_kernel(float* C, float* Ct, float* mu, int r) {
  const double pi = 3.14159265358979323846;
  const long long rr = (long long)r * r;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < rr;
       e += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(e / r), n = (int)(e % r);
    const double a = k == 0 ? sqrt(1.0 / r) : sqrt(2.0 / r);
    const float v = (float)(a * cos(pi * k * (2.0 * n + 1.0) / (2.0 * r)));
    C[(long long)k * r + n] = v;
    Ct[(long long)n * r + k] = v;
    if (n == 0) mu[k] = (float)(2.0 - 2.0 * cos(pi * k / r));
  }
}

}  // namespace npg

static std::mutex g_pc_mutex;
// Device address of g_pc_scratch, per device ordinal, looked up once per
// process: it stays valid as long as the device's primary context does (a
// cudaDeviceReset invalidates it; the header says so).
static float* g_pc_addr[256];

extern "C" int npg_precondition_static(const float* g, float* out, int r, int F, float lambda,
                                       void* stream) {
  if (!g || !out || r < 2 || F < 1 || F > NPG_MAX_F || !(lambda >= 0.f))
    return npg::set_error_message(NPG_EINVAL,
                                  "npg_precondition_static: bad arguments (r=%d F=%d)", r, F);
  const long long n = (long long)r * r * r * F;
  if (r > NPG_PC_STATIC_MAX_R || n > NPG_PC_STATIC_MAX_ELEMS)
    return npg::set_error_message(
        NPG_EINVAL,
        "npg_precondition_static: r^3 * F = %lld exceeds the static scratch limit of %d "
        "(r <= %d); use npg_precondition",
        n, NPG_PC_STATIC_MAX_ELEMS, NPG_PC_STATIC_MAX_R);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 256)
    return npg::set_error_message(NPG_ECUDA, "npg_precondition_static: cudaGetDevice: %s",
                                  cudaGetErrorString(e));
  float* base = nullptr;
  {
    // set-up, once per device, with that device current: the host-side name
    // of the array is not a device address
    std::lock_guard<std::mutex> lk(g_pc_mutex);
    if (!g_pc_addr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_pc_scratch);
      if (e != cudaSuccess || !p)
        return npg::set_error_message(NPG_ECUDA,
                                      "npg_precondition_static: cudaGetSymbolAddress: %s",
                                      cudaGetErrorString(e));
      g_pc_addr[dev] = static_cast<float*>(p);
    }
    base = g_pc_addr[dev];
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float* t0 = base;
  float* t1 = base + NPG_PC_STATIC_MAX_ELEMS;
  float* C = base + 2 * NPG_PC_STATIC_MAX_ELEMS;
  float* Ct = C + (long long)r * r;
  float* mu = Ct + (long long)r * r;
  // every element a pass reads is written earlier in this call: nothing in the
  // array has to start at zero
  const long long rr = (long long)r * r;
  npg::dct_tables_kernel<<<(int)((rr + 255) / 256), 256, 0, s>>>(C, Ct, mu, r);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = npg::launch_precondition(g, out, t0, t1, C, Ct, mu, r, F, lambda, s);
  if (e != cudaSuccess)
    return npg::set_error_message(NPG_ECUDA, "npg_precondition_static: %s", cudaGetErrorString(e));
  return NPG_OK;
}
