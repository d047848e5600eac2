// Evaluation metrics of a reconstruction (Sec. 4): per frame, the decoded
// vertices x-hat against ground-truth vertices with the same connectivity
// (known trajectories): bidirectional l2 Chamfer distance, precision /
// recall / F-score at a threshold relative to the ground truth's bounding
// box, normal consistency of nearest pairs (area-weighted vertex normals),
// and the mean correspondence error |x-hat_i - g_i|. The nearest neighbours
// come from the exact bucketed search (k_chamfer.cu); the per-frame sums are
// FP64 partials in a fixed order. Also the per-frame spatial extent that
// keyframe selection rates (Sec. 3.1).
#include <float.h>

#include "npg_internal.cuh"

namespace npg {

// Area-weighted vertex normals of every frame: the sum of the incident faces'
// cross products (vertex -> face lists in a fixed order), normalised.
__global__ void eval_normals_kernel(const float4* __restrict__ v, const int3* __restrict__ faces,
                                    const int* __restrict__ vf_off, const int* __restrict__ vf,
                                    int N, long long NT, float4* __restrict__ nrm) {
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < NT;
       k += (long long)gridDim.x * blockDim.x) {
    const long long base = (k / N) * N;
    const int i = (int)(k - base);
    float nx = 0.f, ny = 0.f, nz = 0.f;
    for (int e = vf_off[i]; e < vf_off[i + 1]; ++e) {
      const int3 f = faces[vf[e]];
      const float4 a = v[base + f.x], b = v[base + f.y], c = v[base + f.z];
      const float ux = b.x - a.x, uy = b.y - a.y, uz = b.z - a.z;
      const float wx = c.x - a.x, wy = c.y - a.y, wz = c.z - a.z;
      nx += uy * wz - uz * wy;
      ny += uz * wx - ux * wz;
      nz += ux * wy - uy * wx;
    }
    const float l = sqrtf(nx * nx + ny * ny + nz * nz);
    const float s = l > 0.f ? 1.f / l : 0.f;
    nrm[k] = make_float4(nx * s, ny * s, nz * s, 0.f);
  }
}

// One block per frame: tau^2 = (tau_rel x bounding-box diagonal of g_t)^2.
__global__ void __launch_bounds__(256) eval_tau_kernel(const float4* __restrict__ g, int N,
                                                       float tau_rel, float* __restrict__ tau2) {
  __shared__ float sh[6][256];
  const float4* gt = g + (long long)blockIdx.x * N;
  float lo[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, hi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const float4 p = gt[i];
    lo[0] = fminf(lo[0], p.x); lo[1] = fminf(lo[1], p.y); lo[2] = fminf(lo[2], p.z);
    hi[0] = fmaxf(hi[0], p.x); hi[1] = fmaxf(hi[1], p.y); hi[2] = fmaxf(hi[2], p.z);
  }
  for (int d = 0; d < 3; ++d) {
    sh[d][threadIdx.x] = lo[d];
    sh[3 + d][threadIdx.x] = hi[d];
  }
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o)
      for (int d = 0; d < 3; ++d) {
        sh[d][threadIdx.x] = fminf(sh[d][threadIdx.x], sh[d][threadIdx.x + o]);
        sh[3 + d][threadIdx.x] = fmaxf(sh[3 + d][threadIdx.x], sh[3 + d][threadIdx.x + o]);
      }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int d = 0; d < 3; ++d) {
      const double e = (double)sh[3 + d][0] - (double)sh[d][0];
      s += e * e;
    }
    const double tau = (double)tau_rel * sqrt(s);
    tau2[blockIdx.x] = (float)(tau * tau);
  }
}

constexpr int EVAL_SPLIT = 8, EVAL_TERMS = 7;

__device__ double eval_block_sum(double v, double* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += sh[w];
  return r;
}

// Grid (T, EVAL_SPLIT): block (t, b) sums a strided share of frame t's
// vertices: d_x, d_g, [d_x < tau^2], [d_g < tau^2], |n_x . n_g(nn)|,
// |n_g . n_x(nn)|, |x - g|.
__global__ void __launch_bounds__(256) eval_frame_kernel(
    const float4* __restrict__ x, const float4* __restrict__ g, const float4* __restrict__ nx,
    const float4* __restrict__ ng, const int* __restrict__ idx_x, const float* __restrict__ d_x,
    const int* __restrict__ idx_g, const float* __restrict__ d_g, const float* __restrict__ tau2,
    int N, double* __restrict__ part) {
  __shared__ double sh[32];
  const int t = blockIdx.x;
  const long long base = (long long)t * N;
  const float tt = tau2[t];
  double acc[EVAL_TERMS] = {0, 0, 0, 0, 0, 0, 0};
  for (int i = blockIdx.y * blockDim.x + threadIdx.x; i < N; i += blockDim.x * EVAL_SPLIT) {
    const long long k = base + i;
    const float dx = d_x[k], dg = d_g[k];
    acc[0] += dx;
    acc[1] += dg;
    acc[2] += dx < tt ? 1.0 : 0.0;
    acc[3] += dg < tt ? 1.0 : 0.0;
    const float4 a = nx[k], b = ng[base + idx_x[k]];
    acc[4] += fabsf(a.x * b.x + a.y * b.y + a.z * b.z);
    const float4 c = ng[k], e = nx[base + idx_g[k]];
    acc[5] += fabsf(c.x * e.x + c.y * e.y + c.z * e.z);
    const float4 p = x[k], q = g[k];
    const float ex = p.x - q.x, ey = p.y - q.y, ez = p.z - q.z;
    acc[6] += sqrtf(ex * ex + ey * ey + ez * ez);
  }
  for (int m = 0; m < EVAL_TERMS; ++m) {
    const double s = eval_block_sum(acc[m], sh);
    if (threadIdx.x == 0) part[((long long)t * EVAL_SPLIT + blockIdx.y) * EVAL_TERMS + m] = s;
  }
}

cudaError_t launch_eval_normals(const float4* v, const int3* faces, const int* vf_off,
                                const int* vf, int N, long long NT, float4* nrm,
                                cudaStream_t s) {
  long long blocks = (NT + 255) / 256;
  if (blocks > 65535LL * 16) blocks = 65535LL * 16;
  eval_normals_kernel<<<(int)blocks, 256, 0, s>>>(v, faces, vf_off, vf, N, NT, nrm);
  return cudaGetLastError();
}

cudaError_t launch_eval_tau(const float4* g, int N, int T, float tau_rel, float* tau2,
                            cudaStream_t s) {
  eval_tau_kernel<<<T, 256, 0, s>>>(g, N, tau_rel, tau2);
  return cudaGetLastError();
}

cudaError_t launch_eval_frames(const float4* x, const float4* g, const float4* nx,
                               const float4* ng, const int* idx_x, const float* d_x,
                               const int* idx_g, const float* d_g, const float* tau2, int N,
                               int T, double* part, cudaStream_t s) {
  eval_frame_kernel<<<dim3(T, EVAL_SPLIT), 256, 0, s>>>(x, g, nx, ng, idx_x, d_x, idx_g, d_g,
                                                        tau2, N, part);
  return cudaGetLastError();
}

// Keyframe selection (Sec. 3.1): one block per frame computes the RMS radius
// of the frame's points about their centroid in FP64, in two passes (the
// centroid, then the squared distances), each a strided per-thread sum and a
// block reduction. off: T + 1 offsets into pts (x, y, z per point).
__global__ void __launch_bounds__(256) keyframe_extent_kernel(const float* __restrict__ pts,
                                                              const long long* __restrict__ off,
                                                              double* __restrict__ extent) {
  __shared__ double sh[32];
  __shared__ double cen[3];
  const long long a = off[blockIdx.x], b = off[blockIdx.x + 1];
  const double n = (double)(b - a);
  double s[3] = {0.0, 0.0, 0.0};
  for (long long j = a + threadIdx.x; j < b; j += blockDim.x)
    for (int d = 0; d < 3; ++d) s[d] += (double)pts[3 * j + d];
  for (int d = 0; d < 3; ++d) {
    const double r = eval_block_sum(s[d], sh);
    if (threadIdx.x == 0) cen[d] = r / n;
  }
  __syncthreads();
  double s2 = 0.0;
  for (long long j = a + threadIdx.x; j < b; j += blockDim.x)
    for (int d = 0; d < 3; ++d) {
      const double u = (double)pts[3 * j + d] - cen[d];
      s2 += u * u;
    }
  const double r = eval_block_sum(s2, sh);
  if (threadIdx.x == 0) extent[blockIdx.x] = sqrt(r / n);
}

cudaError_t launch_keyframe_extent(const float* pts, const long long* off, int T, double* extent,
                                   cudaStream_t s) {
  keyframe_extent_kernel<<<T, 256, 0, s>>>(pts, off, extent);
  return cudaGetLastError();
}

int eval_split() { return EVAL_SPLIT; }
int eval_terms() { return EVAL_TERMS; }

}  // namespace npg
