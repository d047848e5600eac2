// FP32 SIMT MLP decode and backward (Sec. 3.3-3.4) for hidden widths beyond
// 64 (multiples of 32 up to 512, the paper's own width): the rows are
// processed in chunks of at most WIDE_CHUNK, layer by layer, with the chunk's
// activations kept in a scratch area of the context, so that each layer is a
// tiled FP32 GEMM with its elementwise work fused into the epilogue:
//   forward      h1 = act(U_i + V_t); h_l = act(h_{l-1} W_l^T + b_l);
//                o = h_D Wo^T + bo and Eq. 5-7 (x-hat) or, in the backward
//                pass, dL/do (their Jacobians) and dpre_D = (dL/do Wo) act'(h_D)
//   backward     dW_l += dpre_l^T h_{l-1}, db_l += column sums of dpre_l,
//                dpre_{l-1} = (dpre_l W_l) act'(h_{l-1}); dWo += dL/do^T h_D;
//                dW1 += dpre_1^T y, y = (z_i, gamma_t); dL/dz_i += dpre_1 W1[:, :Z]
// Weight-gradient GEMMs reduce over the chunk's rows in slices, one atomic add
// per output value and slice.
#include <algorithm>
#include <utility>

#include "npg_device.cuh"
#include "npg_internal.cuh"

namespace npg {

namespace {
constexpr int GBM = 128, GBN = 128, GBK = 16;
constexpr int TN_SLICE = 1024;  // rows per block of a weight-gradient GEMM

enum { G_NT_ACT = 0, G_NN_DACT = 1, G_TN_ADD = 2, G_NN_DZ = 3 };

struct GemmArgs {
  const float* A;
  const float* B;
  float* Y;
  const float* bias;  // G_NT_ACT
  const float* Hin;   // G_NN_DACT: the layer input's activation (post-LeakyReLU)
  int M, N, K;
  int lda, ldb, ldy, ldh;
  float slope;
  long long r0;       // G_NN_DZ: global row of the chunk's first row
  int nvert;          // G_NN_DZ: N vertices (row r belongs to vertex r mod N)
};

// One 128 x 128 output tile per block, 16-deep K steps, 8 x 8 outputs per
// thread at rows ty + 16 i and columns tx + 16 j.
//   G_NT_ACT   Y = act(A B^T + bias)          A: M x K, B: N x K (row-major)
//   G_NN_DACT  Y = (A B) act'(Hin)            A: M x K, B: K x N
//   G_TN_ADD   Y += A^T B (atomic)            A: K x M, B: K x N; K sliced by blockIdx.z
//   G_NN_DZ    dz[(r0 + m) mod nvert] += A B  A: M x K, B: K x N
template <int MODE>
__global__ void __launch_bounds__(256) wide_gemm_kernel(GemmArgs p) {
  __shared__ float As[GBK][GBM + 4];
  __shared__ float Bs[GBK][GBN + 4];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;
  int kb = 0, ke = p.K;
  if (MODE == G_TN_ADD) {
    kb = blockIdx.z * TN_SLICE;
    ke = min(p.K, kb + TN_SLICE);
  }
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
  for (int k0 = kb; k0 < ke; k0 += GBK) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int e = tid + 256 * q;
      if (MODE == G_TN_ADD) {
        const int kk = e >> 7, mm = e & 127;
        const int k = k0 + kk, m = m0 + mm;
        As[kk][mm] = (k < ke && m < p.M) ? p.A[(long long)k * p.lda + m] : 0.f;
      } else {
        const int mm = e >> 4, kk = e & 15;
        const int k = k0 + kk, m = m0 + mm;
        As[kk][mm] = (k < ke && m < p.M) ? p.A[(long long)m * p.lda + k] : 0.f;
      }
      if (MODE == G_NT_ACT) {
        const int nn = e >> 4, kk = e & 15;
        const int k = k0 + kk, n = n0 + nn;
        Bs[kk][nn] = (k < ke && n < p.N) ? p.B[(long long)n * p.ldb + k] : 0.f;
      } else {
        const int kk = e >> 7, nn = e & 127;
        const int k = k0 + kk, n = n0 + nn;
        Bs[kk][nn] = (k < ke && n < p.N) ? p.B[(long long)k * p.ldb + n] : 0.f;
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GBK; ++kk) {
      float a[8], b[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 8; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int m = m0 + ty + 16 * i;
    if (m >= p.M) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int n = n0 + tx + 16 * j;
      if (n >= p.N) continue;
      const float v = acc[i][j];
      if (MODE == G_NT_ACT)
        p.Y[(long long)m * p.ldy + n] = leaky(v + p.bias[n], p.slope);
      else if (MODE == G_NN_DACT)
        p.Y[(long long)m * p.ldy + n] = v * dleaky_h(p.Hin[(long long)m * p.ldh + n], p.slope);
      else if (MODE == G_TN_ADD)
        atomicAdd(p.Y + (long long)m * p.ldy + n, v);
      else
        atomicAdd(p.Y + ((p.r0 + m) % p.nvert) * p.ldy + n, v);
    }
  }
}

template <int MODE>
cudaError_t gemm(const GemmArgs& p, cudaStream_t s) {
  if (p.M <= 0 || p.N <= 0 || p.K <= 0) return cudaSuccess;
  dim3 grid((p.N + GBN - 1) / GBN, (p.M + GBM - 1) / GBM,
            MODE == G_TN_ADD ? (p.K + TN_SLICE - 1) / TN_SLICE : 1);
  wide_gemm_kernel<MODE><<<grid, 256, 0, s>>>(p);
  return cudaGetLastError();
}

// h1 = act(U_i + V_t) of rows [r0, r0 + rows) (row r = t N + i) into act0.
__global__ void wide_h1_kernel(const float* __restrict__ U, const float* __restrict__ V,
                               float* __restrict__ act0, long long r0, int rows, int N, int H,
                               float slope) {
  const int H4 = H / 4;
  const long long n4 = (long long)rows * H4;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n4;
       e += (long long)gridDim.x * blockDim.x) {
    const long long rr = e / H4;
    const int k4 = (int)(e - rr * H4);
    const long long row = r0 + rr;
    const int t = (int)(row / N), i = (int)(row - (long long)t * N);
    const float4 u = reinterpret_cast<const float4*>(U + (long long)i * H)[k4];
    const float4 v = reinterpret_cast<const float4*>(V + (long long)t * H)[k4];
    reinterpret_cast<float4*>(act0 + rr * H)[k4] =
        make_float4(leaky(u.x + v.x, slope), leaky(u.y + v.y, slope), leaky(u.z + v.z, slope),
                    leaky(u.w + v.w, slope));
  }
}

// One warp per row: o = Wo h_D + bo (lane l holds features l + 32 k), then
// either Eq. 5-7 (x-hat, displacement) or dL/do (their Jacobians) with
// dpre_D = (dL/do Wo) act'(h_D). Wo and bo live in shared memory.
template <int ROT, bool BACKWARD>
__global__ void __launch_bounds__(256) wide_out_kernel(
    const float* __restrict__ mlp_out, const float* __restrict__ hD, const float4* __restrict__ xr,
    float4* __restrict__ xhat, float4* __restrict__ disp, const float4* __restrict__ dxhat,
    float* __restrict__ go_out, float* __restrict__ dp_out, long long r0, int rows, int N, int H,
    int NO, float slope, float alpha) {
  extern __shared__ float wo[];  // NO x H, then bo (NO)
  for (int k = threadIdx.x; k < NO * H + NO; k += blockDim.x) wo[k] = mlp_out[k];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int warps = (int)(gridDim.x * blockDim.x / 32);
  const int nk = H / 32;
  for (int rr = (int)((blockIdx.x * blockDim.x + threadIdx.x) / 32); rr < rows; rr += warps) {
    const long long row = r0 + rr;
    const int t = (int)(row / N), i = (int)(row - (long long)t * N);
    const float* h = hD + (long long)rr * H;
    float o[7];
#pragma unroll
    for (int q = 0; q < 7; ++q) {
      float s = 0.f;
      if (q < NO)
        for (int k = 0; k < nk; ++k) s = fmaf(wo[q * H + lane + 32 * k], h[lane + 32 * k], s);
#pragma unroll
      for (int o2 = 16; o2 > 0; o2 >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o2);
      o[q] = q < NO ? s + wo[NO * H + q] : 0.f;
    }
    if (!BACKWARD) {
      if (lane == 0) {
        float4 xh, dl;
        transform<ROT>(o, alpha, xr[i], xh, dl);
        xhat[row] = xh;
        disp[row] = dl;
      }
    } else {
      float go[7];
#pragma unroll
      for (int q = 0; q < 7; ++q) go[q] = 0.f;
      transform_backward<ROT>(o, alpha, xr[i], dxhat[row], go);
      float gl = 0.f;
#pragma unroll
      for (int q = 0; q < 7; ++q)
        if (lane == q && q < NO) gl = go[q];
      if (lane < 8) go_out[(long long)rr * 8 + lane] = gl;
      for (int k = 0; k < nk; ++k) {
        const int m = lane + 32 * k;
        float s = 0.f;
#pragma unroll
        for (int q = 0; q < 7; ++q)
          if (q < NO) s = fmaf(wo[q * H + m], go[q], s);
        dp_out[(long long)rr * H + m] = s * dleaky_h(h[m], slope);
      }
    }
  }
}

// Column sums over rows: out[n] += sum_m A[m][n] (n < ncol, A row-major, lda).
__global__ void wide_colsum_kernel(const float* __restrict__ A, float* __restrict__ out, int rows,
                                   int ncol, int lda) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= ncol) return;
  const int per = (rows + gridDim.y - 1) / gridDim.y;
  const int b = blockIdx.y * per, e = min(rows, b + per);
  float s = 0.f;
  for (int m = b; m < e; ++m) s += A[(long long)m * lda + n];
  if (e > b) atomicAdd(out + n, s);
}

cudaError_t colsum(const float* A, float* out, int rows, int ncol, int lda, cudaStream_t s) {
  dim3 grid((ncol + 127) / 128, (unsigned)max(1, min(256, rows / 512)));
  wide_colsum_kernel<<<grid, 128, 0, s>>>(A, out, rows, ncol, lda);
  return cudaGetLastError();
}

// Per-frame column sums: dV[t][n] += sum of A[m][n] over the chunk's rows m of
// frame t = (r0 + m) / N (rows are frame-major, so a slice of rows spans few
// frames; one atomic add per column and frame met).
__global__ void wide_frame_colsum_kernel(const float* __restrict__ A, float* __restrict__ dV,
                                         long long r0, int rows, int N, int H) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= H) return;
  const int per = (rows + gridDim.y - 1) / gridDim.y;
  const int b = blockIdx.y * per, e = min(rows, b + per);
  if (b >= e) return;
  long long t = (r0 + b) / N;
  float s = 0.f;
  for (int m = b; m < e; ++m) {
    const long long tm = (r0 + m) / N;
    if (tm != t) {
      atomicAdd(dV + t * H + n, s);
      s = 0.f;
      t = tm;
    }
    s += A[(long long)m * H + n];
  }
  atomicAdd(dV + t * H + n, s);
}

// y = (z_i, gamma_t) of the chunk's rows, K wide.
__global__ void wide_y_kernel(const float* __restrict__ z, const float* __restrict__ gamma,
                              float* __restrict__ y, long long r0, int rows, int N, int Z, int K) {
  const long long n = (long long)rows * K;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const long long rr = e / K;
    const int k = (int)(e - rr * K);
    const long long row = r0 + rr;
    const int t = (int)(row / N), i = (int)(row - (long long)t * N);
    y[e] = k < Z ? z[(long long)i * Z + k] : gamma[(long long)t * (K - Z) + (k - Z)];
  }
}

int grid1d(long long n, int threads, int num_sms) {
  long long b = (n + threads - 1) / threads;
  return (int)std::max(1LL, std::min(b, (long long)num_sms * 16));
}

struct WideLayout {  // offsets (floats) of the chunk buffers in c->wide
  long long act, dp0, dp1, go, y;
};

WideLayout wide_layout(const npg_ctx* c) {
  const long long C = c->wide_rows, H = c->md.H;
  WideLayout w;
  w.act = 0;
  w.dp0 = w.act + (long long)c->md.D * C * H;
  w.dp1 = w.dp0 + C * H;
  w.go = w.dp1 + C * H;
  w.y = w.go + C * 8;
  return w;
}

template <int ROT>
cudaError_t wide_out(npg_ctx* c, bool backward, const float* hD, float* go, float* dp, long long r0,
                     int rows, cudaStream_t s) {
  const MlpDims& md = c->md;
  const float* po = c->mlp + (long long)md.H * md.K + md.H +
                    (long long)(md.D - 1) * (md.H * md.H + md.H);
  const size_t smem = sizeof(float) * ((size_t)md.NO * md.H + md.NO);
  const int blocks = grid1d((long long)rows * 32, 256, c->num_sms);
  if (backward)
    wide_out_kernel<ROT, true><<<blocks, 256, smem, s>>>(po, hD, c->xr, c->xhat, c->disp,
                                                         c->dxhat, go, dp, r0, rows, c->N, md.H,
                                                         md.NO, md.slope, c->cfg.alpha);
  else
    wide_out_kernel<ROT, false><<<blocks, 256, smem, s>>>(po, hD, c->xr, c->xhat, c->disp,
                                                          c->dxhat, go, dp, r0, rows, c->N, md.H,
                                                          md.NO, md.slope, c->cfg.alpha);
  return cudaGetLastError();
}

cudaError_t wide_out_rot(npg_ctx* c, bool backward, const float* hD, float* go, float* dp,
                         long long r0, int rows, cudaStream_t s) {
  switch (c->cfg.rot_mode) {
    case NPG_ROT_QUAT: return wide_out<0>(c, backward, hD, go, dp, r0, rows, s);
    case NPG_ROT_EXPMAP: return wide_out<1>(c, backward, hD, go, dp, r0, rows, s);
    default: return wide_out<2>(c, backward, hD, go, dp, r0, rows, s);
  }
}

// h1 .. h_D of rows [r0, r0 + rows) into the chunk's activation buffers.
cudaError_t wide_forward_chunk(npg_ctx* c, long long r0, int rows, cudaStream_t s) {
  const MlpDims& md = c->md;
  const int H = md.H;
  const WideLayout L = wide_layout(c);
  float* act = c->wide + L.act;
  const long long C = c->wide_rows;
  wide_h1_kernel<<<grid1d((long long)rows * H / 4, 256, c->num_sms), 256, 0, s>>>(
      c->U, c->V, act, r0, rows, c->N, H, md.slope);
  cudaError_t e = cudaGetLastError();
  const float* W = c->mlp + (long long)H * md.K + H;
  for (int l = 1; l < md.D && e == cudaSuccess; ++l) {
    GemmArgs p{};
    p.A = act + (l - 1) * C * H;
    p.B = W;
    p.Y = act + l * C * H;
    p.bias = W + (long long)H * H;
    p.M = rows;
    p.N = H;
    p.K = H;
    p.lda = p.ldb = p.ldy = H;
    p.slope = md.slope;
    e = gemm<G_NT_ACT>(p, s);
    W += (long long)H * H + H;
  }
  return e;
}
}  // namespace

bool wide_fp32_supported(int H) { return H > 64 && H <= 512 && H % 32 == 0; }

long long wide_fp32_scratch_floats(int H, int D, int K, long long rows, long long* chunk_rows) {
  const long long C = std::min<long long>(rows, WIDE_CHUNK);
  if (chunk_rows) *chunk_rows = C;
  return (long long)(D + 2) * C * H + C * 8 + C * K;
}

cudaError_t launch_decode_fp32_wide(npg_ctx* c) {
  const long long rows = (long long)c->N * c->T;
  const long long C = c->wide_rows;
  const WideLayout L = wide_layout(c);
  cudaStream_t s = c->stream;
  for (long long r0 = 0; r0 < rows; r0 += C) {
    const int n = (int)std::min(C, rows - r0);
    cudaError_t e = wide_forward_chunk(c, r0, n, s);
    if (e == cudaSuccess)
      e = wide_out_rot(c, false, c->wide + L.act + (long long)(c->md.D - 1) * C * c->md.H,
                       nullptr, nullptr, r0, n, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_mlp_backward_fp32_wide(npg_ctx* c) {
  const MlpDims& md = c->md;
  const int H = md.H, K = md.K, Z = md.Z, D = md.D, NO = md.NO;
  const long long rows = (long long)c->N * c->T;
  const long long C = c->wide_rows;
  const WideLayout L = wide_layout(c);
  cudaStream_t s = c->stream;
  float* act = c->wide + L.act;
  float* go = c->wide + L.go;
  float* y = c->wide + L.y;
  // gradient layout = parameter layout
  float* gW1 = c->g_mlp;
  float* gb1 = gW1 + (long long)H * K;
  float* gh = gb1 + H;  // hidden layers: W (H x H) then b (H) each
  float* gWo = gh + (long long)(D - 1) * (H * H + H);
  float* gbo = gWo + (long long)NO * H;
  const float* W1 = c->mlp;
  const float* Wh = c->mlp + (long long)H * K + H;
  for (long long r0 = 0; r0 < rows; r0 += C) {
    const int n = (int)std::min(C, rows - r0);
    cudaError_t e = wide_forward_chunk(c, r0, n, s);
    float* dp = c->wide + L.dp0;
    float* dq = c->wide + L.dp1;
    const float* hD = act + (long long)(D - 1) * C * H;
    if (e == cudaSuccess) e = wide_out_rot(c, true, hD, go, dp, r0, n, s);
    // output layer: dWo += dL/do^T h_D, dbo += column sums of dL/do
    if (e == cudaSuccess) {
      GemmArgs p{};
      p.A = go;
      p.lda = 8;
      p.B = hD;
      p.ldb = H;
      p.Y = gWo;
      p.ldy = H;
      p.M = NO;
      p.N = H;
      p.K = n;
      e = gemm<G_TN_ADD>(p, s);
    }
    if (e == cudaSuccess) e = colsum(go, gbo, n, NO, 8, s);
    // hidden layers, last to first: dp holds dpre_l
    for (int l = D - 1; l >= 1 && e == cudaSuccess; --l) {
      const float* W = Wh + (long long)(l - 1) * (H * H + H);
      float* gW = gh + (long long)(l - 1) * (H * H + H);
      const float* hin = act + (long long)(l - 1) * C * H;
      GemmArgs p{};
      p.A = dp;
      p.lda = H;
      p.B = hin;
      p.ldb = H;
      p.Y = gW;
      p.ldy = H;
      p.M = H;
      p.N = H;
      p.K = n;
      e = gemm<G_TN_ADD>(p, s);
      if (e == cudaSuccess) e = colsum(dp, gW + (long long)H * H, n, H, H, s);
      if (e == cudaSuccess) {
        GemmArgs q{};
        q.A = dp;
        q.lda = H;
        q.B = W;
        q.ldb = H;
        q.Y = dq;
        q.ldy = H;
        q.Hin = hin;
        q.ldh = H;
        q.M = n;
        q.N = H;
        q.K = H;
        q.slope = md.slope;
        e = gemm<G_NN_DACT>(q, s);
      }
      std::swap(dp, dq);
    }
    // first layer: dW1 += dpre_1^T y, db1, dL/dz
    if (e == cudaSuccess) {
      wide_y_kernel<<<grid1d((long long)n * K, 256, c->num_sms), 256, 0, s>>>(
          c->z, c->gamma, y, r0, n, c->N, Z, K);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
      GemmArgs p{};
      p.A = dp;
      p.lda = H;
      p.B = y;
      p.ldb = K;
      p.Y = gW1;
      p.ldy = K;
      p.M = H;
      p.N = K;
      p.K = n;
      e = gemm<G_TN_ADD>(p, s);
    }
    if (e == cudaSuccess) e = colsum(dp, gb1, n, H, H, s);
    if (e == cudaSuccess && c->dV) {
      dim3 grid((H + 127) / 128, (unsigned)std::max(1, std::min(1024, n / 512)));
      wide_frame_colsum_kernel<<<grid, 128, 0, s>>>(dp, c->dV, r0, n, c->N, H);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
      GemmArgs p{};
      p.A = dp;
      p.lda = H;
      p.B = W1;
      p.ldb = K;
      p.Y = c->dz;
      p.ldy = Z;
      p.M = n;
      p.N = Z;
      p.K = H;
      p.r0 = r0;
      p.nvert = c->N;
      e = gemm<G_NN_DZ>(p, s);
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace npg
