// Forward kernels: latent-grid lookup (Sec. 3.2), time modulation and the
// FP32 SIMT decode + rigid transform (Sec. 3.3-3.4).
#include "npg_device.cuh"
#include "npg_internal.cuh"

namespace npg {

// ----------------------------------------------------------------- encode
// Block = 16 lookups (levels 0..L-1 and the normal grid at L) x 16 vertices.
// Phase 1: each thread interpolates one lookup of one vertex (8 corners x F).
// Phase 2: level mean (Eq. 1) -> z = (z_n, z_p); U = W1[:, :Z] z + b1.
struct EncodeArgs {
  const float4* xr;
  const float4* nr;
  const float* grid;
  const float* mlp;  // W1 (H x K) then b1
  float* z;
  float* U;
  int N, L, F, Fn, H, K, Z;
  int r[NPG_MAX_LEVELS + 1];
  long long off[NPG_MAX_LEVELS + 1];
};

__global__ void __launch_bounds__(256) encode_kernel(EncodeArgs a) {
  __shared__ float part[16][NPG_MAX_LEVELS + 1][NPG_MAX_F];
  __shared__ float zs[16][NPG_MAX_Z];
  const int lk = threadIdx.x, vy = threadIdx.y;
  const int i = blockIdx.x * 16 + vy;
  const int nl = a.L + 1;
  if (i < a.N && lk < nl) {
    const bool normal = (lk == a.L);
    const int r = a.r[lk], F = normal ? a.Fn : a.F;
    const float4 p = normal ? a.nr[i] : a.xr[i];
    int ix, iy, iz;
    float fx, fy, fz;
    tri_axis(p.x, r, ix, fx);
    tri_axis(p.y, r, iy, fy);
    tri_axis(p.z, r, iz, fz);
    const float* g = a.grid + a.off[lk];
    float acc[NPG_MAX_F];
#pragma unroll
    for (int f = 0; f < NPG_MAX_F; ++f) acc[f] = 0.f;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int bx = c & 1, by = (c >> 1) & 1, bz = (c >> 2) & 1;
      const float w = (bx ? fx : 1.f - fx) * (by ? fy : 1.f - fy) * (bz ? fz : 1.f - fz);
      const long long node = ((long long)(iz + bz) * r + (iy + by)) * r + (ix + bx);
      const float* gp = g + node * F;
      if (F == 4) {
        const float4 v = *reinterpret_cast<const float4*>(gp);
        acc[0] = fmaf(w, v.x, acc[0]);
        acc[1] = fmaf(w, v.y, acc[1]);
        acc[2] = fmaf(w, v.z, acc[2]);
        acc[3] = fmaf(w, v.w, acc[3]);
      } else {
#pragma unroll
        for (int f = 0; f < NPG_MAX_F; ++f)
          if (f < F) acc[f] = fmaf(w, __ldg(gp + f), acc[f]);
      }
    }
#pragma unroll
    for (int f = 0; f < NPG_MAX_F; ++f)
      if (f < F) part[vy][lk][f] = acc[f];
  }
  __syncthreads();
  // level mean and z
  const int tid = vy * 16 + lk;
  for (int e = tid; e < 16 * a.Z; e += 256) {
    const int v = e / a.Z, k = e % a.Z;
    const int ii = blockIdx.x * 16 + v;
    float val = 0.f;
    if (ii < a.N) {
      if (k < a.Fn) {
        val = part[v][a.L][k];
      } else {
        float s = 0.f;
        for (int l = 0; l < a.L; ++l) s += part[v][l][k - a.Fn];
        val = s / (float)a.L;
      }
      a.z[(long long)ii * a.Z + k] = val;
    }
    zs[v][k] = val;
  }
  __syncthreads();
  // U = W1[:, :Z] z + b1
  const float* W1 = a.mlp;
  const float* b1 = a.mlp + (long long)a.H * a.K;
  for (int e = tid; e < 16 * a.H; e += 256) {
    const int v = e / a.H, j = e % a.H;
    const int ii = blockIdx.x * 16 + v;
    if (ii >= a.N) continue;
    float s = b1[j];
    for (int k = 0; k < a.Z; ++k) s = fmaf(W1[(long long)j * a.K + k], zs[v][k], s);
    a.U[(long long)ii * a.H + j] = s;
  }
}

cudaError_t launch_encode(npg_ctx* c) {
  EncodeArgs a;
  a.xr = c->xr;
  a.nr = c->nr;
  a.grid = c->grid;
  a.mlp = c->mlp;
  a.z = c->z;
  a.U = c->U;
  a.N = c->N;
  a.L = c->cfg.L;
  a.F = c->cfg.F_p;
  a.Fn = c->cfg.F_n;
  a.H = c->md.H;
  a.K = c->md.K;
  a.Z = c->md.Z;
  for (int l = 0; l < c->nlev; ++l) {
    a.r[l] = c->lev[l].r;
    a.off[l] = c->lev[l].off;
  }
  dim3 block(16, 16), grid((c->N + 15) / 16);
  encode_kernel<<<grid, block, 0, c->stream>>>(a);
  return cudaGetLastError();
}

// ----------------------------------------------------------------- time modulation
// gamma(t) of every frame (T x 2M), once per context: the encoding is fixed.
struct TimeFreqs {
  float B[NPG_MAX_FREQ];
};

__global__ void time_table_kernel(float* gamma, int T, int M, int mode, TimeFreqs f) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < T) time_embedding_mode(t, T, M, mode, f.B, gamma + (long long)t * 2 * M);
}

// V_t = W1[:, Z:] gamma(t) (Eq. 2-3; the bias lives in U).
__global__ void time_mod_kernel(const float* mlp, const float* gamma, float* V, int T, int H,
                                int K, int Z, int M) {
  const int t = blockIdx.x;
  const float* g = gamma + (long long)t * 2 * M;
  for (int j = threadIdx.x; j < H; j += blockDim.x) {
    float s = 0.f;
    for (int k = 0; k < 2 * M; ++k) s = fmaf(mlp[(long long)j * K + Z + k], g[k], s);
    V[(long long)t * H + j] = s;
  }
}

// Learned time embedding (the time-encoding ablation, Sec. 4): per frame,
// h = act(a t~ + b) (Ht values), gamma = W h + c (2M values); the parameters
// follow the decoder's in the MLP vector. One block per frame.
__global__ void learned_time_kernel(const float* __restrict__ tp, float* __restrict__ gamma,
                                    int T, int M, int Ht, float slope) {
  extern __shared__ float hs[];
  const int t = blockIdx.x;
  const float tt = T > 1 ? (float)t / (float)(T - 1) : 0.f;
  const float* a = tp;
  const float* b = a + Ht;
  const float* W = b + Ht;
  const float* cc = W + 2 * M * Ht;
  for (int j = threadIdx.x; j < Ht; j += blockDim.x) hs[j] = leaky(fmaf(a[j], tt, b[j]), slope);
  __syncthreads();
  for (int k = threadIdx.x; k < 2 * M; k += blockDim.x) {
    float s = cc[k];
    for (int j = 0; j < Ht; ++j) s = fmaf(W[k * Ht + j], hs[j], s);
    gamma[(long long)t * 2 * M + k] = s;
  }
}

cudaError_t launch_learned_time(npg_ctx* c) {
  const MlpDims& md = c->md;
  learned_time_kernel<<<c->T, 64, sizeof(float) * md.Ht, c->stream>>>(
      c->mlp + md.dec_len, c->gamma, c->T, md.M, md.Ht, md.slope);
  return cudaGetLastError();
}

// Reverse of the above, one block per frame: dL/dgamma_t = W1[:, Z:]^T dV_t
// (dV_t = the sum over vertices of dL/d(first-layer pre-activation) at frame
// t), then back through gamma = W h + c and h = act(a t~ + b) into psi_t's
// gradient (atomic adds over frames).
__global__ void learned_time_backward_kernel(const float* __restrict__ mlp,
                                             const float* __restrict__ dV,
                                             float* __restrict__ g_tp, int T, int H, int K, int Z,
                                             int M, int Ht, long long dec_len, float slope) {
  __shared__ float gg[2 * NPG_MAX_FREQ];
  const int t = blockIdx.x;
  const float tt = T > 1 ? (float)t / (float)(T - 1) : 0.f;
  const int G2 = 2 * M;
  for (int k = threadIdx.x; k < G2; k += blockDim.x) {
    float s = 0.f;
    for (int j = 0; j < H; ++j) s = fmaf(mlp[(long long)j * K + Z + k], dV[(long long)t * H + j], s);
    gg[k] = s;
  }
  __syncthreads();
  const float* a = mlp + dec_len;
  const float* b = a + Ht;
  const float* W = b + Ht;
  float* ga = g_tp;
  float* gb = ga + Ht;
  float* gW = gb + Ht;
  float* gc = gW + G2 * Ht;
  for (int j = threadIdx.x; j < Ht; j += blockDim.x) {
    const float hp = fmaf(a[j], tt, b[j]);
    const float h = leaky(hp, slope);
    float dh = 0.f;
    for (int k = 0; k < G2; ++k) {
      atomicAdd(gW + k * Ht + j, gg[k] * h);
      dh = fmaf(W[k * Ht + j], gg[k], dh);
    }
    const float dp = dh * (hp > 0.f ? 1.f : slope);
    atomicAdd(ga + j, dp * tt);
    atomicAdd(gb + j, dp);
  }
  for (int k = threadIdx.x; k < G2; k += blockDim.x) atomicAdd(gc + k, gg[k]);
}

cudaError_t launch_learned_time_backward(npg_ctx* c) {
  const MlpDims& md = c->md;
  learned_time_backward_kernel<<<c->T, 64, 0, c->stream>>>(c->mlp, c->dV, c->g_mlp + md.dec_len,
                                                            c->T, md.H, md.K, md.Z, md.M, md.Ht,
                                                            md.dec_len, md.slope);
  return cudaGetLastError();
}

cudaError_t launch_time_table(npg_ctx* c) {
  if (c->md.Ht > 0) return launch_learned_time(c);
  TimeFreqs f;
  for (int j = 0; j < NPG_MAX_FREQ; ++j) f.B[j] = c->cfg.time_B[j];
  time_table_kernel<<<(c->T + 127) / 128, 128, 0, c->stream>>>(c->gamma, c->T, c->md.M,
                                                               c->cfg.time_enc, f);
  return cudaGetLastError();
}

cudaError_t launch_time_mod(npg_ctx* c) {
  time_mod_kernel<<<c->T, 128, 0, c->stream>>>(c->mlp, c->gamma, c->V, c->T, c->md.H, c->md.K,
                                              c->md.Z, c->md.M);
  return cudaGetLastError();
}

// ----------------------------------------------------------------- FP32 decode
// One thread per row (i, t), rows frame-major. h1 = act(U_i + V_t); hidden
// layers from shared memory (row-major W[j][k], read as float4 broadcasts);
// output layer; Eq. 5-7. Writes x-hat[t][i].
template <int H, int ROT>
__global__ void __launch_bounds__(128) decode_fp32_kernel(const float* __restrict__ mlp,
                                                          const float* __restrict__ U,
                                                          const float* __restrict__ V,
                                                          const float4* __restrict__ xr,
                                                          float4* __restrict__ xhat,
                                                          float4* __restrict__ disp, int N, int T,
                                                          int K, int D, int NO, float slope,
                                                          float alpha) {
  extern __shared__ float4 smem4[];
  float* sm = reinterpret_cast<float*>(smem4);
  const long long hid_len = (long long)(D - 1) * (H * H + H);
  const float* src = mlp + (long long)H * K + H;
  const int nload = (int)(hid_len + NO * H + NO);
  for (int k = threadIdx.x; k < nload; k += blockDim.x) sm[k] = src[k];
  __syncthreads();
  const long long rows = (long long)N * T;
  for (long long row = (long long)blockIdx.x * blockDim.x + threadIdx.x; row < rows;
       row += (long long)gridDim.x * blockDim.x) {
    const int t = (int)(row / N), i = (int)(row - (long long)t * N);
    float h[H];
    const float4* u4 = reinterpret_cast<const float4*>(U + (long long)i * H);
    const float4* v4 = reinterpret_cast<const float4*>(V + (long long)t * H);
#pragma unroll
    for (int k = 0; k < H / 4; ++k) {
      const float4 u = u4[k], v = v4[k];
      h[4 * k + 0] = leaky(u.x + v.x, slope);
      h[4 * k + 1] = leaky(u.y + v.y, slope);
      h[4 * k + 2] = leaky(u.z + v.z, slope);
      h[4 * k + 3] = leaky(u.w + v.w, slope);
    }
    for (int layer = 1; layer < D; ++layer) {
      const float* W = sm + (long long)(layer - 1) * (H * H + H);
      const float* b = W + H * H;
      float hn[H];
#pragma unroll
      for (int j = 0; j < H; ++j) {
        const float4* w4 = reinterpret_cast<const float4*>(W + j * H);
        float s = b[j];
#pragma unroll
        for (int k = 0; k < H / 4; ++k) {
          const float4 w = w4[k];
          s = fmaf(w.x, h[4 * k + 0], s);
          s = fmaf(w.y, h[4 * k + 1], s);
          s = fmaf(w.z, h[4 * k + 2], s);
          s = fmaf(w.w, h[4 * k + 3], s);
        }
        hn[j] = s;
      }
#pragma unroll
      for (int j = 0; j < H; ++j) h[j] = leaky(hn[j], slope);
    }
    const float* Wo = sm + hid_len;
    const float* bo = Wo + NO * H;
    float o[7];
#pragma unroll
    for (int j = 0; j < 7; ++j) {
      if (j < NO) {
        const float4* w4 = reinterpret_cast<const float4*>(Wo + j * H);
        float s = bo[j];
#pragma unroll
        for (int k = 0; k < H / 4; ++k) {
          const float4 w = w4[k];
          s = fmaf(w.x, h[4 * k + 0], s);
          s = fmaf(w.y, h[4 * k + 1], s);
          s = fmaf(w.z, h[4 * k + 2], s);
          s = fmaf(w.w, h[4 * k + 3], s);
        }
        o[j] = s;
      } else {
        o[j] = 0.f;
      }
    }
    float4 xh, dl;
    transform<ROT>(o, alpha, xr[i], xh, dl);
    xhat[row] = xh;
    disp[row] = dl;
  }
}

bool decode_fp32_supported(int H, int D) {
  return (H == 16 || H == 32 || H == 64) && D >= 1 && D <= NPG_MAX_DEPTH;
}

template <int H, int ROT>
static cudaError_t decode_fp32_h(npg_ctx* c) {
  const int D = c->md.D, NO = c->md.NO;
  const size_t smem = sizeof(float) * ((size_t)(D - 1) * (H * H + H) + NO * H + NO + 4);
  auto k = decode_fp32_kernel<H, ROT>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long rows = (long long)c->N * c->T;
  long long blocks = (rows + 127) / 128;
  const long long cap = (long long)c->num_sms * 8;
  if (blocks > cap) blocks = cap;
  k<<<(int)blocks, 128, smem, c->stream>>>(c->mlp, c->U, c->V, c->xr, c->xhat, c->disp, c->N, c->T,
                                           c->md.K, D, NO, c->md.slope, c->cfg.alpha);
  return cudaGetLastError();
}

cudaError_t launch_decode_fp32(npg_ctx* c) {
  const int H = c->md.H;
  if (H > 64) return launch_decode_fp32_wide(c);
  const int rm = c->cfg.rot_mode;
#define NPG_DECODE_H(HH)                                                                    \
  if (H == HH)                                                                              \
    return rm == NPG_ROT_QUAT     ? decode_fp32_h<HH, 0>(c)                                 \
           : rm == NPG_ROT_EXPMAP ? decode_fp32_h<HH, 1>(c)                                 \
                                  : decode_fp32_h<HH, 2>(c);
  NPG_DECODE_H(16)
  NPG_DECODE_H(32)
  NPG_DECODE_H(64)
#undef NPG_DECODE_H
  return cudaErrorInvalidValue;
}

// ----------------------------------------------------------------- helpers

__global__ void points_to_float4_kernel(const float* __restrict__ s, float4* __restrict__ d,
                                        long long n) {
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x)
    d[k] = make_float4(s[3 * k], s[3 * k + 1], s[3 * k + 2], 0.f);
}

cudaError_t launch_points_to_float4(const float* src, float4* dst, long long n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  long long b = (n + 255) / 256;
  if (b > 65535) b = 65535;
  points_to_float4_kernel<<<(int)b, 256, 0, s>>>(src, dst, n);
  return cudaGetLastError();
}

__global__ void xhat_out_kernel(const float4* __restrict__ x, float* __restrict__ o, long long n) {
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    const float4 v = x[k];
    o[3 * k] = v.x;
    o[3 * k + 1] = v.y;
    o[3 * k + 2] = v.z;
  }
}

cudaError_t launch_xhat_out(const float4* xhat, float* out, long long n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  long long b = (n + 255) / 256;
  if (b > 65535) b = 65535;
  xhat_out_kernel<<<(int)b, 256, 0, s>>>(xhat, out, n);
  return cudaGetLastError();
}

}  // namespace npg
