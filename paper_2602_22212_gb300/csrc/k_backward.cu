// Backward kernels: FP32 SIMT MLP backward with forward recompute (reverse
// of Sec. 3.3-3.4) and the grid scatter-add (reverse of Sec. 3.2, Eq. 1).
#include "npg_device.cuh"
#include "npg_internal.cuh"

namespace npg {

// ----------------------------------------------------------------- MLP backward
// A tile is 8 vertices x 8 frames = 64 rows. Each row is handled by a thread
// pair (half = tid & 1 owns output features [half H/2, (half+1) H/2)). The
// forward pass is recomputed into shared memory, then dL/do (Eq. 5-7
// Jacobians) is propagated back layer by layer. Weight gradients are tiled
// outer products over the 64 rows accumulated in shared memory across the
// block's tiles and added to global memory once per block. dL/dz is reduced
// over the tile's frames before one atomic add per vertex.
struct BwdArgs {
  const float* mlp;
  const float* U;
  const float* V;
  const float* z;
  const float4* xr;
  const float4* dxhat;
  const float* gamma;  // T x 2M time encoding
  float* g_mlp;
  float* dz;
  float* dV;  // T x H, nullable: per-frame sums of dpre1 (learned time embedding)
  int N, T, K, Z, M, D, NO;
  float slope, alpha;
};

struct BwdLayout {
  int oWh, oBh, oWo, oBo, oW1, oAct, oDpA, oDpB, oDO, oY, oGWh, oGBh, oGWo, oGBo, oGW1, oGB1,
      oDZ, total;
};

__host__ __device__ inline BwdLayout bwd_layout(int H, int D, int K, int Z, int M) {
  BwdLayout L;
  int o = 0;
  auto take = [&](int n) {
    const int r = o;
    o += (n + 3) & ~3;
    return r;
  };
  L.oWh = take((D - 1) * H * H);
  L.oBh = take((D - 1) * H);
  L.oWo = take(8 * H);
  L.oBo = take(8);
  L.oW1 = take(H * K);
  L.oAct = take(D * 64 * H);
  L.oDpA = take(64 * H);
  L.oDpB = take(64 * H);
  L.oDO = take(64 * 8);
  L.oY = take(8 * Z + 8 * 2 * M);
  L.oGWh = take((D - 1) * H * H);
  L.oGBh = take((D - 1) * H);
  L.oGWo = take(8 * H);
  L.oGBo = take(8);
  L.oGW1 = take(H * K);
  L.oGB1 = take(H);
  L.oDZ = take(64 * Z);
  L.total = o;
  return L;
}

size_t mlp_bwd_fp32_smem(const MlpDims& md) {
  return sizeof(float) * (size_t)bwd_layout(md.H, md.D, md.K, md.Z, md.M).total;
}

template <int H, int ROT>
__global__ void __launch_bounds__(128, 1) mlp_bwd_fp32_kernel(BwdArgs a) {
  extern __shared__ float4 smem4[];
  float* sm = reinterpret_cast<float*>(smem4);
  const int D = a.D, K = a.K, Z = a.Z, M = a.M, NO = a.NO;
  const BwdLayout Ly = bwd_layout(H, D, K, Z, M);
  float* Wh = sm + Ly.oWh;
  float* Bh = sm + Ly.oBh;
  float* Wo = sm + Ly.oWo;
  float* Bo = sm + Ly.oBo;
  float* W1 = sm + Ly.oW1;
  float* act = sm + Ly.oAct;
  float* dpA = sm + Ly.oDpA;
  float* dpB = sm + Ly.oDpB;
  float* dO = sm + Ly.oDO;
  float* Ys = sm + Ly.oY;
  float* gWh = sm + Ly.oGWh;
  float* gBh = sm + Ly.oGBh;
  float* gWo = sm + Ly.oGWo;
  float* gBo = sm + Ly.oGBo;
  float* gW1 = sm + Ly.oGW1;
  float* gB1 = sm + Ly.oGB1;
  float* dZ = sm + Ly.oDZ;
  const int tid = threadIdx.x;

  // parameters: W1 (H x K), b1, hidden (W, b) x (D-1), Wo (NO x H), bo
  const float* p = a.mlp;
  for (int k = tid; k < H * K; k += 128) W1[k] = p[k];
  p += H * K + H;
  for (int l = 0; l < D - 1; ++l) {
    for (int k = tid; k < H * H; k += 128) Wh[l * H * H + k] = p[k];
    for (int k = tid; k < H; k += 128) Bh[l * H + k] = p[H * H + k];
    p += H * H + H;
  }
  for (int k = tid; k < 8 * H; k += 128) Wo[k] = k < NO * H ? p[k] : 0.f;
  for (int k = tid; k < 8; k += 128) Bo[k] = k < NO ? p[NO * H + k] : 0.f;
  const int nacc = Ly.oDZ - Ly.oGWh;
  for (int k = tid; k < nacc; k += 128) gWh[k] = 0.f;  // all accumulators are contiguous
  __syncthreads();

  const int r = tid >> 1, half = tid & 1;
  const int il = r & 7, tl = r >> 3;
  constexpr int HH = H / 2;
  const int n_ib = (a.N + 7) / 8, n_tb = (a.T + 7) / 8;
  const long long n_tiles = (long long)n_ib * n_tb;
  // weight-gradient tile of this thread: j in [jb TJ, +TJ), m in [mb TM, +TM)
  constexpr int TJ = H / 16, TM = H / 8;
  const int jb = tid >> 3, mb = tid & 7;

  for (long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int i0 = (int)(tile / n_tb) * 8, t0 = (int)(tile % n_tb) * 8;
    const int i = i0 + il, t = t0 + tl;
    const bool valid = (i < a.N) && (t < a.T);
    // y = (z_i, gamma_t) of the tile
    for (int k = tid; k < 8 * Z; k += 128) {
      const int v = k / Z, q = k % Z;
      Ys[k] = (i0 + v < a.N) ? a.z[(long long)(i0 + v) * Z + q] : 0.f;
    }
    if (tid < 8)
      for (int k = 0; k < 2 * M; ++k)
        Ys[8 * Z + tid * 2 * M + k] = a.gamma[(long long)min(t0 + tid, a.T - 1) * 2 * M + k];

    // ---- forward recompute
    float h[H];
    if (valid) {
      const float4* u4 = reinterpret_cast<const float4*>(a.U + (long long)i * H);
      const float4* v4 = reinterpret_cast<const float4*>(a.V + (long long)t * H);
#pragma unroll
      for (int k = 0; k < H / 4; ++k) {
        const float4 u = u4[k], v = v4[k];
        h[4 * k + 0] = leaky(u.x + v.x, a.slope);
        h[4 * k + 1] = leaky(u.y + v.y, a.slope);
        h[4 * k + 2] = leaky(u.z + v.z, a.slope);
        h[4 * k + 3] = leaky(u.w + v.w, a.slope);
      }
    } else {
#pragma unroll
      for (int k = 0; k < H; ++k) h[k] = 0.f;
    }
#pragma unroll
    for (int j = 0; j < HH; ++j) act[r * H + half * HH + j] = h[half * HH + j];
    for (int l = 1; l < D; ++l) {
      const float* W = Wh + (l - 1) * H * H;
      const float* b = Bh + (l - 1) * H;
      float hn[HH];
#pragma unroll
      for (int jj = 0; jj < HH; ++jj) {
        const int j = half * HH + jj;
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
        hn[jj] = valid ? leaky(s, a.slope) : 0.f;
      }
      float* out = act + l * 64 * H + r * H + half * HH;
#pragma unroll
      for (int jj = 0; jj < HH; ++jj) out[jj] = hn[jj];
      __syncthreads();
      const float4* full = reinterpret_cast<const float4*>(act + l * 64 * H + r * H);
#pragma unroll
      for (int k = 0; k < H / 4; ++k) {
        const float4 v = full[k];
        h[4 * k + 0] = v.x;
        h[4 * k + 1] = v.y;
        h[4 * k + 2] = v.z;
        h[4 * k + 3] = v.w;
      }
    }
    // output layer and dL/do
    float o[7], go[7];
#pragma unroll
    for (int j = 0; j < 7; ++j) {
      const float4* w4 = reinterpret_cast<const float4*>(Wo + j * H);
      float s = Bo[j];
#pragma unroll
      for (int k = 0; k < H / 4; ++k) {
        const float4 w = w4[k];
        s = fmaf(w.x, h[4 * k + 0], s);
        s = fmaf(w.y, h[4 * k + 1], s);
        s = fmaf(w.z, h[4 * k + 2], s);
        s = fmaf(w.w, h[4 * k + 3], s);
      }
      o[j] = s;
      go[j] = 0.f;
    }
    if (valid) {
      const long long row = (long long)t * a.N + i;
      transform_backward<ROT>(o, a.alpha, a.xr[i], a.dxhat[row], go);
    }
    if (half == 0) {
#pragma unroll
      for (int j = 0; j < 8; ++j) dO[r * 8 + j] = (j < NO) ? go[j] : 0.f;
    }
    // dpre_D = (Wo^T do) * act'(h_D), my half of the features
    {
      const float* hD = act + (D - 1) * 64 * H + r * H;
#pragma unroll 8
      for (int jj = 0; jj < HH; ++jj) {
        const int m = half * HH + jj;
        float s = 0.f;
#pragma unroll
        for (int q = 0; q < 7; ++q) s = fmaf(Wo[q * H + m], go[q], s);
        dpA[r * H + m] = s * dleaky_h(hD[m], a.slope);
      }
    }
    __syncthreads();
    // output-layer weight gradients
    for (int e = tid; e < 8 * H; e += 128) {
      const int q = e / H, m = e % H;
      if (q >= NO) continue;
      float s = gWo[e];
      const float* hD = act + (D - 1) * 64 * H;
      for (int rr = 0; rr < 64; ++rr) s = fmaf(dO[rr * 8 + q], hD[rr * H + m], s);
      gWo[e] = s;
    }
    if (tid < 8) {
      float s = gBo[tid];
      for (int rr = 0; rr < 64; ++rr) s += dO[rr * 8 + tid];
      gBo[tid] = s;
    }
    // hidden layers, last to first
    float* cur = dpA;
    float* nxt = dpB;
    for (int l = D - 1; l >= 1; --l) {
      const float* hin = act + (l - 1) * 64 * H;  // input of hidden layer l
      float* gW = gWh + (l - 1) * H * H;
      // gW[j][m] += sum_r cur[r][j] hin[r][m]
      {
        float accw[TJ][TM];
#pragma unroll
        for (int x = 0; x < TJ; ++x)
#pragma unroll
          for (int y = 0; y < TM; ++y) accw[x][y] = gW[(jb * TJ + x) * H + mb * TM + y];
        for (int rr = 0; rr < 64; ++rr) {
          float dj[TJ], hm[TM];
#pragma unroll
          for (int x = 0; x < TJ; ++x) dj[x] = cur[rr * H + jb * TJ + x];
#pragma unroll
          for (int y = 0; y < TM; ++y) hm[y] = hin[rr * H + mb * TM + y];
#pragma unroll
          for (int x = 0; x < TJ; ++x)
#pragma unroll
            for (int y = 0; y < TM; ++y) accw[x][y] = fmaf(dj[x], hm[y], accw[x][y]);
        }
#pragma unroll
        for (int x = 0; x < TJ; ++x)
#pragma unroll
          for (int y = 0; y < TM; ++y) gW[(jb * TJ + x) * H + mb * TM + y] = accw[x][y];
      }
      for (int j = tid; j < H; j += 128) {
        float s = gBh[(l - 1) * H + j];
        for (int rr = 0; rr < 64; ++rr) s += cur[rr * H + j];
        gBh[(l - 1) * H + j] = s;
      }
      // nxt[r][m] = (sum_j W[j][m] cur[r][j]) * act'(hin[r][m])
      {
        const float* W = Wh + (l - 1) * H * H;
        float dr[H];
        const float4* c4 = reinterpret_cast<const float4*>(cur + r * H);
#pragma unroll
        for (int k = 0; k < H / 4; ++k) {
          const float4 v = c4[k];
          dr[4 * k] = v.x;
          dr[4 * k + 1] = v.y;
          dr[4 * k + 2] = v.z;
          dr[4 * k + 3] = v.w;
        }
        float acc[HH];
#pragma unroll
        for (int jj = 0; jj < HH; ++jj) acc[jj] = 0.f;
#pragma unroll
        for (int j = 0; j < H; ++j) {
          const float4* w4 = reinterpret_cast<const float4*>(W + j * H + half * HH);
#pragma unroll
          for (int k = 0; k < HH / 4; ++k) {
            const float4 w = w4[k];
            acc[4 * k + 0] = fmaf(w.x, dr[j], acc[4 * k + 0]);
            acc[4 * k + 1] = fmaf(w.y, dr[j], acc[4 * k + 1]);
            acc[4 * k + 2] = fmaf(w.z, dr[j], acc[4 * k + 2]);
            acc[4 * k + 3] = fmaf(w.w, dr[j], acc[4 * k + 3]);
          }
        }
        const float* hr = hin + r * H + half * HH;
#pragma unroll
        for (int jj = 0; jj < HH; ++jj)
          nxt[r * H + half * HH + jj] = acc[jj] * dleaky_h(hr[jj], a.slope);
      }
      __syncthreads();
      float* tmp = cur;
      cur = nxt;
      nxt = tmp;
    }
    // first layer: gW1 += dpre1 (x) y, gb1 += dpre1, dz rows
    for (int e = tid; e < H * K; e += 128) {
      const int j = e / K, q = e % K;
      float s = gW1[e];
      for (int rr = 0; rr < 64; ++rr) {
        const float yv = q < Z ? Ys[(rr & 7) * Z + q] : Ys[8 * Z + (rr >> 3) * 2 * M + (q - Z)];
        s = fmaf(cur[rr * H + j], yv, s);
      }
      gW1[e] = s;
    }
    for (int j = tid; j < H; j += 128) {
      float s = gB1[j];
      for (int rr = 0; rr < 64; ++rr) s += cur[rr * H + j];
      gB1[j] = s;
    }
    for (int q = half; q < Z; q += 2) {
      float s = 0.f;
      for (int j = 0; j < H; ++j) s = fmaf(W1[j * K + q], cur[r * H + j], s);
      dZ[r * Z + q] = s;
    }
    if (a.dV) {  // per-frame sums over the tile's 8 vertices (rows tl * 8 + il)
      for (int e = tid; e < 8 * H; e += 128) {
        const int ft = e / H, j = e % H;
        if (t0 + ft >= a.T) continue;
        float s = 0.f;
        for (int v = 0; v < 8; ++v) s += cur[(ft * 8 + v) * H + j];
        atomicAdd(a.dV + (long long)(t0 + ft) * H + j, s);
      }
    }
    __syncthreads();
    for (int e = tid; e < 8 * Z; e += 128) {
      const int v = e / Z, q = e % Z;
      if (i0 + v >= a.N) continue;
      float s = 0.f;
      for (int tt = 0; tt < 8; ++tt) s += dZ[(tt * 8 + v) * Z + q];
      atomicAdd(a.dz + (long long)(i0 + v) * Z + q, s);
    }
    __syncthreads();
  }
  // block partials -> global gradient (same layout as the parameters)
  float* g = a.g_mlp;
  for (int k = tid; k < H * K; k += 128) atomicAdd(g + k, gW1[k]);
  for (int k = tid; k < H; k += 128) atomicAdd(g + H * K + k, gB1[k]);
  float* gh = g + H * K + H;
  for (int l = 0; l < D - 1; ++l) {
    for (int k = tid; k < H * H; k += 128) atomicAdd(gh + k, gWh[l * H * H + k]);
    for (int k = tid; k < H; k += 128) atomicAdd(gh + H * H + k, gBh[l * H + k]);
    gh += H * H + H;
  }
  for (int k = tid; k < NO * H; k += 128) atomicAdd(gh + k, gWo[k]);
  for (int k = tid; k < NO; k += 128) atomicAdd(gh + NO * H + k, gBo[k]);
}

template <int H, int ROT>
static cudaError_t mlp_bwd_h(npg_ctx* c) {
  BwdArgs a;
  a.mlp = c->mlp;
  a.U = c->U;
  a.V = c->V;
  a.z = c->z;
  a.xr = c->xr;
  a.dxhat = c->dxhat;
  a.g_mlp = c->g_mlp;
  a.dz = c->dz;
  a.dV = c->dV;
  a.N = c->N;
  a.T = c->T;
  a.K = c->md.K;
  a.Z = c->md.Z;
  a.M = c->md.M;
  a.gamma = c->gamma;
  a.D = c->md.D;
  a.NO = c->md.NO;
  a.slope = c->md.slope;
  a.alpha = c->cfg.alpha;
  const size_t smem = mlp_bwd_fp32_smem(c->md);
  auto k = mlp_bwd_fp32_kernel<H, ROT>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long tiles = (long long)((c->N + 7) / 8) * ((c->T + 7) / 8);
  long long blocks = c->num_sms;
  if (blocks > tiles) blocks = tiles;
  k<<<(int)blocks, 128, smem, c->stream>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_mlp_backward_fp32(npg_ctx* c) {
  if (c->md.H > 64) return launch_mlp_backward_fp32_wide(c);
  const int rm = c->cfg.rot_mode;
#define NPG_BWD_H(HH)                                                                       \
  case HH:                                                                                  \
    return rm == NPG_ROT_QUAT ? mlp_bwd_h<HH, 0>(c)                                         \
                              : rm == NPG_ROT_EXPMAP ? mlp_bwd_h<HH, 1>(c) : mlp_bwd_h<HH, 2>(c);
  switch (c->md.H) {
    NPG_BWD_H(16)
    NPG_BWD_H(32)
    NPG_BWD_H(64)
  }
#undef NPG_BWD_H
  return cudaErrorInvalidValue;
}

// ----------------------------------------------------------------- scatter
// dL/dG_l[corner] += w_c dz_p / L (Eq. 1 reversed), dL/dG_n[corner] += w_c dz_n.
// Block = 16 lookups x 16 vertices; the small normal grid is pre-reduced in
// shared memory before one global atomic per node.
struct ScatterArgs {
  const float4* xr;
  const float4* nr;
  const float* dz;
  float* g;
  int N, L, F, Fn, Z, nn_nodes;
  int r[NPG_MAX_LEVELS + 1];
  long long off[NPG_MAX_LEVELS + 1];
};

__global__ void __launch_bounds__(256) scatter_kernel(ScatterArgs a) {
  extern __shared__ float gn_sm[];
  const int lk = threadIdx.x, vy = threadIdx.y, tid = vy * 16 + lk;
  const int nsm = a.nn_nodes * a.Fn;
  for (int k = tid; k < nsm; k += 256) gn_sm[k] = 0.f;
  __syncthreads();
  const int i = blockIdx.x * 16 + vy;
  if (i < a.N && lk <= a.L) {
    const bool normal = lk == a.L;
    const int r = a.r[lk], F = normal ? a.Fn : a.F;
    const float4 p = normal ? a.nr[i] : a.xr[i];
    int ix, iy, iz;
    float fx, fy, fz;
    tri_axis(p.x, r, ix, fx);
    tri_axis(p.y, r, iy, fy);
    tri_axis(p.z, r, iz, fz);
    const float* dzi = a.dz + (long long)i * a.Z + (normal ? 0 : a.Fn);
    const float sc = normal ? 1.f : 1.f / (float)a.L;
    float gv[NPG_MAX_F];
#pragma unroll
    for (int f = 0; f < NPG_MAX_F; ++f) gv[f] = f < F ? dzi[f] * sc : 0.f;
    float* g = a.g + a.off[lk];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int bx = c & 1, by = (c >> 1) & 1, bz = (c >> 2) & 1;
      const float w = (bx ? fx : 1.f - fx) * (by ? fy : 1.f - fy) * (bz ? fz : 1.f - fz);
      const long long node = ((long long)(iz + bz) * r + (iy + by)) * r + (ix + bx);
      if (normal && nsm > 0) {
#pragma unroll
        for (int f = 0; f < NPG_MAX_FN; ++f)
          if (f < F) atomicAdd(gn_sm + node * F + f, w * gv[f]);
      } else if (F == 4) {
        float* gp = g + node * 4;
        atomicAdd(reinterpret_cast<float4*>(gp),
                  make_float4(w * gv[0], w * gv[1], w * gv[2], w * gv[3]));
      } else {
        float* gp = g + node * F;
#pragma unroll
        for (int f = 0; f < NPG_MAX_F; ++f)
          if (f < F) atomicAdd(gp + f, w * gv[f]);
      }
    }
  }
  __syncthreads();
  if (nsm > 0) {
    float* g = a.g + a.off[a.L];
    for (int k = tid; k < nsm; k += 256)
      if (gn_sm[k] != 0.f) atomicAdd(g + k, gn_sm[k]);
  }
}

cudaError_t launch_scatter(npg_ctx* c) {
  ScatterArgs a;
  a.xr = c->xr;
  a.nr = c->nr;
  a.dz = c->dz;
  a.g = c->g_grid;
  a.N = c->N;
  a.L = c->cfg.L;
  a.F = c->cfg.F_p;
  a.Fn = c->cfg.F_n;
  a.Z = c->md.Z;
  for (int l = 0; l < c->nlev; ++l) {
    a.r[l] = c->lev[l].r;
    a.off[l] = c->lev[l].off;
  }
  const long long nn = (long long)c->cfg.res_n * c->cfg.res_n * c->cfg.res_n;
  a.nn_nodes = (nn * c->cfg.F_n <= 8192) ? (int)nn : 0;
  const size_t smem = sizeof(float) * (size_t)a.nn_nodes * c->cfg.F_n;
  dim3 block(16, 16), grid((c->N + 15) / 16);
  scatter_kernel<<<grid, block, smem, c->stream>>>(a);
  return cudaGetLastError();
}

}  // namespace npg
