// Pieces shared by the BF16 tensor-core MLP kernels (hidden width 64 in
// k_mlp_tc.cu, 128 in k_mlp_tc128.cu): kernel arguments, bounded mbarrier
// waits folded into CTA barriers, BF16 stores into 128B-swizzled K-major
// tiles and TMEM column loads.
#pragma once

#include <cuda_bf16.h>

#include "npg_device.cuh"
#include "npg_internal.cuh"
#include "tc_sm100.cuh"

namespace npg {

constexpr int TC_ROWS = 128;
constexpr uint32_t TC_TILE = TC_ROWS * 128;  // bytes of one [128][64] BF16 swizzled tile
constexpr uint32_t WAIT_TRIES = 1u << 24;

struct TcArgs {
  const float* mlp;
  const float* U;
  const float* V;
  const float4* xr;
  float4* xhat;
  float4* disp;
  const float4* dxhat;
  const float* z;
  const float* gamma;  // T x 2M time encoding
  float* g_mlp;
  float* dz;
  float* dV;  // T x H, nullable: per-frame sums of dpre1 (learned time embedding)
  int* err;
  int N, T, K, Z, M, NO;
  float slope, alpha;
};

inline TcArgs make_tc_args(npg_ctx* c) {
  TcArgs a;
  a.mlp = c->mlp;
  a.U = c->U;
  a.V = c->V;
  a.xr = c->xr;
  a.xhat = c->xhat;
  a.disp = c->disp;
  a.dxhat = c->dxhat;
  a.z = c->z;
  a.g_mlp = c->g_mlp;
  a.dz = c->dz;
  a.dV = c->dV;
  a.err = c->d_err;
  a.N = c->N;
  a.T = c->T;
  a.K = c->md.K;
  a.Z = c->md.Z;
  a.M = c->md.M;
  a.gamma = c->gamma;
  a.NO = c->md.NO;
  a.slope = c->md.slope;
  a.alpha = c->cfg.alpha;
  return a;
}

// Grid of a persistent kernel: per_sm CTAs per SM, at most one per tile.
inline int tc_grid(const npg_ctx* c, long long tiles, int per_sm) {
  long long b = (long long)c->num_sms * per_sm;
  if (b > tiles) b = tiles;
  if (b < 1) b = 1;
  return (int)b;
}

__device__ __forceinline__ void st_bf16(uint8_t* tile, int row, int col, float v) {
  *reinterpret_cast<__nv_bfloat16*>(tile + tc::sw128_off(row, col)) = __float2bfloat16_rn(v);
}

// 8 FP32 values as BF16 into columns [c0, c0 + 8) (c0 % 8 == 0, c0 < 64) of
// one row of a K-major [rows][64] tile.
__device__ __forceinline__ void st_bf16x8(uint8_t* tile, int row, int c0, const float* v) {
  uint4 q;
  q.x = tc::pack_bf16(v[0], v[1]);
  q.y = tc::pack_bf16(v[2], v[3]);
  q.z = tc::pack_bf16(v[4], v[5]);
  q.w = tc::pack_bf16(v[6], v[7]);
  *reinterpret_cast<uint4*>(tile + tc::sw128_off(row, c0)) = q;
}

// Every thread polls the barrier; the outcome is folded into the next
// CTA-wide barrier (tc_sync_ok), so a wait that gives up ends the kernel
// uniformly without an extra barrier per wait.
__device__ __forceinline__ void tc_wait(uint64_t* bar, uint32_t& phase, bool& ok) {
  ok = ok && tc::mbar_wait(bar, phase, WAIT_TRIES);
  phase ^= 1u;
  tc::fence_after_sync();
}

// The same wait for a phase parity the caller derives (a barrier committed a
// fixed number of times per tile completes a fixed parity pattern).
__device__ __forceinline__ void tc_wait_parity(uint64_t* bar, uint32_t parity, bool& ok) {
  ok = ok && tc::mbar_wait(bar, parity, WAIT_TRIES);
  tc::fence_after_sync();
}

// Shared-memory writes -> async proxy, TMEM reads complete, then a CTA
// barrier that also agrees on `ok`.
__device__ __forceinline__ bool tc_sync_ok(bool ok, int* err) {
  tc::fence_async_smem();
  tc::fence_before_sync();
  ok = __syncthreads_and(ok) != 0;
  tc::fence_after_sync();
  if (!ok && threadIdx.x == 0) atomicExch(err, 1);
  return ok;
}

__device__ __forceinline__ void ld_col16(uint32_t taddr, float* v) {
  uint32_t r[16];
  tc::tmem_ld16(taddr, r);
  tc::tmem_ld_wait();
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// Per-frame sums of n values per thread over the 16 lanes of each half-warp
// (the 16 vertices of one frame in a 16 x 8 tile whose row = 16 frame +
// vertex sits in TMEM lane row % 32 of warp row / 32), added to
// dV[t0 + frame][col0 + j]. Every lane of the warp takes part.
template <int NV>
__device__ __forceinline__ void frame_sums(const float* v, float* dV, int t0, int frame, int T,
                                           int H, int col0) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    float s = v[j];
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((lane & 15) == 0 && t0 + frame < T) atomicAdd(dV + (long long)(t0 + frame) * H + col0 + j, s);
  }
}

// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void ld_col32(uint32_t taddr, float* v) {
  uint32_t r[32];
  tc::tmem_ld16(taddr, r);
  tc::tmem_ld16(taddr + 16, r + 16);
  tc::tmem_ld_wait();
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

}  // namespace npg
