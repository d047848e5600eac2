// BF16 tensor-core (tcgen05) MLP decode (Sec. 3.3-3.4) for hidden width 64
// and 3 hidden layers: operands in 128B-swizzled shared
// memory, FP32 accumulators in TMEM, FP32 epilogues (bias, LeakyReLU, the
// rotation/translation mapping and its Jacobian) on the CUDA cores.
//
// A CTA of 128 threads owns tiles of 128 consecutive rows (row = t N + i);
// thread t owns row t of the tile and TMEM lane t. One elected lane of warp 0
// issues the MMAs; completion is tracked by an mbarrier whose waits are bounded: a
// wait that gives up sets *err and the CTA frees its TMEM and exits.
#include "mlp_tc_common.cuh"

namespace npg {

constexpr int TC_H = 64;

// Hidden width 64 here, 128 in k_mlp_tc128.cu; three hidden layers.
bool decode_bf16_supported(int H, int D) { return (H == TC_H || H == 128) && D == 3; }

// Write 64 FP32 values of one row as BF16 into a K-major swizzled tile.
__device__ __forceinline__ void st_row64(uint8_t* tile, int row, const float* v) {
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    uint4 q;
    q.x = tc::pack_bf16(v[8 * c + 0], v[8 * c + 1]);
    q.y = tc::pack_bf16(v[8 * c + 2], v[8 * c + 3]);
    q.z = tc::pack_bf16(v[8 * c + 4], v[8 * c + 5]);
    q.w = tc::pack_bf16(v[8 * c + 6], v[8 * c + 7]);
    *reinterpret_cast<uint4*>(tile + tc::sw128_off(row, 8 * c)) = q;
  }
}

// Issue D = A * B^T with K = 64 (4 steps of 16), K-major operand descriptors
// (a K step of 16 advances the start address by 32 B, 2 in its 16 B units).
__device__ __forceinline__ void mma_k64(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc) {
#pragma unroll
  for (int ks = 0; ks < 4; ++ks) tc::mma_bf16(d, a + 2 * ks, b + 2 * ks, idesc, ks > 0);
}

// Shared layout of the decode kernel (offsets from a 1024-byte aligned base).
struct DecodeSmem {
  static constexpr uint32_t W2 = 0;                 // [64][64] K-major (B operand)
  static constexpr uint32_t W3 = W2 + TC_TILE / 2;  // 8 KB each
  static constexpr uint32_t WO = W3 + TC_TILE / 2;  // [16][64] (rows >= NO zero)
  static constexpr uint32_t ACT = WO + 2048;        // [128][64] activations (A operand)
  static constexpr uint32_t BIAS = ACT + TC_TILE;   // b2, b3 (64 each), bo (16) FP32
  static constexpr uint32_t BAR = BIAS + (64 + 64 + 16) * 4;
  static constexpr uint32_t TMEMP = BAR + 8;
  static constexpr uint32_t TOTAL = TMEMP + 8;
};

// Convert a row-major FP32 [rows][64] weight block into a K-major BF16 tile.
__device__ void load_weight_tile(uint8_t* tile, const float* W, int rows, int valid_rows) {
  for (int e = threadIdx.x; e < rows * 64; e += blockDim.x) {
    const int r = e >> 6, k = e & 63;
    st_bf16(tile, r, k, r < valid_rows ? W[r * 64 + k] : 0.f);
  }
}

template <int ROT>
__global__ void __launch_bounds__(128) decode_tc_kernel(TcArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = tc::align1024(smem_raw);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + DecodeSmem::BAR);
  uint32_t* tmem_ptr = reinterpret_cast<uint32_t*>(sm + DecodeSmem::TMEMP);
  float* bias = reinterpret_cast<float*>(sm + DecodeSmem::BIAS);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int H = TC_H, K = a.K, NO = a.NO;

  // weights: W1 (H x K) + b1 | W2 + b2 | W3 + b3 | Wo (NO x H) + bo
  const float* p2 = a.mlp + H * K + H;
  const float* p3 = p2 + H * H + H;
  const float* po = p3 + H * H + H;
  load_weight_tile(sm + DecodeSmem::W2, p2, 64, 64);
  load_weight_tile(sm + DecodeSmem::W3, p3, 64, 64);
  load_weight_tile(sm + DecodeSmem::WO, po, 16, NO);
  for (int k = tid; k < 64; k += 128) {
    bias[k] = p2[H * H + k];
    bias[64 + k] = p3[H * H + k];
  }
  if (tid < 16) bias[128 + tid] = tid < NO ? po[NO * H + tid] : 0.f;
  if (tid == 0) {
    tc::mbar_init(bar, 1);
    tc::fence_mbar_init();
  }
  if (warp == 0) {
    tc::tmem_alloc(tmem_ptr, 64);
    tc::tmem_relinquish();
  }
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_ptr;
  const uint32_t lane = tmem + ((uint32_t)(warp * 32) << 16);
  const uint32_t s_act = tc::smem_u32(sm + DecodeSmem::ACT);
  const uint32_t s_w2 = tc::smem_u32(sm + DecodeSmem::W2);
  const uint32_t s_w3 = tc::smem_u32(sm + DecodeSmem::W3);
  const uint32_t s_wo = tc::smem_u32(sm + DecodeSmem::WO);
  constexpr uint32_t ID64 = tc::idesc_bf16(128, 64, false, false);
  constexpr uint32_t ID16 = tc::idesc_bf16(128, 16, false, false);
  uint32_t phase = 0;
  bool ok = true, run = true;
  const long long rows = (long long)a.N * a.T;
  const long long ntiles = (rows + TC_ROWS - 1) / TC_ROWS;
  uint8_t* act = sm + DecodeSmem::ACT;

  // One barrier per layer: it publishes the activation tile to the tensor
  // core, orders every lane's TMEM reads of the previous layer before the
  // next MMA overwrites the accumulator, and agrees on the waits' outcome.
  // A thread writes the next activation into `act` right after its own wait
  // (the MMA that read `act` has completed).
  for (long long tile = blockIdx.x; tile < ntiles && run; tile += gridDim.x) {
    const long long row = tile * TC_ROWS + tid;
    const bool valid = row < rows;
    const int t = valid ? (int)(row / a.N) : 0;
    const int i = valid ? (int)(row - (long long)t * a.N) : 0;
    float v[64];
    if (valid) {
      const float4* u4 = reinterpret_cast<const float4*>(a.U + (long long)i * H);
      const float4* v4 = reinterpret_cast<const float4*>(a.V + (long long)t * H);
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const float4 u = u4[k], w = v4[k];
        v[4 * k + 0] = leaky(u.x + w.x, a.slope);
        v[4 * k + 1] = leaky(u.y + w.y, a.slope);
        v[4 * k + 2] = leaky(u.z + w.z, a.slope);
        v[4 * k + 3] = leaky(u.w + w.w, a.slope);
      }
    } else {
#pragma unroll
      for (int k = 0; k < 64; ++k) v[k] = 0.f;
    }
    st_row64(act, tid, v);
    // two hidden layers, then the output layer
#pragma unroll 1
    for (int layer = 0; layer < 3; ++layer) {
      tc::fence_async_smem();
      tc::fence_before_sync();
      run = __syncthreads_and(ok) != 0;
      tc::fence_after_sync();
      if (!run) break;
      if (warp == 0) {  // descriptors from the whole warp, one elected lane issues
        const uint64_t da = tc::kmajor_sw128(s_act);
        const uint64_t db = tc::kmajor_sw128(layer == 0 ? s_w2 : layer == 1 ? s_w3 : s_wo);
        if (tc::elect_one()) {
          mma_k64(tmem, da, db, layer < 2 ? ID64 : ID16);
          tc::mma_commit(bar);
        }
        __syncwarp();
      }
      if (!tc::mbar_wait(bar, phase, WAIT_TRIES)) {
        ok = false;
        atomicExch(a.err, 1);
      }
      phase ^= 1u;
      tc::fence_after_sync();
      if (layer < 2) {
        uint32_t r[64];
        tc::tmem_ld64_wait(lane, r);
        const float* b = bias + 64 * layer;
#pragma unroll
        for (int k = 0; k < 64; ++k) v[k] = leaky(__uint_as_float(r[k]) + b[k], a.slope);
        st_row64(act, tid, v);
      } else {
        uint32_t r[16];
        tc::tmem_ld16(lane, r);
        tc::tmem_ld_wait();
        float o[7];
#pragma unroll
        for (int j = 0; j < 7; ++j) o[j] = __uint_as_float(r[j]) + bias[128 + j];
        if (valid) {
          float4 xh, dl;
          transform<ROT>(o, a.alpha, a.xr[i], xh, dl);
          a.xhat[row] = xh;
          a.disp[row] = dl;
        }
      }
    }
  }
  // every lane's TMEM reads are complete before the columns are freed
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, 64);
}

cudaError_t launch_decode_bf16(npg_ctx* c) {
  if (c->md.H == 128) return launch_decode_bf16_h128(c);
  const size_t smem = DecodeSmem::TOTAL + 1024;
  auto k = c->cfg.rot_mode == NPG_ROT_QUAT     ? decode_tc_kernel<0>
           : c->cfg.rot_mode == NPG_ROT_EXPMAP ? decode_tc_kernel<1>
                                               : decode_tc_kernel<2>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long tiles = ((long long)c->N * c->T + TC_ROWS - 1) / TC_ROWS;
  k<<<tc_grid(c, tiles, c->dec_per_sm), 128, smem, c->stream>>>(make_tc_args(c));
  return cudaGetLastError();
}

// ----------------------------------------------------------------- backward
// Hidden width 64: k_mlp_tc64.cu (two CTAs per SM); 128: k_mlp_tc128.cu.
bool backward_bf16_supported(int K, int Z) { return K <= 15 && Z <= 8; }

cudaError_t launch_mlp_backward_bf16(npg_ctx* c) {
  if (c->md.H == 128) return launch_mlp_backward_bf16_h128(c);
  return launch_mlp_backward_bf16_h64(c);
}

}  // namespace npg
