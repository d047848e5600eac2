// BF16 tensor-core (tcgen05) MLP decode and backward (Sec. 3.3-3.4) for
// hidden width 64 and 3 hidden layers: operands in 128B-swizzled shared
// memory, FP32 accumulators in TMEM, FP32 epilogues (bias, LeakyReLU, the
// rotation/translation mapping and its Jacobian) on the CUDA cores.
//
// A CTA of 128 threads owns tiles of 128 consecutive rows (row = t N + i);
// thread t owns row t of the tile and TMEM lane t. One elected thread issues
// the MMAs; completion is tracked by an mbarrier whose waits are bounded: a
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

// Issue D = A * B^T with K = 64 (4 steps of 16), K-major operands.
__device__ __forceinline__ void mma_k64(uint32_t d, uint32_t a_smem, uint32_t b_smem,
                                        uint32_t idesc) {
#pragma unroll
  for (int ks = 0; ks < 4; ++ks)
    tc::mma_bf16(d, tc::kmajor_sw128(a_smem + 32 * ks), tc::kmajor_sw128(b_smem + 32 * ks),
                 idesc, ks > 0);
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
  uint8_t* sm = reinterpret_cast<uint8_t*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
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
      if (tid == 0) {
        if (layer < 2)
          mma_k64(tmem, s_act, layer == 0 ? s_w2 : s_w3, ID64);
        else
          mma_k64(tmem, s_act, s_wo, ID16);
        tc::mma_commit(bar);
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
  k<<<tc_grid(c, tiles, 6), 128, smem, c->stream>>>(make_tc_args(c));
  return cudaGetLastError();
}

// ----------------------------------------------------------------- backward
// Tile = 16 vertices x 8 frames (row r = tl 16 + il). Per tile:
//   forward recompute  h1 = act(U + V), h2, h3 (layer MMAs), o (output MMA)
//   dL/do              Eq. 5-7 Jacobians in FP32 -> gO tile
//   dh3 = gO Wo, dpre3 = dh3 act'(h3); dh2 = dpre3 W3, dpre2; dh1 = dpre2 W2, dpre1
//   weight gradients, accumulated in TMEM over all tiles of the CTA:
//     ACC_W += [dpre3 | dpre2]^T [h2 | h1 | y]   (M 128, N 144, K = 128 rows)
//     ACC_X += [gO | dpre1]^T [y | h3]           (M 128, N 128)
//   where y = (z_i, gamma_t, 0.., 1 at column 15): the diagonal blocks are
//   dW3, dW2 and dW_out, dW1, the column of ones gives the bias gradients.
//   dL/dz rows = dpre1 W1[:, :Z] (an N = 16 MMA), summed over the tile's frames.
//
// A CTA of 512 threads (16 warps) owns one tile at a time: warp w serves TMEM
// lanes 32 (w % 4) .. + 31 (its tile rows) and the 16-column quarter
// c = w / 4 of every 64-wide activation, so each thread converts, masks and
// stores 16 values per layer. Per-row scalar work is spread over the
// quarters and overlapped in one phase: while c = 0 forms dL/do, c = 1 writes
// the y row and c >= 2 sums and adds the previous tile's dL/dz partials. The
// output-bias gradient stays in per-thread FP32 registers until the CTA ends.
// Warps 2..15 issue the bulk copies of the next tile's inputs (U, V, x,
// dL/dx-hat, z and gamma rows) into a second shared staging buffer during the
// current tile's first MMA. The next tile's h1 is written before the current
// tile's last barrier, and the last weight-gradient MMA is not waited for:
// the next tile's first MMA commit covers it.
struct BwdStage {  // inputs of one tile, FP32
  static constexpr uint32_t U_PITCH = 272;    // 256 B + 16: the 16 vertex rows hit distinct banks
  static constexpr uint32_t U = 0;            // [16 vertices][64], rows U_PITCH apart
  static constexpr uint32_t V = 4352;         // [8 frames][64]
  static constexpr uint32_t X = 6400;         // [16] float4 x_i
  static constexpr uint32_t G = 6656;         // [8][16] float4 dL/dx-hat
  static constexpr uint32_t Z = 8704;         // [16][Z] z_i (Z <= 8)
  static constexpr uint32_t GAM = 9216;       // [8 frames][2M] gamma_t (2M <= 16)
  static constexpr uint32_t BYTES = 9728;
};
struct BwdSmem {
  // B operands of the forward and dh MMAs (K-major)
  static constexpr uint32_t W2 = 0, W3 = 8192, WO = 16384, W2T = 18432, W3T = 26624,
                            WOT = 34816;  // [64][64]: (m, q) = Wo[q][m]
  // [h2 | h1 | y | h3] then [gO | dpre3 | dpre2], 16 KB tiles
  static constexpr uint32_t H2 = 43008, H1 = H2 + TC_TILE, Y = H1 + TC_TILE, H3 = Y + TC_TILE;
  static constexpr uint32_t GO = H3 + TC_TILE, DP3 = GO + TC_TILE, DP2 = DP3 + TC_TILE;
  static constexpr uint32_t W1Z = DP2 + TC_TILE;  // BF16 K-major [16][64]: W1[:, :Z]^T, rows >= Z zero
  static constexpr uint32_t BIAS = W1Z + 2048;                  // b2, b3, bo FP32
  static constexpr uint32_t DZP = BIAS + (64 + 64 + 16) * 4;    // FP32 [8 qz][4 q4][16 vertices]
  static constexpr uint32_t STG = DZP + 8 * 64 * 4;             // 2 x BwdStage
  static constexpr uint32_t DBO = STG + 2 * BwdStage::BYTES;    // FP32 [8] output-bias gradient
  // mbarriers: chain MMAs, final drain, dL/dz MMA, staging buffer 0 and 1
  static constexpr uint32_t BAR = DBO + 8 * 4;
  static constexpr uint32_t TMEMP = BAR + 5 * 8;
  static constexpr uint32_t TOTAL = TMEMP + 8;
};
constexpr uint32_t ACC_W_COL = 0, ACC_X_COL = 256, WORK_COL = 384, DZ_COL = 448;
constexpr int BWD_THREADS = 512;

bool backward_bf16_supported(int K, int Z) { return K <= 15 && Z <= 8; }

// 16 FP32 values as BF16 into columns [c0, c0 + 16) of a row of a K-major tile.
__device__ __forceinline__ void st_row16(uint8_t* tile, int row, int c0, const float* v) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    uint4 q;
    q.x = tc::pack_bf16(v[8 * h + 0], v[8 * h + 1]);
    q.y = tc::pack_bf16(v[8 * h + 2], v[8 * h + 3]);
    q.z = tc::pack_bf16(v[8 * h + 4], v[8 * h + 5]);
    q.w = tc::pack_bf16(v[8 * h + 6], v[8 * h + 7]);
    *reinterpret_cast<uint4*>(tile + tc::sw128_off(row, c0 + 8 * h)) = q;
  }
}

// D (128 x N) += A^T B with A, B MN-major [128 rows][64] tiles placed 16 KB
// apart along M / N; K = the 128 rows of the tile (8 steps of 16).
__device__ __forceinline__ void mma_rows(uint32_t d, uint32_t a_smem, uint32_t b_smem,
                                         uint32_t idesc, bool first) {
#pragma unroll
  for (int ks = 0; ks < 8; ++ks)
    tc::mma_bf16(d, tc::mnmajor_sw128(a_smem + 2048 * ks, TC_TILE, 1024),
                 tc::mnmajor_sw128(b_smem + 2048 * ks, TC_TILE, 1024), idesc,
                 (first && ks == 0) ? 0u : 1u);
}

// Issue the bulk copies of one tile's inputs into a staging buffer. The 28
// pieces (16 U rows, 8 dL/dx-hat frame rows, V, x, z, gamma) are spread over
// STAGE_WARPS warps, lane l of part p taking piece p + STAGE_WARPS l; each
// warp announces its own bytes on *sbar (initialised with one arrival per
// warp). Vertices past N and frames past T are not copied: their staging rows
// keep stale (or never written) values, which every reader replaces by zero
// through a select. The z and gamma copies round up to 16 B; those arrays
// carry 16 B of padding.
constexpr int STAGE_WARPS = 14, STAGE_PIECES = 28;
__device__ void bwd_stage(const TcArgs& a, int i0, int t0, uint8_t* stg, uint64_t* sbar,
                          int part, int lane) {
  const int nv = min(16, a.N - i0), nf = min(8, a.T - t0);
  const uint32_t zb = ((uint32_t)(nv * a.Z * 4) + 15u) & ~15u;
  const uint32_t gb = ((uint32_t)(nf * 2 * a.M * 4) + 15u) & ~15u;
  // bytes of piece k (0: not copied)
  auto piece_bytes = [&](int k) -> uint32_t {
    if (k < 16) return k < nv ? 256u : 0u;
    if (k < 24) return k - 16 < nf ? (uint32_t)nv * 16u : 0u;
    if (k == 24) return (uint32_t)nf * 256u;
    if (k == 25) return (uint32_t)nv * 16u;
    return k == 26 ? zb : gb;
  };
  if (lane == 0) {
    uint32_t total = 0u;
    for (int k = part; k < STAGE_PIECES; k += STAGE_WARPS) total += piece_bytes(k);
    tc::mbar_arrive_expect_tx(sbar, total);
  }
  __syncwarp();
  const int k = part + STAGE_WARPS * lane;
  if (k >= STAGE_PIECES) return;
  const uint32_t n = piece_bytes(k);
  if (n == 0u) return;
  if (k < 16)
    tc::bulk_g2s(stg + BwdStage::U + k * BwdStage::U_PITCH, a.U + (long long)(i0 + k) * TC_H, n,
                 sbar);
  else if (k < 24)
    tc::bulk_g2s(stg + BwdStage::G + (k - 16) * 256, a.dxhat + (long long)(t0 + k - 16) * a.N + i0,
                 n, sbar);
  else if (k == 24)
    tc::bulk_g2s(stg + BwdStage::V, a.V + (long long)t0 * TC_H, n, sbar);
  else if (k == 25)
    tc::bulk_g2s(stg + BwdStage::X, a.xr + i0, n, sbar);
  else if (k == 26)
    tc::bulk_g2s(stg + BwdStage::Z, a.z + (long long)i0 * a.Z, n, sbar);
  else
    tc::bulk_g2s(stg + BwdStage::GAM, a.gamma + (long long)t0 * 2 * a.M, n, sbar);
}

template <int ROT>
__global__ void __launch_bounds__(BWD_THREADS, 1) mlp_bwd_tc_kernel(TcArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + BwdSmem::BAR);
  uint32_t* tmem_ptr = reinterpret_cast<uint32_t*>(sm + BwdSmem::TMEMP);
  float* bias = reinterpret_cast<float*>(sm + BwdSmem::BIAS);
  float* dzp = reinterpret_cast<float*>(sm + BwdSmem::DZP);
  float* dbo = reinterpret_cast<float*>(sm + BwdSmem::DBO);
  uint64_t* sbar = bar + 3;  // staging buffers
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int q4 = warp & 3, c = warp >> 2;  // lane quarter, column quarter
  const int row = 32 * q4 + lane, il = row & 15, tl = row >> 4;
  const int H = TC_H, K = a.K, Z = a.Z, NO = a.NO;
  if (tid < 8) dbo[tid] = 0.f;

  const float* p2 = a.mlp + H * K + H;
  const float* p3 = p2 + H * H + H;
  const float* po = p3 + H * H + H;
  load_weight_tile(sm + BwdSmem::W2, p2, 64, 64);
  load_weight_tile(sm + BwdSmem::W3, p3, 64, 64);
  load_weight_tile(sm + BwdSmem::WO, po, 16, NO);
  for (int e = tid; e < 64 * 64; e += BWD_THREADS) {
    const int m = e >> 6, j = e & 63;
    st_bf16(sm + BwdSmem::W2T, m, j, p2[j * H + m]);
    st_bf16(sm + BwdSmem::W3T, m, j, p3[j * H + m]);
    st_bf16(sm + BwdSmem::WOT, m, j, j < NO ? po[j * H + m] : 0.f);
  }
  {  // gO and y start zero; their columns >= 16 stay zero, y column 15 stays 1
    const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
    for (int e = tid; e < 2 * TC_TILE / 16; e += BWD_THREADS) {
      const uint32_t off = (uint32_t)(e % (TC_TILE / 16)) * 16u;
      *reinterpret_cast<uint4*>(sm + (e < TC_TILE / 16 ? BwdSmem::GO : BwdSmem::Y) + off) = zero;
    }
  }
  for (int e = tid; e < 16 * 64; e += BWD_THREADS) {
    const int qz = e >> 6, m = e & 63;
    st_bf16(sm + BwdSmem::W1Z, qz, m, qz < Z ? a.mlp[m * K + qz] : 0.f);
  }
  for (int k = tid; k < 64; k += BWD_THREADS) {
    bias[k] = p2[H * H + k];
    bias[64 + k] = p3[H * H + k];
  }
  if (tid < 16) bias[128 + tid] = tid < NO ? po[NO * H + tid] : 0.f;
  if (tid == 0) {
    for (int b = 0; b < 3; ++b) tc::mbar_init(bar + b, 1);
    for (int b = 3; b < 5; ++b) tc::mbar_init(bar + b, STAGE_WARPS);
    tc::fence_mbar_init();
  }
  if (warp == 0) {
    tc::tmem_alloc(tmem_ptr, 512);
    tc::tmem_relinquish();
  }
  // tile = ib n_tb + tb covers vertices 16 ib.. and frames 8 tb.. (the host
  // checks that the tile count fits an int)
  const int n_tb = (a.T + 7) / 8;
  const int ntiles = ((a.N + 15) / 16) * n_tb;
  int tile = blockIdx.x;
  int i0 = 0, t0 = 0;  // first vertex and frame of `tile`
  if (tile < ntiles) {
    i0 = tile / n_tb * 16;
    t0 = (tile - i0 / 16 * n_tb) * 8;
  }
  __syncthreads();  // zeroed y before its column 15 is set; barriers initialised
  if (c == 1) st_bf16(sm + BwdSmem::Y, row, 15, 1.f);
  bool ok = tc_sync_ok(true, a.err);
  // staging: warps 16 - STAGE_WARPS .. 15 (two pieces each; warp 0 issues the
  // MMAs) issue a tile's copies, every thread waits on the buffer's barrier
  // before its first read (parity and in-flight bit per buffer)
  uint32_t sphase = 0u, pending = 0u;
  auto stage_issue = [&](int b, int i0_, int t0_) {
    const int part = warp - (16 - STAGE_WARPS);
    if (part >= 0)
      bwd_stage(a, i0_, t0_, sm + BwdSmem::STG + b * BwdStage::BYTES, sbar + b, part, lane);
    pending |= 1u << b;
  };
  auto stage_wait = [&](int b) {
    ok = ok && tc::mbar_wait(sbar + b, (sphase >> b) & 1u, WAIT_TRIES);
    sphase ^= 1u << b;
    pending &= ~(1u << b);
  };
  if (tile < ntiles) stage_issue(0, i0, t0);
  const uint32_t tmem = *tmem_ptr;
  const uint32_t lane_addr = tmem + ((uint32_t)(q4 * 32) << 16);
  auto sa = [&](uint32_t off) { return tc::smem_u32(sm + off); };
  constexpr uint32_t ID64 = tc::idesc_bf16(128, 64, false, false);
  constexpr uint32_t ID16 = tc::idesc_bf16(128, 16, false, false);
  constexpr uint32_t IDW = tc::idesc_bf16(128, 144, true, true);
  constexpr uint32_t IDX = tc::idesc_bf16(128, 128, true, true);
  uint32_t phase = 0, phase_dz = 0;
  bool first = true;
  const float* b2 = bias + 16 * c;
  const float* b3 = bias + 64 + 16 * c;

  // h1 of the tile staged in `stg`: act' mask and the H1 store
  auto put_h1 = [&](const uint8_t* stg, bool valid) {
    const float4* u4 =
        reinterpret_cast<const float4*>(stg + BwdStage::U + il * BwdStage::U_PITCH + 64 * c);
    const float4* v4 = reinterpret_cast<const float4*>(stg + BwdStage::V + tl * 256 + 64 * c);
    float v[16];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float4 u = u4[k], w = v4[k];
      v[4 * k + 0] = valid ? leaky(u.x + w.x, a.slope) : 0.f;
      v[4 * k + 1] = valid ? leaky(u.y + w.y, a.slope) : 0.f;
      v[4 * k + 2] = valid ? leaky(u.z + w.z, a.slope) : 0.f;
      v[4 * k + 3] = valid ? leaky(u.w + w.w, a.slope) : 0.f;
    }
    uint32_t m = 0u;
#pragma unroll
    for (int k = 0; k < 16; ++k) m |= (v[k] > 0.f ? 1u : 0u) << k;
    st_row16(sm + BwdSmem::H1, row, 16 * c, v);
    return m;
  };
  auto row_valid = [&](int i0_, int t0_) { return i0_ + il < a.N && t0_ + tl < a.T; };

  uint32_t m1 = 0u;
  int buf = 0;
  int dz_i0 = -1;  // first vertex of the tile whose dL/dz partials wait in dzp
  float dbo_acc[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  // dL/dz of the tile whose partials are in dzp: sum over its 8 frames (two
  // per warp quarter, pre-summed), one global add per value
  auto flush_dz = [&](int e0, int stride) {
    for (int e = e0; e < 16 * Z; e += stride) {
      const int vi = e & 15, qz = e >> 4;
      if (dz_i0 + vi >= a.N) continue;
      float s = 0.f;
#pragma unroll
      for (int q = 0; q < 4; ++q) s += dzp[(qz * 4 + q) * 16 + vi];
      atomicAdd(a.dz + (long long)(dz_i0 + vi) * Z + qz, s);
    }
  };
  if (tile < ntiles) {
    stage_wait(0);
    m1 = put_h1(sm + BwdSmem::STG, row_valid(i0, t0));
  }
  // `ok` leaves the loop only through tc_sync_ok, so every thread breaks at
  // the same barrier
  for (; tile < ntiles; tile += gridDim.x) {
    uint8_t* stg = sm + BwdSmem::STG + buf * BwdStage::BYTES;
    const bool valid = row_valid(i0, t0);
    // ---- forward: layer 2
    if (!(ok = tc_sync_ok(ok, a.err))) break;
    if (tid == 0) {
      mma_k64(tmem + WORK_COL, sa(BwdSmem::H1), sa(BwdSmem::W2), ID64);
      tc::mma_commit(bar);
    }
    // the next tile's coordinates, while the MMA runs
    const int next = tile + (int)gridDim.x;
    int ni0 = 0, nt0 = 0;
    if (next < ntiles) {
      ni0 = next / n_tb * 16;
      nt0 = (next - ni0 / 16 * n_tb) * 8;
    }
    // the next tile's inputs copy while this tile computes (the buffer's last
    // readers, the previous tile's dL/do and y row, are behind several barriers)
    if (next < ntiles) stage_issue(buf ^ 1, ni0, nt0);
    tc_wait(bar, phase, ok);
    uint32_t m2 = 0u, m3 = 0u;
    {
      float v[16];
      ld_col16(lane_addr + WORK_COL + 16 * c, v);
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        v[k] = leaky(v[k] + b2[k], a.slope);
        m2 |= (v[k] > 0.f ? 1u : 0u) << k;
      }
      st_row16(sm + BwdSmem::H2, row, 16 * c, v);
    }
    // ---- layer 3
    if (!(ok = tc_sync_ok(ok, a.err))) break;
    if (tid == 0) {
      mma_k64(tmem + WORK_COL, sa(BwdSmem::H2), sa(BwdSmem::W3), ID64);
      tc::mma_commit(bar);
    }
    tc_wait(bar, phase, ok);
    {
      float v[16];
      ld_col16(lane_addr + WORK_COL + 16 * c, v);
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        v[k] = leaky(v[k] + b3[k], a.slope);
        m3 |= (v[k] > 0.f ? 1u : 0u) << k;
      }
      st_row16(sm + BwdSmem::H3, row, 16 * c, v);
    }
    // ---- output layer, then dL/do (quarter 0)
    if (!(ok = tc_sync_ok(ok, a.err))) break;
    if (tid == 0) {
      mma_k64(tmem + WORK_COL, sa(BwdSmem::H3), sa(BwdSmem::WO), ID16);
      tc::mma_commit(bar);
    }
    tc_wait(bar, phase, ok);
    if (c == 0) {
      float r[16];
      ld_col16(lane_addr + WORK_COL, r);
      float o[7], go[7];
#pragma unroll
      for (int j = 0; j < 7; ++j) {
        o[j] = r[j] + bias[128 + j];
        go[j] = 0.f;
      }
      if (valid) {
        const float4 x = reinterpret_cast<const float4*>(stg + BwdStage::X)[il];
        const float4 g = reinterpret_cast<const float4*>(stg + BwdStage::G)[tl * 16 + il];
        transform_backward<ROT>(o, a.alpha, x, g, go);
      }
      // output-bias gradient: summed in FP32 (rows cancel strongly; a BF16
      // rounding of each row's dL/do would dominate the sum)
#pragma unroll
      for (int j = 0; j < 7; ++j) dbo_acc[j] += go[j];
      uint4 q0;
      q0.x = tc::pack_bf16(go[0], go[1]);
      q0.y = tc::pack_bf16(go[2], go[3]);
      q0.z = tc::pack_bf16(go[4], go[5]);
      q0.w = tc::pack_bf16(NO > 6 ? go[6] : 0.f, 0.f);
      *reinterpret_cast<uint4*>(sm + BwdSmem::GO + tc::sw128_off(row, 0)) = q0;
    } else if (c == 1) {
      // y row: z_i, gamma_t in columns 0..K-1, zeros, 1 in column 15 (first
      // read by the ACC_W MMA, after the dh2 step)
      const float* zs = reinterpret_cast<const float*>(stg + BwdStage::Z) + il * Z;
      const float* gt = reinterpret_cast<const float*>(stg + BwdStage::GAM) + tl * (K - Z);
      float y[16];
#pragma unroll
      for (int k = 0; k < 16; ++k)
        y[k] = k == 15 ? 1.f : !valid ? 0.f : k < Z ? zs[k] : k < K ? gt[k - Z] : 0.f;
      st_row16(sm + BwdSmem::Y, row, 0, y);
    } else if (dz_i0 >= 0) {
      flush_dz(tid - 256, 256);  // 16 Z <= 128 values: warps 8..11
    }
    // ---- backward: dh3 = gO Wo (K = 16)
    if (!(ok = tc_sync_ok(ok, a.err))) break;
    if (tid == 0) {
      tc::mma_bf16(tmem + WORK_COL, tc::kmajor_sw128(sa(BwdSmem::GO)),
                   tc::kmajor_sw128(sa(BwdSmem::WOT)), ID64, 0u);
      tc::mma_commit(bar);
    }
    tc_wait(bar, phase, ok);
    {
      float v[16];
      ld_col16(lane_addr + WORK_COL + 16 * c, v);
#pragma unroll
      for (int k = 0; k < 16; ++k) v[k] *= ((m3 >> k) & 1u) ? 1.f : a.slope;
      st_row16(sm + BwdSmem::DP3, row, 16 * c, v);
    }
    // ---- dh2 = dpre3 W3
    if (!(ok = tc_sync_ok(ok, a.err))) break;
    if (tid == 0) {
      mma_k64(tmem + WORK_COL, sa(BwdSmem::DP3), sa(BwdSmem::W3T), ID64);
      tc::mma_commit(bar);
    }
    tc_wait(bar, phase, ok);
    {
      float v[16];
      ld_col16(lane_addr + WORK_COL + 16 * c, v);
#pragma unroll
      for (int k = 0; k < 16; ++k) v[k] *= ((m2 >> k) & 1u) ? 1.f : a.slope;
      st_row16(sm + BwdSmem::DP2, row, 16 * c, v);
    }
    // ---- ACC_W += [dpre3 | dpre2]^T [h2 | h1 | y]; dh1 = dpre2 W2
    if (!(ok = tc_sync_ok(ok, a.err))) break;
    if (tid == 0) {
      mma_rows(tmem + ACC_W_COL, sa(BwdSmem::DP3), sa(BwdSmem::H2), IDW, first);
      mma_k64(tmem + WORK_COL, sa(BwdSmem::DP2), sa(BwdSmem::W2T), ID64);
      tc::mma_commit(bar);
    }
    tc_wait(bar, phase, ok);
    {
      float v[16];
      ld_col16(lane_addr + WORK_COL + 16 * c, v);
#pragma unroll
      for (int k = 0; k < 16; ++k) v[k] *= ((m1 >> k) & 1u) ? 1.f : a.slope;
      st_row16(sm + BwdSmem::DP3, row, 16 * c, v);  // dpre1 (ACC_W has consumed dpre3)
    }
    // the next tile's h1 (ACC_W, the last reader of H1, has completed); the
    // current m1 is used up
    if (next < ntiles) {
      stage_wait(buf ^ 1);
      m1 = put_h1(sm + BwdSmem::STG + (buf ^ 1) * BwdStage::BYTES, row_valid(ni0, nt0));
    }
    // ---- dL/dz rows = dpre1 W1[:, :Z] (N = 16); ACC_X += [gO | dpre1]^T [y | h3]
    if (!(ok = tc_sync_ok(ok, a.err))) break;
    // ACC_X is not waited for here: the next tile's first commit also covers
    // it, and nothing before that wait writes a tile ACC_X reads
    if (tid == 0) {
      mma_k64(tmem + DZ_COL, sa(BwdSmem::DP3), sa(BwdSmem::W1Z), ID16);
      tc::mma_commit(bar + 2);
      mma_rows(tmem + ACC_X_COL, sa(BwdSmem::GO), sa(BwdSmem::Y), IDX, first);
    }
    first = false;
    dz_i0 = i0;
    // dL/dz partials (quarter 1; warp 0 is issuing), summed with lane ^ 16
    // (the same vertex, the warp's other frame)
    if (c == 1) {
      tc_wait(bar + 2, phase_dz, ok);
      float r[16];
      ld_col16(lane_addr + DZ_COL, r);
#pragma unroll
      for (int qz = 0; qz < 8; ++qz) {
        if (qz < Z) {
          const float s = r[qz] + __shfl_xor_sync(0xffffffffu, r[qz], 16);
          if (lane < 16) dzp[(qz * 4 + q4) * 16 + lane] = s;
        }
      }
    }
    buf ^= 1;
    i0 = ni0;
    t0 = nt0;
  }
  // the last ACC_X
  if (!first) {
    if (tid == 0) tc::mma_commit(bar);
    tc_wait(bar, phase, ok);
  }
  // the last tile's dL/dz partials; the output-bias gradient of quarter 0
  ok = tc_sync_ok(ok, a.err);
  if (ok && dz_i0 >= 0) flush_dz(tid, BWD_THREADS);
  if (c == 0) {
#pragma unroll
    for (int j = 0; j < 7; ++j) {
      float sj = dbo_acc[j];
#pragma unroll
      for (int o2 = 16; o2 > 0; o2 >>= 1) sj += __shfl_xor_sync(0xffffffffu, sj, o2);
      if (lane == 0 && j < NO) atomicAdd(dbo + j, sj);
    }
  }
  // ---- accumulators -> global gradient (parameter layout), once per CTA
  ok = tc_sync_ok(ok, a.err);
  if (ok && !first) {
    float* g = a.g_mlp;
    float* gW1 = g;
    float* gb1 = g + H * K;
    float* gW2 = gb1 + H;
    float* gb2 = gW2 + H * H;
    float* gW3 = gb2 + H;
    float* gb3 = gW3 + H * H;
    float* gWo = gb3 + H;
    float* gbo = gWo + NO * H;
    float v[16];
    // ACC_W rows 0..63: dW3 (cols 0..63), db3 (col 143); rows 64..127: dW2
    // (cols 64..127), db2 (col 143)
    const int wr = row < 64 ? row : row - 64;
    ld_col16(lane_addr + ACC_W_COL + (row < 64 ? 0 : 64) + 16 * c, v);
    float* gW = row < 64 ? gW3 : gW2;
#pragma unroll
    for (int k = 0; k < 16; ++k) atomicAdd(gW + wr * H + 16 * c + k, v[k]);
    if (c == 0) {
      ld_col16(lane_addr + ACC_W_COL + 128, v);
      atomicAdd((row < 64 ? gb3 : gb2) + wr, v[15]);
    }
    // ACC_X rows 0..NO-1: dW_out (cols 64..127); rows 64..127: dW1 (cols
    // 0..K-1), db1 (col 15)
    if (q4 < 2) {  // rows 0..63
      ld_col16(lane_addr + ACC_X_COL + 64 + 16 * c, v);
      if (row < NO) {
#pragma unroll
        for (int k = 0; k < 16; ++k) atomicAdd(gWo + row * H + 16 * c + k, v[k]);
        if (c == 0) atomicAdd(gbo + row, dbo[row]);
      }
    } else if (c == 0) {
      ld_col16(lane_addr + ACC_X_COL, v);
#pragma unroll
      for (int k = 0; k < 16; ++k)
        if (k < K) atomicAdd(gW1 + (row - 64) * K + k, v[k]);
      atomicAdd(gb1 + (row - 64), v[15]);
    }
  }
  // drain (bounded): no copy or MMA of this CTA may be in flight when it exits
  for (int b = 0; b < 2; ++b)
    if (pending & (1u << b)) tc::mbar_wait(sbar + b, (sphase >> b) & 1u, WAIT_TRIES);
  if (tid == 0) {
    tc::mma_commit(bar + 1);
    tc::mbar_wait(bar + 1, 0, WAIT_TRIES);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

cudaError_t launch_mlp_backward_bf16(npg_ctx* c) {
  if (c->md.H == 128) return launch_mlp_backward_bf16_h128(c);
  if (c->md.H == 64) return launch_mlp_backward_bf16_h64(c);
  const size_t smem = BwdSmem::TOTAL + 1024;
  auto k = c->cfg.rot_mode == NPG_ROT_QUAT     ? mlp_bwd_tc_kernel<0>
           : c->cfg.rot_mode == NPG_ROT_EXPMAP ? mlp_bwd_tc_kernel<1>
                                               : mlp_bwd_tc_kernel<2>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long tiles = (long long)((c->N + 15) / 16) * ((c->T + 7) / 8);
  if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;  // tile indices are ints
  k<<<tc_grid(c, tiles, 1), BWD_THREADS, smem, c->stream>>>(make_tc_args(c));
  return cudaGetLastError();
}

}  // namespace npg
