// BF16 tensor-core (tcgen05) MLP decode and backward (Sec. 3.3-3.4) for
// hidden width 128 and 3 hidden layers: operands in 128B-swizzled shared
// memory, FP32 accumulators in TMEM, FP32 epilogues on the CUDA cores.
//
// A [128 rows][128] BF16 activation tile is two K-major [128][64] blocks, 16 KB
// apart. The same two blocks are the MN-major operand (K = rows, M or N = the
// 128 features, the 64-wide halves 16 KB apart) that the weight-gradient
// MMAs read, and a K-major [out][in] weight tile is also the MN-major
// operand of the input-gradient MMAs, so no transposed copies are kept.
#include "mlp_tc_common.cuh"

namespace npg {

namespace {
constexpr int H2X = 128;
constexpr uint32_t ACT = 2 * TC_TILE;  // one [128][128] BF16 tile: 32 KB

// 32 FP32 values as BF16 into columns [c0, c0 + 32) of one row of a
// [128][128] tile (c0 % 32 == 0).
__device__ __forceinline__ void st_row32(uint8_t* tile, int row, int c0, const float* v) {
  uint8_t* blk = tile + (c0 >> 6) * TC_TILE;
  const int cb = c0 & 63;
#pragma unroll
  for (int h = 0; h < 4; ++h) st_bf16x8(blk, row, cb + 8 * h, v + 8 * h);
}

// [rows][128] FP32 row-major weights (rows >= valid_rows zero) into a K-major
// [rows][128] BF16 tile: two [rows][64] blocks `blk` bytes apart.
__device__ void load_weight128(uint8_t* tile, uint32_t blk, const float* W, int rows,
                               int valid_rows, int ld, int nthreads) {
  for (int e = threadIdx.x; e < rows * 128; e += nthreads) {
    const int r = e >> 7, k = e & 127;
    st_bf16(tile + (k >> 6) * blk, r, k & 63, r < valid_rows ? W[(long long)r * ld + k] : 0.f);
  }
}

// The MMA helpers take descriptors that warp 0 computed as a whole (one
// elected lane issues): a K step of 16 advances a K-major descriptor's start
// address by 32 B (2 in its 16-byte units), an MN-major one by 2048 B (128);
// the start field cannot carry out of its 14 bits below 256 KB.
__device__ __forceinline__ uint64_t kdesc(uint32_t saddr) { return tc::kmajor_sw128(saddr); }
// MN-major operand whose 64-wide feature halves are one [128][64] tile apart
__device__ __forceinline__ uint64_t mdesc2(uint32_t saddr, uint32_t lbo = TC_TILE) {
  return tc::mnmajor_sw128(saddr, lbo, 1024);
}

// D (M 128 x N) = A B^T over K = 128 features, K-major A (a [128][128] tile)
// and B (rows of `bblk` bytes per 64-K block).
__device__ __forceinline__ void mma_feat(uint32_t d, uint64_t a, uint64_t b, uint32_t bblk,
                                         uint32_t idesc) {
#pragma unroll
  for (int kb = 0; kb < 2; ++kb)
#pragma unroll
    for (int ks = 0; ks < 4; ++ks)
      tc::mma_bf16(d, a + kb * (TC_TILE >> 4) + 2 * ks, b + kb * (bblk >> 4) + 2 * ks, idesc,
                   (kb | ks) ? 1u : 0u);
}

// D (M 128 x N 128) = A W over K = 128 (the weight's output rows): K-major A
// (a [128][128] tile, K = its features), w the MN-major descriptor of a
// K-major [128 out][128 in] weight tile (K = out rows, N = in features).
__device__ __forceinline__ void mma_wT(uint32_t d, uint64_t a, uint64_t w, uint32_t idesc) {
#pragma unroll
  for (int kb = 0; kb < 2; ++kb)
#pragma unroll
    for (int ks = 0; ks < 4; ++ks)
      tc::mma_bf16(d, a + kb * (TC_TILE >> 4) + 2 * ks, w + 128 * (4 * kb + ks), idesc,
                   (kb | ks) ? 1u : 0u);
}

// D (M 128 x N) (+)= A^T B over K = the 128 rows of a tile: A and B MN-major
// descriptors (feature halves 16 KB apart).
__device__ __forceinline__ void mma_rows128(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                            bool first) {
#pragma unroll
  for (int ks = 0; ks < 8; ++ks)
    tc::mma_bf16(d, a + 128 * ks, b + 128 * ks, idesc, (first && ks == 0) ? 0u : 1u);
}
}  // namespace

// ----------------------------------------------------------------- decode
// 256 threads: warp w serves TMEM lanes 32 (w % 4) .. + 31 (its tile rows)
// and the 64-column half w / 4 of every activation. Per 128-row tile: h1 from
// U + V on the CUDA cores, two 128 x 128 x 128 layer MMAs and a 128 x 16 x 128
// output MMA, bias + LeakyReLU and the Eq. 5-7 mapping in the epilogues.
struct Dec128Smem {
  static constexpr uint32_t W2 = 0, W3 = W2 + ACT, WO = W3 + ACT;  // WO: [16][128], 2 KB blocks
  static constexpr uint32_t X = WO + 4096;                        // activation tile
  static constexpr uint32_t BIAS = X + ACT;                       // b2, b3 (128 each), bo (16)
  static constexpr uint32_t BAR = BIAS + (128 + 128 + 16) * 4;
  static constexpr uint32_t TMEMP = BAR + 8;
  static constexpr uint32_t TOTAL = TMEMP + 8;
};
constexpr int DEC128_THREADS = 256;

template <int ROT>
__global__ void __launch_bounds__(DEC128_THREADS, 2) decode_tc128_kernel(TcArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = tc::align1024(smem_raw);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + Dec128Smem::BAR);
  uint32_t* tmem_ptr = reinterpret_cast<uint32_t*>(sm + Dec128Smem::TMEMP);
  float* bias = reinterpret_cast<float*>(sm + Dec128Smem::BIAS);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int q4 = warp & 3, half = warp >> 2;
  const int row_t = 32 * q4 + (tid & 31);
  const int H = H2X, K = a.K, NO = a.NO;
  const float* p2 = a.mlp + H * K + H;
  const float* p3 = p2 + H * H + H;
  const float* po = p3 + H * H + H;
  load_weight128(sm + Dec128Smem::W2, TC_TILE, p2, 128, 128, H, DEC128_THREADS);
  load_weight128(sm + Dec128Smem::W3, TC_TILE, p3, 128, 128, H, DEC128_THREADS);
  load_weight128(sm + Dec128Smem::WO, 2048, po, 16, NO, H, DEC128_THREADS);
  for (int k = tid; k < 128; k += DEC128_THREADS) {
    bias[k] = p2[H * H + k];
    bias[128 + k] = p3[H * H + k];
  }
  if (tid < 16) bias[256 + tid] = tid < NO ? po[NO * H + tid] : 0.f;
  if (tid == 0) {
    tc::mbar_init(bar, 1);
    tc::fence_mbar_init();
  }
  if (warp == 0) {
    tc::tmem_alloc(tmem_ptr, 128);
    tc::tmem_relinquish();
  }
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_ptr;
  const uint32_t lane = tmem + ((uint32_t)(q4 * 32) << 16);
  const uint32_t s_x = tc::smem_u32(sm + Dec128Smem::X);
  const uint32_t s_w2 = tc::smem_u32(sm + Dec128Smem::W2);
  const uint32_t s_w3 = tc::smem_u32(sm + Dec128Smem::W3);
  const uint32_t s_wo = tc::smem_u32(sm + Dec128Smem::WO);
  constexpr uint32_t ID128 = tc::idesc_bf16(128, 128, false, false);
  constexpr uint32_t ID16 = tc::idesc_bf16(128, 16, false, false);
  uint32_t phase = 0;
  bool ok = true;
  const long long rows = (long long)a.N * a.T;
  const long long ntiles = (rows + TC_ROWS - 1) / TC_ROWS;
  uint8_t* xt = sm + Dec128Smem::X;
  const int c0 = 64 * half;

  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long row = tile * TC_ROWS + row_t;
    const bool valid = row < rows;
    const int t = valid ? (int)(row / a.N) : 0;
    const int i = valid ? (int)(row - (long long)t * a.N) : 0;
    {
      float v[64];
      const float4* u4 = reinterpret_cast<const float4*>(a.U + (long long)i * H + c0);
      const float4* v4 = reinterpret_cast<const float4*>(a.V + (long long)t * H + c0);
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const float4 u = valid ? u4[k] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 w = valid ? v4[k] : make_float4(0.f, 0.f, 0.f, 0.f);
        v[4 * k + 0] = leaky(u.x + w.x, a.slope);
        v[4 * k + 1] = leaky(u.y + w.y, a.slope);
        v[4 * k + 2] = leaky(u.z + w.z, a.slope);
        v[4 * k + 3] = leaky(u.w + w.w, a.slope);
      }
#pragma unroll
      for (int h = 0; h < 8; ++h) st_bf16x8(xt + half * TC_TILE, row_t, 8 * h, v + 8 * h);
    }
#pragma unroll 1
    for (int layer = 0; layer < 3; ++layer) {
      if (!(ok = tc_sync_ok(ok, a.err))) break;
      if (warp == 0) {
        const uint64_t da = kdesc(s_x);
        const uint64_t db = kdesc(layer == 0 ? s_w2 : layer == 1 ? s_w3 : s_wo);
        if (tc::elect_one()) {
          if (layer < 2)
            mma_feat(tmem, da, db, TC_TILE, ID128);
          else
            mma_feat(tmem, da, db, 2048, ID16);
          tc::mma_commit(bar);
        }
        __syncwarp();
      }
      tc_wait(bar, phase, ok);
      if (layer < 2) {
        // the MMA that read the tile has completed: overwrite it in place
        const float* b = bias + 128 * layer + c0;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          float v[32];
          ld_col32(lane + c0 + 32 * q, v);
#pragma unroll
          for (int k = 0; k < 32; ++k) v[k] = leaky(v[k] + b[32 * q + k], a.slope);
          st_row32(xt, row_t, c0 + 32 * q, v);
        }
      } else if (half == 0) {
        float r[16];
        ld_col16(lane, r);
        float o[7];
#pragma unroll
        for (int j = 0; j < 7; ++j) o[j] = r[j] + bias[256 + j];
        if (valid) {
          float4 xh, dl;
          transform<ROT>(o, a.alpha, a.xr[i], xh, dl);
          a.xhat[row] = xh;
          a.disp[row] = dl;
        }
      }
    }
    if (!ok) break;
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, 128);
}

cudaError_t launch_decode_bf16_h128(npg_ctx* c) {
  const size_t smem = Dec128Smem::TOTAL + 1024;
  auto k = c->cfg.rot_mode == NPG_ROT_QUAT     ? decode_tc128_kernel<0>
           : c->cfg.rot_mode == NPG_ROT_EXPMAP ? decode_tc128_kernel<1>
                                               : decode_tc128_kernel<2>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long tiles = ((long long)c->N * c->T + TC_ROWS - 1) / TC_ROWS;
  k<<<tc_grid(c, tiles, 2), DEC128_THREADS, smem, c->stream>>>(make_tc_args(c));
  return cudaGetLastError();
}

// ----------------------------------------------------------------- backward
// Tile = 16 vertices x 8 frames (row r = tl 16 + il), 512 threads: warp w
// serves TMEM lanes 32 (w % 4) .. + 31 (its rows) and the 32-column quarter
// c = w / 4 of every 128-wide activation. Three activation tiles X[a], X[b],
// X[c] rotate roles from tile to tile:
//   1  h1 = act(U + V)                        -> X[a]   (during the previous tile)
//   2  h2 = act(h1 W2^T + b2)                 -> X[b]
//   3  h3 = act(h2 W3^T + b3)                 -> X[c]
//   4  o = h3 Wo^T + bo, dL/do (Eq. 5-7)      -> GO;  y = (z, gamma, .., 1) -> Y
//   5  dh3 = gO Wo, ACC_O += h3^T gO          dpre3 -> X[c]
//   6  dh2 = dpre3 W3, ACC_3 += dpre3^T h2, ACC_B3 += dpre3^T y   dpre2 -> X[b]
//   7  dh1 = dpre2 W2, ACC_2 += dpre2^T h1, ACC_B2 += dpre2^T y   dpre1 -> X[a],
//      the next tile's h1 -> X[b]
//   8  dL/dz rows = dpre1 W1[:, :Z], ACC_B1 += dpre1^T y
// and the next tile uses (a, b, c) <- (b, c, a). ACC_3 / ACC_2 hold dW3 / dW2,
// ACC_O dWo^T, the ACC_B blocks the bias gradients (the column of ones in y)
// and dW1 | db1; all accumulate in TMEM over the CTA's tiles. Every MMA
// issued before a commit is complete when that commit's wait returns, so a
// buffer read by step 8 is free after the next tile's step 2. Warp 0 computes
// every MMA's descriptors and one elected lane issues them; the weight-
// gradient MMAs of steps 5-7 commit to their own barrier, which the epilogue
// waits for only before it overwrites the tile they read.
// The staged inputs of the next tile arrive by bulk copies into one staging
// buffer: U and V rows (read in step 7 of the current tile) are issued in
// step 2, the rest (x, dL/dx-hat, z, gamma; read in step 4) in step 5.
struct Bwd128Stage {
  static constexpr uint32_t U_PITCH = 528;  // 512 B + 16: the 16 vertex rows hit distinct banks
  static constexpr uint32_t U = 0;          // [16 vertices][128]
  static constexpr uint32_t V = 16 * U_PITCH;  // [8 frames][128]
  static constexpr uint32_t X = V + 8 * 512;   // [16] float4
  static constexpr uint32_t G = X + 256;       // [8][16] float4
  static constexpr uint32_t Z = G + 2048;      // [16][Z] (Z <= 8)
  static constexpr uint32_t GAM = Z + 512;     // [8][2M] (2M <= 16)
  static constexpr uint32_t BYTES = GAM + 512;
};
struct Bwd128Smem {
  static constexpr uint32_t W2 = 0, W3 = W2 + ACT;
  static constexpr uint32_t XB = W3 + ACT;           // X[0..2]
  static constexpr uint32_t GO = XB + 3 * ACT;       // [128][64], columns >= 16 zero
  static constexpr uint32_t Y = GO + TC_TILE;        // [128][64], columns >= 16 zero but 15
  static constexpr uint32_t WO = Y + TC_TILE;        // [16][128] K-major, 2 KB blocks
  static constexpr uint32_t W1Z = WO + 4096;         // [16][128]: W1[:, :Z]^T, rows >= Z zero
  static constexpr uint32_t STG = W1Z + 4096;
  static constexpr uint32_t BIAS = STG + Bwd128Stage::BYTES;   // b2, b3, bo
  static constexpr uint32_t DZP = BIAS + (128 + 128 + 16) * 4;  // [8 qz][4 q4][16 vertices]
  static constexpr uint32_t DBO = DZP + 8 * 64 * 4;
  // mbarriers: chain MMAs, final drain, dL/dz MMA, staged U/V, staged rest,
  // weight-gradient MMAs
  static constexpr uint32_t BAR = DBO + 8 * 4;
  static constexpr uint32_t TMEMP = BAR + 6 * 8;
  static constexpr uint32_t TOTAL = TMEMP + 8;
};
static_assert(Bwd128Smem::TOTAL + 1024 <= 227 * 1024, "backward H = 128 shared memory");
constexpr uint32_t C_WORK = 0, C_ACC3 = 128, C_ACC2 = 256, C_ACCB = 384, C_ACCO = 432,
                   C_DZ = 448;
constexpr int BWD128_THREADS = 512;

// The two staged groups of one tile: U and V rows (part 0, 17 pieces) or x,
// dL/dx-hat, z and gamma (part 1, 11 pieces). One thread announces a group's
// bytes on its barrier before a CTA barrier; after it warps 1..15 issue the
// pieces, at most two lanes each (one warp issuing a whole group became the
// next barrier's straggler). Rows past N or T are not copied: the readers
// replace their stale values by zero. The z and gamma copies round up to 16 B
// (those arrays carry 16 B of padding).
constexpr int STAGE_PIECES = 17, STAGE_WARPS128 = 15;

__device__ __forceinline__ uint32_t bwd128_piece_bytes(const TcArgs& a, int i0, int t0,
                                                       int part, int k) {
  const int nv = min(16, a.N - i0), nf = min(8, a.T - t0);
  if (part == 0) {
    if (k < 16) return k < nv ? 512u : 0u;
    return k == 16 ? (uint32_t)nf * 512u : 0u;
  }
  if (k < 8) return k < nf ? (uint32_t)nv * 16u : 0u;
  if (k == 8) return (uint32_t)nv * 16u;
  if (k == 9) return ((uint32_t)(nv * a.Z * 4) + 15u) & ~15u;
  return k == 10 ? ((uint32_t)(nf * 2 * a.M * 4) + 15u) & ~15u : 0u;
}

__device__ void bwd128_stage_expect(const TcArgs& a, int i0, int t0, uint64_t* sbar, int part) {
  uint32_t total = 0u;
  for (int k = 0; k < STAGE_PIECES; ++k) total += bwd128_piece_bytes(a, i0, t0, part, k);
  tc::mbar_arrive_expect_tx(sbar, total);
}

__device__ void bwd128_stage_issue(const TcArgs& a, int i0, int t0, uint8_t* stg,
                                   uint64_t* sbar, int part, int warp, int lane) {
  if (warp < 1) return;
  const int k = lane * STAGE_WARPS128 + (warp - 1);
  if (k >= STAGE_PIECES) return;
  const uint32_t n = bwd128_piece_bytes(a, i0, t0, part, k);
  if (n == 0u) return;
  if (part == 0) {
    if (k < 16)
      tc::bulk_g2s(stg + Bwd128Stage::U + k * Bwd128Stage::U_PITCH,
                   a.U + (long long)(i0 + k) * H2X, n, sbar);
    else
      tc::bulk_g2s(stg + Bwd128Stage::V, a.V + (long long)t0 * H2X, n, sbar);
  } else {
    if (k < 8)
      tc::bulk_g2s(stg + Bwd128Stage::G + k * 256, a.dxhat + (long long)(t0 + k) * a.N + i0, n,
                   sbar);
    else if (k == 8)
      tc::bulk_g2s(stg + Bwd128Stage::X, a.xr + i0, n, sbar);
    else if (k == 9)
      tc::bulk_g2s(stg + Bwd128Stage::Z, a.z + (long long)i0 * a.Z, n, sbar);
    else
      tc::bulk_g2s(stg + Bwd128Stage::GAM, a.gamma + (long long)t0 * 2 * a.M, n, sbar);
  }
}

// TSUM: also the per-frame sums of dpre1 into a.dV (learned time embedding).
template <int ROT, bool TSUM>
__global__ void __launch_bounds__(BWD128_THREADS, 1) mlp_bwd_tc128_kernel(TcArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = tc::align1024(smem_raw);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + Bwd128Smem::BAR);
  uint32_t* tmem_ptr = reinterpret_cast<uint32_t*>(sm + Bwd128Smem::TMEMP);
  float* bias = reinterpret_cast<float*>(sm + Bwd128Smem::BIAS);
  float* dzp = reinterpret_cast<float*>(sm + Bwd128Smem::DZP);
  float* dbo = reinterpret_cast<float*>(sm + Bwd128Smem::DBO);
  uint64_t* sbar = bar + 3;  // [0] U/V, [1] the rest
  uint8_t* stg = sm + Bwd128Smem::STG;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int q4 = warp & 3, c = warp >> 2;  // lane quarter, column quarter
  const int row = 32 * q4 + lane, il = row & 15, tl = row >> 4;
  const int H = H2X, K = a.K, Z = a.Z, NO = a.NO;
  const int c0 = 32 * c;
  if (tid < 8) dbo[tid] = 0.f;

  const float* p2 = a.mlp + H * K + H;
  const float* p3 = p2 + H * H + H;
  const float* po = p3 + H * H + H;
  load_weight128(sm + Bwd128Smem::W2, TC_TILE, p2, 128, 128, H, BWD128_THREADS);
  load_weight128(sm + Bwd128Smem::W3, TC_TILE, p3, 128, 128, H, BWD128_THREADS);
  load_weight128(sm + Bwd128Smem::WO, 2048, po, 16, NO, H, BWD128_THREADS);
  // W1Z row qz = column qz of W1 (H x K): W1[m][qz]
  for (int e = tid; e < 16 * 128; e += BWD128_THREADS) {
    const int qz = e >> 7, m = e & 127;
    st_bf16(sm + Bwd128Smem::W1Z + (m >> 6) * 2048, qz, m & 63,
            qz < Z ? a.mlp[(long long)m * K + qz] : 0.f);
  }
  {  // GO and Y start zero; their columns >= 16 stay zero, Y column 15 stays 1
    const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
    for (int e = tid; e < 2 * TC_TILE / 16; e += BWD128_THREADS)
      *reinterpret_cast<uint4*>(sm + Bwd128Smem::GO + (uint32_t)e * 16u) = zero;
  }
  for (int k = tid; k < 128; k += BWD128_THREADS) {
    bias[k] = p2[H * H + k];
    bias[128 + k] = p3[H * H + k];
  }
  if (tid < 16) bias[256 + tid] = tid < NO ? po[NO * H + tid] : 0.f;
  if (tid == 0) {
    for (int b = 0; b < 6; ++b) tc::mbar_init(bar + b, 1);
    tc::fence_mbar_init();
  }
  const int n_tb0 = (a.T + 7) / 8;
  if (tid == 0 && (int)blockIdx.x < ((a.N + 15) / 16) * n_tb0) {  // the first tile's groups
    const int fi0 = (int)blockIdx.x / n_tb0 * 16, ft0 = ((int)blockIdx.x - fi0 / 16 * n_tb0) * 8;
    bwd128_stage_expect(a, fi0, ft0, bar + 3, 0);
    bwd128_stage_expect(a, fi0, ft0, bar + 4, 1);
  }
  if (warp == 0) {
    tc::tmem_alloc(tmem_ptr, 512);
    tc::tmem_relinquish();
  }
  const int n_tb = (a.T + 7) / 8;
  const int ntiles = ((a.N + 15) / 16) * n_tb;
  int tile = blockIdx.x;
  int i0 = 0, t0 = 0;
  if (tile < ntiles) {
    i0 = tile / n_tb * 16;
    t0 = (tile - i0 / 16 * n_tb) * 8;
  }
  __syncthreads();  // zeroed Y before its column 15 is set; barriers initialised
  if (c == 1) st_bf16(sm + Bwd128Smem::Y, row, 15, 1.f);
  bool ok = tc_sync_ok(true, a.err);
  uint32_t sphase = 0u, pending = 0u;
  // a group's bytes are announced (thread 0) before the CTA barrier that
  // precedes its issue; after it warps 1-15 issue the group's pieces, at most
  // two each
  auto stage_expect = [&](int part, int i0_, int t0_) {
    if (tid == 0) bwd128_stage_expect(a, i0_, t0_, sbar + part, part);
  };
  auto stage_issue = [&](int part, int i0_, int t0_) {
    bwd128_stage_issue(a, i0_, t0_, stg, sbar + part, part, warp, lane);
    pending |= 1u << part;
  };
  auto stage_wait = [&](int part) {
    ok = ok && tc::mbar_wait(sbar + part, (sphase >> part) & 1u, WAIT_TRIES);
    sphase ^= 1u << part;
    pending &= ~(1u << part);
  };
  if (tile < ntiles) {
    stage_issue(0, i0, t0);
    stage_issue(1, i0, t0);
  }
  const uint32_t tmem = *tmem_ptr;
  const uint32_t lane_addr = tmem + ((uint32_t)(q4 * 32) << 16);
  auto sa = [&](uint32_t off) { return tc::smem_u32(sm + off); };
  constexpr uint32_t ID128 = tc::idesc_bf16(128, 128, false, false);
  constexpr uint32_t ID16 = tc::idesc_bf16(128, 16, false, false);
  constexpr uint32_t IDW = tc::idesc_bf16(128, 128, false, true);   // A K-major, B MN-major
  constexpr uint32_t IDR = tc::idesc_bf16(128, 128, true, true);    // A^T B over rows
  constexpr uint32_t IDR16 = tc::idesc_bf16(128, 16, true, true);
  // bar + 5: the weight-gradient MMAs of a step, committed after its chain
  // MMA: the epilogue loads and scales its values meanwhile and waits for
  // them only before it overwrites the tile they read.
  // Phase parities from the tile count lt: per tile the chain barrier
  // completes 6 phases (steps 2-7: parities 0, 1, 0, 1, 0, 1), the weight
  // barrier 3 (steps 5-7: lt, lt + 1, lt), the dL/dz barrier 1 (lt).
  int lt = 0;  // tiles done (0: the weight gradients' first MMAs overwrite)
  const float* b2 = bias + c0;
  const float* b3 = bias + 128 + c0;
  auto xbuf = [&](int k) { return Bwd128Smem::XB + (uint32_t)k * ACT; };
  // descriptors of the fixed operands (the weights, dL/do and y tiles)
  const uint64_t d_w2k = kdesc(sa(Bwd128Smem::W2)), d_w3k = kdesc(sa(Bwd128Smem::W3));
  const uint64_t d_w2m = mdesc2(sa(Bwd128Smem::W2)), d_w3m = mdesc2(sa(Bwd128Smem::W3));
  const uint64_t d_wok = kdesc(sa(Bwd128Smem::WO)), d_wom = mdesc2(sa(Bwd128Smem::WO), 2048);
  const uint64_t d_gok = kdesc(sa(Bwd128Smem::GO)), d_gom = mdesc2(sa(Bwd128Smem::GO));
  const uint64_t d_ym = mdesc2(sa(Bwd128Smem::Y)), d_w1z = kdesc(sa(Bwd128Smem::W1Z));

  // h1 of the tile staged in `stg` into X[k]: act' mask of this thread's columns
  auto put_h1 = [&](int k, bool valid) {
    const float4* u4 = reinterpret_cast<const float4*>(stg + Bwd128Stage::U +
                                                       il * Bwd128Stage::U_PITCH + 4 * c0);
    const float4* v4 = reinterpret_cast<const float4*>(stg + Bwd128Stage::V + tl * 512 + 4 * c0);
    float v[32];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const float4 u = u4[q], w = v4[q];
      v[4 * q + 0] = valid ? leaky(u.x + w.x, a.slope) : 0.f;
      v[4 * q + 1] = valid ? leaky(u.y + w.y, a.slope) : 0.f;
      v[4 * q + 2] = valid ? leaky(u.z + w.z, a.slope) : 0.f;
      v[4 * q + 3] = valid ? leaky(u.w + w.w, a.slope) : 0.f;
    }
    uint32_t m = 0u;
#pragma unroll
    for (int q = 0; q < 32; ++q) m |= (v[q] > 0.f ? 1u : 0u) << q;
    st_row32(sm + xbuf(k), row, c0, v);
    return m;
  };
  auto row_valid = [&](int i0_, int t0_) { return i0_ + il < a.N && t0_ + tl < a.T; };

  int xa = 0, xb = 1, xc = 2;
  uint32_t m1 = 0u;
  int dz_i0 = -1;
  float dbo_acc[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
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
    m1 = put_h1(xa, row_valid(i0, t0));
  }
  for (; tile < ntiles; tile += gridDim.x) {
    const bool valid = row_valid(i0, t0);
    const int next = tile + (int)gridDim.x;
    int ni0 = 0, nt0 = 0;
    if (next < ntiles) {
      ni0 = next / n_tb * 16;
      nt0 = (next - ni0 / 16 * n_tb) * 8;
      // the U/V group of this tile has been waited for (before its h1): the
      // next tile's is announced before step 2's barrier and issued after it
      stage_expect(0, ni0, nt0);
    }
    // ---- 2: h2
    if (!(ok = tc_sync_ok(ok, a.err))) break;
    if (warp == 0) {
      const uint64_t da = kdesc(sa(xbuf(xa)));
      if (tc::elect_one()) {
        mma_feat(tmem + C_WORK, da, d_w2k, TC_TILE, ID128);
        tc::mma_commit(bar);
      }
      __syncwarp();
    }
    // the U/V rows of this tile were read (step 7 of the previous tile)
    if (next < ntiles) stage_issue(0, ni0, nt0);
    tc_wait_parity(bar, 0u, ok);
    uint32_t m2 = 0u, m3 = 0u;
    {
      float v[32];
      ld_col32(lane_addr + C_WORK + c0, v);
#pragma unroll
      for (int k = 0; k < 32; ++k) {
        v[k] = leaky(v[k] + b2[k], a.slope);
        m2 |= (v[k] > 0.f ? 1u : 0u) << k;
      }
      st_row32(sm + xbuf(xb), row, c0, v);
    }
    // ---- 3: h3
    if (!(ok = tc_sync_ok(ok, a.err))) break;
    if (warp == 0) {
      const uint64_t da = kdesc(sa(xbuf(xb)));
      if (tc::elect_one()) {
        mma_feat(tmem + C_WORK, da, d_w3k, TC_TILE, ID128);
        tc::mma_commit(bar);
      }
      __syncwarp();
    }
    tc_wait_parity(bar, 1u, ok);
    {
      float v[32];
      ld_col32(lane_addr + C_WORK + c0, v);
#pragma unroll
      for (int k = 0; k < 32; ++k) {
        v[k] = leaky(v[k] + b3[k], a.slope);
        m3 |= (v[k] > 0.f ? 1u : 0u) << k;
      }
      st_row32(sm + xbuf(xc), row, c0, v);
    }
    // ---- 4: o, dL/do (quarter 0), y (quarter 1), previous dL/dz (quarters 2, 3)
    if (!(ok = tc_sync_ok(ok, a.err))) break;
    if (warp == 0) {
      const uint64_t da = kdesc(sa(xbuf(xc)));
      if (tc::elect_one()) {
        mma_feat(tmem + C_WORK, da, d_wok, 2048, ID16);
        tc::mma_commit(bar);
      }
      __syncwarp();
    }
    stage_wait(1);
    if (next < ntiles) stage_expect(1, ni0, nt0);  // issued after step 5's barrier
    tc_wait_parity(bar, 0u, ok);
    if (c == 0) {
      float r[16];
      ld_col16(lane_addr + C_WORK, r);
      float o[7], go[7];
#pragma unroll
      for (int j = 0; j < 7; ++j) {
        o[j] = r[j] + bias[256 + j];
        go[j] = 0.f;
      }
      if (valid) {
        const float4 x = reinterpret_cast<const float4*>(stg + Bwd128Stage::X)[il];
        const float4 g = reinterpret_cast<const float4*>(stg + Bwd128Stage::G)[tl * 16 + il];
        transform_backward<ROT>(o, a.alpha, x, g, go);
      }
      // output-bias gradient summed in FP32 (rows cancel strongly)
#pragma unroll
      for (int j = 0; j < 7; ++j) dbo_acc[j] += go[j];
      uint4 q0;
      q0.x = tc::pack_bf16(go[0], go[1]);
      q0.y = tc::pack_bf16(go[2], go[3]);
      q0.z = tc::pack_bf16(go[4], go[5]);
      q0.w = tc::pack_bf16(NO > 6 ? go[6] : 0.f, 0.f);
      *reinterpret_cast<uint4*>(sm + Bwd128Smem::GO + tc::sw128_off(row, 0)) = q0;
    } else if (c == 1) {
      // y = (z_i, gamma_t, 0.., 1): both sources read at fixed offsets from
      // per-thread bases (zs[k], and gamma through gz = gt - Z), unconditionally
      // and then selected, every read inside the staging area (Z <= 8 floats
      // per vertex, K - Z <= 12 per frame, 128 floats each)
      const float* zs = reinterpret_cast<const float*>(stg + Bwd128Stage::Z) + il * Z;
      const float* gz = reinterpret_cast<const float*>(stg + Bwd128Stage::GAM) + tl * (K - Z) - Z;
      float y[16];
#pragma unroll
      for (int k = 0; k < 15; ++k) {
        const float zk = k < 8 ? zs[k] : 0.f;
        const float gk = k >= 1 ? gz[k] : 0.f;
        y[k] = !valid ? 0.f : k < Z ? zk : k < K ? gk : 0.f;
      }
      y[15] = 1.f;
      st_bf16x8(sm + Bwd128Smem::Y, row, 0, y);
      st_bf16x8(sm + Bwd128Smem::Y, row, 8, y + 8);
    } else if (dz_i0 >= 0) {
      flush_dz(tid - 256, 256);
    }
    // ---- 5: dh3 = gO Wo, ACC_O += h3^T gO
    if (!(ok = tc_sync_ok(ok, a.err))) break;
    if (warp == 0) {
      const uint64_t dc = mdesc2(sa(xbuf(xc)));
      if (tc::elect_one()) {
        tc::mma_bf16(tmem + C_WORK, d_gok, d_wom, IDW, 0u);
        tc::mma_commit(bar);
        mma_rows128(tmem + C_ACCO, dc, d_gom, IDR16, lt == 0);
        tc::mma_commit(bar + 5);
      }
      __syncwarp();
    }
    // x, dL/dx-hat, z and gamma of this tile were read in step 4
    if (next < ntiles) stage_issue(1, ni0, nt0);
    tc_wait_parity(bar, 1u, ok);
    {
      float v[32];
      ld_col32(lane_addr + C_WORK + c0, v);
#pragma unroll
      for (int k = 0; k < 32; ++k) v[k] *= ((m3 >> k) & 1u) ? 1.f : a.slope;
      tc_wait_parity(bar + 5, (uint32_t)(lt & 1), ok);         // ACC_O has read h3
      st_row32(sm + xbuf(xc), row, c0, v);  // dpre3
    }
    // ---- 6: dh2 = dpre3 W3, ACC_3 += dpre3^T h2, ACC_B3 += dpre3^T y
    if (!(ok = tc_sync_ok(ok, a.err))) break;
    if (warp == 0) {
      const uint64_t dck = kdesc(sa(xbuf(xc))), dc = mdesc2(sa(xbuf(xc)));
      const uint64_t db = mdesc2(sa(xbuf(xb)));
      if (tc::elect_one()) {
        mma_wT(tmem + C_WORK, dck, d_w3m, IDW);
        tc::mma_commit(bar);
        mma_rows128(tmem + C_ACC3, dc, db, IDR, lt == 0);
        mma_rows128(tmem + C_ACCB, dc, d_ym, IDR16, lt == 0);
        tc::mma_commit(bar + 5);
      }
      __syncwarp();
    }
    tc_wait_parity(bar, 0u, ok);
    {
      float v[32];
      ld_col32(lane_addr + C_WORK + c0, v);
#pragma unroll
      for (int k = 0; k < 32; ++k) v[k] *= ((m2 >> k) & 1u) ? 1.f : a.slope;
      tc_wait_parity(bar + 5, (uint32_t)((lt + 1) & 1), ok);         // ACC_3 has read h2
      st_row32(sm + xbuf(xb), row, c0, v);  // dpre2
    }
    // ---- 7: dh1 = dpre2 W2, ACC_2 += dpre2^T h1, ACC_B2 += dpre2^T y
    if (!(ok = tc_sync_ok(ok, a.err))) break;
    if (warp == 0) {
      const uint64_t dbk = kdesc(sa(xbuf(xb))), db = mdesc2(sa(xbuf(xb)));
      const uint64_t da = mdesc2(sa(xbuf(xa)));
      if (tc::elect_one()) {
        mma_wT(tmem + C_WORK, dbk, d_w2m, IDW);
        tc::mma_commit(bar);
        mma_rows128(tmem + C_ACC2, db, da, IDR, lt == 0);
        mma_rows128(tmem + C_ACCB + 16, db, d_ym, IDR16, lt == 0);
        tc::mma_commit(bar + 5);
      }
      __syncwarp();
    }
    tc_wait_parity(bar, 1u, ok);
    {
      float v[32];
      ld_col32(lane_addr + C_WORK + c0, v);
#pragma unroll
      for (int k = 0; k < 32; ++k) v[k] *= ((m1 >> k) & 1u) ? 1.f : a.slope;
      if (TSUM) frame_sums<32>(v, a.dV, t0, tl, a.T, H, c0);
      tc_wait_parity(bar + 5, (uint32_t)(lt & 1), ok);         // ACC_2 has read h1 (and dpre2)
      st_row32(sm + xbuf(xa), row, c0, v);  // dpre1
    }
    // the next tile's h1 into X[b] (dpre2 is used up)
    if (next < ntiles) {
      stage_wait(0);
      m1 = put_h1(xb, row_valid(ni0, nt0));
    }
    // ---- 8: dL/dz rows = dpre1 W1[:, :Z]; ACC_B1 += dpre1^T y
    if (!(ok = tc_sync_ok(ok, a.err))) break;
    // ACC_B1 is not waited for here: the next tile's first commit covers it
    if (warp == 0) {
      const uint64_t dak = kdesc(sa(xbuf(xa))), da = mdesc2(sa(xbuf(xa)));
      if (tc::elect_one()) {
        mma_feat(tmem + C_DZ, dak, d_w1z, 2048, ID16);
        tc::mma_commit(bar + 2);
        mma_rows128(tmem + C_ACCB + 32, da, d_ym, IDR16, lt == 0);
      }
      __syncwarp();
    }
    dz_i0 = i0;
    if (c == 1) {
      tc_wait_parity(bar + 2, (uint32_t)(lt & 1), ok);
      float r[16];
      ld_col16(lane_addr + C_DZ, r);
#pragma unroll
      for (int qz = 0; qz < 8; ++qz) {
        if (qz < Z) {
          const float s = r[qz] + __shfl_xor_sync(0xffffffffu, r[qz], 16);
          if (lane < 16) dzp[(qz * 4 + q4) * 16 + lane] = s;
        }
      }
    }
    ++lt;
    const int t_ = xa;
    xa = xb;
    xb = xc;
    xc = t_;
    i0 = ni0;
    t0 = nt0;
  }
  if (lt > 0) {  // drain: every MMA issued (by warp 0's elected lane) has completed
    if (warp == 0) {
      if (tc::elect_one()) tc::mma_commit(bar);
      __syncwarp();
    }
    tc_wait_parity(bar, 0u, ok);
  }
  ok = tc_sync_ok(ok, a.err);
  if (ok && dz_i0 >= 0) flush_dz(tid, BWD128_THREADS);
  if (c == 0) {
#pragma unroll
    for (int j = 0; j < 7; ++j) {
      float sj = dbo_acc[j];
#pragma unroll
      for (int o2 = 16; o2 > 0; o2 >>= 1) sj += __shfl_xor_sync(0xffffffffu, sj, o2);
      if (lane == 0 && j < NO) atomicAdd(dbo + j, sj);
    }
  }
  ok = tc_sync_ok(ok, a.err);
  if (ok && lt > 0) {
    // accumulators (TMEM lane = output feature j or m) -> the gradient, once per CTA
    float* g = a.g_mlp;
    float* gW1 = g;
    float* gb1 = g + H * K;
    float* gW2 = gb1 + H;
    float* gb2 = gW2 + H * H;
    float* gW3 = gb2 + H;
    float* gb3 = gW3 + H * H;
    float* gWo = gb3 + H;
    float* gbo = gWo + NO * H;
    const int j = row;
    float v[32];
    ld_col32(lane_addr + C_ACC3 + c0, v);
#pragma unroll
    for (int k = 0; k < 32; ++k) atomicAdd(gW3 + j * H + c0 + k, v[k]);
    ld_col32(lane_addr + C_ACC2 + c0, v);
#pragma unroll
    for (int k = 0; k < 32; ++k) atomicAdd(gW2 + j * H + c0 + k, v[k]);
    if (c == 0) {
      ld_col16(lane_addr + C_ACCB, v);
      atomicAdd(gb3 + j, v[15]);
      ld_col16(lane_addr + C_ACCB + 16, v);
      atomicAdd(gb2 + j, v[15]);
    } else if (c == 1) {
      ld_col16(lane_addr + C_ACCB + 32, v);
#pragma unroll
      for (int k = 0; k < 15; ++k)
        if (k < K) atomicAdd(gW1 + j * K + k, v[k]);
      atomicAdd(gb1 + j, v[15]);
    } else if (c == 2) {
      ld_col16(lane_addr + C_ACCO, v);  // row m of dWo^T
#pragma unroll
      for (int q = 0; q < 7; ++q)
        if (q < NO) atomicAdd(gWo + q * H + j, v[q]);
    } else if (tid - 384 < NO) {
      atomicAdd(gbo + (tid - 384), dbo[tid - 384]);
    }
  }
  for (int b = 0; b < 2; ++b)
    if (pending & (1u << b)) tc::mbar_wait(sbar + b, (sphase >> b) & 1u, WAIT_TRIES);
  if (warp == 0) {
    if (tc::elect_one()) {
      tc::mma_commit(bar + 1);
      tc::mbar_wait(bar + 1, 0, WAIT_TRIES);
    }
    __syncwarp();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

cudaError_t launch_mlp_backward_bf16_h128(npg_ctx* c) {
  const size_t smem = Bwd128Smem::TOTAL + 1024;
  const bool ts = c->dV != nullptr;
  auto k = c->cfg.rot_mode == NPG_ROT_QUAT
               ? (ts ? mlp_bwd_tc128_kernel<0, true> : mlp_bwd_tc128_kernel<0, false>)
           : c->cfg.rot_mode == NPG_ROT_EXPMAP
               ? (ts ? mlp_bwd_tc128_kernel<1, true> : mlp_bwd_tc128_kernel<1, false>)
               : (ts ? mlp_bwd_tc128_kernel<2, true> : mlp_bwd_tc128_kernel<2, false>);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long tiles = (long long)((c->N + 15) / 16) * ((c->T + 7) / 8);
  if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;  // tile indices are ints
  k<<<tc_grid(c, tiles, 1), BWD128_THREADS, smem, c->stream>>>(make_tc_args(c));
  return cudaGetLastError();
}

}  // namespace npg
