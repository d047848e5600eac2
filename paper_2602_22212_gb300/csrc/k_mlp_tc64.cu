// BF16 tensor-core MLP backward (reverse of Sec. 3.3-3.4) for hidden width 64
// and 3 hidden layers, sized so that two CTAs share an SM: while one waits on
// its MMAs or its barriers the other runs its epilogues, which is what the
// chain of dependent MMA -> TMEM -> CUDA-core steps of one tile cannot do by
// itself. Each CTA takes 112 KB of shared memory and 256 TMEM columns.
//
// Tile = 16 vertices x 8 frames = 128 rows (row r = tl 16 + il); 256 threads:
// warp w serves TMEM lanes 32 (w % 4) .. + 31 (its rows) and the 32-column
// half c = w / 4 of every 64-wide activation. Four [128][64] activation
// tiles P, Q, R, S hold, per tile: h1 (P), h2 (Q), h3 (R), then dpre3 (S),
// dpre2 (R), dpre1 (Q) and the next tile's h1 (S); the next tile's roles are
// (P, Q, R, S) <- (S, P, Q, R). No epilogue writes a tile that a weight-
// gradient MMA still reads, so those MMAs are not waited for in their own
// step: each is covered by the next step's commit. A fifth tile YG holds
// y = (z_i, gamma_t, 0.., 1) in columns 0..15 and dL/do in columns 16..22.
// The weight gradients accumulate in TMEM over all of a CTA's tiles:
//   ACC_3 = [h2 | y]^T dpre3   M = 128: lanes 0..63 dW3^T, lane 79 db3
//   ACC_2 = [h1 | y]^T dpre2   likewise ([h | y] is one MN-major operand
//                              whose second 64-row block is YG: the
//                              descriptor's leading-byte offset is YG - h)
//   ACC_O = [h3 | y]^T dL/do   M = 128 (lanes 0..63; y's block only pads
//   ACC_1 = [dpre1 | y]^T y    M up to the faster 128): dWo^T; dW1 in
//                              columns 0..K-1, db1 in column 15
// Warp 0 computes every MMA's descriptors and one elected lane issues them.
#include "mlp_tc_common.cuh"

namespace npg {

namespace {
constexpr int H64 = 64;

struct Bwd64Stage {  // inputs of one tile, FP32
  static constexpr uint32_t U_PITCH = 272;  // 256 B + 16: the 16 vertex rows hit distinct banks
  static constexpr uint32_t U = 0;          // [16 vertices][64]
  static constexpr uint32_t V = 16 * U_PITCH;   // [8 frames][64]
  static constexpr uint32_t X = V + 8 * 256;    // [16] float4
  static constexpr uint32_t G = X + 256;        // [8][16] float4
  static constexpr uint32_t Z = G + 2048;       // [16][Z] (Z <= 8)
  static constexpr uint32_t GAM = Z + 512;      // [8][2M] (2M <= 16)
  static constexpr uint32_t BYTES = GAM + 512;
};
struct Bwd64Smem {
  static constexpr uint32_t W2 = 0, W3 = W2 + TC_TILE / 2;  // [64][64] K-major, 8 KB each
  static constexpr uint32_t XB = W3 + TC_TILE / 2;          // four activation tiles, 16 KB each
  static constexpr uint32_t YG = XB + 4 * TC_TILE;          // y | dL/do (after every X tile)
  static constexpr uint32_t WO = YG + TC_TILE;              // [16][64] K-major
  static constexpr uint32_t W1Z = WO + 2048;                // [16][64]: W1[:, :Z]^T
  static constexpr uint32_t STG = W1Z + 2048;
  static constexpr uint32_t DZP = STG + Bwd64Stage::BYTES;  // [8 qz][4 q4][16 vertices]
  static constexpr uint32_t DBO = DZP + 8 * 64 * 4;
  static constexpr uint32_t BAR = DBO + 8 * 4;  // chain, drain, dL/dz, staged U/V, staged rest
  static constexpr uint32_t TMEMP = BAR + 5 * 8;
  static constexpr uint32_t TOTAL = TMEMP + 8;
};
static_assert(2 * (Bwd64Smem::TOTAL + 1024) <= 226 * 1024, "two CTAs per SM");
constexpr uint32_t C_WORK = 0, C_ACC3 = 64, C_ACC2 = 128, C_ACCO = 192, C_ACC1 = 208;
constexpr int BWD64_THREADS = 256;

__device__ void load_weight64(uint8_t* tile, const float* W, int rows, int valid_rows) {
  for (int e = threadIdx.x; e < rows * 64; e += BWD64_THREADS) {
    const int r = e >> 6, k = e & 63;
    st_bf16(tile, r, k, r < valid_rows ? W[r * 64 + k] : 0.f);
  }
}

// The MMA helpers take descriptors that warp 0 computed as a whole (one
// elected lane issues). A K step of 16 advances a K-major descriptor's start
// address by 32 B (2 in its 16-byte units) and an MN-major one by 2048 B
// (128); the start field cannot carry out of its 14 bits below 256 KB.

// M 128 x N (= idesc) over K = 64 features: K-major A and B ([rows][64]).
__device__ __forceinline__ void mma_f64(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc) {
#pragma unroll
  for (int ks = 0; ks < 4; ++ks) tc::mma_bf16(d, a + 2 * ks, b + 2 * ks, idesc, ks > 0);
}

// M 128 x N 64 = A W over K = 64 (the weight's output rows): A K-major, w the
// MN-major descriptor of a K-major [64 out][64 in] weight tile.
__device__ __forceinline__ void mma_w64T(uint32_t d, uint64_t a, uint64_t w, uint32_t idesc) {
#pragma unroll
  for (int ks = 0; ks < 4; ++ks) tc::mma_bf16(d, a + 2 * ks, w + 128 * ks, idesc, ks > 0);
}

// M x N (+)= A^T B over K = the 128 rows of a tile, A and B MN-major
// descriptors (a second 64-wide block at their leading-byte offsets).
__device__ __forceinline__ void mma_rows(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                         bool first) {
#pragma unroll
  for (int ks = 0; ks < 8; ++ks)
    tc::mma_bf16(d, a + 128 * ks, b + 128 * ks, idesc, (first && ks == 0) ? 0u : 1u);
}

__device__ __forceinline__ uint64_t kdesc(uint32_t saddr) { return tc::kmajor_sw128(saddr); }
__device__ __forceinline__ uint64_t mdesc(uint32_t saddr, uint32_t lbo = 0) {
  return tc::mnmajor_sw128(saddr, lbo, 1024);
}

// The two staged groups of a tile (part 0: the U rows and V, 17 pieces;
// part 1: dL/dx-hat rows, x, z, gamma, 11 pieces). One thread announces a
// group's bytes on its barrier before a CTA barrier (bwd64_stage_expect);
// after that barrier warps 1..7 issue the pieces, at most three lanes each
// (bwd64_stage_issue): a bulk copy costs its issuing lane tens of cycles, and
// a group issued by one warp made that warp the straggler of the next barrier.
constexpr int STAGE_PIECES = 17, STAGE_WARPS = 7;

__device__ __forceinline__ uint32_t bwd64_piece_bytes(const TcArgs& a, int i0, int t0, int part,
                                                      int k) {
  const int nv = min(16, a.N - i0), nf = min(8, a.T - t0);
  if (part == 0) {
    if (k < 16) return k < nv ? 256u : 0u;
    return k == 16 ? (uint32_t)nf * 256u : 0u;
  }
  if (k < 8) return k < nf ? (uint32_t)nv * 16u : 0u;
  if (k == 8) return (uint32_t)nv * 16u;
  if (k == 9) return ((uint32_t)(nv * a.Z * 4) + 15u) & ~15u;
  return k == 10 ? ((uint32_t)(nf * 2 * a.M * 4) + 15u) & ~15u : 0u;
}

__device__ void bwd64_stage_expect(const TcArgs& a, int i0, int t0, uint64_t* sbar, int part) {
  uint32_t total = 0u;
  for (int k = 0; k < STAGE_PIECES; ++k) total += bwd64_piece_bytes(a, i0, t0, part, k);
  tc::mbar_arrive_expect_tx(sbar, total);
}

__device__ void bwd64_stage_issue(const TcArgs& a, int i0, int t0, uint8_t* stg, uint64_t* sbar,
                                  int part, int warp, int lane) {
  if (warp < 1) return;
  const int k = lane * STAGE_WARPS + (warp - 1);
  if (k >= STAGE_PIECES) return;
  const uint32_t n = bwd64_piece_bytes(a, i0, t0, part, k);
  if (n == 0u) return;
  if (part == 0) {
    if (k < 16)
      tc::bulk_g2s(stg + Bwd64Stage::U + k * Bwd64Stage::U_PITCH, a.U + (long long)(i0 + k) * H64,
                   n, sbar);
    else
      tc::bulk_g2s(stg + Bwd64Stage::V, a.V + (long long)t0 * H64, n, sbar);
  } else {
    if (k < 8)
      tc::bulk_g2s(stg + Bwd64Stage::G + k * 256, a.dxhat + (long long)(t0 + k) * a.N + i0, n,
                   sbar);
    else if (k == 8)
      tc::bulk_g2s(stg + Bwd64Stage::X, a.xr + i0, n, sbar);
    else if (k == 9)
      tc::bulk_g2s(stg + Bwd64Stage::Z, a.z + (long long)i0 * a.Z, n, sbar);
    else
      tc::bulk_g2s(stg + Bwd64Stage::GAM, a.gamma + (long long)t0 * 2 * a.M, n, sbar);
  }
}
}  // namespace

// TSUM: also the per-frame sums of dpre1 into a.dV (learned time embedding).
template <int ROT, bool TSUM>
__global__ void __launch_bounds__(BWD64_THREADS, 2) mlp_bwd_tc2_kernel(TcArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = tc::align1024(smem_raw);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + Bwd64Smem::BAR);
  uint32_t* tmem_ptr = reinterpret_cast<uint32_t*>(sm + Bwd64Smem::TMEMP);
  float* dzp = reinterpret_cast<float*>(sm + Bwd64Smem::DZP);
  float* dbo = reinterpret_cast<float*>(sm + Bwd64Smem::DBO);
  uint64_t* sbar = bar + 3;
  uint8_t* stg = sm + Bwd64Smem::STG;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int q4 = warp & 3, c = warp >> 2;
  const int row = 32 * q4 + lane, il = row & 15, tl = row >> 4;
  const int H = H64, K = a.K, Z = a.Z, NO = a.NO;
  const int c0 = 32 * c;
  if (tid < 8) dbo[tid] = 0.f;

  const float* p2 = a.mlp + H * K + H;
  const float* p3 = p2 + H * H + H;
  const float* po = p3 + H * H + H;
  load_weight64(sm + Bwd64Smem::W2, p2, 64, 64);
  load_weight64(sm + Bwd64Smem::W3, p3, 64, 64);
  load_weight64(sm + Bwd64Smem::WO, po, 16, NO);
  for (int e = tid; e < 16 * 64; e += BWD64_THREADS) {
    const int qz = e >> 6, m = e & 63;
    st_bf16(sm + Bwd64Smem::W1Z, qz, m, qz < Z ? a.mlp[m * K + qz] : 0.f);
  }
  {  // YG starts zero; its columns >= 23 stay zero, column 15 stays 1
    const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
    for (int e = tid; e < TC_TILE / 16; e += BWD64_THREADS)
      *reinterpret_cast<uint4*>(sm + Bwd64Smem::YG + (uint32_t)e * 16u) = zero;
  }
  if (tid == 0) {
    for (int b = 0; b < 5; ++b) tc::mbar_init(bar + b, 1);
    tc::fence_mbar_init();
  }
  const int n_tb0 = (a.T + 7) / 8;
  if (tid == 0 && (int)blockIdx.x < ((a.N + 15) / 16) * n_tb0) {  // the first tile's groups
    const int fi0 = (int)blockIdx.x / n_tb0 * 16, ft0 = ((int)blockIdx.x - fi0 / 16 * n_tb0) * 8;
    bwd64_stage_expect(a, fi0, ft0, bar + 3, 0);
    bwd64_stage_expect(a, fi0, ft0, bar + 4, 1);
  }
  if (warp == 0) {
    tc::tmem_alloc(tmem_ptr, 256);
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
  __syncthreads();
  if (c == 1) st_bf16(sm + Bwd64Smem::YG, row, 15, 1.f);
  bool ok = tc_sync_ok(true, a.err);
  uint32_t sphase = 0u, pending = 0u;
  // a group's bytes are announced (thread 0) before the CTA barrier that
  // precedes its issue
  auto stage_expect = [&](int part, int i0_, int t0_) {
    if (tid == 0) bwd64_stage_expect(a, i0_, t0_, sbar + part, part);
  };
  auto stage_issue = [&](int part, int i0_, int t0_) {
    bwd64_stage_issue(a, i0_, t0_, stg, sbar + part, part, warp, lane);
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
  constexpr uint32_t ID64 = tc::idesc_bf16(128, 64, false, false);
  constexpr uint32_t ID16 = tc::idesc_bf16(128, 16, false, false);
  constexpr uint32_t IDW = tc::idesc_bf16(128, 64, false, true);    // A K-major, B MN-major
  constexpr uint32_t IDR128 = tc::idesc_bf16(128, 64, true, true);  // A^T B over rows
  constexpr uint32_t IDR16 = tc::idesc_bf16(128, 16, true, true);
  // phase parities from the tile count lt (below): per tile the chain barrier
  // completes 6 phases (steps 2-7: parities 0, 1, 0, 1, 0, 1), the dL/dz
  // barrier one (lt)
  // biases from global memory (read-only, L1-resident)
  const float* b2 = p2 + H * H + c0;
  const float* b3 = p3 + H * H + c0;
  auto xbuf = [&](int k) { return Bwd64Smem::XB + (uint32_t)k * TC_TILE; };
  const uint32_t s_yg = sa(Bwd64Smem::YG);
  const uint64_t d_w2k = kdesc(sa(Bwd64Smem::W2)), d_w3k = kdesc(sa(Bwd64Smem::W3));
  const uint64_t d_w2m = mdesc(sa(Bwd64Smem::W2)), d_w3m = mdesc(sa(Bwd64Smem::W3));
  const uint64_t d_wok = kdesc(sa(Bwd64Smem::WO)), d_wom = mdesc(sa(Bwd64Smem::WO));
  const uint64_t d_w1z = kdesc(sa(Bwd64Smem::W1Z));
  const uint64_t d_ygk32 = kdesc(s_yg + 32), d_ygm = mdesc(s_yg), d_ygm32 = mdesc(s_yg + 32);
  // [h | y]: the activation tile and YG as one MN-major operand of 128
  auto d_hy = [&](int k) { return mdesc(sa(xbuf(k)), Bwd64Smem::YG - xbuf(k)); };

  // (every epilogue below works on 16 columns at a time: fewer live registers)
  auto put_h1 = [&](int k, bool valid) {
    uint32_t m = 0u;
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
      const float4* u4 = reinterpret_cast<const float4*>(
          stg + Bwd64Stage::U + il * Bwd64Stage::U_PITCH + 4 * (c0 + 16 * hh));
      const float4* v4 =
          reinterpret_cast<const float4*>(stg + Bwd64Stage::V + tl * 256 + 4 * (c0 + 16 * hh));
      float v[16];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float4 u = u4[q], w = v4[q];
        v[4 * q + 0] = valid ? leaky(u.x + w.x, a.slope) : 0.f;
        v[4 * q + 1] = valid ? leaky(u.y + w.y, a.slope) : 0.f;
        v[4 * q + 2] = valid ? leaky(u.z + w.z, a.slope) : 0.f;
        v[4 * q + 3] = valid ? leaky(u.w + w.w, a.slope) : 0.f;
      }
#pragma unroll
      for (int q = 0; q < 16; ++q) m |= (v[q] > 0.f ? 1u : 0u) << (16 * hh + q);
      st_bf16x8(sm + xbuf(k), row, c0 + 16 * hh, v);
      st_bf16x8(sm + xbuf(k), row, c0 + 16 * hh + 8, v + 8);
    }
    return m;
  };
  // act(WORK + bias) of this thread's 32 columns into tile k; returns the mask
  auto fwd_epi = [&](const float* bias_c, int k) {
    uint32_t m = 0u;
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
      float v[16];
      ld_col16(lane_addr + C_WORK + c0 + 16 * hh, v);
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        v[q] = leaky(v[q] + __ldg(bias_c + 16 * hh + q), a.slope);
        m |= (v[q] > 0.f ? 1u : 0u) << (16 * hh + q);
      }
      st_bf16x8(sm + xbuf(k), row, c0 + 16 * hh, v);
      st_bf16x8(sm + xbuf(k), row, c0 + 16 * hh + 8, v + 8);
    }
    return m;
  };
  // WORK x act'(h) (from the mask) of this thread's 32 columns into tile k;
  // with `sums` (dpre1 of a learned time embedding) also its per-frame sums
  auto bwd_epi = [&](uint32_t msk, int k, bool sums) {
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
      float v[16];
      ld_col16(lane_addr + C_WORK + c0 + 16 * hh, v);
#pragma unroll
      for (int q = 0; q < 16; ++q) v[q] *= ((msk >> (16 * hh + q)) & 1u) ? 1.f : a.slope;
      st_bf16x8(sm + xbuf(k), row, c0 + 16 * hh, v);
      st_bf16x8(sm + xbuf(k), row, c0 + 16 * hh + 8, v + 8);
      if (sums) frame_sums<16>(v, a.dV, t0, tl, a.T, H, c0 + 16 * hh);
    }
  };
  auto row_valid = [&](int i0_, int t0_) { return i0_ + il < a.N && t0_ + tl < a.T; };

  int xp = 0, xq = 1, xr = 2, xs = 3;  // tiles P, Q, R, S
  uint32_t m1 = 0u;
  // dL/dz of a tile's 16 vertices: per-quarter partial sums over its frames
  // (step 8), added to global memory in step 4 of the next tile
  int dz_prev = -1, lt = 0;  // i0 of the previous tile; tiles done (0: the weight
                             // gradients' first MMAs overwrite their accumulators)
  float dbo_acc[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  auto flush_dz = [&](int e0, int stride) {
    for (int e = e0; e < 16 * Z; e += stride) {
      const int vi = e & 15, qz = e >> 4;
      if (dz_prev + vi >= a.N) continue;
      float s = 0.f;
#pragma unroll
      for (int q = 0; q < 4; ++q) s += dzp[(qz * 4 + q) * 16 + vi];
      atomicAdd(a.dz + (long long)(dz_prev + vi) * Z + qz, s);
    }
  };
  if (tile < ntiles) {
    stage_wait(0);
    m1 = put_h1(xp, row_valid(i0, t0));
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
    // ---- 2: h2 (P W2^T) -> Q
    if (!(ok = tc_sync_ok(ok, a.err))) break;
    if (warp == 0) {
      const uint64_t da = kdesc(sa(xbuf(xp)));
      if (tc::elect_one()) {
        mma_f64(tmem + C_WORK, da, d_w2k, ID64);
        tc::mma_commit(bar);
      }
      __syncwarp();
    }
    if (next < ntiles) stage_issue(0, ni0, nt0);
    tc_wait_parity(bar, 0u, ok);
    const uint32_t m2 = fwd_epi(b2, xq);
    // ---- 3: h3 (Q W3^T) -> R
    if (!(ok = tc_sync_ok(ok, a.err))) break;
    if (warp == 0) {
      const uint64_t da = kdesc(sa(xbuf(xq)));
      if (tc::elect_one()) {
        mma_f64(tmem + C_WORK, da, d_w3k, ID64);
        tc::mma_commit(bar);
      }
      __syncwarp();
    }
    tc_wait_parity(bar, 1u, ok);
    const uint32_t m3 = fwd_epi(b3, xr);
    // ---- 4: o; dL/do (half 0); y and the previous tile's dL/dz (half 1)
    if (!(ok = tc_sync_ok(ok, a.err))) break;
    if (warp == 0) {
      const uint64_t da = kdesc(sa(xbuf(xr)));
      if (tc::elect_one()) {
        mma_f64(tmem + C_WORK, da, d_wok, ID16);
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
      float o[7], go[8];
#pragma unroll
      for (int j = 0; j < 7; ++j) {
        o[j] = r[j] + (j < NO ? __ldg(po + NO * H + j) : 0.f);
        go[j] = 0.f;
      }
      go[7] = 0.f;
      if (valid) {
        const float4 x = reinterpret_cast<const float4*>(stg + Bwd64Stage::X)[il];
        const float4 g = reinterpret_cast<const float4*>(stg + Bwd64Stage::G)[tl * 16 + il];
        transform_backward<ROT>(o, a.alpha, x, g, go);
      }
      if (NO < 7) go[6] = 0.f;
#pragma unroll
      for (int j = 0; j < 7; ++j) dbo_acc[j] += go[j];
      st_bf16x8(sm + Bwd64Smem::YG, row, 16, go);
    } else {
      // y = (z_i, gamma_t, 0.., 1): both sources read at fixed offsets from
      // per-thread bases (zs[k], and gamma through gz = gt - Z), unconditionally
      // and then selected, every read inside the staging area (Z <= 8 floats
      // per vertex, K - Z <= 12 per frame, 128 floats each)
      const float* zs = reinterpret_cast<const float*>(stg + Bwd64Stage::Z) + il * Z;
      const float* gz = reinterpret_cast<const float*>(stg + Bwd64Stage::GAM) + tl * (K - Z) - Z;
      float y[16];
#pragma unroll
      for (int k = 0; k < 15; ++k) {
        const float zk = k < 8 ? zs[k] : 0.f;
        const float gk = k >= 1 ? gz[k] : 0.f;
        y[k] = !valid ? 0.f : k < Z ? zk : k < K ? gk : 0.f;
      }
      y[15] = 1.f;
      st_bf16x8(sm + Bwd64Smem::YG, row, 0, y);
      st_bf16x8(sm + Bwd64Smem::YG, row, 8, y + 8);
      if (dz_prev >= 0) flush_dz(tid - 128, 128);
    }
    // ---- 5: dh3 = dL/do Wo (waited); ACC_O += h3^T dL/do (covered by step 6)
    if (!(ok = tc_sync_ok(ok, a.err))) break;
    if (warp == 0) {
      const uint64_t dhy = d_hy(xr);
      if (tc::elect_one()) {
        tc::mma_bf16(tmem + C_WORK, d_ygk32, d_wom, IDW, 0u);
        tc::mma_commit(bar);
        mma_rows(tmem + C_ACCO, dhy, d_ygm32, IDR16, lt == 0);
      }
      __syncwarp();
    }
    if (next < ntiles) stage_issue(1, ni0, nt0);
    tc_wait_parity(bar, 1u, ok);
    bwd_epi(m3, xs, false);  // dpre3 -> S
    // ---- 6: dh2 = dpre3 W3; ACC_3 += [h2 | y]^T dpre3
    if (!(ok = tc_sync_ok(ok, a.err))) break;
    if (warp == 0) {
      const uint64_t dsk = kdesc(sa(xbuf(xs))), dsm = mdesc(sa(xbuf(xs))), dhy = d_hy(xq);
      if (tc::elect_one()) {
        mma_w64T(tmem + C_WORK, dsk, d_w3m, IDW);
        tc::mma_commit(bar);
        mma_rows(tmem + C_ACC3, dhy, dsm, IDR128, lt == 0);
      }
      __syncwarp();
    }
    tc_wait_parity(bar, 0u, ok);
    bwd_epi(m2, xr, false);  // dpre2 -> R (h3's last reader, ACC_O, came before)
    // ---- 7: dh1 = dpre2 W2; ACC_2 += [h1 | y]^T dpre2
    if (!(ok = tc_sync_ok(ok, a.err))) break;
    if (warp == 0) {
      const uint64_t drk = kdesc(sa(xbuf(xr))), drm = mdesc(sa(xbuf(xr))), dhy = d_hy(xp);
      if (tc::elect_one()) {
        mma_w64T(tmem + C_WORK, drk, d_w2m, IDW);
        tc::mma_commit(bar);
        mma_rows(tmem + C_ACC2, dhy, drm, IDR128, lt == 0);
      }
      __syncwarp();
    }
    tc_wait_parity(bar, 1u, ok);
    bwd_epi(m1, xq, TSUM);  // dpre1 -> Q (h2's last reader, ACC_3, came before)
    if (next < ntiles) {
      stage_wait(0);
      m1 = put_h1(xs, row_valid(ni0, nt0));  // the next h1 -> S (dpre3 is done)
    }
    // ---- 8: dL/dz rows = dpre1 W1[:, :Z] (into WORK); ACC_1 += dpre1^T y
    if (!(ok = tc_sync_ok(ok, a.err))) break;
    if (warp == 0) {
      const uint64_t dqk = kdesc(sa(xbuf(xq))), dqy = d_hy(xq);
      if (tc::elect_one()) {
        mma_f64(tmem + C_WORK, dqk, d_w1z, ID16);
        tc::mma_commit(bar + 2);
        mma_rows(tmem + C_ACC1, dqy, d_ygm, IDR16, lt == 0);
      }
      __syncwarp();
    }
    if (c == 1) {
      tc_wait_parity(bar + 2, (uint32_t)(lt & 1), ok);
      float r[16];
      ld_col16(lane_addr + C_WORK, r);
#pragma unroll
      for (int qz = 0; qz < 8; ++qz) {
        if (qz < Z) {
          const float s = r[qz] + __shfl_xor_sync(0xffffffffu, r[qz], 16);
          if (lane < 16) dzp[(qz * 4 + q4) * 16 + lane] = s;
        }
      }
    }
    dz_prev = i0;
    ++lt;
    const int t_ = xs;
    xs = xr;
    xr = xq;
    xq = xp;
    xp = t_;
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
  if (ok && dz_prev >= 0) flush_dz(tid, BWD64_THREADS);
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
    float* g = a.g_mlp;
    float* gW1 = g;
    float* gb1 = g + H * K;
    float* gW2 = gb1 + H;
    float* gb2 = gW2 + H * H;
    float* gW3 = gb2 + H;
    float* gb3 = gW3 + H * H;
    float* gWo = gb3 + H;
    float* gbo = gWo + NO * H;
    float v[32];
    // M = 128 accumulators ACC_3, ACC_2: lane m < 64 is input feature m of
    // the layer, lane 79 the bias (y's constant column); column n is output
    // feature n (this thread's half: c0 .. c0 + 31)
    // (the TMEM loads are warp-collective: every lane loads)
    ld_col32(lane_addr + C_ACC3 + c0, v);
    if (row < 64) {
#pragma unroll
      for (int k = 0; k < 32; ++k) atomicAdd(gW3 + (c0 + k) * H + row, v[k]);
    } else if (row == 79) {
#pragma unroll
      for (int k = 0; k < 32; ++k) atomicAdd(gb3 + c0 + k, v[k]);
    }
    ld_col32(lane_addr + C_ACC2 + c0, v);
    if (row < 64) {
#pragma unroll
      for (int k = 0; k < 32; ++k) atomicAdd(gW2 + (c0 + k) * H + row, v[k]);
    } else if (row == 79) {
#pragma unroll
      for (int k = 0; k < 32; ++k) atomicAdd(gb2 + c0 + k, v[k]);
    }
    // ACC_O, ACC_1 (M = 128 over [h | y]): lane m < 64 is feature m of h3 or
    // of dpre1 (the lanes of y's block are not used)
    if (c == 0) {
      ld_col16(lane_addr + C_ACCO, v);  // row m of dWo^T
      if (row < 64)
#pragma unroll
        for (int q = 0; q < 7; ++q)
          if (q < NO) atomicAdd(gWo + q * H + row, v[q]);
    } else {
      ld_col16(lane_addr + C_ACC1, v);
      if (row < 64) {
#pragma unroll
        for (int k = 0; k < 15; ++k)
          if (k < K) atomicAdd(gW1 + row * K + k, v[k]);
        atomicAdd(gb1 + row, v[15]);
      }
      if (q4 == 0 && lane < NO) atomicAdd(gbo + lane, dbo[lane]);
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
  if (warp == 0) tc::tmem_dealloc(tmem, 256);
}

cudaError_t launch_mlp_backward_bf16_h64(npg_ctx* c) {
  const size_t smem = Bwd64Smem::TOTAL + 1024;
  const bool ts = c->dV != nullptr;
  auto k = c->cfg.rot_mode == NPG_ROT_QUAT
               ? (ts ? mlp_bwd_tc2_kernel<0, true> : mlp_bwd_tc2_kernel<0, false>)
           : c->cfg.rot_mode == NPG_ROT_EXPMAP
               ? (ts ? mlp_bwd_tc2_kernel<1, true> : mlp_bwd_tc2_kernel<1, false>)
               : (ts ? mlp_bwd_tc2_kernel<2, true> : mlp_bwd_tc2_kernel<2, false>);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long tiles = (long long)((c->N + 15) / 16) * ((c->T + 7) / 8);
  if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;  // tile indices are ints
  k<<<tc_grid(c, tiles, 2), BWD64_THREADS, smem, c->stream>>>(make_tc_args(c));
  return cudaGetLastError();
}

}  // namespace npg
