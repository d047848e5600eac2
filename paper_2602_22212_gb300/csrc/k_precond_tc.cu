// Tensor-core DCT pass of the Sobolev preconditioner (Eq. 9).
//
// Same pass as dct_pass_kernel (k_step.cu): out[p][k][c] = s(p,k) sum_n
// Mx[k][n] in[n][p F + c], with Mx = C or C^T and the optional spectral
// scaling s = 1 / (1 + lambda (mu_kz + mu_ky + mu_kx))^2, but the contraction
// runs on tcgen05 in split BF16: every FP32 value x is carried as
// hi = bf16(x), lo = bf16(x - hi) (16 significant bits), and
//   Mx . In ~ Mx_hi In_hi + Mx_hi In_lo + Mx_lo In_hi
// (the dropped lo.lo term is below 2^-16 relative), accumulated in FP32 in
// TMEM: about 1e-5 relative per pass.
//
// Persistent, warp-specialised CTA, one per SM, looping over column tiles of
// 128: the tile covers all r output rows (one or two 128-row MMA blocks); K
// (the transformed axis n) is streamed in chunks of 64. The table blocks (one
// 128-row block of C's hi and lo rows per K chunk, 32 KB, pre-swizzled, from
// L2) and the input chunks (64 rows x 128 columns, hi and lo, 32 KB, from HBM)
// come through two separate shared-memory rings of four and three slots, so
// that the input of the next two chunks and the table of the next one are in
// flight while one chunk is multiplied. One thread issues 12 MMAs per table
// block into one of two TMEM accumulators while the epilogue warps drain the
// other with coalesced rotated stores (8-byte hi / lo pieces for F = 4).
//
// Between the passes of one preconditioner call the data stays split: a pass
// may store its output as the hi and lo BF16 arrays (the same bytes as FP32,
// rows padded to a multiple of 8 elements), and the next pass then loads its
// input tiles with TMA straight into the swizzled operand layout, so that its
// producer warps move no data through registers. Only the first pass reads
// FP32 (by TMA into the input slot, where its producers split it in place) and
// only the last one writes FP32.
#include <cuda.h>  // CUtensorMap and its encoder's types (the encoder is fetched at run time)
#include <cuda_bf16.h>

#include <mutex>

#include "npg_internal.cuh"
#include "tc_sm100.cuh"

namespace npg {

namespace {
constexpr uint32_t TILE_A = 128 * 128;  // [128][64] BF16, 128B-swizzled
constexpr uint32_t ATOM_B = 64 * 128;   // MN-major atom: 64 K-rows x 64 columns BF16
constexpr uint32_t A_SLOT = 2 * TILE_A;  // hi and lo of one 128-row table block
constexpr uint32_t B_SLOT = 4 * ATOM_B;  // hi (2 atoms) and lo (2 atoms) of one input chunk
constexpr int NA = 4, NB = 3;            // ring depths (table blocks, input chunks)
constexpr uint32_t WAIT = 1u << 22;
// Warp roles: input producers [0, BW), the table warp BW, (FP32 input) the raw
// warp BW + 1, epilogue [PW, PW + EW), the MMA warp PW + EW. A pass that splits
// FP32 input needs 4 input warps, which split the raw chunks that the raw warp
// brings by TMA (or load them themselves); one whose input comes split by TMA
// needs one thread to issue it. Both have 8 epilogue warps, two per TMEM lane
// quarter, each draining half of the tile's columns. The table blocks have a
// warp of their own so that the input copies run ahead of them, as far as the
// input ring allows.
template <bool IN_SPLIT> struct Roles {
  static constexpr int BW = IN_SPLIT ? 1 : 4, PW = IN_SPLIT ? BW + 1 : BW + 2;
  static constexpr int EW = 8;
  static constexpr int PRODUCERS = BW * 32, EPILOGUE = EW * 32, MMA_WARP = PW + EW;
  static constexpr int THREADS = (PW + EW + 1) * 32;
};
constexpr int PRODUCERS = Roles<false>::PRODUCERS;


// Table ring (NA blocks [hi, lo] of 128 rows x 64 K), input ring (NB chunks
// [hi atom 0, hi atom 1, lo atom 0, lo atom 1]), the spectral weights mu (r <=
// 256) and the barriers.
struct PcSmem {
  static constexpr uint32_t A = 0;
  static constexpr uint32_t B = A + NA * A_SLOT;
  static constexpr uint32_t MU = B + NB * B_SLOT;
  // a_full[NA], a_empty[NA], b_full[NB], b_empty[NB], acc_full[2], acc_empty[2], fin,
  // raw_full[NB], raw_read[NB]
  static constexpr uint32_t BAR = MU + 256 * 4;
  static constexpr uint32_t NBAR = 2 * NA + 4 * NB + 5;
  static constexpr uint32_t FLAGS = BAR + NBAR * 8;
  static constexpr uint32_t TOTAL = FLAGS + 16;
};
static_assert(PcSmem::TOTAL + 1024 <= 232448, "shared memory of one CTA");

__device__ __forceinline__ uint32_t mn_off(uint32_t m, uint32_t k) {
  return (m >> 6) * ATOM_B + (k >> 3) * 1024u + (k & 7u) * 128u +
         (((((m & 63u) >> 3) ^ (k & 7u)) & 7u) << 4) + (m & 7u) * 2u;
}

__device__ __forceinline__ void split8(const float* x, uint4& hi, uint4& lo) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const __nv_bfloat16 a = __float2bfloat16_rn(x[2 * j]);
    const __nv_bfloat16 b = __float2bfloat16_rn(x[2 * j + 1]);
    const float ra = x[2 * j] - __bfloat162float(a);
    const float rb = x[2 * j + 1] - __bfloat162float(b);
    h[j] = (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
    l[j] = tc::pack_bf16(ra, rb);
  }
  hi = make_uint4(h[0], h[1], h[2], h[3]);
  lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// hi = bf16(x), lo = bf16(x - hi) of 4 values, packed in pairs.
__device__ __forceinline__ void split4(float4 x, uint2& hi, uint2& lo) {
  const float v[4] = {x.x, x.y, x.z, x.w};
  uint32_t h[2], l[2];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const __nv_bfloat16 a = __float2bfloat16_rn(v[2 * j]);
    const __nv_bfloat16 b = __float2bfloat16_rn(v[2 * j + 1]);
    h[j] = (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
    l[j] = tc::pack_bf16(v[2 * j] - __bfloat162float(a), v[2 * j + 1] - __bfloat162float(b));
  }
  hi = make_uint2(h[0], h[1]);
  lo = make_uint2(l[0], l[1]);
}

// Bounded wait shared by every role; gives up (and flags the CTA) once any
// thread of the CTA has timed out.
__device__ __forceinline__ bool pc_wait(uint64_t* bar, uint32_t phase, volatile int* abort,
                                        int* err) {
  for (uint32_t k = 0; k < WAIT; ++k) {
    if (tc::mbar_try_wait(bar, phase)) return true;
    if ((k & 1023u) == 1023u && *abort) return false;
  }
  *abort = 1;
  atomicExch(err, 1);
  return false;
}
}  // namespace

// One pass, persistent and warp-specialised: the producer warps (bulk copies
// of the table blocks into the table ring; TMA loads, or load + split, of the
// input chunks into the input ring), the epilogue warps draining one TMEM
// accumulator to global memory and the MMA warp filling the other. CTAs loop
// over column tiles of 128.
// tabs: pre-swizzled 32 KB slots [kc][mt][hi, lo] (dct_tc_tables).
// IN_SPLIT: the input is hi / lo BF16 rows loaded by TMA (tm_hi, tm_lo, boxes
// of 64 rows x 64 columns, 128B swizzle); else FP32 `in`, split by the
// producers after the raw warp brought it by TMA (tm_raw, boxes of 64 rows x
// 32 columns, 128B swizzle; raw_tma != 0) or loaded by themselves (raw_tma ==
// 0: rows that are not 16-byte multiples or an unaligned base). OUT_SPLIT: the
// output goes to hi / lo BF16 arrays `ohi`, `olo` with row pitch `pitch`; else
// FP32 `out`.
template <bool SCALE, bool IN_SPLIT, bool OUT_SPLIT>
__global__ void __launch_bounds__(Roles<IN_SPLIT>::THREADS, 1) dct_pass_tc_kernel(
    const float* __restrict__ in, float* __restrict__ out, const uint8_t* __restrict__ tabs,
    const float* __restrict__ mu, int r, int F, float lambda, int* err,
    const __grid_constant__ CUtensorMap tm_hi, const __grid_constant__ CUtensorMap tm_lo,
    __nv_bfloat16* __restrict__ ohi, __nv_bfloat16* __restrict__ olo, long long pitch,
    const __grid_constant__ CUtensorMap tm_raw, int raw_tma) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = tc::align1024(smem_raw);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + PcSmem::BAR);
  uint64_t* a_full = bars;
  uint64_t* a_empty = a_full + NA;
  uint64_t* b_full = a_empty + NA;
  uint64_t* b_empty = b_full + NB;
  uint64_t* acc_full = b_empty + NB;
  uint64_t* acc_empty = acc_full + 2;
  uint64_t* fin = acc_empty + 2;
  uint64_t* raw_full = fin + 1;
  uint64_t* raw_read = raw_full + NB;
  volatile int* abort = reinterpret_cast<volatile int*>(sm + PcSmem::FLAGS);
  uint32_t* tmem_ptr = reinterpret_cast<uint32_t*>(sm + PcSmem::FLAGS + 4);
  float* smu = reinterpret_cast<float*>(sm + PcSmem::MU);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int nM = (r + 127) >> 7, nK = (r + 63) >> 6;
  const uint32_t acc_cols = (uint32_t)nM * 128u;
  const uint32_t tm_cols = nM == 2 ? 512u : 256u;
  const long long ncol = (long long)r * r * F;
  const long long ntiles = (ncol + 127) / 128;
  using RL = Roles<IN_SPLIT>;
  for (int k = tid; k < r; k += RL::THREADS) smu[k] = mu[k];
  if (tid == 0) {
    for (int b = 0; b < NA; ++b) {
      tc::mbar_init(a_full + b, 1);
      tc::mbar_init(a_empty + b, 1);
    }
    for (int b = 0; b < NB; ++b) {
      // TMA input: thread 0 arrives with the transaction count; split input:
      // every producer arrives once its share of the chunk is stored
      tc::mbar_init(b_full + b, IN_SPLIT ? 1 : RL::PRODUCERS);
      tc::mbar_init(b_empty + b, 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(acc_full + b, 1);
      tc::mbar_init(acc_empty + b, RL::EPILOGUE);
    }
    tc::mbar_init(fin, 1);
    for (int b = 0; b < NB; ++b) {
      tc::mbar_init(raw_full + b, 1);
      tc::mbar_init(raw_read + b, RL::PRODUCERS);
    }
    *abort = 0;
    tc::fence_mbar_init();
  }
  if (warp == RL::MMA_WARP) {
    tc::tmem_alloc(tmem_ptr, tm_cols);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_ptr;

  if (warp < RL::BW) {
    // ------------------------------------------------------------ input producers
    // TMA input: thread 0 issues the chunk's four loads. FP32 input: every
    // producer loads, splits and stores its share of the chunk.
    uint32_t ub = 0;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
      const long long col0 = tile * 128;
      for (int kc = 0; kc < nK; ++kc, ++ub) {
        const uint32_t sbi = ub % NB, bph = (ub / NB) & 1u;
        if (!pc_wait(b_empty + sbi, bph ^ 1u, abort, err)) goto inputs_done;
        uint8_t* sb = sm + PcSmem::B + sbi * B_SLOT;
        if (IN_SPLIT) {
          if (tid == 0) {
            tc::mbar_arrive_expect_tx(b_full + sbi, B_SLOT);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              tc::tma_load_2d(sb + h * ATOM_B, &tm_hi, (int)(col0 + 64 * h), kc * 64,
                              b_full + sbi);
              tc::tma_load_2d(sb + (2 + h) * ATOM_B, &tm_lo, (int)(col0 + 64 * h), kc * 64,
                              b_full + sbi);
            }
          }
          continue;
        }
        // 64 K-rows x 16 groups of 8 columns, in two halves of 32 rows; each
        // half's loads are issued before its stores. The raw rows 0-31 and the
        // split rows 0-31 both lie in the first 4 KB of each 8 KB box / atom of
        // the slot, rows 32-63 in the second: a half's stores overwrite only
        // raw values of the same half.
        constexpr int PER = 32 * 16 / PRODUCERS;
        if (raw_tma && !pc_wait(raw_full + sbi, bph, abort, err)) goto inputs_done;
#pragma unroll 1
        for (int half = 0; half < 2; ++half) {
          float x[PER][8];
          if (raw_tma) {
            // the raw FP32 chunk is in this slot (four 128B-swizzled boxes of
            // 64 rows x 32 columns); every producer reads its values of the
            // half before any of them overwrites it with the split operand
#pragma unroll
            for (int i = 0; i < PER; ++i) {
              const int e = tid + i * PRODUCERS;
              const uint32_t n = (uint32_t)(32 * half + (e >> 4)), g = (uint32_t)(e & 15);
              const uint8_t* row = sb + (g >> 2) * 8192u + n * 128u;
              const uint32_t c0 = (g & 3u) * 2u;
              const float4 a = *reinterpret_cast<const float4*>(row + ((c0 ^ (n & 7u)) << 4));
              const float4 b =
                  *reinterpret_cast<const float4*>(row + (((c0 + 1u) ^ (n & 7u)) << 4));
              x[i][0] = a.x; x[i][1] = a.y; x[i][2] = a.z; x[i][3] = a.w;
              x[i][4] = b.x; x[i][5] = b.y; x[i][6] = b.z; x[i][7] = b.w;
            }
            // one phase per half: the phase of half h has parity h
            tc::mbar_arrive(raw_read + sbi);
            if (!pc_wait(raw_read + sbi, (uint32_t)half, abort, err)) goto inputs_done;
          } else
#pragma unroll
          for (int i = 0; i < PER; ++i) {
            const int e = tid + i * PRODUCERS;
            const int n = kc * 64 + 32 * half + (e >> 4);
            const long long c0 = col0 + (e & 15) * 8;
            if (n < r && (ncol & 3) == 0 && c0 + 8 <= ncol) {
              const float4* p = reinterpret_cast<const float4*>(in + (long long)n * ncol + c0);
              const float4 a = __ldcs(p), b = __ldcs(p + 1);
              x[i][0] = a.x; x[i][1] = a.y; x[i][2] = a.z; x[i][3] = a.w;
              x[i][4] = b.x; x[i][5] = b.y; x[i][6] = b.z; x[i][7] = b.w;
            } else {
#pragma unroll
              for (int j = 0; j < 8; ++j)
                x[i][j] = (n < r && c0 + j < ncol) ? in[(long long)n * ncol + c0 + j] : 0.f;
            }
          }
#pragma unroll
          for (int i = 0; i < PER; ++i) {
            const int e = tid + i * PRODUCERS;
            uint4 hi, lo;
            split8(x[i], hi, lo);
            const uint32_t o =
                mn_off((uint32_t)((e & 15) * 8), (uint32_t)(32 * half + (e >> 4)));
            *reinterpret_cast<uint4*>(sb + o) = hi;
            *reinterpret_cast<uint4*>(sb + 2 * ATOM_B + o) = lo;
          }
        }
        tc::fence_async_smem();
        tc::mbar_arrive(b_full + sbi);
      }
    }
  inputs_done:
    // Do not leave with a copy in flight: wait (bounded) for the last copy
    // issued into every slot. A slot whose copies were all consumed has
    // completed that phase, and the wait returns at once.
    if (IN_SPLIT && tid == 0)
      for (uint32_t i = 0; i < NB && i < ub; ++i) {
        const uint32_t last = ub - 1 - ((ub - 1 - i) % NB);  // latest u < ub with u % NB == i
        tc::mbar_wait(b_full + i, (last / NB) & 1u, WAIT);
      }
  } else if (warp == RL::BW) {
    // ------------------------------------------------------------ table blocks
    if ((tid & 31) == 0) {
      uint32_t ua = 0;
      for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x)
        for (int kc = 0; kc < nK; ++kc)
          for (int mt = 0; mt < nM; ++mt, ++ua) {
            const uint32_t sai = ua % NA, aph = (ua / NA) & 1u;
            if (!pc_wait(a_empty + sai, aph ^ 1u, abort, err)) goto tables_done;
            tc::mbar_arrive_expect_tx(a_full + sai, A_SLOT);
            tc::bulk_g2s(sm + PcSmem::A + sai * A_SLOT, tabs + ((size_t)kc * nM + mt) * A_SLOT,
                         A_SLOT, a_full + sai);
          }
    tables_done:
      for (uint32_t i = 0; i < NA && i < ua; ++i) {
        const uint32_t last = ua - 1 - ((ua - 1 - i) % NA);
        tc::mbar_wait(a_full + i, (last / NA) & 1u, WAIT);
      }
    }
  } else if (!IN_SPLIT && warp == RL::BW + 1) {
    // ------------------------------------------------------------ raw FP32 chunks
    // Lane 0 brings each input chunk as FP32 into its slot of the input ring
    // (four 128B-swizzled TMA boxes of 64 rows x 32 columns; rows and columns
    // outside the level read as 0), as far ahead as the ring allows.
    if (raw_tma && (tid & 31) == 0) {
      uint32_t ub = 0;
      for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x)
        for (int kc = 0; kc < nK; ++kc, ++ub) {
          const uint32_t sbi = ub % NB, bph = (ub / NB) & 1u;
          if (!pc_wait(b_empty + sbi, bph ^ 1u, abort, err)) goto raw_done;
          uint8_t* sb = sm + PcSmem::B + sbi * B_SLOT;
          tc::mbar_arrive_expect_tx(raw_full + sbi, B_SLOT);
#pragma unroll
          for (int b = 0; b < 4; ++b)
            tc::tma_load_2d(sb + b * 8192, &tm_raw, (int)(tile * 128 + 32 * b), kc * 64,
                            raw_full + sbi);
        }
    raw_done:
      for (uint32_t i = 0; i < NB && i < ub; ++i) {
        const uint32_t last = ub - 1 - ((ub - 1 - i) % NB);
        tc::mbar_wait(raw_full + i, (last / NB) & 1u, WAIT);
      }
    }
  } else if (warp == RL::MMA_WARP) {
    // ------------------------------------------------------------ MMA issuer
    // The whole warp follows the barriers; lane 0 issues.
    const bool leader = (tid & 31) == 0;
    constexpr uint32_t IDESC = tc::idesc_bf16(128, 128, false, true);
    uint32_t ua = 0, ub = 0, lt = 0;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++lt) {
      const uint32_t acc = lt & 1u, aph = (lt >> 1) & 1u;
      if (!pc_wait(acc_empty + acc, aph ^ 1u, abort, err)) break;
      tc::fence_after_sync();
      const uint32_t d0 = tmem + acc * acc_cols;
      bool ok = true;
      for (int kc = 0; kc < nK && ok; ++kc, ++ub) {
        const uint32_t sbi = ub % NB;
        if (!pc_wait(b_full + sbi, (ub / NB) & 1u, abort, err)) {
          ok = false;
          break;
        }
        const uint32_t sB = tc::smem_u32(sm + PcSmem::B + sbi * B_SLOT);
        for (int mt = 0; mt < nM; ++mt, ++ua) {
          const uint32_t sai = ua % NA;
          if (!pc_wait(a_full + sai, (ua / NA) & 1u, abort, err)) {
            ok = false;
            break;
          }
          tc::fence_after_sync();
          if (leader) {
            const uint32_t sA = tc::smem_u32(sm + PcSmem::A + sai * A_SLOT);
            const uint32_t d = d0 + mt * 128;
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
              const uint64_t ah = tc::kmajor_sw128(sA + 32 * ks);
              const uint64_t al = tc::kmajor_sw128(sA + TILE_A + 32 * ks);
              const uint64_t bh = tc::mnmajor_sw128(sB + 2048 * ks, ATOM_B, 1024);
              const uint64_t bl = tc::mnmajor_sw128(sB + 2 * ATOM_B + 2048 * ks, ATOM_B, 1024);
              tc::mma_bf16(d, ah, bh, IDESC, (kc > 0 || ks > 0) ? 1u : 0u);
              tc::mma_bf16(d, ah, bl, IDESC, 1u);
              tc::mma_bf16(d, al, bh, IDESC, 1u);
            }
            tc::mma_commit(a_empty + sai);
          }
          __syncwarp();
        }
        if (ok && leader) tc::mma_commit(b_empty + sbi);
        __syncwarp();
      }
      if (!ok) break;
      if (leader) tc::mma_commit(acc_full + acc);
      __syncwarp();
    }
    __syncwarp();
    // Do not free TMEM with MMAs in flight (bounded).
    if (leader) tc::mma_commit(fin);
    __syncwarp();
    tc::mbar_wait(fin, 0, WAIT);
  } else {
    // ------------------------------------------------------------ epilogue
    const int et = 32 * (warp & 3) + (tid & 31);  // TMEM lane of this thread
    // column range of the tile this warp drains
    const int cg_lo = RL::EW == 8 ? 64 * ((warp - RL::PW) >> 2) : 0;
    const int cg_hi = RL::EW == 8 ? cg_lo + 64 : 128;
    const uint32_t qlane = (uint32_t)((warp & 3) * 32) << 16;
    const long long rF = (long long)r * F;
    uint32_t lt = 0;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++lt) {
      const uint32_t acc = lt & 1u, aph = (lt >> 1) & 1u;
      if (!pc_wait(acc_full + acc, aph, abort, err)) break;
      tc::fence_after_sync();
      const long long col0 = tile * 128;
      // (pa, pb): the two untransformed axes of the tile's first column
      // (F = 4); later columns step pb, carrying into pa (32-bit, no division
      // per element)
      const int p0 = (int)(col0 >> 2);
      const int pa0 = p0 / r, pb0 = p0 - pa0 * r;
      for (int mt = 0; mt < nM; ++mt) {
        const int k = mt * 128 + et;
        const uint32_t lane = tmem + acc * acc_cols + mt * 128 + qlane;
        for (int cg = cg_lo; cg < cg_hi; cg += 16) {
          uint32_t v[16];
          tc::tmem_ld16(lane + cg, v);
          tc::tmem_ld_wait();
          if (k >= r) continue;
          if (F == 4) {
            int pa = pa0, pb = pb0 + (cg >> 2);
            while (pb >= r) {
              pb -= r;
              ++pa;
            }
            int pq[4], bq[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              if (q > 0 && ++pb == r) {
                pb = 0;
                ++pa;
              }
              pq[q] = pa;
              bq[q] = pb;
            }
            // the four scale factors first (independent of the stores; pa runs
            // past r - 1 only for columns beyond the level, never stored)
            float sc[4] = {1.f, 1.f, 1.f, 1.f};
            if (SCALE) {
              const float mk = smu[k];
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                const float dd = 1.f + lambda * (smu[min(pq[q], r - 1)] + smu[bq[q]] + mk);
                sc[q] = __frcp_rn(dd * dd);  // = 1 / dd^2, correctly rounded
              }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const int pa = pq[q], pb = bq[q];
              const long long col = col0 + cg + 4 * q;
              if (col >= ncol) break;
              const float x0 = __uint_as_float(v[4 * q]) * sc[q];
              const float x1 = __uint_as_float(v[4 * q + 1]) * sc[q];
              const float x2 = __uint_as_float(v[4 * q + 2]) * sc[q];
              const float x3 = __uint_as_float(v[4 * q + 3]) * sc[q];
              if (OUT_SPLIT) {
                const long long o = (long long)pa * pitch + (long long)pb * rF + (long long)k * 4;
                uint2 hi, lo;
                split4(make_float4(x0, x1, x2, x3), hi, lo);
                __stcs(reinterpret_cast<uint2*>(ohi + o), hi);
                __stcs(reinterpret_cast<uint2*>(olo + o), lo);
              } else {
                const long long o = ((long long)pa * r + pb) * rF + (long long)k * 4;
                __stcs(reinterpret_cast<float4*>(out + o), make_float4(x0, x1, x2, x3));
              }
            }
          } else {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const long long col = col0 + cg + j;
              if (col >= ncol) break;
              const int pi = (int)col / F;
              const int c = (int)col - pi * F;
              const int pa = pi / r, pb = pi - pa * r;
              float sc = 1.f;
              if (SCALE) {
                const float dd = 1.f + lambda * (smu[pa] + smu[pb] + smu[k]);
                sc = __frcp_rn(dd * dd);  // = 1 / dd^2, correctly rounded
              }
              const float x = __uint_as_float(v[j]) * sc;
              if (OUT_SPLIT) {
                const long long o =
                    (long long)pa * pitch + (long long)pb * rF + (long long)k * F + c;
                const __nv_bfloat16 h = __float2bfloat16_rn(x);
                ohi[o] = h;
                olo[o] = __float2bfloat16_rn(x - __bfloat162float(h));
              } else {
                out[(long long)pi * rF + (long long)k * F + c] = x;
              }
            }
          }
        }
      }
      tc::fence_before_sync();
      tc::mbar_arrive(acc_empty + acc);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == RL::MMA_WARP) {
    __syncwarp();
    tc::tmem_dealloc(tmem, tm_cols);
  }
}

size_t dct_tc_table_elems(int r) {
  const int nM = (r + 127) / 128, nK = (r + 63) / 64;
  return (size_t)nK * nM * 2 * (TILE_A / 2);  // BF16 elements
}

static uint16_t bf16_bits_rne(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) == 0x7f800000u) return (uint16_t)(u >> 16);
  const uint32_t lsb = (u >> 16) & 1u;
  u += 0x7fffu + lsb;
  return (uint16_t)(u >> 16);
}

static float bf16_to_float(uint16_t b) {
  const uint32_t u = (uint32_t)b << 16;
  float f;
  memcpy(&f, &u, 4);
  return f;
}

// Split BF16 hi / lo tables of an FP32 r x r matrix (row-major), stored as the
// shared-memory images the kernel copies: for K chunk kc and row block mt, the
// 32 KB slot [hi, lo], each [128 rows][64 columns] 128B-swizzled.
void dct_tc_tables(int r, const float* Mx, uint16_t* dst) {
  const int nM = (r + 127) / 128, nK = (r + 63) / 64;
  uint8_t* base = reinterpret_cast<uint8_t*>(dst);
  memset(base, 0, dct_tc_table_elems(r) * 2);
  for (int kc = 0; kc < nK; ++kc)
    for (int part = 0; part < 2; ++part)
      for (int mt = 0; mt < nM; ++mt) {
        uint8_t* blk = base + ((size_t)kc * nM + mt) * A_SLOT + part * TILE_A;
        for (int rr = 0; rr < 128; ++rr)
          for (int k = 0; k < 64; ++k) {
            const int i = mt * 128 + rr, j = kc * 64 + k;
            const float v = (i < r && j < r) ? Mx[(size_t)i * r + j] : 0.f;
            const uint16_t h = bf16_bits_rne(v);
            const uint16_t b = part == 0 ? h : bf16_bits_rne(v - bf16_to_float(h));
            const uint32_t off = (uint32_t)(rr >> 3) * 1024u + (uint32_t)(rr & 7) * 128u +
                                 ((((uint32_t)(k >> 3)) ^ (uint32_t)(rr & 7)) << 4) +
                                 (uint32_t)(k & 7) * 2u;
            memcpy(blk + off, &b, 2);
          }
      }
}

// Row pitch (elements) of the split hi / lo intermediates of an r^3 x F level:
// r^2 F rounded up to 8, so that every row starts 16-byte aligned for TMA.
long long dct_tc_split_pitch(int r, int F) { return (((long long)r * r * F) + 7) & ~7LL; }

size_t dct_tc_scratch_elems(int r, int F) {
  // hi + lo BF16 of r rows of `pitch` elements, in units of floats
  return (size_t)r * (size_t)dct_tc_split_pitch(r, F);
}

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_tiled() {
  static std::once_flag once;
  static EncodeTiledFn fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    cudaGetLastError();
  });
  return fn;
}

// Tensor map of one split array: `rows` rows of `cols` BF16 with row pitch
// `pitch` elements; boxes of 64 x 64, 128-byte swizzle, zero fill outside.
static bool split_map(CUtensorMap* m, const __nv_bfloat16* base, int rows, long long cols,
                      long long pitch) {
  EncodeTiledFn enc = encode_tiled();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)pitch * 2};
  const cuuint32_t box[2] = {64, 64};
  const cuuint32_t estr[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(base), dims,
             strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

// Tensor map of the FP32 input: r rows of `cols` floats; boxes of 64 rows x 32
// columns, 128-byte swizzle, zero fill outside. Needs 16-byte aligned rows.
static bool raw_map(CUtensorMap* m, const float* base, int rows, long long cols) {
  EncodeTiledFn enc = encode_tiled();
  if (!enc || (cols & 3) != 0 || (reinterpret_cast<uintptr_t>(base) & 15) != 0) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)cols * 4};
  const cuuint32_t box[2] = {32, 64};
  const cuuint32_t estr[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box,
             estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

// t0, t1: scratch of dct_tc_scratch_elems(r, F) floats each, holding the split
// intermediates (hi then lo BF16 arrays).
cudaError_t launch_precondition_tc(const float* g, float* out, float* t0, float* t1,
                                   const uint16_t* tabC, const uint16_t* tabCt, const float* mu,
                                   int r, int F, float lambda, int* err, cudaStream_t s) {
  const size_t smem = PcSmem::TOTAL + 1024;
  static bool attr = false;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(dct_pass_tc_kernel<false, false, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(dct_pass_tc_kernel<false, true, true>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(dct_pass_tc_kernel<true, true, true>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(dct_pass_tc_kernel<false, true, false>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const long long ncol = (long long)r * r * F;
  const long long pitch = dct_tc_split_pitch(r, F);
  const long long tiles = (ncol + 127) / 128;
  const unsigned grid = (unsigned)(tiles < sms ? tiles : sms);
  const uint8_t* C = reinterpret_cast<const uint8_t*>(tabC);
  const uint8_t* Ct = reinterpret_cast<const uint8_t*>(tabCt);
  __nv_bfloat16* h0 = reinterpret_cast<__nv_bfloat16*>(t0);
  __nv_bfloat16* l0 = h0 + (long long)r * pitch;
  __nv_bfloat16* h1 = reinterpret_cast<__nv_bfloat16*>(t1);
  __nv_bfloat16* l1 = h1 + (long long)r * pitch;
  CUtensorMap mh0, ml0, mh1, ml1;
  if (!split_map(&mh0, h0, r, ncol, pitch) || !split_map(&ml0, l0, r, ncol, pitch) ||
      !split_map(&mh1, h1, r, ncol, pitch) || !split_map(&ml1, l1, r, ncol, pitch))
    return cudaErrorInvalidValue;
  // g -> t0 (split) -> t1 -> t0 (scaled) -> t1 -> t0 -> out (FP32)
  constexpr int T0 = Roles<false>::THREADS, T1 = Roles<true>::THREADS;
  // the first pass reads its FP32 input by TMA where the rows allow it (else
  // its producers load it)
  CUtensorMap mraw;
  const int raw = raw_map(&mraw, g, r, ncol) ? 1 : 0;
  if (!raw) mraw = mh0;  // not read
  dct_pass_tc_kernel<false, false, true><<<grid, T0, smem, s>>>(
      g, nullptr, C, mu, r, F, lambda, err, mh1, ml1, h0, l0, pitch, mraw, raw);
  dct_pass_tc_kernel<false, true, true><<<grid, T1, smem, s>>>(
      nullptr, nullptr, C, mu, r, F, lambda, err, mh0, ml0, h1, l1, pitch, mh0, 0);
  dct_pass_tc_kernel<true, true, true><<<grid, T1, smem, s>>>(
      nullptr, nullptr, C, mu, r, F, lambda, err, mh1, ml1, h0, l0, pitch, mh0, 0);
  dct_pass_tc_kernel<false, true, true><<<grid, T1, smem, s>>>(
      nullptr, nullptr, Ct, mu, r, F, lambda, err, mh0, ml0, h1, l1, pitch, mh0, 0);
  dct_pass_tc_kernel<false, true, true><<<grid, T1, smem, s>>>(
      nullptr, nullptr, Ct, mu, r, F, lambda, err, mh1, ml1, h0, l0, pitch, mh0, 0);
  dct_pass_tc_kernel<false, true, false><<<grid, T1, smem, s>>>(
      nullptr, out, Ct, mu, r, F, lambda, err, mh0, ml0, nullptr, nullptr, pitch, mh0, 0);
  return cudaGetLastError();
}

}  // namespace npg
