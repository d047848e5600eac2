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
// CTA = 128 threads, tile = all r output rows (one or two 128-row MMA
// blocks) x 128 columns; K (the transformed axis n) streamed in chunks of 64.
// Each chunk: the tables' hi/lo rows are copied into K-major swizzled tiles,
// the input columns are loaded, split and written as MN-major tiles, then one
// thread issues 12 MMAs per 128-row block. The epilogue stores the rotated
// layout with coalesced float4 writes (F = 4) or scalar writes.
#include <cuda_bf16.h>

#include "npg_internal.cuh"
#include "tc_sm100.cuh"

namespace npg {

namespace {
constexpr uint32_t TILE_A = 128 * 128;  // [128][64] BF16
constexpr uint32_t ATOM_B = 64 * 128;   // MN-major atom: 64 K-rows x 64 columns BF16
constexpr uint32_t WAIT = 1u << 24;

struct PcSmem {
  // A: [hi m0, hi m1, lo m0, lo m1], B: [hi (2 atoms), lo (2 atoms)]
  static constexpr uint32_t A = 0;
  static constexpr uint32_t B = 4 * TILE_A;
  static constexpr uint32_t MU = B + 4 * ATOM_B;
  static constexpr uint32_t BAR = MU + 1024 * 4;
  static constexpr uint32_t TMEMP = BAR + 8;
  static constexpr uint32_t TOTAL = TMEMP + 8;
};

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
}  // namespace

// tabs: hi then lo, each [rm][rk] BF16 row-major (rm = nM * 128, rk = K chunks * 64),
// zero-padded.
template <bool SCALE>
__global__ void __launch_bounds__(128) dct_pass_tc_kernel(const float* __restrict__ in,
                                                          float* __restrict__ out,
                                                          const __nv_bfloat16* __restrict__ tabs,
                                                          const float* __restrict__ mu, int r,
                                                          int F, float lambda, int* err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + PcSmem::BAR);
  uint32_t* tmem_ptr = reinterpret_cast<uint32_t*>(sm + PcSmem::TMEMP);
  float* smu = reinterpret_cast<float*>(sm + PcSmem::MU);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int nM = (r + 127) >> 7, nK = (r + 63) >> 6;
  const int rm = nM * 128, rk = nK * 64;
  const long long ncol = (long long)r * r * F;
  const long long col0 = (long long)blockIdx.x * 128;
  for (int k = tid; k < r; k += 128) smu[k] = mu[k];
  if (tid == 0) {
    tc::mbar_init(bar, 1);
    tc::fence_mbar_init();
  }
  if (warp == 0) {
    tc::tmem_alloc(tmem_ptr, 256);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_ptr;
  const uint32_t sA = tc::smem_u32(sm + PcSmem::A), sB = tc::smem_u32(sm + PcSmem::B);
  constexpr uint32_t IDESC = tc::idesc_bf16(128, 128, false, true);
  const bool vec = (ncol & 3) == 0;
  uint32_t phase = 0;
  bool ok = true;

  for (int kc = 0; kc < nK && ok; ++kc) {
    // A: table rows [mt 128, +128) x columns [kc 64, +64), hi and lo
    const __nv_bfloat16* th = tabs;
    const __nv_bfloat16* tl = tabs + (long long)rm * rk;
    for (int e = tid; e < nM * 128 * 8; e += 128) {
      const int row = e >> 3, c = e & 7;  // row < nM * 128, 16-byte chunk c
      const long long g = (long long)row * rk + kc * 64 + c * 8;
      const uint4 vh = *reinterpret_cast<const uint4*>(th + g);
      const uint4 vl = *reinterpret_cast<const uint4*>(tl + g);
      const int mt = row >> 7, rr = row & 127;
      *reinterpret_cast<uint4*>(sm + PcSmem::A + mt * TILE_A + tc::sw128_off(rr, c * 8)) = vh;
      *reinterpret_cast<uint4*>(sm + PcSmem::A + (2 + mt) * TILE_A + tc::sw128_off(rr, c * 8)) =
          vl;
    }
    // B: input rows n in [kc 64, +64) x columns [col0, col0 + 128), split hi / lo
    for (int e = tid; e < 64 * 16; e += 128) {
      const int kk = e >> 4, g8 = e & 15;  // K-row, group of 8 columns
      const int n = kc * 64 + kk;
      const long long c0 = col0 + g8 * 8;
      float x[8];
      if (n < r && vec && c0 + 8 <= ncol) {
        const float4* p = reinterpret_cast<const float4*>(in + (long long)n * ncol + c0);
        const float4 a = p[0], b = p[1];
        x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
        x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
      } else {
#pragma unroll
        for (int j = 0; j < 8; ++j)
          x[j] = (n < r && c0 + j < ncol) ? in[(long long)n * ncol + c0 + j] : 0.f;
      }
      uint4 hi, lo;
      split8(x, hi, lo);
      const uint32_t o = mn_off((uint32_t)(g8 * 8), (uint32_t)kk);
      *reinterpret_cast<uint4*>(sm + PcSmem::B + o) = hi;
      *reinterpret_cast<uint4*>(sm + PcSmem::B + 2 * ATOM_B + o) = lo;
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (tid == 0) {
      for (int mt = 0; mt < nM; ++mt) {
        const uint32_t d = tmem + mt * 128;
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
          const uint64_t ah = tc::kmajor_sw128(sA + mt * TILE_A + 32 * ks);
          const uint64_t al = tc::kmajor_sw128(sA + (2 + mt) * TILE_A + 32 * ks);
          const uint64_t bh = tc::mnmajor_sw128(sB + 2048 * ks, ATOM_B, 1024);
          const uint64_t bl = tc::mnmajor_sw128(sB + 2 * ATOM_B + 2048 * ks, ATOM_B, 1024);
          tc::mma_bf16(d, ah, bh, IDESC, (kc > 0 || ks > 0) ? 1u : 0u);
          tc::mma_bf16(d, ah, bl, IDESC, 1u);
          tc::mma_bf16(d, al, bh, IDESC, 1u);
        }
      }
      tc::mma_commit(bar);
    }
    bool w = tc::mbar_wait(bar, phase, WAIT);
    phase ^= 1u;
    w = __syncthreads_and(w) != 0;
    if (!w) {
      ok = false;
      if (tid == 0) atomicExch(err, 1);
    }
    tc::fence_after_sync();
  }
  if (ok) {
    const long long rF = (long long)r * F;
    for (int mt = 0; mt < nM; ++mt) {
      const int k = mt * 128 + tid;  // output row of this lane
      const uint32_t lane = tmem + mt * 128 + ((uint32_t)(warp * 32) << 16);
      for (int cg = 0; cg < 128; cg += 16) {
        uint32_t v[16];
        tc::tmem_ld16(lane + cg, v);
        tc::tmem_ld_wait();
        if (k >= r) continue;
        if (F == 4) {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const long long col = col0 + cg + 4 * q;
            if (col >= ncol) break;
            const long long p = col >> 2;
            float s = 1.f;
            if (SCALE) {
              const float d = 1.f + lambda * (smu[p / r] + smu[p % r] + smu[k]);
              s = 1.f / (d * d);
            }
            float4 o4 = make_float4(__uint_as_float(v[4 * q]) * s, __uint_as_float(v[4 * q + 1]) * s,
                                    __uint_as_float(v[4 * q + 2]) * s,
                                    __uint_as_float(v[4 * q + 3]) * s);
            *reinterpret_cast<float4*>(out + p * rF + (long long)k * 4) = o4;
          }
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const long long col = col0 + cg + j;
            if (col >= ncol) break;
            const long long p = col / F;
            const int c = (int)(col - p * F);
            float s = 1.f;
            if (SCALE) {
              const float d = 1.f + lambda * (smu[p / r] + smu[p % r] + smu[k]);
              s = 1.f / (d * d);
            }
            out[p * rF + (long long)k * F + c] = __uint_as_float(v[j]) * s;
          }
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, 256);
}

size_t dct_tc_table_elems(int r) {
  const int nM = (r + 127) / 128, nK = (r + 63) / 64;
  return (size_t)2 * (nM * 128) * (nK * 64);  // hi and lo
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

// Split BF16 tables of an FP32 r x r matrix (row-major) into the padded
// layout the kernel reads: hi block then lo block.
void dct_tc_tables(int r, const float* Mx, uint16_t* dst) {
  const int nM = (r + 127) / 128, nK = (r + 63) / 64;
  const int rm = nM * 128, rk = nK * 64;
  uint16_t* hi = dst;
  uint16_t* lo = dst + (size_t)rm * rk;
  for (int i = 0; i < rm; ++i)
    for (int j = 0; j < rk; ++j) {
      const float v = (i < r && j < r) ? Mx[(size_t)i * r + j] : 0.f;
      const uint16_t h = bf16_bits_rne(v);
      hi[(size_t)i * rk + j] = h;
      lo[(size_t)i * rk + j] = bf16_bits_rne(v - bf16_to_float(h));
    }
}

cudaError_t launch_precondition_tc(const float* g, float* out, float* t0, float* t1,
                                   const uint16_t* tabC, const uint16_t* tabCt, const float* mu,
                                   int r, int F, float lambda, int* err, cudaStream_t s) {
  const size_t smem = PcSmem::TOTAL + 1024;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(dct_pass_tc_kernel<false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(dct_pass_tc_kernel<true>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const long long ncol = (long long)r * r * F;
  const unsigned grid = (unsigned)((ncol + 127) / 128);
  const __nv_bfloat16* C = reinterpret_cast<const __nv_bfloat16*>(tabC);
  const __nv_bfloat16* Ct = reinterpret_cast<const __nv_bfloat16*>(tabCt);
  dct_pass_tc_kernel<false><<<grid, 128, smem, s>>>(g, t0, C, mu, r, F, lambda, err);
  dct_pass_tc_kernel<false><<<grid, 128, smem, s>>>(t0, t1, C, mu, r, F, lambda, err);
  dct_pass_tc_kernel<true><<<grid, 128, smem, s>>>(t1, t0, C, mu, r, F, lambda, err);
  dct_pass_tc_kernel<false><<<grid, 128, smem, s>>>(t0, t1, Ct, mu, r, F, lambda, err);
  dct_pass_tc_kernel<false><<<grid, 128, smem, s>>>(t1, t0, Ct, mu, r, F, lambda, err);
  dct_pass_tc_kernel<false><<<grid, 128, smem, s>>>(t0, out, Ct, mu, r, F, lambda, err);
  return cudaGetLastError();
}

}  // namespace npg
