// Bidirectional Chamfer term (Sec. 3.5): per-frame uniform-grid bucketing
// (counting sort), exact bucketed nearest-neighbour search in both directions,
// the per-frame FP64 reductions of cd_t and L_iso, the confidence weights
// (Eq. 11-12), the loss (Eq. 8, 10, 13), and dL/dx-hat.
#include <float.h>

#include "npg_device.cuh"
#include "npg_internal.cuh"

namespace npg {

__device__ __forceinline__ int set_of(long long k, long long uniform, const long long* off,
                                      int nsets) {
  if (off == nullptr) return (int)(k / uniform);
  int lo = 0, hi = nsets - 1;  // largest s with off[s] <= k
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= k) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ long long set_base(int s, long long uniform, const long long* off) {
  return off == nullptr ? (long long)s * uniform : off[s];
}

__device__ __forceinline__ int cell_axis(float v, int G) {
  int c = (int)floorf((v + 1.f) * (0.5f * (float)G));
  return min(max(c, 0), G - 1);
}

// ----------------------------------------------------------------- bucketing

__global__ void bucket_count_kernel(const float4* __restrict__ pts, const long long* off,
                                    long long uniform, int nsets, long long total, int G,
                                    int* __restrict__ counts, int* __restrict__ slot) {
  const long long G3 = (long long)G * G * G;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < total;
       k += (long long)gridDim.x * blockDim.x) {
    const int s = set_of(k, uniform, off, nsets);
    const float4 p = pts[k];
    const int cell = (cell_axis(p.z, G) * G + cell_axis(p.y, G)) * G + cell_axis(p.x, G);
    slot[k] = atomicAdd(&counts[s * G3 + cell], 1);
  }
}

// One block per set: exclusive scan of G^3 counts -> G^3 + 1 starts, in
// tiles of SCAN_TILE counts. A tile is loaded with coalesced thread-strided
// reads (the next tile's loads are issued before the current tile is
// scanned), transposed through padded shared memory so that each thread owns
// SCAN_PER consecutive counts, scanned, and stored back coalesced.
constexpr int SCAN_THREADS = 1024, SCAN_PER = 8, SCAN_TILE = SCAN_THREADS * SCAN_PER;

__device__ __forceinline__ int scan_pad(int i) { return i + (i >> 5); }

__global__ void __launch_bounds__(SCAN_THREADS) bucket_scan_kernel(const int* __restrict__ counts,
                                                                    int* __restrict__ starts,
                                                                    int G) {
  __shared__ int tile[SCAN_TILE + SCAN_TILE / 32];
  __shared__ int warp_sums[32];
  const long long G3 = (long long)G * G * G;
  const int* cnt = counts + blockIdx.x * G3;
  int* st = starts + blockIdx.x * (G3 + 1);
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  int next[SCAN_PER];
#pragma unroll
  for (int j = 0; j < SCAN_PER; ++j) {
    const long long k = (long long)j * SCAN_THREADS + tid;
    next[j] = k < G3 ? __ldcs(cnt + k) : 0;
  }
  int carry = 0;
  for (long long base = 0; base < G3; base += SCAN_TILE) {
#pragma unroll
    for (int j = 0; j < SCAN_PER; ++j) tile[scan_pad(j * SCAN_THREADS + tid)] = next[j];
    const long long nb = base + SCAN_TILE;
#pragma unroll
    for (int j = 0; j < SCAN_PER; ++j) {
      const long long k = nb + (long long)j * SCAN_THREADS + tid;
      next[j] = k < G3 ? __ldcs(cnt + k) : 0;
    }
    __syncthreads();
    int v[SCAN_PER], local = 0;
#pragma unroll
    for (int j = 0; j < SCAN_PER; ++j) {
      v[j] = local;
      local += tile[scan_pad(tid * SCAN_PER + j)];
    }
    int inc = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int n = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += n;
    }
    if (lane == 31) warp_sums[wid] = inc;
    __syncthreads();
    if (wid == 0) {
      int w = warp_sums[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int n = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += n;
      }
      warp_sums[lane] = w;
    }
    __syncthreads();
    const int before = carry + (inc - local) + (wid > 0 ? warp_sums[wid - 1] : 0);
#pragma unroll
    for (int j = 0; j < SCAN_PER; ++j) tile[scan_pad(tid * SCAN_PER + j)] = before + v[j];
    carry += warp_sums[31];
    __syncthreads();
#pragma unroll
    for (int j = 0; j < SCAN_PER; ++j) {
      const long long k = base + (long long)j * SCAN_THREADS + tid;
      if (k < G3) st[k] = tile[scan_pad(j * SCAN_THREADS + tid)];
    }
    __syncthreads();
  }
  if (tid == 0) st[G3] = carry;
}

__global__ void bucket_scatter_kernel(const float4* __restrict__ pts, const long long* off,
                                      long long uniform, int nsets, long long total, int G,
                                      const int* __restrict__ starts, const int* __restrict__ slot,
                                      float4* __restrict__ sorted) {
  const long long G3 = (long long)G * G * G;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < total;
       k += (long long)gridDim.x * blockDim.x) {
    const int s = set_of(k, uniform, off, nsets);
    const long long base = set_base(s, uniform, off);
    float4 p = pts[k];
    const int cell = (cell_axis(p.z, G) * G + cell_axis(p.y, G)) * G + cell_axis(p.x, G);
    const long long dst = base + starts[s * (G3 + 1) + cell] + slot[k];
    p.w = __int_as_float((int)(k - base));
    sorted[dst] = p;
  }
}

static int grid_blocks(long long n, int per) {
  long long b = (n + per - 1) / per;
  if (b > 65535 * 16) b = 65535 * 16;
  if (b < 1) b = 1;
  return (int)b;
}

cudaError_t bucket_build(const float4* pts, const long long* d_off, long long uniform_count,
                         int nsets, long long total, int G, Buckets& b, cudaStream_t s) {
  const long long G3 = (long long)G * G * G;
  b.src = pts;
  cudaError_t e = cudaMemsetAsync(b.counts, 0, sizeof(int) * G3 * nsets, s);
  if (e != cudaSuccess) return e;
  if (total > 0)
    bucket_count_kernel<<<grid_blocks(total, 256), 256, 0, s>>>(pts, d_off, uniform_count, nsets,
                                                                total, G, b.counts, b.slot);
  bucket_scan_kernel<<<nsets, SCAN_THREADS, 0, s>>>(b.counts, b.cell_start, G);
  if (total > 0)
    bucket_scatter_kernel<<<grid_blocks(total, 256), 256, 0, s>>>(
        pts, d_off, uniform_count, nsets, total, G, b.cell_start, b.slot, b.sorted);
  return cudaGetLastError();
}

int auto_cells(long long points_per_set, int nsets) {
  // surface data: about 2.8 G^2 occupied cells; aim at ~8 points per occupied
  // cell, capped so that nsets * G^3 cell starts stay below 32M entries
  double g = sqrt((double)points_per_set / 8.0);
  int G = (int)(g + 0.5);
  if (G < 1) G = 1;
  if (G > 96) G = 96;
  while (G > 1 && (double)G * G * G * nsets > 32.0e6) --G;
  return G;
}

// ----------------------------------------------------------------- NN search
// Exact nearest neighbour by growing Chebyshev rings of cells around the
// query's cell; a search stops once its best squared distance is below the
// squared distance to every unexplored cell (with a safety margin for FP32
// rounding of the cell assignment). Ties go to the lowest candidate index.
//
// Two passes balance the work: pass 1 (one thread per query, queries in cell
// order) searches rings 0..NN_NEAR_RINGS and finishes most queries; a query
// that is still open is appended to a queue with its best so far. Pass 2
// (a group of 8 lanes per queued query, the lanes splitting the cell rows)
// finishes the far queries, whose rings hold many (mostly empty) cells.
//
// Seeded search: when a starting candidate is known (the previous result of
// an optimisation loop; any index in range will do), its distance bounds the
// ball that can hold the nearest neighbour. The ball is then covered directly,
// one row segment per (z, y) cell row within reach, instead of ring by ring:
// every cell row costs two loads of cell starts, however many cells its
// segment spans. Balls of up to `near_rows` rows (set per direction) are covered
// in pass 1, wider ones in pass 2. The result is the same exact nearest neighbour; the
// seed only changes how much of the grid is visited.
constexpr int NN_NEAR_RINGS = 1;

struct NnGeom {
  const float4* qs;
  long long q_uniform;
  const long long* q_off;
  int nsets;
  long long q_total;
  const float4* cs;
  const int* cstart;
  int G;
  const long long* c_off;
  long long c_uniform;
  int* out_idx;
  float* out_d;
  unsigned long long* stats;
  int* qcount;  // [0] pushed, [1] popped
  int4* qitems;
  const float4* csrc;  // candidates in their own order (seed lookups)
  bool seeded;         // out_idx holds a starting candidate per query (or an invalid index)
  int near_rows;       // widest seed ball (cell rows) that pass 1 covers
};

// Candidates [lo, hi) of one cell row against the best (distance, index)
// pair, the lowest index winning ties. (Loading them four at a time measured
// slower: a row's candidates are contiguous and mostly hit L1 after the
// first, and short rows paid for the padding.)
__device__ __forceinline__ void scan_range(const float4* __restrict__ cs, long long cb, int lo,
                                           int hi, float4 q, float& best, int& bi) {
  for (int j = lo; j < hi; ++j) {
    const float4 p = cs[cb + j];
    const float d = sqdist(q.x, q.y, q.z, p.x, p.y, p.z);
    const int id = __float_as_int(p.w);
    if (d < best || (d == best && id < bi)) {
      best = d;
      bi = id;
    }
  }
}

// Distance from coordinate v to the extent of cell c along one axis, less a
// slack for FP32 rounding of the cell assignment; the boundary cells extend
// to infinity (they hold the clamped points).
__device__ __forceinline__ float axis_gap(float v, int c, int G, float h) {
  const float lo = c == 0 ? -FLT_MAX : fmaf((float)c, h, -1.f);
  const float hi = c == G - 1 ? FLT_MAX : fmaf((float)(c + 1), h, -1.f);
  const float gap = v < lo ? lo - v : (v > hi ? v - hi : 0.f);
  return fmaxf(gap - 4e-6f, 0.f);
}

// Scan the cells of row (z, y) that belong to the shell of ring `ring` and
// can still hold a point at squared distance <= best: a row whose (y, z)
// extent is farther than best is skipped, and only the x cells within reach
// of the best-ball are read (with a relative margin, so ties are kept).
// Returns whether the row's cell starts were read.
__device__ __forceinline__ bool scan_row(const NnGeom& g, const int* st, long long cb, int z,
                                         int y, int cx, int cy, int cz, int ring, float4 q,
                                         float h, float& best, int& bi,
                                         unsigned long long& nc) {
  const int G = g.G;
  const float gz = axis_gap(q.z, z, G, h), gy = axis_gap(q.y, y, G, h);
  const float base = gz * gz + gy * gy;
  const float reach = best * (1.f + 2e-5f);
  if (base > reach) return false;
  const float rx = fminf(sqrtf(reach - base) + 4e-6f, 8.f);
  const int xlo = cell_axis(q.x - rx, G), xhi = cell_axis(q.x + rx, G);
  const int x0 = cx - ring, x1 = cx + ring;
  const bool full = (z == cz - ring || z == cz + ring || y == cy - ring || y == cy + ring);
  const int row = (z * G + y) * G;
  if (full) {
    const int a = max(max(x0, 0), xlo), b = min(min(x1, G - 1), xhi);
    if (a > b) return false;
    const int lo = st[row + a], hi = st[row + b + 1];
    nc += (unsigned long long)(hi - lo);
    scan_range(g.cs, cb, lo, hi, q, best, bi);
  } else {
    bool any = false;
    if (x0 >= 0 && x0 >= xlo && x0 <= xhi) {
      const int lo = st[row + x0], hi = st[row + x0 + 1];
      nc += (unsigned long long)(hi - lo);
      scan_range(g.cs, cb, lo, hi, q, best, bi);
      any = true;
    }
    if (x1 <= G - 1 && x1 != x0 && x1 >= xlo && x1 <= xhi) {
      const int lo = st[row + x1], hi = st[row + x1 + 1];
      nc += (unsigned long long)(hi - lo);
      scan_range(g.cs, cb, lo, hi, q, best, bi);
      any = true;
    }
    if (!any) return false;
  }
  return true;
}

// Scan the part of cell row (z, y) that can hold a point at squared distance
// <= best (with the same margins as scan_row): one contiguous range of the
// cell-sorted candidates. Returns whether the row's cell starts were read.
__device__ __forceinline__ bool ball_row(const NnGeom& g, const int* st, long long cb, int z,
                                         int y, float4 q, float h, float& best, int& bi,
                                         unsigned long long& nc) {
  const int G = g.G;
  const float gz = axis_gap(q.z, z, G, h), gy = axis_gap(q.y, y, G, h);
  const float base = gz * gz + gy * gy;
  const float reach = best * (1.f + 2e-5f);
  if (base > reach) return false;
  const float rx = fminf(sqrtf(reach - base) + 4e-6f, 8.f);
  const int xlo = cell_axis(q.x - rx, G), xhi = cell_axis(q.x + rx, G);
  const int row = (z * G + y) * G;
  const int lo = st[row + xlo], hi = st[row + xhi + 1];
  nc += (unsigned long long)(hi - lo);
  scan_range(g.cs, cb, lo, hi, q, best, bi);
  return true;
}

// Cell range [a, b] along one axis that a ball of squared radius best
// (with margins) around v can reach.
__device__ __forceinline__ void ball_axis(float v, float best, int G, int& a, int& b) {
  const float R = fminf(sqrtf(best * (1.f + 2e-5f)) + 8e-6f, 8.f);
  a = cell_axis(v - R, G);
  b = cell_axis(v + R, G);
}

// The seed of query `ob`: its candidate and squared distance, if in range.
__device__ __forceinline__ void seed_start(const NnGeom& g, long long ob, long long cb,
                                           long long ccount, float4 q, float& best, int& bi) {
  if (!g.seeded) return;
  const int sd = g.out_idx[ob];
  if (sd < 0 || sd >= ccount) return;
  const float4 p = g.csrc[cb + sd];
  best = sqdist(q.x, q.y, q.z, p.x, p.y, p.z);
  bi = sd;
}

__device__ __forceinline__ long long set_count(int s, long long uniform, const long long* off) {
  return off == nullptr ? uniform : off[s + 1] - off[s];
}

// Squared lower bound on the distance to any cell outside rings 0..ring
// (FLT_MAX when the rings cover the whole grid).
__device__ __forceinline__ float ring_bound(float4 q, int cx, int cy, int cz, int ring, int G,
                                            float h) {
  const int x0 = cx - ring, x1 = cx + ring, y0 = cy - ring, y1 = cy + ring;
  const int z0 = cz - ring, z1 = cz + ring;
  float lb = FLT_MAX;
  if (x0 > 0) lb = fminf(lb, q.x - fmaf((float)x0, h, -1.f));
  if (x1 < G - 1) lb = fminf(lb, fmaf((float)(x1 + 1), h, -1.f) - q.x);
  if (y0 > 0) lb = fminf(lb, q.y - fmaf((float)y0, h, -1.f));
  if (y1 < G - 1) lb = fminf(lb, fmaf((float)(y1 + 1), h, -1.f) - q.y);
  if (z0 > 0) lb = fminf(lb, q.z - fmaf((float)z0, h, -1.f));
  if (z1 < G - 1) lb = fminf(lb, fmaf((float)(z1 + 1), h, -1.f) - q.z);
  return lb;
}

// true when no unexplored cell can hold a point closer than best
__device__ __forceinline__ bool ring_done(float lb, float best) {
  if (lb == FLT_MAX) return true;
  lb -= 4e-6f;
  return lb > 0.f && best < lb * lb * (1.f - 1e-5f);
}

__device__ __forceinline__ void warp_stats(unsigned long long* stats, unsigned long long nc,
                                           unsigned long long nr) {
  if (!stats) return;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    nc += __shfl_xor_sync(0xffffffffu, nc, o);
    nr += __shfl_xor_sync(0xffffffffu, nr, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(stats, nc);
    atomicAdd(stats + 1, nr);
  }
}

__global__ void __launch_bounds__(128) nn_near_kernel(NnGeom g) {
  const int G = g.G;
  const long long G3 = (long long)G * G * G;
  const float h = 2.f / (float)G;
  unsigned long long n_cand = 0, n_rows = 0;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < g.q_total;
       k += (long long)gridDim.x * blockDim.x) {
    const int s = set_of(k, g.q_uniform, g.q_off, g.nsets);
    const float4 q = g.qs[k];
    const long long cb = set_base(s, g.c_uniform, g.c_off);
    const int* st = g.cstart + s * (G3 + 1);
    const int cx = cell_axis(q.x, G), cy = cell_axis(q.y, G), cz = cell_axis(q.z, G);
    const long long ob = set_base(s, g.q_uniform, g.q_off) + __float_as_int(q.w);
    float best = FLT_MAX;
    int bi = 0x7fffffff;
    bool done = false;
    seed_start(g, ob, cb, set_count(s, g.c_uniform, g.c_off), q, best, bi);
    if (best < FLT_MAX) {
      int za, zb, ya, yb;
      ball_axis(q.z, best, G, za, zb);
      ball_axis(q.y, best, G, ya, yb);
      if ((zb - za + 1) * (yb - ya + 1) <= g.near_rows) {
        for (int z = za; z <= zb; ++z)
          for (int y = ya; y <= yb; ++y)
            n_rows += ball_row(g, st, cb, z, y, q, h, best, bi, n_cand) ? 1 : 0;
        done = true;
      }
    } else {
      for (int ring = 0; ring <= NN_NEAR_RINGS && ring < G; ++ring) {
        for (int z = max(cz - ring, 0); z <= min(cz + ring, G - 1); ++z)
          for (int y = max(cy - ring, 0); y <= min(cy + ring, G - 1); ++y)
            n_rows += scan_row(g, st, cb, z, y, cx, cy, cz, ring, q, h, best, bi, n_cand) ? 1 : 0;
        if (ring_done(ring_bound(q, cx, cy, cz, ring, G, h), best)) {
          done = true;
          break;
        }
      }
    }
    if (done) {
      g.out_idx[ob] = bi;
      if (g.out_d) g.out_d[ob] = best;
    } else {
      const int pos = atomicAdd(g.qcount, 1);
      g.qitems[pos] = make_int4((int)k, __float_as_int(best), bi, 0);
    }
  }
  warp_stats(g.stats, n_cand, n_rows);
}

// ----------------------------------------------------------------- far queries, lane groups
// The queued queries (a seed ball wider than `near_rows` cell rows, or
// no seed and still open after rings 0..1) are served by groups of NN_GROUP
// lanes: a group takes the next item of the queue and deals the cell rows of
// the seed's ball (nearest rows first: the query's own row, then rows
// stepping out in z and y alternately) or of each further ring to its lanes,
// NN_GROUP rows per round, agreeing on the best candidate after every round so
// that later rows are pruned by it. Groups of one warp proceed independently
// (their shuffles name only the group's lanes).
constexpr int NN_GROUP = 8;

// i-th index of [a, b] ordered by distance from c (c, c + 1, c - 1, c + 2, ...).
__device__ __forceinline__ int center_out(int i, int a, int b, int c) {
  const int up = b - c, dn = c - a, m = min(up, dn);
  if (i <= 2 * m) return c + ((i & 1) ? (i + 1) / 2 : -(i / 2));
  return up > dn ? c + (i - m) : c - (i - m);
}

// minimum of (best, index) over the group's lanes, lowest index on ties
__device__ __forceinline__ void group_min(unsigned mask, float& best, int& bi) {
#pragma unroll
  for (int o = NN_GROUP / 2; o > 0; o >>= 1) {
    const float ob = __shfl_xor_sync(mask, best, o);
    const int oi = __shfl_xor_sync(mask, bi, o);
    if (ob < best || (ob == best && oi < bi)) {
      best = ob;
      bi = oi;
    }
  }
}

__global__ void __launch_bounds__(128) nn_far_group_kernel(NnGeom g) {
  const int G = g.G;
  const long long G3 = (long long)G * G * G;
  const float h = 2.f / (float)G;
  const int lane = threadIdx.x & 31, gl = lane & (NN_GROUP - 1);
  const unsigned mask = 0xffu << (lane & ~(NN_GROUP - 1));
  const int nq = *g.qcount;
  unsigned long long n_cand = 0, n_rows = 0;
  while (true) {
    int item = 0;
    if (gl == 0) item = atomicAdd(g.qcount + 1, 1);
    item = __shfl_sync(mask, item, lane & ~(NN_GROUP - 1));
    if (item >= nq) break;
    const int4 it = g.qitems[item];
    const long long k = it.x;
    const int s = set_of(k, g.q_uniform, g.q_off, g.nsets);
    const float4 q = g.qs[k];
    const long long cb = set_base(s, g.c_uniform, g.c_off);
    const int* st = g.cstart + s * (G3 + 1);
    const int cx = cell_axis(q.x, G), cy = cell_axis(q.y, G), cz = cell_axis(q.z, G);
    float best = __int_as_float(it.y);
    int bi = it.z;
    if (best < FLT_MAX) {
      int za, zb, ya, yb;
      ball_axis(q.z, best, G, za, zb);
      ball_axis(q.y, best, G, ya, yb);
      const int ny = yb - ya + 1, nrows = (zb - za + 1) * ny;
      for (int p0 = 0; p0 < nrows; p0 += NN_GROUP) {
        const int p = p0 + gl;
        if (p < nrows) {
          const int z = center_out(p / ny, za, zb, cz), y = center_out(p % ny, ya, yb, cy);
          n_rows += ball_row(g, st, cb, z, y, q, h, best, bi, n_cand) ? 1 : 0;
        }
        group_min(mask, best, bi);
      }
    } else {
      for (int ring = NN_NEAR_RINGS + 1; ring < G; ++ring) {
        const int za = max(cz - ring, 0), zb = min(cz + ring, G - 1);
        const int ya = max(cy - ring, 0), yb = min(cy + ring, G - 1);
        const int ny = yb - ya + 1, nrows = (zb - za + 1) * ny;
        for (int p = gl; p < nrows; p += NN_GROUP) {
          const int z = za + p / ny, y = ya + p % ny;
          n_rows += scan_row(g, st, cb, z, y, cx, cy, cz, ring, q, h, best, bi, n_cand) ? 1 : 0;
        }
        group_min(mask, best, bi);
        if (ring_done(ring_bound(q, cx, cy, cz, ring, G, h), best)) break;
      }
    }
    if (gl == 0) {
      const long long ob = set_base(s, g.q_uniform, g.q_off) + __float_as_int(q.w);
      g.out_idx[ob] = bi;
      if (g.out_d) g.out_d[ob] = best;
    }
  }
  // the work counters: every group has left the loop; reduce over the warp
  __syncwarp();
  warp_stats(g.stats, n_cand, n_rows);
}

cudaError_t launch_nn(const float4* queries_sorted, long long q_uniform, const long long* q_off,
                      int nsets, long long q_total, const Buckets& cand,
                      const long long* c_off, long long c_uniform, int* out_idx, float* out_d,
                      NnQueue queue, cudaStream_t s, unsigned long long* stats,
                      bool seeded) {
  if (q_total == 0) return cudaSuccess;
  NnGeom g{queries_sorted, q_uniform, q_off, nsets, q_total, cand.sorted, cand.cell_start,
           cand.G, c_off, c_uniform, out_idx, out_d, stats, queue.counters, queue.items,
           cand.src, seeded && cand.src != nullptr, queue.near_rows};
  cudaError_t e = cudaMemsetAsync(queue.counters, 0, 2 * sizeof(int), s);
  if (e != cudaSuccess) return e;
  nn_near_kernel<<<grid_blocks(q_total, 128), 128, 0, s>>>(g);
  nn_far_group_kernel<<<queue.far_blocks, 128, 0, s>>>(g);
  return cudaGetLastError();
}

// ----------------------------------------------------------------- loss
// One block per frame, fixed reduction order (deterministic). The squared
// distances are re-formed from the displacement, |(x_i - p_j) + delta_i|^2,
// and the isometry terms from iso_diff, so both keep their relative precision
// when the motion is small; sums in FP64.
__device__ double block_sum(double v, double* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += sh[w];
  __syncthreads();
  return r;
}

__device__ __forceinline__ float resid_sq(float4 x, float4 d, float4 p) {
  const float rx = (x.x - p.x) + d.x, ry = (x.y - p.y) + d.y, rz = (x.z - p.z) + d.z;
  return rx * rx + ry * ry + rz * rz;
}

// Grid (T, LOSS_SPLIT): block (t, b) sums a strided share of frame t; the
// partial sums are combined in a fixed order by loss_final_kernel.
constexpr int LOSS_SPLIT = 8;

__global__ void __launch_bounds__(256) loss_frame_kernel(
    const int* __restrict__ nn_x, const int* __restrict__ nn_p, const long long* __restrict__ off,
    const float4* __restrict__ praw, const float4* __restrict__ xr,
    const float4* __restrict__ disp, const int2* __restrict__ edges, int N, int E, int t_key,
    double* __restrict__ part) {
  __shared__ double sh[32];
  const int t = blockIdx.x;
  const int stride = blockDim.x * LOSS_SPLIT;
  const int first = blockIdx.y * blockDim.x + threadIdx.x;
  const long long b = off[t], e = off[t + 1];
  const float4* Dl = disp + (long long)t * N;
  const float4* Dk = disp + (long long)t_key * N;
  double sx = 0.0, sp = 0.0, si = 0.0;
  for (int i = first; i < N; i += stride)
    sx += (double)resid_sq(xr[i], Dl[i], praw[b + nn_x[(long long)t * N + i]]);
  for (long long j = b + first; j < e; j += stride) {
    const int i = nn_p[j];
    sp += (double)resid_sq(xr[i], Dl[i], praw[j]);
  }
  if (t != t_key) {
    for (int k = first; k < E; k += stride) {
      const int a0 = edges[k].x, b0 = edges[k].y;
      const float4 xa = xr[a0], xb = xr[b0], da = Dl[a0], db = Dl[b0], ka = Dk[a0], kb = Dk[b0];
      float3 et;
      float lt;
      const float df = iso_diff(make_float3(xa.x - xb.x, xa.y - xb.y, xa.z - xb.z),
                                make_float3(da.x - db.x, da.y - db.y, da.z - db.z),
                                make_float3(ka.x - kb.x, ka.y - kb.y, ka.z - kb.z), et, lt);
      si += fabs((double)df);
    }
  }
  sx = block_sum(sx, sh);
  sp = block_sum(sp, sh);
  si = block_sum(si, sh);
  if (threadIdx.x == 0) {
    double* o = part + ((long long)t * LOSS_SPLIT + blockIdx.y) * 3;
    o[0] = sx;
    o[1] = sp;
    o[2] = si;
  }
}

__global__ void loss_combine_kernel(const double* __restrict__ part,
                                    const long long* __restrict__ off, int N, int T,
                                    double* __restrict__ cd, double* __restrict__ iso_t) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= T) return;
  double sx = 0.0, sp = 0.0, si = 0.0;
  for (int b = 0; b < LOSS_SPLIT; ++b) {
    const double* o = part + ((long long)t * LOSS_SPLIT + b) * 3;
    sx += o[0];
    sp += o[1];
    si += o[2];
  }
  cd[t] = sx / (double)N + sp / (double)(off[t + 1] - off[t]);
  iso_t[t] = si;
}

// Eq. 11-12 (cumulative products outward from the keyframe), Eq. 10, 13, 8.
// The per-frame factors (one FP64 power each) are computed in parallel; one
// thread then forms the products outward from the keyframe; the sums use the
// block's fixed-order reduction.
// Variants (the stability ablation): delta_mode NPG_DELTA_* picks the
// catch-up variable, omega_mode NPG_OMEGA_* replaces the cumulative product by
// a direct weight omega(t)^delta; NPG_DELTA_INTERP blends the delta = 1
// weight W(t) as (1 - e~) W(t) + e~.
__global__ void __launch_bounds__(256) loss_final_kernel(
    const double* __restrict__ cd, const double* __restrict__ iso_t, const int* __restrict__ epoch,
    int e_max, int T, int t_key, int E, double w_iso, int delta_mode, int omega_mode,
    double* __restrict__ w, double* __restrict__ loss) {
  __shared__ double sh[32];
  double eb = e_max > 0 ? (double)(*epoch) / (double)e_max : 1.0;
  eb = fmin(fmax(eb, 0.0), 1.0);
  double delta = 1.0 - sqrt(eb);
  if (delta_mode == NPG_DELTA_CONST || delta_mode == NPG_DELTA_INTERP) delta = 1.0;
  if (delta_mode == NPG_DELTA_LINEAR) delta = 1.0 - eb;
  if (delta_mode == NPG_DELTA_EXP) delta = exp(-5.0 * eb);
  const double ck = cd[t_key];
  for (int t = threadIdx.x; t < T; t += blockDim.x) {
    const double ex = cd[t] - ck;
    const double om = omega_mode == NPG_OMEGA_CONST  ? 1.0
                      : omega_mode == NPG_OMEGA_HALF ? 0.5
                                                     : 1.0 / (1.0 + (ex > 0 ? ex : 0.0));
    w[t] = (t == t_key && omega_mode == NPG_OMEGA_CUMULATIVE) ? 1.0 : pow(om, delta);
  }
  __syncthreads();
  if (threadIdx.x == 0 && omega_mode == NPG_OMEGA_CUMULATIVE) {
    for (int t = t_key + 1; t < T; ++t) w[t] *= w[t - 1];
    for (int t = t_key - 1; t >= 0; --t) w[t] *= w[t + 1];
  }
  __syncthreads();
  if (delta_mode == NPG_DELTA_INTERP) {
    for (int t = threadIdx.x; t < T; t += blockDim.x) w[t] = (1.0 - eb) * w[t] + eb;
    __syncthreads();
  }
  double ld = 0.0, li = 0.0;
  for (int t = threadIdx.x; t < T; t += blockDim.x) {
    ld += w[t] * cd[t];
    li += iso_t[t];
  }
  ld = block_sum(ld, sh);
  li = block_sum(li, sh);
  if (threadIdx.x == 0) {
    ld /= (double)T;
    li = E > 0 ? li / ((double)T * (double)E) : 0.0;
    loss[0] = ld + w_iso * li;
    loss[1] = ld;
    loss[2] = li;
  }
}

cudaError_t launch_loss(npg_ctx* c) {
  loss_frame_kernel<<<dim3(c->T, LOSS_SPLIT), 256, 0, c->stream>>>(
      c->nn_x, c->nn_p, c->p_off, c->praw, c->xr, c->disp, c->edges, c->N, c->E, c->t_key,
      c->loss_part);
  loss_combine_kernel<<<(c->T + 127) / 128, 128, 0, c->stream>>>(c->loss_part, c->p_off, c->N,
                                                                 c->T, c->cd, c->iso_t);
  loss_final_kernel<<<1, 256, 0, c->stream>>>(c->cd, c->iso_t, c->d_epoch, c->cfg.e_max,
                                             c->T, c->t_key, c->E, (double)c->cfg.w_iso,
                                             c->cfg.conf_delta, c->cfg.conf_omega, c->wconf,
                                             c->loss);
  return cudaGetLastError();
}

// ----------------------------------------------------------------- dL/dx-hat

// Vertex side of the Chamfer term plus the isometry term (vertex-centric over
// the edge adjacency, no atomics); writes dxhat. The sign of |e_t| - |e_key|
// is 0 at the keyframe (stop-grad reference, d|u|/du at 0 taken as 0).
// The per-frame coefficients of the Chamfer terms of dL/dx-hat, formed once in
// FP64 and rounded to FP32 (the FP64 divisions per row would cost more than
// the rest of the dL/dx-hat kernels: FP64 runs at a small fraction of FP32
// here): coef[t] = w_t / T * 2 / N (vertex side), coef[T + t] = w_t / T * 2 /
// M_t (point side).
__global__ void dx_coef_kernel(const double* __restrict__ w, const long long* __restrict__ off,
                               int N, int T, float* __restrict__ coef) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += gridDim.x * blockDim.x) {
    coef[t] = (float)(w[t] / (double)T * 2.0 / (double)N);
    coef[T + t] = (float)(w[t] / (double)T * 2.0 / (double)(off[t + 1] - off[t]));
  }
}

// ci: the isometry coefficient w_iso / (T E), rounded to FP32.
__global__ void __launch_bounds__(256) dxhat_vertex_kernel(
    const float4* __restrict__ xr, const float4* __restrict__ disp, const int* __restrict__ nn_x,
    const long long* __restrict__ off, const float4* __restrict__ praw,
    const float* __restrict__ coef, const int* __restrict__ adj_off, const int* __restrict__ adj,
    int N, int T, int E, int t_key, float ci, float4* __restrict__ dxhat) {
  const long long total = (long long)N * T;
  for (long long row = (long long)blockIdx.x * blockDim.x + threadIdx.x; row < total;
       row += (long long)gridDim.x * blockDim.x) {
    const int t = (int)(row / N), i = (int)(row - (long long)t * N);
    const float4 xi = xr[i], di = disp[row];
    const float4 p = praw[off[t] + nn_x[row]];
    const float cx = coef[t];
    float gx = cx * ((xi.x - p.x) + di.x), gy = cx * ((xi.y - p.y) + di.y),
          gz = cx * ((xi.z - p.z) + di.z);
    if (E > 0 && t != t_key) {
      const float4* Dl = disp + (long long)t * N;
      const float4* Dk = disp + (long long)t_key * N;
      const float4 ki = Dk[i];
      for (int a = adj_off[i]; a < adj_off[i + 1]; ++a) {
        const int j = adj[a];
        const float4 xj = xr[j], dj = Dl[j], kj = Dk[j];
        // orient as (lower id) - (higher id), the orientation of the edge list
        const float sg = i < j ? 1.f : -1.f;
        float3 et;
        float lt;
        const float df = iso_diff(
            make_float3(sg * (xi.x - xj.x), sg * (xi.y - xj.y), sg * (xi.z - xj.z)),
            make_float3(sg * (di.x - dj.x), sg * (di.y - dj.y), sg * (di.z - dj.z)),
            make_float3(sg * (ki.x - kj.x), sg * (ki.y - kj.y), sg * (ki.z - kj.z)), et, lt);
        if (lt > 0.f && df != 0.f) {
          // d|e_t|/dx_i = sg * e_t / |e_t|
          const float sc = (df > 0.f ? ci : -ci) * sg / lt;
          gx = fmaf(sc, et.x, gx);
          gy = fmaf(sc, et.y, gy);
          gz = fmaf(sc, et.z, gz);
        }
      }
    }
    dxhat[row] = make_float4(gx, gy, gz, 0.f);
  }
}

// Point side of the Chamfer term: every point adds to its nearest vertex.
__global__ void __launch_bounds__(256) dxhat_point_kernel(
    const float4* __restrict__ praw, const long long* __restrict__ off, int T, long long MT,
    const int* __restrict__ nn_p, const float4* __restrict__ xr, const float4* __restrict__ disp,
    const float* __restrict__ coef, int N, float4* __restrict__ dxhat) {
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < MT;
       k += (long long)gridDim.x * blockDim.x) {
    const int t = set_of(k, 0, off, T);
    const float cp = coef[T + t];
    const int i = nn_p[k];
    const float4 p = praw[k];
    const long long row = (long long)t * N + i;
    const float4 x = xr[i], d = disp[row];
    float* g = reinterpret_cast<float*>(dxhat + row);
    atomicAdd(g + 0, cp * ((x.x - p.x) + d.x));
    atomicAdd(g + 1, cp * ((x.y - p.y) + d.y));
    atomicAdd(g + 2, cp * ((x.z - p.z) + d.z));
  }
}

cudaError_t launch_dxhat(npg_ctx* c) {
  const long long rows = (long long)c->N * c->T;
  dx_coef_kernel<<<(c->T + 255) / 256, 256, 0, c->stream>>>(c->wconf, c->p_off, c->N, c->T,
                                                            c->dx_coef);
  const float ci =
      c->E > 0 ? (float)((double)c->cfg.w_iso / ((double)c->T * (double)c->E)) : 0.f;
  dxhat_vertex_kernel<<<grid_blocks(rows, 256), 256, 0, c->stream>>>(
      c->xr, c->disp, c->nn_x, c->p_off, c->praw, c->dx_coef, c->adj_off, c->adj, c->N, c->T,
      c->E, c->t_key, ci, c->dxhat);
  dxhat_point_kernel<<<grid_blocks(c->MT, 256), 256, 0, c->stream>>>(
      c->praw, c->p_off, c->T, c->MT, c->nn_p, c->xr, c->disp, c->dx_coef, c->N, c->dxhat);
  return cudaGetLastError();
}

}  // namespace npg
