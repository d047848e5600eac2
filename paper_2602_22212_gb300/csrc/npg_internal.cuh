// Internal declarations shared by the libnpg.so translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/npg.h"

#define NPG_MAX_F 32
#define NPG_MAX_FN 8
#define NPG_MAX_Z (NPG_MAX_F + NPG_MAX_FN)
#define NPG_MAX_K (NPG_MAX_Z + 2 * NPG_MAX_FREQ)
#define NPG_MAX_DEPTH 8

namespace npg {

// One grid block: a position level (l < L) or the normal grid (l == L).
struct Level {
  int r;           // nodes per axis
  int F;           // features per node
  long long off;   // float offset in the device grid vector (256-byte aligned)
  long long flat;  // float offset in the flat (unpadded) layout
  long long n;     // r^3 * F
  float lr;        // Adam learning rate
  float lambda;    // Sobolev smoothing
};

// Bucket grid over [-1, 1]^3 used by the exact nearest-neighbour search.
struct Buckets {
  int G = 0;                // cells per axis
  int nsets = 0;            // number of independent point sets (frames)
  int* cell_start = nullptr;  // nsets x (G^3 + 1), set-local offsets
  int* counts = nullptr;      // nsets x G^3 scratch
  int* slot = nullptr;        // per point: rank within its cell
  float4* sorted = nullptr;   // per point, in cell order: (x, y, z, bits(local index))
  const float4* src = nullptr;  // the points in their own order (set by bucket_build)
};

// Work queue of the far-query pass of the nearest-neighbour search.
struct NnQueue {
  int* counters = nullptr;  // 2 ints: pushed, popped
  int4* items = nullptr;    // capacity >= number of queries
  int far_blocks = 1;
  int near_rows = 12;       // seed balls of up to this many cell rows stay in pass 1
};

struct MlpDims {
  int H, D, K, Z, NO, M;  // hidden width, hidden layers, first-layer inputs, latent, outputs, freqs
  float slope;
  int Ht;                 // hidden width of the learned time embedding (0: a fixed encoding)
  long long dec_len;      // decoder parameters; psi_t's follow them
};

}  // namespace npg

struct npg_ctx {
  npg_config cfg;
  // tunable launch shapes (npg_autotune): bucket cells per axis of the two
  // search grids are pb.G / xb.G below; CTAs per SM of the BF16 decode
  int dec_per_sm = 6;
  int G_cap_p = 0, G_cap_x = 0;  // the bucket arrays hold up to this many cells per axis
  cudaStream_t stream = nullptr;
  int dev = 0;
  int N = 0, T = 0, t_key = 0, E = 0;
  long long MT = 0, MT_cap = 0;
  npg::MlpDims md;
  int nlev = 0;  // L + 1
  npg::Level lev[NPG_MAX_LEVELS + 1];
  long long grid_dev_len = 0;   // padded
  long long grid_flat_len = 0;  // oracle-compatible
  long long mlp_len = 0;
  int max_r = 0;
  long long max_level_n = 0;

  // constant inputs
  float4* xr = nullptr;       // N reference vertices (w = 0)
  float4* nr = nullptr;       // N unit normals
  int* adj_off = nullptr;     // N + 1
  int* adj = nullptr;         // 2E neighbour vertex ids
  int* adj_edge = nullptr;    // 2E edge ids
  int2* edges = nullptr;      // E (a < b)
  long long* p_off = nullptr; // T + 1 (device)
  long long* h_off = nullptr; // T + 1 (host copy)
  float4* praw = nullptr;     // MT_cap points in input order (w = 0)
  npg::Buckets pb;            // static point buckets
  npg::Buckets xb;            // per-iteration x-hat buckets

  // per-iteration buffers
  float* z = nullptr;      // N x Z
  float* U = nullptr;      // N x H
  float* V = nullptr;      // T x H
  float* gamma = nullptr;  // T x 2M time encoding gamma(t)
  float4* xhat = nullptr;  // T x N deformed vertices
  float4* disp = nullptr;  // T x N displacements x-hat - x
  float4* dxhat = nullptr; // T x N
  int* nn_x = nullptr;     // T x N
  float* d_x = nullptr;    // T x N
  int* nn_p = nullptr;     // MT
  float* d_p = nullptr;    // MT
  float* dz = nullptr;     // N x Z
  double* cd = nullptr;    // T
  double* wconf = nullptr; // T
  double* iso_t = nullptr; // T
  double* loss_part = nullptr;  // T x 8 x 3 partial sums
  float* dx_coef = nullptr;  // 2 T: per-frame Chamfer coefficients of dL/dx-hat (vertex, point)
  double* loss = nullptr;  // 3: L, L_def, L_iso
  double* h_loss = nullptr;  // pinned host mirror (3 + T)

  // parameters, gradients, optimiser state
  float* grid = nullptr;
  float* g_grid = nullptr;
  float* g_pc = nullptr;
  float* m_grid = nullptr;
  float* v_grid = nullptr;
  float* mlp = nullptr;
  float* g_mlp = nullptr;
  float* m_mlp = nullptr;
  float* v_mlp = nullptr;
  float* mlp_bf16 = nullptr;  // packed tensor-core weights (BF16 path)
  float* dV = nullptr;        // T x H: sum over vertices of dL/d(first-layer pre-activation)
                              // (learned time embedding)
  float* wide = nullptr;      // FP32 path with H > 64: per-chunk activations and gradients
  long long wide_rows = 0;    // rows per chunk of that path

  // preconditioner tables and scratch
  float* dct = nullptr;          // per level: C (r x r) then C^T (r x r) then mu (r)
  long long dct_off[NPG_MAX_LEVELS + 1];
  uint16_t* dct_tc = nullptr;     // split BF16 tables per level: C then C^T (hi, lo each)
  long long dct_tc_off[NPG_MAX_LEVELS + 1][2];
  float* pc_tmp0 = nullptr;
  float* pc_tmp1 = nullptr;

  // Stream lanes: the grid levels' preconditioner + Adam, and the two search
  // directions, run concurrently on the main stream (lane 0) and auxiliary
  // streams forked from it and joined back (also inside a captured graph).
  static constexpr int NLANE = 4;
  cudaStream_t lane[NLANE] = {};   // lane[0] = stream
  cudaEvent_t ev_fork = nullptr;
  cudaEvent_t ev_join[NLANE] = {};
  float* lane_tmp[NLANE][2] = {};  // preconditioner scratch of each lane
  int level_lane[NPG_MAX_LEVELS + 1] = {};

  // per-stage timing (event ring) and launch accounting
  cudaEvent_t* tev = nullptr;  // t_slots x (NPG_NUM_STAGES + 1)
  unsigned* t_mask = nullptr;  // per slot: which marks were recorded
  int t_slots = 0, t_next = 0, t_cur = -1;
  int capturing = 0;
  long long launches = 0;
  unsigned long long* d_nnstats = nullptr;  // per direction: candidates, cell rows (timing mode)
  npg::NnQueue nnq;    // vertex -> point search
  npg::NnQueue nnq_p;  // point -> vertex search (runs concurrently)
  long long graph_launches = 0;  // kernels in one replay of the captured graph
  int* d_epoch = nullptr;  // device copy of e (read by graph-captured kernels)
  float* d_adam_c = nullptr;  // 1 - beta1^s, 1 - beta2^s of the current step
  int* d_err = nullptr;       // set by a kernel whose bounded wait gave up
  float* xhat3 = nullptr;     // T x N x 3 staging for npg_get
  void* allocs[128];
  int n_allocs = 0;
  int phase = 0;  // 0 ready, 1 forward done, 2 loss done, 3 backward done
  int e = 0;
  int sticky = 0;
  int num_sms = 0;
  cudaGraphExec_t graph_exec = nullptr;
  cudaGraph_t graph = nullptr;
  std::string err;
  // evaluation metrics: faces (host copy) and, once built, their device form
  std::vector<int32_t> faces_h;
  int3* d_faces = nullptr;
  int* d_vf_off = nullptr;  // vertex -> incident faces, CSR
  int* d_vf = nullptr;
};

namespace npg {

// kernels (launchers return cudaGetLastError())
cudaError_t launch_encode(npg_ctx* c);
cudaError_t launch_time_table(npg_ctx* c);
cudaError_t launch_time_mod(npg_ctx* c);
// learned time embedding: gamma from psi_t's parameters; the reverse pass from dV
cudaError_t launch_learned_time(npg_ctx* c);
cudaError_t launch_learned_time_backward(npg_ctx* c);
cudaError_t launch_decode_fp32(npg_ctx* c);
cudaError_t launch_decode_bf16(npg_ctx* c);
cudaError_t launch_decode_bf16_h128(npg_ctx* c);

cudaError_t bucket_build(const float4* pts, const long long* d_off, long long uniform_count,
                         int nsets, long long total, int G, Buckets& b, cudaStream_t s);
cudaError_t launch_nn(const float4* queries_sorted, long long q_uniform, const long long* q_off,
                      int nsets, long long q_total, const Buckets& cand,
                      const long long* c_off, long long c_uniform, int* out_idx, float* out_d,
                      NnQueue queue, cudaStream_t s, unsigned long long* stats = nullptr,
                      bool seeded = false);
cudaError_t launch_loss(npg_ctx* c);
cudaError_t launch_dxhat(npg_ctx* c);
cudaError_t launch_mlp_backward_fp32(npg_ctx* c);
// FP32 MLP for hidden widths beyond 64 (k_mlp_fp32_wide.cu): rows in chunks of
// at most WIDE_CHUNK, layer by layer through a scratch area of
// wide_fp32_scratch_floats() floats (c->wide, c->wide_rows rows per chunk).
constexpr long long WIDE_CHUNK = 262144;
bool wide_fp32_supported(int H);
long long wide_fp32_scratch_floats(int H, int D, int K, long long rows, long long* chunk_rows);
cudaError_t launch_decode_fp32_wide(npg_ctx* c);
cudaError_t launch_mlp_backward_fp32_wide(npg_ctx* c);
cudaError_t launch_mlp_backward_bf16(npg_ctx* c);
cudaError_t launch_mlp_backward_bf16_h128(npg_ctx* c);
cudaError_t launch_mlp_backward_bf16_h64(npg_ctx* c);
cudaError_t launch_scatter(npg_ctx* c);
cudaError_t launch_precondition(const float* g, float* out, float* tmp0, float* tmp1,
                                const float* C, const float* Ct, const float* mu, int r, int F,
                                float lambda, cudaStream_t s);
cudaError_t launch_adam(float* p, const float* g, float* m, float* v, long long n, float lr,
                        float b1, float b2, float eps, const float* cc, cudaStream_t s);
cudaError_t launch_step_prepare(const int* epoch, float b1, float b2, float* cc, cudaStream_t s);
cudaError_t launch_step_finish(int* epoch, cudaStream_t s);
void dct_tables(int r, float* C, float* Ct, float* mu);
size_t dct_tc_table_elems(int r);
// Scratch (floats, per buffer) the tensor-core preconditioner needs for an
// r^3 x F level: its split hi / lo intermediates with padded rows.
size_t dct_tc_scratch_elems(int r, int F);
void dct_tc_tables(int r, const float* Mx, uint16_t* dst);
// One Adam step of one parameter (Sec. 3.5: Adam on the preconditioned
// gradient), bias corrections c1 = 1 - b1^s, c2 = 1 - b2^s of step s; shared
// by the scalar and the float4 Adam kernels.
__device__ __forceinline__ void adam_update(float g, float& m, float& v, float& p, float lr,
                                            float b1, float b2, float eps, float c1, float c2) {
  m = fmaf(b1, m, (1.f - b1) * g);
  v = fmaf(b2, v, (1.f - b2) * g * g);
  p -= lr * (m / c1) / (sqrtf(v / c2) + eps);
}

cudaError_t launch_precondition_tc(const float* g, float* out, float* t0, float* t1,
                                   const uint16_t* tabC, const uint16_t* tabCt, const float* mu,
                                   int r, int F, float lambda, int* err, cudaStream_t s);
constexpr int PRECOND_TC_MIN_R = 24;
cudaError_t launch_points_to_float4(const float* src, float4* dst, long long n, cudaStream_t s);
cudaError_t launch_xhat_out(const float4* xhat, float* out, long long n, cudaStream_t s);

int auto_cells(long long points_per_set, int nsets);

// evaluation metrics (k_eval.cu)
cudaError_t launch_eval_normals(const float4* v, const int3* faces, const int* vf_off,
                                const int* vf, int N, long long NT, float4* nrm, cudaStream_t s);
cudaError_t launch_eval_tau(const float4* g, int N, int T, float tau_rel, float* tau2,
                            cudaStream_t s);
cudaError_t launch_eval_frames(const float4* x, const float4* g, const float4* nx,
                               const float4* ng, const int* idx_x, const float* d_x,
                               const int* idx_g, const float* d_g, const float* tau2, int N,
                               int T, double* part, cudaStream_t s);
cudaError_t launch_keyframe_extent(const float* pts, const long long* off, int T, double* extent,
                                   cudaStream_t s);
int eval_split();
int eval_terms();
// records a message for npg_last_error(NULL) and returns code
int set_error_message(int code, const char* fmt, ...);
bool decode_fp32_supported(int H, int D);
bool decode_bf16_supported(int H, int D);
bool backward_bf16_supported(int K, int Z);
size_t mlp_bwd_fp32_smem(const MlpDims& md);

}  // namespace npg
