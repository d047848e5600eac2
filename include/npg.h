/*
 * npg.h - C ABI of libnpg.so, the GB300 (sm_103a) implementation of one
 * Neu-PiG per-sequence optimisation iteration.
 *
 * One iteration (Sec. 3 of the paper) is
 *   npg_forward   latent-grid lookup at every reference vertex by position and
 *                 normal (Sec. 3.2, Eq. 1), Fourier time encoding (Sec. 3.3,
 *                 Eq. 3), MLP decode of the input vector of Eq. 2 (Eq. 4),
 *                 quaternion / exponential-map rotation and tanh translation
 *                 (Sec. 3.4, Eq. 5-7) -> deformed vertices x-hat for all frames
 *   npg_loss      bidirectional Chamfer nearest neighbours per frame, the
 *                 confidence weights (Eq. 11-12), L_def (Eq. 10), L_iso (Eq. 13)
 *                 and L (Eq. 8)
 *   npg_backward  reverse-mode gradient of L w.r.t. the grids and the MLP
 *   npg_step      Sobolev preconditioner (I + lambda_l L_l)^-2 on every grid
 *                 level (Eq. 9), then Adam with per-level learning rates
 *                 (Sec. 3.5, implementation details); e += 1
 *
 * Conventions shared by every call:
 *   - every function returns NPG_OK (0) or a negative NPG_E* code and never
 *     aborts; npg_last_error() gives a message. A sticky CUDA error makes the
 *     context unusable (every later call returns NPG_ECUDA).
 *   - inputs are copied at npg_create (the caller keeps ownership); outputs go
 *     to caller buffers. "device" pointers are CUDA device (or managed)
 *     addresses on the context's device; "host" pointers are ordinary memory.
 *   - all device work is ordered on cfg.stream (a cudaStream_t; NULL = the
 *     legacy default stream). Calls that return host data synchronize it.
 *   - calls follow forward -> loss -> backward -> step; a call out of order
 *     returns NPG_ESTATE and changes nothing. forward may be repeated at any
 *     point (it restarts the sequence for the current parameters).
 *   - coordinates are expected in [-1, 1]^3 (Sec. 3.4); grid queries outside
 *     are clamped to the boundary.
 */
#ifndef NPG_H
#define NPG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define NPG_API __attribute__((visibility("default")))
#else
#define NPG_API
#endif

#define NPG_MAX_LEVELS 16
#define NPG_MAX_FREQ 8  /* time-encoding frequencies M <= 8 */

/* status codes */
#define NPG_OK 0
#define NPG_EINVAL (-1)   /* bad argument, shape or configuration            */
#define NPG_ENOMEM (-2)   /* device or host allocation failed                */
#define NPG_ECUDA (-3)    /* CUDA runtime / launch error (may be sticky)     */
#define NPG_ESTATE (-4)   /* call out of order                               */
#define NPG_ETIMEOUT (-5) /* a bounded device wait gave up                   */
#define NPG_ENOTIMPL (-6) /* configuration not supported by this build       */

/* rotation parameterisation of the decoder output */
#define NPG_ROT_QUAT 0   /* Eq. 5: q = (1 + o0, o1, o2, o3) / norm, d = o4..6 */
#define NPG_ROT_EXPMAP 1 /* exponential map: omega = o0..2, d = o3..5        */
#define NPG_ROT_CAYLEY 2 /* Cayley transform (I - K)^-1 (I + K), K = [o0..2]x, d = o3..5
                            (the rotation-representation ablation, Sec. 4)  */

/* arithmetic of the preconditioner's DCT passes */
#define NPG_PRECOND_FP32 0
#define NPG_PRECOND_TC 1

/* arithmetic of the MLP decode and its backward pass */
#define NPG_TIME_FOURIER 0
#define NPG_TIME_POLY 1
#define NPG_TIME_GAUSS 2
#define NPG_TIME_LEARNED 3
#define NPG_DELTA_SQRT 0
#define NPG_DELTA_CONST 1
#define NPG_DELTA_LINEAR 2
#define NPG_DELTA_EXP 3
#define NPG_DELTA_INTERP 4
#define NPG_OMEGA_CUMULATIVE 0
#define NPG_OMEGA_CONST 1
#define NPG_OMEGA_HALF 2
#define NPG_OMEGA_SINGLE 3
#define NPG_FP32 0     /* FP32 SIMT                                          */
#define NPG_BF16_MLP 1 /* BF16 operands, FP32 accumulation on tcgen05 tensor cores */

typedef struct npg_ctx npg_ctx; /* opaque; owns all device memory it allocates */

/*
 * Configuration (POD, copied at npg_create).
 *   L, res[l]        position-grid levels and nodes per axis of level l
 *                    (l = 0 coarsest; res >= 2). Nodes sit at -1 + 2k/(r-1).
 *   F_p, F_n, res_n  features per position node (1..32), per normal node
 *                    (1..8), nodes per axis of the normal grid (Sec. 3.2).
 *   H, depth         hidden width and number of hidden layers (Sec. 3.3);
 *                    NPG_FP32 supports H in {16, 32, 64} and multiples of 32
 *                    in (64, 512] (the paper's own network is 512 wide),
 *                    NPG_BF16_MLP H in {64, 128} with depth 3; depth 1..8.
 *   leaky_slope      LeakyReLU negative slope (0 = ReLU).
 *   rot_mode         NPG_ROT_QUAT, NPG_ROT_EXPMAP or NPG_ROT_CAYLEY.
 *   n_freq           Fourier frequencies M (Eq. 3; 1..8).
 *   alpha            translation squashing factor (Eq. 6).
 *   lr_mlp           Adam learning rate of the MLP.
 *   lr_grid[l]       Adam learning rate of level l; lr_grid[L] = normal grid.
 *   lambda[l]        Sobolev smoothing of level l; lambda[L] = normal grid.
 *   adam_*           Adam beta1, beta2, epsilon.
 *   w_iso            isometry weight (Eq. 8).
 *   e_max            iteration count normalising the catch-up variable delta.
 *   precision        NPG_FP32 or NPG_BF16_MLP.
 *   nn_cells         bucket cells per axis of the Chamfer search grids; 0 =
 *                    chosen from the point and vertex counts.
 *   precond_mode     NPG_PRECOND_FP32: the DCT passes of the preconditioner on
 *                    the CUDA cores in FP32; NPG_PRECOND_TC: on tcgen05 tensor
 *                    cores in split BF16 (hi + lo, three products, FP32
 *                    accumulation; ~1e-5 relative) for levels with r >= 24.
 *   use_graph        npg_iteration replays one captured CUDA graph.
 *   time_enc         time encoding gamma(t) (Sec. 3.3 and its ablation, Sec. 4):
 *                    NPG_TIME_FOURIER (Eq. 3, the method), NPG_TIME_POLY
 *                    (t~^j, j = 1..2M), NPG_TIME_GAUSS (sin / cos(2 pi B_j t~)
 *                    with the caller's frequencies time_B[0..M-1], e.g. drawn
 *                    from N(0, 1)), NPG_TIME_LEARNED (gamma(t) = psi_t(t~), a
 *                    two-layer MLP with time_hidden hidden units and the
 *                    decoder's LeakyReLU, trained with the decoder: its
 *                    parameters a, b (time_hidden each; h = act(a t~ + b)), W
 *                    (2M x time_hidden), c (2M; gamma = W h + c) follow the
 *                    decoder's in the MLP vector).
 *   time_hidden      hidden width of psi_t (NPG_TIME_LEARNED; 1..256).
 *   conf_delta       catch-up variable of the confidence weights (Eq. 11-12 and
 *                    the stability ablation): NPG_DELTA_SQRT (1 - sqrt(e~), the
 *                    method), _CONST (1), _LINEAR (1 - e~), _EXP (exp(-5 e~)),
 *                    _INTERP (w = (1 - e~) W(t) + e~, W the weight at delta 1).
 *   conf_omega       temporal weighting: NPG_OMEGA_CUMULATIVE (Eq. 12, the
 *                    method) or a direct w = omega(t)^delta with omega = 1
 *                    (_CONST), 0.5 (_HALF) or 1 / (1 + max(0, cd_t - cd_key))
 *                    (_SINGLE).
 *   stream           cudaStream_t for all device work.
 *   alloc/free/user  optional device allocator (e.g. PyTorch's caching
 *                    allocator); NULL = cudaMalloc / cudaFree. Blocks must be
 *                    16-byte aligned (a misaligned block fails with
 *                    NPG_ENOMEM).
 */
typedef struct npg_config {
  int L;
  int res[NPG_MAX_LEVELS];
  int F_p;
  int F_n;
  int res_n;
  int H;
  int depth;
  float leaky_slope;
  int rot_mode;
  int n_freq;
  float alpha;
  float lr_mlp;
  float lr_grid[NPG_MAX_LEVELS + 1];
  float lambda[NPG_MAX_LEVELS + 1];
  float adam_beta1;
  float adam_beta2;
  float adam_eps;
  float w_iso;
  int e_max;
  int precision;
  int nn_cells;
  int precond_mode;
  int use_graph;
  void* stream;
  void* (*alloc)(size_t bytes, void* user);
  void (*free)(void* ptr, void* user);
  void* alloc_user;
  int time_enc;
  float time_B[NPG_MAX_FREQ];
  int conf_delta;
  int conf_omega;
  int time_hidden;
} npg_config;

/* Paper defaults (Sec. 3.2-3.5): resolutions r_l = round(r_min + (r_max -
 * r_min)(l-1)/(L-1)), F_n = 2, res_n = 4, LeakyReLU 0.01, quaternions, M = 4,
 * alpha = 0.1, lr_mlp = 1e-3, lr_l = 0.005 * 2.5^(l-1), lambda_l = 0.4 *
 * 1.5^(l-1) (l = 1 coarsest; the normal grid takes the level-1 values), Adam
 * (0.9, 0.999, 1e-8), w_iso = 100, e_max = 1000, FP32, Fourier time encoding,
 * the cumulative confidence weights with delta = 1 - sqrt(e~). */
NPG_API int npg_config_default(npg_config* cfg, int L, int r_min, int r_max, int F_p, int H, int depth);

/*
 * Create a context for one sequence (Sec. 3, problem statement).
 *   ref_xyz, ref_nrm  N x 3 FP32: keyframe reference vertices and unit normals.
 *   faces             F_tri x 3 int32 triangles; the isometry edges are the
 *                     unique undirected edges of these faces.
 *   points            sum_t M_t x 3 FP32, the T clouds concatenated in frame order;
 *   frame_offsets     T + 1 int64, frame t owns points [off[t], off[t+1]);
 *                     every frame needs M_t >= 1.
 *   t_key             keyframe index, 0-based.
 *   mlp_init          flat FP32 MLP parameters (mlp_len floats): layer 0 W
 *                     (H x K, row-major, K = F_n + F_p + 2 n_freq, input order
 *                     (z_n, z_p, gamma)) then b (H); hidden layers W (H x H) + b;
 *                     output W (O x H) + b, O = 7 (quaternion) or 6
 *                     (exponential map); with NPG_TIME_LEARNED the parameters
 *                     of psi_t after those. Zeroing the output layer gives the
 *                     identity initialisation of Sec. 3.1.
 *   inputs_on_device  0: every input pointer is host memory; 1: device memory.
 * Grids and Adam moments start at zero, e = 0. On failure *out is NULL.
 */
NPG_API int npg_create(npg_ctx** out, const npg_config* cfg, const float* ref_xyz, const float* ref_nrm,
               int N, const int32_t* faces, int F_tri, const float* points,
               const int64_t* frame_offsets, int T, int t_key, const float* mlp_init,
               size_t mlp_len, int inputs_on_device);

/* Deformed vertices for every frame. xhat_out: nullable device pointer to
 * T x N x 3 FP32 (frame-major) that receives a copy. */
NPG_API int npg_forward(npg_ctx* ctx, float* xhat_out);

/* Chamfer nearest neighbours, cd_t, w_conf(t), L_def, L_iso and L for the last
 * forward pass. loss_out (host, nullable): 3 doubles {L, L_def, L_iso};
 * cd_out (host, nullable): T doubles. Non-null outputs synchronize the stream. */
NPG_API int npg_loss(npg_ctx* ctx, double* loss_out, double* cd_out);

/* Gradient of L w.r.t. every grid value and MLP parameter (stop-grad on
 * w_conf and on the keyframe edge lengths, as Eq. 11-13 prescribe). */
NPG_API int npg_backward(npg_ctx* ctx);

/* Reverse pass from a given dL/dx-hat: back through Eq. 7-5, the MLP, the
 * input vector (Eq. 2) and the grid lookups (Eq. 1) into the parameter
 * gradients, as npg_backward does after forming dL/dx-hat from the loss.
 * dxhat: nullable device pointer to T x N x 3 FP32 (frame-major); NULL reuses
 * the dL/dx-hat of the last npg_backward. Needs a preceding npg_forward; the
 * next call may be npg_step. Lets a caller differentiate its own loss of x-hat. */
NPG_API int npg_backprop(npg_ctx* ctx, const float* dxhat);

/* Eq. 9 preconditioner on every grid level, then Adam (step e + 1); e += 1. */
NPG_API int npg_step(npg_ctx* ctx);

/* forward + loss + backward + step. loss_out (host, nullable): 3 doubles
 * {L, L_def, L_iso} of this iteration (synchronizes). With cfg.use_graph the
 * four calls are captured once into a CUDA graph and replayed. */
NPG_API int npg_iteration(npg_ctx* ctx, double* loss_out);

/*
 * Reconstruction quality (the evaluation metrics of Sec. 4) of the x-hat of
 * the last npg_forward against ground-truth vertex positions gt_xyz (T x N x 3
 * FP32, host or device per on_device, the reference mesh's connectivity, so
 * vertex i of every frame is the same material point). Per frame t:
 *   cd        mean_i min_j |x_i - g_j|^2 + mean_j min_i |g_j - x_i|^2
 *   precision fraction of x_i with min_j |x_i - g_j| < tau, recall likewise
 *             for g_j, fscore = 2 P R / (P + R) (0 when both are 0)
 *   nc        (mean_i |n_i . n_g(nn(i))| + mean_j |n_g,j . n(nn(j))|) / 2 with
 *             area-weighted vertex normals
 *   corr      mean_i |x_i - g_i| (correspondence error along trajectories)
 * tau = tau_rel x the diagonal of frame t's ground-truth bounding box (the
 * paper's F-score threshold is 0.5%: tau_rel = 0.005). The paper names these
 * metrics without formulas; the definitions above are this library's reading.
 * out (host): (T + 1) x 6 doubles {cd, precision, recall, fscore, nc, corr}
 * per frame, then their mean over frames. Allocates its scratch with
 * cudaMallocAsync on the context's stream and synchronizes.
 */
NPG_API int npg_evaluate(npg_ctx* ctx, const float* gt_xyz, int on_device, float tau_rel,
                         double* out);

/*
 * Batch of independent sequences (many sequences of uneven vertex, frame and
 * point counts optimised together). The caller creates one context per
 * sequence with npg_create, each with its own non-default stream, distinct
 * from the others and from `stream`; the batch does not own them (destroy the
 * batch first). npg_batch_iteration runs one iteration (forward, loss,
 * backward, step) of every sequence: the first call runs them eagerly and
 * captures the next iteration of all of them into one CUDA graph, in which
 * every sequence is a branch forked from and joined back to `stream`, so
 * small sequences share the GPU; later calls replay it. Each context's
 * stream is ordered after the batch iteration (the contexts stay usable with
 * the single-sequence calls, which reset nothing in the batch). loss_out
 * (host, nullable): S x 3 doubles {L, L_def, L_iso} per sequence of this
 * iteration (synchronizes). A context may belong to one batch at a time.
 */
typedef struct npg_batch npg_batch;
NPG_API int npg_batch_create(npg_batch** out, int S, npg_ctx* const* ctxs, void* stream);
NPG_API int npg_batch_iteration(npg_batch* batch, double* loss_out);
/* Concurrency of the batch graph: the sequences form `width` chains, the
 * sequences of one chain run one after the other, the chains concurrently.
 * Sequences go largest first (work N T + M T) onto the chain with the least
 * work so far. width 0 (the default) or >= S: every sequence its own branch;
 * width 1: all of them in sequence (no contention for the GPU between
 * sequences that each fill it). Call before the first npg_batch_iteration
 * (NPG_EINVAL once the graph is captured); negative values count as 0. */
NPG_API int npg_batch_set_width(npg_batch* batch, int width);
/* NULL is allowed. Leaves the contexts alive. */
NPG_API int npg_batch_destroy(npg_batch* batch);

/* Replace the point clouds (same T; per-frame counts may change, total at most
 * the count given at create). on_device as for npg_create. Resets the call
 * order to "before forward". */
NPG_API int npg_set_points(npg_ctx* ctx, const float* points, const int64_t* frame_offsets, int on_device);

/* Buffers readable with npg_get (and writable with npg_set where marked). Grid
 * vectors use the flat layout: levels 0..L-1 then the normal grid; level l is
 * res^3 x F with node (ix,iy,iz) at ((iz r + iy) r + ix) and features innermost.
 * The nearest-neighbour buffers also seed the next search: each search starts
 * from the index already stored for its query (the previous result, -1 after
 * create) and only visits the cells within that candidate's distance. Any
 * value may be written; an index outside the candidate set means no seed. The
 * search result is the exact nearest neighbour whatever the seeds. */
#define NPG_BUF_GRID 0        /* FP32 grid values (settable)                 */
#define NPG_BUF_MLP 1         /* FP32 MLP parameters (settable)              */
#define NPG_BUF_GRID_GRAD 2   /* FP32 dL/dgrid of the last backward           */
#define NPG_BUF_GRID_PC 3     /* FP32 preconditioned grid gradient of the last step */
#define NPG_BUF_MLP_GRAD 4    /* FP32 dL/dmlp of the last backward            */
#define NPG_BUF_XHAT 5        /* FP32 T x N x 3                              */
#define NPG_BUF_NN_X 6        /* int32 T x N: nearest point (frame-local index) (settable) */
#define NPG_BUF_NN_P 7        /* int32 sum M_t: nearest vertex of every point (settable) */
#define NPG_BUF_CD 8          /* FP64 T                                      */
#define NPG_BUF_WCONF 9       /* FP64 T                                      */
#define NPG_BUF_ADAM_M_GRID 10 /* FP32, grid layout (settable)               */
#define NPG_BUF_ADAM_V_GRID 11 /* FP32, grid layout (settable)               */
#define NPG_BUF_ADAM_M_MLP 12  /* FP32 (settable)                            */
#define NPG_BUF_ADAM_V_MLP 13  /* FP32 (settable)                            */
#define NPG_BUF_DIST_X 14     /* FP32 T x N squared NN distances             */
#define NPG_BUF_DIST_P 15     /* FP32 sum M_t squared NN distances           */
#define NPG_BUF_DXHAT 16      /* FP32 T x N x 3 dL/dx-hat of the last backward */
#define NPG_BUF_DISP 17       /* FP32 T x N x 3 displacement x-hat - x of the last forward,
                                 formed directly as (R - I) x + d-hat (keeps its relative
                                 precision when the motion is small) */
#define NPG_BUF_DEVICE_ERROR 18 /* int32 (one value): the device error word that a kernel
                                 sets when one of its bounded waits gives up. Nonzero
                                 makes the next call that synchronises return
                                 NPG_ETIMEOUT (and clears it); npg_get reads it without
                                 clearing. Settable (e.g. to 0, or to nonzero to exercise
                                 a caller's own error handling). */

/* Size in bytes of a buffer (0 for an unknown id). */
NPG_API size_t npg_size(const npg_ctx* ctx, int which);
/* Copy a buffer out (dst host or device per dst_on_device; bytes must equal
 * npg_size). Synchronizes the stream. */
NPG_API int npg_get(npg_ctx* ctx, int which, void* dst, size_t bytes, int dst_on_device);
/* Overwrite a settable buffer (bytes must equal npg_size); resets the call order. */
NPG_API int npg_set(npg_ctx* ctx, int which, const void* src, size_t bytes, int src_on_device);
/* Iteration counter e (0-based index of the next iteration). */
NPG_API int npg_get_epoch(const npg_ctx* ctx);
NPG_API int npg_set_epoch(npg_ctx* ctx, int e);

/* Checkpoint: grids, MLP, Adam moments and e as one host blob. With blob ==
 * NULL, *bytes receives the size. npg_set_state restores it exactly. */
NPG_API int npg_get_state(npg_ctx* ctx, void* blob, size_t* bytes);
NPG_API int npg_set_state(npg_ctx* ctx, const void* blob, size_t bytes);

/* Per-stage device timing (CUDA events on cfg.stream) of eager iterations.
 * npg_timing(ctx, n) keeps event sets for the next n iterations (n = 0 turns
 * timing off and frees them); npg_timing_read synchronizes and returns, for
 * one stage, the summed milliseconds and the number of iterations measured
 * since timing was enabled. Graph replays are not timed per stage. */
#define NPG_STAGE_ENCODE 0   /* grid lookup, level mean, first layer, time modulation */
#define NPG_STAGE_DECODE 1   /* MLP decode + rigid transform                        */
#define NPG_STAGE_BUCKET 2   /* counting sort of x-hat into the search cells         */
#define NPG_STAGE_NN_X 3     /* nearest point of every vertex                       */
#define NPG_STAGE_NN_P 4     /* nearest vertex of every point                       */
#define NPG_STAGE_LOSS 5     /* keyframe edge lengths, cd_t, w_conf, L              */
#define NPG_STAGE_DXHAT 6    /* dL/dx-hat                                           */
#define NPG_STAGE_MLP_BWD 7  /* MLP backward with forward recompute                 */
#define NPG_STAGE_SCATTER 8  /* grid gradient                                       */
#define NPG_STAGE_PRECOND 9  /* Sobolev preconditioner, all levels                  */
#define NPG_STAGE_ADAM 10    /* Adam, all parameters                                */
#define NPG_NUM_STAGES 11
NPG_API int npg_timing(npg_ctx* ctx, int n_iters);
NPG_API int npg_timing_read(npg_ctx* ctx, int stage, double* total_ms, int* n_iters);

/* Work counters of the nearest-neighbour search, summed over the iterations
 * timed since the last npg_timing call: out4 = {candidate pairs evaluated and
 * cell rows visited, vertex -> point; the same, point -> vertex}. */
NPG_API int npg_search_stats(npg_ctx* ctx, long long* out4);

/* Number of kernels this context has launched (graph replays count every
 * kernel node they contain). */
NPG_API long long npg_launch_count(const npg_ctx* ctx);

/*
 * Autotuner of the context's launch shapes (one of the batching tools: each
 * sequence of a batch gets the shapes that suit its sizes). It times `reps`
 * forward (+ loss) passes, after one warm-up, for each candidate and keeps the
 * fastest: the bucket cells per axis of the vertex-side and then of the
 * point-side search grid (the default resolution times 0.7, 0.85, 1, 1.25;
 * the search is exact at every resolution), the widest seed ball (6, 12, 24,
 * 48, 96, 192 or 384 cell rows) that one thread covers before a query of each search
 * direction goes to the lane-group pass, then, for the BF16 form with H = 64,
 * the decode's CTAs per SM (3, 4, 6 or 8). Parameters, Adam state and
 * e are unchanged; the nearest-neighbour buffers hold the last search's
 * (exact) results; the call order restarts before forward, and a captured
 * iteration graph is captured again at the next npg_iteration.
 * chosen (host, nullable): 5 ints {vertex-side cells, point-side cells,
 * decode CTAs per SM, ball rows per thread for vertex -> point, and for point
 * -> vertex}. NPG_EINVAL if cfg.nn_cells fixes the cells. Synchronizes.
 */
NPG_API int npg_autotune(npg_ctx* ctx, int reps, int* chosen);

/* Release everything the context owns; NULL is allowed. */
NPG_API int npg_destroy(npg_ctx* ctx);

/* Message of the last failure on ctx (or of the calling thread when ctx is NULL). */
NPG_API const char* npg_last_error(const npg_ctx* ctx);

/*
 * Standalone exact nearest neighbours (the Chamfer search of Sec. 3.5, one
 * point set). For each of nq queries q[i] the index of the closest of the nc
 * candidates c[j] in squared Euclidean distance, formed in FP32 as
 * d = dx*dx; d = fma(dy,dy,d); d = fma(dz,dz,d); ties go to the lowest index.
 * All pointers are device pointers: q (nq x 3 FP32), c (nc x 3 FP32), idx
 * (nq int32), dist (nq FP32, nullable). cells = bucket cells per axis (0 =
 * automatic). Allocates its bucket scratch with cudaMallocAsync on stream and
 * frees it before returning. nq >= 0, nc >= 1.
 */
NPG_API int npg_nearest(const float* q, int nq, const float* c, int nc, int32_t* idx, float* dist,
                int cells, void* stream);

/*
 * Keyframe selection (Sec. 3.1, Initialization): every frame's point cloud is
 * rated by its spatial extent, weighted toward the temporal midpoint, and the
 * best-rated frame is returned as t_key (the frame whose cloud the caller
 * turns into the reference mesh). The paper defers the formula to an earlier
 * method; this library's reading:
 *   e_t = sqrt(mean_j |p_j - c_t|^2), c_t = mean_j p_j   (RMS radius, FP64)
 *   w_t = 1 - bias |t / (T - 1) - 1/2|                   (T = 1: t_key = 0)
 *   t_key = argmax_t w_t e_t, the lowest t on ties.
 * points: concatenated clouds, frame_offsets[T] x 3 FP32; frame_offsets: T + 1
 * int64, frame_offsets[0] = 0, every frame non-empty. Both are device pointers
 * when on_device, else host pointers; the caller keeps them. 0 <= bias <= 1.
 * extent_out (host, T doubles, nullable) receives e_t, t_key_out (host) the
 * choice. Allocates its scratch with cudaMallocAsync on stream and
 * synchronizes the stream before returning. Bad arguments and invalid offsets
 * return NPG_EINVAL before any device work.
 */
NPG_API int npg_select_keyframe(const float* points, const int64_t* frame_offsets, int T,
                                int on_device, double bias, double* extent_out, int* t_key_out,
                                void* stream);

/*
 * Standalone Sobolev preconditioner (Eq. 9) of one r^3 x F block:
 * out = (I + lambda L)^-2 g per channel, L the 6-neighbour lattice Laplacian
 * with natural (Neumann) boundary. g and out are device pointers (r^3 x F
 * FP32, node-major, features innermost; they may alias). 2 <= r <= 512,
 * 1 <= F <= 32. Allocates its transform scratch with cudaMallocAsync on
 * stream and frees it before returning.
 */
NPG_API int npg_precondition(const float* g, float* out, int r, int F, float lambda, void* stream);

/* npg_precondition with the DCT passes on the tensor cores (split BF16, FP32
 * accumulation, ~1e-5 relative error): same arguments, layout and errors;
 * 2 <= r <= 256. Allocates its scratch and tables with cudaMallocAsync on
 * stream and frees them before returning. */
NPG_API int npg_precondition_tc(const float* g, float* out, int r, int F, float lambda,
                                void* stream);

/*
 * Allocation-free variant of npg_precondition (the paper has no counterpart:
 * this is a deployment convenience). Some callers cannot allocate device
 * memory where they need the preconditioner: a process whose GPU memory is
 * already owned by another allocator (a framework's caching pool that has
 * reserved the device), a loop with a fixed memory budget, or code that must
 * not risk the implicit device synchronisation of cudaMalloc / cudaFree. This
 * entry point takes the same arguments and gives the same result as
 * npg_precondition, but allocates and frees nothing: its scratch is one
 * file-scope device array of about 8.5 MB that every GPU which loads
 * libnpg.so holds until the process exits.
 *   - Limit: r^3 * F <= 1,048,576, hence r <= 101 (e.g. r = 64 with F = 4,
 *     r = 101 with F = 1); larger blocks return NPG_EINVAL (use
 *     npg_precondition).
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current and keeps it for the
 *     rest of the process; make that first call before any stream capture,
 *     and do not call this entry point again after a cudaDeviceReset of that
 *     device (the kept address would be stale).
 *   - The work is queued on stream and not waited for.
 *   - Every call shares the one array. Calls whose work overlaps on the GPU
 *     (different streams or host threads without ordering) race and corrupt
 *     each other's results: order them, e.g. on one stream.
 */
NPG_API int npg_precondition_static(const float* g, float* out, int r, int F, float lambda,
                                    void* stream);

/*
 * Measurement helper (no counterpart in the paper): the FP32 FMA rate of the
 * current device, the peak against which the plain-FP32 stages are placed.
 * Launches a kernel of 16 independent FMA chains per thread on 8 x 256
 * threads per SM (one untimed warm-up launch, one launch timed with CUDA
 * events on stream) and returns *tflops = 2 x FMAs / time in TFLOP/s and
 * *ms_out (nullable) the timed launch's milliseconds. Allocates 1.2 MB of
 * output with cudaMallocAsync on stream and synchronizes it.
 */
NPG_API int npg_fp32_fma_rate(double* tflops, double* ms_out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* NPG_H */
