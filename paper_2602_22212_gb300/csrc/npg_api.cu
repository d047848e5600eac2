// C ABI of libnpg.so (declared in include/npg.h): context lifetime, argument
// validation, device buffers, and the order of kernel launches for one
// Neu-PiG iteration (Sec. 3.2-3.5).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <utility>
#include <vector>

#include "npg_internal.cuh"

using namespace npg;

static thread_local std::string g_thread_err;

static int set_err(npg_ctx* c, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  g_thread_err = buf;
  return code;
}

int npg::set_error_message(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_thread_err = buf;
  return code;
}

static bool is_sticky(cudaError_t e) {
  switch (e) {
    case cudaErrorIllegalAddress:
    case cudaErrorLaunchFailure:
    case cudaErrorIllegalInstruction:
    case cudaErrorMisalignedAddress:
    case cudaErrorInvalidAddressSpace:
    case cudaErrorInvalidPc:
    case cudaErrorHardwareStackError:
    case cudaErrorAssert:
    case cudaErrorLaunchTimeout:
    case cudaErrorECCUncorrectable:
      return true;
    default:
      return false;
  }
}

static int cuda_fail(npg_ctx* c, cudaError_t e, const char* what) {
  if (c && is_sticky(e)) c->sticky = 1;
  return set_err(c, e == cudaErrorMemoryAllocation ? NPG_ENOMEM : NPG_ECUDA, "%s: %s (%s)", what,
                 cudaGetErrorName(e), cudaGetErrorString(e));
}

#define CK(c, call)                                              \
  do {                                                           \
    cudaError_t _e = (call);                                     \
    if (_e != cudaSuccess) return cuda_fail((c), _e, #call);     \
  } while (0)

// ----------------------------------------------------------------- memory

static void* dev_alloc(npg_ctx* c, size_t bytes) {
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~(size_t)255;
  void* p = nullptr;
  if (c->cfg.alloc) {
    p = c->cfg.alloc(bytes, c->cfg.alloc_user);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p && ((uintptr_t)p & 15u) != 0) {  // bulk and vector copies need 16-byte alignment
    if (c->cfg.free) c->cfg.free(p, c->cfg.alloc_user);
    return nullptr;
  }
  if (p && c->n_allocs < 128) c->allocs[c->n_allocs++] = p;
  return p;
}

static void dev_free_all(npg_ctx* c) {
  for (int k = 0; k < c->n_allocs; ++k) {
    if (c->cfg.free)
      c->cfg.free(c->allocs[k], c->cfg.alloc_user);
    else
      cudaFree(c->allocs[k]);
  }
  c->n_allocs = 0;
}

template <class T>
static bool alloc_n(npg_ctx* c, T*& p, long long n) {
  p = static_cast<T*>(dev_alloc(c, sizeof(T) * (size_t)(n > 0 ? n : 1)));
  return p != nullptr;
}

// ----------------------------------------------------------------- timing

static void mark(npg_ctx* c, int k) {
  if (!c->tev || c->capturing || c->t_cur < 0) return;
  if (cudaEventRecord(c->tev[c->t_cur * (NPG_NUM_STAGES + 1) + k], c->stream) == cudaSuccess)
    c->t_mask[c->t_cur] |= 1u << k;
  else
    cudaGetLastError();
}

static void begin_iteration_timing(npg_ctx* c) {
  c->t_cur = (c->tev && !c->capturing && c->t_next < c->t_slots) ? c->t_next : -1;
  if (c->t_cur >= 0) c->t_mask[c->t_cur] = 0;
}

static void end_iteration_timing(npg_ctx* c) {
  if (c->t_cur >= 0) {
    c->t_next++;
    c->t_cur = -1;
  }
}

static void free_timing(npg_ctx* c) {
  if (c->tev) {
    for (int k = 0; k < c->t_slots * (NPG_NUM_STAGES + 1); ++k) cudaEventDestroy(c->tev[k]);
    delete[] c->tev;
    delete[] c->t_mask;
  }
  c->tev = nullptr;
  c->t_mask = nullptr;
  c->t_slots = c->t_next = 0;
  c->t_cur = -1;
}

// ----------------------------------------------------------------- config

extern "C" int npg_config_default(npg_config* cfg, int L, int r_min, int r_max, int F_p, int H,
                                  int depth) {
  if (!cfg) return set_err(nullptr, NPG_EINVAL, "cfg is NULL");
  if (L < 1 || L > NPG_MAX_LEVELS || r_min < 2 || r_max < r_min)
    return set_err(nullptr, NPG_EINVAL, "bad level schedule L=%d r=%d..%d", L, r_min, r_max);
  memset(cfg, 0, sizeof(*cfg));
  cfg->L = L;
  for (int l = 0; l < L; ++l)
    cfg->res[l] = L == 1 ? r_max
                         : (int)lround(r_min + (double)(r_max - r_min) * l / (double)(L - 1));
  cfg->F_p = F_p;
  cfg->F_n = 2;
  cfg->res_n = 4;
  cfg->H = H;
  cfg->depth = depth;
  cfg->leaky_slope = 0.01f;
  cfg->rot_mode = NPG_ROT_QUAT;
  cfg->n_freq = 4;
  cfg->alpha = 0.1f;
  cfg->lr_mlp = 1e-3f;
  for (int l = 0; l < L; ++l) {
    cfg->lr_grid[l] = (float)(0.005 * pow(2.5, l));
    cfg->lambda[l] = (float)(0.4 * pow(1.5, l));
  }
  cfg->lr_grid[L] = 0.005f;
  cfg->lambda[L] = 0.4f;
  cfg->adam_beta1 = 0.9f;
  cfg->adam_beta2 = 0.999f;
  cfg->adam_eps = 1e-8f;
  cfg->w_iso = 100.f;
  cfg->e_max = 1000;
  cfg->precision = NPG_FP32;
  return NPG_OK;
}

static int validate(const npg_config* c, char* why, size_t n) {
  if (c->L < 1 || c->L > NPG_MAX_LEVELS) return snprintf(why, n, "L=%d out of 1..16", c->L), 0;
  for (int l = 0; l < c->L; ++l)
    if (c->res[l] < 2 || c->res[l] > 1024)
      return snprintf(why, n, "res[%d]=%d out of 2..1024", l, c->res[l]), 0;
  if (c->F_p < 1 || c->F_p > NPG_MAX_F) return snprintf(why, n, "F_p=%d out of 1..32", c->F_p), 0;
  if (c->F_n < 1 || c->F_n > NPG_MAX_FN) return snprintf(why, n, "F_n=%d out of 1..8", c->F_n), 0;
  if (c->res_n < 2 || c->res_n > 64) return snprintf(why, n, "res_n=%d out of 2..64", c->res_n), 0;
  if (c->depth < 1 || c->depth > NPG_MAX_DEPTH)
    return snprintf(why, n, "depth=%d out of 1..8", c->depth), 0;
  if (c->n_freq < 1 || c->n_freq > NPG_MAX_FREQ)
    return snprintf(why, n, "n_freq=%d out of 1..8", c->n_freq), 0;
  if (c->time_enc < NPG_TIME_FOURIER || c->time_enc > NPG_TIME_LEARNED)
    return snprintf(why, n, "time_enc=%d", c->time_enc), 0;
  if (c->time_enc == NPG_TIME_LEARNED && (c->time_hidden < 1 || c->time_hidden > 256))
    return snprintf(why, n, "time_hidden=%d out of 1..256", c->time_hidden), 0;
  if (c->conf_delta < NPG_DELTA_SQRT || c->conf_delta > NPG_DELTA_INTERP)
    return snprintf(why, n, "conf_delta=%d", c->conf_delta), 0;
  if (c->conf_omega < NPG_OMEGA_CUMULATIVE || c->conf_omega > NPG_OMEGA_SINGLE)
    return snprintf(why, n, "conf_omega=%d", c->conf_omega), 0;
  if (c->rot_mode != NPG_ROT_QUAT && c->rot_mode != NPG_ROT_EXPMAP &&
      c->rot_mode != NPG_ROT_CAYLEY)
    return snprintf(why, n, "rot_mode=%d", c->rot_mode), 0;
  if (!(c->leaky_slope >= 0.f)) return snprintf(why, n, "leaky_slope must be >= 0"), 0;
  for (int l = 0; l <= c->L; ++l)
    if (!(c->lambda[l] >= 0.f) || !(c->lr_grid[l] >= 0.f))
      return snprintf(why, n, "lambda/lr of level %d must be >= 0", l), 0;
  if (c->e_max < 0) return snprintf(why, n, "e_max < 0"), 0;
  if (c->nn_cells < 0 || c->nn_cells > 256) return snprintf(why, n, "nn_cells out of 0..256"), 0;
  if (c->precond_mode != NPG_PRECOND_FP32 && c->precond_mode != NPG_PRECOND_TC)
    return snprintf(why, n, "precond_mode=%d", c->precond_mode), 0;
  if (c->precond_mode == NPG_PRECOND_TC)
    for (int l = 0; l < c->L; ++l)
      if (c->res[l] > 256) return snprintf(why, n, "tensor-core preconditioner needs res <= 256"), 0;
  return 1;
}

// ----------------------------------------------------------------- create

// Largest bucket resolution the autotuner may try for a set of T frames whose
// default is G: 1.25 G, at most 256, with T G^3 below 32M cell starts.
static int tune_cap(int G, int T) {
  int g = std::min(256, (G * 5 + 3) / 4);
  while (g > G && (double)g * g * g * T > 32.0e6) --g;
  return std::max(g, G);
}

static int copy_in(npg_ctx* c, void* dst, const void* src, size_t bytes, int on_device) {
  if (bytes == 0) return NPG_OK;
  CK(c, cudaMemcpyAsync(dst, src, bytes, on_device ? cudaMemcpyDeviceToDevice
                                                   : cudaMemcpyHostToDevice, c->stream));
  return NPG_OK;
}

static int fetch_host(npg_ctx* c, std::vector<char>& out, const void* src, size_t bytes,
                      int on_device) {
  out.resize(bytes);
  if (bytes == 0) return NPG_OK;
  if (on_device) {
    CK(c, cudaMemcpyAsync(out.data(), src, bytes, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
  } else {
    memcpy(out.data(), src, bytes);
  }
  return NPG_OK;
}

static int build_point_buckets(npg_ctx* c) {
  CK(c, bucket_build(c->praw, c->p_off, 0, c->T, c->MT, c->pb.G, c->pb, c->stream));
  return NPG_OK;
}

static int set_points_impl(npg_ctx* c, const float* points, const int64_t* off, int on_device) {
  std::vector<char> hoff;
  int rc = fetch_host(c, hoff, off, sizeof(int64_t) * (c->T + 1), on_device);
  if (rc) return rc;
  const int64_t* o = reinterpret_cast<const int64_t*>(hoff.data());
  if (o[0] != 0) return set_err(c, NPG_EINVAL, "frame_offsets[0] must be 0");
  for (int t = 0; t < c->T; ++t)
    if (o[t + 1] - o[t] < 1)
      return set_err(c, NPG_EINVAL, "frame %d has no points (every frame needs M_t >= 1)", t);
  const long long MT = o[c->T];
  if (c->MT_cap > 0 && MT > c->MT_cap)
    return set_err(c, NPG_EINVAL, "%lld points exceed the %lld given at create", MT, c->MT_cap);
  if (MT > 0x7fffffffLL) return set_err(c, NPG_EINVAL, "too many points");
  for (int t = 0; t <= c->T; ++t) c->h_off[t] = o[t];
  if (MT != c->MT && c->graph_exec) {  // the total is baked into the captured launches
    cudaGraphExecDestroy(c->graph_exec);
    cudaGraphDestroy(c->graph);
    c->graph_exec = nullptr;
    c->graph = nullptr;
  }
  c->MT = MT;
  rc = copy_in(c, c->p_off, c->h_off, sizeof(long long) * (c->T + 1), 0);
  if (rc) return rc;
  // raw xyz -> float4 (through the d_p buffer area when the input is on the host)
  float* staging = nullptr;
  if (on_device) {
    staging = const_cast<float*>(points);
  } else {
    staging = reinterpret_cast<float*>(c->pb.sorted);  // MT_cap float4 >= 3 MT floats
    rc = copy_in(c, staging, points, sizeof(float) * 3 * MT, 0);
    if (rc) return rc;
  }
  CK(c, launch_points_to_float4(staging, c->praw, MT, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  rc = build_point_buckets(c);
  if (rc) return rc;
  c->phase = 0;
  return NPG_OK;
}

extern "C" int npg_create(npg_ctx** out, const npg_config* cfg, const float* ref_xyz,
                          const float* ref_nrm, int N, const int32_t* faces, int F_tri,
                          const float* points, const int64_t* frame_offsets, int T, int t_key,
                          const float* mlp_init, size_t mlp_len, int inputs_on_device) {
  if (!out) return set_err(nullptr, NPG_EINVAL, "out is NULL");
  *out = nullptr;
  if (!cfg) return set_err(nullptr, NPG_EINVAL, "cfg is NULL");
  char why[256];
  if (!validate(cfg, why, sizeof(why))) return set_err(nullptr, NPG_EINVAL, "config: %s", why);
  if (N < 1 || T < 1 || F_tri < 0 || t_key < 0 || t_key >= T)
    return set_err(nullptr, NPG_EINVAL, "bad sizes N=%d T=%d F_tri=%d t_key=%d", N, T, F_tri,
                   t_key);
  if (!ref_xyz || !ref_nrm || !points || !frame_offsets || !mlp_init || (F_tri > 0 && !faces))
    return set_err(nullptr, NPG_EINVAL, "NULL input pointer");

  npg_ctx* c = new (std::nothrow) npg_ctx();
  if (!c) return set_err(nullptr, NPG_ENOMEM, "host allocation failed");
  c->cfg = *cfg;
  c->stream = static_cast<cudaStream_t>(cfg->stream);
  c->N = N;
  c->T = T;
  c->t_key = t_key;
  auto fail = [&](int rc) {
    g_thread_err = c->err;
    npg_destroy(c);
    return rc;
  };
  if (cudaGetDevice(&c->dev) != cudaSuccess) return fail(cuda_fail(c, cudaGetLastError(), "cudaGetDevice"));
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->dev);
  if (c->num_sms <= 0) c->num_sms = 148;
  c->lane[0] = c->stream;
  {
    cudaError_t e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
    for (int j = 0; j < npg_ctx::NLANE && e == cudaSuccess; ++j) {
      if (j > 0) e = cudaStreamCreateWithFlags(&c->lane[j], cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_join[j], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) return fail(cuda_fail(c, e, "lane streams"));
  }

  MlpDims& md = c->md;
  md.H = cfg->H;
  md.D = cfg->depth;
  md.Z = cfg->F_n + cfg->F_p;
  md.M = cfg->n_freq;
  md.K = md.Z + 2 * md.M;
  md.NO = cfg->rot_mode == NPG_ROT_QUAT ? 7 : 6;
  md.slope = cfg->leaky_slope;
  md.Ht = cfg->time_enc == NPG_TIME_LEARNED ? cfg->time_hidden : 0;
  md.dec_len = (long long)md.H * md.K + md.H + (long long)(md.D - 1) * (md.H * md.H + md.H) +
               (long long)md.NO * md.H + md.NO;
  c->mlp_len = md.dec_len + (md.Ht > 0 ? 2LL * md.Ht + 2LL * md.M * md.Ht + 2 * md.M : 0);
  if ((long long)mlp_len != c->mlp_len)
    return fail(set_err(c, NPG_EINVAL, "mlp_len %zu != expected %lld", mlp_len, c->mlp_len));
  if (cfg->precision == NPG_FP32) {
    if (!decode_fp32_supported(md.H, md.D) && !wide_fp32_supported(md.H))
      return fail(set_err(c, NPG_ENOTIMPL,
                          "FP32 path supports H in {16,32,64} or a multiple of 32 in (64, 512], "
                          "got %d", md.H));
    if (md.H <= 64 && mlp_bwd_fp32_smem(md) > 227 * 1024)
      return fail(set_err(c, NPG_ENOTIMPL, "FP32 backward needs %zu B shared memory (H=%d depth=%d)",
                          mlp_bwd_fp32_smem(md), md.H, md.D));
  } else if (cfg->precision == NPG_BF16_MLP) {
    if (!decode_bf16_supported(md.H, md.D) || !backward_bf16_supported(md.K, md.Z))
      return fail(set_err(c, NPG_ENOTIMPL,
                          "BF16 path supports H in {64, 128}, depth 3, F_n + F_p + 2 n_freq <= 15; "
                          "got H=%d depth=%d K=%d", md.H, md.D, md.K));
  } else {
    return fail(set_err(c, NPG_EINVAL, "precision=%d", cfg->precision));
  }

  // grid levels (l == L is the normal grid); device offsets 256-byte aligned
  c->nlev = cfg->L + 1;
  long long off = 0, flat = 0;
  for (int l = 0; l < c->nlev; ++l) {
    Level& lv = c->lev[l];
    lv.r = l < cfg->L ? cfg->res[l] : cfg->res_n;
    lv.F = l < cfg->L ? cfg->F_p : cfg->F_n;
    lv.n = (long long)lv.r * lv.r * lv.r * lv.F;
    lv.off = off;
    lv.flat = flat;
    lv.lr = cfg->lr_grid[l];
    lv.lambda = cfg->lambda[l];
    off += (lv.n + 63) & ~63LL;
    flat += lv.n;
    c->max_r = std::max(c->max_r, lv.r);
    c->max_level_n = std::max(c->max_level_n, lv.n);
    if (cfg->precond_mode == NPG_PRECOND_TC && lv.r >= PRECOND_TC_MIN_R)
      c->max_level_n = std::max(c->max_level_n, (long long)dct_tc_scratch_elems(lv.r, lv.F));
  }
  c->grid_dev_len = off;
  c->grid_flat_len = flat;

  // host-side copies of the small inputs we need to inspect
  std::vector<char> hoff, hfaces;
  int rc = fetch_host(c, hoff, frame_offsets, sizeof(int64_t) * (T + 1), inputs_on_device);
  if (rc) return fail(rc);
  const int64_t* ho = reinterpret_cast<const int64_t*>(hoff.data());
  c->MT_cap = ho[T];
  rc = fetch_host(c, hfaces, faces, sizeof(int32_t) * 3 * (size_t)F_tri, inputs_on_device);
  if (rc) return fail(rc);

  // edges: unique undirected (a < b), sorted; vertex-centric adjacency
  std::vector<std::pair<int, int>> ev;
  ev.reserve(3 * (size_t)F_tri);
  const int32_t* hf = reinterpret_cast<const int32_t*>(hfaces.data());
  c->faces_h.assign(hf, hf + 3 * (size_t)F_tri);
  for (int f = 0; f < F_tri; ++f)
    for (int k = 0; k < 3; ++k) {
      int a = hf[3 * f + k], b = hf[3 * f + (k + 1) % 3];
      if (a < 0 || a >= N || b < 0 || b >= N)
        return fail(set_err(c, NPG_EINVAL, "face %d references vertex out of range", f));
      if (a == b) continue;
      ev.emplace_back(std::min(a, b), std::max(a, b));
    }
  std::sort(ev.begin(), ev.end());
  ev.erase(std::unique(ev.begin(), ev.end()), ev.end());
  c->E = (int)ev.size();
  std::vector<int> adj_off(N + 1, 0), adj(2 * (size_t)c->E), adj_edge(2 * (size_t)c->E);
  std::vector<int2> edges(c->E);
  for (int e = 0; e < c->E; ++e) {
    edges[e] = make_int2(ev[e].first, ev[e].second);
    adj_off[ev[e].first + 1]++;
    adj_off[ev[e].second + 1]++;
  }
  for (int i = 0; i < N; ++i) adj_off[i + 1] += adj_off[i];
  {
    std::vector<int> fill(adj_off.begin(), adj_off.end() - 1);
    for (int e = 0; e < c->E; ++e) {
      int a = ev[e].first, b = ev[e].second;
      adj[fill[a]] = b;
      adj_edge[fill[a]++] = e;
      adj[fill[b]] = a;
      adj_edge[fill[b]++] = e;
    }
  }

  // bucket resolutions
  const long long Mavg = std::max<long long>(1, c->MT_cap / T);
  c->pb.G = cfg->nn_cells > 0 ? cfg->nn_cells : auto_cells(Mavg, T);
  c->xb.G = cfg->nn_cells > 0 ? cfg->nn_cells : auto_cells(N, T);
  c->pb.nsets = c->xb.nsets = T;
  // room for the autotuner's finer candidates (up to 1.25 x, within the cap of
  // 32M cell starts over all frames)
  c->G_cap_p = tune_cap(c->pb.G, T);
  c->G_cap_x = tune_cap(c->xb.G, T);
  const long long Gp3 = (long long)c->G_cap_p * c->G_cap_p * c->G_cap_p;
  const long long Gx3 = (long long)c->G_cap_x * c->G_cap_x * c->G_cap_x;
  const long long NT = (long long)N * T;

  bool ok = true;
  ok &= alloc_n(c, c->xr, N) && alloc_n(c, c->nr, N);
  ok &= alloc_n(c, c->adj_off, N + 1) && alloc_n(c, c->adj, 2LL * c->E) &&
        alloc_n(c, c->adj_edge, 2LL * c->E) && alloc_n(c, c->edges, c->E);
  ok &= alloc_n(c, c->p_off, T + 1) && alloc_n(c, c->praw, c->MT_cap);
  ok &= alloc_n(c, c->pb.cell_start, T * (Gp3 + 1)) && alloc_n(c, c->pb.counts, T * Gp3) &&
        alloc_n(c, c->pb.slot, c->MT_cap) && alloc_n(c, c->pb.sorted, c->MT_cap);
  ok &= alloc_n(c, c->xb.cell_start, T * (Gx3 + 1)) && alloc_n(c, c->xb.counts, T * Gx3) &&
        alloc_n(c, c->xb.slot, NT) && alloc_n(c, c->xb.sorted, NT);
  // z and gamma carry 16 B of padding: the BF16 backward stages them with
  // bulk copies rounded up to 16 B
  ok &= alloc_n(c, c->z, (long long)N * md.Z + 4) && alloc_n(c, c->U, (long long)N * md.H) &&
        alloc_n(c, c->V, (long long)T * md.H) && alloc_n(c, c->xhat, NT) &&
        alloc_n(c, c->gamma, (long long)T * 2 * md.M + 4) &&
        alloc_n(c, c->disp, NT) &&
        alloc_n(c, c->dxhat, NT) && alloc_n(c, c->nn_x, NT) && alloc_n(c, c->d_x, NT) &&
        alloc_n(c, c->nn_p, c->MT_cap) && alloc_n(c, c->d_p, c->MT_cap) &&
        alloc_n(c, c->dz, (long long)N * md.Z);
  if (md.Ht > 0) ok &= alloc_n(c, c->dV, (long long)T * md.H);
  ok &= alloc_n(c, c->cd, T) && alloc_n(c, c->wconf, T) && alloc_n(c, c->iso_t, T) &&
        alloc_n(c, c->loss_part, (long long)T * 8 * 3) && alloc_n(c, c->dx_coef, 2LL * T) &&
        alloc_n(c, c->loss, 4) && alloc_n(c, c->d_epoch, 1) && alloc_n(c, c->d_adam_c, 2) &&
        alloc_n(c, c->d_err, 1) && alloc_n(c, c->d_nnstats, 4) &&
        alloc_n(c, c->nnq.counters, 4) && alloc_n(c, c->nnq.items, std::max(NT, c->MT_cap));
  c->nnq.far_blocks = c->num_sms * 16;
  // the widest seed ball one thread covers: the autotuner's usual choices
  // (vertex -> point 24-96, point -> vertex 192-384 rows)
  c->nnq.near_rows = 48;
  ok &= alloc_n(c, c->grid, c->grid_dev_len) && alloc_n(c, c->g_grid, c->grid_dev_len) &&
        alloc_n(c, c->g_pc, c->grid_dev_len) && alloc_n(c, c->m_grid, c->grid_dev_len) &&
        alloc_n(c, c->v_grid, c->grid_dev_len);
  ok &= alloc_n(c, c->mlp, c->mlp_len) && alloc_n(c, c->g_mlp, c->mlp_len) &&
        alloc_n(c, c->m_mlp, c->mlp_len) && alloc_n(c, c->v_mlp, c->mlp_len);
  ok &= alloc_n(c, c->pc_tmp0, c->max_level_n) && alloc_n(c, c->pc_tmp1, c->max_level_n);
  if (cfg->precision == NPG_FP32 && md.H > 64)
    ok &= alloc_n(c, c->wide, wide_fp32_scratch_floats(md.H, md.D, md.K, NT, &c->wide_rows));
  ok &= alloc_n(c, c->nnq_p.counters, 4) && alloc_n(c, c->nnq_p.items, c->MT_cap);
  c->nnq_p.far_blocks = c->num_sms * 16;
  c->nnq_p.near_rows = 192;
  // levels to lanes, largest first onto the least loaded lane; each lane's
  // scratch holds its largest level
  {
    long long load[npg_ctx::NLANE] = {}, need[npg_ctx::NLANE] = {};
    int order[NPG_MAX_LEVELS + 1];
    for (int l = 0; l < c->nlev; ++l) order[l] = l;
    std::sort(order, order + c->nlev, [&](int a, int b) { return c->lev[a].n > c->lev[b].n; });
    for (int i = 0; i < c->nlev; ++i) {
      const int l = order[i];
      int best = 0;
      for (int j = 1; j < npg_ctx::NLANE; ++j)
        if (load[j] < load[best]) best = j;
      c->level_lane[l] = best;
      load[best] += c->lev[l].n;
      long long n = c->lev[l].n;
      if (cfg->precond_mode == NPG_PRECOND_TC && c->lev[l].r >= PRECOND_TC_MIN_R)
        n = std::max(n, (long long)dct_tc_scratch_elems(c->lev[l].r, c->lev[l].F));
      need[best] = std::max(need[best], n);
    }
    c->lane_tmp[0][0] = c->pc_tmp0;
    c->lane_tmp[0][1] = c->pc_tmp1;
    for (int j = 1; j < npg_ctx::NLANE; ++j)
      if (need[j] > 0)
        ok &= alloc_n(c, c->lane_tmp[j][0], need[j]) && alloc_n(c, c->lane_tmp[j][1], need[j]);
  }
  long long dct_len = 0;
  for (int l = 0; l < c->nlev; ++l) {
    c->dct_off[l] = dct_len;
    dct_len += ((2LL * c->lev[l].r * c->lev[l].r + c->lev[l].r) + 63) & ~63LL;
  }
  ok &= alloc_n(c, c->dct, dct_len);
  long long tc_len = 0;
  if (cfg->precond_mode == NPG_PRECOND_TC)
    for (int l = 0; l < c->nlev; ++l)
      for (int m = 0; m < 2; ++m) {
        c->dct_tc_off[l][m] = tc_len;
        tc_len += ((long long)dct_tc_table_elems(c->lev[l].r) + 127) & ~127LL;
      }
  if (tc_len > 0) ok &= alloc_n(c, c->dct_tc, tc_len);
  if (!ok) return fail(set_err(c, NPG_ENOMEM, "device allocation failed"));
  if (cudaMallocHost(&c->h_loss, sizeof(double) * (4 + T)) != cudaSuccess ||
      cudaMallocHost(&c->h_off, sizeof(long long) * (T + 1)) != cudaSuccess) {
    cudaGetLastError();
    return fail(set_err(c, NPG_ENOMEM, "pinned host allocation failed"));
  }

  // inputs
  {
    std::vector<char> hx, hn;
    if ((rc = fetch_host(c, hx, ref_xyz, sizeof(float) * 3 * (size_t)N, inputs_on_device)) ||
        (rc = fetch_host(c, hn, ref_nrm, sizeof(float) * 3 * (size_t)N, inputs_on_device)))
      return fail(rc);
    std::vector<float4> x4(N), n4(N);
    const float* px = reinterpret_cast<const float*>(hx.data());
    const float* pn = reinterpret_cast<const float*>(hn.data());
    for (int i = 0; i < N; ++i) {
      x4[i] = make_float4(px[3 * i], px[3 * i + 1], px[3 * i + 2], 0.f);
      n4[i] = make_float4(pn[3 * i], pn[3 * i + 1], pn[3 * i + 2], 0.f);
    }
    if ((rc = copy_in(c, c->xr, x4.data(), sizeof(float4) * N, 0)) ||
        (rc = copy_in(c, c->nr, n4.data(), sizeof(float4) * N, 0)) ||
        (rc = copy_in(c, c->adj_off, adj_off.data(), sizeof(int) * (N + 1), 0)) ||
        (rc = copy_in(c, c->adj, adj.data(), sizeof(int) * adj.size(), 0)) ||
        (rc = copy_in(c, c->adj_edge, adj_edge.data(), sizeof(int) * adj_edge.size(), 0)) ||
        (rc = copy_in(c, c->edges, edges.data(), sizeof(int2) * edges.size(), 0)) ||
        (rc = copy_in(c, c->mlp, mlp_init, sizeof(float) * mlp_len, inputs_on_device)))
      return fail(rc);
    std::vector<float> tab(dct_len, 0.f);
    for (int l = 0; l < c->nlev; ++l) {
      const int r = c->lev[l].r;
      float* base = tab.data() + c->dct_off[l];
      dct_tables(r, base, base + (long long)r * r, base + 2LL * r * r);
    }
    if ((rc = copy_in(c, c->dct, tab.data(), sizeof(float) * tab.size(), 0))) return fail(rc);
    if (tc_len > 0) {
      std::vector<uint16_t> tt((size_t)tc_len, 0);
      for (int l = 0; l < c->nlev; ++l) {
        const int r = c->lev[l].r;
        const float* base = tab.data() + c->dct_off[l];
        dct_tc_tables(r, base, tt.data() + c->dct_tc_off[l][0]);
        dct_tc_tables(r, base + (long long)r * r, tt.data() + c->dct_tc_off[l][1]);
      }
      CK(c, cudaMemcpyAsync(c->dct_tc, tt.data(), sizeof(uint16_t) * tt.size(),
                            cudaMemcpyHostToDevice, c->stream));
      CK(c, cudaStreamSynchronize(c->stream));
    }
    CK(c, cudaStreamSynchronize(c->stream));
  }
  CK(c, cudaMemsetAsync(c->grid, 0, sizeof(float) * c->grid_dev_len, c->stream));
  CK(c, cudaMemsetAsync(c->m_grid, 0, sizeof(float) * c->grid_dev_len, c->stream));
  CK(c, cudaMemsetAsync(c->v_grid, 0, sizeof(float) * c->grid_dev_len, c->stream));
  CK(c, cudaMemsetAsync(c->g_grid, 0, sizeof(float) * c->grid_dev_len, c->stream));
  CK(c, cudaMemsetAsync(c->g_pc, 0, sizeof(float) * c->grid_dev_len, c->stream));
  CK(c, cudaMemsetAsync(c->m_mlp, 0, sizeof(float) * c->mlp_len, c->stream));
  CK(c, cudaMemsetAsync(c->v_mlp, 0, sizeof(float) * c->mlp_len, c->stream));
  CK(c, cudaMemsetAsync(c->g_mlp, 0, sizeof(float) * c->mlp_len, c->stream));
  CK(c, cudaMemsetAsync(c->d_epoch, 0, sizeof(int), c->stream));
  CK(c, cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream));
  CK(c, cudaMemsetAsync(c->d_nnstats, 0, sizeof(unsigned long long) * 4, c->stream));
  CK(c, launch_time_table(c));
  // no nearest-neighbour seeds before the first search
  CK(c, cudaMemsetAsync(c->nn_x, 0xff, sizeof(int) * NT, c->stream));
  CK(c, cudaMemsetAsync(c->nn_p, 0xff, sizeof(int) * c->MT_cap, c->stream));
  if ((rc = set_points_impl(c, points, frame_offsets, inputs_on_device))) return fail(rc);
  CK(c, cudaStreamSynchronize(c->stream));
  c->phase = 0;
  *out = c;
  return NPG_OK;
}

// ----------------------------------------------------------------- the iteration

static int guard(npg_ctx* c) {
  if (!c) return set_err(nullptr, NPG_EINVAL, "ctx is NULL");
  if (c->sticky) return set_err(c, NPG_ECUDA, "context unusable after a sticky CUDA error: %s",
                                c->err.c_str());
  return NPG_OK;
}

static int forward_launch(npg_ctx* c) {
  begin_iteration_timing(c);
  mark(c, 0);
  CK(c, launch_encode(c));
  if (c->md.Ht > 0) {
    CK(c, launch_learned_time(c));
    c->launches += 1;
  }
  CK(c, launch_time_mod(c));
  mark(c, 1);
  if (c->cfg.precision == NPG_BF16_MLP)
    CK(c, launch_decode_bf16(c));
  else
    CK(c, launch_decode_fp32(c));
  mark(c, 2);
  c->launches += 3;
  return NPG_OK;
}

// Lanes 1..n-1 start after everything issued so far on the main stream.
static cudaError_t lanes_fork(npg_ctx* c, int n) {
  cudaError_t e = cudaEventRecord(c->ev_fork, c->stream);
  for (int j = 1; j < n && e == cudaSuccess; ++j) e = cudaStreamWaitEvent(c->lane[j], c->ev_fork, 0);
  return e;
}

// The main stream continues after everything issued on lanes 1..n-1.
static cudaError_t lanes_join(npg_ctx* c, int n) {
  cudaError_t e = cudaSuccess;
  for (int j = 1; j < n && e == cudaSuccess; ++j) {
    e = cudaEventRecord(c->ev_join[j], c->lane[j]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, c->ev_join[j], 0);
  }
  return e;
}

static int loss_launch(npg_ctx* c) {
  const long long NT = (long long)c->N * c->T;
  CK(c, bucket_build(c->xhat, nullptr, c->N, c->T, NT, c->xb.G, c->xb, c->stream));
  mark(c, 3);
  // vertex -> point (queries in x-hat bucket order for coherent warps)
  const bool count = c->tev && !c->capturing && c->t_cur >= 0;
  // point -> vertex on lane 1, concurrently with vertex -> point on the main stream
  CK(c, lanes_fork(c, 2));
  CK(c, launch_nn(c->pb.sorted, 0, c->p_off, c->T, c->MT, c->xb, nullptr, c->N, c->nn_p, c->d_p,
                  c->nnq_p, c->lane[1], count ? c->d_nnstats + 2 : nullptr, true));
  CK(c, launch_nn(c->xb.sorted, c->N, nullptr, c->T, NT, c->pb, c->p_off, 0, c->nn_x, c->d_x,
                  c->nnq, c->stream, count ? c->d_nnstats : nullptr, true));
  mark(c, 4);
  CK(c, lanes_join(c, 2));
  mark(c, 5);
  CK(c, launch_loss(c));
  mark(c, 6);
  c->launches += 3 + 4 + 3;
  return NPG_OK;
}

static int backprop_launch(npg_ctx* c) {
  CK(c, cudaMemsetAsync(c->g_mlp, 0, sizeof(float) * c->mlp_len, c->stream));
  CK(c, cudaMemsetAsync(c->dz, 0, sizeof(float) * (size_t)c->N * c->md.Z, c->stream));
  if (c->dV)
    CK(c, cudaMemsetAsync(c->dV, 0, sizeof(float) * (size_t)c->T * c->md.H, c->stream));
  // the grid gradient (every level; 0.6 GB at the paper's sizes) is cleared on
  // lane 1 while the MLP backward, which neither reads nor writes it, runs
  CK(c, lanes_fork(c, 2));
  CK(c, cudaMemsetAsync(c->g_grid, 0, sizeof(float) * c->grid_dev_len, c->lane[1]));
  if (c->cfg.precision == NPG_BF16_MLP)
    CK(c, launch_mlp_backward_bf16(c));
  else
    CK(c, launch_mlp_backward_fp32(c));
  CK(c, lanes_join(c, 2));
  if (c->md.Ht > 0) {
    CK(c, launch_learned_time_backward(c));
    c->launches += 1;
  }
  mark(c, 8);
  CK(c, launch_scatter(c));
  mark(c, 9);
  c->launches += 2;
  return NPG_OK;
}

static int backward_launch(npg_ctx* c) {
  CK(c, launch_dxhat(c));
  mark(c, 7);
  c->launches += 3;
  return backprop_launch(c);
}

static int step_launch(npg_ctx* c) {
  const npg_config& f = c->cfg;
  CK(c, launch_step_prepare(c->d_epoch, f.adam_beta1, f.adam_beta2, c->d_adam_c, c->stream));
  // each grid level's preconditioner and Adam step on its lane (levels are
  // independent), the lanes joined back before the epoch advances
  CK(c, lanes_fork(c, npg_ctx::NLANE));
  for (int l = 0; l < c->nlev; ++l) {
    const Level& lv = c->lev[l];
    const int j = c->level_lane[l];
    cudaStream_t ls = c->lane[j];
    const float* tab = c->dct + c->dct_off[l];
    const long long rr = (long long)lv.r * lv.r;
    if (c->cfg.precond_mode == NPG_PRECOND_TC && lv.r >= PRECOND_TC_MIN_R)
      CK(c, launch_precondition_tc(c->g_grid + lv.off, c->g_pc + lv.off, c->lane_tmp[j][0],
                                   c->lane_tmp[j][1], c->dct_tc + c->dct_tc_off[l][0],
                                   c->dct_tc + c->dct_tc_off[l][1], tab + 2 * rr, lv.r, lv.F,
                                   lv.lambda, c->d_err, ls));
    else
      CK(c, launch_precondition(c->g_grid + lv.off, c->g_pc + lv.off, c->lane_tmp[j][0],
                                c->lane_tmp[j][1], tab, tab + rr, tab + 2 * rr, lv.r, lv.F,
                                lv.lambda, ls));
    CK(c, launch_adam(c->grid + lv.off, c->g_pc + lv.off, c->m_grid + lv.off,
                      c->v_grid + lv.off, lv.n, lv.lr, f.adam_beta1, f.adam_beta2, f.adam_eps,
                      c->d_adam_c, ls));
  }
  CK(c, lanes_join(c, npg_ctx::NLANE));
  mark(c, 10);
  CK(c, launch_adam(c->mlp, c->g_mlp, c->m_mlp, c->v_mlp, c->mlp_len, f.lr_mlp, f.adam_beta1,
                    f.adam_beta2, f.adam_eps, c->d_adam_c, c->stream));
  CK(c, launch_step_finish(c->d_epoch, c->stream));
  mark(c, 11);
  end_iteration_timing(c);
  c->launches += 1 + 6LL * c->nlev + c->nlev + 1 + 1;
  return NPG_OK;
}

// After a synchronisation: report a kernel whose bounded wait gave up.
static int check_device_error(npg_ctx* c) {
  int e = 0;
  CK(c, cudaMemcpy(&e, c->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (e) {
    CK(c, cudaMemset(c->d_err, 0, sizeof(int)));
    return set_err(c, NPG_ETIMEOUT, "a tensor-core wait timed out; results of this call are invalid");
  }
  return NPG_OK;
}

static int copy_loss_out(npg_ctx* c, double* loss_out, double* cd_out) {
  if (!loss_out && !cd_out) return NPG_OK;
  CK(c, cudaMemcpyAsync(c->h_loss, c->loss, sizeof(double) * 3, cudaMemcpyDeviceToHost,
                        c->stream));
  if (cd_out)
    CK(c, cudaMemcpyAsync(c->h_loss + 4, c->cd, sizeof(double) * c->T, cudaMemcpyDeviceToHost,
                          c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  if (int rc = check_device_error(c)) return rc;
  if (loss_out) memcpy(loss_out, c->h_loss, sizeof(double) * 3);
  if (cd_out) memcpy(cd_out, c->h_loss + 4, sizeof(double) * c->T);
  return NPG_OK;
}

extern "C" int npg_forward(npg_ctx* c, float* xhat_out) {
  int rc = guard(c);
  if (rc) return rc;
  if ((rc = forward_launch(c))) return rc;
  if (xhat_out) CK(c, launch_xhat_out(c->xhat, xhat_out, (long long)c->N * c->T, c->stream));
  c->phase = 1;
  return NPG_OK;
}

extern "C" int npg_loss(npg_ctx* c, double* loss_out, double* cd_out) {
  int rc = guard(c);
  if (rc) return rc;
  if (c->phase != 1) return set_err(c, NPG_ESTATE, "npg_loss needs a preceding npg_forward");
  if ((rc = loss_launch(c))) return rc;
  c->phase = 2;
  return copy_loss_out(c, loss_out, cd_out);
}

extern "C" int npg_backward(npg_ctx* c) {
  int rc = guard(c);
  if (rc) return rc;
  if (c->phase != 2) return set_err(c, NPG_ESTATE, "npg_backward needs a preceding npg_loss");
  if ((rc = backward_launch(c))) return rc;
  c->phase = 3;
  return NPG_OK;
}

extern "C" int npg_backprop(npg_ctx* c, const float* dxhat) {
  int rc = guard(c);
  if (rc) return rc;
  if (c->phase < 1) return set_err(c, NPG_ESTATE, "npg_backprop needs a preceding npg_forward");
  if (dxhat)
    CK(c, launch_points_to_float4(dxhat, c->dxhat, (long long)c->N * c->T, c->stream));
  if ((rc = backprop_launch(c))) return rc;
  c->phase = 3;
  return NPG_OK;
}

extern "C" int npg_step(npg_ctx* c) {
  int rc = guard(c);
  if (rc) return rc;
  if (c->phase != 3) return set_err(c, NPG_ESTATE, "npg_step needs a preceding npg_backward");
  if ((rc = step_launch(c))) return rc;
  c->phase = 0;
  c->e += 1;
  return NPG_OK;
}

static int iteration_launch(npg_ctx* c) {
  int rc;
  if ((rc = forward_launch(c)) || (rc = loss_launch(c)) || (rc = backward_launch(c)) ||
      (rc = step_launch(c)))
    return rc;
  return NPG_OK;
}

extern "C" int npg_iteration(npg_ctx* c, double* loss_out) {
  int rc = guard(c);
  if (rc) return rc;
  if (!c->cfg.use_graph) {
    if ((rc = iteration_launch(c))) return rc;
  } else {
    if (!c->graph_exec) {
      if (c->stream == nullptr)
        return set_err(c, NPG_EINVAL, "use_graph needs a non-default stream");
      // one eager iteration first: function attributes and lazy module loading
      // happen outside the capture
      if ((rc = iteration_launch(c))) return rc;
      CK(c, cudaStreamSynchronize(c->stream));
      c->e += 1;
      c->phase = 0;
      CK(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
      c->capturing = 1;
      const long long before = c->launches;
      rc = iteration_launch(c);
      c->capturing = 0;
      c->graph_launches = c->launches - before;
      c->launches = before;
      cudaGraph_t g = nullptr;
      cudaError_t ce = cudaStreamEndCapture(c->stream, &g);
      if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
      }
      if (ce != cudaSuccess) return cuda_fail(c, ce, "cudaStreamEndCapture");
      c->graph = g;
      CK(c, cudaGraphInstantiate(&c->graph_exec, g, 0));
      // this call's iteration was the eager one; replays start with the next call
      if (loss_out) {
        rc = copy_loss_out(c, loss_out, nullptr);
        if (rc) return rc;
      }
      return NPG_OK;
    }
    CK(c, cudaGraphLaunch(c->graph_exec, c->stream));
    c->launches += c->graph_launches;
  }
  c->e += 1;
  c->phase = 0;
  return copy_loss_out(c, loss_out, nullptr);
}

// ----------------------------------------------------------------- buffers

extern "C" size_t npg_size(const npg_ctx* c, int which) {
  if (!c) return 0;
  const size_t NT = (size_t)c->N * c->T;
  switch (which) {
    case NPG_BUF_GRID: case NPG_BUF_GRID_GRAD: case NPG_BUF_GRID_PC:
    case NPG_BUF_ADAM_M_GRID: case NPG_BUF_ADAM_V_GRID:
      return sizeof(float) * (size_t)c->grid_flat_len;
    case NPG_BUF_MLP: case NPG_BUF_MLP_GRAD: case NPG_BUF_ADAM_M_MLP: case NPG_BUF_ADAM_V_MLP:
      return sizeof(float) * (size_t)c->mlp_len;
    case NPG_BUF_XHAT: case NPG_BUF_DXHAT: case NPG_BUF_DISP: return sizeof(float) * 3 * NT;
    case NPG_BUF_NN_X: return sizeof(int32_t) * NT;
    case NPG_BUF_NN_P: return sizeof(int32_t) * (size_t)c->MT;
    case NPG_BUF_CD: case NPG_BUF_WCONF: return sizeof(double) * (size_t)c->T;
    case NPG_BUF_DIST_X: return sizeof(float) * NT;
    case NPG_BUF_DIST_P: return sizeof(float) * (size_t)c->MT;
    case NPG_BUF_DEVICE_ERROR: return sizeof(int32_t);
  }
  return 0;
}

static float* grid_buf(npg_ctx* c, int which) {
  switch (which) {
    case NPG_BUF_GRID: return c->grid;
    case NPG_BUF_GRID_GRAD: return c->g_grid;
    case NPG_BUF_GRID_PC: return c->g_pc;
    case NPG_BUF_ADAM_M_GRID: return c->m_grid;
    case NPG_BUF_ADAM_V_GRID: return c->v_grid;
  }
  return nullptr;
}

static void* plain_buf(npg_ctx* c, int which) {
  switch (which) {
    case NPG_BUF_MLP: return c->mlp;
    case NPG_BUF_MLP_GRAD: return c->g_mlp;
    case NPG_BUF_ADAM_M_MLP: return c->m_mlp;
    case NPG_BUF_ADAM_V_MLP: return c->v_mlp;
    case NPG_BUF_NN_X: return c->nn_x;
    case NPG_BUF_NN_P: return c->nn_p;
    case NPG_BUF_CD: return c->cd;
    case NPG_BUF_WCONF: return c->wconf;
    case NPG_BUF_DIST_X: return c->d_x;
    case NPG_BUF_DIST_P: return c->d_p;
    case NPG_BUF_DEVICE_ERROR: return c->d_err;
  }
  return nullptr;
}

extern "C" int npg_get(npg_ctx* c, int which, void* dst, size_t bytes, int dst_on_device) {
  int rc = guard(c);
  if (rc) return rc;
  const size_t need = npg_size(c, which);
  if (need == 0) return set_err(c, NPG_EINVAL, "unknown buffer %d", which);
  if (!dst || bytes != need)
    return set_err(c, NPG_EINVAL, "buffer %d needs %zu bytes, got %zu", which, need, bytes);
  const cudaMemcpyKind kind = dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (float* g = grid_buf(c, which)) {
    for (int l = 0; l < c->nlev; ++l)
      CK(c, cudaMemcpyAsync(static_cast<float*>(dst) + c->lev[l].flat, g + c->lev[l].off,
                            sizeof(float) * c->lev[l].n, kind, c->stream));
  } else if (which == NPG_BUF_XHAT || which == NPG_BUF_DXHAT || which == NPG_BUF_DISP) {
    const long long NT = (long long)c->N * c->T;
    const float4* srcv =
        which == NPG_BUF_XHAT ? c->xhat : (which == NPG_BUF_DXHAT ? c->dxhat : c->disp);
    if (dst_on_device) {
      CK(c, launch_xhat_out(srcv, static_cast<float*>(dst), NT, c->stream));
    } else {
      if (!c->xhat3 && !alloc_n(c, c->xhat3, 3 * NT))
        return set_err(c, NPG_ENOMEM, "device allocation failed");
      CK(c, launch_xhat_out(srcv, c->xhat3, NT, c->stream));
      CK(c, cudaMemcpyAsync(dst, c->xhat3, bytes, kind, c->stream));
    }
  } else {
    CK(c, cudaMemcpyAsync(dst, plain_buf(c, which), bytes, kind, c->stream));
  }
  CK(c, cudaStreamSynchronize(c->stream));
  // reading the error word itself reports it without clearing it
  return which == NPG_BUF_DEVICE_ERROR ? NPG_OK : check_device_error(c);
}

extern "C" int npg_set(npg_ctx* c, int which, const void* src, size_t bytes, int src_on_device) {
  int rc = guard(c);
  if (rc) return rc;
  const bool settable = which == NPG_BUF_GRID || which == NPG_BUF_MLP ||
                        which == NPG_BUF_ADAM_M_GRID || which == NPG_BUF_ADAM_V_GRID ||
                        which == NPG_BUF_ADAM_M_MLP || which == NPG_BUF_ADAM_V_MLP ||
                        which == NPG_BUF_NN_X || which == NPG_BUF_NN_P ||
                        which == NPG_BUF_DEVICE_ERROR;
  if (!settable) return set_err(c, NPG_EINVAL, "buffer %d is not settable", which);
  const size_t need = npg_size(c, which);
  if (!src || bytes != need)
    return set_err(c, NPG_EINVAL, "buffer %d needs %zu bytes, got %zu", which, need, bytes);
  const cudaMemcpyKind kind = src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (float* g = grid_buf(c, which)) {
    for (int l = 0; l < c->nlev; ++l)
      CK(c, cudaMemcpyAsync(g + c->lev[l].off, static_cast<const float*>(src) + c->lev[l].flat,
                            sizeof(float) * c->lev[l].n, kind, c->stream));
  } else {
    CK(c, cudaMemcpyAsync(plain_buf(c, which), src, bytes, kind, c->stream));
  }
  CK(c, cudaStreamSynchronize(c->stream));
  c->phase = 0;
  return NPG_OK;
}

extern "C" int npg_get_epoch(const npg_ctx* c) { return c ? c->e : -1; }

extern "C" int npg_set_epoch(npg_ctx* c, int e) {
  int rc = guard(c);
  if (rc) return rc;
  if (e < 0) return set_err(c, NPG_EINVAL, "epoch < 0");
  c->e = e;
  CK(c, cudaMemcpyAsync(c->d_epoch, &c->e, sizeof(int), cudaMemcpyHostToDevice, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  c->phase = 0;
  return NPG_OK;
}

// state blob: magic, version, grid_flat_len, mlp_len, e, then six FP32 arrays
struct StateHeader {
  uint64_t magic, version, grid_len, mlp_len, epoch, pad;
};
static const uint64_t kMagic = 0x4e50475354415445ULL;  // "NPGSTATE"

extern "C" int npg_get_state(npg_ctx* c, void* blob, size_t* bytes) {
  int rc = guard(c);
  if (rc) return rc;
  if (!bytes) return set_err(c, NPG_EINVAL, "bytes is NULL");
  const size_t gsz = sizeof(float) * c->grid_flat_len, msz = sizeof(float) * c->mlp_len;
  const size_t need = sizeof(StateHeader) + 3 * gsz + 3 * msz;
  if (!blob) {
    *bytes = need;
    return NPG_OK;
  }
  if (*bytes < need) return set_err(c, NPG_EINVAL, "state needs %zu bytes", need);
  StateHeader h{kMagic, 1, (uint64_t)c->grid_flat_len, (uint64_t)c->mlp_len, (uint64_t)c->e, 0};
  char* p = static_cast<char*>(blob);
  memcpy(p, &h, sizeof(h));
  p += sizeof(h);
  const int ids[6] = {NPG_BUF_GRID, NPG_BUF_ADAM_M_GRID, NPG_BUF_ADAM_V_GRID,
                      NPG_BUF_MLP,  NPG_BUF_ADAM_M_MLP,  NPG_BUF_ADAM_V_MLP};
  for (int k = 0; k < 6; ++k) {
    const size_t sz = k < 3 ? gsz : msz;
    if ((rc = npg_get(c, ids[k], p, sz, 0))) return rc;
    p += sz;
  }
  *bytes = need;
  return NPG_OK;
}

extern "C" int npg_set_state(npg_ctx* c, const void* blob, size_t bytes) {
  int rc = guard(c);
  if (rc) return rc;
  if (!blob || bytes < sizeof(StateHeader)) return set_err(c, NPG_EINVAL, "state too small");
  StateHeader h;
  memcpy(&h, blob, sizeof(h));
  const size_t gsz = sizeof(float) * c->grid_flat_len, msz = sizeof(float) * c->mlp_len;
  if (h.magic != kMagic || h.version != 1 || h.grid_len != (uint64_t)c->grid_flat_len ||
      h.mlp_len != (uint64_t)c->mlp_len || bytes != sizeof(h) + 3 * gsz + 3 * msz)
    return set_err(c, NPG_EINVAL, "state blob does not match this context");
  const char* p = static_cast<const char*>(blob) + sizeof(h);
  const int ids[6] = {NPG_BUF_GRID, NPG_BUF_ADAM_M_GRID, NPG_BUF_ADAM_V_GRID,
                      NPG_BUF_MLP,  NPG_BUF_ADAM_M_MLP,  NPG_BUF_ADAM_V_MLP};
  for (int k = 0; k < 6; ++k) {
    const size_t sz = k < 3 ? gsz : msz;
    if ((rc = npg_set(c, ids[k], p, sz, 0))) return rc;
    p += sz;
  }
  return npg_set_epoch(c, (int)h.epoch);
}

extern "C" int npg_set_points(npg_ctx* c, const float* points, const int64_t* frame_offsets,
                              int on_device) {
  int rc = guard(c);
  if (rc) return rc;
  if (!points || !frame_offsets) return set_err(c, NPG_EINVAL, "NULL pointer");
  return set_points_impl(c, points, frame_offsets, on_device);
}

extern "C" int npg_timing(npg_ctx* c, int n_iters) {
  int rc = guard(c);
  if (rc) return rc;
  if (n_iters < 0 || n_iters > 100000) return set_err(c, NPG_EINVAL, "n_iters out of 0..100000");
  CK(c, cudaStreamSynchronize(c->stream));
  free_timing(c);
  if (n_iters == 0) return NPG_OK;
  const int per = NPG_NUM_STAGES + 1;
  c->tev = new (std::nothrow) cudaEvent_t[(size_t)n_iters * per];
  c->t_mask = new (std::nothrow) unsigned[n_iters];
  if (!c->tev || !c->t_mask) return set_err(c, NPG_ENOMEM, "host allocation failed");
  for (int k = 0; k < n_iters * per; ++k) {
    cudaError_t e = cudaEventCreate(&c->tev[k]);
    if (e != cudaSuccess) {
      for (int j = 0; j < k; ++j) cudaEventDestroy(c->tev[j]);
      delete[] c->tev;
      delete[] c->t_mask;
      c->tev = nullptr;
      c->t_mask = nullptr;
      return cuda_fail(c, e, "cudaEventCreate");
    }
  }
  for (int k = 0; k < n_iters; ++k) c->t_mask[k] = 0;
  c->t_slots = n_iters;
  c->t_next = 0;
  CK(c, cudaMemsetAsync(c->d_nnstats, 0, sizeof(unsigned long long) * 4, c->stream));
  return NPG_OK;
}

extern "C" int npg_search_stats(npg_ctx* c, long long* out4) {
  int rc = guard(c);
  if (rc) return rc;
  if (!out4) return set_err(c, NPG_EINVAL, "out4 is NULL");
  unsigned long long h[4];
  CK(c, cudaMemcpyAsync(h, c->d_nnstats, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  for (int k = 0; k < 4; ++k) out4[k] = (long long)h[k];
  return NPG_OK;
}

extern "C" int npg_timing_read(npg_ctx* c, int stage, double* total_ms, int* n_iters) {
  int rc = guard(c);
  if (rc) return rc;
  if (stage < 0 || stage >= NPG_NUM_STAGES || !total_ms || !n_iters)
    return set_err(c, NPG_EINVAL, "bad stage or NULL output");
  CK(c, cudaStreamSynchronize(c->stream));
  double tot = 0.0;
  int n = 0;
  const int per = NPG_NUM_STAGES + 1;
  const unsigned need = (1u << stage) | (1u << (stage + 1));
  for (int s = 0; s < c->t_next && s < c->t_slots; ++s) {
    if ((c->t_mask[s] & need) != need) continue;
    float ms = 0.f;
    CK(c, cudaEventElapsedTime(&ms, c->tev[s * per + stage], c->tev[s * per + stage + 1]));
    tot += ms;
    ++n;
  }
  *total_ms = tot;
  *n_iters = n;
  return NPG_OK;
}

extern "C" long long npg_launch_count(const npg_ctx* c) { return c ? c->launches : 0; }

// ----------------------------------------------------------------- autotuner
// Milliseconds per pass of `reps` forward passes (plus the loss when with_loss)
// at the current launch shapes, on the context's stream. Parameters, Adam
// state and e are untouched; the nearest-neighbour results (which are also
// the next search's seeds) are recomputed.
static int time_passes(npg_ctx* c, int reps, bool with_loss, float* ms) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(c, cudaEventCreate(&e0));
  cudaError_t ce = cudaEventCreate(&e1);
  if (ce != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_fail(c, ce, "cudaEventCreate");
  }
  int rc = forward_launch(c);  // warm-up at these shapes
  if (!rc && with_loss) rc = loss_launch(c);
  if (!rc) {
    cudaEventRecord(e0, c->stream);
    for (int k = 0; k < reps && !rc; ++k) {
      rc = forward_launch(c);
      if (!rc && with_loss) rc = loss_launch(c);
    }
    cudaEventRecord(e1, c->stream);
    ce = cudaEventSynchronize(e1);
    if (ce == cudaSuccess) ce = cudaEventElapsedTime(ms, e0, e1);
    if (ce != cudaSuccess) rc = cuda_fail(c, ce, "autotune timing");
    *ms /= (float)reps;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

extern "C" int npg_autotune(npg_ctx* c, int reps, int* chosen) {
  int rc = guard(c);
  if (rc) return rc;
  if (reps < 1 || reps > 100) return set_err(c, NPG_EINVAL, "reps out of 1..100");
  if (c->cfg.nn_cells > 0) return set_err(c, NPG_EINVAL, "nn_cells is fixed by the configuration");
  CK(c, cudaStreamSynchronize(c->stream));
  // search grids: the default resolution G scaled by 0.7 .. 1.25 (the search
  // stays exact at every resolution); the point side is rebuilt per candidate
  const int gx0 = c->xb.G, gp0 = c->pb.G;
  const double scale[4] = {0.7, 0.85, 1.0, 1.25};
  auto cand = [](int g0, double f, int cap) {
    return std::max(1, std::min(cap, (int)lround(g0 * f)));
  };
  float best = 0.f, ms = 0.f;
  int bx = gx0, bp = gp0;
  bool first = true;
  for (int k = 0; k < 4; ++k) {  // vertex side, point side at its default
    c->xb.G = cand(gx0, scale[k], c->G_cap_x);
    if ((rc = time_passes(c, reps, true, &ms))) return rc;
    if (first || ms < best) {
      best = ms;
      bx = c->xb.G;
      first = false;
    }
  }
  c->xb.G = bx;
  first = true;
  for (int k = 0; k < 4; ++k) {  // point side at the chosen vertex side
    c->pb.G = cand(gp0, scale[k], c->G_cap_p);
    if ((rc = build_point_buckets(c))) return rc;
    if ((rc = time_passes(c, reps, true, &ms))) return rc;
    if (first || ms < best) {
      best = ms;
      bp = c->pb.G;
      first = false;
    }
  }
  c->pb.G = bp;
  if ((rc = build_point_buckets(c))) return rc;
  // the widest seed ball that one thread covers before a query goes to the
  // lane-group pass, per search direction
  const int rows_opt[7] = {6, 12, 24, 48, 96, 192, 384};
  for (int dir = 0; dir < 2; ++dir) {
    NnQueue& qd = dir == 0 ? c->nnq : c->nnq_p;
    int brow = qd.near_rows;
    first = true;
    for (int k = 0; k < 7; ++k) {
      qd.near_rows = rows_opt[k];
      if ((rc = time_passes(c, reps, true, &ms))) return rc;
      if (first || ms < best) {
        best = ms;
        brow = rows_opt[k];
        first = false;
      }
    }
    qd.near_rows = brow;
  }
  // CTAs per SM of the BF16 decode (timed on the forward pass alone)
  if (c->cfg.precision == NPG_BF16_MLP && c->md.H == 64) {
    const int opts[4] = {3, 4, 6, 8};
    int bd = c->dec_per_sm;
    first = true;
    for (int k = 0; k < 4; ++k) {
      c->dec_per_sm = opts[k];
      if ((rc = time_passes(c, reps, false, &ms))) return rc;
      if (first || ms < best) {
        best = ms;
        bd = opts[k];
        first = false;
      }
    }
    c->dec_per_sm = bd;
  }
  // the shapes are baked into a captured iteration: capture it again
  if (c->graph_exec) {
    cudaGraphExecDestroy(c->graph_exec);
    cudaGraphDestroy(c->graph);
    c->graph_exec = nullptr;
    c->graph = nullptr;
  }
  c->phase = 0;
  if (chosen) {
    chosen[0] = c->xb.G;
    chosen[1] = c->pb.G;
    chosen[2] = c->dec_per_sm;
    chosen[3] = c->nnq.near_rows;
    chosen[4] = c->nnq_p.near_rows;
  }
  return NPG_OK;
}

// ----------------------------------------------------------------- evaluation
extern "C" int npg_evaluate(npg_ctx* c, const float* gt_xyz, int on_device, float tau_rel,
                            double* out) {
  int rc = guard(c);
  if (rc) return rc;
  if (!gt_xyz || !out || !(tau_rel > 0.f))
    return set_err(c, NPG_EINVAL, "npg_evaluate: gt_xyz and out non-NULL, tau_rel > 0");
  if (c->phase < 1) return set_err(c, NPG_ESTATE, "npg_evaluate needs a preceding npg_forward");
  const int N = c->N, T = c->T;
  const long long NT = (long long)N * T;
  const long long F_tri = (long long)c->faces_h.size() / 3;
  cudaStream_t s = c->stream;
  if (!c->d_faces && F_tri > 0) {  // vertex -> face lists, built once
    std::vector<int> off(N + 1, 0), vf(3 * F_tri);
    for (long long f = 0; f < F_tri; ++f)
      for (int k = 0; k < 3; ++k) off[c->faces_h[3 * f + k] + 1]++;
    for (int i = 0; i < N; ++i) off[i + 1] += off[i];
    std::vector<int> fill(off.begin(), off.end() - 1);
    for (long long f = 0; f < F_tri; ++f)
      for (int k = 0; k < 3; ++k) vf[fill[c->faces_h[3 * f + k]]++] = (int)f;
    if (!alloc_n(c, c->d_faces, F_tri) || !alloc_n(c, c->d_vf_off, N + 1) ||
        !alloc_n(c, c->d_vf, 3 * F_tri))
      return set_err(c, NPG_ENOMEM, "device allocation failed");
    if ((rc = copy_in(c, c->d_faces, c->faces_h.data(), sizeof(int32_t) * 3 * F_tri, 0)) ||
        (rc = copy_in(c, c->d_vf_off, off.data(), sizeof(int) * (N + 1), 0)) ||
        (rc = copy_in(c, c->d_vf, vf.data(), sizeof(int) * 3 * F_tri, 0)))
      return rc;
  }
  const int G = auto_cells(N, T);
  const long long G3 = (long long)G * G * G;
  const int split = eval_split(), terms = eval_terms();
  float4 *g4 = nullptr, *nx = nullptr, *ng = nullptr;
  float *gstage = nullptr, *d_x = nullptr, *d_g = nullptr, *tau2 = nullptr;
  int *idx_x = nullptr, *idx_g = nullptr;
  double* part = nullptr;
  Buckets xs, gs;
  NnQueue q;
  q.far_blocks = c->num_sms * 16;
  cudaError_t e = cudaSuccess;
  auto A = [&](void** p, size_t b) {
    if (e == cudaSuccess) e = cudaMallocAsync(p, b, s);
  };
  A((void**)&g4, sizeof(float4) * NT);
  if (!on_device) A((void**)&gstage, sizeof(float) * 3 * NT);
  A((void**)&nx, sizeof(float4) * NT);
  A((void**)&ng, sizeof(float4) * NT);
  A((void**)&idx_x, sizeof(int) * NT);
  A((void**)&idx_g, sizeof(int) * NT);
  A((void**)&d_x, sizeof(float) * NT);
  A((void**)&d_g, sizeof(float) * NT);
  A((void**)&tau2, sizeof(float) * T);
  A((void**)&part, sizeof(double) * T * split * terms);
  for (Buckets* b : {&xs, &gs}) {
    b->G = G;
    b->nsets = T;
    A((void**)&b->cell_start, sizeof(int) * T * (G3 + 1));
    A((void**)&b->counts, sizeof(int) * T * G3);
    A((void**)&b->slot, sizeof(int) * NT);
    A((void**)&b->sorted, sizeof(float4) * NT);
  }
  A((void**)&q.counters, sizeof(int) * 2);
  A((void**)&q.items, sizeof(int4) * NT);
  const float* gsrc = gt_xyz;
  if (e == cudaSuccess && !on_device) {
    e = cudaMemcpyAsync(gstage, gt_xyz, sizeof(float) * 3 * NT, cudaMemcpyHostToDevice, s);
    gsrc = gstage;
  }
  if (e == cudaSuccess) e = launch_points_to_float4(gsrc, g4, NT, s);
  if (e == cudaSuccess) e = launch_eval_tau(g4, N, T, tau_rel, tau2, s);
  if (e == cudaSuccess)
    e = launch_eval_normals(c->xhat, c->d_faces, c->d_vf_off, c->d_vf, N, NT, nx, s);
  if (e == cudaSuccess) e = launch_eval_normals(g4, c->d_faces, c->d_vf_off, c->d_vf, N, NT, ng, s);
  if (e == cudaSuccess) e = bucket_build(c->xhat, nullptr, N, T, NT, G, xs, s);
  if (e == cudaSuccess) e = bucket_build(g4, nullptr, N, T, NT, G, gs, s);
  if (e == cudaSuccess)
    e = launch_nn(xs.sorted, N, nullptr, T, NT, gs, nullptr, N, idx_x, d_x, q, s);
  if (e == cudaSuccess)
    e = launch_nn(gs.sorted, N, nullptr, T, NT, xs, nullptr, N, idx_g, d_g, q, s);
  if (e == cudaSuccess)
    e = launch_eval_frames(c->xhat, g4, nx, ng, idx_x, d_x, idx_g, d_g, tau2, N, T, part, s);
  std::vector<double> hp((size_t)T * split * terms);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(hp.data(), part, sizeof(double) * hp.size(), cudaMemcpyDeviceToHost, s);
  for (void* p : {(void*)g4, (void*)gstage, (void*)nx, (void*)ng, (void*)idx_x, (void*)idx_g,
                  (void*)d_x, (void*)d_g, (void*)tau2, (void*)part, (void*)q.counters,
                  (void*)q.items, (void*)xs.cell_start, (void*)xs.counts, (void*)xs.slot,
                  (void*)xs.sorted, (void*)gs.cell_start, (void*)gs.counts, (void*)gs.slot,
                  (void*)gs.sorted})
    if (p) cudaFreeAsync(p, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "npg_evaluate");
  double mean[6] = {0, 0, 0, 0, 0, 0};
  for (int t = 0; t < T; ++t) {
    double sum[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int b = 0; b < split; ++b)
      for (int m = 0; m < terms; ++m) sum[m] += hp[((size_t)t * split + b) * terms + m];
    double* o = out + 6 * (size_t)t;
    const double P = sum[2] / N, R = sum[3] / N;
    o[0] = (sum[0] + sum[1]) / N;
    o[1] = P;
    o[2] = R;
    o[3] = P + R > 0 ? 2 * P * R / (P + R) : 0.0;
    o[4] = 0.5 * (sum[4] + sum[5]) / N;
    o[5] = sum[6] / N;
    for (int m = 0; m < 6; ++m) mean[m] += o[m] / T;
  }
  for (int m = 0; m < 6; ++m) out[6 * (size_t)T + m] = mean[m];
  return NPG_OK;
}

// ----------------------------------------------------------------- batch
struct npg_batch {
  std::vector<npg_ctx*> ctx;
  cudaStream_t stream = nullptr;
  cudaEvent_t fork = nullptr, done = nullptr;
  std::vector<cudaEvent_t> join;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<long long> graph_launches;
  int width = 0;  // chains in the graph; 0: every sequence its own branch
};

extern "C" int npg_batch_destroy(npg_batch* b) {
  if (!b) return NPG_OK;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->done) cudaEventDestroy(b->done);
  for (cudaEvent_t e : b->join)
    if (e) cudaEventDestroy(e);
  cudaGetLastError();
  delete b;
  return NPG_OK;
}

extern "C" int npg_batch_create(npg_batch** out, int S, npg_ctx* const* ctxs, void* stream) {
  if (!out) return set_err(nullptr, NPG_EINVAL, "npg_batch_create: out is NULL");
  *out = nullptr;
  if (S < 1 || !ctxs || !stream)
    return set_err(nullptr, NPG_EINVAL, "npg_batch_create: S=%d, ctxs and stream non-NULL", S);
  cudaStream_t bs = static_cast<cudaStream_t>(stream);
  for (int i = 0; i < S; ++i) {
    npg_ctx* c = ctxs[i];
    if (!c) return set_err(nullptr, NPG_EINVAL, "npg_batch_create: context %d is NULL", i);
    if (int rc = guard(c)) return rc;
    if (!c->stream || c->stream == bs)
      return set_err(nullptr, NPG_EINVAL,
                     "npg_batch_create: context %d needs its own non-default stream", i);
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == c || ctxs[j]->stream == c->stream)
        return set_err(nullptr, NPG_EINVAL,
                       "npg_batch_create: contexts %d and %d share a stream", j, i);
  }
  npg_batch* b = new npg_batch;
  b->ctx.assign(ctxs, ctxs + S);
  b->stream = bs;
  b->join.assign(S, nullptr);
  b->graph_launches.assign(S, 0);
  cudaError_t e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming);
  for (int i = 0; i < S && e == cudaSuccess; ++i)
    e = cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming);
  if (e != cudaSuccess) {
    npg_batch_destroy(b);
    return cuda_fail(nullptr, e, "npg_batch_create: cudaEventCreate");
  }
  *out = b;
  return NPG_OK;
}

extern "C" int npg_batch_set_width(npg_batch* b, int width) {
  if (!b) return set_err(nullptr, NPG_EINVAL, "batch is NULL");
  if (b->exec)
    return set_err(nullptr, NPG_EINVAL, "npg_batch_set_width: the batch graph is already captured");
  b->width = width < 0 ? 0 : width;
  return NPG_OK;
}

// Chains of the batch graph: with `width` chains (0 or >= S: S chains of one
// sequence), the sequences go largest first (work N T + M T) onto the chain
// with the least work so far. Returns, per sequence, the index of the
// sequence it follows in its chain (-1: it starts its chain).
static std::vector<int> batch_chains(const npg_batch* b) {
  const int S = (int)b->ctx.size();
  std::vector<int> prev(S, -1);
  const int W = (b->width <= 0 || b->width >= S) ? S : b->width;
  if (W == S) return prev;
  std::vector<int> order(S);
  for (int i = 0; i < S; ++i) order[i] = i;
  auto work = [&](int i) {
    const npg_ctx* c = b->ctx[i];
    return (double)c->N * c->T + (double)c->MT;
  };
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return work(x) > work(y); });
  std::vector<double> load(W, 0.0);
  std::vector<int> tail(W, -1);
  for (int i : order) {
    int best = 0;
    for (int w = 1; w < W; ++w)
      if (load[w] < load[best]) best = w;
    prev[i] = tail[best];
    tail[best] = i;
    load[best] += work(i);
  }
  return prev;
}

// The batch stream waits for every context's stream (prior single-sequence work).
static cudaError_t batch_after_contexts(npg_batch* b) {
  for (size_t i = 0; i < b->ctx.size(); ++i) {
    cudaError_t e = cudaEventRecord(b->join[i], b->ctx[i]->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->join[i], 0);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Every context's stream waits for the batch stream (later single-sequence work).
static cudaError_t contexts_after_batch(npg_batch* b) {
  cudaError_t e = cudaEventRecord(b->done, b->stream);
  for (size_t i = 0; i < b->ctx.size() && e == cudaSuccess; ++i)
    e = cudaStreamWaitEvent(b->ctx[i]->stream, b->done, 0);
  return e;
}

static int batch_loss_out(npg_batch* b, double* loss_out) {
  if (!loss_out) return NPG_OK;
  for (size_t i = 0; i < b->ctx.size(); ++i)
    if (int rc = copy_loss_out(b->ctx[i], loss_out + 3 * i, nullptr)) return rc;
  return NPG_OK;
}

extern "C" int npg_batch_iteration(npg_batch* b, double* loss_out) {
  if (!b) return set_err(nullptr, NPG_EINVAL, "batch is NULL");
  for (npg_ctx* c : b->ctx)
    if (int rc = guard(c)) return rc;
  const int S = (int)b->ctx.size();
  if (!b->exec) {
    // one eager iteration of every sequence, each on its own stream (function
    // attributes and lazy module loading happen outside the capture)
    for (npg_ctx* c : b->ctx) {
      if (int rc = iteration_launch(c)) return rc;
      c->e += 1;
      c->phase = 0;
    }
    for (npg_ctx* c : b->ctx) CK(c, cudaStreamSynchronize(c->stream));
    // capture: the batch stream forks to the first context of every chain;
    // a later context of a chain waits for the one before it; every context
    // joins back into the batch stream
    const std::vector<int> prev = batch_chains(b);
    std::vector<int> seq_order;
    std::vector<char> placed(S, 0);
    while ((int)seq_order.size() < S)  // each context after the one it follows
      for (int i = 0; i < S; ++i)
        if (!placed[i] && (prev[i] < 0 || placed[prev[i]])) {
          placed[i] = 1;
          seq_order.push_back(i);
        }
    CK(nullptr, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    int rc = NPG_OK;
    cudaError_t ce = cudaEventRecord(b->fork, b->stream);
    for (int n = 0; n < S && ce == cudaSuccess && rc == NPG_OK; ++n) {
      const int i = seq_order[n];
      npg_ctx* c = b->ctx[i];
      ce = cudaStreamWaitEvent(c->stream, prev[i] < 0 ? b->fork : b->join[prev[i]], 0);
      if (ce != cudaSuccess) break;
      c->capturing = 1;
      const long long before = c->launches;
      rc = iteration_launch(c);
      c->capturing = 0;
      b->graph_launches[i] = c->launches - before;
      c->launches = before;
      if (rc) break;
      ce = cudaEventRecord(b->join[i], c->stream);
      if (ce == cudaSuccess) ce = cudaStreamWaitEvent(b->stream, b->join[i], 0);
    }
    cudaGraph_t g = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(b->stream, &g);
    if (rc || ce != cudaSuccess || ee != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      if (rc) return rc;
      return cuda_fail(nullptr, ce != cudaSuccess ? ce : ee, "npg_batch_iteration: capture");
    }
    b->graph = g;
    CK(nullptr, cudaGraphInstantiate(&b->exec, g, 0));
    // this call's iteration was the eager one; replays start with the next call
    return batch_loss_out(b, loss_out);
  }
  CK(nullptr, batch_after_contexts(b));
  CK(nullptr, cudaGraphLaunch(b->exec, b->stream));
  CK(nullptr, contexts_after_batch(b));
  for (int i = 0; i < S; ++i) {
    npg_ctx* c = b->ctx[i];
    c->e += 1;
    c->phase = 0;
    c->launches += b->graph_launches[i];
  }
  return batch_loss_out(b, loss_out);
}

extern "C" int npg_destroy(npg_ctx* c) {
  if (!c) return NPG_OK;
  if (c->stream || true) cudaStreamSynchronize(c->stream);
  for (int j = 1; j < npg_ctx::NLANE; ++j)
    if (c->lane[j]) {
      cudaStreamSynchronize(c->lane[j]);
      cudaStreamDestroy(c->lane[j]);
    }
  for (int j = 0; j < npg_ctx::NLANE; ++j)
    if (c->ev_join[j]) cudaEventDestroy(c->ev_join[j]);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  free_timing(c);
  if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
  if (c->graph) cudaGraphDestroy(c->graph);
  dev_free_all(c);
  if (c->h_loss) cudaFreeHost(c->h_loss);
  if (c->h_off) cudaFreeHost(c->h_off);
  cudaGetLastError();
  delete c;
  return NPG_OK;
}

extern "C" const char* npg_last_error(const npg_ctx* c) {
  if (c) return c->err.c_str();
  return g_thread_err.c_str();
}

// ----------------------------------------------------------------- standalone ops

extern "C" int npg_nearest(const float* q, int nq, const float* cand, int nc, int32_t* idx,
                           float* dist, int cells, void* stream) {
  if (nq < 0 || nc < 1 || (nq > 0 && (!q || !idx)) || !cand || cells < 0 || cells > 256)
    return set_err(nullptr, NPG_EINVAL, "npg_nearest: bad arguments (nq=%d nc=%d)", nq, nc);
  if (nq == 0) return NPG_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int G = cells > 0 ? cells : auto_cells(nc, 1);
  const long long G3 = (long long)G * G * G;
  Buckets cb, qb;
  cb.G = G;
  cb.nsets = 1;
  float4 *q4 = nullptr, *c4 = nullptr, *qs = nullptr;
  int *qslot = nullptr;
  NnQueue queue;
  queue.far_blocks = 152 * 16;
  auto cleanup = [&]() {
    cudaFreeAsync(q4, s); cudaFreeAsync(c4, s); cudaFreeAsync(qs, s); cudaFreeAsync(qslot, s);
    cudaFreeAsync(queue.counters, s); cudaFreeAsync(queue.items, s);
    cudaFreeAsync(cb.cell_start, s); cudaFreeAsync(cb.counts, s); cudaFreeAsync(cb.slot, s);
    cudaFreeAsync(cb.sorted, s); cudaFreeAsync(qb.cell_start, s); cudaFreeAsync(qb.counts, s);
  };
  cudaError_t e = cudaSuccess;
  auto A = [&](void** p, size_t b) {
    if (e == cudaSuccess) e = cudaMallocAsync(p, b, s);
  };
  A((void**)&q4, sizeof(float4) * nq);
  A((void**)&c4, sizeof(float4) * nc);
  A((void**)&qs, sizeof(float4) * nq);
  A((void**)&qslot, sizeof(int) * nq);
  A((void**)&cb.cell_start, sizeof(int) * (G3 + 1));
  A((void**)&cb.counts, sizeof(int) * G3);
  A((void**)&cb.slot, sizeof(int) * nc);
  A((void**)&cb.sorted, sizeof(float4) * nc);
  A((void**)&qb.cell_start, sizeof(int) * (G3 + 1));
  A((void**)&qb.counts, sizeof(int) * G3);
  A((void**)&queue.counters, sizeof(int) * 2);
  A((void**)&queue.items, sizeof(int4) * nq);
  if (e == cudaSuccess) e = launch_points_to_float4(q, q4, nq, s);
  if (e == cudaSuccess) e = launch_points_to_float4(cand, c4, nc, s);
  if (e == cudaSuccess) e = bucket_build(c4, nullptr, nc, 1, nc, G, cb, s);
  // queries sorted by the same cells (coherent warps)
  qb.G = G;
  qb.nsets = 1;
  qb.slot = qslot;
  qb.sorted = qs;
  if (e == cudaSuccess) e = bucket_build(q4, nullptr, nq, 1, nq, G, qb, s);
  if (e == cudaSuccess) e = launch_nn(qs, nq, nullptr, 1, nq, cb, nullptr, nc, idx, dist, queue, s);
  cleanup();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "npg_nearest");
  return NPG_OK;
}

extern "C" int npg_select_keyframe(const float* points, const int64_t* frame_offsets, int T,
                                   int on_device, double bias, double* extent_out,
                                   int* t_key_out, void* stream) {
  if (T < 1 || !points || !frame_offsets || !t_key_out || !(bias >= 0.0 && bias <= 1.0))
    return set_err(nullptr, NPG_EINVAL, "npg_select_keyframe: bad arguments (T=%d)", T);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::vector<long long> off(T + 1);
  cudaError_t e = cudaSuccess;
  if (on_device) {
    e = cudaMemcpyAsync(off.data(), frame_offsets, sizeof(long long) * (T + 1),
                        cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "npg_select_keyframe");
  } else {
    for (int t = 0; t <= T; ++t) off[t] = frame_offsets[t];
  }
  if (off[0] != 0) return set_err(nullptr, NPG_EINVAL, "frame_offsets[0] must be 0");
  for (int t = 0; t < T; ++t)
    if (off[t + 1] - off[t] < 1)
      return set_err(nullptr, NPG_EINVAL, "frame %d has no points (every frame needs one)", t);
  const long long MT = off[T];
  const float* d_pts = on_device ? points : nullptr;
  float* own_pts = nullptr;
  long long* d_off = nullptr;
  double* d_ext = nullptr;
  if (!on_device) {
    e = cudaMallocAsync((void**)&own_pts, sizeof(float) * 3 * MT, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(own_pts, points, sizeof(float) * 3 * MT, cudaMemcpyHostToDevice, s);
    d_pts = own_pts;
  }
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&d_off, sizeof(long long) * (T + 1), s);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&d_ext, sizeof(double) * T, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_off, off.data(), sizeof(long long) * (T + 1), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = launch_keyframe_extent(d_pts, d_off, T, d_ext, s);
  std::vector<double> ext(T);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ext.data(), d_ext, sizeof(double) * T, cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(own_pts, s);
  cudaFreeAsync(d_off, s);
  cudaFreeAsync(d_ext, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "npg_select_keyframe");
  // rating and choice on the host, in FP64 (lowest frame on ties)
  int best = 0;
  double best_s = -1.0;
  for (int t = 0; t < T; ++t) {
    const double tt = T > 1 ? (double)t / (double)(T - 1) : 0.5;
    const double sc = (1.0 - bias * fabs(tt - 0.5)) * ext[t];
    if (sc > best_s) {
      best_s = sc;
      best = t;
    }
    if (extent_out) extent_out[t] = ext[t];
  }
  *t_key_out = best;
  return NPG_OK;
}

extern "C" int npg_precondition_tc(const float* g, float* out, int r, int F, float lambda,
                                   void* stream) {
  if (!g || !out || r < 2 || r > 256 || F < 1 || F > NPG_MAX_F || !(lambda >= 0.f))
    return set_err(nullptr, NPG_EINVAL, "npg_precondition_tc: bad arguments (r=%d F=%d)", r, F);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const long long n = (long long)r * r * r * F;
  std::vector<float> tab(2LL * r * r + r);
  dct_tables(r, tab.data(), tab.data() + (long long)r * r, tab.data() + 2LL * r * r);
  const size_t te = dct_tc_table_elems(r);
  std::vector<uint16_t> tt(2 * te);
  dct_tc_tables(r, tab.data(), tt.data());
  dct_tc_tables(r, tab.data() + (long long)r * r, tt.data() + te);
  float *t0 = nullptr, *t1 = nullptr, *dmu = nullptr;
  uint16_t* dtt = nullptr;
  int* derr = nullptr;
  const long long nt = std::max(n, (long long)dct_tc_scratch_elems(r, F));
  cudaError_t e = cudaMallocAsync((void**)&t0, sizeof(float) * nt, s);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&t1, sizeof(float) * nt, s);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&dmu, sizeof(float) * r, s);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&dtt, sizeof(uint16_t) * tt.size(), s);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&derr, sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(derr, 0, sizeof(int), s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dmu, tab.data() + 2LL * r * r, sizeof(float) * r, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dtt, tt.data(), sizeof(uint16_t) * tt.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = launch_precondition_tc(g, out, t0, t1, dtt, dtt + te, dmu, r, F, lambda, derr, s);
  int herr = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(t0, s);
  cudaFreeAsync(t1, s);
  cudaFreeAsync(dmu, s);
  cudaFreeAsync(dtt, s);
  cudaFreeAsync(derr, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "npg_precondition_tc");
  if (herr) return set_err(nullptr, NPG_ETIMEOUT, "npg_precondition_tc: a tensor-core wait timed out");
  return NPG_OK;
}

extern "C" int npg_precondition(const float* g, float* out, int r, int F, float lambda,
                                void* stream) {
  if (!g || !out || r < 2 || r > 512 || F < 1 || F > NPG_MAX_F || !(lambda >= 0.f))
    return set_err(nullptr, NPG_EINVAL, "npg_precondition: bad arguments (r=%d F=%d)", r, F);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const long long n = (long long)r * r * r * F;
  std::vector<float> tab(2LL * r * r + r);
  dct_tables(r, tab.data(), tab.data() + (long long)r * r, tab.data() + 2LL * r * r);
  float *t0 = nullptr, *t1 = nullptr, *dtab = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&t0, sizeof(float) * n, s);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&t1, sizeof(float) * n, s);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&dtab, sizeof(float) * tab.size(), s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dtab, tab.data(), sizeof(float) * tab.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = launch_precondition(g, out, t0, t1, dtab, dtab + (long long)r * r, dtab + 2LL * r * r, r,
                            F, lambda, s);
  cudaFreeAsync(t0, s);
  cudaFreeAsync(t1, s);
  cudaFreeAsync(dtab, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "npg_precondition");
  return NPG_OK;
}
