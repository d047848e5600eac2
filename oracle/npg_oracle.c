/*
 * Neu-PiG per-sequence optimization: plain, slow FP64 CPU oracle.
 *
 * TEST INFRASTRUCTURE. Only the test suite, the package's smoke check and the
 * benchmark's CPU-baseline leg load this library. The product path (libnpg.so
 * and its Python binding) never calls, links or includes anything here, and
 * this file includes nothing from the product path.
 *
 * Every routine restates the paper's definitions directly, in the paper's
 * order and notation, with no blocking, fusion or reordering:
 *   Sec. 3.2  multi-resolution latent grids, trilinear lookup, Eq. 1 level mean
 *   Sec. 3.3  input vector (Eq. 2), Fourier time encoding (Eq. 3), MLP (Eq. 4)
 *   Sec. 3.4  quaternion offset + normalisation (Eq. 5), tanh translation
 *             (Eq. 6), rigid transform (Eq. 7); supplementary rotation study:
 *             exponential map
 *   Sec. 3.5  total loss (Eq. 8), Sobolev preconditioner (Eq. 9), L_def
 *             (Eq. 10), confidence weight (Eq. 11-12), L_iso (Eq. 13), Adam
 *             with per-level learning rates (implementation details)
 * The reverse-mode gradient is written by hand, step by step, in the reverse
 * order of the forward pass. The preconditioner solves (I + lambda L) u = g
 * twice by conjugate gradients in FP64.
 *
 * Readings where the paper is silent (each mirrored by the GPU library):
 *   - nodes sit at -1 + 2k/(r-1) per axis; queries are clamped to [-1,1];
 *     the cell index is min(floor(u), r-2); corner c = bx + 2 by + 4 bz;
 *     node (ix,iy,iz) is stored at ((iz r + iy) r + ix), features innermost.
 *   - the Chamfer distance is the plain bidirectional squared-L2 one:
 *     cd = mean_i min_j |x_i - p_j|^2 + mean_j min_i |p_j - x_i|^2; nearest
 *     neighbour ties go to the lowest index.
 *   - the Laplacian is the combinatorial graph Laplacian of the 6-connected
 *     node lattice (natural Neumann boundary), applied per feature channel.
 *   - the preconditioned gradient replaces the raw gradient as Adam's input
 *     for grid parameters; MLP parameters use the raw gradient.
 *   - L_iso reference lengths are the current keyframe lengths, stop-grad;
 *     d|u|/du at u = 0 is 0 and d|e|/de at e = 0 is 0.
 *   - frames are 0-based here; t~ = t / (T-1) (t~ = 0 when T = 1); the
 *     Fourier features are interleaved (sin_1, cos_1, ..., sin_M, cos_M).
 *   - a zero-norm quaternion (1 + q_w = q_x = q_y = q_z = 0) maps to the
 *     identity rotation with zero gradient.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAX_LEVELS 16

typedef struct {
  int L;                   /* number of position-grid levels                 */
  int res[OR_MAX_LEVELS];  /* nodes per axis of level l (l = 0 is coarsest)  */
  int F;                   /* features per position-grid node                */
  int Fn;                  /* features per normal-grid node                  */
  int rn;                  /* nodes per axis of the normal grid              */
  int H;                   /* hidden width                                   */
  int D;                   /* number of hidden layers                        */
  int rot_mode;            /* 0: quaternion (Eq. 5), 1: exponential map,
                              2: Cayley transform                            */
  int n_freq;              /* Fourier frequencies M (Eq. 3)                  */
  double slope;            /* LeakyReLU negative slope                       */
  double alpha;            /* translation squashing factor (Eq. 6)           */
  double w_iso;            /* isometry weight (Eq. 8)                        */
  /* variants of the ablations (Sec. 4): 0 is the method itself */
  int time_enc;            /* time encoding: 0 Fourier (Eq. 3), 1 polynomial,
                              2 Gaussian Fourier with frequencies time_B,
                              3 learned: psi_t(t~), a two-layer MLP           */
  double time_B[8];        /* Gaussian Fourier frequencies B_j (j < n_freq)  */
  int conf_delta;          /* catch-up delta: 0 1 - sqrt(e~), 1 constant 1,
                              2 linear 1 - e~, 3 exp(-5 e~), 4 interpolated  */
  int conf_omega;          /* 0 cumulative product of omega (Eq. 11-12);
                              direct w = omega(t)^delta with omega 1 constant,
                              2 one half, 3 the single-frame omega(t)        */
  int Ht;                  /* hidden width of the learned time embedding
                              psi_t (time_enc 3)                             */
} or_cfg;

/* ---------------------------------------------------------------- threads */

/* Loops over independent queries, rows and lattice nodes may run on several
 * host threads (OpenMP, when compiled with it); every such loop writes
 * disjoint outputs and has no reduction, so results do not depend on the
 * thread count. Returns the thread count in effect (1 without OpenMP). */
int or_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

/* ------------------------------------------------------------------ sizes */

int or_n_out(const or_cfg* c) { return c->rot_mode == 0 ? 7 : 6; }
int or_k_in(const or_cfg* c) { return c->Fn + c->F + 2 * c->n_freq; }

static long cube(long r) { return r * r * r; }

/* Offset of level l's block in the flat grid vector; l == L is the normal grid. */
long or_level_offset(const or_cfg* c, int l) {
  long off = 0;
  for (int k = 0; k < l && k < c->L; ++k) off += cube(c->res[k]) * c->F;
  return off;
}

long or_grid_len(const or_cfg* c) {
  return or_level_offset(c, c->L) + cube(c->rn) * c->Fn;
}

/* MLP layout: layer 0 W (H x K) row-major then b (H); hidden layers
 * 1..D-1 W (H x H), b (H); output layer W (O x H), b (O). */
/* Parameters of psi_t (time_enc 3), stored after the decoder's: first layer
 * a, b (Ht each: h = act(a t~ + b)), then W (2M x Ht, row-major) and c (2M):
 * gamma = W h + c. Zero for the other encodings. */
long or_time_params(const or_cfg* c) {
  long Ht = c->Ht, G2 = 2L * c->n_freq;
  return c->time_enc == 3 ? 2 * Ht + G2 * Ht + G2 : 0;
}

static long decoder_len(const or_cfg* c) {
  long K = or_k_in(c), H = c->H, D = c->D, O = or_n_out(c);
  return H * K + H + (D - 1) * (H * H + H) + O * H + O;
}

long or_mlp_len(const or_cfg* c) { return decoder_len(c) + or_time_params(c); }

/* -------------------------------------------- Sec. 3.2: trilinear lookup */

void or_trilinear(int r, const double* p, long* idx, double* w) {
  long i0[3];
  double f[3];
  for (int a = 0; a < 3; ++a) {
    double q = p[a];
    if (q < -1.0) q = -1.0;
    if (q > 1.0) q = 1.0;
    double u = (q + 1.0) * 0.5 * (double)(r - 1);
    long i = (long)floor(u);
    if (i > r - 2) i = r - 2;
    if (i < 0) i = 0;
    i0[a] = i;
    f[a] = u - (double)i;
  }
  for (int c = 0; c < 8; ++c) {
    int bx = c & 1, by = (c >> 1) & 1, bz = (c >> 2) & 1;
    idx[c] = ((i0[2] + bz) * r + (i0[1] + by)) * r + (i0[0] + bx);
    w[c] = (bx ? f[0] : 1.0 - f[0]) * (by ? f[1] : 1.0 - f[1]) *
           (bz ? f[2] : 1.0 - f[2]);
  }
}

/* Sec. 3.2: z_p(x) = (1/L) sum_l z_p^l(x) (Eq. 1); z_n(n) from the normal grid.
 * z is N x (Fn + F), ordered (z_n, z_p) as in the input vector of Eq. 2. */
void or_encode(const or_cfg* c, int N, const double* x, const double* n,
               const double* grid, double* z) {
  int F = c->F, Fn = c->Fn, Z = Fn + F;
  long idx[8];
  double w[8];
  for (int i = 0; i < N; ++i) {
    double* zi = z + (long)i * Z;
    for (int k = 0; k < Z; ++k) zi[k] = 0.0;
    or_trilinear(c->rn, n + 3L * i, idx, w);
    const double* gn = grid + or_level_offset(c, c->L);
    for (int k = 0; k < 8; ++k)
      for (int f = 0; f < Fn; ++f) zi[f] += w[k] * gn[idx[k] * Fn + f];
    for (int l = 0; l < c->L; ++l) {
      const double* gl = grid + or_level_offset(c, l);
      or_trilinear(c->res[l], x + 3L * i, idx, w);
      for (int k = 0; k < 8; ++k)
        for (int f = 0; f < F; ++f)
          zi[Fn + f] += w[k] * gl[idx[k] * F + f] / (double)c->L;
    }
  }
}

/* ------------------------------------- Sec. 3.3, Eq. 3: time embedding */

/* Sec. 3.3, Eq. 3 (and the ablation's variants): time_enc 1 is the
 * polynomial basis gamma_j = t~^j, j = 1..2M; time_enc 2 the Gaussian Fourier
 * mapping (sin(2 pi B_j t~), cos(2 pi B_j t~)) with given B, interleaved
 * like Eq. 3. */
void or_time_embedding(const or_cfg* c, int T, double* gamma) {
  const double pi = 3.14159265358979323846;
  int M = c->n_freq;
  for (int t = 0; t < T; ++t) {
    double tt = T > 1 ? (double)t / (double)(T - 1) : 0.0;
    double* g = gamma + (long)t * 2 * M;
    if (c->time_enc == 1) {
      for (int j = 0; j < 2 * M; ++j) g[j] = pow(tt, (double)(j + 1));
      continue;
    }
    for (int j = 0; j < M; ++j) {
      double a = c->time_enc == 2 ? 2.0 * c->time_B[j] * tt
                                  : ldexp(1.0, j) * tt; /* nu_j = 2^(j-1), 1-based */
      g[2 * j] = sin(pi * a);
      g[2 * j + 1] = cos(pi * a);
    }
  }
}

/* ------------------------------------------ Sec. 3.3: the MLP psi (Eq. 4) */

static double act(double s, double slope) { return s > 0.0 ? s : slope * s; }
static double dact(double s, double slope) { return s > 0.0 ? 1.0 : slope; }

/* The time embedding of every frame from the parameter vector mlp: the
 * learned one of the ablation (time_enc 3: gamma(t) = psi_t(t~), a two-layer
 * MLP with Ht hidden units and the decoder's activation, parameters after the
 * decoder's), else the fixed encodings of or_time_embedding. */
void or_time_embedding_params(const or_cfg* c, const double* mlp, int T, double* gamma) {
  if (c->time_enc != 3) {
    or_time_embedding(c, T, gamma);
    return;
  }
  int Ht = c->Ht, G2 = 2 * c->n_freq;
  const double* a = mlp + decoder_len(c);
  const double* b = a + Ht;
  const double* W = b + Ht;
  const double* cc = W + (long)G2 * Ht;
  for (int t = 0; t < T; ++t) {
    double tt = T > 1 ? (double)t / (double)(T - 1) : 0.0;
    for (int k = 0; k < G2; ++k) {
      double s = cc[k];
      for (int j = 0; j < Ht; ++j) s += W[(long)k * Ht + j] * act(a[j] * tt + b[j], c->slope);
      gamma[(long)t * G2 + k] = s;
    }
  }
}

/* One row: pre[k*H + j] and h[k*H + j] for hidden layer k, then o (O). */
static void mlp_row(const or_cfg* c, const double* mlp, const double* y,
                    double* pre, double* h, double* o) {
  int K = or_k_in(c), H = c->H, D = c->D, O = or_n_out(c);
  const double* W = mlp;
  const double* b = W + (long)H * K;
  for (int j = 0; j < H; ++j) {
    double s = b[j];
    for (int k = 0; k < K; ++k) s += W[(long)j * K + k] * y[k];
    pre[j] = s;
    h[j] = act(s, c->slope);
  }
  const double* p = b + H;
  for (int layer = 1; layer < D; ++layer) {
    W = p;
    b = W + (long)H * H;
    p = b + H;
    const double* hin = h + (long)(layer - 1) * H;
    for (int j = 0; j < H; ++j) {
      double s = b[j];
      for (int k = 0; k < H; ++k) s += W[(long)j * H + k] * hin[k];
      pre[(long)layer * H + j] = s;
      h[(long)layer * H + j] = act(s, c->slope);
    }
  }
  W = p;
  b = W + (long)O * H;
  const double* hl = h + (long)(D - 1) * H;
  for (int j = 0; j < O; ++j) {
    double s = b[j];
    for (int k = 0; k < H; ++k) s += W[(long)j * H + k] * hl[k];
    o[j] = s;
  }
}

void or_mlp_forward(const or_cfg* c, const double* mlp, int rows,
                    const double* y, double* o) {
  int H = c->H, D = c->D, K = or_k_in(c), O = or_n_out(c);
  double* pre = (double*)malloc(sizeof(double) * H * D);
  double* h = (double*)malloc(sizeof(double) * H * D);
  for (int r = 0; r < rows; ++r)
    mlp_row(c, mlp, y + (long)r * K, pre, h, o + (long)r * O);
  free(pre);
  free(h);
}

/* ---------------------------------------- Sec. 3.4: transformation mapping */

static void quat_to_R(const double* q, double* R) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z); R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z); R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y); R[7] = 2 * (y * z + w * x); R[8] = 1 - 2 * (x * x + y * y);
}

/* Exponential map R = I + A K + B K^2, K = [w]x, A = sin t / t, B = (1-cos t)/t^2,
 * with the Taylor series below t = 1e-2. Also returns A'/t and B'/t. */
static void expmap_coeffs(double th, double* A, double* B, double* dA, double* dB) {
  double t2 = th * th;
  if (th < 1e-2) {
    *A = 1.0 - t2 / 6.0 + t2 * t2 / 120.0;
    *B = 0.5 - t2 / 24.0 + t2 * t2 / 720.0;
    *dA = -1.0 / 3.0 + t2 / 30.0 - t2 * t2 / 840.0;
    *dB = -1.0 / 12.0 + t2 / 180.0 - t2 * t2 / 6720.0;
  } else {
    double s = sin(th), co = cos(th), omc = 2.0 * sin(0.5 * th) * sin(0.5 * th);
    *A = s / th;
    *B = omc / t2;
    *dA = (th * co - s) / (t2 * th);
    *dB = (th * s - 2.0 * omc) / (t2 * t2);
  }
}

/* Cayley transform (the rotation-representation ablation, Sec. 4):
 * R = (I - K)^-1 (I + K) with K = [w]x, in closed form I + c (K + K^2),
 * c = 2 / (1 + |w|^2); as for the exponential map, dA = dB = (dc/d|w|) / |w|. */
static void cayley_coeffs(double th, double* A, double* B, double* dA, double* dB) {
  const double cc = 2.0 / (1.0 + th * th);
  *A = *B = cc;
  *dA = *dB = -cc * cc;
}

static void rot_coeffs(int rot_mode, double th, double* A, double* B, double* dA, double* dB) {
  if (rot_mode == 2)
    cayley_coeffs(th, A, B, dA, dB);
  else
    expmap_coeffs(th, A, B, dA, dB);
}

static void skew(const double* w, double* K) {
  K[0] = 0; K[1] = -w[2]; K[2] = w[1];
  K[3] = w[2]; K[4] = 0; K[5] = -w[0];
  K[6] = -w[1]; K[7] = w[0]; K[8] = 0;
}

static void matmul3(const double* A, const double* B, double* C) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0;
      for (int k = 0; k < 3; ++k) s += A[i * 3 + k] * B[k * 3 + j];
      C[i * 3 + j] = s;
    }
}

static void expmap_R(int rot_mode, const double* w, double* R) {
  double th = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
  double A, B, dA, dB, K[9], K2[9];
  rot_coeffs(rot_mode, th, &A, &B, &dA, &dB);
  skew(w, K);
  matmul3(K, K, K2);
  for (int i = 0; i < 9; ++i) R[i] = (i % 4 == 0 ? 1.0 : 0.0) + A * K[i] + B * K2[i];
}

/* Rotation matrix R (row-major) and translation d-hat from one output row o. */
void or_rotation_translation(const or_cfg* c, const double* o, double* R, double* d) {
  if (c->rot_mode == 0) {
    double q[4] = {1.0 + o[0], o[1], o[2], o[3]};
    double nq = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    if (nq > 0.0) {
      for (int k = 0; k < 4; ++k) q[k] /= nq;
    } else {
      q[0] = 1.0; q[1] = q[2] = q[3] = 0.0;
    }
    quat_to_R(q, R);
    for (int a = 0; a < 3; ++a) d[a] = tanh(c->alpha * o[4 + a]);
  } else {
    expmap_R(c->rot_mode, o, R);
    for (int a = 0; a < 3; ++a) d[a] = tanh(c->alpha * o[3 + a]);
  }
}

/* Eq. 7: x-hat = R(q-hat) x + d-hat. */
static void transform_row(const or_cfg* c, const double* o, const double* x, double* xh) {
  double R[9], d[3];
  or_rotation_translation(c, o, R, d);
  for (int a = 0; a < 3; ++a)
    xh[a] = R[a * 3 + 0] * x[0] + R[a * 3 + 1] * x[1] + R[a * 3 + 2] * x[2] + d[a];
}

/* Given g = dL/dx-hat of one row, write dL/do (length O). */
static void transform_row_backward(const or_cfg* c, const double* o, const double* x,
                                   const double* g, double* go) {
  double G[9];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) G[a * 3 + b] = g[a] * x[b];
  if (c->rot_mode == 0) {
    double q[4] = {1.0 + o[0], o[1], o[2], o[3]};
    double nq = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    if (nq > 0.0) {
      double w = q[0] / nq, X = q[1] / nq, Y = q[2] / nq, Z = q[3] / nq;
      double gq[4];
      gq[0] = 2 * (-Z * G[1] + Y * G[2] + Z * G[3] - X * G[5] - Y * G[6] + X * G[7]);
      gq[1] = 2 * (Y * G[1] + Z * G[2] + Y * G[3] - 2 * X * G[4] - w * G[5] + Z * G[6] +
                   w * G[7] - 2 * X * G[8]);
      gq[2] = 2 * (-2 * Y * G[0] + X * G[1] + w * G[2] + X * G[3] + Z * G[5] - w * G[6] +
                   Z * G[7] - 2 * Y * G[8]);
      gq[3] = 2 * (-2 * Z * G[0] - w * G[1] + X * G[2] + w * G[3] - 2 * Z * G[4] + Y * G[5] +
                   X * G[6] + Y * G[7]);
      double qh[4] = {w, X, Y, Z};
      double dot = 0;
      for (int k = 0; k < 4; ++k) dot += qh[k] * gq[k];
      for (int k = 0; k < 4; ++k) go[k] = (gq[k] - qh[k] * dot) / nq;
    } else {
      for (int k = 0; k < 4; ++k) go[k] = 0.0;
    }
    for (int a = 0; a < 3; ++a) {
      double th = tanh(c->alpha * o[4 + a]);
      go[4 + a] = g[a] * c->alpha * (1.0 - th * th);
    }
  } else {
    const double* w = o;
    double th = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    double A, B, dA, dB, K[9], K2[9];
    rot_coeffs(c->rot_mode, th, &A, &B, &dA, &dB);
    skew(w, K);
    matmul3(K, K, K2);
    for (int k = 0; k < 3; ++k) {
      double e[3] = {0, 0, 0}, Ek[9], EK[9], KE[9];
      e[k] = 1.0;
      skew(e, Ek);
      matmul3(Ek, K, EK);
      matmul3(K, Ek, KE);
      double s = 0;
      for (int i = 0; i < 9; ++i) {
        double dR = dA * w[k] * K[i] + A * Ek[i] + dB * w[k] * K2[i] + B * (EK[i] + KE[i]);
        s += G[i] * dR;
      }
      go[k] = s;
    }
    for (int a = 0; a < 3; ++a) {
      double t = tanh(c->alpha * o[3 + a]);
      go[3 + a] = g[a] * c->alpha * (1.0 - t * t);
    }
  }
}

/* Full decode of all rows (i, t): y = (z_i, gamma_t) (Eq. 2), o = psi(y),
 * x-hat[t][i] = R x_i + d (Eq. 5-7). xhat is T x N x 3. */
void or_decode(const or_cfg* c, int N, int T, const double* x, const double* z,
               const double* gamma, const double* mlp, double* xhat) {
  int K = or_k_in(c), Z = c->Fn + c->F, G2 = 2 * c->n_freq;
  int H = c->H, D = c->D;
  long rows = (long)N * T;
#pragma omp parallel
  {
    double* y = (double*)malloc(sizeof(double) * K);
    double* pre = (double*)malloc(sizeof(double) * H * D);
    double* h = (double*)malloc(sizeof(double) * H * D);
    double o[8];
#pragma omp for schedule(static)
    for (long row = 0; row < rows; ++row) {
      long t = row / N, i = row % N;
      for (int k = 0; k < Z; ++k) y[k] = z[i * Z + k];
      for (int k = 0; k < G2; ++k) y[Z + k] = gamma[t * G2 + k];
      mlp_row(c, mlp, y, pre, h, o);
      transform_row(c, o, x + 3L * i, xhat + (t * N + i) * 3);
    }
    free(y);
    free(pre);
    free(h);
  }
}

/* ------------------------------------------- Sec. 3.5: Chamfer distance */

/* Brute-force nearest neighbour of each query among the candidates; ties go
 * to the lowest index. decide_f32 != 0 takes the argmin decision in FP32 on
 * the inputs rounded to float, with the distance formed as
 * d = dx*dx; d = fma(dy, dy, d); d = fma(dz, dz, d). The returned distance is
 * always the FP64 squared distance of the chosen pair. */
void or_nn(int nq, const double* q, int nc, const double* cand, int decide_f32,
           int32_t* idx, double* dist) {
#pragma omp parallel for schedule(dynamic, 64)
  for (int i = 0; i < nq; ++i) {
    const double* a = q + 3L * i;
    int best = -1;
    if (decide_f32) {
      float ax = (float)a[0], ay = (float)a[1], az = (float)a[2];
      float bd = 0.0f;
      for (int j = 0; j < nc; ++j) {
        float dx = ax - (float)cand[3L * j];
        float dy = ay - (float)cand[3L * j + 1];
        float dz = az - (float)cand[3L * j + 2];
        float d = dx * dx;
        d = fmaf(dy, dy, d);
        d = fmaf(dz, dz, d);
        if (best < 0 || d < bd) { bd = d; best = j; }
      }
    } else {
      double bd = 0.0;
      for (int j = 0; j < nc; ++j) {
        double dx = a[0] - cand[3L * j], dy = a[1] - cand[3L * j + 1], dz = a[2] - cand[3L * j + 2];
        double d = dx * dx + dy * dy + dz * dz;
        if (best < 0 || d < bd) { bd = d; best = j; }
      }
    }
    idx[i] = best;
    const double* b = cand + 3L * best;
    double dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
    dist[i] = dx * dx + dy * dy + dz * dz;
  }
}

/* cd_t of Eq. 10's Chamfer term for given nearest-neighbour choices: the mean
 * squared distance of every vertex to its chosen point plus that of every
 * point to its chosen vertex, FP64, summed in index order. nn_x is T x N
 * (frame-local point indices), nn_p follows the point order. */
void or_chamfer_from_nn(int T, int N, const double* xhat, const int64_t* off, const double* pts,
                        const int32_t* nn_x, const int32_t* nn_p, double* cd) {
  for (int t = 0; t < T; ++t) {
    const double* X = xhat + (long)t * N * 3;
    long M = off[t + 1] - off[t];
    const double* P = pts + 3 * off[t];
    double sx = 0, sp = 0;
    for (int i = 0; i < N; ++i) {
      const double* a = X + 3L * i;
      const double* b = P + 3L * nn_x[(long)t * N + i];
      double dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
      sx += dx * dx + dy * dy + dz * dz;
    }
    for (long j = 0; j < M; ++j) {
      const double* a = P + 3L * j;
      const double* b = X + 3L * nn_p[off[t] + j];
      double dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
      sp += dx * dx + dy * dy + dz * dz;
    }
    cd[t] = sx / N + sp / (double)M;
  }
}

/* Per frame t: cd_t = mean_i min_j |x-hat_i - p_j|^2 + mean_j min_i |p_j - x-hat_i|^2.
 * off has T+1 entries; points of frame t are pts[off[t] .. off[t+1]).
 * nn_x, d_x are T x N; nn_p, d_p follow the point order (off[T] entries). */
void or_chamfer(int T, int N, const double* xhat, const int64_t* off, const double* pts,
                int decide_f32, int32_t* nn_x, double* d_x, int32_t* nn_p, double* d_p,
                double* cd) {
  for (int t = 0; t < T; ++t) {
    const double* X = xhat + (long)t * N * 3;
    long M = off[t + 1] - off[t];
    const double* P = pts + 3 * off[t];
    or_nn(N, X, (int)M, P, decide_f32, nn_x + (long)t * N, d_x + (long)t * N);
    or_nn((int)M, P, N, X, decide_f32, nn_p + off[t], d_p + off[t]);
  }
  or_chamfer_from_nn(T, N, xhat, off, pts, nn_x, nn_p, cd);
}

/* ---------------------------------- Sec. 3.5, Eq. 11-12: confidence weight */

/* w(t) = prod_{tau between t_key and t, inclusive} omega(tau)^delta,
 * omega(tau) = 1 / (1 + max(0, cd_tau - cd_tkey)), delta = 1 - sqrt(e / e_max)
 * with e / e_max clamped to [0, 1]. */
/* The ablation's schedules (Sec. 4, stability function): delta_mode picks
 * the catch-up variable (0: 1 - sqrt(e~), the method; 1: 1; 2: 1 - e~;
 * 3: exp(-5 e~); 4: interpolated, w = (1 - e~) W(t) + e~ with W(t) the
 * weight at delta = 1), omega_mode the temporal weighting (0: the cumulative
 * product of Eq. 11-12; 1, 2, 3: direct w = omega(t)^delta with omega = 1,
 * 0.5, or 1 / (1 + max(0, cd_t - cd_key))). */
void or_conf_weights_mode(int T, const double* cd, int t_key, double e, double e_max,
                          int delta_mode, int omega_mode, double* w) {
  double eb = e_max > 0 ? e / e_max : 1.0;
  if (eb < 0) eb = 0;
  if (eb > 1) eb = 1;
  double delta = 1.0 - sqrt(eb);
  if (delta_mode == 1 || delta_mode == 4) delta = 1.0;
  if (delta_mode == 2) delta = 1.0 - eb;
  if (delta_mode == 3) delta = exp(-5.0 * eb);
  for (int t = 0; t < T; ++t) {
    double wt;
    if (omega_mode == 0) {
      int lo = t < t_key ? t : t_key, hi = t < t_key ? t_key : t;
      double prod = 1.0;
      for (int tau = lo; tau <= hi; ++tau) {
        double ex = cd[tau] - cd[t_key];
        double om = 1.0 / (1.0 + (ex > 0 ? ex : 0.0));
        prod *= pow(om, delta);
      }
      wt = prod;
    } else {
      double ex = cd[t] - cd[t_key];
      double om = omega_mode == 1 ? 1.0
                : omega_mode == 2 ? 0.5
                                  : 1.0 / (1.0 + (ex > 0 ? ex : 0.0));
      wt = pow(om, delta);
    }
    w[t] = delta_mode == 4 ? (1.0 - eb) * wt + eb : wt;
  }
}

void or_conf_weights(int T, const double* cd, int t_key, double e, double e_max, double* w) {
  or_conf_weights_mode(T, cd, t_key, e, e_max, 0, 0, w);
}

/* ------------------------------------------------------ mesh edges */

static int cmp_edge(const void* a, const void* b) {
  const int32_t* x = (const int32_t*)a;
  const int32_t* y = (const int32_t*)b;
  if (x[0] != y[0]) return x[0] < y[0] ? -1 : 1;
  if (x[1] != y[1]) return x[1] < y[1] ? -1 : 1;
  return 0;
}

/* Unique undirected edges (i < j), sorted; edges must hold 3 * F_tri pairs.
 * Returns the number of edges. */
long or_edges(int F_tri, const int32_t* faces, int32_t* edges) {
  long n = 0;
  for (int f = 0; f < F_tri; ++f)
    for (int k = 0; k < 3; ++k) {
      int32_t a = faces[3L * f + k], b = faces[3L * f + (k + 1) % 3];
      if (a == b) continue;
      edges[2 * n] = a < b ? a : b;
      edges[2 * n + 1] = a < b ? b : a;
      ++n;
    }
  qsort(edges, (size_t)n, 2 * sizeof(int32_t), cmp_edge);
  long u = 0;
  for (long k = 0; k < n; ++k)
    if (u == 0 || cmp_edge(edges + 2 * k, edges + 2 * (u - 1)) != 0) {
      edges[2 * u] = edges[2 * k];
      edges[2 * u + 1] = edges[2 * k + 1];
      ++u;
    }
  return u;
}

/* Edge lengths |x-hat_i - x-hat_j| of frame t (E entries). */
void or_edge_lengths(int N, const double* xhat, int t, long E, const int32_t* edges,
                     double* len) {
  const double* X = xhat + (long)t * N * 3;
  for (long e = 0; e < E; ++e) {
    const double* a = X + 3L * edges[2 * e];
    const double* b = X + 3L * edges[2 * e + 1];
    double dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
    len[e] = sqrt(dx * dx + dy * dy + dz * dz);
  }
}

/* Eq. 13 with the reference lengths given (their stop-grad values). */
double or_iso(int T, int N, const double* xhat, long E, const int32_t* edges,
              const double* lref) {
  double s = 0;
  double* len = (double*)malloc(sizeof(double) * (E > 0 ? E : 1));
  for (int t = 0; t < T; ++t) {
    or_edge_lengths(N, xhat, t, E, edges, len);
    for (long e = 0; e < E; ++e) s += fabs(len[e] - lref[e]);
  }
  free(len);
  return E > 0 ? s / ((double)T * (double)E) : 0.0;
}

/* ------------------------------ loss and hand-written reverse-mode gradient */

/* Reverse pass from a given dL/dx-hat (T x N x 3): back through Eq. 7-5, the
 * MLP (Eq. 4), the input vector (Eq. 2), the trilinear lookups and the level
 * mean (Eq. 1). g_grid and g_mlp (nullable) are overwritten.
 * With mag != 0 the same pass runs on magnitudes: dL/do, the weights, the
 * activations and the inputs enter by their absolute values, so every output
 * is the sum of |each product| that makes up the true gradient (the usual
 * companion computation of a forward rounding-error bound: an operand rounding
 * of relative size u perturbs each gradient value by at most u times it). */
static void backprop_impl(const or_cfg* c, int N, const double* x, const double* n, int T,
                          const double* grid, const double* mlp, const double* gx,
                          double* g_grid, double* g_mlp, int mag) {
  int F = c->F, Fn = c->Fn, Z = Fn + F, G2 = 2 * c->n_freq, K = or_k_in(c);
  int H = c->H, D = c->D, O = or_n_out(c);
  double* z = (double*)malloc(sizeof(double) * (size_t)N * Z);
  double* gamma = (double*)malloc(sizeof(double) * (size_t)T * G2);
  or_encode(c, N, x, n, grid, z);
  or_time_embedding_params(c, mlp, T, gamma);
  /* back through Eq. 7-5, the MLP (Eq. 4) and the input vector (Eq. 2) */
  double* gm = (double*)calloc((size_t)or_mlp_len(c), sizeof(double));
  double* gz = (double*)calloc((size_t)N * Z, sizeof(double));
  double* y = (double*)malloc(sizeof(double) * K);
  double* pre = (double*)malloc(sizeof(double) * H * D);
  double* h = (double*)malloc(sizeof(double) * H * D);
  double* dh = (double*)malloc(sizeof(double) * H);
  double* dp = (double*)malloc(sizeof(double) * H);
  double* ggam = (double*)calloc((size_t)T * G2, sizeof(double)); /* dL/dgamma_t */
  double o[8], go[8];
#define W(idx) (mag ? fabs(mlp[idx]) : mlp[idx])
  for (int t = 0; t < T; ++t)
    for (int i = 0; i < N; ++i) {
      for (int k = 0; k < Z; ++k) y[k] = z[(long)i * Z + k];
      for (int k = 0; k < G2; ++k) y[Z + k] = gamma[(long)t * G2 + k];
      mlp_row(c, mlp, y, pre, h, o);
      transform_row_backward(c, o, x + 3L * i, gx + ((long)t * N + i) * 3, go);
      if (mag) {
        for (int j = 0; j < O; ++j) go[j] = fabs(go[j]);
        for (int k = 0; k < H * D; ++k) h[k] = fabs(h[k]);
        for (int k = 0; k < K; ++k) y[k] = fabs(y[k]);
      }
      /* layer offsets in the flat parameter vector */
      long offW0 = 0, offb0 = (long)H * K;
      long offHid = offb0 + H; /* hidden layer k>=1 at offHid + (k-1)(H*H+H) */
      long offWo = offHid + (long)(D - 1) * (H * H + H), offbo = offWo + (long)O * H;
      /* output layer */
      const double* hl = h + (long)(D - 1) * H;
      for (int k = 0; k < H; ++k) dh[k] = 0.0;
      for (int j = 0; j < O; ++j) {
        gm[offbo + j] += go[j];
        for (int k = 0; k < H; ++k) {
          gm[offWo + (long)j * H + k] += go[j] * hl[k];
          dh[k] += W(offWo + (long)j * H + k) * go[j];
        }
      }
      /* hidden layers D-1 .. 1 */
      for (int layer = D - 1; layer >= 1; --layer) {
        long offW = offHid + (long)(layer - 1) * (H * H + H), offb = offW + (long)H * H;
        const double* hin = h + (long)(layer - 1) * H;
        for (int j = 0; j < H; ++j) dp[j] = dh[j] * dact(pre[(long)layer * H + j], c->slope);
        for (int k = 0; k < H; ++k) dh[k] = 0.0;
        for (int j = 0; j < H; ++j) {
          gm[offb + j] += dp[j];
          for (int k = 0; k < H; ++k) {
            gm[offW + (long)j * H + k] += dp[j] * hin[k];
            dh[k] += W(offW + (long)j * H + k) * dp[j];
          }
        }
      }
      /* first layer */
      for (int j = 0; j < H; ++j) dp[j] = dh[j] * dact(pre[j], c->slope);
      for (int j = 0; j < H; ++j) {
        gm[offb0 + j] += dp[j];
        for (int k = 0; k < K; ++k) gm[offW0 + (long)j * K + k] += dp[j] * y[k];
        for (int k = 0; k < Z; ++k) gz[(long)i * Z + k] += W(offW0 + (long)j * K + k) * dp[j];
        for (int k = 0; k < G2; ++k)
          ggam[(long)t * G2 + k] += W(offW0 + (long)j * K + Z + k) * dp[j];
      }
    }
  /* back through the learned time embedding psi_t (time_enc 3) */
  if (c->time_enc == 3) {
    int Ht = c->Ht;
    long oa = decoder_len(c), ob = oa + Ht, oW = ob + Ht, oc = oW + (long)G2 * Ht;
    for (int t = 0; t < T; ++t) {
      double tt = T > 1 ? (double)t / (double)(T - 1) : 0.0;
      const double* gg = ggam + (long)t * G2;
      for (int j = 0; j < Ht; ++j) {
        double hp = mlp[oa + j] * tt + mlp[ob + j];
        double hj = act(hp, c->slope);
        if (mag) hj = fabs(hj);
        double dhj = 0.0;
        for (int k = 0; k < G2; ++k) {
          gm[oW + (long)k * Ht + j] += gg[k] * hj;
          dhj += W(oW + (long)k * Ht + j) * gg[k];
        }
        double dpj = dhj * dact(hp, c->slope);
        gm[oa + j] += dpj * tt;
        gm[ob + j] += dpj;
      }
      for (int k = 0; k < G2; ++k) gm[oc + k] += gg[k];
    }
  }
#undef W
  free(ggam);
  if (g_mlp) memcpy(g_mlp, gm, sizeof(double) * (size_t)or_mlp_len(c));

  /* back through the trilinear lookups and the level mean (Eq. 1) */
  if (g_grid) {
    memset(g_grid, 0, sizeof(double) * (size_t)or_grid_len(c));
    long idx[8];
    double w[8];
    for (int i = 0; i < N; ++i) {
      const double* gzi = gz + (long)i * Z;
      or_trilinear(c->rn, n + 3L * i, idx, w);
      double* gn = g_grid + or_level_offset(c, c->L);
      for (int k = 0; k < 8; ++k)
        for (int f = 0; f < Fn; ++f) gn[idx[k] * Fn + f] += w[k] * gzi[f];
      for (int l = 0; l < c->L; ++l) {
        double* gl = g_grid + or_level_offset(c, l);
        or_trilinear(c->res[l], x + 3L * i, idx, w);
        for (int k = 0; k < 8; ++k)
          for (int f = 0; f < F; ++f) gl[idx[k] * F + f] += w[k] * gzi[Fn + f] / (double)c->L;
      }
    }
  }
  free(gm); free(gz); free(y); free(pre); free(h); free(dh); free(dp); free(z); free(gamma);
}

void or_backprop(const or_cfg* c, int N, const double* x, const double* n, int T,
                 const double* grid, const double* mlp, const double* gx, double* g_grid,
                 double* g_mlp) {
  backprop_impl(c, N, x, n, T, grid, mlp, gx, g_grid, g_mlp, 0);
}

/* The magnitude companion of or_backprop (see backprop_impl). */
void or_backprop_magnitude(const or_cfg* c, int N, const double* x, const double* n, int T,
                           const double* grid, const double* mlp, const double* gx,
                           double* g_grid, double* g_mlp) {
  backprop_impl(c, N, x, n, T, grid, mlp, gx, g_grid, g_mlp, 1);
}

/* L = L_def + w_iso L_iso (Eq. 8, 10, 13) with the stop-grad quantities held
 * fixed: w_fixed (T confidence weights) and lref (E keyframe edge lengths).
 * Writes dL/d grid and dL/d mlp when the pointers are non-null (they are
 * overwritten, not accumulated). parts (nullable) receives {L_def, L_iso}.
 * xhat_out (nullable, T x N x 3), cd_out (nullable, T). nn_x/nn_p (nullable)
 * receive the nearest-neighbour indices; gx_out (nullable, T x N x 3) dL/dx-hat. */
double or_loss_grad(const or_cfg* c, int N, const double* x, const double* n, int T,
                    const int64_t* off, const double* pts, long E, const int32_t* edges,
                    const double* grid, const double* mlp, const double* w_fixed,
                    const double* lref, int decide_f32, double* g_grid, double* g_mlp,
                    double* xhat_out, double* cd_out, double* parts, int32_t* nn_x_out,
                    int32_t* nn_p_out, double* gx_out) {
  int Z = c->Fn + c->F, G2 = 2 * c->n_freq;
  long MT = off[T];
  double* z = (double*)malloc(sizeof(double) * (size_t)N * Z);
  double* gamma = (double*)malloc(sizeof(double) * (size_t)T * G2);
  double* xhat = (double*)malloc(sizeof(double) * (size_t)T * N * 3);
  or_encode(c, N, x, n, grid, z);
  or_time_embedding_params(c, mlp, T, gamma);
  or_decode(c, N, T, x, z, gamma, mlp, xhat);

  int32_t* nn_x = (int32_t*)malloc(sizeof(int32_t) * (size_t)T * N);
  double* d_x = (double*)malloc(sizeof(double) * (size_t)T * N);
  int32_t* nn_p = (int32_t*)malloc(sizeof(int32_t) * (size_t)(MT > 0 ? MT : 1));
  double* d_p = (double*)malloc(sizeof(double) * (size_t)(MT > 0 ? MT : 1));
  double* cd = (double*)malloc(sizeof(double) * T);
  or_chamfer(T, N, xhat, off, pts, decide_f32, nn_x, d_x, nn_p, d_p, cd);

  /* Eq. 10 and Eq. 13 */
  double Ldef = 0;
  for (int t = 0; t < T; ++t) Ldef += w_fixed[t] * cd[t];
  Ldef /= T;
  double Liso = or_iso(T, N, xhat, E, edges, lref);
  double Lval = Ldef + c->w_iso * Liso;
  if (parts) { parts[0] = Ldef; parts[1] = Liso; }

  if (g_grid || g_mlp || gx_out) {
    /* dL/dx-hat (T x N x 3) */
    double* gx = (double*)calloc((size_t)T * N * 3, sizeof(double));
    for (int t = 0; t < T; ++t) {
      double ct = w_fixed[t] / T; /* dL/dcd_t */
      long M = off[t + 1] - off[t];
      const double* P = pts + 3 * off[t];
      const double* X = xhat + (long)t * N * 3;
      double* GX = gx + (long)t * N * 3;
      for (int i = 0; i < N; ++i) {
        const double* p = P + 3L * nn_x[(long)t * N + i];
        for (int a = 0; a < 3; ++a) GX[3L * i + a] += ct * (2.0 / N) * (X[3L * i + a] - p[a]);
      }
      for (long j = 0; j < M; ++j) {
        int i = nn_p[off[t] + j];
        for (int a = 0; a < 3; ++a)
          GX[3L * i + a] += ct * (2.0 / (double)M) * (X[3L * i + a] - P[3 * j + a]);
      }
      if (E > 0) {
        double ci = c->w_iso / ((double)T * (double)E);
        for (long e = 0; e < E; ++e) {
          int a0 = edges[2 * e], b0 = edges[2 * e + 1];
          double v[3];
          for (int a = 0; a < 3; ++a) v[a] = X[3L * a0 + a] - X[3L * b0 + a];
          double len = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
          double diff = len - lref[e];
          double s = diff > 0 ? 1.0 : (diff < 0 ? -1.0 : 0.0);
          if (len > 0 && s != 0) {
            for (int a = 0; a < 3; ++a) {
              GX[3L * a0 + a] += ci * s * v[a] / len;
              GX[3L * b0 + a] -= ci * s * v[a] / len;
            }
          }
        }
      }
    }

    or_backprop(c, N, x, n, T, grid, mlp, gx, g_grid, g_mlp);
    if (gx_out) memcpy(gx_out, gx, sizeof(double) * (size_t)T * N * 3);
    free(gx);
  }

  if (xhat_out) memcpy(xhat_out, xhat, sizeof(double) * (size_t)T * N * 3);
  if (cd_out) memcpy(cd_out, cd, sizeof(double) * T);
  if (nn_x_out) memcpy(nn_x_out, nn_x, sizeof(int32_t) * (size_t)T * N);
  if (nn_p_out && MT > 0) memcpy(nn_p_out, nn_p, sizeof(int32_t) * (size_t)MT);
  free(z); free(gamma); free(xhat); free(nn_x); free(d_x); free(nn_p); free(d_p); free(cd);
  return Lval;
}

/* The loss as the method evaluates it at iteration e: the stop-grad inputs
 * (w_conf from this forward pass's cd, Eq. 11-12, and the keyframe edge
 * lengths of this forward pass, Eq. 13) are computed first, then held fixed.
 * w_out (T) and lref_out (E) are nullable. */
double or_loss_full(const or_cfg* c, int N, const double* x, const double* n, int T,
                    const int64_t* off, const double* pts, long E, const int32_t* edges,
                    int t_key, double e, double e_max, const double* grid, const double* mlp,
                    int decide_f32, double* g_grid, double* g_mlp, double* xhat_out,
                    double* cd_out, double* w_out, double* parts, int32_t* nn_x_out,
                    int32_t* nn_p_out, double* gx_out) {
  int Z = c->Fn + c->F, G2 = 2 * c->n_freq;
  long MT = off[T];
  double* z = (double*)malloc(sizeof(double) * (size_t)N * Z);
  double* gamma = (double*)malloc(sizeof(double) * (size_t)T * G2);
  double* xhat = (double*)malloc(sizeof(double) * (size_t)T * N * 3);
  or_encode(c, N, x, n, grid, z);
  or_time_embedding_params(c, mlp, T, gamma);
  or_decode(c, N, T, x, z, gamma, mlp, xhat);
  int32_t* nn_x = (int32_t*)malloc(sizeof(int32_t) * (size_t)T * N);
  double* d_x = (double*)malloc(sizeof(double) * (size_t)T * N);
  int32_t* nn_p = (int32_t*)malloc(sizeof(int32_t) * (size_t)(MT > 0 ? MT : 1));
  double* d_p = (double*)malloc(sizeof(double) * (size_t)(MT > 0 ? MT : 1));
  double* cd = (double*)malloc(sizeof(double) * T);
  double* w = (double*)malloc(sizeof(double) * T);
  double* lref = (double*)malloc(sizeof(double) * (E > 0 ? E : 1));
  or_chamfer(T, N, xhat, off, pts, decide_f32, nn_x, d_x, nn_p, d_p, cd);
  or_conf_weights_mode(T, cd, t_key, e, e_max, c->conf_delta, c->conf_omega, w);
  or_edge_lengths(N, xhat, t_key, E, edges, lref);
  double L = or_loss_grad(c, N, x, n, T, off, pts, E, edges, grid, mlp, w, lref, decide_f32,
                          g_grid, g_mlp, xhat_out, cd_out, parts, nn_x_out, nn_p_out, gx_out);
  if (w_out) memcpy(w_out, w, sizeof(double) * T);
  free(z); free(gamma); free(xhat); free(nn_x); free(d_x); free(nn_p); free(d_p);
  free(cd); free(w); free(lref);
  return L;
}

/* ------------------------------------------- Sec. 3.5, Eq. 9: preconditioner */

/* y = (I + lambda L) u on an r^3 node lattice, one channel (stride F). */
static void apply_A(int r, int F, int ch, double lambda, const double* u, double* y) {
#pragma omp parallel for schedule(static)
  for (long iz = 0; iz < r; ++iz)
    for (long iy = 0; iy < r; ++iy)
      for (long ix = 0; ix < r; ++ix) {
        long k = (iz * r + iy) * r + ix;
        double uk = u[k * F + ch];
        double lap = 0.0;
        if (ix > 0) lap += uk - u[(k - 1) * F + ch];
        if (ix < r - 1) lap += uk - u[(k + 1) * F + ch];
        if (iy > 0) lap += uk - u[(k - r) * F + ch];
        if (iy < r - 1) lap += uk - u[(k + r) * F + ch];
        if (iz > 0) lap += uk - u[(k - (long)r * r) * F + ch];
        if (iz < r - 1) lap += uk - u[(k + (long)r * r) * F + ch];
        y[k * F + ch] = uk + lambda * lap;
      }
}

/* Solve (I + lambda L) u = b for channel ch by conjugate gradients. */
static int cg_solve(int r, int F, int ch, double lambda, const double* b, double* u,
                    double tol, int max_iter) {
  long n = cube(r);
  double* res = (double*)malloc(sizeof(double) * n * F);
  double* p = (double*)malloc(sizeof(double) * n * F);
  double* Ap = (double*)malloc(sizeof(double) * n * F);
  double bb = 0;
  for (long k = 0; k < n; ++k) {
    u[k * F + ch] = 0.0;
    res[k * F + ch] = b[k * F + ch];
    p[k * F + ch] = b[k * F + ch];
    bb += b[k * F + ch] * b[k * F + ch];
  }
  double rr = bb;
  int it = 0;
  while (rr > tol * tol * bb && it < max_iter) {
    apply_A(r, F, ch, lambda, p, Ap);
    double pAp = 0;
    for (long k = 0; k < n; ++k) pAp += p[k * F + ch] * Ap[k * F + ch];
    double al = rr / pAp;
    double rr2 = 0;
    for (long k = 0; k < n; ++k) {
      u[k * F + ch] += al * p[k * F + ch];
      res[k * F + ch] -= al * Ap[k * F + ch];
      rr2 += res[k * F + ch] * res[k * F + ch];
    }
    double be = rr2 / rr;
    for (long k = 0; k < n; ++k) p[k * F + ch] = res[k * F + ch] + be * p[k * F + ch];
    rr = rr2;
    ++it;
  }
  free(res);
  free(p);
  free(Ap);
  return it;
}

/* out = (I + lambda L)^-2 g for every channel of one r^3 x F block.
 * Returns the largest CG iteration count used. */
int or_precondition(int r, int F, double lambda, const double* g, double* out, double tol,
                    int max_iter) {
  long n = cube(r);
  double* tmp = (double*)malloc(sizeof(double) * n * F);
  int worst = 0;
  for (int ch = 0; ch < F; ++ch) {
    int a = cg_solve(r, F, ch, lambda, g, tmp, tol, max_iter);
    int b = cg_solve(r, F, ch, lambda, tmp, out, tol, max_iter);
    if (a > worst) worst = a;
    if (b > worst) worst = b;
  }
  free(tmp);
  return worst;
}

/* ------------------------------------------------------------ Adam */

/* Kingma & Ba, bias-corrected; step is 1-based. */
void or_adam(long n, double* p, const double* g, double* m, double* v, double lr, double b1,
             double b2, double eps, int step) {
  double c1 = 1.0 - pow(b1, step), c2 = 1.0 - pow(b2, step);
  for (long k = 0; k < n; ++k) {
    m[k] = b1 * m[k] + (1.0 - b1) * g[k];
    v[k] = b2 * v[k] + (1.0 - b2) * g[k] * g[k];
    double mh = m[k] / c1, vh = v[k] / c2;
    p[k] -= lr * mh / (sqrt(vh) + eps);
  }
}

/* ------------------------------------------------- one whole iteration */

/* One optimisation iteration e (0-based): loss and gradient at the current
 * parameters, the preconditioner of Eq. 9 on every grid level (lambda[l],
 * l = L for the normal grid), then Adam (lr_grid[l] per level, lr_mlp on the
 * MLP) with step count e + 1. Parameters and moments are updated in place.
 * g_grid_pc (nullable) receives the preconditioned grid gradient.
 * Returns the loss before the update. */
double or_iteration(const or_cfg* c, int N, const double* x, const double* n, int T,
                    const int64_t* off, const double* pts, long E, const int32_t* edges,
                    int t_key, int e, int e_max, double* grid, double* mlp, double* m_grid,
                    double* v_grid, double* m_mlp, double* v_mlp, const double* lr_grid,
                    double lr_mlp, const double* lambda, double b1, double b2, double eps,
                    int decide_f32, double cg_tol, double* cd_out, double* g_grid_out,
                    double* g_grid_pc, double* g_mlp_out) {
  long GL = or_grid_len(c), ML = or_mlp_len(c);
  double* gg = (double*)malloc(sizeof(double) * GL);
  double* gp = (double*)malloc(sizeof(double) * GL);
  double* gm = (double*)malloc(sizeof(double) * ML);
  double L = or_loss_full(c, N, x, n, T, off, pts, E, edges, t_key, (double)e, (double)e_max,
                          grid, mlp, decide_f32, gg, gm, NULL, cd_out, NULL, NULL, NULL, NULL, NULL);
  for (int l = 0; l <= c->L; ++l) {
    int r = l < c->L ? c->res[l] : c->rn;
    int F = l < c->L ? c->F : c->Fn;
    long o = or_level_offset(c, l);
    or_precondition(r, F, lambda[l], gg + o, gp + o, cg_tol, 100000);
  }
  for (int l = 0; l <= c->L; ++l) {
    int r = l < c->L ? c->res[l] : c->rn;
    int F = l < c->L ? c->F : c->Fn;
    long o = or_level_offset(c, l), len = cube(r) * F;
    or_adam(len, grid + o, gp + o, m_grid + o, v_grid + o, lr_grid[l], b1, b2, eps, e + 1);
  }
  or_adam(ML, mlp, gm, m_mlp, v_mlp, lr_mlp, b1, b2, eps, e + 1);
  if (g_grid_out) memcpy(g_grid_out, gg, sizeof(double) * GL);
  if (g_grid_pc) memcpy(g_grid_pc, gp, sizeof(double) * GL);
  if (g_mlp_out) memcpy(g_mlp_out, gm, sizeof(double) * ML);
  free(gg);
  free(gp);
  free(gm);
  return L;
}

/* ---------------------------------- Sec. 4: evaluation metrics */

/* Area-weighted vertex normals of one frame (sum of the incident faces'
 * cross products, normalised; a vertex without area gets (0, 0, 0)). */
static void vertex_normals(int N, const double* v, int F_tri, const int32_t* faces, double* nrm) {
  for (long i = 0; i < 3L * N; ++i) nrm[i] = 0.0;
  for (int f = 0; f < F_tri; ++f) {
    const int32_t* t = faces + 3L * f;
    const double* a = v + 3L * t[0];
    const double* b = v + 3L * t[1];
    const double* c = v + 3L * t[2];
    const double u[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    const double w[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
    const double n[3] = {u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2],
                         u[0] * w[1] - u[1] * w[0]};
    for (int k = 0; k < 3; ++k)
      for (int d = 0; d < 3; ++d) nrm[3L * t[k] + d] += n[d];
  }
  for (int i = 0; i < N; ++i) {
    double* p = nrm + 3L * i;
    const double l = sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
    if (l > 0.0)
      for (int d = 0; d < 3; ++d) p[d] /= l;
  }
}

/* Per frame t, the reconstruction xhat (reference connectivity) against the
 * ground truth gt (same connectivity, known trajectories), both T x N x 3:
 *   cd        mean_i min_j |xh_i - g_j|^2 + mean_j min_i |g_j - xh_i|^2
 *   precision fraction of xh_i with min_j |xh_i - g_j| < tau
 *   recall    fraction of g_j with min_i |g_j - xh_i| < tau
 *   fscore    2 P R / (P + R), 0 when P + R = 0
 *   nc        (mean_i |n_i . n_g(nn(i))| + mean_j |n_g,j . n(nn(j))|) / 2
 *   corr      mean_i |xh_i - g_i|
 * with tau = tau_rel x the diagonal of frame t's ground-truth bounding box
 * and area-weighted vertex normals. out: T x 6 in that order. */
void or_evaluate(int T, int N, const double* xhat, const double* gt, int F_tri,
                 const int32_t* faces, double tau_rel, double* out) {
  double* nx = (double*)malloc(sizeof(double) * 3 * N);
  double* ng = (double*)malloc(sizeof(double) * 3 * N);
  int32_t* ix = (int32_t*)malloc(sizeof(int32_t) * N);
  int32_t* ig = (int32_t*)malloc(sizeof(int32_t) * N);
  double* dx = (double*)malloc(sizeof(double) * N);
  double* dg = (double*)malloc(sizeof(double) * N);
  for (int t = 0; t < T; ++t) {
    const double* X = xhat + 3L * N * t;
    const double* G = gt + 3L * N * t;
    double lo[3], hi[3];
    for (int d = 0; d < 3; ++d) lo[d] = hi[d] = G[d];
    for (int i = 0; i < N; ++i)
      for (int d = 0; d < 3; ++d) {
        lo[d] = fmin(lo[d], G[3L * i + d]);
        hi[d] = fmax(hi[d], G[3L * i + d]);
      }
    const double diag = sqrt((hi[0] - lo[0]) * (hi[0] - lo[0]) + (hi[1] - lo[1]) * (hi[1] - lo[1]) +
                             (hi[2] - lo[2]) * (hi[2] - lo[2]));
    const double tau = tau_rel * diag;
    vertex_normals(N, X, F_tri, faces, nx);
    vertex_normals(N, G, F_tri, faces, ng);
    or_nn(N, X, N, G, 0, ix, dx);
    or_nn(N, G, N, X, 0, ig, dg);
    double sx = 0, sg = 0, cx = 0, cg = 0, nsx = 0, nsg = 0, sc = 0;
    for (int i = 0; i < N; ++i) {
      sx += dx[i];
      sg += dg[i];
      if (dx[i] < tau * tau) cx += 1;
      if (dg[i] < tau * tau) cg += 1;
      const double* a = nx + 3L * i;
      const double* b = ng + 3L * ix[i];
      nsx += fabs(a[0] * b[0] + a[1] * b[1] + a[2] * b[2]);
      const double* c = ng + 3L * i;
      const double* e = nx + 3L * ig[i];
      nsg += fabs(c[0] * e[0] + c[1] * e[1] + c[2] * e[2]);
      const double* p = X + 3L * i;
      const double* q = G + 3L * i;
      sc += sqrt((p[0] - q[0]) * (p[0] - q[0]) + (p[1] - q[1]) * (p[1] - q[1]) +
                 (p[2] - q[2]) * (p[2] - q[2]));
    }
    double* o = out + 6L * t;
    const double P = cx / N, R = cg / N;
    o[0] = sx / N + sg / N;
    o[1] = P;
    o[2] = R;
    o[3] = P + R > 0 ? 2 * P * R / (P + R) : 0.0;
    o[4] = 0.5 * (nsx / N + nsg / N);
    o[5] = sc / N;
  }
  free(nx);
  free(ng);
  free(ix);
  free(ig);
  free(dx);
  free(dg);
}

/* Keyframe selection (Sec. 3.1, Initialization): each frame's point cloud is
 * rated by its spatial extent, weighted by a term that favours the temporal
 * midpoint, and the best-rated frame becomes t_key. The paper defers the
 * formula to an earlier method; the reading taken here:
 *   e_t = sqrt( mean_j |p_j - c_t|^2 ),  c_t = mean_j p_j   (RMS radius of P_t)
 *   w_t = 1 - bias |t~ - 1/2|,  t~ = t / (T - 1)  (t~ = 1/2 when T = 1)
 *   t_key = argmax_t w_t e_t, the lowest t on ties.
 * Two passes per frame (centroid, then squared distances), FP64, points in
 * input order. pts: off[T] x 3; extent (T, nullable) receives e_t. */
int or_select_keyframe(int T, const int64_t* off, const double* pts, double bias,
                       double* extent) {
  int best = 0;
  double best_s = -1.0;
  for (int t = 0; t < T; ++t) {
    const int64_t a = off[t], b = off[t + 1];
    const double n = (double)(b - a);
    double c[3] = {0.0, 0.0, 0.0};
    for (int64_t j = a; j < b; ++j)
      for (int d = 0; d < 3; ++d) c[d] += pts[3 * j + d];
    for (int d = 0; d < 3; ++d) c[d] /= n;
    double s2 = 0.0;
    for (int64_t j = a; j < b; ++j)
      for (int d = 0; d < 3; ++d) {
        const double u = pts[3 * j + d] - c[d];
        s2 += u * u;
      }
    const double e = sqrt(s2 / n);
    if (extent) extent[t] = e;
    const double tt = T > 1 ? (double)t / (double)(T - 1) : 0.5;
    const double s = (1.0 - bias * fabs(tt - 0.5)) * e;
    if (s > best_s) {
      best_s = s;
      best = t;
    }
  }
  return best;
}
