// Device helpers shared by the libnpg.so kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include "../../include/npg.h"

namespace npg {

// Sec. 3.2: nodes at -1 + 2k/(r-1); queries clamped to [-1, 1]; cell index
// min(floor(u), r-2); returns the cell and the fractional offset in it.
__device__ __forceinline__ void tri_axis(float q, int r, int& i0, float& f) {
  q = fminf(fmaxf(q, -1.f), 1.f);
  const float h = 0.5f * (float)(r - 1);
  const float u = fmaf(q, h, h);
  int i = (int)floorf(u);
  i = min(max(i, 0), r - 2);
  i0 = i;
  f = u - (float)i;
}

__device__ __forceinline__ float leaky(float s, float slope) { return s > 0.f ? s : slope * s; }
// derivative from the post-activation value (valid for slope >= 0: h > 0 <=> s > 0)
__device__ __forceinline__ float dleaky_h(float h, float slope) { return h > 0.f ? 1.f : slope; }

// Squared distance with the fixed operation order of the nearest-neighbour rule.
__device__ __forceinline__ float sqdist(float ax, float ay, float az, float bx, float by, float bz) {
  const float dx = __fsub_rn(ax, bx), dy = __fsub_rn(ay, by), dz = __fsub_rn(az, bz);
  float d = __fmul_rn(dx, dx);
  d = __fmaf_rn(dy, dy, d);
  d = __fmaf_rn(dz, dz, d);
  return d;
}


// ------------------------------------------------------- Sec. 3.4 mapping

// Exponential map coefficients A = sin t / t, B = (1 - cos t)/t^2 and
// A'/t, B'/t, Taylor series below t = 0.5.
__device__ __forceinline__ void expmap_coeffs(float th, float& A, float& B, float& dA, float& dB) {
  const float t2 = th * th;
  if (th < 0.5f) {
    A = 1.f + t2 * (-1.f / 6.f + t2 * (1.f / 120.f + t2 * (-1.f / 5040.f + t2 * (1.f / 362880.f))));
    B = 0.5f + t2 * (-1.f / 24.f + t2 * (1.f / 720.f + t2 * (-1.f / 40320.f + t2 * (1.f / 3628800.f))));
    dA = -1.f / 3.f + t2 * (1.f / 30.f + t2 * (-1.f / 840.f + t2 * (1.f / 45360.f)));
    dB = -1.f / 12.f + t2 * (1.f / 180.f + t2 * (-1.f / 6720.f + t2 * (1.f / 453600.f)));
  } else {
    float s, co;
    sincosf(th, &s, &co);
    const float sh = sinf(0.5f * th);
    const float omc = 2.f * sh * sh;
    A = s / th;
    B = omc / t2;
    dA = (th * co - s) / (t2 * th);
    dB = (th * s - 2.f * omc) / (t2 * t2);
  }
}

// Cayley transform R = (I - K)^-1 (I + K) = I + c (K + K^2), c = 2 / (1 + |w|^2):
// the same form as the exponential map with A = B = c and
// dA = dB = (dc/d|w|) / |w| = -c^2.
__device__ __forceinline__ void cayley_coeffs(float th, float& A, float& B, float& dA, float& dB) {
  const float c = 2.f / (1.f + th * th);
  A = B = c;
  dA = dB = -c * c;
}

template <int ROT>
__device__ __forceinline__ void rot_coeffs(float th, float& A, float& B, float& dA, float& dB) {
  if (ROT == 2)
    cayley_coeffs(th, A, B, dA, dB);
  else
    expmap_coeffs(th, A, B, dA, dB);
}

// Rotation R (row-major) and translation d from one decoder output row
// (ROT: NPG_ROT_QUAT, NPG_ROT_EXPMAP or NPG_ROT_CAYLEY).
template <int ROT>
__device__ __forceinline__ void rot_trans(const float* o, float alpha, float* R, float* d) {
  if (ROT == 0) {
    float w = 1.f + o[0], x = o[1], y = o[2], z = o[3];
    const float n2 = w * w + x * x + y * y + z * z;
    if (n2 > 0.f) {
      // correctly rounded sqrt and division: a zero output gives R = I exactly
      const float nq = __fsqrt_rn(n2);
      w = __fdiv_rn(w, nq); x = __fdiv_rn(x, nq); y = __fdiv_rn(y, nq); z = __fdiv_rn(z, nq);
    } else {
      w = 1.f; x = y = z = 0.f;
    }
    R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z); R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z); R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y); R[7] = 2.f * (y * z + w * x); R[8] = 1.f - 2.f * (x * x + y * y);
    d[0] = tanhf(alpha * o[4]);
    d[1] = tanhf(alpha * o[5]);
    d[2] = tanhf(alpha * o[6]);
  } else {
    const float wx = o[0], wy = o[1], wz = o[2];
    const float th = sqrtf(wx * wx + wy * wy + wz * wz);
    float A, B, dA, dB;
    rot_coeffs<ROT>(th, A, B, dA, dB);
    // K = [w]x, K^2 = w w^T - |w|^2 I
    const float xx = wx * wx, yy = wy * wy, zz = wz * wz, xy = wx * wy, xz = wx * wz, yz = wy * wz;
    R[0] = 1.f + B * (-(yy + zz)); R[1] = -A * wz + B * xy;       R[2] = A * wy + B * xz;
    R[3] = A * wz + B * xy;       R[4] = 1.f + B * (-(xx + zz)); R[5] = -A * wx + B * yz;
    R[6] = -A * wy + B * xz;      R[7] = A * wx + B * yz;       R[8] = 1.f + B * (-(xx + yy));
    d[0] = tanhf(alpha * o[3]);
    d[1] = tanhf(alpha * o[4]);
    d[2] = tanhf(alpha * o[5]);
  }
}

// Eq. 7: x-hat = R x + d, formed as x + delta with the displacement
// delta = (R - I) x + d computed directly (R - I from the rotation parameters,
// without the cancellation of 1 - 2(y^2 + z^2) - 1), so that near-rigid
// motions keep their relative precision in delta.
template <int ROT>
__device__ __forceinline__ void transform(const float* o, float alpha, float4 x, float4& xh,
                                          float4& dl) {
  float R[9], d[3];
  rot_trans<ROT>(o, alpha, R, d);
  R[0] -= 1.f;
  R[4] -= 1.f;
  R[8] -= 1.f;
  dl.x = fmaf(R[0], x.x, fmaf(R[1], x.y, fmaf(R[2], x.z, d[0])));
  dl.y = fmaf(R[3], x.x, fmaf(R[4], x.y, fmaf(R[5], x.z, d[1])));
  dl.z = fmaf(R[6], x.x, fmaf(R[7], x.y, fmaf(R[8], x.z, d[2])));
  dl.w = 0.f;
  xh = make_float4(x.x + dl.x, x.y + dl.y, x.z + dl.z, 0.f);
}

// |e_t| - |e_key| for one edge (Eq. 13) from the reference edge e0 = x_a - x_b
// and the displacement differences Dt = delta_a(t) - delta_b(t), Dk at the
// keyframe: (|e_t|^2 - |e_k|^2) / (|e_t| + |e_k|) with
// |e_t|^2 - |e_k|^2 = (Dt - Dk) . (2 e0 + Dt + Dk), so the (often tiny)
// difference keeps its relative precision; exactly 0 at the keyframe.
// Also returns e_t and |e_t|.
__device__ __forceinline__ float iso_diff(float3 e0, float3 Dt, float3 Dk, float3& et,
                                          float& lt) {
  et = make_float3(e0.x + Dt.x, e0.y + Dt.y, e0.z + Dt.z);
  const float3 ek = make_float3(e0.x + Dk.x, e0.y + Dk.y, e0.z + Dk.z);
  lt = sqrtf(et.x * et.x + et.y * et.y + et.z * et.z);
  const float lk = sqrtf(ek.x * ek.x + ek.y * ek.y + ek.z * ek.z);
  const float num = (Dt.x - Dk.x) * (et.x + ek.x) + (Dt.y - Dk.y) * (et.y + ek.y) +
                    (Dt.z - Dk.z) * (et.z + ek.z);
  const float den = lt + lk;
  return den > 0.f ? num / den : 0.f;
}

// dL/do for one row given g = dL/dx-hat.
template <int ROT>
__device__ __forceinline__ void transform_backward(const float* o, float alpha, float4 x, float4 g,
                                                   float* go) {
  float G[9] = {g.x * x.x, g.x * x.y, g.x * x.z, g.y * x.x, g.y * x.y,
                g.y * x.z, g.z * x.x, g.z * x.y, g.z * x.z};
  if (ROT == 0) {
    const float qw = 1.f + o[0], qx = o[1], qy = o[2], qz = o[3];
    const float n2 = qw * qw + qx * qx + qy * qy + qz * qz;
    if (n2 > 0.f) {
      // a gradient, not a decision: one reciprocal square root suffices
      const float inv = rsqrtf(n2);
      const float w = qw * inv, X = qx * inv, Y = qy * inv, Z = qz * inv;
      float gq0 = 2.f * (-Z * G[1] + Y * G[2] + Z * G[3] - X * G[5] - Y * G[6] + X * G[7]);
      float gq1 = 2.f * (Y * G[1] + Z * G[2] + Y * G[3] - 2.f * X * G[4] - w * G[5] + Z * G[6] +
                         w * G[7] - 2.f * X * G[8]);
      float gq2 = 2.f * (-2.f * Y * G[0] + X * G[1] + w * G[2] + X * G[3] + Z * G[5] - w * G[6] +
                         Z * G[7] - 2.f * Y * G[8]);
      float gq3 = 2.f * (-2.f * Z * G[0] - w * G[1] + X * G[2] + w * G[3] - 2.f * Z * G[4] +
                         Y * G[5] + X * G[6] + Y * G[7]);
      const float dot = w * gq0 + X * gq1 + Y * gq2 + Z * gq3;
      go[0] = (gq0 - w * dot) * inv;
      go[1] = (gq1 - X * dot) * inv;
      go[2] = (gq2 - Y * dot) * inv;
      go[3] = (gq3 - Z * dot) * inv;
    } else {
      go[0] = go[1] = go[2] = go[3] = 0.f;
    }
    const float t0 = tanhf(alpha * o[4]), t1 = tanhf(alpha * o[5]), t2 = tanhf(alpha * o[6]);
    go[4] = g.x * alpha * (1.f - t0 * t0);
    go[5] = g.y * alpha * (1.f - t1 * t1);
    go[6] = g.z * alpha * (1.f - t2 * t2);
  } else {
    const float w[3] = {o[0], o[1], o[2]};
    const float th = sqrtf(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    float A, B, dA, dB;
    rot_coeffs<ROT>(th, A, B, dA, dB);
    float K[9] = {0.f, -w[2], w[1], w[2], 0.f, -w[0], -w[1], w[0], 0.f};
    float K2[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        K2[i * 3 + j] = K[i * 3 + 0] * K[0 * 3 + j] + K[i * 3 + 1] * K[1 * 3 + j] +
                        K[i * 3 + 2] * K[2 * 3 + j];
    // s_K = <G, K>, s_K2 = <G, K^2>
    float sK = 0.f, sK2 = 0.f;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      sK = fmaf(G[i], K[i], sK);
      sK2 = fmaf(G[i], K2[i], sK2);
    }
    // <G, E_k> with E_k = [e_k]x: E_0 = (0,0,0;0,0,-1;0,1,0) etc.
    const float gE[3] = {G[7] - G[5], G[2] - G[6], G[3] - G[1]};
    // <G, E_k K + K E_k>
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      float Ek[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      if (k == 0) { Ek[5] = -1.f; Ek[7] = 1.f; }
      if (k == 1) { Ek[2] = 1.f; Ek[6] = -1.f; }
      if (k == 2) { Ek[1] = -1.f; Ek[3] = 1.f; }
      float s = 0.f;
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          const float m = Ek[i * 3 + 0] * K[0 * 3 + j] + Ek[i * 3 + 1] * K[1 * 3 + j] +
                          Ek[i * 3 + 2] * K[2 * 3 + j] + K[i * 3 + 0] * Ek[0 * 3 + j] +
                          K[i * 3 + 1] * Ek[1 * 3 + j] + K[i * 3 + 2] * Ek[2 * 3 + j];
          s = fmaf(G[i * 3 + j], m, s);
        }
      go[k] = dA * w[k] * sK + A * gE[k] + dB * w[k] * sK2 + B * s;
    }
    const float t0 = tanhf(alpha * o[3]), t1 = tanhf(alpha * o[4]), t2 = tanhf(alpha * o[5]);
    go[3] = g.x * alpha * (1.f - t0 * t0);
    go[4] = g.y * alpha * (1.f - t1 * t1);
    go[5] = g.z * alpha * (1.f - t2 * t2);
  }
}

// Sec. 3.3, Eq. 3: gamma_t (interleaved sin/cos, nu_j = 2^(j-1)).
__device__ __forceinline__ void time_embedding(int t, int T, int M, float* g) {
  const float tt = T > 1 ? (float)t / (float)(T - 1) : 0.f;
  for (int j = 0; j < M; ++j) {
    const float a = ldexpf(tt, j);
    float s, c;
    sincospif(a, &s, &c);
    g[2 * j] = s;
    g[2 * j + 1] = c;
  }
}

// gamma(t) of the chosen encoding (NPG_TIME_*): Eq. 3, the polynomial basis
// t~^j (j = 1..2M), or the Gaussian Fourier mapping sin / cos(2 pi B_j t~).
__device__ __forceinline__ void time_embedding_mode(int t, int T, int M, int mode,
                                                    const float* B, float* g) {
  if (mode == NPG_TIME_FOURIER) {
    time_embedding(t, T, M, g);
    return;
  }
  const float tt = T > 1 ? (float)t / (float)(T - 1) : 0.f;
  if (mode == NPG_TIME_POLY) {
    float p = 1.f;
    for (int j = 0; j < 2 * M; ++j) {
      p *= tt;
      g[j] = p;
    }
    return;
  }
  for (int j = 0; j < M; ++j) {
    float s, c;
    sincospif(2.f * B[j] * tt, &s, &c);
    g[2 * j] = s;
    g[2 * j + 1] = c;
  }
}

}  // namespace npg
