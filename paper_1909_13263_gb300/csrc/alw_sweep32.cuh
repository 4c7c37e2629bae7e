// Streaming float sweep of the WENO reconstruction along one line segment.
//
// Same arithmetic as weno_sweep<float> (alw_device.cuh), reorganised so that
// each step of the sliding window computes only the quantities that become
// newly needed (one Delta^+ value, one second difference, three F values,
// three interval means, one T value) and hands each node's (phi^-, phi^+) to
// a callback as soon as it is complete; dead values retire at once, which
// keeps register pressure low.
//
// Weights and the compact form are folded into one reciprocal per side:
// with A0 = q1 q2, A1 = q0 q2, A2 = q0 q1 (q_k = (eps + beta_k)^2),
//   den = A0 + 6 A1 + 3 A2  ( = 10 sum_k d_k prod_{l != k} q_l ),
//   omega_0 = A0 / den, omega_2 = 3 A2 / den,
//   phi^- = (c + T_b/12) - (A0 T_a / 3 + A2 T_b / 2) / den,
//   phi^+ = (c - T_b/12) + (A0' T_c / 3 + A2' T_b / 2) / den'.
#pragma once
#include "alw_device.cuh"

namespace alw {

struct FVal {
  float F, s;  // F(u) = u sqrt(1+u^2) + asinh(u), s = sqrt(1+u^2)
};

__device__ __forceinline__ FVal f_eval(float u) {
  FVal r;
  const float t = fmaf(u, u, 1.0f);
  r.s = t * rsqrtf(t);
  const float l = __log2f(fabsf(u) + r.s);
  r.F = fmaf(0.693147180559945f, copysignf(l, u), u * r.s);
  return r;
}

// q = (eps + (dx G)^2)^2 for the interval [a, b], hdx = dx/2.
__device__ __forceinline__ float q_interval(float a, FVal fa, float b, FVal fb, float hdx, float eps) {
  const float h = b - a;
  const float ss = fa.s + fb.s;
  const float gd = __fdividef(hdx * (fb.F - fa.F), h);  // dx * divided difference
  const float gt = hdx * ss;                             // dx * trapezoid mean
  const float g = (fabsf(h) > 0.015625f * ss) ? gd : gt;
  const float e = fmaf(g, g, eps);
  return e * e;
}

// (T_a/3, T_b/2) terms and the side's reciprocal combination.
__device__ __forceinline__ float side_corr(float q0, float q1, float q2, float ta3, float tb2, float ta, float tb) {
  const float A0 = q1 * q2, A1 = q0 * q2, A2 = q0 * q1;
  const float den = fmaf(6.0f, A1, fmaf(3.0f, A2, A0));
  if (den > 1e-30f && den < 1e30f) {
    return __fdividef(fmaf(A0, ta3, A2 * tb2), den);
  }
  // products out of range: per-weight reciprocals
  const float a0 = __fdividef(0.1f, q0), a1 = __fdividef(0.6f, q1), a2 = __fdividef(0.3f, q2);
  const float r = __fdividef(1.0f, a0 + a1 + a2);
  const float w0 = a0 * r, w2 = a2 * r;
  return w0 * ta * (1.0f / 3.0f) + w2 * tb * (1.0f / 6.0f);
}

// v(m) returns Delta^+ phi at position i0 - 3 + m (m = 0..K+4); emit(p, dm, dp)
// receives node i0 + p.
template <int K, int WEIGHTS, class LoadV, class Emit>
__device__ __forceinline__ void sweep_stream(LoadV v_at, float rdx, float hdx, float eps, Emit emit) {
  // window state (indices are positions m as in weno_sweep)
  float v[K + 5];
  float s[K + 5];
  float T[K + 5];
  float qX[K + 6], qY[K + 6], qZ[K + 6];
  // arc length: D2 and F(D2) per position
  float D2[K + 6];
  FVal FD[K + 6];

  auto pos_s = [&](int m) {                  // s, and D2 for arc length
    s[m] = v[m] - v[m - 1];
    if (WEIGHTS == W_ARCLEN) D2[m] = s[m] * rdx;
  };
  auto pos_T = [&](int m) { T[m] = fmaf(-2.0f, s[m], s[m - 1] + s[m + 1]); };
  auto al_qX = [&](int m) {                  // interval (D2_m, R_m), R = 2 D2_m - D2_{m-1}
    const float R = fmaf(2.0f, D2[m], -D2[m - 1]);
    qX[m] = q_interval(D2[m], FD[m], R, f_eval(R), hdx, eps);
  };
  auto al_qY = [&](int m) { qY[m] = q_interval(D2[m], FD[m], D2[m + 1], FD[m + 1], hdx, eps); };
  auto al_qZ = [&](int m) {                  // interval (L_m, D2_m), L = 2 D2_m - D2_{m+1}
    const float Lv = fmaf(2.0f, D2[m], -D2[m + 1]);
    qZ[m] = q_interval(Lv, f_eval(Lv), D2[m], FD[m], hdx, eps);
  };
  auto jp_pair = [&](int m) {                // Jiang-Peng quantities of the pair (s_m, s_{m+1})
    const float x = s[m], y = s[m + 1];
    const float d = x - y, d13 = 13.0f * d * d;
    const float a = fmaf(-3.0f, y, x), b = x + y, c = fmaf(3.0f, x, -y);
    const float ea = fmaf(3.0f * a, a, d13) + eps, eb = fmaf(3.0f * b, b, d13) + eps, ec = fmaf(3.0f * c, c, d13) + eps;
    qX[m] = ea * ea;
    qY[m] = eb * eb;
    qZ[m] = ec * ec;
  };

  // ---- prologue: everything node 0 needs
#pragma unroll
  for (int m = 0; m <= 5; ++m) v[m] = v_at(m);
#pragma unroll
  for (int m = 1; m <= 5; ++m) pos_s(m);
#pragma unroll
  for (int m = 2; m <= 4; ++m) pos_T(m);
  if (WEIGHTS == W_ARCLEN) {
#pragma unroll
    for (int m = 2; m <= 4; ++m) FD[m] = f_eval(D2[m]);
    al_qX(2); al_qY(2); al_qZ(3);
    al_qX(3); al_qY(3); al_qZ(4);
  } else {
#pragma unroll
    for (int m = 1; m <= 4; ++m) jp_pair(m);
  }

#pragma unroll
  for (int p = 0; p < K; ++p) {
    // node p
    const float c = fmaf(7.0f / 12.0f, v[p + 2] + v[p + 3], -(1.0f / 12.0f) * (v[p + 1] + v[p + 4]));
    const float tb = T[p + 3];
    const float tb12 = tb * (1.0f / 12.0f), tb2 = 0.5f * tb;
    float cm, cp;
    if (WEIGHTS == W_ARCLEN) {
      cm = side_corr(qX[p + 2], qY[p + 2], qZ[p + 3], T[p + 2] * (1.0f / 3.0f), tb2, T[p + 2], tb);
      cp = side_corr(qZ[p + 4], qY[p + 3], qX[p + 3], T[p + 4] * (1.0f / 3.0f), tb2, T[p + 4], tb);
    } else {
      cm = side_corr(qX[p + 1], qY[p + 2], qZ[p + 3], T[p + 2] * (1.0f / 3.0f), tb2, T[p + 2], tb);
      cp = side_corr(qZ[p + 4], qY[p + 3], qX[p + 2], T[p + 4] * (1.0f / 3.0f), tb2, T[p + 4], tb);
    }
    emit(p, (c + tb12) - cm, (c - tb12) + cp);
    // advance the window by one position
    if (p + 1 < K) {
      v[p + 6] = v_at(p + 6);
      pos_s(p + 6);
      pos_T(p + 5);
      if (WEIGHTS == W_ARCLEN) {
        FD[p + 5] = f_eval(D2[p + 5]);
        al_qX(p + 4);
        al_qY(p + 4);
        al_qZ(p + 5);
      } else {
        jp_pair(p + 5);
      }
    }
  }
}

}  // namespace alw
