// Streaming float sweep of the WENO reconstruction along line segments, in a
// scalar (float) and a packed two-lane (float2) form.
//
// Same arithmetic as weno_sweep<float> (alw_device.cuh), reorganised so that
// each step of the sliding window computes only the quantities that become
// newly needed (one Delta^+ value, one second difference, three F values,
// three interval means, one T value) and hands each node's (phi^-, phi^+) to
// a callback as soon as it is complete; dead values retire at once, which
// keeps register pressure low.  In the float2 form the two lanes are two
// independent segments (the 2D stage kernel puts a row segment in .x and a
// column segment in .y) that run the same instruction stream, so every
// float add/mul/fma is one packed sm_100+ instruction for both.
//
// Indicators: q_k = (eps + beta_k)^2 with beta_k = (dx G_k)^2 enters the
// weights only through ratios, so all q_k may be scaled by one factor: with
// G2 = 2 G (the divided difference (F(b) - F(a)) / (b - a) without the 1/2)
// the kernel uses q_k = (4 eps / dx^2 + G2_k^2)^2 = 16 q_k / dx^4.
//
// Weights and the compact form are folded into one reciprocal per side:
// with A0 = q1 q2, A1 = q0 q2, A2 = q0 q1,
//   den = A0 + 6 A1 + 3 A2  ( = 10 sum_k d_k prod_{l != k} q_l ),
//   omega_0 = A0 / den, omega_2 = 3 A2 / den,
//   phi^- = (c + T_b/12) - (A0 T_a / 3 + A2 T_b / 2) / den,
//   phi^+ = (c - T_b/12) + (A0' T_c / 3 + A2' T_b / 2) / den'.
#pragma once
#include "alw_device.cuh"

namespace alw {

// ---- lane-wise operations on float and float2 ------------------------------------------
__device__ __forceinline__ float vadd(float a, float b) { return a + b; }
__device__ __forceinline__ float vsub(float a, float b) { return a - b; }
__device__ __forceinline__ float vmul(float a, float b) { return a * b; }
__device__ __forceinline__ float vfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ float vsplat(float x, float) { return x; }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 vsub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 vsplat(float x, float2) { return make_float2(x, x); }

// Special-function-unit approximations in their flush-to-zero PTX forms (reciprocal square root,
// base-2 logarithm, reciprocal).  No input here is subnormal -- 1 + u^2 >= 1, |u| + sqrt(1 + u^2) >= 1,
// weight denominators >= 1e-24 -- except 1/h for a vanishing interval, whose quotient the trapezoid
// branch discards, so the results equal those of the non-flushing forms.
__device__ __forceinline__ float sfu_rsqrt(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float sfu_lg2(float x) {
  float r;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float sfu_rcp(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
// sine and cosine of the Hamiltonians (absolute error about 2^-20 for moderate arguments; a subnormal argument
// gives 0 instead of itself)
__device__ __forceinline__ float sfu_sin(float x) {
  float r;
  asm("sin.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float sfu_cos(float x) {
  float r;
  asm("cos.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

template <class V> struct Lanes;
template <> struct Lanes<float> {
  static constexpr int n = 1;
  __device__ __forceinline__ static float &at(float &v, int) { return v; }
  __device__ __forceinline__ static float get(const float &v, int) { return v; }
};
template <> struct Lanes<float2> {
  static constexpr int n = 2;
  __device__ __forceinline__ static float &at(float2 &v, int i) { return i == 0 ? v.x : v.y; }
  __device__ __forceinline__ static float get(const float2 &v, int i) { return i == 0 ? v.x : v.y; }
};

template <class V> struct FValV {
  V F, s;  // F(u) = u sqrt(1+u^2) + asinh(u), s = sqrt(1+u^2)
};

template <class V>
__device__ __forceinline__ FValV<V> f_eval_v(V u) {
  using LN = Lanes<V>;
  FValV<V> r;
  const V t = vfma(u, u, vsplat(1.0f, u));
  V rs, lsg;
#pragma unroll
  for (int i = 0; i < LN::n; ++i) LN::at(rs, i) = sfu_rsqrt(LN::get(t, i));
  r.s = vmul(t, rs);
  // |u| + s per lane (the absolute value is an operand modifier of the scalar add)
#pragma unroll
  for (int i = 0; i < LN::n; ++i)
    LN::at(lsg, i) = copysignf(sfu_lg2(fabsf(LN::get(u, i)) + LN::get(r.s, i)), LN::get(u, i));
  // asinh|u| = ln(|u| + sqrt(1+u^2)); absolute error of the base-2 log ~ 2^-22
  r.F = vfma(vsplat(0.693147180559945f, u), lsg, vmul(u, r.s));
  return r;
}

// q = (eps4 + G2^2)^2 for the interval [a, b] (eps4 = 4 eps / dx^2; see the header comment).
template <class V>
__device__ __forceinline__ V q_interval_v(V a, FValV<V> fa, V b, FValV<V> fb, V eps4) {
  using LN = Lanes<V>;
  const V h = vsub(b, a);
  const V ss = vadd(fa.s, fb.s);          // trapezoid value of G2
  const V dF = vsub(fb.F, fa.F);
  const V thr = vmul(vsplat(0.015625f, h), ss);
  V rh;
#pragma unroll
  for (int i = 0; i < LN::n; ++i) LN::at(rh, i) = sfu_rcp(LN::get(h, i));
  const V gd = vmul(dF, rh);
  V g;
#pragma unroll
  for (int i = 0; i < LN::n; ++i) {
    // divided difference, or the trapezoid mean when the interval is short compared with its ends
    LN::at(g, i) = (fabsf(LN::get(h, i)) > LN::get(thr, i)) ? LN::get(gd, i) : LN::get(ss, i);
  }
  const V e = vfma(g, g, eps4);
  return vmul(e, e);
}

// Slow path of side_corr_v for one lane, when the q products leave the safe float range
// (kept out of line: it is rare and would otherwise be inlined at every node).
static __device__ __noinline__ float side_corr_wide(float q0, float q1, float q2, float ta3, float tb2) {
  const float a0 = __fdividef(0.1f, q0), a1 = __fdividef(0.6f, q1), a2 = __fdividef(0.3f, q2);
  const float r = __fdividef(1.0f, a0 + a1 + a2);
  return (a0 * r) * ta3 + (a2 * r) * (1.0f / 3.0f) * tb2;
}

// The side's correction (A0 T_a / 3 + A2 T_b / 2) / den; ta3 = T_a / 3, tb2 = T_b / 2.
template <class V>
__device__ __forceinline__ V side_corr_v(V q0, V q1, V q2, V ta3, V tb2) {
  using LN = Lanes<V>;
  const V A0 = vmul(q1, q2), A1 = vmul(q0, q2), A2 = vmul(q0, q1);
  const V den = vfma(vsplat(6.0f, q0), A1, vfma(vsplat(3.0f, q0), A2, A0));
  const V num = vfma(A0, ta3, vmul(A2, tb2));
  // den >= A0 > 0 cannot underflow (arc length: q >= 16; Jiang-Peng: q >= eps^2), so only the
  // upper end of the float range needs a check (NaN fails it too)
  V rd;
  bool ok = true;
#pragma unroll
  for (int i = 0; i < LN::n; ++i) {
    const float dn = LN::get(den, i);
    ok = ok && (dn < 1e30f);
    LN::at(rd, i) = sfu_rcp(dn);
  }
  V out = vmul(num, rd);
  if (!ok) {
#pragma unroll
    for (int i = 0; i < LN::n; ++i) {
      const float dn = LN::get(den, i);
      if (!(dn < 1e30f))
        LN::at(out, i) = side_corr_wide(LN::get(q0, i), LN::get(q1, i), LN::get(q2, i), LN::get(ta3, i),
                                        LN::get(tb2, i));
    }
  }
  return out;
}

// v_at(m) returns Delta^+ phi at position i0 - 3 + m (m = 0..K+4) per lane; emit(p, dm, dp)
// receives node i0 + p.  rdx = 1/dx, eps4 = 4 eps / dx^2 (per lane).
template <int K, int WEIGHTS, class V, class LoadV, class Emit>
__device__ __forceinline__ void sweep_stream(LoadV v_at, V rdx, V eps4, V eps, Emit emit) {
  V v[K + 5];
  V s[K + 5];
  V T[K + 5];
  V qX[K + 6], qY[K + 6], qZ[K + 6];
  V D2[K + 6];
  FValV<V> FD[K + 6];
  const V two = vsplat(2.0f, eps), mtwo = vsplat(-2.0f, eps);

  auto pos_s = [&](int m) {                  // s, and D2 for arc length
    s[m] = vsub(v[m], v[m - 1]);
    if (WEIGHTS == W_ARCLEN) D2[m] = vmul(s[m], rdx);
  };
  auto pos_T = [&](int m) { T[m] = vfma(mtwo, s[m], vadd(s[m - 1], s[m + 1])); };
  auto al_qX = [&](int m) {                  // interval (D2_m, R_m), R = 2 D2_m - D2_{m-1}
    const V R = vsub(vmul(two, D2[m]), D2[m - 1]);
    qX[m] = q_interval_v(D2[m], FD[m], R, f_eval_v(R), eps4);
  };
  auto al_qY = [&](int m) { qY[m] = q_interval_v(D2[m], FD[m], D2[m + 1], FD[m + 1], eps4); };
  auto al_qZ = [&](int m) {                  // interval (L_m, D2_m), L = 2 D2_m - D2_{m+1}
    const V Lv = vsub(vmul(two, D2[m]), D2[m + 1]);
    qZ[m] = q_interval_v(Lv, f_eval_v(Lv), D2[m], FD[m], eps4);
  };
  auto jp_pair = [&](int m) {                // Jiang-Peng quantities of the pair (s_m, s_{m+1})
    const V x = s[m], y = s[m + 1];
    const V d = vsub(x, y);
    const V d13 = vmul(vsplat(13.0f, x), vmul(d, d));
    const V a = vfma(vsplat(-3.0f, x), y, x), b = vadd(x, y), c = vsub(vmul(vsplat(3.0f, x), x), y);
    const V three = vsplat(3.0f, x);
    const V ea = vadd(vfma(vmul(three, a), a, d13), eps), eb = vadd(vfma(vmul(three, b), b, d13), eps);
    const V ec = vadd(vfma(vmul(three, c), c, d13), eps);
    qX[m] = vmul(ea, ea);
    qY[m] = vmul(eb, eb);
    qZ[m] = vmul(ec, ec);
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
    for (int m = 2; m <= 4; ++m) FD[m] = f_eval_v(D2[m]);
    al_qX(2); al_qY(2); al_qZ(3);
    al_qX(3); al_qY(3); al_qZ(4);
  } else {
#pragma unroll
    for (int m = 1; m <= 4; ++m) jp_pair(m);
  }

  const V c712 = vsplat(7.0f / 12.0f, eps), cm112 = vsplat(-1.0f / 12.0f, eps);
  const V c13 = vsplat(1.0f / 3.0f, eps), c12 = vsplat(0.5f, eps);
#pragma unroll
  for (int p = 0; p < K; ++p) {
    // node p
    const V c = vfma(c712, vadd(v[p + 2], v[p + 3]), vmul(cm112, vadd(v[p + 1], v[p + 4])));
    const V tb = T[p + 3];
    const V tb12 = vmul(tb, vsplat(1.0f / 12.0f, eps)), tb2 = vmul(c12, tb);
    V cm, cp;
    if (WEIGHTS == W_ARCLEN) {
      cm = side_corr_v(qX[p + 2], qY[p + 2], qZ[p + 3], vmul(T[p + 2], c13), tb2);
      cp = side_corr_v(qZ[p + 4], qY[p + 3], qX[p + 3], vmul(T[p + 4], c13), tb2);
    } else {
      cm = side_corr_v(qX[p + 1], qY[p + 2], qZ[p + 3], vmul(T[p + 2], c13), tb2);
      cp = side_corr_v(qZ[p + 4], qY[p + 3], qX[p + 2], vmul(T[p + 4], c13), tb2);
    }
    emit(p, vsub(vadd(c, tb12), cm), vadd(vsub(c, tb12), cp));
    // advance the window by one position
    if (p + 1 < K) {
      v[p + 6] = v_at(p + 6);
      pos_s(p + 6);
      pos_T(p + 5);
      if (WEIGHTS == W_ARCLEN) {
        FD[p + 5] = f_eval_v(D2[p + 5]);
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
