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
// The central parts are formed from d_m = s_{m+1} - s_m (s_m = v_m - v_{m-1}): for the node between
// v_2 and v_3 of its window, c + T_b/12 = (v_2 + v_3)/2 - d_2/6 and c - T_b/12 = (v_2 + v_3)/2 - d_3/6,
// and T_m = d_m - d_{m-1}; the widths d_m / dx are those of the arc-length intervals.
//
// Short intervals.  The interval mean G takes the trapezoid value (s_a + s_b) / 2 whenever the
// interval [a, b] is short against its end values (|b - a| <= (s_a + s_b) / 64, s = sqrt(1 + u^2)).
// On smooth data at fine grids every interval of a segment is that short (its width is a third
// difference of phi over dx^2, about phi_xxx dx), and then F, its logarithm and the interval
// reciprocals are never used.  sweep_stream_short computes only what the trapezoid branch needs
// and reports whether the segment qualifies: every width W_m = d_m / dx of the segment at most
// kShortH (which implies the trapezoid branch for all three interval kinds, because D2_{m+1} - D2_m,
// R_m - D2_m and D2_m - L_m all equal such a width up to the rounding of D2, R or L -- below 1e-4
// while |D2| <= kShortD2, against the margin 1/32 - kShortH -- and s >= 1), |D2| at the segment
// start at most kShortD2 and eps4 at most kShortEps4 (together
// these keep every weight denominator below 1e29, so the overflow branch of side_corr_v cannot be
// taken).  When the segment qualifies, both sweeps evaluate the same formulas on the same branches;
// their results agree to rounding (the compiler may select instructions for the two code paths
// differently), and the stage kernel decides between them from the segment's own data only.
#pragma once
#include "alw_device.cuh"

namespace alw {

constexpr float kShortH = 0.03f;      // largest width D2_{m+1} - D2_m of a short segment
constexpr float kShortD2 = 400.0f;    // largest |D2| at the start of a short segment
constexpr float kShortEps4 = 1.0e6f;  // largest 4 eps / dx^2 of a short segment

// ---- lane-wise operations on float and float2 ------------------------------------------
// Every add, subtract and multiply is rounded as written: the packed forms are PTX instructions
// with an explicit rounding mode, which the compiler does not contract into a fused multiply-add
// (the f32x2 intrinsics were contracted with a following subtraction in some contexts and not
// in others).  Fused multiply-adds are written as vfma.
__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float vsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float vfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ float vsplat(float x, float) { return x; }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) {
  float2 r;
  asm("{\n .reg .b64 a, b, d;\n mov.b64 a, {%2, %3};\n mov.b64 b, {%4, %5};\n add.rn.f32x2 d, a, b;\n"
      " mov.b64 {%0, %1}, d;\n}"
      : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
__device__ __forceinline__ float2 vsub(float2 a, float2 b) {
  float2 r;
  asm("{\n .reg .b64 a, b, d;\n mov.b64 a, {%2, %3};\n mov.b64 b, {%4, %5};\n sub.rn.f32x2 d, a, b;\n"
      " mov.b64 {%0, %1}, d;\n}"
      : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
__device__ __forceinline__ float2 vmul(float2 a, float2 b) {
  float2 r;
  asm("{\n .reg .b64 a, b, d;\n mov.b64 a, {%2, %3};\n mov.b64 b, {%4, %5};\n mul.rn.f32x2 d, a, b;\n"
      " mov.b64 {%0, %1}, d;\n}"
      : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 vsplat(float x, float2) { return make_float2(x, x); }

// Special-function-unit approximations in their flush-to-zero PTX forms (reciprocal square root,
// square root, base-2 logarithm, reciprocal).  No input here is subnormal -- 1 + u^2 >= 1, |u| + sqrt(1 + u^2) >= 1,
// weight denominators >= 1e-24 -- except 1/h for a vanishing interval, whose quotient the trapezoid
// branch discards, so the results equal those of the non-flushing forms.
__device__ __forceinline__ float sfu_rsqrt(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float sfu_sqrt(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
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

// s = sqrt(1 + u^2) as one square-root instruction per lane (a single rounding step, so that every
// code path that evaluates it gets the same bits)
template <class V>
__device__ __forceinline__ V s_eval_v(V u) {
  using LN = Lanes<V>;
  const V t = vfma(u, u, vsplat(1.0f, u));
  V r;
#pragma unroll
  for (int i = 0; i < LN::n; ++i) LN::at(r, i) = sfu_sqrt(LN::get(t, i));
  return r;
}

template <class V>
__device__ __forceinline__ FValV<V> f_eval_v(V u) {
  using LN = Lanes<V>;
  FValV<V> r;
  V lsg;
  r.s = s_eval_v(u);
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

// The side's correction (A0 T_a / 3 + A2 T_b / 2) / den as a pair (num, r) with correction =
// num * r (r = 1 / den; on the rare lanes whose products leave the float range, num = the
// correction and r = 1); ta3 = T_a / 3, tb2 = T_b / 2.  NEG (the "-" side, whose correction is
// subtracted) gives r = -1 / den (or -1), so that the caller adds num * r to the central part with
// one fused multiply-add on either side.
template <bool NEG, class V>
__device__ __forceinline__ void side_corr_v(V q0, V q1, V q2, V ta3, V tb2, V &num_out, V &r_out) {
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
    LN::at(rd, i) = sfu_rcp(NEG ? -dn : dn);
  }
  V nm = num;
  if (!ok) {
#pragma unroll
    for (int i = 0; i < LN::n; ++i) {
      const float dn = LN::get(den, i);
      if (!(dn < 1e30f)) {
        LN::at(nm, i) = side_corr_wide(LN::get(q0, i), LN::get(q1, i), LN::get(q2, i), LN::get(ta3, i),
                                       LN::get(tb2, i));
        LN::at(rd, i) = NEG ? -1.0f : 1.0f;
      }
    }
  }
  num_out = nm;
  r_out = rd;
}

// v_at(m) returns Delta^+ phi at position i0 - 3 + m (m = 0..K+4) per lane; emit(p, dm, dp)
// receives node i0 + p.  rdx = 1/dx, eps4 = 4 eps / dx^2 (per lane).
// Every lane of v holds a width at most kShortH (NaN fails).
template <class V>
__device__ __forceinline__ bool short_width(V h) {
  using LN = Lanes<V>;
  bool ok = true;
#pragma unroll
  for (int i = 0; i < LN::n; ++i) ok &= fabsf(LN::get(h, i)) <= kShortH;
  return ok;
}

// The size conditions of a short segment on |D2| at its start and on eps4 (NaN fails).
template <class V>
__device__ __forceinline__ bool short_sizes(V d2, V eps4) {
  using LN = Lanes<V>;
  bool ok = true;
#pragma unroll
  for (int i = 0; i < LN::n; ++i)
    ok &= (fabsf(LN::get(d2, i)) <= kShortD2) & (LN::get(eps4, i) <= kShortEps4);
  return ok;
}

// The extrapolated interval ends R_m = 2 D2_m - D2_{m-1} and L_m = 2 D2_m - D2_{m+1}, formed as
// D2_m plus or minus the neighbouring width W = d / dx (the quantity the short-interval test
// inspects; one operation each).
template <class V>
__device__ __forceinline__ V r_end(V d2m, V w_prev) { return vadd(d2m, w_prev); }
template <class V>
__device__ __forceinline__ V l_end(V d2m, V w_m) { return vsub(d2m, w_m); }

template <int K, int WEIGHTS, class V, class LoadV, class Emit>
__device__ __forceinline__ void sweep_stream(LoadV v_at, V rdx, V eps4, V eps, Emit emit) {
  V v[K + 5];
  V s[K + 5];
  V dd[K + 5];                               // d_m = s_{m+1} - s_m
  V T[K + 5];
  V T3[K + 5];                               // T_m / 3
  V qX[K + 6], qY[K + 6], qZ[K + 6];
  V D2[K + 6];
  V W[K + 6];                                // W_m = d_m / dx = D2_{m+1} - D2_m up to rounding
  FValV<V> FD[K + 6];

  auto pos_s = [&](int m) {                  // s, d, and D2 and W for arc length
    s[m] = vsub(v[m], v[m - 1]);
    if (WEIGHTS == W_ARCLEN) D2[m] = vmul(s[m], rdx);
    if (m >= 2) {
      dd[m - 1] = vsub(s[m], s[m - 1]);
      if (WEIGHTS == W_ARCLEN) W[m - 1] = vmul(dd[m - 1], rdx);
    }
  };
  const V c13 = vsplat(1.0f / 3.0f, eps);
  auto pos_T = [&](int m) {
    T[m] = vsub(dd[m], dd[m - 1]);
    T3[m] = vmul(T[m], c13);
  };
  auto al_qX = [&](int m) {                  // interval (D2_m, R_m), R = 2 D2_m - D2_{m-1}
    const V R = r_end(D2[m], W[m - 1]);
    qX[m] = q_interval_v(D2[m], FD[m], R, f_eval_v(R), eps4);
  };
  auto al_qY = [&](int m) { qY[m] = q_interval_v(D2[m], FD[m], D2[m + 1], FD[m + 1], eps4); };
  auto al_qZ = [&](int m) {                  // interval (L_m, D2_m), L = 2 D2_m - D2_{m+1}
    const V Lv = l_end(D2[m], W[m]);
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

  const V cm16 = vsplat(-1.0f / 6.0f, eps), c12 = vsplat(0.5f, eps);
#pragma unroll
  for (int p = 0; p < K; ++p) {
    // node p: phi^- = (c + T_b/12) - corr^-, phi^+ = (c - T_b/12) + corr^+
    const V mid = vmul(c12, vadd(v[p + 2], v[p + 3]));
    const V tb2 = vmul(c12, T[p + 3]);
    V nm, rm, np, rp;
    if (WEIGHTS == W_ARCLEN) {
      side_corr_v<true>(qX[p + 2], qY[p + 2], qZ[p + 3], T3[p + 2], tb2, nm, rm);
      side_corr_v<false>(qZ[p + 4], qY[p + 3], qX[p + 3], T3[p + 4], tb2, np, rp);
    } else {
      side_corr_v<true>(qX[p + 1], qY[p + 2], qZ[p + 3], T3[p + 2], tb2, nm, rm);
      side_corr_v<false>(qZ[p + 4], qY[p + 3], qX[p + 2], T3[p + 4], tb2, np, rp);
    }
    emit(p, vfma(nm, rm, vfma(dd[p + 2], cm16, mid)), vfma(np, rp, vfma(dd[p + 3], cm16, mid)));
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

// Arc-length sweep of segments on which every interval takes the trapezoid branch (see the header
// comment): the square roots s = sqrt(1 + u^2) of the interval ends, the trapezoid values and the
// weights, with the operations of sweep_stream on those branches.  Called by all 32 threads of a
// warp; returns, uniformly across the warp, whether every segment of the warp (both lanes of all
// threads) met the conditions (checked after the prologue, where a failing warp stops at once,
// and after the last node).  When it returns false the emitted values, if any, are not to be
// used and the caller sweeps the warp's segments again with sweep_stream.
template <int K, class V, class LoadV, class Emit>
__device__ __forceinline__ bool sweep_stream_short(LoadV v_at, V rdx, V eps4, Emit emit) {
  using LN = Lanes<V>;
  V v[K + 5];
  V s[K + 5];
  V dd[K + 5];
  V T[K + 5];
  V T3[K + 5];
  V D2[K + 6];
  V W[K + 6];
  V S[K + 6];                                // S_m = sqrt(1 + D2_m^2)
  V qX[K + 6], qY[K + 6], qZ[K + 6];
  bool ok = true;

  auto sq = [&](V u) { return s_eval_v(u); };   // FValV::s of f_eval_v
  auto qv = [&](V sa, V sb) {                // q of q_interval_v on its trapezoid branch
    const V ss = vadd(sa, sb);
    const V e = vfma(ss, ss, eps4);
    return vmul(e, e);
  };
  auto pos_s = [&](int m) {
    s[m] = vsub(v[m], v[m - 1]);
    D2[m] = vmul(s[m], rdx);
    if (m >= 2) {
      dd[m - 1] = vsub(s[m], s[m - 1]);
      W[m - 1] = vmul(dd[m - 1], rdx);
      ok &= short_width(W[m - 1]);
    }
  };
  const V c13 = vsplat(1.0f / 3.0f, rdx);
  auto pos_T = [&](int m) {
    T[m] = vsub(dd[m], dd[m - 1]);
    T3[m] = vmul(T[m], c13);
  };
  auto al_qX = [&](int m) { qX[m] = qv(S[m], sq(r_end(D2[m], W[m - 1]))); };
  auto al_qY = [&](int m) { qY[m] = qv(S[m], S[m + 1]); };
  auto al_qZ = [&](int m) { qZ[m] = qv(sq(l_end(D2[m], W[m])), S[m]); };
  // side_corr_v when the denominator is known to be in range (neg: r = -1 / den)
  auto corr = [&](V q0, V q1, V q2, V ta3, V tb2, bool neg, V &num, V &rd) {
    const V A0 = vmul(q1, q2), A1 = vmul(q0, q2), A2 = vmul(q0, q1);
    const V den = vfma(vsplat(6.0f, q0), A1, vfma(vsplat(3.0f, q0), A2, A0));
    num = vfma(A0, ta3, vmul(A2, tb2));
#pragma unroll
    for (int i = 0; i < LN::n; ++i) LN::at(rd, i) = sfu_rcp(neg ? -LN::get(den, i) : LN::get(den, i));
  };

#pragma unroll
  for (int m = 0; m <= 5; ++m) v[m] = v_at(m);
#pragma unroll
  for (int m = 1; m <= 5; ++m) pos_s(m);
#pragma unroll
  for (int m = 2; m <= 4; ++m) pos_T(m);
#pragma unroll
  for (int m = 2; m <= 4; ++m) S[m] = sq(D2[m]);
  al_qX(2); al_qY(2); al_qZ(3);
  al_qX(3); al_qY(3); al_qZ(4);
  ok &= short_sizes(D2[2], eps4);
  if (!__all_sync(0xffffffffu, ok)) return false;

  const V cm16 = vsplat(-1.0f / 6.0f, rdx), c12 = vsplat(0.5f, rdx);
#pragma unroll
  for (int p = 0; p < K; ++p) {
    const V mid = vmul(c12, vadd(v[p + 2], v[p + 3]));
    const V tb2 = vmul(c12, T[p + 3]);
    V nm, rm, np, rp;
    corr(qX[p + 2], qY[p + 2], qZ[p + 3], T3[p + 2], tb2, true, nm, rm);
    corr(qZ[p + 4], qY[p + 3], qX[p + 3], T3[p + 4], tb2, false, np, rp);
    emit(p, vfma(nm, rm, vfma(dd[p + 2], cm16, mid)), vfma(np, rp, vfma(dd[p + 3], cm16, mid)));
    if (p + 1 < K) {
      v[p + 6] = v_at(p + 6);
      pos_s(p + 6);
      pos_T(p + 5);
      S[p + 5] = sq(D2[p + 5]);
      al_qX(p + 4);
      al_qY(p + 4);
      al_qZ(p + 5);
    }
  }
  return __all_sync(0xffffffffu, ok);
}

}  // namespace alw
