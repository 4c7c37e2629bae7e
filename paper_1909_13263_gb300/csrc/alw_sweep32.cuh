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
// and T_m = d_m - d_{m-1}; the widths d_m / dx are those of the arc-length intervals.  The arc-length
// sweeps take their input as u = v / dx (the differences pass scales by 1/dx^2), so that the second
// differences D2_m = u_m - u_{m-1} and the widths W_m = D2_{m+1} - D2_m = d_m / dx come without a
// multiply; dx enters once, in the constants dx/2, dx/3, -dx/6 of the central parts and of T_a/3, T_b/2.
// The Jiang-Peng sweep needs no D2 and keeps v.
//
// Short intervals.  The interval mean G takes the trapezoid value (s_a + s_b) / 2 whenever the
// interval [a, b] is short against its end values (|b - a| <= (s_a + s_b) / 64, s = sqrt(1 + u^2)).
// On smooth data at fine grids every interval of a segment is that short (its width is a third
// difference of phi over dx^2, about phi_xxx dx), and then F, its logarithm and the interval
// reciprocals are never used.  sweep_stream_short computes only what the trapezoid branch needs
// and reports whether the segment qualifies: every width W_m of the segment at most
// kShortH (which implies the trapezoid branch for all three interval kinds, because D2_{m+1} - D2_m
// is such a width and R_m - D2_m and D2_m - L_m equal one up to the rounding of R or L -- below 1e-4
// while |D2| <= kShortD2, against the margin 1/32 - kShortH -- and s >= 1), |D2| at the segment
// start at most kShortD2 and eps4 at most kShortEps4 (together
// these keep every weight denominator below 1e29, so the overflow branch of group_corr_v is not
// needed).  When the segment qualifies, both sweeps evaluate the same formulas on the same branches;
// their results agree to rounding (the compiler may select instructions for the two code paths
// differently), and the stage kernel decides between them from the segment's own data only.
#pragma once
#include <type_traits>

#include "alw_device.cuh"

// The sweeps' window arrays are filled position by position after the lambdas that read them are defined;
// the front end's "used before its value is set" (549) fires at each such capture although every element
// is written before it is read.
#pragma nv_diagnostic push
#pragma nv_diag_suppress 549

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

// Slow path of group_corr_v for one lane, when the q products leave the safe float range
// (kept out of line: it is rare and would otherwise be inlined at every node).
static __device__ __noinline__ float side_corr_wide(float q0, float q1, float q2, float ta3, float tb2) {
  const float a0 = __fdividef(0.1f, q0), a1 = __fdividef(0.6f, q1), a2 = __fdividef(0.3f, q2);
  const float r = __fdividef(1.0f, a0 + a1 + a2);
  return (a0 * r) * ta3 + (a2 * r) * (1.0f / 3.0f) * tb2;
}

// Per-lane constants of an arc-length sweep (x lane: dx; y lane: dy).
template <class V> struct SweepConsts {
  V eps4;          // 4 eps / dx^2
  V h2, h3, mh6;   // dx / 2, dx / 3, -dx / 6 (the central parts and T_a / 3, T_b / 2 back in units of phi_x)
};

// The corrections of the two sides that read one stencil of indicators.  The "-" side of node j reads
// (q0, q1, q2) = (g0, g1, g2) and the "+" side of node j - 1 reads the same three indicators mirrored,
// (q0, q1, q2) = (g2, g1, g0); the products g1 g2, g0 g2, g0 g1 therefore serve both sides:
//   "-": A0 = g1 g2, A1 = g0 g2, A2 = g0 g1;     "+": A0 = g0 g1, A1 = g0 g2, A2 = g1 g2,
// den = A0 + 6 A1 + 3 A2 and num = A0 T_a / 3 + A2 T_b / 2 on either side (ta = T_a / 3, tb = T_b / 2 of
// that side).  Each side's correction num / den is returned as a pair (num, r) with correction = num * r:
// r = -1 / den on the "-" side (whose correction is subtracted) and 1 / den on the "+" side, so that the
// caller adds num * r to the central part with one fused multiply-add.  CHECKED: on lanes whose
// denominator leaves the safe float range (or is NaN), num = the correction from side_corr_wide and
// r = -1 or 1.  MINUS / PLUS select the sides wanted.  (The sweeps with the range check form each
// side on its own -- sharing the products there measured slower, the rare out-of-line fallback
// making the shared values live across its call -- and the short-interval sweep forms both.)
template <bool CHECKED, bool MINUS, bool PLUS, class V>
__device__ __forceinline__ void group_corr_v(V g0, V g1, V g2, V ta_m, V tb_m, V ta_p, V tb_p, V &num_m, V &r_m,
                                             V &num_p, V &r_p) {
  using LN = Lanes<V>;
  const V p12 = vmul(g1, g2), p02 = vmul(g0, g2), p01 = vmul(g0, g1);
  // den >= A0 > 0 cannot underflow (arc length: q >= 16; Jiang-Peng: q >= eps^2), so only the upper end
  // of the float range needs a check (NaN fails it too)
  auto side = [&](V a0, V a2, V ta, V tb, bool neg, V q0, V q1, V q2, V &num_out, V &r_out) {
    const V den = vfma(vsplat(6.0f, q0), p02, vfma(vsplat(3.0f, q0), a2, a0));
    V nm = vfma(a0, ta, vmul(a2, tb));
    V rd;
    bool ok = true;
#pragma unroll
    for (int i = 0; i < LN::n; ++i) {
      const float dn = LN::get(den, i);
      if (CHECKED) ok = ok && (dn < 1e30f);
      LN::at(rd, i) = sfu_rcp(neg ? -dn : dn);
    }
    if (CHECKED && !ok) {
#pragma unroll
      for (int i = 0; i < LN::n; ++i) {
        const float dn = LN::get(den, i);
        if (!(dn < 1e30f)) {
          LN::at(nm, i) = side_corr_wide(LN::get(q0, i), LN::get(q1, i), LN::get(q2, i), LN::get(ta, i),
                                         LN::get(tb, i));
          LN::at(rd, i) = neg ? -1.0f : 1.0f;
        }
      }
    }
    num_out = nm;
    r_out = rd;
  };
  if (MINUS) side(p12, p01, ta_m, tb_m, true, g0, g1, g2, num_m, r_m);
  if (PLUS) side(p01, p12, ta_p, tb_p, false, g2, g1, g0, num_p, r_p);
}

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
// D2_m plus or minus the neighbouring width W (the quantity the short-interval test inspects; one
// operation each).
template <class V>
__device__ __forceinline__ V r_end(V d2m, V w_prev) { return vadd(d2m, w_prev); }
template <class V>
__device__ __forceinline__ V l_end(V d2m, V w_m) { return vsub(d2m, w_m); }

// The window of the arc-length sweeps.  u_at(m) returns u = Delta^+ phi / dx^2 at position i0 - 3 + m
// (m = 0..K+4) per lane; in these units the second differences D2_m = u_m - u_{m-1} and the widths
// W_m = D2_{m+1} - D2_m need no scaling, and T_m = W_m - W_{m-1} is T / dx of the first-difference
// form.  Per position: D2_m, W_{m-1} and the two scaled copies of T_{m-1}, ta = T dx / 3, tb = T dx / 2.
template <int N, class V>
struct Window {
  V u[N], D2[N], W[N], Ta[N], Tb[N];
  __device__ __forceinline__ void pos(int m, const SweepConsts<V> &c) {
    D2[m] = vsub(u[m], u[m - 1]);
    if (m >= 2) W[m - 1] = vsub(D2[m], D2[m - 1]);
    if (m >= 3) {
      const V T = vsub(W[m - 1], W[m - 2]);
      Ta[m - 1] = vmul(T, c.h3);
      Tb[m - 1] = vmul(T, c.h2);
    }
  }
  // node p: phi^- = (c + T_b / 12) - corr^-, phi^+ = (c - T_b / 12) + corr^+, with
  // c +- T_b / 12 = dx ((u_{p+2} + u_{p+3}) / 2 - W_{p+2 or p+3} / 6)
  template <class Emit>
  __device__ __forceinline__ void emit_node(int p, const SweepConsts<V> &c, V nm, V rm, V np, V rp, Emit &emit) {
    const V mid = vmul(c.h2, vadd(u[p + 2], u[p + 3]));
    emit(p, vfma(nm, rm, vfma(W[p + 2], c.mh6, mid)), vfma(np, rp, vfma(W[p + 3], c.mh6, mid)));
  }
};

// Stencil j of an arc-length segment, (X_{j+2}, Y_{j+2}, Z_{j+3}) with T_{j+2}, T_{j+3}, serves the "-"
// side of node j and the "+" side of node j - 1 (see group_corr_v).  emit(p, dm, dp) receives node i0 + p.
template <int K, class V, class LoadV, class Emit>
__device__ __forceinline__ void sweep_stream(LoadV u_at, const SweepConsts<V> &c, Emit emit) {
  Window<K + 5, V> w;
  V qX[K + 6], qY[K + 6], qZ[K + 6];
  FValV<V> FD[K + 6];

  auto al_qX = [&](int m) {                  // interval (D2_m, R_m), R = 2 D2_m - D2_{m-1}
    const V R = r_end(w.D2[m], w.W[m - 1]);
    qX[m] = q_interval_v(w.D2[m], FD[m], R, f_eval_v(R), c.eps4);
  };
  auto al_qY = [&](int m) { qY[m] = q_interval_v(w.D2[m], FD[m], w.D2[m + 1], FD[m + 1], c.eps4); };
  auto al_qZ = [&](int m) {                  // interval (L_m, D2_m), L = 2 D2_m - D2_{m+1}
    const V Lv = l_end(w.D2[m], w.W[m]);
    qZ[m] = q_interval_v(Lv, f_eval_v(Lv), w.D2[m], FD[m], c.eps4);
  };

  // ---- prologue: everything node 0 needs
#pragma unroll
  for (int m = 0; m <= 5; ++m) w.u[m] = u_at(m);
#pragma unroll
  for (int m = 1; m <= 5; ++m) w.pos(m, c);
#pragma unroll
  for (int m = 2; m <= 4; ++m) FD[m] = f_eval_v(w.D2[m]);
  al_qX(2); al_qY(2); al_qZ(3);
  al_qX(3); al_qY(3); al_qZ(4);

#pragma unroll
  for (int p = 0; p < K; ++p) {
    V nm, rm, np, rp, unused0, unused1;
    group_corr_v<true, true, false>(qX[p + 2], qY[p + 2], qZ[p + 3], w.Ta[p + 2], w.Tb[p + 3], w.Ta[p + 2],
                                    w.Tb[p + 3], nm, rm, unused0, unused1);
    group_corr_v<true, false, true>(qX[p + 3], qY[p + 3], qZ[p + 4], w.Ta[p + 3], w.Tb[p + 4], w.Ta[p + 4],
                                    w.Tb[p + 3], unused0, unused1, np, rp);
    w.emit_node(p, c, nm, rm, np, rp, emit);
    // advance the window by one position
    if (p + 1 < K) {
      w.u[p + 6] = u_at(p + 6);
      w.pos(p + 6, c);
      FD[p + 5] = f_eval_v(w.D2[p + 5]);
      al_qX(p + 4);
      al_qY(p + 4);
      al_qZ(p + 5);
    }
  }
}

// Jiang-Peng sweep, in units of the first differences: v_at(m) returns Delta^+ phi / dx at position
// i0 - 3 + m; s_m = v_m - v_{m-1}, d_m = s_{m+1} - s_m, T_m = d_m - d_{m-1}.  Stencil j is
// (X_{j+1}, Y_{j+2}, Z_{j+3}), the indicators of the pairs (s_m, s_{m+1}).
template <int K, class V, class LoadV, class Emit>
__device__ __forceinline__ void sweep_stream_jp(LoadV v_at, V eps, Emit emit) {
  V v[K + 5];
  V s[K + 5];
  V dd[K + 5];
  V T[K + 5];
  V T3[K + 5];                               // T_m / 3
  V qX[K + 6], qY[K + 6], qZ[K + 6];

  auto pos_s = [&](int m) {
    s[m] = vsub(v[m], v[m - 1]);
    if (m >= 2) dd[m - 1] = vsub(s[m], s[m - 1]);
  };
  const V c13 = vsplat(1.0f / 3.0f, eps);
  auto pos_T = [&](int m) {
    T[m] = vsub(dd[m], dd[m - 1]);
    T3[m] = vmul(T[m], c13);
  };
  auto jp_pair = [&](int m) {
    const V x = s[m], y = s[m + 1];
    const V d = vsub(x, y);
    const V d13 = vmul(vsplat(13.0f, x), vmul(d, d));
    const V a = vfma(vsplat(-3.0f, x), y, x), b = vadd(x, y), cc = vsub(vmul(vsplat(3.0f, x), x), y);
    const V three = vsplat(3.0f, x);
    const V ea = vadd(vfma(vmul(three, a), a, d13), eps), eb = vadd(vfma(vmul(three, b), b, d13), eps);
    const V ec = vadd(vfma(vmul(three, cc), cc, d13), eps);
    qX[m] = vmul(ea, ea);
    qY[m] = vmul(eb, eb);
    qZ[m] = vmul(ec, ec);
  };

#pragma unroll
  for (int m = 0; m <= 5; ++m) v[m] = v_at(m);
#pragma unroll
  for (int m = 1; m <= 5; ++m) pos_s(m);
#pragma unroll
  for (int m = 2; m <= 4; ++m) pos_T(m);
#pragma unroll
  for (int m = 1; m <= 4; ++m) jp_pair(m);

  const V cm16 = vsplat(-1.0f / 6.0f, eps), c12 = vsplat(0.5f, eps);
#pragma unroll
  for (int p = 0; p < K; ++p) {
    const V mid = vmul(c12, vadd(v[p + 2], v[p + 3]));
    const V tb2 = vmul(c12, T[p + 3]);
    V nm, rm, np, rp, unused0, unused1;
    group_corr_v<true, true, false>(qX[p + 1], qY[p + 2], qZ[p + 3], T3[p + 2], tb2, T3[p + 2], tb2, nm, rm,
                                    unused0, unused1);
    group_corr_v<true, false, true>(qX[p + 2], qY[p + 3], qZ[p + 4], T3[p + 4], tb2, T3[p + 4], tb2, unused0,
                                    unused1, np, rp);
    emit(p, vfma(nm, rm, vfma(dd[p + 2], cm16, mid)), vfma(np, rp, vfma(dd[p + 3], cm16, mid)));
    if (p + 1 < K) {
      v[p + 6] = v_at(p + 6);
      pos_s(p + 6);
      pos_T(p + 5);
      jp_pair(p + 5);
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
__device__ __forceinline__ bool sweep_stream_short(LoadV u_at, const SweepConsts<V> &c, Emit emit) {
  Window<K + 5, V> w;
  V S[K + 6];                                // S_m = sqrt(1 + D2_m^2)
  V qX[K + 6], qY[K + 6], qZ[K + 6];
  bool ok = true;

  auto sq = [&](V u) { return s_eval_v(u); };   // FValV::s of f_eval_v
  auto qv = [&](V sa, V sb) {                // q of q_interval_v on its trapezoid branch
    const V ss = vadd(sa, sb);
    const V e = vfma(ss, ss, c.eps4);
    return vmul(e, e);
  };
  auto pos = [&](int m) {
    w.pos(m, c);
    if (m >= 2) ok &= short_width(w.W[m - 1]);
  };
  auto al_qX = [&](int m) { qX[m] = qv(S[m], sq(r_end(w.D2[m], w.W[m - 1]))); };
  auto al_qY = [&](int m) { qY[m] = qv(S[m], S[m + 1]); };
  auto al_qZ = [&](int m) { qZ[m] = qv(sq(l_end(w.D2[m], w.W[m])), S[m]); };
  // the denominators stay in range on short segments: no check
  auto stencil = [&](int j, auto minus_c, auto plus_c, V &nm, V &rm, V &np, V &rp) {
    constexpr bool MI = decltype(minus_c)::value, PL = decltype(plus_c)::value;
    group_corr_v<false, MI, PL>(qX[j + 2], qY[j + 2], qZ[j + 3], w.Ta[j + 2], w.Tb[j + 3], w.Ta[j + 3],
                                w.Tb[j + 2], nm, rm, np, rp);
  };

#pragma unroll
  for (int m = 0; m <= 5; ++m) w.u[m] = u_at(m);
#pragma unroll
  for (int m = 1; m <= 5; ++m) pos(m);
#pragma unroll
  for (int m = 2; m <= 4; ++m) S[m] = sq(w.D2[m]);
  al_qX(2); al_qY(2); al_qZ(3);
  al_qX(3); al_qY(3); al_qZ(4);
  ok &= short_sizes(w.D2[2], c.eps4);
  if (!__all_sync(0xffffffffu, ok)) return false;

  V nm, rm, dummy0, dummy1;
  stencil(0, std::true_type{}, std::false_type{}, nm, rm, dummy0, dummy1);
#pragma unroll
  for (int p = 0; p < K; ++p) {
    V nm1, rm1, np, rp;
    if (p + 1 < K) stencil(p + 1, std::true_type{}, std::true_type{}, nm1, rm1, np, rp);
    else stencil(p + 1, std::false_type{}, std::true_type{}, nm1, rm1, np, rp);
    w.emit_node(p, c, nm, rm, np, rp, emit);
    nm = nm1;
    rm = rm1;
    if (p + 1 < K) {
      w.u[p + 6] = u_at(p + 6);
      pos(p + 6);
      S[p + 5] = sq(w.D2[p + 5]);
      al_qX(p + 4);
      al_qY(p + 4);
      al_qZ(p + 5);
    }
  }
  return __all_sync(0xffffffffu, ok);
}

}  // namespace alw

#pragma nv_diagnostic pop
