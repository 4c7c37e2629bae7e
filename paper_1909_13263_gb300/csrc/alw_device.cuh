// Device code of the WENO-L stage kernel (sm_103a).
//
// One launch = one TVD-RK3 stage (Step 5) over a 2D (or 1D) grid tile by tile.
// Per tile: load phi and a 3-node halo into shared memory, sweep rows for
// phi_x^-/+ and columns for phi_y^-/+ (Steps 1-4, dimension by dimension as in
// the Sec. 2 Note), form the Lax-Friedrichs numerical Hamiltonian, combine the
// RK stage, write the interior and the periodic ghost copies it owns, and fold
// max |dH/dp|, max |dH/dq| into a device scalar.
//
// The reconstruction uses the algebraically identical compact form
//   phi_x^-_i = c_i - (1/3) w0 T_{i-1} - (1/6)(w2 - 1/2) T_i,
//   phi_x^+_i = c_i + (1/3) w0' T_{i+1} + (1/6)(w2' - 1/2) T_i,
// with c_i = (-v_{i-2} + 7 v_{i-1} + 7 v_i - v_{i+1})/12 (v = Delta^+ phi),
// s_j = v_j - v_{j-1}, T_j = s_{j-1} - 2 s_j + s_{j+1}; it equals
// sum_k omega_k phi_x^{-,k} of Steps 2-4 for any weights (omega_1 = 1 - omega_0
// - omega_2), and the "+" side is the mirror image about x_i.
//
// Arc-length indicators (Step 4, Eq. newbeta): the derivative of each
// candidate p_i^k is linear on its cell, with end values that are second
// differences D2_j = s_j / dx: "-" side k = 0: (D2_{i-1}, R_{i-1}), k = 1:
// (D2_{i-1}, D2_i), k = 2: (L_i, D2_i); "+" side mirrored, with R_j = 2 D2_j -
// D2_{j-1}, L_j = 2 D2_j - D2_{j+1}.  The arc length over a cell is
// dx * G(a, b), G = mean of sqrt(1+u^2) over [a, b] = (F(b) - F(a)) / (2 (b - a)),
// F(u) = u sqrt(1+u^2) + asinh(u)  (the primitive I[b,c,z] of Sec. 2).  Each F
// and each G is evaluated once per node and shared with the neighbours.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "alw_internal.h"

namespace alw {

enum { BC_PERIODIC = 0, BC_LINEXTRAP = 1 };
enum { H_BURGERS2D = 0, H_NEGCOS2D = 1, H_SIN2D = 2, H_ADVECT1D = 3, H_BURGERS1D = 4, H_NEGCOS1D = 5,
       H_EIKONAL2D = 6, H_NONCONVEX1D = 7, H_OPTCTRL2D = 8 };
enum { W_ARCLEN = 0, W_JP = 1 };
enum { A_LOCAL_LAGGED = 0, A_LOCAL_EXACT = 1, A_GLOBAL_LAGGED = 2, A_GLOBAL_EXACT = 3, A_FIXED = 4 };

// --------------------------------------------------------------------------
// Arithmetic per compute type.

template <typename T> struct Arith;

template <> struct Arith<double> {
  // F(u) = u s + asinh(u) and s = sqrt(1+u^2), with asinh|u| = log(|u| + s) reusing s.  F only
  // enters divided differences (F(b) - F(a)) / (b - a) over intervals longer than 1e-3 s, so
  // its absolute error is what counts: log of the rounded |u| + s >= 1 errs by about one unit
  // of 1, like a correctly rounded F of size one.
  __device__ __forceinline__ static void F(double u, double &Fu, double &s) {
    s = sqrt(fma(u, u, 1.0));
    Fu = fma(u, s, copysign(log(fabs(u) + s), u));
  }
  // mean of sqrt(1+u^2) over [a, b]; near a == b the divided difference is 0/0, so its Taylor
  // series about the midpoint is summed instead (below 1e-3 of the mean of the end values
  // sa, sb, which bounds sqrt(1 + m^2) from above; both forms are accurate near the switch).
  __device__ __forceinline__ static double G(double a, double Fa, double sa, double b, double Fb, double sb) {
    const double h = b - a;
    if (fabs(h) > 5e-4 * (sa + sb)) return (Fb - Fa) / (2.0 * h);
    const double m = 0.5 * (a + b);
    const double s2 = fma(m, m, 1.0), s = sqrt(s2);
    const double r = 1.0 / s2, m2 = m * m, h2 = h * h;
    // f'' = s2^{-3/2}, f'''' = (12 m^2 - 3) s2^{-7/2}, f^(6) = (45 - 540 m^2 + 360 m^4) s2^{-11/2}
    const double f2 = r / s;
    const double f4 = (12.0 * m2 - 3.0) * r * r * r / s;
    const double f6 = (45.0 - 540.0 * m2 + 360.0 * m2 * m2) * r * r * r * r * r / s;
    return s + h2 * (f2 / 24.0 + h2 * (f4 / 1920.0 + h2 * f6 / 322560.0));
  }
  // nonlinear weights (Eq. WLOC1): returns omega_0, omega_2 from q_k = (eps + beta_k)^2 in the
  // product form omega_k = d_k prod_{l != k} q_l / sum_m d_m prod_{l != m} q_l (one division;
  // the quotients d_k / q_k of Eq. WLOC1 when the products leave the double range)
  __device__ __forceinline__ static void weights(double q0, double q1, double q2, double &w0, double &w2) {
    const double n0 = 0.1 * (q1 * q2), n2 = 0.3 * (q0 * q1);
    const double den = fma(0.6, q0 * q2, n0 + n2);
    if (den > 1e-290 && den < 1e290) {
      const double r = 1.0 / den;
      w0 = n0 * r;
      w2 = n2 * r;
    } else {
      const double a0 = 0.1 / q0, a1 = 0.6 / q1, a2 = 0.3 / q2;
      const double sum = a0 + a1 + a2;
      w0 = a0 / sum;
      w2 = a2 / sum;
    }
  }
  __device__ __forceinline__ static double cosv(double x) { return cos(x); }
  __device__ __forceinline__ static double sinv(double x) { return sin(x); }
  __device__ __forceinline__ static double sqrtv(double x) { return sqrt(x); }
  __device__ __forceinline__ static double rcp(double x) { return 1.0 / x; }
};

template <> struct Arith<float> {
  __device__ __forceinline__ static void F(float u, float &Fu, float &s) {
    const float t = fmaf(u, u, 1.0f);
    s = t * rsqrtf(t);
    // asinh|u| = ln(|u| + sqrt(1+u^2)); absolute error of the base-2 log ~ 2^-22
    const float l = __log2f(fabsf(u) + s) * 0.693147180559945f;
    Fu = fmaf(u, s, copysignf(l, u));
  }
  // divided difference, or the trapezoid mean (relative error <= h^2/12) when the
  // interval is short compared with its end values
  __device__ __forceinline__ static float G(float a, float Fa, float sa, float b, float Fb, float sb) {
    const float h = b - a;
    const float dd = __fdividef(0.5f * (Fb - Fa), h);
    const float tr = 0.5f * (sa + sb);
    return (fabsf(h) > 0.015625f * (1.0f + fabsf(a) + fabsf(b))) ? dd : tr;
  }
  // product form: omega_k = d_k prod_{l != k} q_l / sum_m d_m prod_{l != m} q_l (one reciprocal);
  // falls back to per-weight reciprocals when the products leave the safe range
  __device__ __forceinline__ static void weights(float q0, float q1, float q2, float &w0, float &w2) {
    const float p12 = q1 * q2, p02 = q0 * q2, p01 = q0 * q1;
    const float n0 = 0.1f * p12, n2 = 0.3f * p01;
    const float den = fmaf(0.6f, p02, n0 + n2);
    if (den > 1e-36f && den < 1e36f) {
      const float r = __frcp_rn(den);
      w0 = n0 * r;
      w2 = n2 * r;
    } else {
      const float a0 = __fdividef(0.1f, q0), a1 = __fdividef(0.6f, q1), a2 = __fdividef(0.3f, q2);
      const float r = __frcp_rn(a0 + a1 + a2);
      w0 = a0 * r;
      w2 = a2 * r;
    }
  }
  __device__ __forceinline__ static float cosv(float x) { return __cosf(x); }
  __device__ __forceinline__ static float sinv(float x) { return __sinf(x); }
  __device__ __forceinline__ static float sqrtv(float x) { return sqrtf(x); }
  __device__ __forceinline__ static float rcp(float x) { return __frcp_rn(x); }
};

// --------------------------------------------------------------------------
// One-direction sweep over K consecutive nodes i0..i0+K-1.
// v[m] = Delta^+ phi_{i0-3+m}, m = 0..K+4.  Outputs phi^-, phi^+ per node.
template <typename T, int K, int WEIGHTS>
__device__ __forceinline__ void weno_sweep(const T (&v)[K + 5], T rdx, T dx, T eps, T (&dm)[K], T (&dp)[K]) {
  using A = Arith<T>;
  T s[K + 5];
#pragma unroll
  for (int m = 1; m <= K + 4; ++m) s[m] = v[m] - v[m - 1];
  T T2[K + 5];
#pragma unroll
  for (int m = 2; m <= K + 3; ++m) T2[m] = (s[m - 1] + s[m + 1]) - T(2) * s[m];

  // q = (eps + beta)^2 per shared interval; index conventions below
  T qX[K + 5], qY[K + 5], qZ[K + 5];
  if (WEIGHTS == W_ARCLEN) {
    T D2[K + 5];
#pragma unroll
    for (int m = 1; m <= K + 4; ++m) D2[m] = s[m] * rdx;
    T FD[K + 5], SD[K + 5];
#pragma unroll
    for (int m = 2; m <= K + 3; ++m) A::F(D2[m], FD[m], SD[m]);
    // qX[m] <- G(D2_m, R_m), m = 2..K+2;  qY[m] <- G(D2_m, D2_{m+1}), m = 2..K+2;
    // qZ[m] <- G(L_m, D2_m), m = 3..K+3
#pragma unroll
    for (int m = 2; m <= K + 2; ++m) {
      const T R = T(2) * D2[m] - D2[m - 1];
      T FR, SR;
      A::F(R, FR, SR);
      const T g = A::G(D2[m], FD[m], SD[m], R, FR, SR);
      const T b = dx * g;
      const T e = eps + b * b;
      qX[m] = e * e;
      const T g2 = A::G(D2[m], FD[m], SD[m], D2[m + 1], FD[m + 1], SD[m + 1]);
      const T b2 = dx * g2;
      const T e2 = eps + b2 * b2;
      qY[m] = e2 * e2;
    }
#pragma unroll
    for (int m = 3; m <= K + 3; ++m) {
      const T Lv = T(2) * D2[m] - D2[m + 1];
      T FL, SL;
      A::F(Lv, FL, SL);
      const T g = A::G(Lv, FL, SL, D2[m], FD[m], SD[m]);
      const T b = dx * g;
      const T e = eps + b * b;
      qZ[m] = e * e;
    }
#pragma unroll
    for (int p = 0; p < K; ++p) {
      T w0, w2, u0, u2;
      A::weights(qX[p + 2], qY[p + 2], qZ[p + 3], w0, w2);   // "-": k = 0, 1, 2
      A::weights(qZ[p + 4], qY[p + 3], qX[p + 3], u0, u2);   // "+": mirrored k = 0, 1, 2
      const T c = ((v[p + 2] + v[p + 3]) * T(7) - v[p + 1] - v[p + 4]) * T(1.0 / 12.0);
      dm[p] = c - w0 * T2[p + 2] * T(1.0 / 3.0) - (w2 - T(0.5)) * T2[p + 3] * T(1.0 / 6.0);
      dp[p] = c + u0 * T2[p + 4] * T(1.0 / 3.0) + (u2 - T(0.5)) * T2[p + 3] * T(1.0 / 6.0);
    }
  } else {
    // Jiang-Peng: for the pair (x, y) = (s_m, s_{m+1}):
    //   qX[m] <- 13(x-y)^2 + 3(x-3y)^2,  qY[m] <- 13(x-y)^2 + 3(x+y)^2,  qZ[m] <- 13(x-y)^2 + 3(3x-y)^2
#pragma unroll
    for (int m = 1; m <= K + 3; ++m) {
      const T x = s[m], y = s[m + 1];
      const T d = x - y, d13 = T(13) * d * d;
      const T a = x - T(3) * y, b = x + y, c = T(3) * x - y;
      const T ea = eps + (d13 + T(3) * a * a), eb = eps + (d13 + T(3) * b * b), ec = eps + (d13 + T(3) * c * c);
      qX[m] = ea * ea;
      qY[m] = eb * eb;
      qZ[m] = ec * ec;
    }
#pragma unroll
    for (int p = 0; p < K; ++p) {
      T w0, w2, u0, u2;
      A::weights(qX[p + 1], qY[p + 2], qZ[p + 3], w0, w2);   // "-"
      A::weights(qZ[p + 4], qY[p + 3], qX[p + 2], u0, u2);   // "+"
      const T c = ((v[p + 2] + v[p + 3]) * T(7) - v[p + 1] - v[p + 4]) * T(1.0 / 12.0);
      dm[p] = c - w0 * T2[p + 2] * T(1.0 / 3.0) - (w2 - T(0.5)) * T2[p + 3] * T(1.0 / 6.0);
      dp[p] = c + u0 * T2[p + 4] * T(1.0 / 3.0) + (u2 - T(0.5)) * T2[p + 3] * T(1.0 / 6.0);
    }
  }
}

// --------------------------------------------------------------------------
// Hamiltonians (runtime kind, uniform across the grid).

// (x, y) is the node's position; only Example 11's H depends on it.
template <typename T>
__device__ __forceinline__ T ham_value(int kind, T p, T q, T x, T y) {
  using A = Arith<T>;
  switch (kind) {
    case H_BURGERS2D: { const T z = p + q + T(1); return T(0.5) * z * z; }
    case H_NEGCOS2D: return -A::cosv(p + q + T(1));
    case H_SIN2D: return A::sinv(p + q);
    case H_ADVECT1D: return p;
    case H_BURGERS1D: { const T z = p + T(1); return T(0.5) * z * z; }
    case H_NEGCOS1D: return -A::cosv(p + T(1));
    case H_EIKONAL2D: return A::sqrtv(p * p + q * q + T(1));
    case H_NONCONVEX1D: return T(0.25) * (p * p - T(1)) * (p * p - T(4));
    case H_OPTCTRL2D: {
      // sin(y) p + (sin(x) + sign q) q - sin^2(y)/2 - (1 - cos x), with (sign q) q = |q|
      const T sy = A::sinv(y);
      return sy * p + A::sinv(x) * q + fabs(q) - T(0.5) * sy * sy - (T(1) - A::cosv(x));
    }
    default: return T(0);
  }
}

// Node alpha: max over the four (u, v) combinations of |H_p| and |H_q|; for the
// non-convex Example 8 Hamiltonian, max of |H_p| over the whole interval [u-, u+].
template <typename T>
__device__ __forceinline__ void node_alpha(int kind, T um, T up, T vm, T vp, T x, T y, T &ax, T &ay) {
  using A = Arith<T>;
  switch (kind) {
    case H_BURGERS2D: {
      const T a = fabs(um + vm + T(1)), b = fabs(um + vp + T(1)), c = fabs(up + vm + T(1)), d = fabs(up + vp + T(1));
      ax = ay = fmax(fmax(a, b), fmax(c, d));
    } break;
    case H_NEGCOS2D: {
      const T a = fabs(A::sinv(um + vm + T(1))), b = fabs(A::sinv(um + vp + T(1)));
      const T c = fabs(A::sinv(up + vm + T(1))), d = fabs(A::sinv(up + vp + T(1)));
      ax = ay = fmax(fmax(a, b), fmax(c, d));
    } break;
    case H_SIN2D: {
      const T a = fabs(A::cosv(um + vm)), b = fabs(A::cosv(um + vp));
      const T c = fabs(A::cosv(up + vm)), d = fabs(A::cosv(up + vp));
      ax = ay = fmax(fmax(a, b), fmax(c, d));
    } break;
    case H_ADVECT1D: ax = T(1); ay = T(0); break;
    case H_BURGERS1D: ax = fmax(fabs(um + T(1)), fabs(up + T(1))); ay = T(0); break;
    case H_NEGCOS1D: ax = fmax(fabs(A::sinv(um + T(1))), fabs(A::sinv(up + T(1)))); ay = T(0); break;
    case H_EIKONAL2D: {
      T mx = T(0), my = T(0);
      const T us[2] = {um, up}, vs[2] = {vm, vp};
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          const T r = A::rcp(A::sqrtv(us[a] * us[a] + vs[b] * vs[b] + T(1)));
          mx = fmax(mx, fabs(us[a]) * r);
          my = fmax(my, fabs(vs[b]) * r);
        }
      ax = mx; ay = my;
    } break;
    case H_NONCONVEX1D: {
      // H_p = p^3 - 5p/2; interior extrema of H_p at p = +-sqrt(5/6), where |H_p| = (5/3) sqrt(5/6)
      const T lo = fmin(um, up), hi = fmax(um, up);
      const T c = T(0.91287092917527690), hc = c * c * c - T(2.5) * c;
      T a = fmax(fabs(um * um * um - T(2.5) * um), fabs(up * up * up - T(2.5) * up));
      if ((lo < c && hi > c) || (lo < -c && hi > -c)) a = fmax(a, fabs(hc));
      ax = a; ay = T(0);
    } break;
    case H_OPTCTRL2D: {
      // H_p = sin y; H_q = sin x + sign q over [min v, max v], both signs when the interval
      // contains the kink of |q| at 0
      const T sx = A::sinv(x), lo = fmin(vm, vp), hi = fmax(vm, vp);
      ax = fabs(A::sinv(y));
      ay = (lo <= T(0) && hi >= T(0)) ? fabs(sx) + T(1) : fabs(sx + (lo > T(0) ? T(1) : T(-1)));
    } break;
    default: ax = ay = T(0);
  }
  // propagate NaN (fmax drops it) so that the caller can flag it
  if (isnan(um) || isnan(up) || isnan(vm) || isnan(vp)) ax = ay = T(NAN);
}

__device__ __forceinline__ double bits_to_double(unsigned long long b) { return __longlong_as_double((long long)b); }
__device__ __forceinline__ unsigned long long double_to_bits(double d) { return (unsigned long long)__double_as_longlong(d); }

// Double-float: (hi, lo) + d with hi, lo, d floats; result renormalised.
__device__ __forceinline__ void df_add(float hi, float lo, float d, float &ohi, float &olo) {
  const float s = hi + d;
  const float bb = s - hi;
  const float e = (hi - (s - bb)) + (d - bb);    // TwoSum error
  const float l2 = lo + e;
  const float h2 = s + l2;
  olo = l2 - (h2 - s);
  ohi = h2;
}

// Store one output value at interior node (gi, gj) and at every periodic ghost
// position that holds a copy of it (a cross-shaped stencil never reads corners).
template <typename S, int DIM>
__device__ __noinline__ void store_ghosts(S *arr, int pitch, int nx, int ny, int gi, int gj, S val) {
  const int gy = (DIM == 2) ? GY : 0;
  S *row = arr + (size_t)(gj + gy) * pitch;
  if (gi < 3 || gi >= nx - 3) {
#pragma unroll
    for (int k = 1; k <= 3; ++k) {
      int g = -k, w = ((g % nx) + nx) % nx;
      if (w == gi) row[g + GX] = val;
      g = nx - 1 + k;
      w = g % nx;
      if (w == gi) row[g + GX] = val;
    }
  }
  if (DIM == 2 && (gj < 3 || gj >= ny - 3)) {
#pragma unroll
    for (int k = 1; k <= 3; ++k) {
      int g = -k, w = ((g % ny) + ny) % ny;
      if (w == gj) arr[(size_t)(g + GY) * pitch + gi + GX] = val;
      g = ny - 1 + k;
      w = g % ny;
      if (w == gj) arr[(size_t)(g + GY) * pitch + gi + GX] = val;
    }
  }
}

template <typename S, int DIM>
__device__ __forceinline__ void store_node(S *arr, int pitch, int nx, int ny, int bc, int gi, int gj, S val) {
  const int gy = (DIM == 2) ? GY : 0;
  S *row = arr + (size_t)(gj + gy) * pitch;
  row[gi + GX] = val;
  if (bc != BC_PERIODIC) return;
  if (nx >= 3 && (DIM == 1 || ny >= 3)) {
    // with at least 3 nodes per direction a node is the periodic image of at most one ghost on
    // each side: left ghost gi - nx for the last three nodes, right ghost gi + nx for the first three
    if (gi >= nx - 3) row[gi - nx + GX] = val;
    if (gi < 3) row[gi + nx + GX] = val;
    if (DIM == 2) {
      if (gj >= ny - 3) arr[(size_t)(gj - ny + GY) * pitch + gi + GX] = val;
      if (gj < 3) arr[(size_t)(gj + ny + GY) * pitch + gi + GX] = val;
    }
  } else if (gi < 3 || gi >= nx - 3 || (DIM == 2 && (gj < 3 || gj >= ny - 3))) {
    store_ghosts<S, DIM>(arr, pitch, nx, ny, gi, gj, val);  // tiny grids: several images per node
  }
}

}  // namespace alw
