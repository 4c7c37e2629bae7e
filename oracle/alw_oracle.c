/*
 * Plain, slow, FP64 CPU oracle for the arc-length WENO scheme (WENO-L) for
 * Hamilton-Jacobi equations  phi_t + H(D phi) = 0   (paper Sec. 2, Steps 1-5).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links or calls this
 * file; it is used by the tests, by the smoke check and by the timed CPU
 * baseline.  It shares no code, header, table or constant with the CUDA path.
 *
 * Every function follows the paper's steps in the paper's order, in double
 * precision, with plain loops (compiled with -ffp-contract=off, no FMA).
 * Readings of passages the paper leaves silent, ambiguous or garbled:
 *   R1  Step 1 / Step 3 coefficient signs: the linear combination is the
 *       d-weighted sum of the Step-2 candidates (printed signs inconsistent).
 *   R2  The "+" side is the mirror image of the "-" side about x_i
 *       (Step 2, last sentence): phi_x^+(phi)_i = -phi_x^-(psi)_{-i},
 *       psi_j = phi_{-j}; so its smoothness interval is [x_i, x_{i+1}].
 *   R3  p_i^k in the arc-length indicator (Eq. newbeta) is the quadratic
 *       candidate p_{k,1}^- of Step 2; b_i^k, c_i^k are the printed closed
 *       forms evaluated in a coordinate centred on x_i (arc length is
 *       translation invariant), which avoids cancellation for |x_i| >> dx.
 *   R4  The primitive I[b,c,z] difference is evaluated as printed
 *       ((F(u1)-F(u0))/(4c), F(u) = u sqrt(1+u^2) + asinh u) unless
 *       |u1-u0| <= 1e-3 sqrt(1+m^2) (m the midpoint), where the identical
 *       mean-value integral is summed as its Taylor series (the printed form
 *       is 0/0 there); c == 0 uses the printed c = 0 branch.
 *   R5  alpha of the Lax-Friedrichs flux ("max over u of |H_1(u)|", range
 *       unstated): by default the node's own maximum of |dH/dp| (|dH/dq|)
 *       over the four combinations (u^-/u^+, v^-/v^+) -- the local form
 *       (for the non-convex H of Example 8, whose H_p is not monotone, the
 *       maximum over the whole interval between u^- and u^+; for Example
 *       11, |sin y| and the maximum of |sin x + sign q| over the interval
 *       between v^- and v^+, both signs when it contains 0),
 *       which reproduces Table 2; the grid-wide maximum of the same values
 *       (global form) and fixed constants are the other modes.  The time
 *       step always uses a grid-wide maximum: of the previous stage
 *       (LAGGED; a prime pass over phi^0 supplies the first) or of phi^n
 *       (EXACT).
 *   R6  dt = cfl / (alpha_x/dx + alpha_y/dy), or with dx^{5/3}, dy^{5/3} in
 *       place of dx, dy (convergence studies); the last step is clipped to
 *       reach t_final exactly.
 *   R7  Periodic grids have N nodes on [a, b), x_i = a + i dx, dx = (b-a)/N.
 *       Linear-extrapolation grids have N nodes on [a, b] including both
 *       ends; ghost values phi_{-m} = (1+m) phi_0 - m phi_1 (mirror image at
 *       the right end).
 *   R8  Jiang-Peng indicators (cited, not printed): with a=v2-v1, b=v3-v2,
 *       c=v4-v3, d=v5-v4:  IS0 = 13(a-b)^2 + 3(a-3b)^2,
 *       IS1 = 13(b-c)^2 + 3(b+c)^2,  IS2 = 13(c-d)^2 + 3(3c-d)^2.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { ORC_BC_PERIODIC = 0, ORC_BC_LINEXTRAP = 1 };
enum { ORC_W_ARCLEN = 0, ORC_W_JP = 1 };
enum {
  ORC_H_BURGERS2D = 0, /* (p+q+1)^2/2       Example 3 */
  ORC_H_NEGCOS2D = 1,  /* -cos(p+q+1)       Example 4 */
  ORC_H_SIN2D = 2,     /* sin(p+q)          Example 10 */
  ORC_H_ADVECT1D = 3,  /* p                 Example 1 */
  ORC_H_BURGERS1D = 4, /* (p+1)^2/2         Example 6 */
  ORC_H_NEGCOS1D = 5,  /* -cos(p+1)         Example 2 */
  ORC_H_EIKONAL2D = 6, /* sqrt(p^2+q^2+1)   Example 12 */
  ORC_H_NONCONVEX1D = 7, /* (p^2-1)(p^2-4)/4 Example 8 */
  ORC_H_OPTCTRL2D = 8    /* sin(y)p + (sin(x)+sign q)q - sin^2(y)/2 - (1-cos x)   Example 11 */
};
enum {
  ORC_ALPHA_LOCAL_LAGGED = 0,  /* flux: per-node alpha; dt: previous stage's grid max */
  ORC_ALPHA_LOCAL_EXACT = 1,   /* flux: per-node alpha; dt: grid max over phi^n */
  ORC_ALPHA_GLOBAL_LAGGED = 2, /* flux and dt: previous stage's grid max */
  ORC_ALPHA_GLOBAL_EXACT = 3,  /* flux: the stage's own grid max; dt: grid max over phi^n */
  ORC_ALPHA_FIXED = 4          /* flux and dt: given constants */
};
enum { ORC_DT_CFL = 0, ORC_DT_DX53 = 1 };
enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_ENONFINITE = 4, ORC_ENOMEM = 2 };

typedef struct {
  int32_t dim;        /* 1 or 2 */
  int32_t nx, ny;     /* nodes per direction (ny = 1 in 1D) */
  int32_t bc;         /* ORC_BC_* */
  double dx, dy;      /* mesh widths */
  int32_t ham;        /* ORC_H_* */
  int32_t weights;    /* ORC_W_* */
  double eps;         /* epsilon of Eq. WLOC1 */
  double cfl;         /* CFL number */
  int32_t dt_mode;    /* ORC_DT_* */
  int32_t alpha_mode; /* ORC_ALPHA_* */
  double alpha_fixed[2];
  double xlo, ylo;    /* coordinates of node (0, 0): x_i = xlo + i dx, y_j = ylo + j dy */
} orc_cfg;

/* ------------------------------------------------------------------------ */
/* Step 2: the three third-order candidates phi_x^{-,k} from v_1..v_5 =     */
/* Delta^+ phi_{i-3..i+1}.                                                 */
static void candidates_minus(const double v[5], double cand[3]) {
  cand[0] = v[0] / 3.0 - 7.0 * v[1] / 6.0 + 11.0 * v[2] / 6.0;
  cand[1] = -v[1] / 6.0 + 5.0 * v[2] / 6.0 + v[3] / 3.0;
  cand[2] = v[2] / 3.0 + 5.0 * v[3] / 6.0 - v[4] / 6.0;
}

/* sqrt(1+u^2) and its antiderivative times two: F(u) = u sqrt(1+u^2) + asinh u */
static double arc_F(double u) { return u * sqrt(1.0 + u * u) + asinh(u); }

/* Arc length of a polynomial P with P'(z) = b + 2 c z over [z0, z1]
 * (Eq. length with the primitive I[b,c,z]; reading R4). */
double orc_arclength(double b, double c, double z0, double z1) {
  if (c == 0.0) return sqrt(1.0 + b * b) * (z1 - z0); /* printed c = 0 branch */
  const double u0 = b + 2.0 * c * z0, u1 = b + 2.0 * c * z1;
  const double h = u1 - u0, m = 0.5 * (u0 + u1);
  const double s2 = 1.0 + m * m, s = sqrt(s2);
  if (fabs(h) <= 1e-3 * s) {
    /* mean of f(u) = sqrt(1+u^2) over [u0,u1]:
       f(m) + f''(m) h^2/24 + f''''(m) h^4/1920 + f^(6)(m) h^6/322560     */
    const double f0 = s;
    const double f2 = 1.0 / (s2 * s);                                      /* (1+m^2)^{-3/2}  */
    const double f4 = (12.0 * m * m - 3.0) / (s2 * s2 * s2 * s);           /* (1+m^2)^{-7/2}  */
    const double f6 = (45.0 - 540.0 * m * m + 360.0 * m * m * m * m) /
                      (s2 * s2 * s2 * s2 * s2 * s);                        /* (1+m^2)^{-11/2} */
    const double h2 = h * h;
    const double mean = f0 + f2 * h2 / 24.0 + f4 * h2 * h2 / 1920.0 + f6 * h2 * h2 * h2 / 322560.0;
    return mean * (z1 - z0);
  }
  /* I[b,c,z1] - I[b,c,z0] as printed */
  return (arc_F(u1) - arc_F(u0)) / (4.0 * c);
}

/* Step 4, Eq. newbeta: beta_k = (L_{[x_{i-1},x_i]}(p_i^k))^2 from the printed
 * b_i^k, c_i^k in a coordinate with x_i = 0 (reading R3).  p[0..5] = phi_{i-3..i+2}. */
static void beta_arclength(const double p[6], double dx, double beta[3]) {
  const double dx3 = dx * dx * dx;
  double b[3], c[3];
  c[0] = (-3.0 * p[0] + 9.0 * p[1] - 9.0 * p[2] + 3.0 * p[3]) / (6.0 * dx3);
  b[0] = (-6.0 * dx * p[0] + 24.0 * dx * p[1] - 30.0 * dx * p[2] + 12.0 * dx * p[3]) / (6.0 * dx3);
  c[1] = (-3.0 * p[1] + 9.0 * p[2] - 9.0 * p[3] + 3.0 * p[4]) / (6.0 * dx3);
  b[1] = (6.0 * dx * p[2] - 12.0 * dx * p[3] + 6.0 * dx * p[4]) / (6.0 * dx3);
  c[2] = (-3.0 * p[2] + 9.0 * p[3] - 9.0 * p[4] + 3.0 * p[5]) / (6.0 * dx3);
  b[2] = (6.0 * dx * p[2] - 12.0 * dx * p[3] + 6.0 * dx * p[4]) / (6.0 * dx3);
  for (int k = 0; k < 3; ++k) {
    const double len = orc_arclength(b[k], c[k], -dx, 0.0); /* [x_{i-1}, x_i] */
    beta[k] = len * len;
  }
}

/* Jiang-Peng indicators on v_1..v_5 (reading R8). */
static void beta_jp(const double v[5], double beta[3]) {
  const double a = v[1] - v[0], b = v[2] - v[1], c = v[3] - v[2], d = v[4] - v[3];
  beta[0] = 13.0 * (a - b) * (a - b) + 3.0 * (a - 3.0 * b) * (a - 3.0 * b);
  beta[1] = 13.0 * (b - c) * (b - c) + 3.0 * (b + c) * (b + c);
  beta[2] = 13.0 * (c - d) * (c - d) + 3.0 * (3.0 * c - d) * (3.0 * c - d);
}

/* Steps 2-4 at one point: phi_x^- from p[0..5] = phi_{i-3..i+2}.
 * Optional outputs: candidates, indicators and nonlinear weights. */
double orc_phix_minus(const double p[6], double dx, int weights, double eps,
                      double *cand_out, double *beta_out, double *omega_out) {
  double v[5], cand[3], beta[3], alpha[3], omega[3];
  for (int m = 0; m < 5; ++m) v[m] = (p[m + 1] - p[m]) / dx; /* Delta^+ phi_j */
  candidates_minus(v, cand);                                   /* Step 2 */
  if (weights == ORC_W_JP) beta_jp(v, beta);
  else beta_arclength(p, dx, beta);                            /* Step 4 */
  const double d[3] = {1.0 / 10.0, 6.0 / 10.0, 3.0 / 10.0};   /* Step 3 */
  double sum = 0.0;
  for (int k = 0; k < 3; ++k) {                                /* Eq. WLOC1 */
    alpha[k] = d[k] / ((eps + beta[k]) * (eps + beta[k]));
    sum += alpha[k];
  }
  double phix = 0.0;
  for (int k = 0; k < 3; ++k) {
    omega[k] = alpha[k] / sum;
    phix += omega[k] * cand[k];
  }
  if (cand_out) memcpy(cand_out, cand, sizeof cand);
  if (beta_out) memcpy(beta_out, beta, sizeof beta);
  if (omega_out) memcpy(omega_out, omega, sizeof omega);
  return phix;
}

/* phi_x^+ from q[0..5] = phi_{i-2..i+3}, by the symmetric procedure about x_i
 * (reading R2): mirror the data, apply the "-" procedure, negate. */
double orc_phix_plus(const double q[6], double dx, int weights, double eps,
                     double *cand_out, double *beta_out, double *omega_out) {
  double r[6];
  for (int m = 0; m < 6; ++m) r[m] = q[5 - m]; /* phi_{i+3}, ..., phi_{i-2} */
  double cand[3];
  const double v = -orc_phix_minus(r, dx, weights, eps, cand, beta_out, omega_out);
  if (cand_out)
    for (int k = 0; k < 3; ++k) cand_out[k] = -cand[k];
  return v;
}

/* ------------------------------------------------------------------------ */
/* Hamiltonians H(x,y,p,q) and partial derivatives in p, q (Examples 1-4, 6, */
/* 8, 10-12).  Only Example 11 depends on the position (x, y).              */
static double sign_of(double q) { return q > 0.0 ? 1.0 : (q < 0.0 ? -1.0 : 0.0); }

int orc_ham(int kind, double x, double y, double p, double q, double *H, double *Hp, double *Hq) {
  double h = 0, hp = 0, hq = 0;
  switch (kind) {
    case ORC_H_BURGERS2D: h = 0.5 * (p + q + 1.0) * (p + q + 1.0); hp = hq = p + q + 1.0; break;
    case ORC_H_NEGCOS2D: h = -cos(p + q + 1.0); hp = hq = sin(p + q + 1.0); break;
    case ORC_H_SIN2D: h = sin(p + q); hp = hq = cos(p + q); break;
    case ORC_H_ADVECT1D: h = p; hp = 1.0; hq = 0.0; break;
    case ORC_H_BURGERS1D: h = 0.5 * (p + 1.0) * (p + 1.0); hp = p + 1.0; hq = 0.0; break;
    case ORC_H_NEGCOS1D: h = -cos(p + 1.0); hp = sin(p + 1.0); hq = 0.0; break;
    case ORC_H_EIKONAL2D: {
      const double r = sqrt(p * p + q * q + 1.0);
      h = r; hp = p / r; hq = q / r;
    } break;
    case ORC_H_NONCONVEX1D:
      h = 0.25 * (p * p - 1.0) * (p * p - 4.0); hp = p * p * p - 2.5 * p; hq = 0.0; break;
    case ORC_H_OPTCTRL2D:
      /* the printed form; (sign q) q = |q| is not differentiable at q = 0, where H_q is
         returned with sign(0) = 0 (orc_node_alpha handles the generalised derivative) */
      h = sin(y) * p + (sin(x) + sign_of(q)) * q - 0.5 * sin(y) * sin(y) - (1.0 - cos(x));
      hp = sin(y); hq = sin(x) + sign_of(q); break;
    default: return ORC_EINVAL;
  }
  if (H) *H = h;
  if (Hp) *Hp = hp;
  if (Hq) *Hq = hq;
  return ORC_OK;
}

/* Lax-Friedrichs numerical Hamiltonian, applied per direction in 2D. */
double orc_hhat(int kind, double x, double y, double up, double um, double vp, double vm, double ax, double ay) {
  double H = 0.0;
  orc_ham(kind, x, y, 0.5 * (up + um), 0.5 * (vp + vm), &H, NULL, NULL);
  return H - ax * 0.5 * (up - um) - ay * 0.5 * (vp - vm);
}

/* ------------------------------------------------------------------------ */
/* Grid values with boundary conditions (reading R7), i in [-3, n+2].       */
static double bc_value(const double *line, ptrdiff_t stride, int n, int bc, int i) {
  if (i >= 0 && i < n) return line[(ptrdiff_t)i * stride];
  if (bc == ORC_BC_PERIODIC) {
    int k = i % n;
    if (k < 0) k += n;
    return line[(ptrdiff_t)k * stride];
  }
  if (i < 0) {
    const int m = -i;
    return (1.0 + m) * line[0] - m * line[stride];
  }
  const int m = i - (n - 1);
  return (1.0 + m) * line[(ptrdiff_t)(n - 1) * stride] - m * line[(ptrdiff_t)(n - 2) * stride];
}

/* phi_x^-, phi_x^+ at node i of a line of n values with the given stride. */
static void line_derivs(const double *line, ptrdiff_t stride, int n, int bc, int i, double h,
                        int weights, double eps, double *dm, double *dp) {
  double p[6], q[6];
  for (int m = 0; m < 6; ++m) p[m] = bc_value(line, stride, n, bc, i - 3 + m);
  for (int m = 0; m < 6; ++m) q[m] = bc_value(line, stride, n, bc, i - 2 + m);
  *dm = orc_phix_minus(p, h, weights, eps, NULL, NULL, NULL);
  *dp = orc_phix_plus(q, h, weights, eps, NULL, NULL, NULL);
}

/* One-sided derivatives at one node (i, j); out = {u^-, u^+, v^-, v^+}. */
void orc_point_derivs(const orc_cfg *cfg, const double *phi, int i, int j, double out[4]) {
  const int nx = cfg->nx, ny = cfg->ny;
  line_derivs(phi + (ptrdiff_t)j * nx, 1, nx, cfg->bc, i, cfg->dx, cfg->weights, cfg->eps, &out[0], &out[1]);
  if (cfg->dim == 2)
    line_derivs(phi + i, nx, ny, cfg->bc, j, cfg->dy, cfg->weights, cfg->eps, &out[2], &out[3]);
  else
    out[2] = out[3] = 0.0;
}

/* Derivatives at every node; arrays of nx*ny values, row-major. */
void orc_derivs(const orc_cfg *cfg, const double *phi, double *um, double *up, double *vm, double *vp) {
  for (int j = 0; j < cfg->ny; ++j)
    for (int i = 0; i < cfg->nx; ++i) {
      double d[4];
      orc_point_derivs(cfg, phi, i, j, d);
      const ptrdiff_t k = (ptrdiff_t)j * cfg->nx + i;
      um[k] = d[0]; up[k] = d[1]; vm[k] = d[2]; vp[k] = d[3];
    }
}

/* Coordinates of the node with row-major index k (reading R7). */
static double node_x(const orc_cfg *cfg, ptrdiff_t k) { return cfg->xlo + (double)(k % cfg->nx) * cfg->dx; }
static double node_y(const orc_cfg *cfg, ptrdiff_t k) {
  return cfg->dim == 2 ? cfg->ylo + (double)(k / cfg->nx) * cfg->dy : 0.0;
}

/* Reading R5, local form: the node's own alpha = max over the four (u, v)
 * combinations at that node of |H_p| (resp. |H_q|). */
void orc_node_alpha(int ham, int dim, double x, double y, double um, double up, double vm, double vp,
                    double out[2]) {
  const double us[2] = {um, up}, vs[2] = {vm, vp};
  double ax = 0.0, ay = 0.0;
  if (ham == ORC_H_OPTCTRL2D) {
    /* H_p = sin y does not depend on (p, q).  H_q = sin x + sign q is piecewise constant: over
       [min(v), max(v)] its values are sin x + s for s in the signs the interval holds, where an
       interval containing q = 0 holds both (the generalised derivative of |q| at 0 is [-1, 1]) */
    const double lo = fmin(vm, vp), hi = fmax(vm, vp);
    ax = fabs(sin(y));
    if (lo <= 0.0 && hi >= 0.0) ay = fmax(fabs(sin(x) + 1.0), fabs(sin(x) - 1.0));
    else ay = fabs(sin(x) + sign_of(lo));
    if (isnan(um) || isnan(up) || isnan(vm) || isnan(vp)) ax = ay = NAN;
    out[0] = ax;
    out[1] = ay;
    return;
  }
  if (ham == ORC_H_NONCONVEX1D) {
    /* H_p = p^3 - 5p/2 is not monotone: its largest modulus on [min(u), max(u)] is at an end or
       where H_pp = 3p^2 - 5/2 vanishes, p = +-sqrt(5/6) */
    const double lo = fmin(um, up), hi = fmax(um, up), c = sqrt(5.0 / 6.0);
    const double cand[4] = {lo, hi, -c, c};
    for (int k = 0; k < 4; ++k) {
      if (k >= 2 && !(cand[k] > lo && cand[k] < hi)) continue;
      double hp;
      orc_ham(ham, x, y, cand[k], 0.0, NULL, &hp, NULL);
      if (fabs(hp) > ax || isnan(hp)) ax = fabs(hp);
    }
    if (isnan(um) || isnan(up)) ax = NAN;
    out[0] = ax;
    out[1] = 0.0;
    return;
  }
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      double hp, hq;
      orc_ham(ham, x, y, us[a], vs[b], NULL, &hp, &hq);
      if (fabs(hp) > ax || isnan(hp)) ax = fabs(hp);
      if (fabs(hq) > ay || isnan(hq)) ay = fabs(hq);
    }
  out[0] = ax;
  out[1] = (dim == 2) ? ay : 0.0;
}

/* Reading R5: alpha_x = max |H_p|, alpha_y = max |H_q| over nodes and the four
 * (u, v) combinations.  Returns ORC_ENONFINITE if a value is not finite. */
int orc_alpha_max(const orc_cfg *cfg, const double *um, const double *up, const double *vm,
                  const double *vp, double out[2]) {
  double ax = 0.0, ay = 0.0;
  int bad = 0;
  const ptrdiff_t n = (ptrdiff_t)cfg->nx * cfg->ny;
  for (ptrdiff_t k = 0; k < n; ++k) {
    double a[2];
    orc_node_alpha(cfg->ham, cfg->dim, node_x(cfg, k), node_y(cfg, k), um[k], up[k], vm[k], vp[k], a);
    if (!isfinite(a[0]) || !isfinite(a[1])) bad = 1;
    if (a[0] > ax) ax = a[0];
    if (a[1] > ay) ay = a[1];
  }
  out[0] = ax;
  out[1] = (cfg->dim == 2) ? ay : 0.0;
  return bad ? ORC_ENONFINITE : ORC_OK;
}

/* Eq. SDE: L(phi) = -Hhat at every node.  alpha_mode selects the alpha of the
 * Lax-Friedrichs flux: per node (LOCAL_*), or the given grid-wide pair. */
void orc_L_from_derivs(const orc_cfg *cfg, const double *um, const double *up, const double *vm,
                       const double *vp, const double alpha[2], double *L) {
  const ptrdiff_t n = (ptrdiff_t)cfg->nx * cfg->ny;
  const int local = (cfg->alpha_mode == ORC_ALPHA_LOCAL_LAGGED || cfg->alpha_mode == ORC_ALPHA_LOCAL_EXACT);
  for (ptrdiff_t k = 0; k < n; ++k) {
    double a[2] = {alpha[0], alpha[1]};
    const double x = node_x(cfg, k), y = node_y(cfg, k);
    if (local) orc_node_alpha(cfg->ham, cfg->dim, x, y, um[k], up[k], vm[k], vp[k], a);
    L[k] = -orc_hhat(cfg->ham, x, y, up[k], um[k], vp[k], vm[k], a[0], cfg->dim == 2 ? a[1] : 0.0);
  }
}

/* Reading R6. */
static double cfl_dt(const orc_cfg *cfg, const double alpha[2]) {
  double lx = cfg->dx, ly = cfg->dy;
  if (cfg->dt_mode == ORC_DT_DX53) {
    lx = pow(cfg->dx, 5.0 / 3.0);
    ly = pow(cfg->dy, 5.0 / 3.0);
  }
  double den = alpha[0] / lx;
  if (cfg->dim == 2) den += alpha[1] / ly;
  return den > 0.0 ? cfg->cfl / den : INFINITY;
}

typedef struct {
  double *um, *up, *vm, *vp, *L, *phi1, *phi2;
} orc_work;

static void work_free(orc_work *w) {
  free(w->um); free(w->up); free(w->vm); free(w->vp); free(w->L); free(w->phi1); free(w->phi2);
}

static int work_alloc(orc_work *w, size_t n) {
  memset(w, 0, sizeof *w);
  w->um = malloc(n * sizeof(double)); w->up = malloc(n * sizeof(double));
  w->vm = malloc(n * sizeof(double)); w->vp = malloc(n * sizeof(double));
  w->L = malloc(n * sizeof(double)); w->phi1 = malloc(n * sizeof(double));
  w->phi2 = malloc(n * sizeof(double));
  if (!w->um || !w->up || !w->vm || !w->vp || !w->L || !w->phi1 || !w->phi2) {
    work_free(w);
    return ORC_ENOMEM;
  }
  return ORC_OK;
}

/* Prime pass: grid-wide alpha of phi's own derivatives. */
int orc_alpha_of(const orc_cfg *cfg, const double *phi, double out[2]) {
  orc_work w;
  const size_t n = (size_t)cfg->nx * cfg->ny;
  if (work_alloc(&w, n)) return ORC_ENOMEM;
  orc_derivs(cfg, phi, w.um, w.up, w.vm, w.vp);
  const int st = orc_alpha_max(cfg, w.um, w.up, w.vm, w.vp, out);
  work_free(&w);
  return st;
}

/* One RK stage's spatial operator on src: derivatives, the flux alpha of the
 * mode, L.  alpha_state (in/out) is the most recent grid-wide reduction; every
 * stage replaces it by the reduction over its own derivatives. */
static int stage_operator(const orc_cfg *cfg, const double *src, double alpha_state[2], orc_work *w) {
  orc_derivs(cfg, src, w->um, w->up, w->vm, w->vp);
  double a_new[2];
  const int st = orc_alpha_max(cfg, w->um, w->up, w->vm, w->vp, a_new);
  double a_use[2] = {alpha_state[0], alpha_state[1]};          /* GLOBAL_LAGGED */
  if (cfg->alpha_mode == ORC_ALPHA_FIXED) {
    a_use[0] = cfg->alpha_fixed[0]; a_use[1] = cfg->alpha_fixed[1];
  } else if (cfg->alpha_mode == ORC_ALPHA_GLOBAL_EXACT) {
    a_use[0] = a_new[0]; a_use[1] = a_new[1];
  }
  orc_L_from_derivs(cfg, w->um, w->up, w->vm, w->vp, a_use, w->L); /* LOCAL_*: per node */
  alpha_state[0] = a_new[0];
  alpha_state[1] = a_new[1];
  return st;
}

/* Step 5: TVD-RK3 time loop from t0 to t_final (in place on phi).
 * alpha_state: the most recent grid-wide alpha reduction, carried between
 * calls.  If alpha_state[0] < 0 on entry, a prime pass sets it from phi.
 * dt of a step uses: FIXED the fixed pair; *_EXACT the reduction over phi^n;
 * *_LAGGED alpha_state (the reduction of the previous stage).
 * Returns ORC_OK, ORC_EINVAL, ORC_ENOMEM or ORC_ENONFINITE. */
int orc_solve(const orc_cfg *cfg, double *phi, double t0, double t_final, int64_t max_steps,
              double alpha_state[2], int64_t *steps_out, double *t_out) {
  if (!cfg || !phi || cfg->nx < 1 || cfg->ny < 1 || (cfg->dim != 1 && cfg->dim != 2)) return ORC_EINVAL;
  if (cfg->dim == 1 && cfg->ny != 1) return ORC_EINVAL;
  if (cfg->bc == ORC_BC_LINEXTRAP && (cfg->nx < 2 || (cfg->dim == 2 && cfg->ny < 2))) return ORC_EINVAL;
  const size_t n = (size_t)cfg->nx * cfg->ny;
  orc_work w;
  if (work_alloc(&w, n)) return ORC_ENOMEM;
  int st = ORC_OK;
  if (alpha_state[0] < 0.0) {
    orc_derivs(cfg, phi, w.um, w.up, w.vm, w.vp);
    st = orc_alpha_max(cfg, w.um, w.up, w.vm, w.vp, alpha_state);
  }
  double t = t0;
  int64_t steps = 0;
  while (st == ORC_OK && t < t_final && steps < max_steps) {
    double a_dt[2] = {alpha_state[0], alpha_state[1]};
    if (cfg->alpha_mode == ORC_ALPHA_FIXED) {
      a_dt[0] = cfg->alpha_fixed[0]; a_dt[1] = cfg->alpha_fixed[1];
    } else if (cfg->alpha_mode == ORC_ALPHA_GLOBAL_EXACT || cfg->alpha_mode == ORC_ALPHA_LOCAL_EXACT) {
      orc_derivs(cfg, phi, w.um, w.up, w.vm, w.vp);
      st = orc_alpha_max(cfg, w.um, w.up, w.vm, w.vp, a_dt);
      alpha_state[0] = a_dt[0]; alpha_state[1] = a_dt[1];
    }
    double dt = cfl_dt(cfg, a_dt);
    int last = 0;
    if (t + dt >= t_final) { dt = t_final - t; last = 1; }
    /* phi_1 = phi_0 + dt L(phi_0) */
    st |= stage_operator(cfg, phi, alpha_state, &w);
    for (size_t k = 0; k < n; ++k) w.phi1[k] = phi[k] + dt * w.L[k];
    /* phi_2 = 3/4 phi_0 + 1/4 (phi_1 + dt L(phi_1)) */
    st |= stage_operator(cfg, w.phi1, alpha_state, &w);
    for (size_t k = 0; k < n; ++k) w.phi2[k] = 0.75 * phi[k] + 0.25 * (w.phi1[k] + dt * w.L[k]);
    /* phi^{n+1} = 1/3 phi_0 + 2/3 (phi_2 + dt L(phi_2)) */
    st |= stage_operator(cfg, w.phi2, alpha_state, &w);
    for (size_t k = 0; k < n; ++k) phi[k] = phi[k] / 3.0 + 2.0 * (w.phi2[k] + dt * w.L[k]) / 3.0;
    t = last ? t_final : t + dt;
    ++steps;
  }
  work_free(&w);
  if (steps_out) *steps_out = steps;
  if (t_out) *t_out = t;
  return st ? ORC_ENONFINITE : ORC_OK;
}

/* Step 5 alone, for a user-supplied operator L (used to pin the RK3
 * combination against its amplification polynomial). */
typedef void (*orc_L_fn)(int64_t n, const double *y, double *out, void *ctx);

int orc_rk3_step_generic(int64_t n, double *y, double dt, orc_L_fn Lf, void *ctx) {
  double *L = malloc((size_t)n * sizeof(double));
  double *y1 = malloc((size_t)n * sizeof(double));
  double *y2 = malloc((size_t)n * sizeof(double));
  if (!L || !y1 || !y2) { free(L); free(y1); free(y2); return ORC_ENOMEM; }
  Lf(n, y, L, ctx);
  for (int64_t k = 0; k < n; ++k) y1[k] = y[k] + dt * L[k];
  Lf(n, y1, L, ctx);
  for (int64_t k = 0; k < n; ++k) y2[k] = 0.75 * y[k] + 0.25 * (y1[k] + dt * L[k]);
  Lf(n, y2, L, ctx);
  for (int64_t k = 0; k < n; ++k) y[k] = y[k] / 3.0 + 2.0 * (y2[k] + dt * L[k]) / 3.0;
  free(L); free(y1); free(y2);
  return ORC_OK;
}

/* One stage of Step 5 at a single node, for sampled comparisons on grids
 * too large for the whole-grid oracle: returns L at (i, j) of phi. */
double orc_point_L(const orc_cfg *cfg, const double *phi, int i, int j, const double alpha[2]) {
  double d[4], a[2] = {alpha[0], alpha[1]};
  orc_point_derivs(cfg, phi, i, j, d);
  if (cfg->alpha_mode == ORC_ALPHA_LOCAL_LAGGED || cfg->alpha_mode == ORC_ALPHA_LOCAL_EXACT)
    orc_node_alpha(cfg->ham, cfg->dim, cfg->xlo + i * cfg->dx, cfg->ylo + j * cfg->dy, d[0], d[1], d[2], d[3], a);
  return -orc_hhat(cfg->ham, cfg->xlo + i * cfg->dx, cfg->ylo + j * cfg->dy, d[1], d[0], d[3], d[2], a[0],
                   cfg->dim == 2 ? a[1] : 0.0);
}
