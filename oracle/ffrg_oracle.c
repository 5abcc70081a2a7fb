/*
 * ffrg_oracle.c -- plain, slow, FP64 CPU oracle for the momentum-loop
 * right-hand side of functional-RG vertex-expansion flows (DiFfRG,
 * arXiv:2412.13043) and for the explicit RK stepper that integrates it.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library may link, load or
 * call this file; only tests/, the smoke check and the CPU-baseline leg of the
 * benchmark use it.  It shares no code, header, table or constant with the
 * CUDA path: every formula below is written out again from the paper's
 * definitions (Sec. 2.1 Eq. GenfRG / FlowGamman, Sec. 5.2.2 Eq. assVar /
 * flowVar, Sec. 5.3.1 regulator API, Sec. 5.3.2 quadrature integrators,
 * App. F interpolator types, App. C time-stepping parameters) and from the
 * synthetic integrands of this library's models where the paper is silent
 * (propagator, regulator and vertex diagrams of the d=3, d=4 and finite-T
 * models, each written out at its function below).
 *
 * Style: nested loops in the order the definitions are written (external point,
 * then Matsubara index, radial node, angular nodes), Neumaier-compensated sums
 * in that fixed order, libm's exp/expm1/log/sqrt.  No blocking, no hoisting of
 * factors across loops beyond what a definition names, no vectorisation.  An
 * optional OpenMP pragma parallelises over external points only (each point's
 * sum keeps its fixed order, so results do not depend on the thread count).
 *
 * Parity pins: see tests/test_oracle_pins.py.  Every function here is pinned
 * by at least one closed form, library routine, invariant or brute-force case.
 * With non-constant tables away from p = 0 every RHS summand is also pinned
 * against an independent route to the same integral: the d=3, finite-T and
 * d=4 two-point integrands through the substitution s = |q + p| and adaptive
 * quadrature; the d=4 three-point block and the full-vertex blocks through
 * summands written from the model definitions over explicit 4-vectors (the
 * full vertex with its shape variables from the leg vectors).  The feedback
 * maps of flow_deriv (d=3: m^2 and Z_i; d=4: Z_i, the psi average of lambda3,
 * lambda4) are pinned by flat-regulator closed forms, by the p -> 0 limit of
 * their difference quotients (d/d(p^2) of the angle average) and by the same
 * independent routes at finite p; the d=4 state Jacobian by central
 * differences of that pinned map (tests/test_oracle_feedback_pins.py).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2
#define ORC_ENONFINITE 3
#define ORC_ESTEP_UNDERFLOW 4
#define ORC_EMAXSTEPS 5

#define ORC_D3 1
#define ORC_D4_VERTEX 2
#define ORC_FINITE_T 3
#define ORC_D4_FULL 4
#define ORC_FINITE_T_4D 5

#define ORC_REG_EXP 0
#define ORC_REG_LITIM 1

static const double ORC_PI = 3.14159265358979323846264338327950288;

/* Problem description, oracle-side layout (the Python wrapper fills it). */
typedef struct {
  int model, regulator;
  int n_rad, n_ang1, n_ang2;
  int n_ext_p, n_ext_ang, n_matsubara, include_p0;
  int n_tables, n_pts, n_stack;
  int statistics; /* finite T: 0 bosonic loop frequencies, 1 fermionic */
  int n_va, n_vb; /* D4_FULL: nodes of the three-point vertex in its two shape variables */
  int n_x0;       /* FINITE_T_4D: Gauss-Legendre nodes of the frequency quadrature */
  double m2_over_k2, m2_shift, lam, T;
  double p_min, p_max, qmax_over_k, prefactor;
  double x_min, x_max;
} orc_problem;

typedef struct {
  double t0, t1, dt0, dt_min, dt_max, atol, rtol;
  long max_steps;
} orc_step_opts;

typedef struct {
  long steps, rejects, rhs_evals;
} orc_flow_stats;

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* ------------------------------------------------------------------ */
/* Neumaier-compensated running sum (fixed order).                      */
/* ------------------------------------------------------------------ */
typedef struct { double sum, comp; } acc_t;

static void acc_add(acc_t *a, double x) {
  double t = a->sum + x;
  if (fabs(a->sum) >= fabs(x))
    a->comp += (a->sum - t) + x;
  else
    a->comp += (x - t) + a->sum;
  a->sum = t;
}
static double acc_get(const acc_t *a) { return a->sum + a->comp; }

/* ------------------------------------------------------------------ */
/* Quadrature rules ("multi-dimensional quadrature rules of arbitrary   */
/* order", Sec. 5.3.2).                                                 */
/* ------------------------------------------------------------------ */

/* Gauss-Legendre rule on [a,b]: nodes are the roots of P_n found by Newton's
 * method on the three-term Legendre recurrence
 *   j P_j(x) = (2j-1) x P_{j-1}(x) - (j-1) P_{j-2}(x),
 * with P_n'(x) = n (x P_n - P_{n-1}) / (x^2 - 1); weights 2/((1-x^2) P_n'(x)^2).
 * Output in ascending order. */
int orc_gauss_legendre(int n, double a, double b, double *x, double *w) {
  if (n < 1) return ORC_EINVAL;
  int m = (n + 1) / 2;
  for (int i = 0; i < m; ++i) {
    double z = cos(ORC_PI * (i + 0.75) / (n + 0.5));
    double dpn = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z; /* P_0, P_1; after the loop p1 = P_n, p0 = P_{n-1} */
      for (int j = 2; j <= n; ++j) {
        double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
        p0 = p1;
        p1 = p2;
      }
      dpn = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dpn;
      z -= dz;
      if (fabs(dz) < 1e-15) break;
    }
    { /* P_n' at the converged root */
      double p0 = 1.0, p1 = z;
      for (int j = 2; j <= n; ++j) {
        double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
        p0 = p1;
        p1 = p2;
      }
      dpn = n * (z * p1 - p0) / (z * z - 1.0);
    }
    double wi = 2.0 / ((1.0 - z * z) * dpn * dpn);
    /* z is the i-th largest root; store +z at the top, -z at the bottom */
    x[n - 1 - i] = z;
    x[i] = -z;
    w[n - 1 - i] = wi;
    w[i] = wi;
  }
  if (n % 2 == 1) x[m - 1] = 0.0;
  double half = 0.5 * (b - a), mid = 0.5 * (a + b);
  for (int i = 0; i < n; ++i) {
    x[i] = mid + half * x[i];
    w[i] = half * w[i];
  }
  return ORC_OK;
}

/* Gauss-Chebyshev rule of the second kind on [-1,1] for the weight
 * sqrt(1-x^2): x_j = cos(j pi/(n+1)), w_j = pi/(n+1) sin^2(j pi/(n+1)),
 * j = 1..n (closed form). */
int orc_gauss_chebyshev2(int n, double *x, double *w) {
  if (n < 1) return ORC_EINVAL;
  for (int j = 1; j <= n; ++j) {
    double th = j * ORC_PI / (n + 1.0);
    x[j - 1] = cos(th);
    w[j - 1] = ORC_PI / (n + 1.0) * sin(th) * sin(th);
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Regulators (Sec. 5.3.1 RB / RBdot; flat regulator of Fig. polyExpReg). */
/* R_k(q) = Z(q) k^2 r(x), x = q^2/k^2; k d_k R_k = Z(q) k^2 rdot(x) at   */
/* fixed Z (k d_k x = -2x).                                               */
/* ------------------------------------------------------------------ */

/* exponential shape r(x) = x/(e^x - 1); flat (Litim) shape (1-x) Theta(1-x). */
double orc_reg_r(int reg, double x) {
  if (reg == ORC_REG_LITIM) return x < 1.0 ? 1.0 - x : 0.0;
  if (x > 700.0) return 0.0;
  if (x < 1e-100) return 1.0;
  return x / expm1(x);
}

/* k d_k of k^2 r(q^2/k^2), divided by k^2:  2 r(x) - 2 x r'(x).
 * exponential: 2 x^2 e^{-x} / (1 - e^{-x})^2 ;  flat: 2 Theta(1-x). */
double orc_reg_rdot(int reg, double x) {
  if (reg == ORC_REG_LITIM) return x < 1.0 ? 2.0 : 0.0;
  if (x > 700.0) return 0.0;
  if (x < 1e-100) return 2.0;
  double em = expm1(-x);
  return 2.0 * x * x * exp(-x) / (em * em);
}

/* ------------------------------------------------------------------ */
/* Logarithmic-grid linear interpolation (App. F: LinearInterpolator1D   */
/* with LogarithmicCoordinates1D).  Grid x_j = x_min (x_max/x_min)^{j/(n-1)}; */
/* linear in the value between neighbouring nodes in ln s; clamped.       */
/* ------------------------------------------------------------------ */
static void lerp_pos(int n, double xmin, double xmax, double s, int *i0, double *w) {
  double sc = s < xmin ? xmin : s;
  double u = (n - 1) * log(sc / xmin) / log(xmax / xmin);
  if (u < 0.0) u = 0.0;
  if (u > n - 1.0) u = n - 1.0;
  int i = (int)floor(u);
  if (i > n - 2) i = n - 2;
  *i0 = i;
  *w = u - i;
}

double orc_lerp_log(const double *T, int n, double xmin, double xmax, double s) {
  int i0;
  double w;
  lerp_pos(n, xmin, xmax, s, &i0, &w);
  return (1.0 - w) * T[i0] + w * T[i0 + 1];
}

/* ------------------------------------------------------------------ */
/* Dual numbers (forward-mode AD, the paper's approach to Jacobians,      */
/* Sec. 5.2.2 "AD" mixin).  Derivatives flow only through table values:   */
/* lookup positions depend on momenta alone.                              */
/* ------------------------------------------------------------------ */
typedef struct { double v, d; } dual;
static dual dl(double v) { dual r = {v, 0.0}; return r; }
static dual dadd(dual a, dual b) { dual r = {a.v + b.v, a.d + b.d}; return r; }
static dual dmul(dual a, dual b) { dual r = {a.v * b.v, a.d * b.v + a.v * b.d}; return r; }
static dual dscale(dual a, double s) { dual r = {a.v * s, a.d * s}; return r; }
static dual drecip(dual a) { dual r = {1.0 / a.v, -a.d / (a.v * a.v)}; return r; }

static dual lerp_dual(const double *T, const double *dT, int n, double xmin, double xmax, double s) {
  int i0;
  double w;
  lerp_pos(n, xmin, xmax, s, &i0, &w);
  dual r;
  r.v = (1.0 - w) * T[i0] + w * T[i0 + 1];
  r.d = dT ? (1.0 - w) * dT[i0] + w * dT[i0 + 1] : 0.0;
  return r;
}

/* ------------------------------------------------------------------ */
/* Shared per-problem helpers.                                            */
/* ------------------------------------------------------------------ */
static double ext_p(const orc_problem *pb, int i) {
  if (pb->n_ext_p == 1) return pb->p_min;
  return pb->p_min * pow(pb->p_max / pb->p_min, (double)i / (pb->n_ext_p - 1));
}

static double m2_of(const orc_problem *pb, double k) { return pb->m2_over_k2 * k * k + pb->m2_shift; }

int orc_n_ext(const orc_problem *pb) {
  switch (pb->model) {
  case ORC_D3: return pb->n_ext_p + (pb->include_p0 ? 1 : 0);
  case ORC_D4_VERTEX:
  case ORC_D4_FULL: return 2 * pb->n_ext_p + 1 + pb->n_ext_p * pb->n_ext_ang;
  case ORC_FINITE_T:
  case ORC_FINITE_T_4D: return pb->n_ext_p * pb->n_ext_ang;
  default: return -1;
  }
}

static int check_problem(const orc_problem *pb) {
  if (!pb) return ORC_EINVAL;
  if (pb->model < ORC_D3 || pb->model > ORC_FINITE_T_4D) return ORC_EINVAL;
  if (pb->model == ORC_FINITE_T_4D &&
      (pb->n_ext_ang < 1 || pb->n_matsubara < 0 || pb->n_tables < 2 || pb->n_stack != 1 || pb->n_x0 < 1 ||
       !(pb->T > 0.0) || (pb->statistics == 1 && pb->n_ext_ang != 1)))
    return ORC_EINVAL;
  if (pb->model == ORC_D4_FULL && (pb->n_va < 1 || pb->n_vb < 1 || pb->n_stack != pb->n_va * pb->n_vb ||
                                   pb->n_ang2 < 1 || pb->n_ext_ang < 1 || pb->n_tables < 3))
    return ORC_EINVAL;
  if (pb->n_rad < 1 || pb->n_ang1 < 1 || pb->n_ext_p < 1 || pb->n_pts < 2) return ORC_EINVAL;
  if (pb->model == ORC_D4_VERTEX && (pb->n_ang2 < 1 || pb->n_ext_ang < 1 || pb->n_tables < 3)) return ORC_EINVAL;
  if (pb->model == ORC_FINITE_T && (pb->n_ext_ang < 1 || pb->n_matsubara < 0 || pb->n_tables < 2 || pb->n_stack < 1))
    return ORC_EINVAL;
  if (pb->model == ORC_D3 && pb->n_tables < 1) return ORC_EINVAL;
  if (pb->statistics != 0 && (pb->statistics != 1 || (pb->model != ORC_FINITE_T && pb->model != ORC_FINITE_T_4D)))
    return ORC_EINVAL;
  if (!(pb->x_min > 0.0) || !(pb->x_max > pb->x_min) || !(pb->p_min > 0.0)) return ORC_EINVAL;
  return ORC_OK;
}

/* Propagator with a Z-dressed regulator (App. G bosonic propagator form,
 * with dressing Z and spatial regulator):
 *   G = 1 / ( Z (omega^2 + s^2) + m^2 + Z k^2 r(s^2/k^2) ). */
static double propagator(int reg, double Z, double om2, double s2, double m2, double k) {
  double k2 = k * k;
  return 1.0 / (Z * (om2 + s2) + m2 + Z * k2 * orc_reg_r(reg, s2 / k2));
}

static dual propagator_dual(int reg, dual Z, double om2, double s2, double m2, double k) {
  double k2 = k * k;
  dual den = dadd(dmul(Z, dl(om2 + s2 + k2 * orc_reg_r(reg, s2 / k2))), dl(m2));
  return drecip(den);
}

/* ------------------------------------------------------------------ */
/* Model d=3, T=0: scalar two-point flow                                  */
/*   I(p) = pref lam^2 int d^3q/(2pi)^3 dR(q) G(q)^2 G(|q+p|)             */
/* with the one-angle reduction d^3q/(2pi)^3 = q^2 dq dcos / (4 pi^2).     */
/* ------------------------------------------------------------------ */

/* summand without measure: dR(q) G(q)^2 G(s), s^2 = |q+p|^2 */
double orc_d3_summand(const orc_problem *pb, const double *tab, double k, double q2, double s2) {
  int n = pb->n_pts, reg = pb->regulator;
  double k2 = k * k, m2 = m2_of(pb, k);
  if (s2 < 0.0) s2 = 0.0;
  double q = sqrt(q2), s = sqrt(s2);
  double Zq = orc_lerp_log(tab, n, pb->x_min, pb->x_max, q);
  double Zs = orc_lerp_log(tab, n, pb->x_min, pb->x_max, s);
  double dR = Zq * k2 * orc_reg_rdot(reg, q2 / k2);
  double Gq = propagator(reg, Zq, 0.0, q2, m2, k);
  double Gs = propagator(reg, Zs, 0.0, s2, m2, k);
  return dR * Gq * Gq * Gs;
}

static dual d3_summand_dual(const orc_problem *pb, const double *tab, const double *dtab, double k, double q2,
                            double s2) {
  int n = pb->n_pts, reg = pb->regulator;
  double k2 = k * k, m2 = m2_of(pb, k);
  if (s2 < 0.0) s2 = 0.0;
  double q = sqrt(q2), s = sqrt(s2);
  dual Zq = lerp_dual(tab, dtab, n, pb->x_min, pb->x_max, q);
  dual Zs = lerp_dual(tab, dtab, n, pb->x_min, pb->x_max, s);
  dual dR = dscale(Zq, k2 * orc_reg_rdot(reg, q2 / k2));
  dual Gq = propagator_dual(reg, Zq, 0.0, q2, m2, k);
  dual Gs = propagator_dual(reg, Zs, 0.0, s2, m2, k);
  return dmul(dmul(dR, dmul(Gq, Gq)), Gs);
}

static int rhs_d3(const orc_problem *pb, const double *tab, const double *dtab, double k, double *out,
                  double *dout, const int *sel, int nsel) {
  int nr = pb->n_rad, na = pb->n_ang1, ne = orc_n_ext(pb);
  double *xr = malloc(sizeof(double) * nr), *wr = malloc(sizeof(double) * nr);
  double *xa = malloc(sizeof(double) * na), *wa = malloc(sizeof(double) * na);
  if (!xr || !wr || !xa || !wa) { free(xr); free(wr); free(xa); free(wa); return ORC_ENOMEM; }
  orc_gauss_legendre(nr, 0.0, pb->qmax_over_k * k, xr, wr);
  orc_gauss_legendre(na, -1.0, 1.0, xa, wa);
  double norm = pb->prefactor * pb->lam * pb->lam / (4.0 * ORC_PI * ORC_PI);
  int nloop = sel ? nsel : ne;
#pragma omp parallel for schedule(dynamic, 1)
  for (int ie = 0; ie < nloop; ++ie) {
    int e = sel ? sel[ie] : ie;
    double p = (e < pb->n_ext_p) ? ext_p(pb, e) : 0.0;
    acc_t acc = {0, 0}, dacc = {0, 0};
    for (int i = 0; i < nr; ++i) {
      double q = xr[i];
      for (int j = 0; j < na; ++j) {
        double s2 = q * q + p * p + 2.0 * q * p * xa[j];
        double wgt = wr[i] * wa[j] * q * q;
        if (dout) {
          dual f = d3_summand_dual(pb, tab, dtab, k, q * q, s2);
          acc_add(&acc, wgt * f.v);
          acc_add(&dacc, wgt * f.d);
        } else {
          acc_add(&acc, wgt * orc_d3_summand(pb, tab, k, q * q, s2));
        }
      }
    }
    out[ie] = norm * acc_get(&acc);
    if (dout) dout[ie] = norm * acc_get(&dacc);
  }
  free(xr); free(wr); free(xa); free(wa);
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Model d=4, T=0, vertex expansion with three dressings                  */
/* Z(S), lambda3(S), lambda4(S) and the average momentum                  */
/* S0 = sqrt(sum_i |p_i|^2 / n) of the n legs (Sec. 3.3).                 */
/* Measure: d^4q/(2pi)^4 = q^3 dq sqrt(1-c1^2) dc1 dc2 / (8 pi^3)          */
/* (third angle integrated), c1 with a Gauss-Chebyshev-II rule, c2 GL.     */
/* External legs: p1 = p e1, p2 = p (cos psi e1 + sin psi e2).             */
/* ------------------------------------------------------------------ */

/* Propagator-flow diagrams:  dR G(q)^2 [ -1/2 lambda4(S0(q,-q,p,-p))
 *                                        + lambda3(S0(q,q+p,p))^2 G(|q+p|) ]   */
/* D4_FULL: three-point vertex lambda3(S0, a, b) on the log grid in S0 times
 * uniform grids of n_va and n_vb nodes on [-1, 1] in its shape variables,
 * stored as stack rows ia * n_vb + ib of table 1 (the "Full" vertex
 * dependence of Sec. 3.3 and the 3-D interpolators of App. F).  For a vertex
 * with legs k1, k2, k3 (k1 + k2 + k3 = 0) and squared magnitudes s1, s2, s3:
 *   S0^2 = (s1 + s2 + s3)/3,
 *   a = k1.k2/(|k1||k2|) = (s3 - s1 - s2)/(2 sqrt(s1 s2)),
 *   b = (s1 - s2)/(s1 + s2),
 * each of a, b clamped to [-1, 1] (NaN to -1); linear in the value between
 * nodes in ln S0, a and b (trilinear), clamped at the grid ends. */
static double clamp_shape(double v) { return v >= -1.0 ? (v <= 1.0 ? v : 1.0) : -1.0; }

static void shape_pos(double v, int m, int *i0, double *w) {
  if (m < 2) {
    *i0 = 0;
    *w = 0.0;
    return;
  }
  double u = 0.5 * (v + 1.0) * (m - 1);
  int i = (int)u;
  if (i > m - 2) i = m - 2;
  *i0 = i;
  *w = u - i;
}

double orc_d4_shape(double s1, double s2, double s3, int which) {
  if (which == 0) return clamp_shape((s3 - s1 - s2) / (2.0 * sqrt(s1 * s2)));
  return clamp_shape((s1 - s2) / (s1 + s2));
}

double orc_lam3_full(const orc_problem *pb, const double *tab, double s1, double s2, double s3) {
  const int n = pb->n_pts, na = pb->n_va, nb = pb->n_vb;
  const double S = sqrt((s1 + s2 + s3) / 3.0);
  int ia, ib;
  double wa, wb;
  shape_pos(orc_d4_shape(s1, s2, s3, 0), na, &ia, &wa);
  shape_pos(orc_d4_shape(s1, s2, s3, 1), nb, &ib, &wb);
  const int da = na > 1 ? nb : 0, db = nb > 1 ? 1 : 0;
  const double *L3 = tab + (size_t)pb->n_stack * n;
  const int r = ia * nb + ib;
  double v00 = orc_lerp_log(L3 + (size_t)r * n, n, pb->x_min, pb->x_max, S);
  double v01 = orc_lerp_log(L3 + (size_t)(r + db) * n, n, pb->x_min, pb->x_max, S);
  double v10 = orc_lerp_log(L3 + (size_t)(r + da) * n, n, pb->x_min, pb->x_max, S);
  double v11 = orc_lerp_log(L3 + (size_t)(r + da + db) * n, n, pb->x_min, pb->x_max, S);
  return (1.0 - wa) * ((1.0 - wb) * v00 + wb * v01) + wa * ((1.0 - wb) * v10 + wb * v11);
}

/* lambda3 at the vertex with legs of squared magnitudes s1, s2, s3 */
static double lam3_at(const orc_problem *pb, const double *tab, double s1, double s2, double s3) {
  if (pb->model == ORC_D4_FULL) return orc_lam3_full(pb, tab, s1, s2, s3);
  return orc_lerp_log(tab + (size_t)pb->n_stack * pb->n_pts, pb->n_pts, pb->x_min, pb->x_max,
                      sqrt((s1 + s2 + s3) / 3.0));
}

double orc_d4_summand_z(const orc_problem *pb, const double *tab, double k, double q2, double p2, double A2) {
  int n = pb->n_pts, reg = pb->regulator;
  const double *Zt = tab, *L4 = tab + (size_t)2 * pb->n_stack * n;
  double k2 = k * k, m2 = m2_of(pb, k);
  if (A2 < 0.0) A2 = 0.0;
  double Zq = orc_lerp_log(Zt, n, pb->x_min, pb->x_max, sqrt(q2));
  double ZA = orc_lerp_log(Zt, n, pb->x_min, pb->x_max, sqrt(A2));
  double l4 = orc_lerp_log(L4, n, pb->x_min, pb->x_max, sqrt((2.0 * q2 + 2.0 * p2) / 4.0));
  double l3 = lam3_at(pb, tab, q2, A2, p2);   /* legs q, q+p, p */
  double dR = Zq * k2 * orc_reg_rdot(reg, q2 / k2);
  double Gq = propagator(reg, Zq, 0.0, q2, m2, k);
  double GA = propagator(reg, ZA, 0.0, A2, m2, k);
  return dR * Gq * Gq * (-0.5 * l4 + l3 * l3 * GA);
}

/* Three-point-vertex flow:
 * 3 dR G(q)^2 G(|q+p1|) G(|q-p2|) l3(S0(q,q+p1,p1)) l3(S0(q,q-p2,p2)) l3(S0(q+p1,q-p2,p1+p2)) */
double orc_d4_summand_3(const orc_problem *pb, const double *tab, double k, double q2, double p2, double A2,
                        double B2, double C2) {
  int n = pb->n_pts, reg = pb->regulator;
  const double *Zt = tab;
  double k2 = k * k, m2 = m2_of(pb, k);
  if (A2 < 0.0) A2 = 0.0;
  if (B2 < 0.0) B2 = 0.0;
  double Zq = orc_lerp_log(Zt, n, pb->x_min, pb->x_max, sqrt(q2));
  double ZA = orc_lerp_log(Zt, n, pb->x_min, pb->x_max, sqrt(A2));
  double ZB = orc_lerp_log(Zt, n, pb->x_min, pb->x_max, sqrt(B2));
  double la = lam3_at(pb, tab, q2, A2, p2);   /* legs q, q+p1, p1 */
  double lb = lam3_at(pb, tab, q2, B2, p2);   /* legs q, q-p2, p2 */
  double lc = lam3_at(pb, tab, A2, B2, C2);   /* legs q+p1, q-p2, p1+p2 */
  double dR = Zq * k2 * orc_reg_rdot(reg, q2 / k2);
  double Gq = propagator(reg, Zq, 0.0, q2, m2, k);
  double GA = propagator(reg, ZA, 0.0, A2, m2, k);
  double GB = propagator(reg, ZB, 0.0, B2, m2, k);
  return 3.0 * dR * Gq * Gq * GA * GB * la * lb * lc;
}

/* Four-point-vertex flow:  3/2 dR G(q)^2 G(|q+p|) lambda4(S0(q,q+p,p,p))^2 */
double orc_d4_summand_4(const orc_problem *pb, const double *tab, double k, double q2, double p2, double A2) {
  int n = pb->n_pts, reg = pb->regulator;
  const double *Zt = tab, *L4 = tab + (size_t)2 * pb->n_stack * n;
  double k2 = k * k, m2 = m2_of(pb, k);
  if (A2 < 0.0) A2 = 0.0;
  double Zq = orc_lerp_log(Zt, n, pb->x_min, pb->x_max, sqrt(q2));
  double ZA = orc_lerp_log(Zt, n, pb->x_min, pb->x_max, sqrt(A2));
  double l4 = orc_lerp_log(L4, n, pb->x_min, pb->x_max, sqrt((q2 + A2 + 2.0 * p2) / 4.0));
  double dR = Zq * k2 * orc_reg_rdot(reg, q2 / k2);
  double Gq = propagator(reg, Zq, 0.0, q2, m2, k);
  double GA = propagator(reg, ZA, 0.0, A2, m2, k);
  return 1.5 * dR * Gq * Gq * GA * l4 * l4;
}

/* dual versions of the three summands (same expressions, dual arithmetic) */
static dual d4_summand_dual(int block, const orc_problem *pb, const double *tab, const double *dtab, double k,
                            double q2, double p2, double A2, double B2, double C2) {
  int n = pb->n_pts, reg = pb->regulator;
  const double *Zt = tab, *L3 = tab + n, *L4 = tab + 2 * n;
  const double *dZt = dtab, *dL3 = dtab + n, *dL4 = dtab + 2 * n;
  double k2 = k * k, m2 = m2_of(pb, k);
  if (A2 < 0.0) A2 = 0.0;
  if (B2 < 0.0) B2 = 0.0;
  dual Zq = lerp_dual(Zt, dZt, n, pb->x_min, pb->x_max, sqrt(q2));
  dual ZA = lerp_dual(Zt, dZt, n, pb->x_min, pb->x_max, sqrt(A2));
  dual dR = dscale(Zq, k2 * orc_reg_rdot(reg, q2 / k2));
  dual Gq = propagator_dual(reg, Zq, 0.0, q2, m2, k);
  dual GA = propagator_dual(reg, ZA, 0.0, A2, m2, k);
  dual base = dmul(dR, dmul(Gq, Gq));
  if (block == 0) {
    dual l4 = lerp_dual(L4, dL4, n, pb->x_min, pb->x_max, sqrt((2.0 * q2 + 2.0 * p2) / 4.0));
    dual l3 = lerp_dual(L3, dL3, n, pb->x_min, pb->x_max, sqrt((q2 + A2 + p2) / 3.0));
    return dmul(base, dadd(dscale(l4, -0.5), dmul(dmul(l3, l3), GA)));
  } else if (block == 1) {
    dual ZB = lerp_dual(Zt, dZt, n, pb->x_min, pb->x_max, sqrt(B2));
    dual la = lerp_dual(L3, dL3, n, pb->x_min, pb->x_max, sqrt((q2 + A2 + p2) / 3.0));
    dual lb = lerp_dual(L3, dL3, n, pb->x_min, pb->x_max, sqrt((q2 + B2 + p2) / 3.0));
    dual lc = lerp_dual(L3, dL3, n, pb->x_min, pb->x_max, sqrt((A2 + B2 + C2) / 3.0));
    dual GB = propagator_dual(reg, ZB, 0.0, B2, m2, k);
    return dscale(dmul(dmul(dmul(base, GA), GB), dmul(dmul(la, lb), lc)), 3.0);
  } else {
    dual l4 = lerp_dual(L4, dL4, n, pb->x_min, pb->x_max, sqrt((q2 + A2 + 2.0 * p2) / 4.0));
    return dscale(dmul(dmul(base, GA), dmul(l4, l4)), 1.5);
  }
}

static int rhs_d4(const orc_problem *pb, const double *tab, const double *dtab, double k, double *out,
                  double *dout, const int *sel, int nsel) {
  int nr = pb->n_rad, n1 = pb->n_ang1, n2 = pb->n_ang2, np = pb->n_ext_p, npsi = pb->n_ext_ang;
  int ne = orc_n_ext(pb);
  double *xr = malloc(sizeof(double) * nr), *wr = malloc(sizeof(double) * nr);
  double *x1 = malloc(sizeof(double) * n1), *w1 = malloc(sizeof(double) * n1);
  double *x2 = malloc(sizeof(double) * n2), *w2 = malloc(sizeof(double) * n2);
  double *xp = malloc(sizeof(double) * npsi), *wp = malloc(sizeof(double) * npsi);
  if (!xr || !wr || !x1 || !w1 || !x2 || !w2 || !xp || !wp) {
    free(xr); free(wr); free(x1); free(w1); free(x2); free(w2); free(xp); free(wp);
    return ORC_ENOMEM;
  }
  orc_gauss_legendre(nr, 0.0, pb->qmax_over_k * k, xr, wr);
  orc_gauss_chebyshev2(n1, x1, w1);
  orc_gauss_legendre(n2, -1.0, 1.0, x2, w2);
  orc_gauss_legendre(npsi, -1.0, 1.0, xp, wp);
  double norm = pb->prefactor / (8.0 * ORC_PI * ORC_PI * ORC_PI);
  int nloop = sel ? nsel : ne;
#pragma omp parallel for schedule(dynamic, 1)
  for (int ie = 0; ie < nloop; ++ie) {
    int e = sel ? sel[ie] : ie;
    /* external-point layout: [Z: p_0..p_{np-1}, p=0][lambda3: p x psi][lambda4: p] */
    int block;
    double p, cpsi = 1.0, spsi = 0.0;
    if (e <= np) {
      block = 0;
      p = (e < np) ? ext_p(pb, e) : 0.0;
    } else if (e < np + 1 + np * npsi) {
      block = 1;
      int r = e - (np + 1);
      p = ext_p(pb, r / npsi);
      cpsi = xp[r % npsi];
      spsi = sqrt(1.0 - cpsi * cpsi);
    } else {
      block = 2;
      p = ext_p(pb, e - (np + 1 + np * npsi));
    }
    double p2 = p * p;
    double C2 = 2.0 * p2 * (1.0 + cpsi);
    acc_t acc = {0, 0}, dacc = {0, 0};
    for (int i = 0; i < nr; ++i) {
      double q = xr[i], q2 = q * q;
      for (int a = 0; a < n1; ++a) {
        double c1 = x1[a], s1 = sqrt(1.0 - c1 * c1);
        for (int b = 0; b < n2; ++b) {
          double c2 = x2[b];
          double A2 = q2 + p2 + 2.0 * q * p * c1;
          double qp2 = q * p * (cpsi * c1 + spsi * s1 * c2);
          double B2 = q2 + p2 - 2.0 * qp2;
          double wgt = wr[i] * w1[a] * w2[b] * q2 * q;
          if (dout) {
            dual f = d4_summand_dual(block, pb, tab, dtab, k, q2, p2, A2, B2, C2);
            acc_add(&acc, wgt * f.v);
            acc_add(&dacc, wgt * f.d);
          } else {
            double f;
            if (block == 0) f = orc_d4_summand_z(pb, tab, k, q2, p2, A2);
            else if (block == 1) f = orc_d4_summand_3(pb, tab, k, q2, p2, A2, B2, C2);
            else f = orc_d4_summand_4(pb, tab, k, q2, p2, A2);
            acc_add(&acc, wgt * f);
          }
        }
      }
    }
    out[ie] = norm * acc_get(&acc);
    if (dout) dout[ie] = norm * acc_get(&dacc);
  }
  free(xr); free(wr); free(x1); free(w1); free(x2); free(w2); free(xp); free(wp);
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Model finite T (Quadratureq0, Sec. 5.3.2): spatial regulator (Sec. 3.1). */
/* Bosonic loop: omega_n = 2 pi T n, |n| <= N, tables stacked over |n|     */
/* (App. F BosonicCoordinates1DFiniteT stack).  Fermionic loop: nu_n =     */
/* (2n+1) pi T, -N-1 <= n <= N (2N+2 frequencies, symmetric about 0),      */
/* tables stacked over j = n (n >= 0) or -n-1 (n < 0), so that row j holds */
/* nu_j = (2j+1) pi T (App. F FermionicCoordinates1DFiniteT stack).  The   */
/* external frequency is bosonic, omega_m = 2 pi T m; the shifted line     */
/* carries nu_n + omega_m = nu_{n+m}.  Stack indices are clamped.          */
/*   I(m,p) = pref lam^2 T sum_n int d^3q/(2pi)^3                          */
/*            dR(n,q) G(n,q)^2 L(n,q) L(n+m,|q+p|) G(n+m,|q+p|)            */
/* ------------------------------------------------------------------ */
static const double *stack_row(const double *tab, const orc_problem *pb, int t, int n) {
  int a;
  if (pb->statistics) a = n >= 0 ? n : -n - 1;
  else a = n < 0 ? -n : n;
  if (a > pb->n_stack - 1) a = pb->n_stack - 1;
  return tab + ((size_t)t * pb->n_stack + a) * pb->n_pts;
}

/* Matsubara frequency of loop index n */
static double matsubara(const orc_problem *pb, int n) {
  return pb->statistics ? (2.0 * n + 1.0) * ORC_PI * pb->T : 2.0 * ORC_PI * pb->T * n;
}

double orc_ft_summand(const orc_problem *pb, const double *tab, double k, int n, int m, double q2, double s2) {
  int np = pb->n_pts, reg = pb->regulator;
  double k2 = k * k, m2 = m2_of(pb, k);
  if (s2 < 0.0) s2 = 0.0;
  double q = sqrt(q2), s = sqrt(s2);
  double wn = matsubara(pb, n), wnm = matsubara(pb, n + m);
  double Zq = orc_lerp_log(stack_row(tab, pb, 0, n), np, pb->x_min, pb->x_max, q);
  double Lq = orc_lerp_log(stack_row(tab, pb, 1, n), np, pb->x_min, pb->x_max, q);
  double Zs = orc_lerp_log(stack_row(tab, pb, 0, n + m), np, pb->x_min, pb->x_max, s);
  double Ls = orc_lerp_log(stack_row(tab, pb, 1, n + m), np, pb->x_min, pb->x_max, s);
  double dR = Zq * k2 * orc_reg_rdot(reg, q2 / k2);
  double Gq = propagator(reg, Zq, wn * wn, q2, m2, k);
  double Gs = propagator(reg, Zs, wnm * wnm, s2, m2, k);
  return dR * Gq * Gq * Lq * Ls * Gs;
}

static int rhs_ft(const orc_problem *pb, const double *tab, double k, double *out, const int *sel, int nsel) {
  int nr = pb->n_rad, na = pb->n_ang1, N = pb->n_matsubara, nm = pb->n_ext_ang;
  int ne = orc_n_ext(pb);
  double *xr = malloc(sizeof(double) * nr), *wr = malloc(sizeof(double) * nr);
  double *xa = malloc(sizeof(double) * na), *wa = malloc(sizeof(double) * na);
  if (!xr || !wr || !xa || !wa) { free(xr); free(wr); free(xa); free(wa); return ORC_ENOMEM; }
  orc_gauss_legendre(nr, 0.0, pb->qmax_over_k * k, xr, wr);
  orc_gauss_legendre(na, -1.0, 1.0, xa, wa);
  double norm = pb->prefactor * pb->lam * pb->lam * pb->T / (4.0 * ORC_PI * ORC_PI);
  int nloop = sel ? nsel : ne;
#pragma omp parallel for schedule(dynamic, 1)
  for (int ie = 0; ie < nloop; ++ie) {
    int e = sel ? sel[ie] : ie;
    int ip = e / nm, m = e % nm;
    double p = ext_p(pb, ip);
    acc_t acc = {0, 0};
    for (int n = pb->statistics ? -N - 1 : -N; n <= N; ++n) {
      for (int i = 0; i < nr; ++i) {
        double q = xr[i];
        for (int j = 0; j < na; ++j) {
          double s2 = q * q + p * p + 2.0 * q * p * xa[j];
          acc_add(&acc, wr[i] * wa[j] * q * q * orc_ft_summand(pb, tab, k, n, m, q * q, s2));
        }
      }
    }
    out[ie] = norm * acc_get(&acc);
  }
  free(xr); free(wr); free(xa); free(wa);
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Model finite T with a 4-dimensional regulator on a k-scaled frequency    */
/* domain (Sec. 5.3.2: "Quadraturex0" integrators treat the time direction */
/* as a Matsubara sum over a domain that scales with k, efficient with     */
/* 4-dimensional regulators; App. G: external fermion legs at             */
/* p0f = pi T exp(-k/(pi T))).  With Q = (q0, q), P = (p0, p):              */
/*   I(m,p) = pref lam^2 [T sum_n | int dq0/2pi] int d^3q/(2pi)^3          */
/*            dR(Q) G(Q)^2 L(|Q|) L(|Q+P|) G(Q+P),                         */
/* R(Q) = Z(|Q|) k^2 r(|Q|^2/k^2) (4D), G(Q) = 1/(Z(|Q|) |Q|^2 + m^2 + R),  */
/* dressings Z and L on one log grid in |Q|.  Frequency domain |q0| <=      */
/* L0 = qmax_over_k k.  Loop frequencies in the domain: bosonic 2 pi T n,   */
/* |n| <= floor(L0/(2 pi T)); fermionic (2n+1) pi T, -N_k-1 <= n <= N_k,    */
/* N_k = floor((L0/(pi T) - 1)/2) (none if L0 < pi T).  While their number */
/* is at most the cap 2 n_matsubara + 1 (+1 fermionic) the frequency       */
/* integral is that Matsubara sum with weight T; beyond it, the T -> 0     */
/* form: Gauss-Legendre with n_x0 nodes on [-L0, L0], weights w/(2 pi).    */
/* External frequency p0: bosonic 2 pi T m; fermionic (n_ext_ang = 1) the  */
/* external fermion leg's p0f = pi T exp(-k/(pi T)).                        */
/* ------------------------------------------------------------------ */
int orc_ft4_frequencies(const orc_problem *pb, double k, double *w, double *wt) {
  double L0 = pb->qmax_over_k * k, T = pb->T;
  int cap = 2 * pb->n_matsubara + 1 + (pb->statistics ? 1 : 0);
  int count;
  if (pb->statistics) {
    double x = L0 / (ORC_PI * T);
    int Nk = x < 1.0 ? -1 : (int)floor((x - 1.0) / 2.0);
    count = 2 * Nk + 2;
    if (count <= cap) {
      for (int n = -Nk - 1; n <= Nk; ++n) {
        w[n + Nk + 1] = (2.0 * n + 1.0) * ORC_PI * T;
        wt[n + Nk + 1] = T;
      }
      return count;
    }
  } else {
    int Nk = (int)floor(L0 / (2.0 * ORC_PI * T));
    count = 2 * Nk + 1;
    if (count <= cap) {
      for (int n = -Nk; n <= Nk; ++n) {
        w[n + Nk] = 2.0 * ORC_PI * T * n;
        wt[n + Nk] = T;
      }
      return count;
    }
  }
  orc_gauss_legendre(pb->n_x0, -L0, L0, w, wt);
  for (int i = 0; i < pb->n_x0; ++i) wt[i] /= 2.0 * ORC_PI;
  return pb->n_x0;
}

double orc_ft4_external_frequency(const orc_problem *pb, double k, int m) {
  if (pb->statistics) return ORC_PI * pb->T * exp(-k / (ORC_PI * pb->T));
  return 2.0 * ORC_PI * pb->T * m;
}

double orc_ft4_summand(const orc_problem *pb, const double *tab, double k, double Q2, double QP2) {
  int np = pb->n_pts, reg = pb->regulator;
  double k2 = k * k, m2 = m2_of(pb, k);
  if (QP2 < 0.0) QP2 = 0.0;
  const double *Zt = tab, *Lt = tab + np;
  double Zq = orc_lerp_log(Zt, np, pb->x_min, pb->x_max, sqrt(Q2));
  double Lq = orc_lerp_log(Lt, np, pb->x_min, pb->x_max, sqrt(Q2));
  double Zs = orc_lerp_log(Zt, np, pb->x_min, pb->x_max, sqrt(QP2));
  double Ls = orc_lerp_log(Lt, np, pb->x_min, pb->x_max, sqrt(QP2));
  double dR = Zq * k2 * orc_reg_rdot(reg, Q2 / k2);
  double Gq = propagator(reg, Zq, 0.0, Q2, m2, k);
  double Gs = propagator(reg, Zs, 0.0, QP2, m2, k);
  return dR * Gq * Gq * Lq * Ls * Gs;
}

static int rhs_ft4(const orc_problem *pb, const double *tab, double k, double *out, const int *sel, int nsel) {
  int nr = pb->n_rad, na = pb->n_ang1, nm = pb->n_ext_ang;
  int ne = orc_n_ext(pb), nmax = 2 * pb->n_matsubara + 2 + pb->n_x0;
  double *xr = malloc(sizeof(double) * nr), *wr = malloc(sizeof(double) * nr);
  double *xa = malloc(sizeof(double) * na), *wa = malloc(sizeof(double) * na);
  double *wf = malloc(sizeof(double) * nmax), *wtf = malloc(sizeof(double) * nmax);
  if (!xr || !wr || !xa || !wa || !wf || !wtf) {
    free(xr); free(wr); free(xa); free(wa); free(wf); free(wtf);
    return ORC_ENOMEM;
  }
  orc_gauss_legendre(nr, 0.0, pb->qmax_over_k * k, xr, wr);
  orc_gauss_legendre(na, -1.0, 1.0, xa, wa);
  int nf = orc_ft4_frequencies(pb, k, wf, wtf);
  double norm = pb->prefactor * pb->lam * pb->lam / (4.0 * ORC_PI * ORC_PI);
  int nloop = sel ? nsel : ne;
#pragma omp parallel for schedule(dynamic, 1)
  for (int ie = 0; ie < nloop; ++ie) {
    int e = sel ? sel[ie] : ie;
    int ip = e / nm, m = e % nm;
    double p = ext_p(pb, ip), p0 = orc_ft4_external_frequency(pb, k, m);
    acc_t acc = {0, 0};
    for (int f = 0; f < nf; ++f) {
      for (int i = 0; i < nr; ++i) {
        double q = xr[i];
        double Q2 = wf[f] * wf[f] + q * q;
        for (int j = 0; j < na; ++j) {
          double s2 = q * q + p * p + 2.0 * q * p * xa[j];
          double QP2 = (wf[f] + p0) * (wf[f] + p0) + s2;
          acc_add(&acc, wtf[f] * wr[i] * wa[j] * q * q * orc_ft4_summand(pb, tab, k, Q2, QP2));
        }
      }
    }
    out[ie] = norm * acc_get(&acc);
  }
  free(xr); free(wr); free(xa); free(wa); free(wf); free(wtf);
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Finite T: the sum over many loop-side states sharing the shifted line   */
/* (the angle-integrated kernel K(p, q) of Sec. 5.3.2, contracted with     */
/* more than one radial factor).  A state F_s is the loop-side factor      */
/* sampled at the loop frequencies and radial nodes, F_s[n - n_lo][i]      */
/* (n_lo = -N bosonic, -N-1 fermionic), without quadrature weights:        */
/*   out[s][e] = pref lam^2 T/(4 pi^2) sum_n sum_i sum_j wr_i wa_j q_i^2   */
/*               F_s[n - n_lo][i] L(n+m, s_ij) G(n+m, s_ij),               */
/* s_ij = |q_i + p| at the angle node j, e = (p, m) as in the RHS layout.  */
/* With F_s = dR(n, q) G(n, q)^2 L(n, q) (orc_ft_loop_factors) this is the */
/* finite-T RHS.                                                           */
/* ------------------------------------------------------------------ */
int orc_ft_loop_factors(const orc_problem *pb, const double *tab, double k, double *F) {
  int st = check_problem(pb);
  if (st) return st;
  if (pb->model != ORC_FINITE_T || !(k > 0.0) || !tab || !F) return ORC_EINVAL;
  int nr = pb->n_rad, N = pb->n_matsubara, n_lo = pb->statistics ? -N - 1 : -N;
  double *xr = malloc(sizeof(double) * nr), *wr = malloc(sizeof(double) * nr);
  if (!xr || !wr) { free(xr); free(wr); return ORC_ENOMEM; }
  orc_gauss_legendre(nr, 0.0, pb->qmax_over_k * k, xr, wr);
  double k2 = k * k, m2 = m2_of(pb, k);
  for (int n = n_lo; n <= N; ++n) {
    double wn = matsubara(pb, n);
    for (int i = 0; i < nr; ++i) {
      double q = xr[i];
      double Zq = orc_lerp_log(stack_row(tab, pb, 0, n), pb->n_pts, pb->x_min, pb->x_max, q);
      double Lq = orc_lerp_log(stack_row(tab, pb, 1, n), pb->n_pts, pb->x_min, pb->x_max, q);
      double dR = Zq * k2 * orc_reg_rdot(pb->regulator, q * q / k2);
      double Gq = propagator(pb->regulator, Zq, wn * wn, q * q, m2, k);
      F[(size_t)(n - n_lo) * nr + i] = dR * Gq * Gq * Lq;
    }
  }
  free(xr); free(wr);
  return ORC_OK;
}

int orc_ft_states(const orc_problem *pb, const double *tab, double k, int n_states, const double *F, double *out) {
  int st = check_problem(pb);
  if (st) return st;
  if (pb->model != ORC_FINITE_T || !(k > 0.0) || !tab || !F || !out || n_states < 0) return ORC_EINVAL;
  int nr = pb->n_rad, na = pb->n_ang1, N = pb->n_matsubara, nm = pb->n_ext_ang;
  int ne = orc_n_ext(pb), n_lo = pb->statistics ? -N - 1 : -N, nfreq = N - n_lo + 1;
  double *xr = malloc(sizeof(double) * nr), *wr = malloc(sizeof(double) * nr);
  double *xa = malloc(sizeof(double) * na), *wa = malloc(sizeof(double) * na);
  if (!xr || !wr || !xa || !wa) { free(xr); free(wr); free(xa); free(wa); return ORC_ENOMEM; }
  orc_gauss_legendre(nr, 0.0, pb->qmax_over_k * k, xr, wr);
  orc_gauss_legendre(na, -1.0, 1.0, xa, wa);
  double norm = pb->prefactor * pb->lam * pb->lam * pb->T / (4.0 * ORC_PI * ORC_PI);
  double m2 = m2_of(pb, k);
#pragma omp parallel for collapse(2) schedule(dynamic, 1)
  for (int s = 0; s < n_states; ++s) {
    for (int e = 0; e < ne; ++e) {
      const double *Fs = F + (size_t)s * nfreq * nr;
      int ip = e / nm, m = e % nm;
      double p = ext_p(pb, ip);
      acc_t acc = {0, 0};
      for (int n = n_lo; n <= N; ++n) {
        double wnm = matsubara(pb, n + m);
        const double *Zrow = stack_row(tab, pb, 0, n + m), *Lrow = stack_row(tab, pb, 1, n + m);
        for (int i = 0; i < nr; ++i) {
          double q = xr[i];
          for (int j = 0; j < na; ++j) {
            double s2 = q * q + p * p + 2.0 * q * p * xa[j];
            if (s2 < 0.0) s2 = 0.0;
            double sv = sqrt(s2);
            double Zs = orc_lerp_log(Zrow, pb->n_pts, pb->x_min, pb->x_max, sv);
            double Ls = orc_lerp_log(Lrow, pb->n_pts, pb->x_min, pb->x_max, sv);
            double Gs = propagator(pb->regulator, Zs, wnm * wnm, s2, m2, k);
            acc_add(&acc, wr[i] * wa[j] * q * q * Fs[(size_t)(n - n_lo) * nr + i] * Ls * Gs);
          }
        }
      }
      out[(size_t)s * ne + e] = norm * acc_get(&acc);
    }
  }
  free(xr); free(wr); free(xa); free(wa);
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Public RHS entry points.                                               */
/* ------------------------------------------------------------------ */
int orc_rhs(const orc_problem *pb, const double *tables, double k, double *out) {
  int st = check_problem(pb);
  if (st) return st;
  if (!(k > 0.0) || !tables || !out) return ORC_EINVAL;
  switch (pb->model) {
  case ORC_D3: return rhs_d3(pb, tables, NULL, k, out, NULL, NULL, 0);
  case ORC_D4_VERTEX:
  case ORC_D4_FULL: return rhs_d4(pb, tables, NULL, k, out, NULL, NULL, 0);
  case ORC_FINITE_T: return rhs_ft(pb, tables, k, out, NULL, 0);
  case ORC_FINITE_T_4D: return rhs_ft4(pb, tables, k, out, NULL, 0);
  }
  return ORC_EINVAL;
}

/* The same sums restricted to the external points sel[0..nsel-1]
 * (out[i] belongs to sel[i]); used to sample full-size problems. */
int orc_rhs_subset(const orc_problem *pb, const double *tables, double k, const int *sel, int nsel, double *out) {
  int st = check_problem(pb);
  if (st) return st;
  if (!(k > 0.0) || !tables || !out || !sel || nsel < 0) return ORC_EINVAL;
  int ne = orc_n_ext(pb);
  for (int i = 0; i < nsel; ++i)
    if (sel[i] < 0 || sel[i] >= ne) return ORC_EINVAL;
  switch (pb->model) {
  case ORC_D3: return rhs_d3(pb, tables, NULL, k, out, NULL, sel, nsel);
  case ORC_D4_VERTEX:
  case ORC_D4_FULL: return rhs_d4(pb, tables, NULL, k, out, NULL, sel, nsel);
  case ORC_FINITE_T: return rhs_ft(pb, tables, k, out, sel, nsel);
  case ORC_FINITE_T_4D: return rhs_ft4(pb, tables, k, out, sel, nsel);
  }
  return ORC_EINVAL;
}

/* Directional derivative of the RHS along a table perturbation dtables
 * (forward-mode AD).  out receives the RHS, dout the derivative. */
int orc_rhs_jvp(const orc_problem *pb, const double *tables, const double *dtables, double k, double *out,
                double *dout) {
  int st = check_problem(pb);
  if (st) return st;
  if (!(k > 0.0) || !tables || !dtables || !out || !dout) return ORC_EINVAL;
  switch (pb->model) {
  case ORC_D3: return rhs_d3(pb, tables, dtables, k, out, dout, NULL, 0);
  case ORC_D4_VERTEX: return rhs_d4(pb, tables, dtables, k, out, dout, NULL, 0);
  default: return ORC_EINVAL;
  }
}

/* Full Jacobian J[e][j] = d out_e / d table_j, one forward-mode sweep per
 * table entry j (row-major, n_ext x table_size). */
int orc_rhs_jacobian(const orc_problem *pb, const double *tables, double k, double *J) {
  int st = check_problem(pb);
  if (st) return st;
  int ne = orc_n_ext(pb);
  int nt = pb->n_tables * pb->n_stack * pb->n_pts;
  double *dt = calloc(nt, sizeof(double)), *o = malloc(sizeof(double) * ne), *d = malloc(sizeof(double) * ne);
  if (!dt || !o || !d) { free(dt); free(o); free(d); return ORC_ENOMEM; }
  for (int j = 0; j < nt; ++j) {
    dt[j] = 1.0;
    st = orc_rhs_jvp(pb, tables, dt, k, o, d);
    dt[j] = 0.0;
    if (st) break;
    for (int e = 0; e < ne; ++e) J[(size_t)e * nt + j] = d[e];
  }
  free(dt); free(o); free(d);
  return st;
}

/* ------------------------------------------------------------------ */
/* Flow in RG time t = t_+ = ln(Lambda/k) (Sec. 2.1): the variable        */
/* assembler's residual is Flow(lambda) = k d_k lambda, so                */
/* d_t y = -Flow (Sec. 5.2.2, Eqs. assVar and flowVar).                   */
/* ------------------------------------------------------------------ */
typedef struct {
  const orc_problem *pb;
  const double *tables;   /* frozen tables */
  double Lambda;
  int feedback;
  double *work_out;       /* n_ext */
  double *work_tab;       /* table_size */
  double *psi_x, *psi_w;  /* external-angle rule (d=4) */
  long rhs_evals;
} flow_ctx;

static int flow_deriv(flow_ctx *fc, double t, const double *y, double *dy, int ny) {
  const orc_problem *pb0 = fc->pb;
  double k = fc->Lambda * exp(-t);
  int st;
  fc->rhs_evals++;
  if (!fc->feedback) {
    st = orc_rhs(pb0, fc->tables, k, fc->work_out);
    if (st) return st;
    for (int i = 0; i < ny; ++i) dy[i] = -fc->work_out[i];
    return ORC_OK;
  }
  if (pb0->model == ORC_D3) {
    /* state (m^2, Z_0..Z_{n-1}); d_t m^2 = -I(0), d_t Z_i = -(I(p_i)-I(0))/p_i^2 */
    orc_problem pb = *pb0;
    int n = pb.n_pts;
    pb.m2_over_k2 = 0.0;
    pb.m2_shift = y[0];
    pb.include_p0 = 1;
    for (int i = 0; i < n; ++i) fc->work_tab[i] = y[1 + i];
    st = orc_rhs(&pb, fc->work_tab, k, fc->work_out);
    if (st) return st;
    double I0 = fc->work_out[n];
    dy[0] = -I0;
    for (int i = 0; i < n; ++i) {
      double p = ext_p(&pb, i);
      dy[1 + i] = -(fc->work_out[i] - I0) / (p * p);
    }
    return ORC_OK;
  }
  if (pb0->model == ORC_D4_VERTEX) {
    /* state = tables (Z, lambda3, lambda4);  d_t Z_i = -(D2(p_i) - D2(0))/p_i^2,
     * d_t lambda3_i = - sum_psi (w_psi/2) Flow3(p_i,psi),  d_t lambda4_i = -Flow4(p_i) */
    int n = pb0->n_pts, npsi = pb0->n_ext_ang;
    st = orc_rhs(pb0, y, k, fc->work_out);
    if (st) return st;
    const double *o = fc->work_out;
    double D0 = o[n];
    for (int i = 0; i < n; ++i) {
      double p = ext_p(pb0, i);
      dy[i] = -(o[i] - D0) / (p * p);
      acc_t a = {0, 0};
      for (int j = 0; j < npsi; ++j) acc_add(&a, 0.5 * fc->psi_w[j] * o[n + 1 + i * npsi + j]);
      dy[n + i] = -acc_get(&a);
      dy[2 * n + i] = -o[n + 1 + n * npsi + i];
    }
    return ORC_OK;
  }
  return ORC_EINVAL;
}

int orc_flow_state_size(const orc_problem *pb, int feedback) {
  if (!feedback) return orc_n_ext(pb);
  if (pb->model == ORC_D3) return 1 + pb->n_pts;
  if (pb->model == ORC_D4_VERTEX) return 3 * pb->n_pts;
  return -1;
}

/* Dormand-Prince 5(4) tableau (Dormand & Prince, J. Comput. Appl. Math. 6,
 * 1980), written from the published coefficients. */
static const double DP_C[7] = {0.0, 1.0 / 5, 3.0 / 10, 4.0 / 5, 8.0 / 9, 1.0, 1.0};
static const double DP_A[7][6] = {
    {0, 0, 0, 0, 0, 0},
    {1.0 / 5, 0, 0, 0, 0, 0},
    {3.0 / 40, 9.0 / 40, 0, 0, 0, 0},
    {44.0 / 45, -56.0 / 15, 32.0 / 9, 0, 0, 0},
    {19372.0 / 6561, -25360.0 / 2187, 64448.0 / 6561, -212.0 / 729, 0, 0},
    {9017.0 / 3168, -355.0 / 33, 46732.0 / 5247, 49.0 / 176, -5103.0 / 18656, 0},
    {35.0 / 384, 0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84}};
/* fifth-order weights (= last row of A, first-same-as-last) and the
 * embedded fourth-order weights */
static const double DP_B5[7] = {35.0 / 384, 0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84, 0};
static const double DP_B4[7] = {5179.0 / 57600, 0, 7571.0 / 16695, 393.0 / 640, -92097.0 / 339200, 187.0 / 2100,
                                1.0 / 40};

typedef int (*deriv_fn)(void *ctx, double t, const double *y, double *dy, int ny);

/* Adaptive DP5(4) over [t0, t1] (App. C "explicit" parameters: dt is the
 * initial step, [minimal_dt, maximal_dt] bound it, abort when stuck at
 * minimal_dt; abs_tol / rel_tol control the error).  Controller reading:
 *   err = max_i |y5_i - y4_i| / (atol + rtol max(|y_i|, |y5_i|))
 *   accept if err <= 1; factor = clamp(0.9 err^(-1/5), 0.2, 5) (5 if err = 0),
 *   factor <= 1 on the step after a rejection; next dt = clamp(h factor,
 *   dt_min, dt_max); the last step is shortened to hit t1.  A rejected step
 *   taken with h <= dt_min aborts (underflow). */
static int dp45_run(deriv_fn f, void *ctx, int ny, double *y, const orc_step_opts *o, long *n_steps,
                    long *n_rejects) {
  int st = ORC_OK;
  double *K = malloc(sizeof(double) * 7 * ny);
  double *ys = malloc(sizeof(double) * ny), *y5 = malloc(sizeof(double) * ny);
  if (!K || !ys || !y5) { free(K); free(ys); free(y5); return ORC_ENOMEM; }
  double t = o->t0, dt = o->dt0;
  long steps = 0, rejects = 0;
  int last_rejected = 0;
  if (dt > o->dt_max) dt = o->dt_max;
  if (dt < o->dt_min) dt = o->dt_min;
  st = f(ctx, t, y, K, ny);
  double span = fabs(o->t1 - o->t0);
  while (!st && o->t1 - t > 1e-13 * (span > 1.0 ? span : 1.0)) {
    if (steps + rejects >= o->max_steps) { st = ORC_EMAXSTEPS; break; }
    double h = dt;
    if (h > o->t1 - t) h = o->t1 - t;
    for (int s = 1; s < 7 && !st; ++s) {
      for (int i = 0; i < ny; ++i) {
        double v = y[i];
        for (int r = 0; r < s; ++r) v += h * DP_A[s][r] * K[r * ny + i];
        ys[i] = v;
      }
      if (s == 6) memcpy(y5, ys, sizeof(double) * ny);
      st = f(ctx, t + DP_C[s] * h, ys, K + s * ny, ny);
    }
    if (st) break;
    double err = 0.0;
    int finite = 1;
    for (int i = 0; i < ny; ++i) {
      double e = 0.0;
      for (int r = 0; r < 7; ++r) e += (DP_B5[r] - DP_B4[r]) * K[r * ny + i];
      e *= h;
      double sc = o->atol + o->rtol * fmax(fabs(y[i]), fabs(y5[i]));
      double ei = fabs(e) / sc;
      if (!isfinite(ei) || !isfinite(y5[i])) finite = 0;
      if (ei > err) err = ei;
    }
    if (!finite) { st = ORC_ENONFINITE; break; }
    if (err <= 1.0) {
      t += h;
      memcpy(y, y5, sizeof(double) * ny);
      memcpy(K, K + 6 * ny, sizeof(double) * ny);
      ++steps;
      double fac = (err == 0.0) ? 5.0 : 0.9 * pow(err, -0.2);
      if (fac > 5.0) fac = 5.0;
      if (fac < 0.2) fac = 0.2;
      if (last_rejected && fac > 1.0) fac = 1.0;
      last_rejected = 0;
      dt = h * fac;
    } else {
      ++rejects;
      if (h <= o->dt_min) { st = ORC_ESTEP_UNDERFLOW; break; }
      double fac = 0.9 * pow(err, -0.2);
      if (fac < 0.2) fac = 0.2;
      dt = h * fac;
      last_rejected = 1;
    }
    if (dt > o->dt_max) dt = o->dt_max;
    if (dt < o->dt_min) dt = o->dt_min;
  }
  *n_steps = steps;
  *n_rejects = rejects;
  free(K); free(ys); free(y5);
  return st;
}

static int flow_deriv_cb(void *ctx, double t, const double *y, double *dy, int ny) {
  return flow_deriv((flow_ctx *)ctx, t, y, dy, ny);
}

static int flow_ctx_init(flow_ctx *fc, const orc_problem *pb, const double *tables, int feedback, double Lambda) {
  fc->pb = pb;
  fc->tables = tables;
  fc->Lambda = Lambda;
  fc->feedback = feedback;
  fc->rhs_evals = 0;
  fc->work_out = malloc(sizeof(double) * (orc_n_ext(pb) + 1));
  fc->work_tab = malloc(sizeof(double) * (pb->n_tables * pb->n_stack * pb->n_pts + 1));
  int npsi = pb->n_ext_ang > 0 ? pb->n_ext_ang : 1;
  fc->psi_x = malloc(sizeof(double) * npsi);
  fc->psi_w = malloc(sizeof(double) * npsi);
  if (!fc->work_out || !fc->work_tab || !fc->psi_x || !fc->psi_w) return ORC_ENOMEM;
  orc_gauss_legendre(npsi, -1.0, 1.0, fc->psi_x, fc->psi_w);
  return ORC_OK;
}

static void flow_ctx_free(flow_ctx *fc) {
  free(fc->work_out); free(fc->work_tab); free(fc->psi_x); free(fc->psi_w);
}

/* Flow of the state y from t_+ = t0 to t1 with DP5(4).  y is overwritten. */
int orc_flow(const orc_problem *pb, const double *tables, int feedback, double Lambda, double *y,
             const orc_step_opts *o, orc_flow_stats *stats) {
  int st = check_problem(pb);
  if (st) return st;
  if (!o || !y || !(Lambda > 0.0) || !(o->t1 >= o->t0)) return ORC_EINVAL;
  int ny = orc_flow_state_size(pb, feedback);
  if (ny <= 0) return ORC_EINVAL;
  if (feedback && (pb->n_ext_p != pb->n_pts || pb->p_min != pb->x_min || pb->p_max != pb->x_max))
    return ORC_EINVAL;
  flow_ctx fc;
  st = flow_ctx_init(&fc, pb, tables, feedback, Lambda);
  long steps = 0, rejects = 0;
  if (!st) st = dp45_run(flow_deriv_cb, &fc, ny, y, o, &steps, &rejects);
  if (stats) {
    stats->steps = steps;
    stats->rejects = rejects;
    stats->rhs_evals = fc.rhs_evals;
  }
  flow_ctx_free(&fc);
  return st;
}

/* Textbook ODEs with closed-form solutions, integrated by the same DP5(4)
 * driver (pins the tableau and the controller independently of the fRG RHS):
 *   which = 0:  y' = y cos t            -> y = y0 exp(sin t)
 *   which = 1:  y' = -2 t y^2           -> y = 1/(1/y0 + t^2)
 *   which = 2:  y0' = y1, y1' = -y0     -> rotation (harmonic oscillator) */
static int textbook_cb(void *ctx, double t, const double *y, double *dy, int ny) {
  int which = *(int *)ctx;
  (void)ny;
  if (which == 0) dy[0] = y[0] * cos(t);
  else if (which == 1) dy[0] = -2.0 * t * y[0] * y[0];
  else { dy[0] = y[1]; dy[1] = -y[0]; }
  return ORC_OK;
}

int orc_dp45_textbook(int which, double *y, const orc_step_opts *o, orc_flow_stats *stats) {
  if (which < 0 || which > 2 || !y || !o) return ORC_EINVAL;
  long steps = 0, rejects = 0;
  int st = dp45_run(textbook_cb, &which, which == 2 ? 2 : 1, y, o, &steps, &rejects);
  if (stats) {
    stats->steps = steps;
    stats->rejects = rejects;
    stats->rhs_evals = 1 + 6 * (steps + rejects);
  }
  return st;
}

/* Time derivative of the flow state, exposed so tests can integrate it with
 * an independent quadrature/ODE method. */
int orc_flow_deriv(const orc_problem *pb, const double *tables, int feedback, double Lambda, double t,
                   const double *y, double *dy) {
  int st = check_problem(pb);
  if (st) return st;
  int ny = orc_flow_state_size(pb, feedback);
  if (ny <= 0) return ORC_EINVAL;
  flow_ctx fc;
  st = flow_ctx_init(&fc, pb, tables, feedback, Lambda);
  if (!st) st = flow_deriv(&fc, t, y, dy, ny);
  flow_ctx_free(&fc);
  return st;
}

/* Batched summand evaluation (plain loops) for brute-force pins that build
 * the loop momenta themselves (Monte Carlo, rotated frames). */
void orc_d3_summand_batch(const orc_problem *pb, const double *tab, double k, long n, const double *q2,
                          const double *s2, double *out) {
  for (long i = 0; i < n; ++i) out[i] = orc_d3_summand(pb, tab, k, q2[i], s2[i]);
}

void orc_d4_summand_batch(int block, const orc_problem *pb, const double *tab, double k, long n, const double *q2,
                          double p2, const double *A2, const double *B2, double C2, double *out) {
  for (long i = 0; i < n; ++i) {
    if (block == 0) out[i] = orc_d4_summand_z(pb, tab, k, q2[i], p2, A2[i]);
    else if (block == 1) out[i] = orc_d4_summand_3(pb, tab, k, q2[i], p2, A2[i], B2[i], C2);
    else out[i] = orc_d4_summand_4(pb, tab, k, q2[i], p2, A2[i]);
  }
}

/* ------------------------------------------------------------------ */
/* Linearly implicit (Rosenbrock) stepping.  ROS2 of Verwer, Spee, Blom  */
/* and Hundsdorfer (SIAM J. Sci. Comput. 20, 1999), written from its      */
/* published definition, gamma = 1 + 1/sqrt(2):                          */
/*   (I - gamma h J) k1 = f(t, y)                                          */
/*   (I - gamma h J) k2 = f(t + h, y + h k1) - 2 k1                        */
/*   y_new = y + h (3/2 k1 + 1/2 k2);  estimate y_new - (y + h k1).        */
/* Second order for any matrix J (W-method); L-stable with the exact J.    */
/* Step control as for DP5(4) with the exponent 1/2.                       */
/* ------------------------------------------------------------------ */
typedef int (*jac_fn)(void *ctx, double t, const double *y, double *J, int ny);

/* Solve A x = b in place (b -> x) by Gaussian elimination with partial
 * pivoting; A (row-major n x n) is overwritten. */
static int dense_solve(double *A, double *b, int n) {
  for (int k = 0; k < n; ++k) {
    int piv = k;
    for (int i = k + 1; i < n; ++i)
      if (fabs(A[(size_t)i * n + k]) > fabs(A[(size_t)piv * n + k])) piv = i;
    if (A[(size_t)piv * n + k] == 0.0) return ORC_ENONFINITE;
    if (piv != k) {
      for (int j = 0; j < n; ++j) {
        double t = A[(size_t)k * n + j];
        A[(size_t)k * n + j] = A[(size_t)piv * n + j];
        A[(size_t)piv * n + j] = t;
      }
      double t = b[k];
      b[k] = b[piv];
      b[piv] = t;
    }
    for (int i = k + 1; i < n; ++i) {
      double l = A[(size_t)i * n + k] / A[(size_t)k * n + k];
      for (int j = k; j < n; ++j) A[(size_t)i * n + j] -= l * A[(size_t)k * n + j];
      b[i] -= l * b[k];
    }
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = b[i];
    for (int j = i + 1; j < n; ++j) s -= A[(size_t)i * n + j] * b[j];
    b[i] = s / A[(size_t)i * n + i];
  }
  return ORC_OK;
}

static int ros2_run(deriv_fn f, jac_fn jf, void *ctx, int ny, double *y, const orc_step_opts *o, long *n_steps,
                    long *n_rejects, long *n_jac) {
  const double g = 1.0 + 1.0 / sqrt(2.0);
  size_t nn = (size_t)ny * ny;
  double *J = malloc(sizeof(double) * nn), *W = malloc(sizeof(double) * nn);
  double *f0 = malloc(sizeof(double) * ny), *k1 = malloc(sizeof(double) * ny), *k2 = malloc(sizeof(double) * ny);
  double *y1 = malloc(sizeof(double) * ny), *yn = malloc(sizeof(double) * ny);
  int st = (J && W && f0 && k1 && k2 && y1 && yn) ? ORC_OK : ORC_ENOMEM;
  double t = o->t0, dt = fmin(fmax(o->dt0, o->dt_min), o->dt_max);
  long steps = 0, rejects = 0, jacs = 0;
  int last_rejected = 0, have_jac = 0;
  double span = fabs(o->t1 - o->t0);
  if (!st) st = f(ctx, t, y, f0, ny);
  while (!st && o->t1 - t > 1e-13 * (span > 1.0 ? span : 1.0)) {
    if (steps + rejects >= o->max_steps) { st = ORC_EMAXSTEPS; break; }
    double h = dt < o->t1 - t ? dt : o->t1 - t;
    if (!have_jac) {
      st = jf(ctx, t, y, J, ny);
      if (st) break;
      ++jacs;
      have_jac = 1;
    }
    for (size_t q = 0; q < nn; ++q) W[q] = -g * h * J[q];
    for (int i = 0; i < ny; ++i) W[(size_t)i * ny + i] += 1.0;
    memcpy(k1, f0, sizeof(double) * ny);
    st = dense_solve(W, k1, ny);
    if (st) break;
    for (int i = 0; i < ny; ++i) y1[i] = y[i] + h * k1[i];
    st = f(ctx, t + h, y1, k2, ny);
    if (st) break;
    for (int i = 0; i < ny; ++i) k2[i] -= 2.0 * k1[i];
    for (size_t q = 0; q < nn; ++q) W[q] = -g * h * J[q];
    for (int i = 0; i < ny; ++i) W[(size_t)i * ny + i] += 1.0;
    st = dense_solve(W, k2, ny);
    if (st) break;
    double err = 0.0;
    int finite = 1;
    for (int i = 0; i < ny; ++i) {
      yn[i] = y[i] + h * (1.5 * k1[i] + 0.5 * k2[i]);
      double e = fabs(yn[i] - y1[i]) / (o->atol + o->rtol * fmax(fabs(y[i]), fabs(yn[i])));
      if (!isfinite(e)) finite = 0;
      if (e > err) err = e;
    }
    if (!finite) { st = ORC_ENONFINITE; break; }
    if (err <= 1.0) {
      t += h;
      memcpy(y, yn, sizeof(double) * ny);
      ++steps;
      st = f(ctx, t, y, f0, ny);
      have_jac = 0;
      double fac = (err == 0.0) ? 5.0 : 0.9 * pow(err, -0.5);
      if (fac > 5.0) fac = 5.0;
      if (fac < 0.2) fac = 0.2;
      if (last_rejected && fac > 1.0) fac = 1.0;
      last_rejected = 0;
      dt = h * fac;
    } else {
      ++rejects;
      if (h <= o->dt_min) { st = ORC_ESTEP_UNDERFLOW; break; }
      double fac = 0.9 * pow(err, -0.5);
      if (fac < 0.2) fac = 0.2;
      dt = h * fac;
      last_rejected = 1;
    }
    if (dt > o->dt_max) dt = o->dt_max;
    if (dt < o->dt_min) dt = o->dt_min;
  }
  *n_steps = steps;
  *n_rejects = rejects;
  *n_jac = jacs;
  free(J); free(W); free(f0); free(k1); free(k2); free(y1); free(yn);
  return st;
}

/* Textbook problems for the ROS2 driver (closed-form solutions):
 *   0: y' = y cos t, J = cos t                  -> y0 exp(sin t)
 *   1: y' = -2 t y^2, J = -4 t y                -> 1/(1/y0 + t^2)
 *   2: y0' = y1, y1' = -y0 (exact J)            -> rotation
 *   3: y' = -1e4 (y - cos t) - sin t, J = -1e4  -> cos t (stiff, y0 = 1)
 *   4: problem 2 with J := 0 (W-method: still second order) */
static int tb_f(void *ctx, double t, const double *y, double *dy, int ny) {
  int w = *(int *)ctx;
  (void)ny;
  if (w == 0) dy[0] = y[0] * cos(t);
  else if (w == 1) dy[0] = -2.0 * t * y[0] * y[0];
  else if (w == 3) dy[0] = -1e4 * (y[0] - cos(t)) - sin(t);
  else { dy[0] = y[1]; dy[1] = -y[0]; }
  return ORC_OK;
}

static int tb_j(void *ctx, double t, const double *y, double *J, int ny) {
  int w = *(int *)ctx;
  (void)ny;
  if (w == 0) J[0] = cos(t);
  else if (w == 1) J[0] = -4.0 * t * y[0];
  else if (w == 3) J[0] = -1e4;
  else if (w == 2) { J[0] = 0.0; J[1] = 1.0; J[2] = -1.0; J[3] = 0.0; }
  else { J[0] = J[1] = J[2] = J[3] = 0.0; }
  return ORC_OK;
}

int orc_ros2_textbook(int which, double *y, const orc_step_opts *o, orc_flow_stats *stats) {
  if (which < 0 || which > 4 || !y || !o) return ORC_EINVAL;
  long s = 0, r = 0, jn = 0;
  int ny = (which == 2 || which == 4) ? 2 : 1;
  int st = ros2_run(tb_f, tb_j, &which, ny, y, o, &s, &r, &jn);
  if (stats) {
    stats->steps = s;
    stats->rejects = r;
    stats->rhs_evals = jn;  /* Jacobian evaluations */
  }
  return st;
}

/* State Jacobian of the d=4 feedback flow: column j = map(d raw / d T_j),
 * with the map of flow_deriv (d_t Z_i = -(D2(p_i)-D2(0))/p_i^2, d_t lambda3_i =
 * -sum_psi (w/2) Flow3, d_t lambda4_i = -Flow4) applied to a raw derivative. */
static int d4_state_jac(void *ctxp, double t, const double *y, double *J, int ny) {
  flow_ctx *fc = (flow_ctx *)ctxp;
  const orc_problem *pb = fc->pb;
  int n = pb->n_pts, npsi = pb->n_ext_ang, ne = orc_n_ext(pb);
  double k = fc->Lambda * exp(-t);
  double *dt = calloc(ny, sizeof(double)), *o = malloc(sizeof(double) * ne), *d = malloc(sizeof(double) * ne);
  if (!dt || !o || !d) { free(dt); free(o); free(d); return ORC_ENOMEM; }
  int st = ORC_OK;
  for (int j = 0; j < ny && !st; ++j) {
    dt[j] = 1.0;
    st = orc_rhs_jvp(pb, y, dt, k, o, d);
    dt[j] = 0.0;
    for (int i = 0; i < n && !st; ++i) {
      double p = ext_p(pb, i);
      J[(size_t)i * ny + j] = -(d[i] - d[n]) / (p * p);
      acc_t a = {0, 0};
      for (int q = 0; q < npsi; ++q) acc_add(&a, 0.5 * fc->psi_w[q] * d[n + 1 + i * npsi + q]);
      J[(size_t)(n + i) * ny + j] = -acc_get(&a);
      J[(size_t)(2 * n + i) * ny + j] = -d[n + 1 + n * npsi + i];
    }
  }
  free(dt); free(o); free(d);
  return st;
}

/* The d=4 feedback state Jacobian at (t, y), row-major ny x ny, exposed so
 * tests can compare its columns with differences of the flow derivative. */
int orc_d4_state_jacobian(const orc_problem *pb, double Lambda, double t, const double *y, double *J) {
  int st = check_problem(pb);
  if (st) return st;
  if (pb->model != ORC_D4_VERTEX || !y || !J || !(Lambda > 0.0)) return ORC_EINVAL;
  int ny = orc_flow_state_size(pb, 1);
  flow_ctx fc;
  st = flow_ctx_init(&fc, pb, NULL, 1, Lambda);
  if (!st) st = d4_state_jac(&fc, t, y, J, ny);
  flow_ctx_free(&fc);
  return st;
}

/* ROS2 flow of the d=4 feedback state (the tables) with the exact state
 * Jacobian recomputed at every accepted step. */
int orc_ros2_flow(const orc_problem *pb, double Lambda, double *y, const orc_step_opts *o, orc_flow_stats *stats) {
  int st = check_problem(pb);
  if (st) return st;
  if (pb->model != ORC_D4_VERTEX || !o || !y || !(Lambda > 0.0)) return ORC_EINVAL;
  if (pb->n_ext_p != pb->n_pts || pb->p_min != pb->x_min || pb->p_max != pb->x_max) return ORC_EINVAL;
  int ny = orc_flow_state_size(pb, 1);
  flow_ctx fc;
  st = flow_ctx_init(&fc, pb, NULL, 1, Lambda);
  long s = 0, r = 0, jn = 0;
  if (!st) st = ros2_run(flow_deriv_cb, d4_state_jac, &fc, ny, y, o, &s, &r, &jn);
  if (stats) {
    stats->steps = s;
    stats->rejects = r;
    stats->rhs_evals = fc.rhs_evals;
  }
  flow_ctx_free(&fc);
  return st;
}

/* ------------------------------------------------------------------ */
/* Adams-Bashforth-Moulton multistep stepping (the paper's Boost_ABM,    */
/* Sec. 5.2.1), fixed step h = (t1 - t0)/n.  Order s (2..5): predictor    */
/* Adams-Bashforth with s back values, corrector Adams-Moulton of order s */
/* with the predicted value and s-1 back values, each followed by an      */
/* evaluation (PECE: two RHS per step).  The first s-1 steps are classical*/
/* fourth-order Runge-Kutta steps (the starting values).  Coefficients    */
/* are the standard Adams tables (e.g. Hairer, Norsett, Wanner, Solving   */
/* ODE I, Sec. III.1).                                                    */
/* ------------------------------------------------------------------ */
static const double abm_b[6][5] = {/* AB_s: weights of f_n, f_{n-1}, ... */
    {0}, {1.0},
    {3.0 / 2.0, -1.0 / 2.0},
    {23.0 / 12.0, -16.0 / 12.0, 5.0 / 12.0},
    {55.0 / 24.0, -59.0 / 24.0, 37.0 / 24.0, -9.0 / 24.0},
    {1901.0 / 720.0, -2774.0 / 720.0, 2616.0 / 720.0, -1274.0 / 720.0, 251.0 / 720.0}};
static const double abm_a[6][5] = {/* AM_s: weights of f_{n+1}, f_n, f_{n-1}, ... */
    {0}, {1.0},
    {1.0 / 2.0, 1.0 / 2.0},
    {5.0 / 12.0, 8.0 / 12.0, -1.0 / 12.0},
    {9.0 / 24.0, 19.0 / 24.0, -5.0 / 24.0, 1.0 / 24.0},
    {251.0 / 720.0, 646.0 / 720.0, -264.0 / 720.0, 106.0 / 720.0, -19.0 / 720.0}};

static int abm_run(deriv_fn f, void *ctx, int ny, double *y, double t0, double t1, long n, int order,
                   long *rhs_evals) {
  if (order < 2 || order > 5 || n < 1 || ny < 1) return ORC_EINVAL;
  const double h = (t1 - t0) / (double)n;
  /* F[j] = f at t_{m-j} (newest first) */
  double *F = malloc(sizeof(double) * ny * order), *yp = malloc(sizeof(double) * ny);
  double *k2 = malloc(sizeof(double) * ny), *k3 = malloc(sizeof(double) * ny), *k4 = malloc(sizeof(double) * ny);
  double *fp = malloc(sizeof(double) * ny);
  if (!F || !yp || !k2 || !k3 || !k4 || !fp) {
    free(F); free(yp); free(k2); free(k3); free(k4); free(fp);
    return ORC_ENOMEM;
  }
  long ev = 0;
  int st = f(ctx, t0, y, F, ny);
  ++ev;
  for (long m = 0; m < n && !st; ++m) {
    const double t = t0 + h * (double)m;
    if (m < order - 1) {
      /* classical RK4 from (t, y) with k1 = F[0] */
      for (int i = 0; i < ny; ++i) yp[i] = y[i] + 0.5 * h * F[i];
      st = f(ctx, t + 0.5 * h, yp, k2, ny);
      for (int i = 0; i < ny && !st; ++i) yp[i] = y[i] + 0.5 * h * k2[i];
      if (!st) st = f(ctx, t + 0.5 * h, yp, k3, ny);
      for (int i = 0; i < ny && !st; ++i) yp[i] = y[i] + h * k3[i];
      if (!st) st = f(ctx, t + h, yp, k4, ny);
      ev += 3;
      for (int i = 0; i < ny && !st; ++i) y[i] += h / 6.0 * (F[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
    } else {
      /* predict, evaluate, correct */
      for (int i = 0; i < ny; ++i) {
        double s = 0.0;
        for (int j = 0; j < order; ++j) s += abm_b[order][j] * F[(size_t)j * ny + i];
        yp[i] = y[i] + h * s;
      }
      st = f(ctx, t + h, yp, fp, ny);
      ++ev;
      for (int i = 0; i < ny && !st; ++i) {
        double s = abm_a[order][0] * fp[i];
        for (int j = 1; j < order; ++j) s += abm_a[order][j] * F[(size_t)(j - 1) * ny + i];
        y[i] += h * s;
      }
    }
    if (st) break;
    /* evaluate at the new point and push it as the newest back value */
    memmove(F + ny, F, sizeof(double) * ny * (order - 1));
    st = f(ctx, t + h, y, F, ny);
    ++ev;
    for (int i = 0; i < ny && !st; ++i)
      if (!isfinite(y[i])) st = ORC_ENONFINITE;
  }
  if (rhs_evals) *rhs_evals = ev;
  free(F); free(yp); free(k2); free(k3); free(k4); free(fp);
  return st;
}

/* ABM on the textbook ODEs of orc_dp45_textbook, plus
 *   which = 3:  y' = 4 t^3 (y = y0 + t^4; polynomial derivative of degree 3) */
static int textbook_abm_cb(void *ctx, double t, const double *y, double *dy, int ny) {
  if (*(int *)ctx == 3) {
    (void)y;
    (void)ny;
    dy[0] = 4.0 * t * t * t;
    return ORC_OK;
  }
  return textbook_cb(ctx, t, y, dy, ny);
}

int orc_abm_textbook(int which, int order, double t0, double t1, long n, double *y, long *rhs_evals) {
  if (which < 0 || which > 3 || !y) return ORC_EINVAL;
  return abm_run(textbook_abm_cb, &which, which == 2 ? 2 : 1, y, t0, t1, n, order, rhs_evals);
}

/* ABM flow of the state y from t_+ = t0 to t1 in n fixed steps. */
int orc_abm_flow(const orc_problem *pb, const double *tables, int feedback, double Lambda, double *y, double t0,
                 double t1, long n, int order, orc_flow_stats *stats) {
  int st = check_problem(pb);
  if (st) return st;
  if (!y || !(Lambda > 0.0) || !(t1 >= t0)) return ORC_EINVAL;
  int ny = orc_flow_state_size(pb, feedback);
  if (ny <= 0) return ORC_EINVAL;
  if (feedback && (pb->n_ext_p != pb->n_pts || pb->p_min != pb->x_min || pb->p_max != pb->x_max))
    return ORC_EINVAL;
  flow_ctx fc;
  st = flow_ctx_init(&fc, pb, tables, feedback, Lambda);
  long ev = 0;
  if (!st) st = abm_run(flow_deriv_cb, &fc, ny, y, t0, t1, n, order, &ev);
  if (stats) {
    stats->steps = n;
    stats->rejects = 0;
    stats->rhs_evals = fc.rhs_evals;
  }
  flow_ctx_free(&fc);
  return st;
}
