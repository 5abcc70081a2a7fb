/*
 * ffrg.h -- C ABI of the GB300 (sm_103a) library that evaluates the loop-
 * momentum integrals on the right-hand side of functional-RG vertex-expansion
 * flows and integrates those flows in RG time (DiFfRG, arXiv:2412.13043).
 *
 * The calls follow the paper's statement of the problem:
 *   - a per-flow integrator "get(k, args...)" that returns the momentum
 *     integral for a scale k (App. G, model code calling the integrators);
 *   - the variable assembler's residual dt_variables(residual, data), i.e.
 *     d_t v + R(v, t) = 0 with R = Flow (Sec. 5.2.2, Eqs. assVar, flowVar);
 *   - a stepper run(&ic, t0, t1) with dt / minimal_dt / maximal_dt / abs_tol /
 *     rel_tol semantics (Sec. 5.2.1 and App. C, "timestepping" parameters);
 *   - kernel descriptors with Type / Angles / d / ctype (Sec. 5.3.2, App. F).
 *
 * Conventions shared by every call:
 *   - Every call returns an ffrg_status; nothing throws across the ABI.
 *   - Pointers marked "device" must be device memory of the context's GPU;
 *     "host" pointers are ordinary host memory.  Caller-owned buffers are
 *     never retained after a call returns (serving copies its inputs).
 *   - Device work is ordered on the CUDA stream passed as `stream`
 *     (a cudaStream_t cast to void*, NULL = legacy default stream).  Calls
 *     that launch work return before it finishes; errors raised on the device
 *     (non-finite results, bounded-wait timeouts) accumulate in a per-context
 *     status word read by ffrg_status_read().
 *   - A context's scratch memory is shared by its calls: issue the calls of
 *     one context on one stream (or serialise them); use one context per
 *     concurrent stream.
 *   - RG time: ffrg_rhs returns k d_k of the target quantity (the literature
 *     convention t_- = ln(k/Lambda)); ffrg_flow integrates in
 *     t = t_+ = ln(Lambda/k), so d_t y = -Flow (Sec. 2.1, t_+ convention).
 *
 * Synthetic models (the paper's Yang-Mills and four-Fermi systems need input
 * data that is not published with it; these models keep the same structure
 * "regulator derivative x propagators x vertices from interpolated dressing
 * tables", Eq. GenfRG, Eq. FlowGamman, App. G):
 *   FFRG_MODEL_D3        d=3, T=0:  I(p) = pref lam^2 int d^3q/(2pi)^3
 *                                         dR(q) G(q)^2 G(|q+p|)
 *   FFRG_MODEL_D4_VERTEX d=4, T=0, tables Z, lambda3, lambda4 (Sec. 3.3
 *                        average-momentum vertices): propagator, three- and
 *                        four-point diagrams
 *   FFRG_MODEL_FINITE_T  d=3 + bosonic Matsubara sum |n| <= N (Sec. 5.3.2
 *                        "Quadratureq0"), tables stacked over |n|
 * with R = Z(q) k^2 r(q^2/k^2), r(x) = x/(e^x-1) (exponential) or
 * (1-x)Theta(1-x) (flat), dR = k d_k R at fixed Z, and
 * G = 1/(Z (omega^2 + q^2) + m^2 + R), m^2 = m2_over_k2 k^2 + m2_shift.
 */
#ifndef FFRG_H
#define FFRG_H

#include <stddef.h>

#if defined(__GNUC__)
#define FFRG_API __attribute__((visibility("default")))
#else
#define FFRG_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ffrg_ctx ffrg_ctx;       /* library-owned; one per device and stream */
typedef struct ffrg_tables ffrg_tables; /* library-owned device dressing tables */

typedef enum {
  FFRG_OK = 0,
  FFRG_EINVAL = 1,          /* bad argument, shape or pointer */
  FFRG_ENOMEM = 2,          /* allocation failed or the context's HBM budget is exceeded */
  FFRG_ENONFINITE = 3,      /* a result or flow state became NaN/Inf */
  FFRG_ESTEP_UNDERFLOW = 4, /* step rejected at minimal_dt (App. C: evolution aborted) */
  FFRG_EMAXSTEPS = 5,       /* step budget exhausted before t1 */
  FFRG_ETIMEOUT = 6,        /* a bounded device wait gave up */
  FFRG_EPENDING = 7,        /* serving: request not finished yet */
  FFRG_EBUSY = 8,           /* serving: queue full */
  FFRG_ECUDA = 9,           /* a CUDA runtime call failed (see ffrg_last_error) */
  FFRG_ENOTFOUND = 10,      /* serving: unknown ticket */
  FFRG_ECANCELED = 11       /* serving: request cancelled before it finished */
} ffrg_status;

typedef enum { FFRG_FP64 = 0, FFRG_MIXED = 1 } ffrg_precision;
typedef enum { FFRG_RULE_GL = 0, FFRG_RULE_GC2 = 1 } ffrg_rule;
typedef enum {
  FFRG_MODEL_D3 = 1,
  FFRG_MODEL_D4_VERTEX = 2,
  FFRG_MODEL_FINITE_T = 3,
  FFRG_MODEL_D4_FULL = 4,
  FFRG_MODEL_FINITE_T_4D = 5
} ffrg_model;
typedef enum { FFRG_REG_EXP = 0, FFRG_REG_LITIM = 1 } ffrg_regulator;
typedef enum { FFRG_STAT_BOSE = 0, FFRG_STAT_FERMI = 1 } ffrg_statistics;

/* One right-hand-side problem (kernel descriptor: Type/Angles/d of App. F).
 * Quadrature: radial Gauss-Legendre with n_rad nodes on [0, qmax_over_k k];
 * D3/FINITE_T: n_ang1 GL nodes in cos(theta); D4: n_ang1 Gauss-Chebyshev-II
 * nodes in cos1 (weight sqrt(1-c1^2)) x n_ang2 GL nodes in cos2 (App. F angle
 * names).  External momenta p_i = p_min (p_max/p_min)^(i/(n_ext_p-1)).
 * External-point layout of the output (row-major):
 *   D3:       [p_0 .. p_{n_ext_p-1}] then, if include_p0, the point p = 0
 *   D4:       [Z: p_0..p_{n-1}, p=0][lambda3: p_i x psi_j][lambda4: p_i],
 *             psi_j = n_ext_ang GL nodes in cos(psi) between the two legs
 *   D4_FULL:  as D4; the three-point vertex is tabulated on (S0, a, b) (the
 *             "Full" vertex dependence of Sec. 3.3): for a vertex with legs
 *             k1, k2, k3 (sum 0), S0^2 = (k1^2+k2^2+k3^2)/3, a = cosine
 *             between k1 and k2, b = (k1^2-k2^2)/(k1^2+k2^2); n_va x n_vb
 *             uniform nodes on [-1, 1] in a and b, interpolated linearly in
 *             ln S0, a and b.  Tables: n_tables = 3, n_stack = n_va n_vb;
 *             Z and lambda4 in row 0 of tables 0 and 2 (other rows unused),
 *             lambda3 at (a_i, b_j) in row i n_vb + j of table 1.
 *   FINITE_T: [p_i][m], m = 0..n_ext_ang-1 external bosonic frequencies
 *             p0_m = 2 pi T m; Matsubara sum of the loop over
 *             statistics FFRG_STAT_BOSE: omega_n = 2 pi T n, |n| <= n_matsubara
 *             (2N+1 terms), tables stacked over |n|;
 *             statistics FFRG_STAT_FERMI: nu_n = (2n+1) pi T, -N-1 <= n <= N
 *             (2N+2 terms), tables stacked over j = n (n >= 0) or -n-1, row j
 *             at nu_j = (2j+1) pi T (App. F bosonic / fermionic finite-T
 *             coordinate stacks).  The shifted line carries frequency n+m.
 *             Stack indices beyond n_stack-1 are clamped to it.
 *   FINITE_T_4D: [p_i][m] as FINITE_T; finite T with a 4-dimensional
 *             regulator on a frequency domain that scales with k (Sec. 5.3.2
 *             "Quadraturex0"): with Q = (q0, q), P = (p0, p),
 *               I = pref lam^2 [T sum_n | int dq0/(2 pi)] int d^3q/(2pi)^3
 *                   dR(Q) G(Q)^2 L(|Q|) L(|Q+P|) G(Q+P),
 *             R(Q) = Z(|Q|) k^2 r(|Q|^2/k^2), G(Q) = 1/(Z(|Q|)|Q|^2 + m^2
 *             + R(Q)); tables Z and L (n_tables = 2, n_stack = 1) on one log
 *             grid in |Q|.  Loop frequencies in |q0| <= qmax_over_k k:
 *             bosonic 2 pi T n, fermionic (statistics FFRG_STAT_FERMI)
 *             (2n+1) pi T.  While at most 2 n_matsubara + 1 (+1 fermionic)
 *             of them lie in the domain, the frequency integral is their
 *             Matsubara sum (weight T); beyond that, n_x0 Gauss-Legendre
 *             nodes on [-qmax_over_k k, qmax_over_k k] (weights / 2 pi), the
 *             T -> 0 form.  External frequency p0: bosonic 2 pi T m; with
 *             fermionic statistics the external fermion leg's
 *             p0f = pi T exp(-k/(pi T)) (App. G; n_ext_ang = 1). */
typedef struct {
  int model;        /* ffrg_model */
  int regulator;    /* ffrg_regulator */
  int n_rad, n_ang1, n_ang2;
  int n_ext_p, n_ext_ang, n_matsubara, include_p0;
  int statistics;   /* ffrg_statistics of the loop frequencies (FINITE_T; 0 otherwise) */
  double m2_over_k2, m2_shift; /* m^2 = m2_over_k2 k^2 + m2_shift */
  double lam;                  /* coupling: lam^2 multiplies D3 and FINITE_T */
  double T;                    /* temperature (FINITE_T) */
  double p_min, p_max;         /* external log grid */
  double qmax_over_k;          /* radial domain [0, qmax_over_k k] */
  double prefactor;            /* overall multiplier */
  int n_va, n_vb;              /* D4_FULL: vertex nodes in a and b (1 otherwise) */
  int n_x0;                    /* FINITE_T_4D: frequency quadrature nodes (0 otherwise) */
} ffrg_problem;

/* Dressing tables values[table][stack][pt] (doubles, row-major) on the log grid
 * x_j = x_min (x_max/x_min)^(j/(n_pts-1)) (App. F LogarithmicCoordinates1D);
 * stack = |n| for FINITE_T (App. F BosonicCoordinates1DFiniteT), clamped to
 * n_stack-1; lookups are linear in the value between nodes in ln s and clamp
 * at both ends.  D3 needs 1 table (Z), D4 3 (Z, lambda3, lambda4), FINITE_T 2
 * (Z, lam).  n_pts in [2, 4096]. */
typedef struct {
  int n_tables, n_stack, n_pts, reserved0;
  double x_min, x_max;
} ffrg_table_desc;

/* App. C explicit time-stepping parameters (t in t_+). */
typedef struct {
  double t0, t1;          /* integrate from t0 to t1 >= t0 */
  double dt0;             /* initial step ("dt") */
  double dt_min, dt_max;  /* "minimal_dt", "maximal_dt" */
  double atol, rtol;      /* "abs_tol", "rel_tol" */
  long long max_steps;    /* accepted + rejected attempts */
} ffrg_step_opts;

typedef struct {
  long long steps, rejects, rhs_evals;
  double integrand_evals; /* rhs_evals x (external points x quadrature nodes) */
  double t_reached;
  long long jac_evals;    /* Jacobian evaluations (Rosenbrock flows) */
} ffrg_flow_stats;

/* Create a context on CUDA device `device`.  hbm_budget_bytes caps the
 * library's own device allocations (0 = no cap).  Owns *out until destroy.
 * Errors: FFRG_EINVAL (NULL out, bad device), FFRG_ECUDA. */
FFRG_API int ffrg_create(ffrg_ctx **out, int device, size_t hbm_budget_bytes);
/* Release a context: stops its server (requests finish FFRG_ECANCELED),
 * waits for the device and frees every library-owned buffer, including
 * tables not yet freed.  ctx is invalid afterwards.  FFRG_EINVAL for NULL. */
FFRG_API int ffrg_destroy(ffrg_ctx *ctx);

/* Quadrature rule on the host (Sec. 5.3.2 "quadrature rules of arbitrary
 * order").  FFRG_RULE_GL: Gauss-Legendre on [a,b], ascending nodes.
 * FFRG_RULE_GC2: Gauss-Chebyshev of the second kind on [-1,1] for the weight
 * sqrt(1-x^2) (a, b ignored).  x, w: caller-owned host arrays of n doubles.
 * Errors: FFRG_EINVAL for n < 1 or n > 65536 or NULL arrays. */
FFRG_API int ffrg_quad_nodes(int rule, int n, double a, double b, double *x, double *w);

/* Upload dressing tables (App. F interpolator objects).  values: n_tables x
 * n_stack x n_pts doubles, host memory (values_on_device = 0) or device memory
 * (1); copied, not retained.  *out is library-owned until ffrg_tables_free.
 * Errors: FFRG_EINVAL (shape), FFRG_ENOMEM (budget). */
FFRG_API int ffrg_tables_upload(ffrg_ctx *ctx, const ffrg_table_desc *desc, const double *values, int values_on_device,
                       ffrg_tables **out, void *stream);
/* Overwrite the values of existing tables (same shape, host or device
 * source as for upload), stream-ordered on `stream`; a host source must stay
 * valid until the copy has run (pinned memory: until the stream reaches it).
 * Errors: FFRG_EINVAL (NULL arguments), FFRG_ECUDA. */
FFRG_API int ffrg_tables_update(ffrg_ctx *ctx, ffrg_tables *tables, const double *values, int values_on_device,
                       void *stream);
/* Free tables (after the work that reads them).  FFRG_EINVAL for NULL. */
FFRG_API int ffrg_tables_free(ffrg_ctx *ctx, ffrg_tables *tables);
/* Device pointer to the FP64 table values (library-owned, for zero-copy use). */
FFRG_API int ffrg_tables_device_ptr(const ffrg_tables *tables, double **dev_values);

/* Number of external points (output length) and integrand evaluations
 * (external points x quadrature nodes) of one RHS; -1 / <0 on a bad problem. */
FFRG_API int ffrg_n_ext(const ffrg_problem *pb);
FFRG_API double ffrg_evals(const ffrg_problem *pb);

/* One right-hand side at scale k (Eq. GenfRG projected onto the truncation,
 * Eq. FlowGamman): out_dev[e] = k d_k of the target at external point e (raw
 * loop integrals; the D4 Z-block holds the propagator-diagram sum D2(p), see
 * the layout above).  out_dev: caller-owned device array of ffrg_n_ext()
 * doubles.  precision: FFRG_FP64 (all arithmetic FP64) or FFRG_MIXED (FP32
 * integrand and row sums, compensated FP32 accumulation within a work item
 * rounded once to FP64, FP64 across work items, FP64 per-radial-node
 * factors, FP64 propagator near the pole).  Asynchronous; non-finite outputs
 * set FFRG_ENONFINITE in the status word.  The kernels stage the tables and
 * rules in the 227 KB of shared memory of a block; FP64 tables that do not fit
 * (8 bytes per value) are read in place from global memory (L2) instead.
 * Errors: FFRG_EINVAL for a bad problem, tables of another shape, or, in mixed
 * precision, FP32 tables and rules that do not fit in shared memory (8 bytes
 * per table node: one FP32 line-form pair, or the (Z, lambda) pair of finite
 * T, plus the angle rules; FFRG_MODEL_D4_FULL keeps lambda3 as 32-byte cell
 * polynomials where those fit and as line-form pairs otherwise); FFRG_ENOMEM
 * (budget); FFRG_ECUDA. */
FFRG_API int ffrg_rhs(ffrg_ctx *ctx, const ffrg_problem *pb, const ffrg_tables *tables, double k, double *out_dev,
             int precision, void *stream);

/* ffrg_rhs with the outputs in host memory.  out_host: caller-owned host
 * memory of ffrg_n_ext() doubles.  Pinned memory mapped into the device
 * address space (cudaHostAlloc / cudaMallocHost / cudaHostRegister with
 * unified addressing): the kernels write the outputs into it directly and the
 * call returns before they have run (synchronise `stream` before reading).
 * Other host memory: the RHS into a device buffer of the context (allocated
 * on the first call, grown when a larger problem needs it, freed by
 * ffrg_destroy), then a copy to out_host that has completed when the call
 * returns.  Calls of one context on different streams share the device
 * buffer: order them.
 * Errors: as ffrg_rhs; FFRG_EINVAL for a NULL out_host. */
FFRG_API int ffrg_rhs_host(ffrg_ctx *ctx, const ffrg_problem *pb, const ffrg_tables *tables, double k,
                  double *out_host, int precision, void *stream);

/* ffrg_rhs for callers that cannot allocate device memory.  The paper has no
 * counterpart; this is a deployment variant.  It suits, for example, a process
 * whose HBM is already reserved by another allocator (a framework's caching
 * pool), and a latency-critical loop where cudaMalloc/cudaFree would stall
 * other streams.  It computes exactly what ffrg_rhs computes with the same
 * kernels, but needs no context and calls no cudaMalloc, cudaFree or other
 * allocating routine.  Its scratch is one fixed 4 MiB device array inside
 * this library.  Every GPU that loads the library holds that array until the
 * process exits.
 *   pb, desc: problem and table layout (as for ffrg_rhs / ffrg_tables_upload);
 *   tables_dev: caller-owned device array of n_tables x n_stack x n_pts
 *   doubles; out_dev: caller-owned device array of ffrg_n_ext(pb) doubles;
 *   k, precision, stream: as for ffrg_rhs.  Runs on the current CUDA device.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.  A
 * call whose kernels need more dynamic shared memory than any earlier call's
 * on that device also raises the kernels' limit (cudaFuncSetAttribute).  Each
 * call copies its quadrature rules from host memory into the array, ordered
 * on `stream`.  All calls share the one array, which keeps the last call's
 * contents.  Calls whose work overlaps on the GPU (other streams, other host
 * threads) race on it: serialise them.  Errors: FFRG_EINVAL for bad arguments
 * and for problems whose scratch exceeds 4 MiB (quadrature rules + (2N+1)
 * n_rad factors + n_ext x chunk partials + the FP32 table copy, about 460 000
 * doubles); FFRG_ECUDA on a CUDA error.  There is no status word to read:
 * device-side errors show in out_dev.  Non-finite results stay non-finite,
 * and if a bounded device wait gave up (what ffrg_rhs reports as
 * FFRG_ETIMEOUT) every entry of out_dev is NaN. */
FFRG_API int ffrg_rhs_noalloc(const ffrg_problem *pb, const ffrg_table_desc *desc, const double *tables_dev, double k,
                              double *out_dev, int precision, void *stream);

/* Finite-T sums of many loop-side states against one angle-integrated
 * kernel (Sec. 5.3.2 momentum integrals).  The finite-T RHS is a sum over the
 * loop frequencies n and radial nodes q_r of a loop-side factor F(n, q_r)
 * (for the model: dR G^2 lam at (omega_n, q_r)) times the angular sum of
 * the shifted line, K[j(n+m)][p][r] = sum_c v_c lam G(n+m, |q_r + p|).  For
 * n_states states F_s sharing the tables, this call builds K once and returns
 *   out_dev[s * n_ext + e] = norm sum_{n, r} w_r q_r^2 F_s(n, r) K[j(n+m)][p][r]
 * with e = (p, m) as in ffrg_rhs, norm = prefactor lam^2 T / (4 pi^2) and the
 * radial rule (w_r, q_r) of the problem; with F_s = the model's factor it is
 * ffrg_rhs.  F_dev: device, n_states x nfreq x n_rad doubles, row n - n_lo
 * (n_lo = -N bosonic, -N-1 fermionic; nfreq = 2N+1 or 2N+2), the values at
 * the nodes without quadrature weights.  out_dev: device, n_states x n_ext
 * doubles.  precision: the arithmetic of K (FFRG_FP64 or FFRG_MIXED as for
 * ffrg_rhs); the contraction over (n, r) runs on the tensor cores and is
 * FP64-faithful in both: an Ozaki-type split of K and of the states into ten
 * 5-bit fixed-point slices carried in BF16, slice products summed exactly in
 * FP32 over at most 16384 (n, r) terms per pass, passes combined in FP64
 * (error below ~1e-14 of the sum of the terms' magnitudes).  Scratch is kept
 * by the context (slices of both operands and the exact pass sums:
 * about 20 (n_ext + n_states) nfreq n_rad + 220 n_ext n_states bytes).
 * Asynchronous.  FFRG_EINVAL for models other than FFRG_MODEL_FINITE_T and
 * for more than 196608 (loop frequency, radial node) terms. */
FFRG_API int ffrg_ft_states(ffrg_ctx *ctx, const ffrg_problem *pb, const ffrg_tables *tables, double k, int n_states,
                            const double *F_dev, double *out_dev, int precision, void *stream);

/* Vector-Jacobian product of ffrg_rhs with respect to the table values
 * (the paper forms Jacobians by forward-mode AD, Sec. 5.2.2; this is the
 * reverse-mode counterpart): tbar_dev[j] = sum_e gbar_dev[e] d out_e / d T_j,
 * j over all n_tables x n_stack x n_pts values.  gbar_dev: device, ffrg_n_ext
 * doubles; tbar_dev: device, overwritten.  Models FFRG_MODEL_D3 and
 * FFRG_MODEL_D4_VERTEX, precision FFRG_FP64 (FFRG_EINVAL otherwise), tables
 * up to ~2400 values.  Reproducible run to run on a given GPU (fixed
 * reduction order, no floating-point atomics). */
FFRG_API int ffrg_rhs_adjoint(ffrg_ctx *ctx, const ffrg_problem *pb, const ffrg_tables *tables, double k,
                     const double *gbar_dev, double *tbar_dev, int precision, void *stream);

/* Flow of a state vector in RG time t_+ with an adaptive Dormand-Prince 5(4)
 * stepper whose stage combination, error norm and step control run on the
 * device in FP64 (Sec. 5.2.1 explicit RK45 stepper; App. C parameters; abort
 * below minimal_dt).  State layouts (state_dev, device, in: y(t0), out: y(t1)):
 *   feedback = 0 (frozen tables, any model): y_e, d_t y_e = -out_e
 *   feedback = 1, D3: [m^2, Z_0..Z_{n-1}]; tables := Z, m^2 := y_0;
 *       d_t m^2 = -I(0), d_t Z_i = -(I(p_i) - I(0)) / p_i^2
 *   feedback = 1, D4: [Z, lambda3, lambda4] (3 n values) = the tables;
 *       d_t Z_i = -(D2(p_i) - D2(0))/p_i^2, d_t lambda3_i = -sum_j (w_j/2)
 *       Flow3(p_i, psi_j), d_t lambda4_i = -Flow4(p_i)
 * Feedback requires the external grid to equal the table grid.  k(t) = Lambda
 * exp(-t).  tables: frozen tables (feedback = 0) or the grid/shape template
 * (feedback = 1).  Synchronous: returns when the flow ends; stats (host) may be
 * NULL.  Errors: FFRG_ESTEP_UNDERFLOW, FFRG_EMAXSTEPS, FFRG_ENONFINITE. */
FFRG_API int ffrg_flow(ffrg_ctx *ctx, const ffrg_problem *pb, const ffrg_tables *tables, int feedback, double Lambda,
              double *state_dev, const ffrg_step_opts *opts, int precision, ffrg_flow_stats *stats,
              void *stream);
/* Full Jacobian of ffrg_rhs with respect to the table values (one pass of the
 * reverse-mode kernels with a gradient row per external point; Sec. 5.2.2
 * "jacobian_variables" counterpart): J_dev[e * T + j] = d out_e / d T_j,
 * T = n_tables x n_stack x n_pts, device, row-major, overwritten.  Models D3
 * and D4_VERTEX, FP64, tables up to ~2400 values.  Asynchronous. */
FFRG_API int ffrg_rhs_jacobian(ffrg_ctx *ctx, const ffrg_problem *pb, const ffrg_tables *tables, double k,
                               double *J_dev, void *stream);

/* Adams-Bashforth-Moulton flow (the paper's Boost_ABM explicit multistep
 * option, Sec. 5.2.1): n_steps fixed steps h = (t1 - t0)/n_steps in t_+ from
 * state_dev (overwritten with y(t1)); state, feedback modes, Lambda and
 * precision as for ffrg_flow.  order 2..5: PECE with the order-`order`
 * Adams-Bashforth predictor and Adams-Moulton corrector (two RHS per step);
 * the first order-1 steps are classical fourth-order Runge-Kutta steps.  No
 * error control: the caller chooses n_steps.  stats: steps = n_steps,
 * rhs_evals, t_reached; status FFRG_ENONFINITE if the state became NaN/Inf.
 * Synchronous. */
FFRG_API int ffrg_abm_flow(ffrg_ctx *ctx, const ffrg_problem *pb, const ffrg_tables *tables, int feedback,
                           double Lambda, double *state_dev, double t0, double t1, long long n_steps, int order,
                           int precision, ffrg_flow_stats *stats, void *stream);

/* Linearly implicit flow of the d=4 feedback state (the three tables, as for
 * ffrg_flow with feedback = 1) with ROS2 (Verwer, Spee, Blom, Hundsdorfer
 * 1999; the paper's implicit steppers use Jacobians, Sec. 5.2.1 / 5.2.2):
 * W = I - gamma h J, gamma = 1 + 1/sqrt(2), J = d(d_t y)/dy from
 * ffrg_rhs_jacobian; error estimate from the embedded first-order solution,
 * step-size exponent 1/2; FP64 throughout.  Synchronous; state_dev as for
 * ffrg_flow; stats->jac_evals counts Jacobians.  3 n_pts <= 4096. */
FFRG_API int ffrg_rosenbrock_flow(ffrg_ctx *ctx, const ffrg_problem *pb, const ffrg_tables *tables, double Lambda,
                                  double *state_dev, const ffrg_step_opts *opts, ffrg_flow_stats *stats, void *stream);

/* Length of the flow state for (pb, feedback); -1 on a bad combination. */
FFRG_API int ffrg_flow_state_size(const ffrg_problem *pb, const ffrg_table_desc *desc, int feedback);

/* Kernel timing for benchmarks: while enabled, every ffrg_rhs call records a
 * CUDA event pair around its main (integrand) kernel on the call's stream (up
 * to 4096 pairs).  ffrg_profile_read synchronises those events and returns the
 * summed main-kernel time in milliseconds and the number of launches, then
 * clears the record.  Enabling clears it too.  The main kernel is otherwise
 * launched so that it may start while the kernel before it (per-radial
 * factors, FP32 tables) is still running; the event between the two holds
 * it back, so a call takes slightly longer while profiling is enabled. */
FFRG_API int ffrg_set_profiling(ffrg_ctx *ctx, int enable);
FFRG_API int ffrg_profile_read(ffrg_ctx *ctx, double *main_ms, long long *launches);

/* ---- Serving: continuous batching of flow requests (one GPU) ----
 * A scheduler thread keeps up to max_slots flows resident on the device
 * (tables, DP5(4) state and RHS scratch of each), advances all of them one
 * adaptive step per tick with batched launches (one persistent integrand
 * launch per model over every resident flow's work items), retires finished
 * flows and admits queued requests as soon as a slot and enough of
 * hbm_budget_bytes are free.  Requests: frozen-background flows
 * (feedback = 0) of FFRG_MODEL_D3 and FFRG_MODEL_FINITE_T, mixed precision
 * (FP32 integrand, FP64 accumulation and step control).  A flow's result does
 * not depend on which other flows share its launches. */
typedef struct {
  int max_slots;            /* resident flows at once, 1..256 */
  int max_queue;            /* queued requests before submit returns FFRG_EBUSY */
  size_t hbm_budget_bytes;  /* device memory for resident flows (0: 1 GiB), reserved
                               by ffrg_serve_start; slot buffers are carved from it
                               on the host, so admission never calls a device allocator */
} ffrg_serve_opts;

typedef struct {
  long long submitted, admitted, completed, cancelled, rejected;
  long long ticks;          /* batched steps completed */
  int resident, queued, peak_resident, reserved0;
  size_t hbm_in_use;        /* bytes held by resident slots */
} ffrg_serve_stats;

/* Start the server of a context (one per context).  FFRG_EBUSY if running. */
FFRG_API int ffrg_serve_start(ffrg_ctx *ctx, const ffrg_serve_opts *opts);
/* Queue one flow request; inputs are copied (host pointers): tables_host
 * (desc layout), y0_host (ffrg_n_ext doubles), Lambda and the step options
 * (t in t_+).  *ticket identifies it.  FFRG_EBUSY: queue full; FFRG_ENOMEM:
 * the request alone exceeds the HBM budget; FFRG_EINVAL: unsupported request. */
FFRG_API int ffrg_serve_submit(ffrg_ctx *ctx, const ffrg_problem *pb, const ffrg_table_desc *desc,
                               const double *tables_host, const double *y0_host, double Lambda,
                               const ffrg_step_opts *opts, unsigned long long *ticket);
/* FFRG_EPENDING while queued or resident.  When finished: the flow's status
 * (FFRG_OK, FFRG_ESTEP_UNDERFLOW, FFRG_EMAXSTEPS, FFRG_ENONFINITE or
 * FFRG_ECANCELED), result_host (ffrg_n_ext doubles, may be NULL), stats and
 * latency_s (submit to completion, may be NULL) are filled and the ticket is
 * released.  FFRG_ENOTFOUND for unknown tickets. */
FFRG_API int ffrg_serve_poll(ffrg_ctx *ctx, unsigned long long ticket, double *result_host, ffrg_flow_stats *stats,
                             double *latency_s);
/* Cancel a queued or resident request (it finishes with FFRG_ECANCELED). */
FFRG_API int ffrg_serve_cancel(ffrg_ctx *ctx, unsigned long long ticket);
/* Counters of the running server (host copy).  FFRG_EINVAL without a server. */
FFRG_API int ffrg_serve_get_stats(ffrg_ctx *ctx, ffrg_serve_stats *out);
/* Stop the scheduler: resident and queued requests finish with FFRG_ECANCELED. */
FFRG_API int ffrg_serve_stop(ffrg_ctx *ctx);

/* Wait for the stream and return (then clear) the device status word:
 * FFRG_OK, FFRG_ENONFINITE or FFRG_ETIMEOUT; FFRG_ECUDA on a CUDA error. */
FFRG_API int ffrg_status_read(ffrg_ctx *ctx, void *stream);

/* Text for a status code; the last CUDA error text of a context. */
FFRG_API const char *ffrg_strerror(int status);
FFRG_API const char *ffrg_last_error(const ffrg_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* FFRG_H */
