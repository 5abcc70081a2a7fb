// Device-resident adaptive Dormand-Prince 5(4) flow in RG time t = t_+ =
// ln(Lambda/k) (Sec. 2.1), with the variable-assembler residual d_t y = -Flow
// (Sec. 5.2.2, Eqs. assVar / flowVar) and the explicit-stepper parameters dt,
// minimal_dt, maximal_dt, abs_tol, rel_tol (Sec. 5.2.1 RK45, App. C).
//
// One step = six stages of [stage state -> RHS (precompute / main, finite T
// also the contraction) -> derivative map], then one single-CTA control kernel that forms the FP64
// error norm, accepts or rejects, updates the step size and decides the next
// step (or that the flow is done).  All of it reads its scalars (t, h, k, m^2,
// done) from a device control block, so one step is captured once into a CUDA
// graph and relaunched; the host looks at the done flag only every few steps.
// Launches after the flow has finished return at once (skip flag).
#include <math.h>

#include <algorithm>

#include "ffrg_internal.cuh"

namespace ffrg {

// Dormand & Prince (1980) coefficients, from the published tableau.
__constant__ double kDpC[7] = {0.0, 0.2, 0.3, 0.8, 8.0 / 9.0, 1.0, 1.0};
__constant__ double kDpA[7][6] = {
    {0.0, 0.0, 0.0, 0.0, 0.0, 0.0},
    {0.2, 0.0, 0.0, 0.0, 0.0, 0.0},
    {3.0 / 40.0, 9.0 / 40.0, 0.0, 0.0, 0.0, 0.0},
    {44.0 / 45.0, -56.0 / 15.0, 32.0 / 9.0, 0.0, 0.0, 0.0},
    {19372.0 / 6561.0, -25360.0 / 2187.0, 64448.0 / 6561.0, -212.0 / 729.0, 0.0, 0.0},
    {9017.0 / 3168.0, -355.0 / 33.0, 46732.0 / 5247.0, 49.0 / 176.0, -5103.0 / 18656.0, 0.0},
    {35.0 / 384.0, 0.0, 500.0 / 1113.0, 125.0 / 192.0, -2187.0 / 6784.0, 11.0 / 84.0}};
// fifth-order minus embedded fourth-order weights
__constant__ double kDpE[7] = {35.0 / 384.0 - 5179.0 / 57600.0,
                               0.0,
                               500.0 / 1113.0 - 7571.0 / 16695.0,
                               125.0 / 192.0 - 393.0 / 640.0,
                               -2187.0 / 6784.0 + 92097.0 / 339200.0,
                               11.0 / 84.0 - 187.0 / 2100.0,
                               -1.0 / 40.0};

enum { kModeFrozen = 0, kModeD3Feedback = 1, kModeD4Feedback = 2 };

__device__ __forceinline__ double ext_p(const FlowArgs &f, int i) { return f.p_min * exp((double)i * f.p_step); }

// d_t y_i = -Flow_i from the raw loop integrals.
__device__ __forceinline__ double deriv_component(const FlowArgs &f, int i) {
  const double *raw = f.raw;
  if (f.mode == kModeFrozen) return -raw[i];
  if (f.mode == kModeD3Feedback) {
    const int n = f.n;
    if (i == 0) return -raw[n];
    const double p = ext_p(f, i - 1);
    return -(raw[i - 1] - raw[n]) / (p * p);
  }
  const int n = f.n, npsi = f.npsi;
  if (i < n) {
    const double p = ext_p(f, i);
    return -(raw[i] - raw[n]) / (p * p);
  }
  if (i < 2 * n) {
    const int ip = i - n;
    double s = 0.0;
    for (int j = 0; j < npsi; ++j) s += 0.5 * f.psi_w[j] * raw[n + 1 + ip * npsi + j];
    return -s;
  }
  return -raw[n + 1 + n * npsi + (i - 2 * n)];
}

// Stage state for stage s (1..6): ys = y + h sum_{r<s} A[s][r] K_r; s = 0: ys = y.
// Also publishes k and m^2 of the stage and the feedback tables.
__device__ __forceinline__ void write_stage_state(const FlowArgs &f, int s, int i, double h) {
  double v = f.y[i];
  for (int r = 0; r < s; ++r) v += h * kDpA[s][r] * f.K[(size_t)r * f.ny + i];
  f.ys[i] = v;
  if (f.tabbuf && i >= f.tab_off && i < f.tab_off + f.tab_len) f.tabbuf[i - f.tab_off] = v;
  if (i == 0 && f.mode == kModeD3Feedback) f.ctl->m2_stage = v;
}

__device__ __forceinline__ void flow_prep_body(const FlowArgs &f, int s, int i) {
  const FlowCtl *c = f.ctl;
  if (*(volatile const int *)&c->done) return;
  const double h = c->h;
  if (i == 0) f.ctl->k_stage = c->Lambda * exp(-(c->t + kDpC[s] * h));
  if (i < f.ny) write_stage_state(f, s, i, h);
}

__global__ void flow_prep_kernel(FlowArgs f, int s) { flow_prep_body(f, s, blockIdx.x * blockDim.x + threadIdx.x); }

// K_s from the RHS, then (s < 6) the state of stage s+1.
__device__ __forceinline__ void flow_deriv_body(const FlowArgs &f, int s, int i) {
  const FlowCtl *c = f.ctl;
  if (*(volatile const int *)&c->done) return;
  const double h = c->h;
  if (i < f.ny) f.K[(size_t)s * f.ny + i] = deriv_component(f, i);
  if (s >= 1 && s < 6) {
    if (i == 0) f.ctl->k_stage = c->Lambda * exp(-(c->t + kDpC[s + 1] * h));
    if (i < f.ny) write_stage_state(f, s + 1, i, h);
  }
}

__global__ void flow_deriv_kernel(FlowArgs f, int s) { flow_deriv_body(f, s, blockIdx.x * blockDim.x + threadIdx.x); }

__device__ __forceinline__ void decide_next_step(FlowCtl *c) {
  const double remaining = c->t1 - c->t;
  if (!(remaining > c->end_tol)) {
    c->done = 1;
    return;
  }
  if (c->steps + c->rejects >= c->max_steps) {
    c->status = FFRG_EMAXSTEPS;
    c->done = 1;
    return;
  }
  c->h = fmin(c->dt, remaining);
}

__global__ void flow_start_kernel(FlowCtl *c) {
  if (threadIdx.x == 0 && blockIdx.x == 0) decide_next_step(c);
}

// Error norm max_i |h sum_r E_r K_r,i| / (atol + rtol max(|y_i|, |y5_i|)),
// accept / reject, step-size update (same controller as the CPU oracle).
__device__ __forceinline__ void flow_control_body(const FlowArgs &f) {
  FlowCtl *c = f.ctl;
  __shared__ double red[32];
  __shared__ int bad_s[32];
  __shared__ int accept_s;
  if (*(volatile const int *)&c->done) return;
  const double h = c->h, atol = c->atol, rtol = c->rtol;
  double emax = 0.0;
  int bad = 0;
  for (int i = threadIdx.x; i < f.ny; i += blockDim.x) {
    double e = 0.0;
    for (int r = 0; r < 7; ++r) e += kDpE[r] * f.K[(size_t)r * f.ny + i];
    e *= h;
    const double y5 = f.ys[i];
    const double sc = atol + rtol * fmax(fabs(f.y[i]), fabs(y5));
    const double ei = fabs(e) / sc;
    if (!isfinite(ei) || !isfinite(y5)) bad = 1;
    else emax = fmax(emax, ei);
  }
  for (int o = 16; o > 0; o >>= 1) {
    emax = fmax(emax, __shfl_down_sync(0xffffffffu, emax, o));
    bad |= __shfl_down_sync(0xffffffffu, bad, o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    red[warp] = emax;
    bad_s[warp] = bad;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double err = 0.0;
    int anybad = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      err = fmax(err, red[w]);
      anybad |= bad_s[w];
    }
    c->err = err;
    int acc = 0;
    if (anybad) {
      c->status = FFRG_ENONFINITE;
      c->done = 1;
    } else if (err <= 1.0) {
      acc = 1;
      c->t += h;
      c->steps += 1;
      double fac = (err == 0.0) ? 5.0 : 0.9 * pow(err, -0.2);
      fac = fmin(fmax(fac, 0.2), 5.0);
      if (c->last_rejected) fac = fmin(fac, 1.0);
      c->last_rejected = 0;
      c->dt = h * fac;
    } else {
      c->rejects += 1;
      if (h <= c->dt_min) {
        c->status = FFRG_ESTEP_UNDERFLOW;
        c->done = 1;
      } else {
        c->dt = h * fmax(0.9 * pow(err, -0.2), 0.2);
        c->last_rejected = 1;
      }
    }
    c->dt = fmin(fmax(c->dt, c->dt_min), c->dt_max);
    accept_s = acc;
  }
  __syncthreads();
  if (accept_s) {
    for (int i = threadIdx.x; i < f.ny; i += blockDim.x) {
      f.y[i] = f.ys[i];
      f.K[i] = f.K[(size_t)6 * f.ny + i];  // first-same-as-last
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && !c->done) decide_next_step(c);
}

__global__ void __launch_bounds__(1024) flow_control_kernel(FlowArgs f) { flow_control_body(f); }

// ---------------------------------------------------------------------------
// Batched DP5(4) steps of many flows (serving): blockIdx.y (or blockIdx.x for
// the control kernel) selects the flow; each flow keeps its own control block,
// so flows at different times, step sizes and stages advance independently.
// ---------------------------------------------------------------------------
__global__ void batched_flow_prep_kernel(const FlowArgs *fa, int s) {
  const FlowArgs &f = fa[blockIdx.y];
  flow_prep_body(f, s, blockIdx.x * blockDim.x + threadIdx.x);
}

__global__ void batched_flow_deriv_kernel(const FlowArgs *fa, int s) {
  const FlowArgs &f = fa[blockIdx.y];
  flow_deriv_body(f, s, blockIdx.x * blockDim.x + threadIdx.x);
}

__global__ void __launch_bounds__(1024) batched_flow_control_kernel(const FlowArgs *fa) {
  flow_control_body(fa[blockIdx.x]);
}

__global__ void batched_flow_start_kernel(const FlowArgs *fa, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && !fa[i].ctl->done) decide_next_step(fa[i].ctl);
}

// First derivative (first-same-as-last stage 0) and the first step size.
int launch_flow_batched_init(ffrg_ctx *ctx, const FlowArgs *fa, int n, int max_ny, const BatchList &bl,
                             cudaStream_t st) {
  if (n == 0) return FFRG_OK;
  const dim3 g((max_ny + 255) / 256, n);
  batched_flow_prep_kernel<<<g, 256, 0, st>>>(fa, 0);
  int rc = launch_rhs_batched(ctx, bl, st);
  if (rc) return rc;
  batched_flow_deriv_kernel<<<g, 256, 0, st>>>(fa, 0);
  batched_flow_start_kernel<<<(n + 255) / 256, 256, 0, st>>>(fa, n);
  return set_cuda_error(ctx, cudaGetLastError(), "batched flow init");
}

// One adaptive step of every flow in the batch (finished flows skip).
int launch_flow_batched_step(ffrg_ctx *ctx, const FlowArgs *fa, int n, int max_ny, const BatchList &bl,
                             cudaStream_t st) {
  if (n == 0) return FFRG_OK;
  const dim3 g((max_ny + 255) / 256, n);
  batched_flow_prep_kernel<<<g, 256, 0, st>>>(fa, 1);
  for (int s = 1; s <= 6; ++s) {
    int rc = launch_rhs_batched(ctx, bl, st);
    if (rc) return rc;
    batched_flow_deriv_kernel<<<g, 256, 0, st>>>(fa, s);
  }
  batched_flow_control_kernel<<<n, 1024, 0, st>>>(fa);
  return set_cuda_error(ctx, cudaGetLastError(), "batched flow step");
}

// ---------------------------------------------------------------------------
// Linearly implicit ROS2 flow (Verwer, Spee, Blom, Hundsdorfer 1999) of the
// d=4 feedback state, gamma = 1 + 1/sqrt(2):
//   W = I - gamma h J,  W k1 = f(t, y),  W k2 = f(t + h, y + h k1) - 2 k1,
//   y_new = y + h (3/2 k1 + 1/2 k2),  error estimate y_new - (y + h k1).
// J = d(d_t y)/dy from the table Jacobian of the RHS (reverse-mode kernels)
// mapped like the derivative; dense LU with partial pivoting in one CTA.
// ---------------------------------------------------------------------------
constexpr double kRosGamma = 1.7071067811865475244;

// W[i][j] = delta_ij - gh (M Jraw)[i][j], M = the map raw -> d_t y (d=4 feedback)
__global__ void ros_build_w_kernel(FlowArgs f, const double *Jraw, double gh, double *W) {
  const int ny = f.ny, n = f.n, npsi = f.npsi;
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)ny * ny) return;
  const int i = (int)(idx / ny), j = (int)(idx % ny);
  double m;
  if (i < n) {
    const double p = ext_p(f, i);
    m = -(Jraw[(size_t)i * ny + j] - Jraw[(size_t)n * ny + j]) / (p * p);
  } else if (i < 2 * n) {
    double s = 0.0;
    for (int q = 0; q < npsi; ++q) s += 0.5 * f.psi_w[q] * Jraw[(size_t)(n + 1 + (i - n) * npsi + q) * ny + j];
    m = -s;
  } else {
    m = -Jraw[(size_t)(n + 1 + n * npsi + (i - 2 * n)) * ny + j];
  }
  W[idx] = (i == j ? 1.0 : 0.0) - gh * m;
}

// In-place LU with partial pivoting (one CTA); a zero pivot stops the flow.
__global__ void __launch_bounds__(1024) lu_kernel(double *W, int n, int *piv, FlowCtl *ctl) {
  __shared__ double bv[32];
  __shared__ int bi[32];
  __shared__ int p_s;
  for (int k = 0; k < n; ++k) {
    double best = -1.0;
    int bidx = n;
    for (int i = k + threadIdx.x; i < n; i += blockDim.x) {
      const double v = fabs(W[(size_t)i * n + k]);
      if (v > best || (v == best && i < bidx)) { best = v; bidx = i; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_down_sync(0xffffffffu, best, o);
      const int oi = __shfl_down_sync(0xffffffffu, bidx, o);
      if (ov > best || (ov == best && oi < bidx)) { best = ov; bidx = oi; }
    }
    if ((threadIdx.x & 31) == 0) { bv[threadIdx.x >> 5] = best; bi[threadIdx.x >> 5] = bidx; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double b = -1.0;
      int p = n;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
        if (bv[w] > b || (bv[w] == b && bi[w] < p)) { b = bv[w]; p = bi[w]; }
      p_s = (b > 0.0 && isfinite(b)) ? p : -1;
      piv[k] = p;
      if (p_s < 0) { ctl->status = FFRG_ENONFINITE; ctl->done = 1; }
    }
    __syncthreads();
    const int p = p_s;
    if (p < 0) return;
    if (p != k)
      for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const double t = W[(size_t)k * n + j];
        W[(size_t)k * n + j] = W[(size_t)p * n + j];
        W[(size_t)p * n + j] = t;
      }
    __syncthreads();
    const double inv = 1.0 / W[(size_t)k * n + k];
    for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) W[(size_t)i * n + k] *= inv;
    __syncthreads();
    const int m = n - k - 1;
    for (int q = threadIdx.x; q < m * m; q += blockDim.x) {
      const int i = k + 1 + q / m, j = k + 1 + q % m;
      W[(size_t)i * n + j] -= W[(size_t)i * n + k] * W[(size_t)k * n + j];
    }
    __syncthreads();
  }
}

// x = W^{-1} b with the factors of lu_kernel (one CTA); x may alias b.
__global__ void __launch_bounds__(1024) lu_solve_kernel(const double *W, const int *piv, int n, const double *b,
                                                        double *x, const FlowCtl *ctl) {
  if (*(volatile const int *)&ctl->done) return;
  for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] = b[i];
  __syncthreads();
  if (threadIdx.x == 0)
    for (int k = 0; k < n; ++k)
      if (piv[k] != k) {
        const double t = x[k];
        x[k] = x[piv[k]];
        x[piv[k]] = t;
      }
  __syncthreads();
  for (int j = 0; j < n; ++j) {  // unit lower triangle
    const double xj = x[j];
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) x[i] -= W[(size_t)i * n + j] * xj;
    __syncthreads();
  }
  for (int j = n - 1; j >= 0; --j) {  // upper triangle
    if (threadIdx.x == 0) x[j] /= W[(size_t)j * n + j];
    __syncthreads();
    const double xj = x[j];
    for (int i = threadIdx.x; i < j; i += blockDim.x) x[i] -= W[(size_t)i * n + j] * xj;
    __syncthreads();
  }
}

// f = d_t y from the raw RHS (out), optionally minus 2 k1
__global__ void ros_map_kernel(FlowArgs f, double *out, const double *k1) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= f.ny) return;
  double v = deriv_component(f, i);
  if (k1) v -= 2.0 * k1[i];
  out[i] = v;
}

// y1 = y + h k1 (also the tables of the second stage)
__global__ void ros_stage_kernel(FlowArgs f, const double *k1) {
  const FlowCtl *c = f.ctl;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= f.ny) return;
  const double v = f.y[i] + c->h * k1[i];
  f.ys[i] = v;
  f.tabbuf[i] = v;
}

// combine, error estimate, accept / reject, step size (exponent 1/2), next h
__global__ void __launch_bounds__(1024) ros_control_kernel(FlowArgs f, const double *k1, const double *k2) {
  FlowCtl *c = f.ctl;
  __shared__ double red[32];
  __shared__ int bad_s[32];
  __shared__ int acc_s;
  if (*(volatile const int *)&c->done) return;
  const double h = c->h;
  double emax = 0.0;
  int bad = 0;
  for (int i = threadIdx.x; i < f.ny; i += blockDim.x) {
    const double yn = f.y[i] + h * (1.5 * k1[i] + 0.5 * k2[i]);
    const double e = fabs(yn - f.ys[i]) / (c->atol + c->rtol * fmax(fabs(f.y[i]), fabs(yn)));
    if (!isfinite(e)) bad = 1;
    else emax = fmax(emax, e);
  }
  for (int o = 16; o > 0; o >>= 1) {
    emax = fmax(emax, __shfl_down_sync(0xffffffffu, emax, o));
    bad |= __shfl_down_sync(0xffffffffu, bad, o);
  }
  if ((threadIdx.x & 31) == 0) { red[threadIdx.x >> 5] = emax; bad_s[threadIdx.x >> 5] = bad; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double err = 0.0;
    int anybad = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { err = fmax(err, red[w]); anybad |= bad_s[w]; }
    c->err = err;
    int acc = 0;
    if (anybad) {
      c->status = FFRG_ENONFINITE;
      c->done = 1;
    } else if (err <= 1.0) {
      acc = 1;
      c->t += h;
      c->steps += 1;
      double fac = (err == 0.0) ? 5.0 : 0.9 * pow(err, -0.5);
      fac = fmin(fmax(fac, 0.2), 5.0);
      if (c->last_rejected) fac = fmin(fac, 1.0);
      c->last_rejected = 0;
      c->dt = h * fac;
    } else {
      c->rejects += 1;
      if (h <= c->dt_min) {
        c->status = FFRG_ESTEP_UNDERFLOW;
        c->done = 1;
      } else {
        c->dt = h * fmax(0.9 * pow(err, -0.5), 0.2);
        c->last_rejected = 1;
      }
    }
    c->dt = fmin(fmax(c->dt, c->dt_min), c->dt_max);
    c->accepted = acc;
    acc_s = acc;
  }
  __syncthreads();
  if (acc_s)
    for (int i = threadIdx.x; i < f.ny; i += blockDim.x) f.y[i] = f.y[i] + h * (1.5 * k1[i] + 0.5 * k2[i]);
  __syncthreads();
  if (threadIdx.x == 0 && !c->done) decide_next_step(c);
}

static int flow_mode(const ffrg_problem *pb, int feedback) {
  if (!feedback) return kModeFrozen;
  if (pb->model == FFRG_MODEL_D3) return kModeD3Feedback;
  if (pb->model == FFRG_MODEL_D4_VERTEX) return kModeD4Feedback;
  return -1;
}

}  // namespace ffrg

using namespace ffrg;

extern "C" int ffrg_flow_state_size(const ffrg_problem *pb, const ffrg_table_desc *desc, int feedback) {
  if (!pb || validate_problem(pb, desc) != FFRG_OK) return -1;
  int mode = flow_mode(pb, feedback);
  if (mode < 0) return -1;
  if (mode == kModeFrozen) return ffrg_n_ext(pb);
  if (!desc) return -1;
  if (mode == kModeD3Feedback) return 1 + desc->n_pts;
  return 3 * desc->n_pts;
}

extern "C" int ffrg_flow(ffrg_ctx *ctx, const ffrg_problem *pb_in, const ffrg_tables *tables, int feedback,
                         double Lambda, double *state_dev, const ffrg_step_opts *o, int precision,
                         ffrg_flow_stats *stats, void *stream) {
  if (!ctx || !pb_in || !tables || !state_dev || !o) return FFRG_EINVAL;
  if (precision != FFRG_FP64 && precision != FFRG_MIXED) return FFRG_EINVAL;
  if (!(Lambda > 0.0) || !isfinite(Lambda)) return FFRG_EINVAL;
  if (!(o->t1 >= o->t0) || !isfinite(o->t1) || !isfinite(o->t0) || !(o->dt0 > 0.0) || !(o->dt_min > 0.0) ||
      !(o->dt_max >= o->dt_min) || !(o->atol >= 0.0) || !(o->rtol >= 0.0) || !(o->atol + o->rtol > 0.0) ||
      o->max_steps < 1)
    return FFRG_EINVAL;
  ffrg_problem pb = *pb_in;
  const ffrg_table_desc *td = &tables->desc;
  int st = validate_problem(&pb, td);
  if (st) return st;
  const int mode = flow_mode(&pb, feedback);
  if (mode < 0) return FFRG_EINVAL;
  if (mode != kModeFrozen) {
    // feedback: the external grid is the table grid
    if (pb.n_ext_p != td->n_pts || pb.p_min != td->x_min || pb.p_max != td->x_max || td->n_stack != 1)
      return FFRG_EINVAL;
  }
  if (mode == kModeD3Feedback) pb.include_p0 = 1;  // I(0) enters d_t m^2 and d_t Z
  const int ny = ffrg_flow_state_size(&pb, td, feedback);
  if (ny < 1) return FFRG_EINVAL;
  cudaSetDevice(ctx->device);
  Plan *pl = nullptr;
  st = get_plan(ctx, &pb, td, &pl);
  if (st) return st;
  const int n_ext = pl->n_ext;

  // device buffers of this flow: segments of the context's flow scratch
  // (kept between calls, grown when this flow needs more)
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t o_ys = al(sizeof(FlowCtl)), o_K = o_ys + al((size_t)ny * sizeof(double));
  const size_t o_raw = o_K + al((size_t)7 * ny * sizeof(double));
  const size_t o_tab = o_raw + al((size_t)n_ext * sizeof(double));
  const size_t need = o_tab + (mode != kModeFrozen ? al((size_t)pl->tab_count * sizeof(double)) : 0);
  if (ctx->flow_cap < need) {
    dev_free(ctx, ctx->flow_dev, ctx->flow_cap);
    ctx->flow_dev = nullptr;
    ctx->flow_cap = 0;
    st = dev_alloc(ctx, &ctx->flow_dev, need);
    if (st) return st;
    ctx->flow_cap = need;
  }
  if (!ctx->flow_host) {
    st = set_cuda_error(ctx, cudaMallocHost(&ctx->flow_host, sizeof(FlowCtl)), "cudaMallocHost");
    if (st) return st;
  }
  if (!ctx->flow_stream) {
    st = set_cuda_error(ctx, cudaStreamCreateWithFlags(&ctx->flow_stream, cudaStreamNonBlocking),
                        "cudaStreamCreate");
    if (st) return st;
  }
  if (!ctx->flow_ev) {
    st = set_cuda_error(ctx, cudaEventCreateWithFlags(&ctx->flow_ev, cudaEventDisableTiming), "cudaEventCreate");
    if (st) return st;
  }
  unsigned char *fb = (unsigned char *)ctx->flow_dev;
  FlowCtl *ctl = (FlowCtl *)fb;
  double *ys = (double *)(fb + o_ys), *K = (double *)(fb + o_K), *raw = (double *)(fb + o_raw);
  double *tabbuf = mode != kModeFrozen ? (double *)(fb + o_tab) : nullptr;
  FlowCtl *ctl_host = (FlowCtl *)ctx->flow_host;
  cudaStream_t user = (cudaStream_t)stream, fs = ctx->flow_stream;
  cudaEvent_t ev = ctx->flow_ev;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;

  FlowCtl hc;
  memset(&hc, 0, sizeof(hc));
  hc.t = o->t0;
  hc.t0 = o->t0;
  hc.t1 = o->t1;
  hc.dt = fmin(fmax(o->dt0, o->dt_min), o->dt_max);
  hc.dt_min = o->dt_min;
  hc.dt_max = o->dt_max;
  hc.atol = o->atol;
  hc.rtol = o->rtol;
  hc.end_tol = 1e-13 * fmax(fabs(o->t1 - o->t0), 1.0);
  hc.Lambda = Lambda;
  hc.max_steps = o->max_steps;
  hc.status = FFRG_OK;

  FlowArgs f;
  memset(&f, 0, sizeof(f));
  f.ny = ny;
  f.mode = mode;
  f.n = td->n_pts;
  f.npsi = pb.n_ext_ang;
  f.tab_off = mode == kModeD3Feedback ? 1 : 0;
  f.tab_len = mode == kModeFrozen ? 0 : pl->tab_count;
  f.p_min = pb.p_min;
  f.p_step = pb.n_ext_p > 1 ? log(pb.p_max / pb.p_min) / (pb.n_ext_p - 1) : 0.0;
  f.psi_w = pl->psi_w;
  f.y = state_dev;
  f.ys = ys;
  f.K = K;
  f.raw = raw;
  f.tabbuf = tabbuf;
  f.ctl = ctl;

  RhsArgs a;
  fill_args(pl, &pb, td, mode == kModeFrozen ? tables->dev : tabbuf, Lambda, a);
  a.out = raw;
  a.status = ctx->status_dev;
  a.k_dev = &ctl->k_stage;
  a.m2_dev = mode == kModeD3Feedback ? &ctl->m2_stage : nullptr;
  a.skip = &ctl->done;

  const int eb = 256, eg = (ny + eb - 1) / eb;
  long long attempts_done = 0;
  if (!st) {
    // order after the caller's stream, initialise, first derivative (FSAL stage 0)
    st = set_cuda_error(ctx, cudaEventRecord(ev, user), "cudaEventRecord");
    if (!st) st = set_cuda_error(ctx, cudaStreamWaitEvent(fs, ev, 0), "cudaStreamWaitEvent");
    if (!st) st = set_cuda_error(ctx, cudaMemcpyAsync(ctl, &hc, sizeof(FlowCtl), cudaMemcpyHostToDevice, fs),
                                 "cudaMemcpyAsync(ctl)");
    if (!st) {
      flow_prep_kernel<<<eg, eb, 0, fs>>>(f, 0);
      st = launch_rhs(ctx, pl, a, precision, fs);
    }
    if (!st) {
      flow_deriv_kernel<<<eg, eb, 0, fs>>>(f, 0);
      flow_start_kernel<<<1, 32, 0, fs>>>(ctl);
      st = set_cuda_error(ctx, cudaGetLastError(), "flow init");
    }
    // make sure the persistent grids are known before capture (no attribute calls inside)
    if (!st) st = set_cuda_error(ctx, cudaStreamSynchronize(fs), "flow init sync");
  }
  if (!st) {
    // capture one adaptive step
    st = set_cuda_error(ctx, cudaStreamBeginCapture(fs, cudaStreamCaptureModeThreadLocal), "BeginCapture");
    if (!st) {
      int cst = FFRG_OK;
      flow_prep_kernel<<<eg, eb, 0, fs>>>(f, 1);
      for (int s = 1; s <= 6 && !cst; ++s) {
        cst = launch_rhs(ctx, pl, a, precision, fs);
        flow_deriv_kernel<<<eg, eb, 0, fs>>>(f, s);
      }
      flow_control_kernel<<<1, 1024, 0, fs>>>(f);
      cudaError_t ce = cudaStreamEndCapture(fs, &graph);
      st = cst ? cst : set_cuda_error(ctx, ce, "EndCapture");
    }
    if (!st) st = set_cuda_error(ctx, cudaGraphInstantiate(&exec, graph, 0), "cudaGraphInstantiate");
  }
  if (!st) {
    int batch = 2;
    for (;;) {
      for (int b = 0; b < batch && !st; ++b)
        st = set_cuda_error(ctx, cudaGraphLaunch(exec, fs), "cudaGraphLaunch");
      if (st) break;
      st = set_cuda_error(ctx, cudaMemcpyAsync(ctl_host, ctl, sizeof(FlowCtl), cudaMemcpyDeviceToHost, fs),
                          "cudaMemcpyAsync(ctl)");
      if (!st) st = set_cuda_error(ctx, cudaStreamSynchronize(fs), "flow sync");
      if (st) break;
      attempts_done = ctl_host->steps + ctl_host->rejects;
      if (ctl_host->done) break;
      batch = std::min(batch * 2, 32);
    }
  }
  if (!st) {
    if (stats) {
      stats->steps = ctl_host->steps;
      stats->rejects = ctl_host->rejects;
      stats->rhs_evals = 1 + 6 * attempts_done;
      stats->integrand_evals = (double)stats->rhs_evals * ffrg_evals(&pb);
      stats->t_reached = ctl_host->t;
      stats->jac_evals = 0;
    }
    st = ctl_host->status;
    // order the caller's stream after the flow
    if (cudaEventRecord(ev, fs) == cudaSuccess) cudaStreamWaitEvent(user, ev, 0);
  }
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  cudaStreamSynchronize(fs);
  return st;
}

extern "C" int ffrg_rosenbrock_flow(ffrg_ctx *ctx, const ffrg_problem *pb_in, const ffrg_tables *tables,
                                    double Lambda, double *state_dev, const ffrg_step_opts *o, ffrg_flow_stats *stats,
                                    void *stream) {
  if (!ctx || !pb_in || !tables || !state_dev || !o) return FFRG_EINVAL;
  if (!(Lambda > 0.0) || !isfinite(Lambda)) return FFRG_EINVAL;
  if (!(o->t1 >= o->t0) || !(o->dt0 > 0.0) || !(o->dt_min > 0.0) || !(o->dt_max >= o->dt_min) || !(o->atol >= 0.0) ||
      !(o->rtol >= 0.0) || !(o->atol + o->rtol > 0.0) || o->max_steps < 1)
    return FFRG_EINVAL;
  ffrg_problem pb = *pb_in;
  const ffrg_table_desc *td = &tables->desc;
  if (pb.model != FFRG_MODEL_D4_VERTEX) return FFRG_EINVAL;
  int st = validate_problem(&pb, td);
  if (st) return st;
  if (pb.n_ext_p != td->n_pts || pb.p_min != td->x_min || pb.p_max != td->x_max) return FFRG_EINVAL;
  const int ny = 3 * td->n_pts;
  if (ny > 4096) return FFRG_EINVAL;
  cudaSetDevice(ctx->device);
  Plan *pl = nullptr;
  st = get_plan(ctx, &pb, td, &pl);
  if (st) return st;
  const int ne = pl->n_ext;
  cudaStream_t user = (cudaStream_t)stream;
  FlowCtl *ctl = nullptr, *hc_pin = nullptr;
  double *f0 = nullptr, *k1 = nullptr, *k2 = nullptr, *ys = nullptr, *raw = nullptr, *tab = nullptr, *Jraw = nullptr,
         *W = nullptr;
  int *piv = nullptr;
  const size_t d = sizeof(double);
  st = dev_alloc(ctx, (void **)&ctl, sizeof(FlowCtl));
  if (!st) st = dev_alloc(ctx, (void **)&f0, ny * d);
  if (!st) st = dev_alloc(ctx, (void **)&k1, ny * d);
  if (!st) st = dev_alloc(ctx, (void **)&k2, ny * d);
  if (!st) st = dev_alloc(ctx, (void **)&ys, ny * d);
  if (!st) st = dev_alloc(ctx, (void **)&raw, ne * d);
  if (!st) st = dev_alloc(ctx, (void **)&tab, (ny * d + 255) & ~(size_t)255);
  if (!st) st = dev_alloc(ctx, (void **)&Jraw, (size_t)ne * ny * d);
  if (!st) st = dev_alloc(ctx, (void **)&W, (size_t)ny * ny * d);
  if (!st) st = dev_alloc(ctx, (void **)&piv, ny * sizeof(int));
  if (!st) st = set_cuda_error(ctx, cudaMallocHost((void **)&hc_pin, sizeof(FlowCtl)), "cudaMallocHost");
  FlowCtl hc;
  memset(&hc, 0, sizeof(hc));
  hc.t = o->t0;
  hc.t0 = o->t0;
  hc.t1 = o->t1;
  hc.dt = fmin(fmax(o->dt0, o->dt_min), o->dt_max);
  hc.dt_min = o->dt_min;
  hc.dt_max = o->dt_max;
  hc.atol = o->atol;
  hc.rtol = o->rtol;
  hc.end_tol = 1e-13 * fmax(fabs(o->t1 - o->t0), 1.0);
  hc.Lambda = Lambda;
  hc.max_steps = o->max_steps;
  FlowArgs f;
  memset(&f, 0, sizeof(f));
  f.ny = ny;
  f.mode = kModeD4Feedback;
  f.n = td->n_pts;
  f.npsi = pb.n_ext_ang;
  f.tab_len = ny;
  f.p_min = pb.p_min;
  f.p_step = pb.n_ext_p > 1 ? log(pb.p_max / pb.p_min) / (pb.n_ext_p - 1) : 0.0;
  f.psi_w = pl->psi_w;
  f.y = state_dev;
  f.ys = ys;
  f.raw = raw;
  f.tabbuf = tab;
  f.ctl = ctl;
  const int eb = 256, eg = (ny + eb - 1) / eb;
  long long rhs_calls = 0, jacs = 0;
  // RHS (FP64) of the tables in `tab` at scale k into raw
  auto rhs_at = [&](double k) {
    RhsArgs a;
    fill_args(pl, &pb, td, tab, k, a);
    a.out = raw;
    a.status = ctx->status_dev;
    ++rhs_calls;
    return launch_rhs(ctx, pl, a, FFRG_FP64, user);
  };
  auto read_ctl = [&]() {
    cudaError_t e = cudaMemcpyAsync(hc_pin, ctl, sizeof(FlowCtl), cudaMemcpyDeviceToHost, user);
    if (e == cudaSuccess) e = cudaStreamSynchronize(user);
    return set_cuda_error(ctx, e, "rosenbrock sync");
  };
  if (!st) st = set_cuda_error(ctx, cudaMemcpyAsync(ctl, &hc, sizeof(hc), cudaMemcpyHostToDevice, user), "ctl");
  if (!st) st = set_cuda_error(ctx, cudaMemcpyAsync(tab, state_dev, ny * d, cudaMemcpyDeviceToDevice, user), "tab");
  if (!st) st = rhs_at(Lambda * exp(-o->t0));
  if (!st) {
    ros_map_kernel<<<eg, eb, 0, user>>>(f, f0, nullptr);
    flow_start_kernel<<<1, 32, 0, user>>>(ctl);
    st = read_ctl();
  }
  bool need_jac = true;
  while (!st && !hc_pin->done) {
    const double t = hc_pin->t, h = hc_pin->h;
    if (need_jac) {
      st = launch_jacobian(ctx, &pb, td, tab, Lambda * exp(-t), Jraw, user);
      ++jacs;
      need_jac = false;
      if (st) break;
    }
    const size_t nn = (size_t)ny * ny;
    ros_build_w_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, user>>>(f, Jraw, kRosGamma * h, W);
    lu_kernel<<<1, 1024, 0, user>>>(W, ny, piv, ctl);
    lu_solve_kernel<<<1, 1024, 0, user>>>(W, piv, ny, f0, k1, ctl);
    ros_stage_kernel<<<eg, eb, 0, user>>>(f, k1);
    st = rhs_at(Lambda * exp(-(t + h)));
    if (st) break;
    ros_map_kernel<<<eg, eb, 0, user>>>(f, k2, k1);
    lu_solve_kernel<<<1, 1024, 0, user>>>(W, piv, ny, k2, k2, ctl);
    ros_control_kernel<<<1, 1024, 0, user>>>(f, k1, k2);
    st = read_ctl();
    if (st) break;
    if (hc_pin->accepted && !hc_pin->done) {
      st = set_cuda_error(ctx, cudaMemcpyAsync(tab, state_dev, ny * d, cudaMemcpyDeviceToDevice, user), "tab");
      if (!st) st = rhs_at(Lambda * exp(-hc_pin->t));
      if (!st) ros_map_kernel<<<eg, eb, 0, user>>>(f, f0, nullptr);
      need_jac = true;
    } else if (!hc_pin->done) {
      // rejected: same Jacobian, stage tables back to the current state
      st = set_cuda_error(ctx, cudaMemcpyAsync(tab, state_dev, ny * d, cudaMemcpyDeviceToDevice, user), "tab");
    }
  }
  if (!st) {
    if (stats) {
      stats->steps = hc_pin->steps;
      stats->rejects = hc_pin->rejects;
      stats->rhs_evals = rhs_calls;
      stats->integrand_evals = (double)rhs_calls * ffrg_evals(&pb);
      stats->t_reached = hc_pin->t;
      stats->jac_evals = jacs;
    }
    st = hc_pin->status;
  }
  cudaStreamSynchronize(user);
  if (hc_pin) cudaFreeHost(hc_pin);
  dev_free(ctx, ctl, sizeof(FlowCtl));
  dev_free(ctx, f0, ny * d);
  dev_free(ctx, k1, ny * d);
  dev_free(ctx, k2, ny * d);
  dev_free(ctx, ys, ny * d);
  dev_free(ctx, raw, ne * d);
  dev_free(ctx, tab, (ny * d + 255) & ~(size_t)255);
  dev_free(ctx, Jraw, (size_t)ne * ny * d);
  dev_free(ctx, W, (size_t)ny * ny * d);
  dev_free(ctx, piv, ny * sizeof(int));
  return st;
}

// ---------------------------------------------------------------------------
// Adams-Bashforth-Moulton (PECE, fixed step; the paper's Boost_ABM option,
// Sec. 5.2.1).  Standard Adams tables: predictor AB_s with the s newest
// back values of d_t y, corrector AM_s with the predicted value and s-1
// back values; the first s-1 steps are classical RK4.
// ---------------------------------------------------------------------------
namespace ffrg {

static const double kAbmB[6][5] = {{0},
                                   {1.0},
                                   {3.0 / 2.0, -1.0 / 2.0},
                                   {23.0 / 12.0, -16.0 / 12.0, 5.0 / 12.0},
                                   {55.0 / 24.0, -59.0 / 24.0, 37.0 / 24.0, -9.0 / 24.0},
                                   {1901.0 / 720.0, -2774.0 / 720.0, 2616.0 / 720.0, -1274.0 / 720.0, 251.0 / 720.0}};
static const double kAbmA[6][5] = {{0},
                                   {1.0},
                                   {1.0 / 2.0, 1.0 / 2.0},
                                   {5.0 / 12.0, 8.0 / 12.0, -1.0 / 12.0},
                                   {9.0 / 24.0, 19.0 / 24.0, -5.0 / 24.0, 1.0 / 24.0},
                                   {251.0 / 720.0, 646.0 / 720.0, -264.0 / 720.0, 106.0 / 720.0, -19.0 / 720.0}};

struct AbmCombo {
  const double *src[6];
  double c[6];
  int n;
};

// Evaluation state ys = y + h sum_j c_j src_j at t + tf h (write_y: also the
// new state y); publishes k, the feedback tables and m^2 like a DP5(4) stage.
__global__ void abm_stage_kernel(FlowArgs f, AbmCombo cb, double h, double tf, int write_y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  FlowCtl *c = f.ctl;
  if (i == 0) c->k_stage = c->Lambda * exp(-(c->t + tf * h));
  if (i >= f.ny) return;
  double v = f.y[i];
  for (int j = 0; j < cb.n; ++j) v += h * cb.c[j] * cb.src[j][i];
  if (write_y) f.y[i] = v;
  f.ys[i] = v;
  if (f.tabbuf && i >= f.tab_off && i < f.tab_off + f.tab_len) f.tabbuf[i - f.tab_off] = v;
  if (i == 0 && f.mode == kModeD3Feedback) c->m2_stage = v;
}

__global__ void abm_deriv_kernel(FlowArgs f, double *dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < f.ny) dst[i] = deriv_component(f, i);
}

// F[j] <- F[j-1], F[0] <- d_t y at the new point; t = t0 + (steps + 1) h
__global__ void abm_push_kernel(FlowArgs f, double *F, int order, double h) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  FlowCtl *c = f.ctl;
  if (i < f.ny) {
    for (int j = order - 1; j >= 1; --j) F[(size_t)j * f.ny + i] = F[(size_t)(j - 1) * f.ny + i];
    const double d = deriv_component(f, i);
    F[i] = d;
    if (!isfinite(d) || !isfinite(f.y[i])) c->status = FFRG_ENONFINITE;
  }
  if (i == 0) {
    c->steps += 1;
    c->t = c->t0 + (double)c->steps * h;
  }
}

}  // namespace ffrg

extern "C" int ffrg_abm_flow(ffrg_ctx *ctx, const ffrg_problem *pb_in, const ffrg_tables *tables, int feedback,
                             double Lambda, double *state_dev, double t0, double t1, long long n_steps, int order,
                             int precision, ffrg_flow_stats *stats, void *stream) {
  if (!ctx || !pb_in || !tables || !state_dev) return FFRG_EINVAL;
  if (precision != FFRG_FP64 && precision != FFRG_MIXED) return FFRG_EINVAL;
  if (!(Lambda > 0.0) || !isfinite(Lambda) || !isfinite(t0) || !isfinite(t1) || !(t1 >= t0)) return FFRG_EINVAL;
  if (order < 2 || order > 5 || n_steps < 1 || n_steps > (1LL << 40)) return FFRG_EINVAL;
  ffrg_problem pb = *pb_in;
  const ffrg_table_desc *td = &tables->desc;
  int st = validate_problem(&pb, td);
  if (st) return st;
  const int mode = flow_mode(&pb, feedback);
  if (mode < 0) return FFRG_EINVAL;
  if (mode != kModeFrozen &&
      (pb.n_ext_p != td->n_pts || pb.p_min != td->x_min || pb.p_max != td->x_max || td->n_stack != 1))
    return FFRG_EINVAL;
  if (mode == kModeD3Feedback) pb.include_p0 = 1;
  const int ny = ffrg_flow_state_size(&pb, td, feedback);
  if (ny < 1) return FFRG_EINVAL;
  cudaSetDevice(ctx->device);
  Plan *pl = nullptr;
  st = get_plan(ctx, &pb, td, &pl);
  if (st) return st;
  const size_t d = sizeof(double), tab_bytes = ((size_t)pl->tab_count * d + 255) & ~(size_t)255;
  FlowCtl *ctl = nullptr, *ctl_host = nullptr;
  double *ys = nullptr, *F = nullptr, *S = nullptr, *raw = nullptr, *tabbuf = nullptr;  // S: 3 scratch derivatives
  st = dev_alloc(ctx, (void **)&ctl, sizeof(FlowCtl));
  if (!st) st = dev_alloc(ctx, (void **)&ys, (size_t)ny * d);
  if (!st) st = dev_alloc(ctx, (void **)&F, (size_t)order * ny * d);
  if (!st) st = dev_alloc(ctx, (void **)&S, (size_t)3 * ny * d);
  if (!st) st = dev_alloc(ctx, (void **)&raw, (size_t)pl->n_ext * d);
  if (!st && mode != kModeFrozen) st = dev_alloc(ctx, (void **)&tabbuf, tab_bytes);
  if (!st) st = set_cuda_error(ctx, cudaMallocHost((void **)&ctl_host, sizeof(FlowCtl)), "cudaMallocHost");
  cudaStream_t user = (cudaStream_t)stream, fs = nullptr;
  cudaEvent_t ev = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  if (!st) st = set_cuda_error(ctx, cudaStreamCreateWithFlags(&fs, cudaStreamNonBlocking), "cudaStreamCreate");
  if (!st) st = set_cuda_error(ctx, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "cudaEventCreate");

  FlowCtl hc;
  memset(&hc, 0, sizeof(hc));
  hc.t = t0;
  hc.t0 = t0;
  hc.t1 = t1;
  hc.Lambda = Lambda;
  hc.status = FFRG_OK;
  FlowArgs f;
  memset(&f, 0, sizeof(f));
  f.ny = ny;
  f.mode = mode;
  f.n = td->n_pts;
  f.npsi = pb.n_ext_ang;
  f.tab_off = mode == kModeD3Feedback ? 1 : 0;
  f.tab_len = mode == kModeFrozen ? 0 : pl->tab_count;
  f.p_min = pb.p_min;
  f.p_step = pb.n_ext_p > 1 ? log(pb.p_max / pb.p_min) / (pb.n_ext_p - 1) : 0.0;
  f.psi_w = pl->psi_w;
  f.y = state_dev;
  f.ys = ys;
  f.raw = raw;
  f.tabbuf = tabbuf;
  f.ctl = ctl;
  RhsArgs a;
  fill_args(pl, &pb, td, mode == kModeFrozen ? tables->dev : tabbuf, Lambda, a);
  a.out = raw;
  a.status = ctx->status_dev;
  a.k_dev = &ctl->k_stage;
  a.m2_dev = mode == kModeD3Feedback ? &ctl->m2_stage : nullptr;
  a.skip = &ctl->done;  // never set: fixed steps

  const int eb = 256, eg = (ny + eb - 1) / eb;
  const double h = (t1 - t0) / (double)n_steps;
  double *K2 = S, *K3 = S + ny, *K4 = S + 2 * (size_t)ny;  // RK4 stages; K2 also holds the predicted slope
  auto stage = [&](std::initializer_list<std::pair<const double *, double>> terms, double tf, int write_y) {
    AbmCombo cb;
    memset(&cb, 0, sizeof(cb));
    for (const auto &t : terms) {
      cb.src[cb.n] = t.first;
      cb.c[cb.n++] = t.second;
    }
    abm_stage_kernel<<<eg, eb, 0, fs>>>(f, cb, h, tf, write_y);
  };
  const long long n_rk = std::min<long long>(n_steps, order - 1);
  if (!st) {
    st = set_cuda_error(ctx, cudaEventRecord(ev, user), "cudaEventRecord");
    if (!st) st = set_cuda_error(ctx, cudaStreamWaitEvent(fs, ev, 0), "cudaStreamWaitEvent");
    if (!st) st = set_cuda_error(ctx, cudaMemcpyAsync(ctl, &hc, sizeof(FlowCtl), cudaMemcpyHostToDevice, fs),
                                 "cudaMemcpyAsync(ctl)");
    // d_t y at t0
    if (!st) {
      stage({}, 0.0, 0);
      st = launch_rhs(ctx, pl, a, precision, fs);
    }
    if (!st) abm_deriv_kernel<<<eg, eb, 0, fs>>>(f, F);
    // starting steps: classical RK4 with k1 = F[0]
    for (long long m = 0; m < n_rk && !st; ++m) {
      stage({{F, 0.5}}, 0.5, 0);
      st = launch_rhs(ctx, pl, a, precision, fs);
      abm_deriv_kernel<<<eg, eb, 0, fs>>>(f, K2);
      if (!st) {
        stage({{K2, 0.5}}, 0.5, 0);
        st = launch_rhs(ctx, pl, a, precision, fs);
        abm_deriv_kernel<<<eg, eb, 0, fs>>>(f, K3);
      }
      if (!st) {
        stage({{K3, 1.0}}, 1.0, 0);
        st = launch_rhs(ctx, pl, a, precision, fs);
        abm_deriv_kernel<<<eg, eb, 0, fs>>>(f, K4);
      }
      if (!st) {
        stage({{F, 1.0 / 6.0}, {K2, 1.0 / 3.0}, {K3, 1.0 / 3.0}, {K4, 1.0 / 6.0}}, 1.0, 1);
        st = launch_rhs(ctx, pl, a, precision, fs);
        abm_push_kernel<<<eg, eb, 0, fs>>>(f, F, order, h);
      }
    }
    if (!st) st = set_cuda_error(ctx, cudaGetLastError(), "abm start");
    // the persistent grids are known before capture (no attribute calls inside)
    if (!st) st = set_cuda_error(ctx, cudaStreamSynchronize(fs), "abm start sync");
  }
  if (!st && n_steps > n_rk) {
    // capture one PECE step
    st = set_cuda_error(ctx, cudaStreamBeginCapture(fs, cudaStreamCaptureModeThreadLocal), "BeginCapture");
    if (!st) {
      AbmCombo pc, cc;
      memset(&pc, 0, sizeof(pc));
      memset(&cc, 0, sizeof(cc));
      for (int j = 0; j < order; ++j) {
        pc.src[j] = F + (size_t)j * ny;
        pc.c[j] = kAbmB[order][j];
      }
      pc.n = order;
      cc.src[0] = K2;
      cc.c[0] = kAbmA[order][0];
      for (int j = 1; j < order; ++j) {
        cc.src[j] = F + (size_t)(j - 1) * ny;
        cc.c[j] = kAbmA[order][j];
      }
      cc.n = order;
      int cst = FFRG_OK;
      abm_stage_kernel<<<eg, eb, 0, fs>>>(f, pc, h, 1.0, 0);
      cst = launch_rhs(ctx, pl, a, precision, fs);
      abm_deriv_kernel<<<eg, eb, 0, fs>>>(f, K2);
      abm_stage_kernel<<<eg, eb, 0, fs>>>(f, cc, h, 1.0, 1);
      if (!cst) cst = launch_rhs(ctx, pl, a, precision, fs);
      abm_push_kernel<<<eg, eb, 0, fs>>>(f, F, order, h);
      cudaError_t ce = cudaStreamEndCapture(fs, &graph);
      st = cst ? cst : set_cuda_error(ctx, ce, "EndCapture");
    }
    if (!st) st = set_cuda_error(ctx, cudaGraphInstantiate(&exec, graph, 0), "cudaGraphInstantiate");
    for (long long m = n_rk; m < n_steps && !st; ++m)
      st = set_cuda_error(ctx, cudaGraphLaunch(exec, fs), "cudaGraphLaunch");
  }
  if (!st) st = set_cuda_error(ctx, cudaMemcpyAsync(ctl_host, ctl, sizeof(FlowCtl), cudaMemcpyDeviceToHost, fs),
                               "cudaMemcpyAsync(ctl)");
  if (!st) st = set_cuda_error(ctx, cudaStreamSynchronize(fs), "abm sync");
  if (!st) {
    if (stats) {
      stats->steps = n_steps;
      stats->rejects = 0;
      stats->rhs_evals = 1 + 4 * n_rk + 2 * (n_steps - n_rk);
      stats->integrand_evals = (double)stats->rhs_evals * ffrg_evals(&pb);
      stats->t_reached = ctl_host->t;
      stats->jac_evals = 0;
    }
    st = ctl_host->status;
    if (cudaEventRecord(ev, fs) == cudaSuccess) cudaStreamWaitEvent(user, ev, 0);
  }
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  if (fs) cudaStreamSynchronize(fs);
  if (ev) cudaEventDestroy(ev);
  if (fs) cudaStreamDestroy(fs);
  if (ctl_host) cudaFreeHost(ctl_host);
  dev_free(ctx, ctl, sizeof(FlowCtl));
  dev_free(ctx, ys, (size_t)ny * d);
  dev_free(ctx, F, (size_t)order * ny * d);
  dev_free(ctx, S, (size_t)3 * ny * d);
  dev_free(ctx, raw, (size_t)pl->n_ext * d);
  dev_free(ctx, tabbuf, tab_bytes);
  return st;
}
