// Vector-Jacobian product of the momentum-loop RHS with respect to the
// dressing-table values (reverse-mode counterpart of the paper's forward-mode
// Jacobians, Sec. 5.2.2):  tbar_j = sum_e gbar_e d out_e / d T_j.
//
// Every lookup is a lerp between two table nodes, so each integrand
// evaluation scatters (1-w) c and w c into two entries of the gradient, where
// c is the derivative of the term with respect to the looked-up value.  The
// Z(q) dependence of the per-radial factor F (regulator derivative and
// G(q)^2) enters through dF/dZ(q) times the angular row sum.
//
// Determinism: no floating-point atomics.  Each warp accumulates into its own
// shared-memory copy of the gradient, lanes taking turns in a fixed order;
// warps are then summed in a fixed order into one partial per CTA, and a
// second kernel sums the CTA partials in a fixed order.  Results are
// reproducible run to run for a given GPU (the persistent grid size fixes
// which items each CTA owns).
#include <math.h>

#include <algorithm>

#include "ffrg_internal.cuh"

namespace ffrg {

constexpr int kAdjThreads = 256;

struct AdjArgs {
  RhsArgs a;
  const double *gbar;  // [n_ext]
  double *gpart;       // [grid][tab_count]
  double *jrows;       // Jacobian mode: one gradient row per work item [n_items][tab_count]
};

// Jacobian mode: clear the warp-private gradients before a work item ...
__device__ __forceinline__ void jac_item_begin(const AdjArgs &A, double *grad) {
  if (!A.jrows) return;
  __syncthreads();
  const int nw = blockDim.x >> 5;
  for (int i = threadIdx.x; i < nw * A.a.tab_count; i += blockDim.x) grad[i] = 0.0;
  __syncthreads();
}

// ... and sum them (warps in order) into the item's row after it.
__device__ __forceinline__ void jac_item_end(const AdjArgs &A, const double *grad, int item) {
  if (!A.jrows) return;
  __syncthreads();
  const int nw = blockDim.x >> 5, T = A.a.tab_count;
  for (int i = threadIdx.x; i < T; i += blockDim.x) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += grad[(size_t)w * T + i];
    A.jrows[(size_t)item * T + i] = s;
  }
}

// lanes add in turn: lane 0 first, lane 31 last
__device__ __forceinline__ void warp_scatter2(double *g, int i0, double v0, double v1, int lane) {
  for (int l = 0; l < 32; ++l) {
    if (lane == l && (v0 != 0.0 || v1 != 0.0)) {
      g[i0] += v0;
      g[i0 + 1] += v1;
    }
    __syncwarp();
  }
}

struct LerpPos {
  int i0;
  double w;
};

__device__ __forceinline__ LerpPos pos_of(const RhsArgs &a, double s2) {
  LerpPos p;
  lerp_pos(s2, a.u_scale, a.u_off, a.n_pts, p.i0, p.w);
  return p;
}
__device__ __forceinline__ double val_at(const double *t, LerpPos p) { return lerp_at(t, p.i0, p.w); }

// shared memory: tables | angle rules (c1, s1, w1, c2, w2) | per-warp gradients
struct AdjSmem {
  double *tab, *c1, *s1, *w1, *c2, *w2, *grad;
  __device__ AdjSmem(unsigned char *base, const RhsArgs &a) {
    size_t off = ((size_t)a.tab_count * 8 + 15) & ~(size_t)15;
    tab = (double *)base;
    c1 = (double *)(base + off);
    s1 = c1 + a.na1;
    w1 = s1 + a.na1;
    c2 = w1 + a.na1;
    w2 = c2 + a.na2;
    off += (((size_t)(3 * a.na1 + 2 * a.na2)) * 8 + 15) & ~(size_t)15;
    grad = (double *)(base + off);
  }
};

__device__ bool adj_prologue(const RhsArgs &a, AdjSmem &S, uint64_t *bar) {
  bool ok = stage_to_smem<double>(S.tab, a.tab, a.tab_count, bar, a.status);
  for (int i = threadIdx.x; i < a.na1; i += blockDim.x) {
    double c = a.a1_x[i];
    S.c1[i] = c;
    S.s1[i] = sqrt(fmax(0.0, 1.0 - c * c));
    S.w1[i] = a.a1_w[i];
  }
  for (int i = threadIdx.x; i < a.na2; i += blockDim.x) {
    S.c2[i] = a.a2_x[i];
    S.w2[i] = a.a2_w[i];
  }
  const int nw = blockDim.x >> 5;
  for (int i = threadIdx.x; i < nw * a.tab_count; i += blockDim.x) S.grad[i] = 0.0;
  __syncthreads();
  return ok;
}

__device__ void adj_epilogue(const AdjArgs &A, AdjSmem &S) {
  if (A.jrows) return;
  __syncthreads();
  const RhsArgs &a = A.a;
  const int nw = blockDim.x >> 5;
  for (int i = threadIdx.x; i < a.tab_count; i += blockDim.x) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += S.grad[(size_t)w * a.tab_count + i];
    A.gpart[(size_t)blockIdx.x * a.tab_count + i] = s;
  }
}

// Z coefficient of the propagator denominator: Z P + m^2, P = s^2 + k^2 r(s^2/k^2)
__device__ __forceinline__ double zcoef(int reg, double s2, double k2, double inv_k2) {
  return s2 + k2 * reg_r(reg, s2 * inv_k2);
}

// ---------------------------------------------------------------------------
// d = 3:  term = F_r w_j G(s)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kAdjThreads) d3_adjoint(AdjArgs A) {
  const RhsArgs &a = A.a;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t bar;
  AdjSmem S(smem, a);
  if (!adj_prologue(a, S, &bar)) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double *g = S.grad + (size_t)warp * a.tab_count;
  const double k = scale_k(a), k2 = k * k, inv_k2 = 1.0 / k2, m2 = mass2(a, k);
  const int nblk = (a.na1 + a.jb - 1) / a.jb;
  for (int item = blockIdx.x; item < a.n_items; item += gridDim.x) {
    const int e = item / a.n_chunks, c = item - e * a.n_chunks;
    const double p = (e < a.n_ext_p) ? ext_momentum(a, e) : 0.0;
    const double gn = (A.jrows ? 1.0 : A.gbar[e]) * a.norm;
    jac_item_begin(A, S.grad);
    const int o0 = c * a.cr, o1 = min(o0 + a.cr, a.nr);
    const int rows = (o1 - o0) * nblk;
    for (int base = warp * 32; base < rows; base += blockDim.x) {
      const int row = base + lane;
      const bool valid = row < rows;
      const int o = valid ? o0 + row / nblk : o0;
      const int jb0 = valid ? (row % nblk) * a.jb : 0, jb1 = valid ? min(jb0 + a.jb, a.na1) : 0;
      const double q = a.radq[o], F = a.radF[o], dF = a.radD[o];
      double vrow = 0.0;
      for (int jj = 0; jj < a.jb; ++jj) {
        const int j = jb0 + jj;
        double c0 = 0.0, c1 = 0.0;
        int i0 = 0;
        if (j < jb1) {
          const double s2 = fmax(q * q + p * p + 2.0 * q * p * S.c1[j], 0.0);
          const LerpPos ps = pos_of(a, s2);
          const double Z = val_at(S.tab, ps), P = zcoef(a.reg, s2, k2, inv_k2);
          const double G = 1.0 / (Z * P + m2);
          vrow += S.w1[j] * G;
          const double cz = gn * F * S.w1[j] * (-G * G * P);
          i0 = ps.i0;
          c0 = (1.0 - ps.w) * cz;
          c1 = ps.w * cz;
        }
        warp_scatter2(g, i0, c0, c1, lane);
      }
      double q0 = 0.0, q1 = 0.0;
      int iq = 0;
      if (valid) {
        const LerpPos pq = pos_of(a, q * q);
        const double cq = gn * dF * vrow;
        iq = pq.i0;
        q0 = (1.0 - pq.w) * cq;
        q1 = pq.w * cq;
      }
      warp_scatter2(g, iq, q0, q1, lane);
    }
    jac_item_end(A, S.grad, item);
  }
  adj_epilogue(A, S);
}

// ---------------------------------------------------------------------------
// d = 4 vertex expansion (tables Z | lambda3 | lambda4 at offsets 0 | n | 2n)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kAdjThreads) d4_adjoint(AdjArgs A) {
  const RhsArgs &a = A.a;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t bar;
  AdjSmem S(smem, a);
  if (!adj_prologue(a, S, &bar)) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double *g = S.grad + (size_t)warp * a.tab_count;
  const double k = scale_k(a), k2 = k * k, inv_k2 = 1.0 / k2, m2 = mass2(a, k);
  const int np = a.n_pts, np_ = a.n_ext_p, npsi = a.n_ext_ang;
  const double *Zt = S.tab, *L3 = S.tab + np, *L4 = S.tab + 2 * np;
  const int oZ = 0, o3 = np, o4 = 2 * np;
  const double third = 1.0 / 3.0, sw2 = a.sum_w2;
  for (int item = blockIdx.x; item < a.n_items; item += gridDim.x) {
    const int e = item / a.n_chunks, c = item - e * a.n_chunks;
    int block, ip, jp = 0;
    if (e <= np_) {
      block = 0;
      ip = e;
    } else if (e < np_ + 1 + np_ * npsi) {
      block = 1;
      ip = (e - np_ - 1) / npsi;
      jp = (e - np_ - 1) - ip * npsi;
    } else {
      block = 2;
      ip = e - np_ - 1 - np_ * npsi;
    }
    const double p = (block == 0 && ip == np_) ? 0.0 : ext_momentum(a, ip);
    const double cpsi = block == 1 ? a.psi_x[jp] : 1.0, spsi = sqrt(fmax(0.0, 1.0 - cpsi * cpsi));
    const double p2 = p * p, C2 = 2.0 * p2 * (1.0 + cpsi);
    const double coef = block == 1 ? 3.0 : (block == 2 ? 1.5 : 1.0);
    const double gn = (A.jrows ? 1.0 : A.gbar[e]) * a.norm * coef;
    jac_item_begin(A, S.grad);
    const int o0 = c * a.cr, o1 = min(o0 + a.cr, a.nr);
    const int rows = (o1 - o0) * a.na1;
    for (int base = warp * 32; base < rows; base += blockDim.x) {
      const int row = base + lane;
      const bool valid = row < rows;
      const int r = valid ? o0 + row / a.na1 : o0, ia = valid ? row % a.na1 : 0;
      const double q = a.radq[r], F = a.radF[r], dF = a.radD[r];
      const double q2 = q * q, qp = q * p, c1 = S.c1[ia], w1 = S.w1[ia];
      const double A2 = fmax(q2 + p2 + 2.0 * qp * c1, 0.0);
      const LerpPos pA = pos_of(a, A2);
      const double ZA = val_at(Zt, pA), PA = zcoef(a.reg, A2, k2, inv_k2);
      const double GA = 1.0 / (ZA * PA + m2);
      const double gF = valid ? gn * F * w1 : 0.0;  // d(out)/d(row value) x gbar
      double v = 0.0;                               // row value (without F w1)
      if (block == 0) {
        const LerpPos p4 = pos_of(a, (q2 + p2) * 0.5), p3 = pos_of(a, (q2 + A2 + p2) * third);
        const double l4 = val_at(L4, p4), l3 = val_at(L3, p3);
        v = sw2 * (-0.5 * l4 + l3 * l3 * GA);
        double c4 = gF * sw2 * (-0.5), c3 = gF * sw2 * 2.0 * l3 * GA, cA = gF * sw2 * l3 * l3 * (-GA * GA * PA);
        warp_scatter2(g, o4 + p4.i0, (1.0 - p4.w) * c4, p4.w * c4, lane);
        warp_scatter2(g, o3 + p3.i0, (1.0 - p3.w) * c3, p3.w * c3, lane);
        warp_scatter2(g, oZ + pA.i0, (1.0 - pA.w) * cA, pA.w * cA, lane);
      } else if (block == 2) {
        const LerpPos p4 = pos_of(a, (q2 + A2 + 2.0 * p2) * 0.25);
        const double l4 = val_at(L4, p4);
        v = sw2 * GA * l4 * l4;
        double c4 = gF * sw2 * 2.0 * GA * l4, cA = gF * sw2 * l4 * l4 * (-GA * GA * PA);
        warp_scatter2(g, o4 + p4.i0, (1.0 - p4.w) * c4, p4.w * c4, lane);
        warp_scatter2(g, oZ + pA.i0, (1.0 - pA.w) * cA, pA.w * cA, lane);
      } else {
        const LerpPos pa = pos_of(a, (q2 + A2 + p2) * third);
        const double la = val_at(L3, pa);
        const double basev = q2 + p2, t1 = 2.0 * qp * cpsi * c1, t2 = 2.0 * qp * spsi * S.s1[ia];
        const double sab = A2 + C2;
        const double gFA = gF * GA * la;  // common factor of the inner terms
        double rs = 0.0;
        for (int b = 0; b < a.na2; ++b) {
          const double B2 = fmax(basev - t1 - t2 * S.c2[b], 0.0);
          const LerpPos pB = pos_of(a, B2), pb = pos_of(a, (basev + B2) * third), pc = pos_of(a, (sab + B2) * third);
          const double ZB = val_at(Zt, pB), PB = zcoef(a.reg, B2, k2, inv_k2);
          const double GB = 1.0 / (ZB * PB + m2);
          const double lb = val_at(L3, pb), lc = val_at(L3, pc);
          const double w2 = S.w2[b];
          rs += w2 * GB * lb * lc;
          const double cB = gFA * w2 * (-GB * GB * PB) * lb * lc;
          const double cb = gFA * w2 * GB * lc, cc = gFA * w2 * GB * lb;
          warp_scatter2(g, oZ + pB.i0, (1.0 - pB.w) * cB, pB.w * cB, lane);
          warp_scatter2(g, o3 + pb.i0, (1.0 - pb.w) * cb, pb.w * cb, lane);
          warp_scatter2(g, o3 + pc.i0, (1.0 - pc.w) * cc, pc.w * cc, lane);
        }
        v = GA * la * rs;
        const double cA = gF * (-GA * GA * PA) * la * rs, ca = gF * GA * rs;
        warp_scatter2(g, oZ + pA.i0, (1.0 - pA.w) * cA, pA.w * cA, lane);
        warp_scatter2(g, o3 + pa.i0, (1.0 - pa.w) * ca, pa.w * ca, lane);
      }
      // Z(q) through F = w q^3 dR(q) G(q)^2
      const LerpPos pq = pos_of(a, q2);
      const double cq = valid ? gn * dF * w1 * v : 0.0;
      warp_scatter2(g, oZ + pq.i0, (1.0 - pq.w) * cq, pq.w * cq, lane);
    }
    jac_item_end(A, S.grad, item);
  }
  adj_epilogue(A, S);
}

// fixed-order sum of the CTA partials
__global__ void adj_reduce_kernel(const double *gpart, int grid, int count, double *tbar) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  double s = 0.0;
  for (int b = 0; b < grid; ++b) s += gpart[(size_t)b * count + i];
  tbar[i] = s;
}

}  // namespace ffrg

using namespace ffrg;

namespace ffrg {

// fixed-order sum of the chunk rows of each external point: J[e][j]
__global__ void jac_reduce_kernel(const double *jrows, int n_ext, int n_chunks, int T, double *J) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)n_ext * T) return;
  const int e = (int)(idx / T), j = (int)(idx % T);
  double s = 0.0;
  for (int c = 0; c < n_chunks; ++c) s += jrows[((size_t)e * n_chunks + c) * T + j];
  J[idx] = s;
}

// Launch geometry, shared memory and scratch of the adjoint kernels of a plan.
static int adjoint_setup(ffrg_ctx *ctx, Plan *pl, int model, void (**kern_out)(AdjArgs)) {
  void (*kern)(AdjArgs) = model == FFRG_MODEL_D3 ? d3_adjoint : d4_adjoint;
  *kern_out = kern;
  if (pl->adj_grid) return FFRG_OK;
  const int nw = kAdjThreads / 32;
  size_t smem = (((size_t)pl->tab_count * 8 + 15) & ~(size_t)15) +
                ((((size_t)(3 * pl->na1 + 2 * pl->na2)) * 8 + 15) & ~(size_t)15) + (size_t)nw * pl->tab_count * 8;
  if (smem > 200 * 1024) {
    ctx->last_error = "adjoint: tables too large for per-warp shared-memory gradients";
    return FFRG_EINVAL;
  }
  int st = ensure_smem_limit(ctx, (const void *)kern, smem);
  if (st) return st;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kAdjThreads, smem);
  if (e != cudaSuccess || per_sm < 1) return set_cuda_error(ctx, e ? e : cudaErrorInvalidConfiguration, "occupancy");
  int grid = std::max(1, std::min(pl->n_items, per_sm * ctx->num_sms));
  st = dev_alloc(ctx, (void **)&pl->radD, (size_t)pl->nr * pl->nfreq * sizeof(double));
  if (!st) st = dev_alloc(ctx, (void **)&pl->gpart, (size_t)grid * pl->tab_count * sizeof(double));
  if (st) return st;
  pl->adj_smem = smem;
  pl->adj_grid = grid;
  return FFRG_OK;
}

// Full Jacobian d out_e / d T_j (row-major n_ext x table values) at scale k.
int launch_jacobian(ffrg_ctx *ctx, const ffrg_problem *pb, const ffrg_table_desc *td, const double *tab, double k,
                    double *J, cudaStream_t s) {
  if (pb->model != FFRG_MODEL_D3 && pb->model != FFRG_MODEL_D4_VERTEX) return FFRG_EINVAL;
  int st = validate_problem(pb, td);
  if (st) return st;
  Plan *pl = nullptr;
  st = get_plan(ctx, pb, td, &pl);
  if (st) return st;
  void (*kern)(AdjArgs) = nullptr;
  st = adjoint_setup(ctx, pl, pb->model, &kern);
  if (st) return st;
  if (!pl->jrows) {
    st = dev_alloc(ctx, (void **)&pl->jrows, (size_t)pl->n_items * pl->tab_count * sizeof(double));
    if (st) return st;
  }
  AdjArgs A;
  memset(&A, 0, sizeof(A));
  fill_args(pl, pb, td, tab, k, A.a);
  A.a.status = ctx->status_dev;
  A.a.cr = pl->cr;  // block-sized work items
  A.a.jb = pl->jb;
  A.a.n_chunks = pl->n_chunks;
  A.a.n_items = pl->n_items;
  A.a.radD = pl->radD;
  A.jrows = pl->jrows;
  st = launch_precompute(ctx, A.a, s);
  if (st) return st;
  kern<<<pl->adj_grid, kAdjThreads, pl->adj_smem, s>>>(A);
  const size_t tot = (size_t)pl->n_ext * pl->tab_count;
  jac_reduce_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(pl->jrows, pl->n_ext, pl->n_chunks, pl->tab_count, J);
  return set_cuda_error(ctx, cudaGetLastError(), "jacobian launch");
}

}  // namespace ffrg

extern "C" int ffrg_rhs_jacobian(ffrg_ctx *ctx, const ffrg_problem *pb, const ffrg_tables *tables, double k,
                                 double *J_dev, void *stream) {
  if (!ctx || !pb || !tables || !J_dev || !(k > 0.0) || !isfinite(k)) return FFRG_EINVAL;
  cudaSetDevice(ctx->device);
  return launch_jacobian(ctx, pb, &tables->desc, tables->dev, k, J_dev, (cudaStream_t)stream);
}

extern "C" int ffrg_rhs_adjoint(ffrg_ctx *ctx, const ffrg_problem *pb, const ffrg_tables *tables, double k,
                                const double *gbar_dev, double *tbar_dev, int precision, void *stream) {
  if (!ctx || !pb || !tables || !gbar_dev || !tbar_dev) return FFRG_EINVAL;
  if (!(k > 0.0) || !isfinite(k)) return FFRG_EINVAL;
  if (precision != FFRG_FP64) return FFRG_EINVAL;
  if (pb->model != FFRG_MODEL_D3 && pb->model != FFRG_MODEL_D4_VERTEX) return FFRG_EINVAL;
  int st = validate_problem(pb, &tables->desc);
  if (st) return st;
  cudaSetDevice(ctx->device);
  Plan *pl = nullptr;
  st = get_plan(ctx, pb, &tables->desc, &pl);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;
  void (*kern)(AdjArgs) = nullptr;
  st = adjoint_setup(ctx, pl, pb->model, &kern);
  if (st) return st;
  AdjArgs A;
  memset(&A, 0, sizeof(A));
  fill_args(pl, pb, &tables->desc, tables->dev, k, A.a);
  A.a.status = ctx->status_dev;
  A.a.cr = pl->cr;  // block-sized work items
  A.a.jb = pl->jb;
  A.a.n_chunks = pl->n_chunks;
  A.a.n_items = pl->n_items;
  A.a.radD = pl->radD;
  A.gbar = gbar_dev;
  A.gpart = pl->gpart;
  st = launch_precompute(ctx, A.a, s);
  if (st) return st;
  kern<<<pl->adj_grid, kAdjThreads, pl->adj_smem, s>>>(A);
  adj_reduce_kernel<<<(pl->tab_count + 255) / 256, 256, 0, s>>>(pl->gpart, pl->adj_grid, pl->tab_count, tbar_dev);
  return set_cuda_error(ctx, cudaGetLastError(), "adjoint launch");
}
