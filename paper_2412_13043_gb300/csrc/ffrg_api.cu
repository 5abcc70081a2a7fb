// Host side of the ffrg C ABI: contexts, dressing tables, quadrature rules,
// launch plans and argument validation (see include/ffrg.h for the contract).
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "ffrg_internal.cuh"

using namespace ffrg;

namespace ffrg {

int ensure_smem_limit(ffrg_ctx *ctx, const void *func, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<const void *, int>, size_t> limits;
  std::lock_guard<std::mutex> lock(mu);
  size_t &cur = limits[{func, ctx->device}];
  if (bytes <= cur) return FFRG_OK;
  cudaError_t e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return set_cuda_error(ctx, e, "cudaFuncSetAttribute");
  cur = bytes;
  return FFRG_OK;
}

int set_cuda_error(ffrg_ctx *ctx, cudaError_t e, const char *what) {
  if (e == cudaSuccess) return FFRG_OK;
  if (ctx) {
    char buf[256];
    snprintf(buf, sizeof(buf), "%s: %s (%d)", what, cudaGetErrorString(e), (int)e);
    ctx->last_error = buf;
  }
  if (e == cudaErrorMemoryAllocation) return FFRG_ENOMEM;
  return FFRG_ECUDA;
}

int dev_alloc(ffrg_ctx *ctx, void **p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  if (ctx->budget && ctx->used + bytes > ctx->budget) {
    ctx->last_error = "HBM budget exceeded";
    return FFRG_ENOMEM;
  }
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    return set_cuda_error(ctx, e, "cudaMalloc");
  }
  ctx->used += bytes;
  return FFRG_OK;
}

void dev_free(ffrg_ctx *ctx, void *p, size_t bytes) {
  if (!p) return;
  if (bytes == 0) bytes = 16;
  cudaFree(p);
  ctx->used = ctx->used >= bytes ? ctx->used - bytes : 0;
}

// Gauss-Legendre on [a,b].  Roots of P_n by Newton iteration in long double
// starting from the asymptotic guess cos(pi (i - 1/4)/(n + 1/2)); P_n and P_n'
// from the three-term recurrence (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}.
int host_gauss_legendre(int n, double a, double b, double *x, double *w) {
  if (n < 1 || n > kMaxNodes || !x || !w) return FFRG_EINVAL;
  const long double pi = 3.141592653589793238462643383279502884L;
  int half = (n + 1) / 2;
  for (int i = 1; i <= half; ++i) {
    long double z = cosl(pi * ((long double)i - 0.25L) / ((long double)n + 0.5L));
    long double dp = 1.0L;
    for (int it = 0; it < 60; ++it) {
      long double pkm1 = 1.0L, pk = z;
      for (int kk = 1; kk < n; ++kk) {
        long double pkp1 = ((2.0L * kk + 1.0L) * z * pk - (long double)kk * pkm1) / (long double)(kk + 1);
        pkm1 = pk;
        pk = pkp1;
      }
      if (n == 1) { pk = z; pkm1 = 1.0L; }
      dp = (long double)n * (pkm1 - z * pk) / (1.0L - z * z);
      long double dz = pk / dp;
      z -= dz;
      if (fabsl(dz) < 1e-19L) {
        // derivative at the final iterate
        pkm1 = 1.0L;
        pk = z;
        for (int kk = 1; kk < n; ++kk) {
          long double pkp1 = ((2.0L * kk + 1.0L) * z * pk - (long double)kk * pkm1) / (long double)(kk + 1);
          pkm1 = pk;
          pk = pkp1;
        }
        if (n == 1) { pk = z; pkm1 = 1.0L; }
        dp = (long double)n * (pkm1 - z * pk) / (1.0L - z * z);
        break;
      }
    }
    long double wi = 2.0L / ((1.0L - z * z) * dp * dp);
    long double mid = 0.5L * ((long double)a + (long double)b), hw = 0.5L * ((long double)b - (long double)a);
    // i-th root counted from +1: goes to index n-i (ascending order)
    x[n - i] = (double)(mid + hw * z);
    x[i - 1] = (double)(mid - hw * z);
    w[n - i] = (double)(hw * wi);
    w[i - 1] = (double)(hw * wi);
    if (2 * i - 1 == n) x[i - 1] = (double)mid;
  }
  return FFRG_OK;
}

// Gauss-Chebyshev of the second kind: x_j = cos(j pi/(n+1)), w_j = pi/(n+1) sin^2(j pi/(n+1)).
int host_gauss_chebyshev2(int n, double *x, double *w) {
  if (n < 1 || n > kMaxNodes || !x || !w) return FFRG_EINVAL;
  const long double pi = 3.141592653589793238462643383279502884L;
  for (int j = 1; j <= n; ++j) {
    long double th = (long double)j * pi / (long double)(n + 1);
    long double s = sinl(th);
    x[j - 1] = (double)cosl(th);
    w[j - 1] = (double)(pi / (long double)(n + 1) * s * s);
  }
  return FFRG_OK;
}

static int tables_needed(int model) {
  switch (model) {
  case FFRG_MODEL_D3: return 1;
  case FFRG_MODEL_D4_VERTEX:
  case FFRG_MODEL_D4_FULL: return 3;
  case FFRG_MODEL_FINITE_T:
  case FFRG_MODEL_FINITE_T_4D: return 2;
  default: return -1;
  }
}

static int desc_ok(const ffrg_table_desc *td) {
  if (!td) return 0;
  if (td->n_tables < 1 || td->n_tables > 8 || td->n_stack < 1 || td->n_pts < 2 || td->n_pts > kMaxPts) return 0;
  if (!(td->x_min > 0.0) || !(td->x_max > td->x_min) || !isfinite(td->x_max)) return 0;
  if ((long long)td->n_tables * td->n_stack * td->n_pts > (1LL << 22)) return 0;
  return 1;
}

int validate_problem(const ffrg_problem *pb, const ffrg_table_desc *td) {
  if (!pb) return FFRG_EINVAL;
  int need = tables_needed(pb->model);
  if (need < 0) return FFRG_EINVAL;
  if (pb->regulator != FFRG_REG_EXP && pb->regulator != FFRG_REG_LITIM) return FFRG_EINVAL;
  if (pb->n_rad < 1 || pb->n_rad > 4096 || pb->n_ang1 < 1 || pb->n_ang1 > 1024) return FFRG_EINVAL;
  if (pb->n_ext_p < 1 || pb->n_ext_p > (1 << 20)) return FFRG_EINVAL;
  if (!(pb->p_min > 0.0) || !(pb->p_max >= pb->p_min) || !isfinite(pb->p_max)) return FFRG_EINVAL;
  if (!(pb->qmax_over_k > 0.0) || !isfinite(pb->qmax_over_k)) return FFRG_EINVAL;
  if (!isfinite(pb->m2_over_k2) || !isfinite(pb->m2_shift) || !isfinite(pb->lam) || !isfinite(pb->prefactor))
    return FFRG_EINVAL;
  if (is_d4(pb->model)) {
    if (pb->n_ang2 < 1 || pb->n_ang2 > 1024 || pb->n_ext_ang < 1 || pb->n_ext_ang > 1024) return FFRG_EINVAL;
  }
  if (pb->model == FFRG_MODEL_D4_FULL) {
    if (pb->n_va < 1 || pb->n_vb < 1 || pb->n_va > 64 || pb->n_vb > 64) return FFRG_EINVAL;
  } else if (pb->n_va > 1 || pb->n_vb > 1) {
    return FFRG_EINVAL;
  }
  if (pb->model == FFRG_MODEL_FINITE_T || pb->model == FFRG_MODEL_FINITE_T_4D) {
    if (pb->n_ext_ang < 1 || pb->n_ext_ang > 1024 || pb->n_matsubara < 0 || pb->n_matsubara > 4096) return FFRG_EINVAL;
    if (!(pb->T > 0.0) || !isfinite(pb->T)) return FFRG_EINVAL;
    if (pb->statistics != FFRG_STAT_BOSE && pb->statistics != FFRG_STAT_FERMI) return FFRG_EINVAL;
  } else if (pb->statistics != FFRG_STAT_BOSE) {
    return FFRG_EINVAL;
  }
  if (pb->model == FFRG_MODEL_FINITE_T_4D) {
    if (pb->n_x0 < 1 || pb->n_x0 > 4096) return FFRG_EINVAL;
    if (pb->statistics == FFRG_STAT_FERMI && pb->n_ext_ang != 1) return FFRG_EINVAL;  // one fermion leg frequency
  } else if (pb->n_x0 != 0) {
    return FFRG_EINVAL;
  }
  if (td) {
    if (!desc_ok(td)) return FFRG_EINVAL;
    if (td->n_tables < need) return FFRG_EINVAL;
    if (pb->model == FFRG_MODEL_D4_FULL) {
      if (td->n_stack != pb->n_va * pb->n_vb) return FFRG_EINVAL;
    } else if (pb->model != FFRG_MODEL_FINITE_T && td->n_stack != 1) {   // FINITE_T_4D: one row per table
      return FFRG_EINVAL;
    }
  }
  if (ffrg_n_ext(pb) < 1) return FFRG_EINVAL;
  return FFRG_OK;
}

static int upload_rule(ffrg_ctx *ctx, const std::vector<double> &h, double **d) {
  int st = dev_alloc(ctx, (void **)d, h.size() * sizeof(double));
  if (st) return st;
  cudaError_t e = cudaMemcpy(*d, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice);
  return set_cuda_error(ctx, e, "cudaMemcpy(rule)");
}

static void plan_free(ffrg_ctx *ctx, Plan *pl) {
  if (!pl) return;
  double *arrs[] = {pl->rad_x, pl->rad_w, pl->a1_x, pl->a1_w, pl->a2_x, pl->a2_w, pl->psi_x, pl->psi_w,
                    pl->radF, pl->radq, pl->partial, pl->radD, pl->gpart, pl->ext_pd, pl->psi_s, pl->jrows};
  for (double *p : arrs) dev_free(ctx, p, 0);
  dev_free(ctx, pl->tab32, 0);
  dev_free(ctx, pl->radq32, 0);
  dev_free(ctx, pl->work_ctr, 0);
  dev_free(ctx, pl->ext_done, 0);
  dev_free(ctx, pl->kconst, 0);
  dev_free(ctx, pl->radF32, 0);
  dev_free(ctx, pl->tabc, 0);
  dev_free(ctx, pl->kbuf, 0);
  delete pl;
}

// Launch geometry: rows of angle work are grouped into work items (external
// point x chunk of outer rows).  The block-sized items (about two rows of at
// most 8 angle nodes per thread of a 256-thread CTA) serve the adjoint
// kernels.  The forward kernels give each item to one warp: the partial sum
// needs only shuffles, no block barrier, and little FP64 reduction work.
void plan_geometry(Plan *pl, const ffrg_problem *pb, const ffrg_table_desc *td) {
  pl->model = pb->model;
  pl->nr = pb->n_rad;
  pl->na1 = pb->n_ang1;
  pl->na2 = is_d4(pb->model) ? pb->n_ang2 : pb->model == FFRG_MODEL_FINITE_T_4D ? pb->n_x0 : 1;
  pl->n_ext_ang = pb->n_ext_ang;
  pl->n_ext_p = pb->n_ext_p;
  const bool ft = pb->model == FFRG_MODEL_FINITE_T || pb->model == FFRG_MODEL_FINITE_T_4D;
  pl->N = ft ? pb->n_matsubara : 0;
  pl->stat = ft ? pb->statistics : FFRG_STAT_BOSE;
  pl->nfreq = 2 * pl->N + 1 + (pl->stat == FFRG_STAT_FERMI ? 1 : 0);
  // FINITE_T_4D: rows of loop frequencies, the Matsubara cap or the quadrature nodes
  if (pb->model == FFRG_MODEL_FINITE_T_4D) pl->nfreq = std::max(pl->nfreq, pb->n_x0);
  pl->include_p0 = pb->include_p0;
  pl->n_ext = ffrg_n_ext(pb);
  pl->n_tables = td->n_tables;
  pl->n_stack = td->n_stack;
  pl->n_pts = td->n_pts;
  pl->tab_count = td->n_tables * td->n_stack * td->n_pts;
  // FP32 layout: (value, difference) node pairs; finite T: (Z, lambda) node
  // pairs per stack row plus one zero pair (same bytes as single values)
  // D4_FULL: compact [Z row 0 | lambda4 row 0 | lambda3 rows] in both precisions
  pl->n_va = pb->model == FFRG_MODEL_D4_FULL ? pb->n_va : 1;
  pl->n_vb = pb->model == FFRG_MODEL_D4_FULL ? pb->n_vb : 1;
  pl->tabc_count = pb->model == FFRG_MODEL_D4_FULL ? (2 + pl->n_va * pl->n_vb) * td->n_pts : 0;
  pl->tab32_count = pb->model == FFRG_MODEL_FINITE_T ? td->n_stack * td->n_pts + 1
                    : pl->tabc_count                 ? pl->tabc_count
                                                     : pl->tab_count;
  int outer_total, rows_per_outer;
  if (is_d4(pb->model)) {
    pl->jb = pl->na2;
    outer_total = pl->nr;
    rows_per_outer = pl->na1;
  } else {
    pl->jb = std::min(pl->na1, 8);
    outer_total = pl->nr * pl->nfreq;
    rows_per_outer = (pl->na1 + pl->jb - 1) / pl->jb;
  }
  auto chunk = [&](int target_rows) {
    return std::min(std::max(1, (target_rows + rows_per_outer - 1) / rows_per_outer), outer_total);
  };
  pl->cr = chunk(2 * kThreads);
  pl->n_chunks = (outer_total + pl->cr - 1) / pl->cr;
  pl->n_items = pl->n_ext * pl->n_chunks;
  // Forward (warp-sized) items.  d=4: rows (radial, first angle), about
  // eight per lane.  d=3 / finite T: rows = outer index x block of angle
  // nodes; a warp item takes a multiple of 32 rows (1..8 per lane), sized for
  // about eight items per resident warp of a 152-SM GPU.  The mixed kernels
  // keep whole angle rules per row (splitting them was measured slower, also
  // for the serving kernels, which use this geometry so that they compute
  // exactly what the single-flow kernels do).  The FP64 kernels split the
  // angle rule into blocks of at least 4 nodes until there is a row per
  // resident lane: small FP64 problems are bound by each lane's FP64 chain.
  const long long kTargetItems = 8LL * 152 * 32;
  auto forward = [&](bool fp64, int &fcr, int &fn_chunks, int &fn_items, int &fjb) {
    if (is_d4(pb->model)) {
      fjb = pl->na2;
      fcr = chunk(8 * 32);
      fn_chunks = (outer_total + fcr - 1) / fcr;
      fn_items = pl->n_ext * fn_chunks;
    } else if (pb->model == FFRG_MODEL_FINITE_T) {
      // rows of K: (stack row j, |p|) x radial node, the whole angle rule per row
      fjb = pl->na1;
      const long long n_outer = (long long)(pl->N + pl->n_ext_ang) * pl->n_ext_p;
      long long rpi = (n_outer * pl->nr + kTargetItems - 1) / kTargetItems;
      rpi = std::min<long long>(std::max<long long>((rpi + 31) / 32 * 32, 32), 256);
      fcr = (int)std::min<long long>(rpi, pl->nr);
      fn_chunks = (pl->nr + fcr - 1) / fcr;
      fn_items = (int)(n_outer * fn_chunks);
    } else {
      const long long total_outer = (long long)pl->n_ext * outer_total;
      const long long kRowsWanted = 152LL * 2048;
      long long nblk = fp64 ? (kRowsWanted + total_outer - 1) / total_outer : 1;
      nblk = std::max<long long>(1, std::min<long long>(nblk, (pl->na1 + 3) / 4));
      fjb = (int)((pl->na1 + nblk - 1) / nblk);
      nblk = (pl->na1 + fjb - 1) / fjb;
      const int rows_ext = outer_total * (int)nblk;
      long long rpi = ((long long)pl->n_ext * rows_ext + kTargetItems - 1) / kTargetItems;
      rpi = std::min<long long>(std::max<long long>((rpi + 31) / 32 * 32, 32), 256);
      fcr = (int)std::min<long long>(rpi, rows_ext);
      fn_chunks = (rows_ext + fcr - 1) / fcr;
      fn_items = pl->n_ext * fn_chunks;
    }
  };
  pl->kbuf_count = pb->model == FFRG_MODEL_FINITE_T
                       ? (size_t)(pl->N + pl->n_ext_ang) * pl->n_ext_p * pl->nr
                   : pb->model == FFRG_MODEL_FINITE_T_4D ? (size_t)2 * pl->nfreq + 2   // frequency set of the scale
                                                         : 0;
  forward(false, pl->fcr, pl->fn_chunks, pl->fn_items, pl->fjb);
  forward(true, pl->fcr64, pl->fn_chunks64, pl->fn_items64, pl->fjb64);
  // shared memory: tables + angle rules (+ sqrt(1-c1^2) for D4), 16-byte aligned regions
  auto al16 = [](size_t b) { return (b + 15) & ~(size_t)15; };
  const size_t ang = (size_t)pl->na1 * 3 + (size_t)pl->na2 * 2;
  const size_t ang32 = ang + (size_t)4 * ((pl->na2 + 1) / 2);   // + second-angle node pairs
  pl->smem64 = al16((size_t)(pl->tabc_count ? pl->tabc_count : pl->tab_count) * 8) + al16(ang * 8);
  // D4_FULL, mixed: lambda3 as cell polynomials (two float4 per (a, b, S0)
  // cell) after the Z and lambda4 line rows, when that fits in shared memory
  pl->l3cell = 0;
  if (pb->model == FFRG_MODEL_D4_FULL) {
    const int cells = 2 * td->n_pts + 4 * pl->n_va * pl->n_vb * td->n_pts;
    if (al16((size_t)cells * 8) + al16(ang32 * 4) <= kMaxDynSmemBytes) {
      pl->l3cell = 1;
      pl->tab32_count = cells;
    }
  }
  pl->smem32 = al16((size_t)pl->tab32_count * 8) + al16(ang32 * 4);
  pl->smem64g = al16(ang * 8);
}

int get_plan(ffrg_ctx *ctx, const ffrg_problem *pb, const ffrg_table_desc *td, Plan **out) {
  std::vector<long long> key = {pb->model, pb->n_rad, pb->n_ang1, pb->n_ang2, pb->n_ext_p, pb->n_ext_ang,
                                pb->n_matsubara, pb->include_p0, td->n_tables, td->n_stack, td->n_pts,
                                pb->model == FFRG_MODEL_FINITE_T ? pb->statistics : 0,
                                pb->model == FFRG_MODEL_D4_FULL ? pb->n_va : 1,
                                pb->model == FFRG_MODEL_D4_FULL ? pb->n_vb : 1,
                                pb->model == FFRG_MODEL_FINITE_T_4D ? pb->n_x0 : 0};
  auto it = ctx->plans.find(key);
  if (it != ctx->plans.end()) {
    *out = it->second;
    return FFRG_OK;
  }
  Plan *pl = new Plan();  // value-initialised: pointers null, counts zero
  pl->key = key;
  plan_geometry(pl, pb, td);

  int st = FFRG_OK;
  std::vector<double> x(pl->nr), w(pl->nr);
  host_gauss_legendre(pl->nr, 0.0, 1.0, x.data(), w.data());
  st = st ? st : upload_rule(ctx, x, &pl->rad_x);
  st = st ? st : upload_rule(ctx, w, &pl->rad_w);
  std::vector<double> x1(pl->na1), w1(pl->na1);
  if (is_d4(pb->model)) host_gauss_chebyshev2(pl->na1, x1.data(), w1.data());
  else host_gauss_legendre(pl->na1, -1.0, 1.0, x1.data(), w1.data());
  st = st ? st : upload_rule(ctx, x1, &pl->a1_x);
  st = st ? st : upload_rule(ctx, w1, &pl->a1_w);
  std::vector<double> x2(pl->na2), w2(pl->na2);
  host_gauss_legendre(pl->na2, -1.0, 1.0, x2.data(), w2.data());
  pl->sum_w2 = 0.0;
  for (double v : w2) pl->sum_w2 += v;
  st = st ? st : upload_rule(ctx, x2, &pl->a2_x);
  st = st ? st : upload_rule(ctx, w2, &pl->a2_w);
  int npsi = std::max(1, pl->n_ext_ang);
  std::vector<double> xp(npsi), wp(npsi);
  host_gauss_legendre(npsi, -1.0, 1.0, xp.data(), wp.data());
  pl->psi_w_host = wp;
  st = st ? st : upload_rule(ctx, xp, &pl->psi_x);
  st = st ? st : upload_rule(ctx, wp, &pl->psi_w);
  size_t nF = (size_t)pl->nr * pl->nfreq;
  if (!st) st = dev_alloc(ctx, (void **)&pl->radF, nF * sizeof(double));
  if (!st) st = dev_alloc(ctx, (void **)&pl->radF32, nF * sizeof(float));
  if (!st) st = dev_alloc(ctx, (void **)&pl->radq, pl->nr * sizeof(double));
  if (!st) st = dev_alloc(ctx, (void **)&pl->radq32, pl->nr * sizeof(float));
  // work_ctr[0]: item counter of the main kernels; [1..4]: grid counters of
  // the finite-T mixed single-launch RHS (all zero at the start)
  if (!st) st = dev_alloc(ctx, (void **)&pl->work_ctr, 5 * sizeof(unsigned));
  if (!st) st = set_cuda_error(ctx, cudaMemset(pl->work_ctr, 0, 5 * sizeof(unsigned)), "cudaMemset(counters)");
  if (!st) st = dev_alloc(ctx, (void **)&pl->ext_done, (size_t)pl->n_ext * sizeof(unsigned));
  if (!st) st = dev_alloc(ctx, (void **)&pl->kconst, kKConstBytes);
  if (!st && pl->tabc_count) st = dev_alloc(ctx, (void **)&pl->tabc, (size_t)pl->tabc_count * sizeof(double));
  if (!st && pl->kbuf_count) st = dev_alloc(ctx, (void **)&pl->kbuf, pl->kbuf_count * sizeof(double));
  if (!st) st = dev_alloc(ctx, (void **)&pl->ext_pd, (size_t)pl->n_ext_p * sizeof(double));
  if (!st) st = dev_alloc(ctx, (void **)&pl->psi_s, (size_t)npsi * sizeof(double));
  if (!st)
    st = dev_alloc(ctx, (void **)&pl->partial, (size_t)std::max(pl->fn_items, pl->fn_items64) * sizeof(double));
  if (!st) st = dev_alloc(ctx, (void **)&pl->tab32,
                          (size_t)std::max(pl->tab_count, pl->tab32_count) * sizeof(float2));
  if (st) {
    plan_free(ctx, pl);
    return st;
  }
  *out = pl;
  ctx->plans[key] = pl;
  return FFRG_OK;
}

void fill_args(const Plan *pl, const ffrg_problem *pb, const ffrg_table_desc *td, const double *tab, double k,
               RhsArgs &a) {
  memset(&a, 0, sizeof(a));
  a.model = pb->model;
  a.reg = pb->regulator;
  a.nr = pl->nr;
  a.na1 = pl->na1;
  a.na2 = pl->na2;
  a.n_ext_p = pl->n_ext_p;
  a.n_ext_ang = pl->n_ext_ang;
  a.N = pl->N;
  a.stat = pl->stat;
  a.nfreq = pl->nfreq;
  a.include_p0 = pl->include_p0;
  a.n_ext = pl->n_ext;
  a.n_tables = td->n_tables;
  a.n_stack = td->n_stack;
  a.n_pts = td->n_pts;
  a.tab_count = pl->tab_count;
  a.cr = pl->fcr;
  a.n_chunks = pl->fn_chunks;
  a.n_items = pl->fn_items;
  a.jb = pl->fjb;
  a.tab32_count = pl->tab32_count;
  a.tabc_count = pl->tabc_count;
  a.n_va = pl->n_va;
  a.n_vb = pl->n_vb;
  a.l3cell = pl->l3cell;
  a.tabc = pl->tabc;
  a.kbuf = pl->kbuf;
  a.k = k;
  a.m2_over_k2 = pb->m2_over_k2;
  a.m2_shift = pb->m2_shift;
  a.T = pb->T;
  a.p_min = pb->p_min;
  a.p_ratio_step = pb->n_ext_p > 1 ? log(pb->p_max / pb->p_min) / (pb->n_ext_p - 1) : 0.0;
  a.qmax_over_k = pb->qmax_over_k;
  const double pi = kPi;
  switch (pb->model) {
  case FFRG_MODEL_D3: a.norm = pb->prefactor * pb->lam * pb->lam / (4.0 * pi * pi); break;
  case FFRG_MODEL_D4_VERTEX:
  case FFRG_MODEL_D4_FULL: a.norm = pb->prefactor / (8.0 * pi * pi * pi); break;
  case FFRG_MODEL_FINITE_T_4D: a.norm = pb->prefactor * pb->lam * pb->lam / (4.0 * pi * pi); break;  // T in the frequency weights
  default: a.norm = pb->prefactor * pb->lam * pb->lam * pb->T / (4.0 * pi * pi); break;
  }
  double lr = log(td->x_max / td->x_min);
  a.u_scale = 0.5 * (td->n_pts - 1) / lr;
  a.u_off = -(td->n_pts - 1) * log(td->x_min) / lr;
  a.x_min2 = td->x_min * td->x_min;
  // k-independent parts of the table coordinates (the kernels add the k-dependent shift)
  const double nm1 = td->n_pts - 1;
  a.us1f = (float)(a.u_scale * 0.6931471805599453094 / nm1);
  a.us1 = a.u_scale / nm1;
  for (int c = 1; c <= 4; ++c) {
    a.uoc[c - 1] = a.u_off - a.u_scale * log((double)c);
    a.uoc1[c - 1] = a.uoc[c - 1] / nm1;
  }
  a.twopiT = 2.0 * kPi * pb->T;
  a.sum_w2 = pl->sum_w2;
  // FP32 scale constants of this k on the host (the kernels use them unless a
  // flow stage sets k_dev or m2_dev later); every field they read is set above
  a.kc_host = kconst_f32(a, k, a.m2_over_k2 * k * k + a.m2_shift);
  a.kc_host_ok = 1;
  a.tab = tab;
  a.tab32 = pl->tab32;
  a.rad_x = pl->rad_x;
  a.rad_w = pl->rad_w;
  a.a1_x = pl->a1_x;
  a.a1_w = pl->a1_w;
  a.a2_x = pl->a2_x;
  a.a2_w = pl->a2_w;
  a.psi_x = pl->psi_x;
  a.radF = pl->radF;
  a.radq = pl->radq;
  a.radq32 = pl->radq32;
  a.radF32 = pl->radF32;
  a.work_ctr = pl->work_ctr;
  a.fused_ctr = pb->model == FFRG_MODEL_FINITE_T ? pl->work_ctr + 1 : nullptr;
  a.ext_done = pl->ext_done;
  a.kconst = pl->kconst;
  a.ext_pd = pl->ext_pd;
  a.psi_s = pl->psi_s;
  a.partial = pl->partial;
}

}  // namespace ffrg

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

int ffrg_create(ffrg_ctx **out, int device, size_t hbm_budget_bytes) {
  if (!out) return FFRG_EINVAL;
  *out = nullptr;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess) return FFRG_ECUDA;
  if (device < 0 || device >= ndev) return FFRG_EINVAL;
  e = cudaSetDevice(device);
  if (e != cudaSuccess) return FFRG_ECUDA;
  ffrg_ctx *ctx = new ffrg_ctx();
  ctx->device = device;
  ctx->budget = hbm_budget_bytes;
  ctx->used = 0;
  ctx->status_dev = nullptr;
  ctx->status_host = nullptr;
  ctx->server = nullptr;
  ctx->profiling = 0;
  ctx->prof_used = 0;
  cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
  int st = dev_alloc(ctx, (void **)&ctx->status_dev, sizeof(unsigned) * 4);
  if (!st) st = set_cuda_error(ctx, cudaMemset(ctx->status_dev, 0, sizeof(unsigned) * 4), "cudaMemset");
  if (!st) st = set_cuda_error(ctx, cudaMallocHost((void **)&ctx->status_host, sizeof(unsigned) * 4), "cudaMallocHost");
  if (st) {
    ffrg_destroy(ctx);
    return st;
  }
  *out = ctx;
  return FFRG_OK;
}

int ffrg_destroy(ffrg_ctx *ctx) {
  if (!ctx) return FFRG_EINVAL;
  if (ctx->server) ffrg_serve_stop(ctx);
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  for (auto &kv : ctx->plans) {
    Plan *pl = kv.second;
    double *arrs[] = {pl->rad_x, pl->rad_w, pl->a1_x, pl->a1_w, pl->a2_x, pl->a2_w, pl->psi_x, pl->psi_w,
                      pl->radF, pl->radq, pl->partial, pl->radD, pl->gpart, pl->ext_pd, pl->psi_s, pl->jrows};
    for (double *p : arrs) cudaFree(p);
    cudaFree(pl->tab32);
    cudaFree(pl->radq32);
    cudaFree(pl->work_ctr);
    cudaFree(pl->ext_done);
    cudaFree(pl->kconst);
    cudaFree(pl->radF32);
    cudaFree(pl->tabc);
    cudaFree(pl->kbuf);
    delete pl;
  }
  ctx->plans.clear();
  for (void *p : ctx->owned) cudaFree(p);
  for (cudaEvent_t e : ctx->prof_events) cudaEventDestroy(e);
  if (ctx->flow_dev) cudaFree(ctx->flow_dev);
  if (ctx->host_out_dev) cudaFree(ctx->host_out_dev);
  if (ctx->states_dev) cudaFree(ctx->states_dev);
  if (ctx->flow_host) cudaFreeHost(ctx->flow_host);
  if (ctx->flow_ev) cudaEventDestroy(ctx->flow_ev);
  if (ctx->flow_stream) cudaStreamDestroy(ctx->flow_stream);
  if (ctx->status_dev) cudaFree(ctx->status_dev);
  if (ctx->status_host) cudaFreeHost(ctx->status_host);
  delete ctx;
  return FFRG_OK;
}

int ffrg_quad_nodes(int rule, int n, double a, double b, double *x, double *w) {
  if (rule == FFRG_RULE_GL) {
    if (!isfinite(a) || !isfinite(b)) return FFRG_EINVAL;
    return host_gauss_legendre(n, a, b, x, w);
  }
  if (rule == FFRG_RULE_GC2) return host_gauss_chebyshev2(n, x, w);
  return FFRG_EINVAL;
}

int ffrg_tables_upload(ffrg_ctx *ctx, const ffrg_table_desc *desc, const double *values, int values_on_device,
                       ffrg_tables **out, void *stream) {
  if (!ctx || !desc || !values || !out) return FFRG_EINVAL;
  *out = nullptr;
  if (!desc_ok(desc)) return FFRG_EINVAL;
  cudaSetDevice(ctx->device);
  ffrg_tables *t = new ffrg_tables();
  t->desc = *desc;
  t->count = (size_t)desc->n_tables * desc->n_stack * desc->n_pts;
  t->bytes = ((t->count * sizeof(double)) + 255) & ~(size_t)255;
  int st = dev_alloc(ctx, (void **)&t->dev, t->bytes);
  if (st) {
    delete t;
    return st;
  }
  st = ffrg_tables_update(ctx, t, values, values_on_device, stream);
  if (st) {
    dev_free(ctx, t->dev, t->bytes);
    delete t;
    return st;
  }
  *out = t;
  return FFRG_OK;
}

int ffrg_tables_update(ffrg_ctx *ctx, ffrg_tables *t, const double *values, int values_on_device, void *stream) {
  if (!ctx || !t || !values) return FFRG_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(t->dev, values, t->count * sizeof(double),
                                  values_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s);
  return set_cuda_error(ctx, e, "cudaMemcpyAsync(tables)");
}

int ffrg_tables_free(ffrg_ctx *ctx, ffrg_tables *t) {
  if (!ctx || !t) return FFRG_EINVAL;
  cudaSetDevice(ctx->device);
  dev_free(ctx, t->dev, t->bytes);
  delete t;
  return FFRG_OK;
}

int ffrg_tables_device_ptr(const ffrg_tables *t, double **dev_values) {
  if (!t || !dev_values) return FFRG_EINVAL;
  *dev_values = t->dev;
  return FFRG_OK;
}

int ffrg_n_ext(const ffrg_problem *pb) {
  if (!pb || pb->n_ext_p < 1) return -1;
  switch (pb->model) {
  case FFRG_MODEL_D3: return pb->n_ext_p + (pb->include_p0 ? 1 : 0);
  case FFRG_MODEL_D4_FULL:
  case FFRG_MODEL_D4_VERTEX:
    if (pb->n_ext_ang < 1) return -1;
    return 2 * pb->n_ext_p + 1 + pb->n_ext_p * pb->n_ext_ang;
  case FFRG_MODEL_FINITE_T:
  case FFRG_MODEL_FINITE_T_4D:
    if (pb->n_ext_ang < 1) return -1;
    return pb->n_ext_p * pb->n_ext_ang;
  default: return -1;
  }
}

double ffrg_evals(const ffrg_problem *pb) {
  int ne = ffrg_n_ext(pb);
  if (ne < 0) return -1.0;
  double nodes = (double)pb->n_rad * pb->n_ang1;
  if (is_d4(pb->model)) nodes *= pb->n_ang2;
  if (pb->model == FFRG_MODEL_FINITE_T)
    nodes *= (2.0 * pb->n_matsubara + 1.0 + (pb->statistics == FFRG_STAT_FERMI ? 1.0 : 0.0));
  if (pb->model == FFRG_MODEL_FINITE_T_4D)   // at most: the Matsubara cap or the quadrature nodes
    nodes *= std::max(2.0 * pb->n_matsubara + 1.0 + (pb->statistics == FFRG_STAT_FERMI ? 1.0 : 0.0),
                      (double)pb->n_x0);
  return (double)ne * nodes;
}

int ffrg_rhs(ffrg_ctx *ctx, const ffrg_problem *pb, const ffrg_tables *tables, double k, double *out_dev,
             int precision, void *stream) {
  if (!ctx || !pb || !tables || !out_dev) return FFRG_EINVAL;
  if (!(k > 0.0) || !isfinite(k)) return FFRG_EINVAL;
  if (precision != FFRG_FP64 && precision != FFRG_MIXED) return FFRG_EINVAL;
  int st = validate_problem(pb, &tables->desc);
  if (st) return st;
  cudaSetDevice(ctx->device);
  Plan *pl = nullptr;
  st = get_plan(ctx, pb, &tables->desc, &pl);
  if (st) return st;
  RhsArgs a;
  fill_args(pl, pb, &tables->desc, tables->dev, k, a);
  a.out = out_dev;
  a.status = ctx->status_dev;
  return launch_rhs(ctx, pl, a, precision, (cudaStream_t)stream);
}

int ffrg_rhs_host(ffrg_ctx *ctx, const ffrg_problem *pb, const ffrg_tables *tables, double k, double *out_host,
                  int precision, void *stream) {
  if (!ctx || !pb || !tables || !out_host) return FFRG_EINVAL;
  const int ne = ffrg_n_ext(pb);
  if (ne < 0) return FFRG_EINVAL;
  const size_t bytes = (size_t)ne * sizeof(double);
  cudaSetDevice(ctx->device);
  // pinned, mapped host memory: the kernels write the outputs there
  // themselves (over the coherent CPU-GPU link), so no copy follows
  cudaPointerAttributes pa;
  if (cudaPointerGetAttributes(&pa, out_host) == cudaSuccess && pa.type == cudaMemoryTypeHost && pa.devicePointer)
    return ffrg_rhs(ctx, pb, tables, k, (double *)pa.devicePointer, precision, stream);
  cudaGetLastError();   // an unregistered pointer is not an error here
  if (ctx->host_out_cap < bytes) {   // grown on demand (cudaFree waits for the work that reads it)
    dev_free(ctx, ctx->host_out_dev, ctx->host_out_cap);
    ctx->host_out_dev = nullptr;
    ctx->host_out_cap = 0;
    int st = dev_alloc(ctx, &ctx->host_out_dev, bytes);
    if (st) return st;
    ctx->host_out_cap = bytes;
  }
  int st = ffrg_rhs(ctx, pb, tables, k, (double *)ctx->host_out_dev, precision, stream);
  if (st) return st;
  return set_cuda_error(ctx, cudaMemcpyAsync(out_host, ctx->host_out_dev, bytes, cudaMemcpyDeviceToHost,
                                             (cudaStream_t)stream),
                        "cudaMemcpyAsync(outputs)");
}

int ffrg_status_read(ffrg_ctx *ctx, void *stream) {
  if (!ctx) return FFRG_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(ctx->status_host, ctx->status_dev, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return set_cuda_error(ctx, e, "ffrg_status_read");
  unsigned v = ctx->status_host[0];
  e = cudaMemsetAsync(ctx->status_dev, 0, sizeof(unsigned), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return set_cuda_error(ctx, e, "ffrg_status_read");
  if (v & kStatusTimeout) return FFRG_ETIMEOUT;
  if (v & kStatusNonFinite) return FFRG_ENONFINITE;
  return FFRG_OK;
}

int ffrg_set_profiling(ffrg_ctx *ctx, int enable) {
  if (!ctx) return FFRG_EINVAL;
  cudaSetDevice(ctx->device);
  if (enable && ctx->prof_events.empty()) {
    ctx->prof_events.resize(2 * 4096);
    for (auto &e : ctx->prof_events) {
      cudaError_t err = cudaEventCreate(&e);
      if (err != cudaSuccess) return set_cuda_error(ctx, err, "cudaEventCreate");
    }
  }
  ctx->profiling = enable ? 1 : 0;
  ctx->prof_used = 0;
  return FFRG_OK;
}

int ffrg_profile_read(ffrg_ctx *ctx, double *main_ms, long long *launches) {
  if (!ctx || !main_ms || !launches) return FFRG_EINVAL;
  double tot = 0.0;
  for (int i = 0; i < ctx->prof_used; ++i) {
    cudaError_t err = cudaEventSynchronize(ctx->prof_events[2 * i + 1]);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, ctx->prof_events[2 * i], ctx->prof_events[2 * i + 1]);
    if (err != cudaSuccess) return set_cuda_error(ctx, err, "ffrg_profile_read");
    tot += ms;
  }
  *main_ms = tot;
  *launches = ctx->prof_used;
  ctx->prof_used = 0;
  return FFRG_OK;
}

const char *ffrg_strerror(int status) {
  switch (status) {
  case FFRG_OK: return "ok";
  case FFRG_EINVAL: return "invalid argument";
  case FFRG_ENOMEM: return "out of device memory or over the HBM budget";
  case FFRG_ENONFINITE: return "non-finite result";
  case FFRG_ESTEP_UNDERFLOW: return "step size underflow (rejected at minimal_dt)";
  case FFRG_EMAXSTEPS: return "maximum number of steps reached";
  case FFRG_ETIMEOUT: return "bounded device wait timed out";
  case FFRG_EPENDING: return "request pending";
  case FFRG_EBUSY: return "busy";
  case FFRG_ECUDA: return "CUDA error";
  case FFRG_ENOTFOUND: return "unknown ticket";
  case FFRG_ECANCELED: return "request cancelled";
  default: return "unknown status";
  }
}

const char *ffrg_last_error(const ffrg_ctx *ctx) {
  if (!ctx) return "";
  return ctx->last_error.c_str();
}

}  // extern "C"
