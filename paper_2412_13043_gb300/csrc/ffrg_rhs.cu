// Momentum-loop right-hand side on sm_103a: for every external point a sum
// over radial x angular (x Matsubara) quadrature nodes of regulator
// derivative x propagators x vertices read from dressing tables (Sec. 2.1
// Eq. GenfRG / FlowGamman; Sec. 5.3.2 quadrature integrators; App. F
// interpolators).
//
// Kernel sequence per RHS (one stream):
//   1. precompute: per radial node (and Matsubara index) the p-independent
//      factor F = w q^{d-1} dR(q) G(q)^2 [lam(n,q)] in FP64 (the paper's
//      generated kernels hoist repeated regulator/interpolator calls the same
//      way, Sec. 5.3.2), plus the FP32 mirror of the tables;
//   2. main: persistent CTAs walk work items (external point x chunk of
//      radial rows); tables are staged into shared memory by a TMA bulk copy
//      (cp.async.bulk + mbarrier, bounded wait); threads take angular rows,
//      accumulate in FP64 (FP64 path) or sum a row in FP32 and add it into an
//      FP64 accumulator (mixed path); a warp-shuffle + shared-memory tree
//      writes one partial per item;
//   3. finalize: fixed-order sum of the partials of each external point, the
//      overall normalisation, and a non-finite check into the status word.
// The reduction order depends only on the problem shape, never on the grid
// size or on other work in flight.
#include <math.h>

#include <algorithm>

#include "ffrg_internal.cuh"

namespace ffrg {

// FP64 propagator with the FP64 global table.
__device__ __forceinline__ double prop_fp64_global(const RhsArgs &a, const double *zrow, double s2, double om2,
                                                   double m2, double k2, double inv_k2) {
  s2 = fmax(s2, 0.0);
  double Z = lerp(zrow, s2, a.u_scale, a.u_off, a.n_pts);
  return 1.0 / prop_den(a.reg, Z, om2, s2, m2, k2, inv_k2);
}

// Near-pole path of the mixed kernels: recompute one propagator entirely in
// FP64 (momenta from the quadrature indices, Z from the FP64 table).  Kept out
// of line so that none of it is evaluated on the common path.
__device__ __noinline__ float pole_prop(const RhsArgs *a, const double *zrow, double s2, double om2) {
  const double k = scale_k(*a), k2 = k * k;
  return (float)prop_fp64_global(*a, zrow, s2, om2, mass2(*a, k), k2, 1.0 / k2);
}

__device__ __noinline__ float pole_d3(const RhsArgs *a, int e, int r, int j) {
  const double p = (e < a->n_ext_p) ? ext_momentum(*a, e) : 0.0;
  const double q = a->radq[r], c = a->a1_x[j];
  return pole_prop(a, a->tab, q * q + p * p + 2.0 * q * p * c, 0.0);
}

// b < 0: the |q + p1| leg; b >= 0: the |q - p2| leg at second-angle node b
__device__ __noinline__ float pole_d4(const RhsArgs *a, int e, int r, int ia, int b) {
  const int np_ = a->n_ext_p, npsi = a->n_ext_ang;
  int ip, jp = 0;
  bool three = false;
  if (e <= np_) ip = e;
  else if (e < np_ + 1 + np_ * npsi) {
    three = true;
    ip = (e - np_ - 1) / npsi;
    jp = (e - np_ - 1) - ip * npsi;
  } else ip = e - np_ - 1 - np_ * npsi;
  const double p = (e == np_) ? 0.0 : ext_momentum(*a, ip);
  const double q = a->radq[r], c1 = a->a1_x[ia];
  double s2;
  if (b < 0) {
    s2 = q * q + p * p + 2.0 * q * p * c1;
  } else {
    const double cpsi = three ? a->psi_x[jp] : 1.0, spsi = sqrt(fmax(0.0, 1.0 - cpsi * cpsi));
    const double s1 = sqrt(fmax(0.0, 1.0 - c1 * c1));
    s2 = q * q + p * p - 2.0 * q * p * (cpsi * c1 + spsi * s1 * a->a2_x[b]);
  }
  return pole_prop(a, a->tab, s2, 0.0);
}

__device__ __noinline__ float pole_ft(const RhsArgs *a, int e, int n, int r, int j) {
  const int nm = a->n_ext_ang, ip = e / nm, m = e - ip * nm;
  const double p = ext_momentum(*a, ip), q = a->radq[r], c = a->a1_x[j];
  const int srow = min(abs(n + m), a->n_stack - 1);
  const double om = 2.0 * kPi * a->T * (double)(n + m);
  return pole_prop(a, a->tab + (size_t)srow * a->n_pts, q * q + p * p + 2.0 * q * p * c, om * om);
}

// Scale-dependent constants of one RHS in the kernel precision (computed once
// per kernel, or per flow in the batched kernels).  us/uo: table coordinate
// (divided by n-1 in FP32); plim = -2 m^2 (near-pole test).  The kernels pass
// squared momenta to the propagator as y = sy s^2 and omega^2 as som omega^2:
// FP64 sy = som = 1; FP32 sy = log2(e)/k^2 (the regulator's exp2 argument)
// and som = 1/(k^2 ln 2), with the FP32 Z table pre-scaled by k^2 ln 2
// (see reg_g).  lnsy = ln(sy) shifts table coordinates taken in y.
template <typename T>
struct KConst {
  T k2, inv_k2, m2, us, uo, plim, sy, som;
  double lnsy;
};

template <typename T>
__device__ __forceinline__ KConst<T> make_kconst(const RhsArgs &a) {
  const double kd = scale_k(a), m2d = mass2(a, kd);
  KConst<T> c;
  c.k2 = (T)(kd * kd);
  c.inv_k2 = (T)(1.0 / (kd * kd));
  c.m2 = (T)m2d;
  c.us = lerp_scale<T>(a.u_scale, a.n_pts);
  c.uo = lerp_off<T>(a.u_off, a.n_pts);
  c.plim = (T)(-2.0 * m2d);
  const bool f32 = sizeof(T) == 4;
  c.sy = (T)(f32 ? 1.4426950408889634074 / (kd * kd) : 1.0);
  c.som = (T)(f32 ? 1.0 / (kd * kd * 0.6931471805599453094) : 1.0);
  c.lnsy = f32 ? log(1.4426950408889634074 / (kd * kd)) : 0.0;
  return c;
}

// FP32 regulator in propagator form.  With x = s^2/k^2 the kinetic part of the
// inverse propagator is Z (omega^2 + s^2 + k^2 r(x)) = Z (omega^2 + k^2 h(x)),
// = (k^2 ln 2 Z) (g(y) + omega^2/(k^2 ln 2)),
// h(x) = x + r(x); for the exponential shape r = x/(e^x - 1) this is
// h(x) = x/(1 - e^{-x}), for the flat shape h = max(1, x).  Evaluated as
// g(y) = h(x)/ln 2 at y = x log2(e) (so that the hardware exp2 takes y):
//   x >= 1: g = y / (1 - 2^{-y})  (no cancellation, 1 - e^{-x} >= 0.63; for
//           large x, 2^{-y} underflows to 0 and g = y exactly);
//   x < 1:  the Bernoulli series h = 1 + x/2 + x^2/12 - x^4/720 + x^6/30240
//           - x^8/1209600, rewritten in y (first omitted term x^10/47900160
//           < 2.1e-8 relative).
__device__ __forceinline__ float reg_g(int reg, float y) {
  if (reg == FFRG_REG_LITIM) return fmaxf(y, 1.4426950408889634f);
  const float y2 = y * y;
  float t = fmaf(y2, -6.3553057516916001e-8f, 5.2910945025509696e-6f);
  t = fmaf(y2, t, -4.6253423887351317e-4f);
  t = fmaf(y2, t, 5.7762265046662109e-2f);
  const float series = fmaf(y2, t, fmaf(y, 0.5f, 1.4426950408889634f));
  const float direct = y * hw_rcp(1.0f - hw_ex2(-y));
  return y < 1.4426950408889634f ? series : direct;
}

// Inverse propagator in the kernel precision from the table value Zs, the
// scaled momentum y = sy s^2 and om2s = som omega^2 (FP64: Z, s^2, omega^2).
// The FP32 version switches to FP64 when m^2 cancels more than half of
// Z (omega^2 + s^2 + k^2 r), i.e. P < -2 m^2: close to the convexity pole.
// `pole` is only evaluated on that rare branch.  POLE = false drops the test;
// callers use it only when m^2 >= 0 and no Z < 0, where P >= 0 >= -2 m^2.
template <bool POLE = true, typename Pole>
__device__ __forceinline__ double inv_prop(const RhsArgs &a, double Z, double y, double om2s,
                                           const KConst<double> &kc, Pole &&) {
  return 1.0 / prop_den(a.reg, Z, om2s, y, kc.m2, kc.k2, kc.inv_k2);
}

template <bool POLE = true, typename Pole>
__device__ __forceinline__ float inv_prop(const RhsArgs &a, float Zs, float y, float om2s, const KConst<float> &kc,
                                          Pole &&pole) {
  const float P = Zs * (reg_g(a.reg, y) + om2s);
  if (POLE && P < kc.plim) return pole();
  return hw_rcp(P + kc.m2);
}

// resident CTAs per SM requested from the compiler: the FP32 kernels are held
// to 64 registers so that four 256-thread CTAs fit
template <typename T>
struct MinBlocks {
  static constexpr int value = 1;
};
template <>
struct MinBlocks<float> {
  static constexpr int value = 4;
};

// ---------------------------------------------------------------------------
// 1. precompute kernel
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool skipped(const RhsArgs &a) { return a.skip && *(volatile const int *)a.skip; }

__device__ __forceinline__ void precompute_body(const RhsArgs &a, int tid0, int stride) {
  if (a.work_ctr && tid0 == 0) *a.work_ctr = 0u;  // the main kernel runs after this one (stream order)
  const double k = scale_k(a), k2 = k * k, inv_k2 = 1.0 / k2, m2 = mass2(a, k);
  const double L = a.qmax_over_k * k;
  const int total = (2 * a.N + 1) * a.nr;
  for (int idx = tid0; idx < total; idx += stride) {
    int n = idx / a.nr - a.N, r = idx % a.nr;
    double q = L * a.rad_x[r], w = L * a.rad_w[r], q2 = q * q;
    if (n == -a.N) {
      a.radq[r] = q;
      if (a.radq32) a.radq32[r] = (float)q;
    }
    double F;
    if (a.model == FFRG_MODEL_FINITE_T) {
      int row = min(abs(n), a.n_stack - 1);
      const double *zr = a.tab + (size_t)row * a.n_pts;
      const double *lr = a.tab + ((size_t)a.n_stack + row) * a.n_pts;
      int i0;
      double wl;
      lerp_pos(q2, a.u_scale, a.u_off, a.n_pts, i0, wl);
      double Z = lerp_at(zr, i0, wl), Lq = lerp_at(lr, i0, wl);
      double om = 2.0 * kPi * a.T * n;
      double G = 1.0 / prop_den(a.reg, Z, om * om, q2, m2, k2, inv_k2);
      double dR = Z * k2 * reg_rdot(a.reg, q2 * inv_k2);
      F = w * q2 * dR * G * G * Lq;
    } else {
      double Z = lerp(a.tab, q2, a.u_scale, a.u_off, a.n_pts);
      double G = 1.0 / prop_den(a.reg, Z, 0.0, q2, m2, k2, inv_k2);
      double rd = k2 * reg_rdot(a.reg, q2 * inv_k2);
      double dR = Z * rd;
      double meas = (a.model == FFRG_MODEL_D4_VERTEX) ? q2 * q : q2;
      F = w * meas * dR * G * G;
      if (a.radD) {
        // d F / d Z(q): dR = Z k^2 rdot, G = 1/(Z P + m^2) with P = q^2 + k^2 r
        double P = q2 + k2 * reg_r(a.reg, q2 * inv_k2);
        a.radD[idx] = w * meas * rd * G * G * (1.0 - 2.0 * Z * G * P);
      }
    }
    a.radF[idx] = F;
  }
  // FP32 node pairs; the Z table (table 0, every stack row) carries the factor
  // k^2 ln 2 of the FP32 propagator form
  const double kh = k2 * 0.6931471805599453094;
  const int z_count = a.n_stack * a.n_pts;
  for (int i = tid0; i < a.tab_count; i += stride) {
    const double f = i < z_count ? kh : 1.0;
    const float v = (float)(f * a.tab[i]);
    const float d = (i % a.n_pts == a.n_pts - 1) ? 0.0f : (float)(f * a.tab[i + 1]) - v;
    a.tab32[i] = make_float2(v, d);
  }
  if (a.ext_done)
    for (int i = tid0; i < a.n_ext; i += stride) a.ext_done[i] = 0u;
  // per-external-point constants used by every work item of the main kernels
  for (int i = tid0; i < a.n_ext_p; i += stride) a.ext_pd[i] = ext_momentum(a, i);
  if (a.model == FFRG_MODEL_D4_VERTEX) {
    for (int j = tid0; j < a.n_ext_ang; j += stride) {
      const double c = a.psi_x[j];
      a.psi_s[j] = sqrt(fmax(0.0, 1.0 - c * c));
    }
  }
}

__global__ void __launch_bounds__(kThreads) precompute_kernel(RhsArgs a) {
  if (skipped(a)) return;
  precompute_body(a, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

// ---------------------------------------------------------------------------
// shared-memory layout of the main kernels: tables (FP64 values, or FP32 node
// pairs), then the second-angle (node, weight) pairs and the first-angle
// nodes, sines and weights
// ---------------------------------------------------------------------------
template <typename T>
struct TabOf {
  using type = double;
};
template <>
struct TabOf<float> {
  using type = float2;
};
template <typename T>
struct Pair2 {
  using type = double2;
};
template <>
struct Pair2<float> {
  using type = float2;
};

template <typename T>
struct SmemLayout {
  using Tab = typename TabOf<T>::type;
  using P2 = typename Pair2<T>::type;
  Tab *tab;
  P2 *cw2;
  T *c1, *s1, *w1;
  __device__ SmemLayout(unsigned char *base, const RhsArgs &a) {
    tab = (Tab *)base;
    size_t off = ((size_t)a.tab_count * sizeof(Tab) + 15) & ~(size_t)15;
    cw2 = (P2 *)(base + off);
    c1 = (T *)(cw2 + a.na2);
    s1 = c1 + a.na1;
    w1 = s1 + a.na1;
  }
};

template <typename T>
__device__ __forceinline__ const typename TabOf<T>::type *table_src(const RhsArgs &a);
template <>
__device__ __forceinline__ const double *table_src<double>(const RhsArgs &a) { return a.tab; }
template <>
__device__ __forceinline__ const float2 *table_src<float>(const RhsArgs &a) { return a.tab32; }

__device__ __forceinline__ double table_value(double v) { return v; }
__device__ __forceinline__ float table_value(float2 v) { return v.x; }

// angle rules into shared memory in the kernel precision
template <typename T>
__device__ __forceinline__ void stage_angles(const RhsArgs &a, SmemLayout<T> &S) {
  for (int i = threadIdx.x; i < a.na1; i += blockDim.x) {
    double c = a.a1_x[i];
    S.c1[i] = (T)c;
    S.s1[i] = (T)sqrt(fmax(0.0, 1.0 - c * c));
    S.w1[i] = (T)a.a1_w[i];
  }
  for (int i = threadIdx.x; i < a.na2; i += blockDim.x) {
    S.cw2[i].x = (T)a.a2_x[i];
    S.cw2[i].y = (T)a.a2_w[i];
  }
}

template <typename T>
__device__ bool main_prologue(const RhsArgs &a, SmemLayout<T> &S, uint64_t *bar) {
  bool ok = stage_to_smem<typename TabOf<T>::type>(S.tab, table_src<T>(a), a.tab_count, bar, a.status);
  stage_angles<T>(a, S);
  __syncthreads();
  return ok;
}

// ---------------------------------------------------------------------------
// 2a. d=3, T=0:  row (r, angle block): sum_j v_j G(|q+p|)
// One work item: partial sum of external point e over a chunk of radial rows
// (returned in thread 0).  `sa` is the argument block the near-pole path reads.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ double d3_item(const RhsArgs &a, const RhsArgs *sa, const SmemLayout<T> &S,
                                          const KConst<T> &kc, int item, double *red) {
  const T us = kc.us, uo = kc.uo;
  const int np = a.n_pts, nblk = (a.na1 + a.jb - 1) / a.jb;
  const int e = item / a.n_chunks, c = item - e * a.n_chunks;
  const double pd = (e < a.n_ext_p) ? a.ext_pd[e] : 0.0;
  const T p = (T)pd;
  const int o0 = c * a.cr, o1 = min(o0 + a.cr, a.nr);
  const int rows = (o1 - o0) * nblk;
  double acc = 0.0;
  for (int row = threadIdx.x; row < rows; row += blockDim.x) {
    const int o = o0 + row / nblk, jb0 = (row % nblk) * a.jb, jb1 = min(jb0 + a.jb, a.na1);
    const double qd = a.radq[o];
    const T q = (T)qd, q2 = q * q, base = q2 + p * p, tqp = (T)2 * q * p;
    T rs = 0;
    for (int j = jb0; j < jb1; ++j) {
      const T s2 = base + tqp * S.c1[j];   // >= 0 up to rounding; lookups clamp
      T Z = lerp(S.tab, s2, us, uo, np);
      auto pole = [&]() { return pole_d3(sa, e, o, j); };
      rs += S.w1[j] * inv_prop(a, Z, s2 * kc.sy, (T)0, kc, pole);
    }
    acc = fma(a.radF[o], (double)rs, acc);
  }
  return block_sum(acc, red);
}

template <typename T>
__global__ void __launch_bounds__(kThreads, MinBlocks<T>::value) d3_main(RhsArgs a) {
  if (skipped(a)) return;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t bar;
  __shared__ double red[kThreads / 32];
  __shared__ RhsArgs sa;  // for the out-of-line near-pole path
  if (threadIdx.x == 0) sa = a;
  SmemLayout<T> S(smem, a);
  if (!main_prologue<T>(a, S, &bar)) return;
  const KConst<T> kc = make_kconst<T>(a);
  for (int item = blockIdx.x; item < a.n_items; item += gridDim.x) {
    double t = d3_item<T>(a, &sa, S, kc, item, red);
    if (threadIdx.x == 0) a.partial[item] = t;
  }
}

// ---------------------------------------------------------------------------
// 2b. d=4 vertex expansion: row (r, c1 node), inner loop over c2 nodes.
// Work items are warp-sized (about eight rows per lane) and are handed out by
// a device counter, the three-point items (the 16x more expensive ones) first.
// Each item is summed by one warp in a fixed order (rows by lane, then a
// shuffle tree), so the result does not depend on which warp took it.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T radial_q(const RhsArgs &a, int r);
template <>
__device__ __forceinline__ double radial_q<double>(const RhsArgs &a, int r) { return a.radq[r]; }
template <>
__device__ __forceinline__ float radial_q<float>(const RhsArgs &a, int r) { return a.radq32[r]; }

// Output of external point e from the sum s of its partials: diagram
// coefficient (d=4: 1, 3, 3/2 for the Z, lambda3, lambda4 blocks), overall
// normalisation, and the non-finite check into the status word.
__device__ __forceinline__ void write_output(const RhsArgs &a, int e, double s) {
  double coef = 1.0;
  if (a.model == FFRG_MODEL_D4_VERTEX) {
    const int np_ = a.n_ext_p;
    if (e > np_ && e < np_ + 1 + np_ * a.n_ext_ang) coef = 3.0;
    else if (e >= np_ + 1 + np_ * a.n_ext_ang) coef = 1.5;
  }
  const double v = a.norm * coef * s;
  a.out[e] = v;
  if (!isfinite(v)) raise_status(a.status, kStatusNonFinite);
}

// Work loop of the d=4 kernel.  All squared momenta are taken as y = sy s^2;
// table coordinates in y use offsets shifted by -u_scale ln(sy).
template <typename T, bool POLE>
__device__ __forceinline__ void d4_items(const RhsArgs &a, const RhsArgs *sa, const SmemLayout<T> &S,
                                         const KConst<T> &kc) {
  const T us = kc.us, sy = kc.sy;
  // S0^2 = (sum of squares)/c: the 1/c is a shift of the coordinate, -u_scale ln c
  const T uo1 = lerp_off<T>(a.u_off - a.u_scale * kc.lnsy, a.n_pts);
  const T uo2 = lerp_off<T>(a.u_off - a.u_scale * (0.69314718055994530942 + kc.lnsy), a.n_pts);
  const T uo3 = lerp_off<T>(a.u_off - a.u_scale * (1.09861228866810969140 + kc.lnsy), a.n_pts);
  const T uo4 = lerp_off<T>(a.u_off - a.u_scale * (1.38629436111989061883 + kc.lnsy), a.n_pts);
  const int np = a.n_pts, np_ = a.n_ext_p, npsi = a.n_ext_ang, na1 = a.na1;
  const auto *Zt = S.tab, *L3 = S.tab + np, *L4 = S.tab + 2 * np;
  const T sum_w2 = (T)a.sum_w2;
  const int lane = threadIdx.x & 31;
  const int dr = 32 / na1, dia = 32 % na1;  // row step of one lane in (r, ia)
  for (;;) {
    int d = 0;
    if (lane == 0) d = (int)atomicAdd(a.work_ctr, 1u);
    d = __shfl_sync(0xffffffffu, d, 0);
    if (d >= a.n_items) break;
    // rank d -> external point: rotate so that the three-point block comes first
    const int c = d % a.n_chunks;
    const int e = (d / a.n_chunks + np_ + 1) % a.n_ext;
    const int item = e * a.n_chunks + c;
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
    const double pd = (block == 0 && ip == np_) ? 0.0 : a.ext_pd[ip];
    const double cpsid = block == 1 ? a.psi_x[jp] : 1.0;
    const double spsid = block == 1 ? a.psi_s[jp] : 0.0;
    const T p = (T)pd, p2 = p * p, cpsi = (T)cpsid, spsi = (T)spsid;
    const T C2 = (T)2 * p2 * ((T)1 + cpsi);
    const int o0 = c * a.cr, o1 = min(o0 + a.cr, a.nr);
    const int rows = (o1 - o0) * na1;
    double acc = 0.0;
    int r = o0 + lane / na1, ia = lane % na1;
    for (int row = lane; row < rows; row += 32) {
      const T q = radial_q<T>(a, r), q2 = q * q, qp = q * p, c1 = S.c1[ia];
      const T A2 = q2 + p2 + (T)2 * qp * c1;   // >= 0 up to rounding; lookups clamp
      const T Ay = A2 * sy;
      const T ZA = lerp(Zt, Ay, us, uo1, np);
      auto pole_a = [&]() { return pole_d4(sa, e, r, ia, -1); };
      const T GA = inv_prop<POLE>(a, ZA, Ay, (T)0, kc, pole_a);
      T v;
      if (block == 0) {
        const T l4 = lerp(L4, (q2 + p2) * sy, us, uo2, np);
        const T l3 = lerp(L3, (q2 + A2 + p2) * sy, us, uo3, np);
        v = sum_w2 * ((T)(-0.5) * l4 + l3 * l3 * GA);
      } else if (block == 2) {
        const T l4 = lerp(L4, (q2 + A2 + (T)2 * p2) * sy, us, uo4, np);
        v = sum_w2 * GA * l4 * l4;
      } else {
        const T la = lerp(L3, (q2 + A2 + p2) * sy, us, uo3, np);
        const T base = q2 + p2, t1 = (T)2 * qp * cpsi * c1, t2 = (T)2 * qp * spsi * S.s1[ia];
        const T by = base * sy, b0 = (base - t1) * sy, t2y = t2 * sy, sy_ab = (A2 + C2) * sy;
        T rs = 0;
        for (int b = 0; b < a.na2; ++b) {
          const auto cw = S.cw2[b];
          const T By = b0 - t2y * cw.x;   // sy |q - p2|^2
          const T ZB = lerp(Zt, By, us, uo1, np);
          auto pole_b = [&]() { return pole_d4(sa, e, r, ia, b); };
          const T GB = inv_prop<POLE>(a, ZB, By, (T)0, kc, pole_b);
          const T lb = lerp(L3, by + By, us, uo3, np);
          const T lc = lerp(L3, sy_ab + By, us, uo3, np);
          rs += cw.y * GB * lb * lc;
        }
        v = GA * la * rs;
      }
      acc = fma(a.radF[r], (double)(S.w1[ia] * v), acc);
      r += dr;
      ia += dia;
      if (ia >= na1) {
        ia -= na1;
        ++r;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    // the warp that completes external point e sums its partials (fixed order)
    unsigned done = 0;
    if (lane == 0) {
      a.partial[item] = acc;
      __threadfence();
      done = atomicAdd(a.ext_done + e, 1u);
    }
    done = __shfl_sync(0xffffffffu, done, 0);
    if (done == (unsigned)a.n_chunks - 1u) {
      __threadfence();
      const double *pp = a.partial + (size_t)e * a.n_chunks;
      double t = 0.0;
      for (int j = lane; j < a.n_chunks; j += 32) t += __ldcg(pp + j);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
      if (lane == 0) write_output(a, e, t);
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads, MinBlocks<T>::value) d4_main(RhsArgs a) {
  if (skipped(a)) return;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t bar;
  __shared__ RhsArgs sa;  // for the out-of-line near-pole path
  if (threadIdx.x == 0) sa = a;
  SmemLayout<T> S(smem, a);
  if (!main_prologue<T>(a, S, &bar)) return;
  const KConst<T> kc = make_kconst<T>(a);
  // the near-pole test can only fire with m^2 < 0 or a negative Z node
  int neg = 0;
  for (int i = threadIdx.x; i < a.n_pts; i += blockDim.x) neg |= table_value(S.tab[i]) < (T)0;
  const bool may_pole = __syncthreads_or(neg) || kc.m2 < (T)0;
  if (may_pole) d4_items<T, true>(a, &sa, S, kc);
  else d4_items<T, false>(a, &sa, S, kc);
}

// ---------------------------------------------------------------------------
// 2c. finite T: row (Matsubara n, r, angle block)
//     sum_j v_j lam(n+m, s) G(n+m, s), s = |q+p|
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ double ft_item(const RhsArgs &a, const RhsArgs *sa, const SmemLayout<T> &S,
                                          const KConst<T> &kc, int item, double *red) {
  const T us = kc.us, uo = kc.uo;
  const int np = a.n_pts, nm = a.n_ext_ang, nblk = (a.na1 + a.jb - 1) / a.jb;
  const int outer_total = (2 * a.N + 1) * a.nr;
  const int e = item / a.n_chunks, c = item - e * a.n_chunks;
  const int ip = e / nm, m = e - ip * nm;
  const double pd = a.ext_pd[ip];
  const T p = (T)pd;
  const int o0 = c * a.cr, o1 = min(o0 + a.cr, outer_total);
  const int rows = (o1 - o0) * nblk;
  double acc = 0.0;
  for (int row = threadIdx.x; row < rows; row += blockDim.x) {
    const int o = o0 + row / nblk, jb0 = (row % nblk) * a.jb, jb1 = min(jb0 + a.jb, a.na1);
    const int n = o / a.nr - a.N, r = o % a.nr;
    const int srow = min(abs(n + m), a.n_stack - 1);
    const auto *Zr = S.tab + (size_t)srow * np, *Lr = S.tab + ((size_t)a.n_stack + srow) * np;
    const double omd = 2.0 * kPi * a.T * (double)(n + m);
    const T om2s = (T)(omd * omd) * kc.som;
    const double qd = a.radq[r];
    const T q = (T)qd, q2 = q * q, base = q2 + p * p, tqp = (T)2 * q * p;
    T rs = 0;
    for (int j = jb0; j < jb1; ++j) {
      const T s2 = base + tqp * S.c1[j];   // >= 0 up to rounding; lookups clamp
      int i0;
      T w;
      lerp_pos(s2, us, uo, np, i0, w);
      const T Z = lerp_at(Zr, i0, w), Lv = lerp_at(Lr, i0, w);
      auto pole = [&]() { return pole_ft(sa, e, n, r, j); };
      rs += S.w1[j] * Lv * inv_prop(a, Z, s2 * kc.sy, om2s, kc, pole);
    }
    acc = fma(a.radF[o], (double)rs, acc);
  }
  return block_sum(acc, red);
}

template <typename T>
__global__ void __launch_bounds__(kThreads, MinBlocks<T>::value) ft_main(RhsArgs a) {
  if (skipped(a)) return;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t bar;
  __shared__ double red[kThreads / 32];
  __shared__ RhsArgs sa;  // for the out-of-line near-pole path
  if (threadIdx.x == 0) sa = a;
  SmemLayout<T> S(smem, a);
  if (!main_prologue<T>(a, S, &bar)) return;
  const KConst<T> kc = make_kconst<T>(a);
  for (int item = blockIdx.x; item < a.n_items; item += gridDim.x) {
    double t = ft_item<T>(a, &sa, S, kc, item, red);
    if (threadIdx.x == 0) a.partial[item] = t;
  }
}

// ---------------------------------------------------------------------------
// 3. finalize: fixed-order sum over chunks, normalisation, finiteness
// ---------------------------------------------------------------------------
__device__ __forceinline__ void finalize_body(const RhsArgs &a, int e) {
  if (e >= a.n_ext) return;
  double s = 0.0;
  const double *pp = a.partial + (size_t)e * a.n_chunks;
  for (int c = 0; c < a.n_chunks; ++c) s += pp[c];
  write_output(a, e, s);
}

__global__ void finalize_kernel(RhsArgs a) {
  if (skipped(a)) return;
  finalize_body(a, blockIdx.x * blockDim.x + threadIdx.x);
}

// ---------------------------------------------------------------------------
// launch
// ---------------------------------------------------------------------------
template <typename K>
static int persistent_grid(ffrg_ctx *ctx, K kernel, size_t smem, int items, int *grid) {
  static const size_t kMaxSmem = 227 * 1024;
  if (smem > kMaxSmem) {
    ctx->last_error = "dressing tables do not fit in shared memory";
    return FFRG_EINVAL;
  }
  int st = ensure_smem_limit(ctx, (const void *)kernel, smem);
  if (st) return st;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, smem);
  if (e != cudaSuccess) return set_cuda_error(ctx, e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
  if (per_sm < 1) {
    ctx->last_error = "RHS kernel cannot be resident";
    return FFRG_EINVAL;
  }
  *grid = std::max(1, std::min(items, per_sm * ctx->num_sms));
  return FFRG_OK;
}

int launch_precompute(ffrg_ctx *ctx, const RhsArgs &a, cudaStream_t s) {
  const int pre_total = std::max((2 * a.N + 1) * a.nr, a.tab_count);
  const int pre_blocks = std::min((pre_total + kThreads - 1) / kThreads, 4 * ctx->num_sms);
  precompute_kernel<<<pre_blocks, kThreads, 0, s>>>(a);
  return set_cuda_error(ctx, cudaGetLastError(), "precompute launch");
}

int launch_rhs(ffrg_ctx *ctx, const Plan *pl_c, const RhsArgs &a, int precision, cudaStream_t s) {
  Plan *pl = const_cast<Plan *>(pl_c);
  const bool mixed = precision == FFRG_MIXED;
  int st;
  int &grid = mixed ? pl->grid32 : pl->grid64;
  const size_t smem = mixed ? pl->smem32 : pl->smem64;
  void (*kern)(RhsArgs) = nullptr;
  switch (a.model) {
  case FFRG_MODEL_D3: kern = mixed ? d3_main<float> : d3_main<double>; break;
  case FFRG_MODEL_D4_VERTEX: kern = mixed ? d4_main<float> : d4_main<double>; break;
  default: kern = mixed ? ft_main<float> : ft_main<double>; break;
  }
  if (a.model == FFRG_MODEL_D4_VERTEX && (!a.work_ctr || !a.radq32 || !a.ext_done)) {
    ctx->last_error = "d=4 plan without work counter or FP32 radial nodes";
    return FFRG_EINVAL;
  }
  if (grid == 0) {
    st = persistent_grid(ctx, kern, smem, a.n_items, &grid);
    if (st) return st;
  }
  const int pre_total = std::max((2 * a.N + 1) * a.nr, a.tab_count);
  const int pre_blocks = std::min((pre_total + kThreads - 1) / kThreads, 4 * ctx->num_sms);
  precompute_kernel<<<pre_blocks, kThreads, 0, s>>>(a);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cap);
  const bool prof = ctx->profiling && cap == cudaStreamCaptureStatusNone &&
                    ctx->prof_used * 2 + 1 < (int)ctx->prof_events.size();
  if (prof) cudaEventRecord(ctx->prof_events[2 * ctx->prof_used], s);
  kern<<<grid, kThreads, smem, s>>>(a);
  if (prof) {
    cudaEventRecord(ctx->prof_events[2 * ctx->prof_used + 1], s);
    ctx->prof_used++;
  }
  // the d=4 kernel writes its outputs itself (last warp per external point)
  if (a.model != FFRG_MODEL_D4_VERTEX)
    finalize_kernel<<<(a.n_ext + kThreads - 1) / kThreads, kThreads, 0, s>>>(a);
  return set_cuda_error(ctx, cudaGetLastError(), "rhs launch");
}

}  // namespace ffrg

// ---------------------------------------------------------------------------
// Batched RHS of many flows (serving, mixed precision): the same item
// functions as the single-flow kernels, driven by per-flow descriptors.
// ---------------------------------------------------------------------------
namespace ffrg {

__global__ void __launch_bounds__(kThreads) batched_precompute_kernel(const RhsArgs *descs) {
  const RhsArgs &a = descs[blockIdx.y];
  if (skipped(a)) return;
  precompute_body(a, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

__global__ void batched_finalize_kernel(const RhsArgs *descs) {
  const RhsArgs &a = descs[blockIdx.y];
  if (skipped(a)) return;
  finalize_body(a, blockIdx.x * blockDim.x + threadIdx.x);
}

// Each CTA walks a contiguous range of the combined item list; when the range
// crosses into another flow it copies that flow's descriptor and FP32 tables
// into shared memory (plain loads) before continuing.
template <int MODEL>
__global__ void __launch_bounds__(kThreads, 4)
    batched_main_kernel(const RhsArgs *descs, const int *flows, const int *start, int n_fl, int total, int per) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ double red[kThreads / 32];
  __shared__ RhsArgs sa;
  const int g0 = blockIdx.x * per, g1 = min(g0 + per, total);
  int cur = -1, lo = 0, hi = 0;
  SmemLayout<float> S(smem, descs[flows[0]]);
  KConst<float> kc;
  bool skip = false;
  for (int g = g0; g < g1; ++g) {
    if (g >= hi) {  // next flow: find f with start[f] <= g < start[f+1]
      int f = (cur < 0) ? 0 : cur + 1;
      while (f < n_fl && start[f + 1] <= g) ++f;
      cur = f;
      lo = start[f];
      hi = start[f + 1];
      __syncthreads();
      if (threadIdx.x == 0) sa = descs[flows[f]];
      __syncthreads();
      skip = sa.skip && *(volatile const int *)sa.skip;
      if (!skip) {
        S = SmemLayout<float>(smem, sa);
        for (int i = threadIdx.x; i < sa.tab_count; i += blockDim.x) S.tab[i] = sa.tab32[i];
        stage_angles<float>(sa, S);
        kc = make_kconst<float>(sa);
      }
      __syncthreads();
    }
    if (skip) continue;
    const int item = g - lo;
    double t = (MODEL == FFRG_MODEL_D3) ? d3_item<float>(sa, &sa, S, kc, item, red)
                                        : ft_item<float>(sa, &sa, S, kc, item, red);
    if (threadIdx.x == 0) sa.partial[item] = t;
  }
}

template <int MODEL>
static int launch_batched_main(ffrg_ctx *ctx, const BatchList &bl, const int *flows, const int *start, int n,
                               int total, size_t smem, cudaStream_t s) {
  if (n == 0 || total == 0) return FFRG_OK;
  void (*kern)(const RhsArgs *, const int *, const int *, int, int, int) = batched_main_kernel<MODEL>;
  int st = ensure_smem_limit(ctx, (const void *)kern, smem);
  if (st) return st;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
  if (e != cudaSuccess || per_sm < 1) return set_cuda_error(ctx, e ? e : cudaErrorInvalidConfiguration, "occupancy");
  const int grid = std::max(1, std::min(total, per_sm * ctx->num_sms));
  const int per = (total + grid - 1) / grid;
  kern<<<(total + per - 1) / per, kThreads, smem, s>>>(bl.descs, flows, start, n, total, per);
  return FFRG_OK;
}

int launch_rhs_batched(ffrg_ctx *ctx, const BatchList &bl, cudaStream_t s) {
  if (bl.n_flows == 0) return FFRG_OK;
  const int pre_blocks = std::max(1, std::min((bl.max_pre + kThreads - 1) / kThreads, 64));
  batched_precompute_kernel<<<dim3(pre_blocks, bl.n_flows), kThreads, 0, s>>>(bl.descs);
  int st = launch_batched_main<FFRG_MODEL_D3>(ctx, bl, bl.d3_flows, bl.d3_start, bl.n_d3, bl.d3_items,
                                              bl.smem_d3, s);
  if (!st) st = launch_batched_main<FFRG_MODEL_FINITE_T>(ctx, bl, bl.ft_flows, bl.ft_start, bl.n_ft, bl.ft_items,
                                                         bl.smem_ft, s);
  if (st) return st;
  batched_finalize_kernel<<<dim3((bl.max_ext + kThreads - 1) / kThreads, bl.n_flows), kThreads, 0, s>>>(bl.descs);
  return set_cuda_error(ctx, cudaGetLastError(), "batched rhs launch");
}

}  // namespace ffrg
