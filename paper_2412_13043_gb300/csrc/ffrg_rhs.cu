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
//      way, Sec. 5.3.2), the FP32 tables (d=3, d=4: line-form rows; finite T:
//      (Z, lambda) node pairs) and the per-RHS constant block;
//   2. main (rhs_main): persistent CTAs stage the tables into shared memory
//      by a TMA bulk copy (cp.async.bulk + mbarrier, bounded wait); warps take
//      warp-sized work items (external point x chunk of rows) from a device
//      counter; lanes take rows and run the row's angle loop in the kernel
//      precision (FP32: pairs of nodes in packed FP32 where no near-pole test
//      is needed); FP64 accumulation, or Kahan FP32 with an error-free
//      two-sum warp tree (mixed); the warp that completes an external point
//      sums its partials in a fixed order and writes the output.  Finite T:
//      the main kernel fills the angle-integrated kernel K(p, q) instead;
//   3. finite T only: the contraction of K with the radial factors, one
//      block per output.
// Serving runs the same item functions from batched kernels over many flows
// (bottom of this file).  The reduction order depends only on the problem
// shape, never on the grid size or on other work in flight.
#include <math.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>

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

// b < 0: the |q + p1| leg; b >= 0: the |q - p2| leg at second-angle node b.
// One copy per d=4 model (M), so that the two kernels do not share an
// out-of-line callee (sharing it cost the vertex-model kernel registers).
template <int M>
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

// stack row of loop frequency index n: |n| (bosonic), n or -n-1 (fermionic)
__device__ __forceinline__ int stack_index(int stat, int n) { return stat ? (n >= 0 ? n : -n - 1) : abs(n); }

// K row of stack row jk (finite T): frequency of row jk, table row min(jk, n_stack-1)
__device__ __noinline__ float pole_ftk(const RhsArgs *a, int ip, int jk, int r, int j) {
  // q from its definition (the value the precompute stores in radq): the
  // single-launch RHS runs no precompute
  const double p = ext_momentum(*a, ip), q = a->qmax_over_k * scale_k(*a) * a->rad_x[r], c = a->a1_x[j];
  const int srow = min(jk, a->n_stack - 1);
  const double om = kPi * a->T * (2.0 * (double)jk + (a->stat ? 1.0 : 0.0));
  return pole_prop(a, a->tab + (size_t)srow * a->n_pts, q * q + p * p + 2.0 * q * p * c, om * om);
}

// Scale-dependent constants of one RHS in the kernel precision, computed once
// per RHS by the precompute kernel into a small device block (RhsArgs::kconst)
// that every CTA of the main kernel loads.  us/uo: table coordinate
// (divided by n-1 in FP32); plim = -2 m^2 (near-pole test).  The kernels pass
// squared momenta to the propagator as y = sy s^2 and omega^2 as som omega^2:
// FP64 sy = som = 1; FP32 sy = log2(e)/k^2 (the regulator's exp2 argument)
// and som = 1/(k^2 ln 2), with the FP32 Z table pre-scaled by k^2 ln 2
// (see reg_g).
// uy1..uy4: offsets of table coordinates taken in y of S0^2 = (sum of c
// squares)/c (c = 1..4; ln(sy) and ln c folded in); twopiT = 2 pi T;
// sw2 = sum of the second-angle weights.
struct KConstPair {
  KConst<float> f;
  KConst<double> d;
};
static_assert(sizeof(KConstPair) <= kKConstBytes, "constant block too small");

// The k-dependent constants of one RHS: FP32 from kconst_f32 (or the host's
// copy of it), FP64 below; once per RHS on one thread.
template <typename T>
__device__ __forceinline__ KConst<T> make_kconst(const RhsArgs &a);
template <>
__device__ __forceinline__ KConst<float> make_kconst<float>(const RhsArgs &a) {
  // the host's copy when the scale and mass are host values (plain RHS calls)
  if (a.kc_host_ok && !a.k_dev && !a.m2_dev) return a.kc_host;
  const double kd = scale_k(a);
  return kconst_f32(a, kd, mass2(a, kd));
}
template <>
__device__ __forceinline__ KConst<double> make_kconst<double>(const RhsArgs &a) {
  const double kd = scale_k(a), m2d = mass2(a, kd);
  KConst<double> c;
  c.k2 = kd * kd;
  c.inv_k2 = 1.0 / c.k2;
  c.m2 = m2d;
  c.plim = -2.0 * m2d;
  c.us = a.u_scale;
  c.uo = a.u_off;
  c.sy = 1.0;
  c.som = 1.0;
  c.isy = 1.0;
  c.uy1 = a.uoc[0];
  c.uy2 = a.uoc[1];
  c.uy3 = a.uoc[2];
  c.uy4 = a.uoc[3];
  c.twopiT = a.twopiT;
  c.sw2 = a.sum_w2;
  return c;
}

template <typename T>
__device__ __forceinline__ KConst<T> load_kconst(const RhsArgs &a);
template <>
__device__ __forceinline__ KConst<float> load_kconst<float>(const RhsArgs &a) {
  return ((const KConstPair *)a.kconst)->f;
}
template <>
__device__ __forceinline__ KConst<double> load_kconst<double>(const RhsArgs &a) {
  return ((const KConstPair *)a.kconst)->d;
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
  // the denominator is one explicit FMA in both variants and the sum an
  // explicit add (no contraction with reg_g's product), so that kernels with
  // and without the test (serving, single flow) round it identically
  const float t = __fadd_rn(reg_g(a.reg, y), om2s);
  if (POLE && Zs * t < kc.plim) return pole();
  return hw_rcp(fmaf(Zs, t, kc.m2));
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

// blocks of the per-radial precompute: radial nodes x values of |n|
constexpr int kPreR = 64, kPreN = 8;

// template tag of the D4_FULL mixed kernel with lambda3 cells (not a public model)
constexpr int kModelD4FullCell = 100 + FFRG_MODEL_D4_FULL;

// n-independent terms of radial node r (q = L x_r): q^2, weight x measure,
// k^2 r(x), k^2 rdot(x) and the table position of q^2
struct RadialNode {
  double q2, wm, kr, rd, wl;
  int i0;
};
__device__ __forceinline__ RadialNode radial_node(const RhsArgs &a, int r, double L, double k2, double inv_k2) {
  RadialNode t;
  const double q = L * a.rad_x[r], w = L * a.rad_w[r], q2 = q * q, x = q2 * inv_k2;
  t.q2 = q2;
  t.wm = w * (is_d4(a.model) ? q2 * q : q2);
  double rx, rdx;
  reg_r_rdot(a.reg, x, rx, rdx);
  t.kr = k2 * rx;
  t.rd = k2 * rdx;
  lerp_pos(q2, a.u_scale, a.u_off, a.n_pts, t.i0, t.wl);
  return t;
}

// Finite T: F(n, r) = w q^2 Z rdot k^2 G^2 lambda at the loop frequency of
// stack row n (>= 0), written to both loop indices that share it: n and -n
// (bosonic) or -n-1 (fermionic); row of loop index n in radF: n + N + stat.
__device__ __forceinline__ void radial_F_finite_t(const RhsArgs &a, int n, int r, double q2, double wm, double kr,
                                                  double rd, int i0, double wl, double m2) {
  const int row = min(n, a.n_stack - 1);
  const double Z = lerp_at(a.tab + (size_t)row * a.n_pts, i0, wl);
  const double Lq = lerp_at(a.tab + ((size_t)a.n_stack + row) * a.n_pts, i0, wl);
  const double om = a.stat ? (2.0 * n + 1.0) * kPi * a.T : 2.0 * kPi * a.T * n;
  const double G = 1.0 / (Z * (om * om + q2 + kr) + m2);
  const double F = wm * (Z * rd) * G * G * Lq;
  const int nr = a.nr, ip = (a.N + a.stat + n) * nr + r, im = (a.N - n) * nr + r;
  a.radF[ip] = F;
  a.radF[im] = F;
  if (a.radF32) {
    a.radF32[ip] = (float)F;
    a.radF32[im] = (float)F;
  }
}

// Per-radial part of the precompute, blocks blk, blk + nblk, ... of the
// kPreR x kPreN blocks; every thread of the calling block must run it (it
// synchronises the block).
__device__ __forceinline__ void precompute_radial(const RhsArgs &a, int blk, int nblk) {
  const double k = scale_k(a), k2 = k * k, inv_k2 = 1.0 / k2, m2 = mass2(a, k);
  const double L = a.qmax_over_k * k;
  // Per-radial factors F(n, r), in blocks of kPreR radial nodes x kPreN
  // stack rows j.  Phase A: the n-independent part of each node (q^2, weight
  // x measure, k^2 r(x), k^2 rdot(x), the table position of q^2) once per
  // block into shared memory.  Phase B: F for stack row j, written to both
  // loop indices that read row j and share its frequency^2: n = j and
  // n = -j (bosonic, omega_j = 2 pi T j) or n = -j-1 (fermionic, nu_j =
  // (2j+1) pi T).  Row of loop index n in radF: n + N + stat.
  const int nr = a.nr, N = a.N;
  const int n_rt = (nr + kPreR - 1) / kPreR, n_nb = N / kPreN + 1;
  __shared__ double s_q2[kPreR], s_wm[kPreR], s_kr[kPreR], s_rd[kPreR], s_wl[kPreR];
  __shared__ int s_i0[kPreR];
  for (int pb = blk; pb < n_rt * n_nb; pb += nblk) {
    const int rt = pb % n_rt, nb = pb / n_rt;
    const int r0 = rt * kPreR, rn = min(kPreR, nr - r0);
    __syncthreads();  // the previous block's shared values are no longer read
    for (int i = threadIdx.x; i < rn; i += blockDim.x) {
      const RadialNode t = radial_node(a, r0 + i, L, k2, inv_k2);
      s_q2[i] = t.q2;
      s_wm[i] = t.wm;
      s_kr[i] = t.kr;
      s_rd[i] = t.rd;
      s_i0[i] = t.i0;
      s_wl[i] = t.wl;
    }
    __syncthreads();
    const int n0 = nb * kPreN, n1 = min(n0 + kPreN, N + 1);
    for (int j = threadIdx.x; j < (n1 - n0) * rn; j += blockDim.x) {
      const int n = n0 + j / rn, i = j - (j / rn) * rn, r = r0 + i;
      const double q2 = s_q2[i], wl = s_wl[i], rd = s_rd[i];
      const int i0 = s_i0[i];
      if (a.model == FFRG_MODEL_FINITE_T) {
        radial_F_finite_t(a, n, r, q2, s_wm[i], s_kr[i], rd, i0, wl, m2);
      } else {
        double F;
        const double Z = lerp_at(a.tab, i0, wl);
        const double P = q2 + s_kr[i];
        const double G = 1.0 / (Z * P + m2);
        F = s_wm[i] * (Z * rd) * G * G;
        // d F / d Z(q): dR = Z k^2 rdot, G = 1/(Z P + m^2) with P = q^2 + k^2 r
        if (a.radD) a.radD[r] = s_wm[i] * rd * G * G * (1.0 - 2.0 * Z * G * P);
        const int ip = (N + a.stat + n) * nr + r, im = (N - n) * nr + r;
        a.radF[ip] = F;
        a.radF[im] = F;
        if (a.radF32) {
          a.radF32[ip] = (float)F;
          a.radF32[im] = (float)F;
        }
      }
    }
  }
}

// Finite T, the same factors F(n, r) by warps: warp unit u of a grid takes
// 32 radial nodes x kRadN stack rows (one node per lane), so that their FP64
// work (slow on this part) spreads over as many SMs as there are units.
constexpr int kRadN = 4;
__device__ __forceinline__ int radial_units(const RhsArgs &a) {
  return ((a.nr + 31) / 32) * ((a.N + 1 + kRadN - 1) / kRadN);
}
__device__ __forceinline__ void radial_unit(const RhsArgs &a, int u, int lane) {
  const int n_rb = (a.nr + 31) / 32, rb = u % n_rb, n0 = (u / n_rb) * kRadN;
  const int r = rb * 32 + lane;
  if (r >= a.nr) return;
  const double k = scale_k(a), k2 = k * k, inv_k2 = 1.0 / k2, m2 = mass2(a, k);
  const RadialNode t = radial_node(a, r, a.qmax_over_k * k, k2, inv_k2);
  for (int n = n0; n < min(n0 + kRadN, a.N + 1); ++n) radial_F_finite_t(a, n, r, t.q2, t.wm, t.kr, t.rd, t.i0, t.wl, m2);
}

// Every thread of a block of the calling grid (blockIdx.x over the grid,
// blockDim.x threads) must run it: it synchronises the block.
__device__ __forceinline__ void precompute_body(const RhsArgs &a) {
  const double k = scale_k(a), k2 = k * k;
  // The scalar and flat work starts at the first block without per-radial
  // work (blocks 0 .. n_rt n_nb - 1 have some), so that no block has both.
  const int n_phase = ((a.nr + kPreR - 1) / kPreR) * (a.N / kPreN + 1);
  const int first_free = n_phase % gridDim.x;
  const int stride = gridDim.x * blockDim.x;
  const int tid0 = ((blockIdx.x + gridDim.x - first_free) % gridDim.x) * blockDim.x + threadIdx.x;
  // the main kernel runs after this one (stream order)
  if (tid0 == 0 && a.work_ctr) *a.work_ctr = 0u;
  if (a.kconst && (tid0 == 0 || tid0 == 32)) {  // two warps, in parallel
    KConstPair *kp = (KConstPair *)a.kconst;
    if (tid0 == 0) kp->f = make_kconst<float>(a);
    else kp->d = make_kconst<double>(a);
  }
  precompute_radial(a, blockIdx.x, gridDim.x);
  // radial nodes q_r = qmax k x_r
  for (int r = tid0; r < a.nr; r += stride) {
    const double q = a.qmax_over_k * k * a.rad_x[r];
    a.radq[r] = q;
    if (a.radq32) a.radq32[r] = (float)q;
  }
  // FP32 tables; the Z table (table 0, every stack row) carries the factor
  // k^2 ln 2 of the FP32 propagator form.  d=3, d=4: rows in line form
  // (T_i - i d_i, (n-1) d_i), d_i the difference to the next node (0 at a
  // row end), from FP64 values.  Finite T: (Z, lambda) pairs per node of each
  // stack row, then one zero pair (the upper neighbour of the last node, read
  // with weight 0).
  const double kh = k2 * 0.6931471805599453094;
  const int z_count = a.n_stack * a.n_pts;
  if (a.model == FFRG_MODEL_D4_FULL) {
    // compact rows [Z row 0 | lambda4 row 0 | lambda3 rows]: FP64 copy and FP32
    // pairs (with lambda3 cells: the two line rows only)
    const int np = a.n_pts, ns = a.n_stack;
    const int n_line = a.l3cell ? 2 * np : a.tabc_count;
    for (int i = tid0; i < a.tabc_count; i += stride) {
      const int row = i / np, col = i - row * np;
      const size_t src = row == 0 ? (size_t)col : row == 1 ? (size_t)2 * ns * np + col : ((size_t)ns + row - 2) * np + col;
      const double f = row == 0 ? kh : 1.0;
      const double v = a.tab[src];
      a.tabc[i] = v;
      if (i < n_line) {
        const double d = col == np - 1 ? 0.0 : f * (a.tab[src + 1] - v);
        a.tab32[i] = make_float2((float)(f * v - col * d), (float)((np - 1) * d));
      }
    }
    if (a.l3cell) {
      // Cell (ia, ib, is) of lambda3 on the (a, b, S0) grid: the trilinear
      // interpolant on [is, is+1] x [ia, ia+1] x [ib, ib+1] written as a
      // polynomial in the normalised coordinates (u_s, u_a, u_b) in [0, 1]^3
      // (node coordinate = u (n - 1)):
      //   c0 + c1 u_s + c2 u_a + c3 u_b + c4 u_s u_a + c5 u_s u_b + c6 u_a u_b + c7 u_s u_a u_b,
      // from the corner differences; the upper neighbour of a last node is the
      // node itself (zero difference).  Stored as (c0, c3, c1, c5), (c2, c6, c4, c7).
      const int na = a.n_va, nb = a.n_vb;
      const double Ns = np - 1, Na = na - 1, Nb = nb - 1;
      float4 *cell = reinterpret_cast<float4 *>(a.tab32 + 2 * np);
      for (int c = tid0; c < na * nb * np; c += stride) {
        const int is = c % np, ab = c / np, ia = ab / nb, ib = ab - ia * nb;
        const int s1 = min(is + 1, np - 1), a1 = min(ia + 1, na - 1), b1 = min(ib + 1, nb - 1);
        auto f = [&](int sx, int ax, int bx) { return a.tab[((size_t)ns + ax * nb + bx) * np + sx]; };
        const double f000 = f(is, ia, ib), f100 = f(s1, ia, ib), f010 = f(is, a1, ib), f001 = f(is, ia, b1);
        const double f110 = f(s1, a1, ib), f101 = f(s1, ia, b1), f011 = f(is, a1, b1), f111 = f(s1, a1, b1);
        const double Ds = f100 - f000, Da = f010 - f000, Db = f001 - f000;
        const double Dsa = f110 - f100 - f010 + f000, Dsb = f101 - f100 - f001 + f000;
        const double Dab = f011 - f010 - f001 + f000;
        const double Dsab = f111 - f110 - f101 - f011 + f100 + f010 + f001 - f000;
        const double i = is, j = ia, l = ib;
        const double c7 = Ns * Na * Nb * Dsab;
        const double c4 = Ns * Na * (Dsa - l * Dsab), c5 = Ns * Nb * (Dsb - j * Dsab), c6 = Na * Nb * (Dab - i * Dsab);
        const double c1 = Ns * (Ds - j * Dsa - l * Dsb + j * l * Dsab);
        const double c2 = Na * (Da - i * Dsa - l * Dab + i * l * Dsab);
        const double c3 = Nb * (Db - i * Dsb - j * Dab + i * j * Dsab);
        const double c0 = f000 - i * Ds - j * Da - l * Db + i * j * Dsa + i * l * Dsb + j * l * Dab - i * j * l * Dsab;
        cell[2 * c] = make_float4((float)c0, (float)c3, (float)c1, (float)c5);
        cell[2 * c + 1] = make_float4((float)c2, (float)c6, (float)c4, (float)c7);
      }
    }
  } else if (a.model == FFRG_MODEL_FINITE_T) {
    for (int i = tid0; i <= z_count; i += stride)
      a.tab32[i] = i < z_count ? make_float2((float)(kh * a.tab[i]), (float)a.tab[z_count + i]) : make_float2(0.f, 0.f);
  } else {
    const int np = a.n_pts;
    for (int i = tid0; i < a.tab_count; i += stride) {
      const double f = i < z_count ? kh : 1.0;
      const int col = i % np;
      const double d = col == np - 1 ? 0.0 : f * (a.tab[i + 1] - a.tab[i]);
      a.tab32[i] = make_float2((float)(f * a.tab[i] - col * d), (float)((np - 1) * d));
    }
  }
  if (a.ext_done)
    for (int i = tid0; i < a.n_ext; i += stride) a.ext_done[i] = 0u;
  // per-external-point constants used by every work item of the main kernels
  // one FP64 exp per value: value i on CTA i mod G, thread i / G, so that a
  // large grid spreads them over SMs and a small one keeps them in parallel lanes
  for (int i = tid0 / (int)blockDim.x + gridDim.x * threadIdx.x; i < a.n_ext_p; i += stride)
    a.ext_pd[i] = ext_momentum(a, i);
  if (is_d4(a.model)) {
    for (int j = tid0; j < a.n_ext_ang; j += stride) {
      const double c = a.psi_x[j];
      a.psi_s[j] = sqrt(fmax(0.0, 1.0 - c * c));
    }
  }
}

__global__ void __launch_bounds__(kThreads) precompute_kernel(RhsArgs a) {
  // the main kernel, launched as its programmatic dependent, may start now:
  // its CTAs stage what does not depend on this kernel, then wait for it
  pdl_trigger();
  if (skipped(a)) return;
  precompute_body(a);
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
__device__ __forceinline__ const typename TabOf<T>::type *table_src(const RhsArgs &a);
template <>
__device__ __forceinline__ const double *table_src<double>(const RhsArgs &a) { return a.tabc ? a.tabc : a.tab; }
template <>
__device__ __forceinline__ const float2 *table_src<float>(const RhsArgs &a) { return a.tab32; }

template <typename T>
struct SmemLayout {
  using Tab = typename TabOf<T>::type;
  using P2 = typename Pair2<T>::type;
  Tab *tab;
  float4 *cw4;  // FP32 kernels: second-angle nodes in pairs (x_2j, x_2j+1, w_2j, w_2j+1)
  P2 *cw2;
  T *c1, *s1, *w1;
  // table entries in shared memory: FP64 values, or the FP32 layout
  static __device__ int entries(const RhsArgs &a) {
    return sizeof(T) == 4 ? a.tab32_count : (a.tabc_count ? a.tabc_count : a.tab_count);
  }
  // FP64 kernels whose tables exceed shared memory read them in place (L2)
  static __device__ bool in_global(const RhsArgs &a) { return sizeof(T) == 8 && a.tab_global; }
  __device__ SmemLayout(unsigned char *base, const RhsArgs &a) {
    const bool g = in_global(a);
    tab = g ? const_cast<Tab *>(table_src<T>(a)) : (Tab *)base;
    size_t off = g ? 0 : ((size_t)entries(a) * sizeof(Tab) + 15) & ~(size_t)15;
    cw4 = (float4 *)(base + off);
    if (sizeof(T) == 4) off += (size_t)((a.na2 + 1) / 2) * sizeof(float4);
    cw2 = (P2 *)(base + off);
    c1 = (T *)(cw2 + a.na2);
    s1 = c1 + a.na1;
    w1 = s1 + a.na1;
  }
};

__device__ __forceinline__ double table_value(double v) { return v; }
__device__ __forceinline__ float table_value(float2 v) { return v.x; }

// handle of the table row that starts `off` entries into the staged tables:
// an FP64 pointer, or an FP32 line row (Row32)
__device__ __forceinline__ const double *tab_row(const SmemLayout<double> &S, int off) { return S.tab + off; }
__device__ __forceinline__ Row32 tab_row(const SmemLayout<float> &S, int off) { return row32(S.tab + off); }

// angle rules into shared memory in the kernel precision.  S1 = false skips
// sqrt(1 - c^2), which only the d=4 models read (FP64, slow on this part);
// the choice is a template argument because a branch on the model here made
// the mixed d=4 main kernel 2 % slower (0.2107 -> 0.2152 ms on the d=4 vertex
// workload)
template <typename T, bool S1 = true>
__device__ __forceinline__ void stage_angles(const RhsArgs &a, SmemLayout<T> &S) {
  for (int i = threadIdx.x; i < a.na1; i += blockDim.x) {
    double c = a.a1_x[i];
    S.c1[i] = (T)c;
    if constexpr (S1) S.s1[i] = (T)sqrt(fmax(0.0, 1.0 - c * c));
    S.w1[i] = (T)a.a1_w[i];
  }
  for (int i = threadIdx.x; i < a.na2; i += blockDim.x) {
    S.cw2[i].x = (T)a.a2_x[i];
    S.cw2[i].y = (T)a.a2_w[i];
  }
  if (sizeof(T) == 4) {
    // an odd last node is paired with itself at weight 0
    for (int j = threadIdx.x; j < (a.na2 + 1) / 2; j += blockDim.x) {
      const int i0 = 2 * j, i1 = min(2 * j + 1, a.na2 - 1);
      S.cw4[j] = make_float4((float)a.a2_x[i0], (float)a.a2_x[i1], (float)a.a2_w[i0],
                             i1 > i0 ? (float)a.a2_w[i1] : 0.0f);
    }
  }
}

template <typename T>
__device__ bool main_prologue(const RhsArgs &a, SmemLayout<T> &S, uint64_t *bar) {
  bool ok = true;
  stage_angles<T>(a, S);   // rules of the plan: not written by the precompute kernel
  // launched as a programmatic dependent of the precompute kernel: wait here
  // for its writes (FP32 tables, radial factors, constants, counters)
  pdl_wait();
  if (!SmemLayout<T>::in_global(a))   // uniform over the block
    ok = stage_to_smem<typename TabOf<T>::type>(S.tab, table_src<T>(a), SmemLayout<T>::entries(a), bar, a.status);
  __syncthreads();
  return ok;
}

// ---------------------------------------------------------------------------
// 2. main kernels.  Work items are warp-sized: external point e x a chunk of
// `cr` outer rows (d=3: radial nodes; finite T: (Matsubara n, radial node)
// pairs; d=4: (radial node, first-angle node) pairs).  Lane l takes rows
// l, l+32, ... of its item and loops over the remaining angle nodes of each
// row in the kernel precision; each row sum, times the row's radial factor,
// enters the lane's accumulator (RowAcc), and the warp reduces its item with
// shuffles.
// The single-flow kernels take items from a device counter; the warp that
// completes the last item of an external point writes that output.  The
// serving kernel walks per-flow item ranges (outputs by a finalize kernel).
// One warp sums each item in a fixed order, so results depend neither on
// which warp took it nor on the grid.  `sa` is the argument block in shared
// memory that the out-of-line near-pole path reads.  Squared momenta enter
// lookups and propagators as y = sy s^2 (table offsets uy1..uy4).
// ---------------------------------------------------------------------------
// Per-lane accumulation of radial factor x row sum, then the warp's item sum
// (valid in lane 0).  FP64 kernels: FP64 FMA and an FP64 shuffle tree.  FP32
// kernels: Kahan-compensated FP32 over the lane's rows (error ~2u of the lane
// sum), then a shuffle tree on (hi, lo) FP32 pairs with an error-free
// two-sum at every level (Knuth's TwoSum), rounded to FP64 at the end: no
// FP64 arithmetic per row or per tree level.
template <typename T>
struct RowAcc;
template <>
struct RowAcc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double F, double x) { s = fma(F, x, s); }
  __device__ __forceinline__ double item_sum() const {
    double v = s;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
  }
};
template <>
struct RowAcc<float> {
  float s = 0.f, c = 0.f;  // running sum and Kahan compensation (value = s - c)
  __device__ __forceinline__ void add(float F, float x) {
    const float y = fmaf(F, x, -c);
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double item_sum() const {
    float hi = s, lo = -c;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float h2 = __shfl_down_sync(0xffffffffu, hi, o), l2 = __shfl_down_sync(0xffffffffu, lo, o);
      const float S = hi + h2, bp = S - hi;
      const float err = (hi - (S - bp)) + (h2 - bp);  // hi + h2 = S + err exactly
      lo = lo + l2 + err;
      hi = S;
    }
    return (double)hi + (double)lo;
  }
};

template <typename T>
__device__ __forceinline__ T radial_F(const RhsArgs &a, int o);
template <>
__device__ __forceinline__ double radial_F<double>(const RhsArgs &a, int o) { return a.radF[o]; }
template <>
__device__ __forceinline__ float radial_F<float>(const RhsArgs &a, int o) { return a.radF32[o]; }

template <typename T>
__device__ __forceinline__ T radial_q(const RhsArgs &a, int r);
template <>
__device__ __forceinline__ double radial_q<double>(const RhsArgs &a, int r) { return a.radq[r]; }
template <>
__device__ __forceinline__ float radial_q<float>(const RhsArgs &a, int r) { return a.radq32[r]; }

// Two second-angle nodes per step in packed FP32 arithmetic (FFMA2, FMUL2,
// FADD2: two lanes of FP32 in one instruction on sm_100 and later); the
// special functions, the saturating coordinate FMA and the table loads stay
// scalar.  Lookup of an FP32 line row at two arguments:
__device__ __forceinline__ float2 look2(Row32 r, float2 s2, float us, float uo, float2 nm1) {
  float2 u;
  asm("fma.rn.sat.f32 %0, %1, %2, %3;" : "=f"(u.x) : "f"(us), "f"(hw_lg2(s2.x)), "f"(uo));
  asm("fma.rn.sat.f32 %0, %1, %2, %3;" : "=f"(u.y) : "f"(us), "f"(hw_lg2(s2.y)), "f"(uo));
  const float2 t = __ffma2_rd(u, nm1, make_float2(12582912.0f, 12582912.0f));
  return make_float2(line_at(r, {__float_as_uint(t.x) << 3, u.x}), line_at(r, {__float_as_uint(t.y) << 3, u.y}));
}

// Propagator of two lines as G = N R, R = 1/(Zs D + m2e N), with the regulator
// form of reg_g: (N, D) = (1 - 2^{-y}, y) for y >= log2(e), (1, series g(y))
// below, and m2e = m^2 (finite T: m^2 + Zs om2s, the frequency part).  One
// reciprocal instead of two (reg_g's and the propagator's); branch-free
// (setp / selp).  Only for m^2 >= 0 and Z >= 0 (no near-pole test), where the
// denominator is >= 0.
__device__ __forceinline__ void prop2(float2 y, float2 Zs, float2 m2e, float2 &N, float2 &R) {
  const float2 E = make_float2(hw_ex2(-y.x), hw_ex2(-y.y));
  const float2 Nd = __ffma2_rn(E, make_float2(-1.0f, -1.0f), make_float2(1.0f, 1.0f));
  const float2 y2 = __fmul2_rn(y, y);
  float2 t = __ffma2_rn(y2, make_float2(-6.3553057516916001e-8f, -6.3553057516916001e-8f),
                        make_float2(5.2910945025509696e-6f, 5.2910945025509696e-6f));
  t = __ffma2_rn(y2, t, make_float2(-4.6253423887351317e-4f, -4.6253423887351317e-4f));
  t = __ffma2_rn(y2, t, make_float2(5.7762265046662109e-2f, 5.7762265046662109e-2f));
  const float2 gs = __ffma2_rn(y2, t, __ffma2_rn(y, make_float2(0.5f, 0.5f),
                                                 make_float2(1.4426950408889634f, 1.4426950408889634f)));
  float2 D;
  asm("{\n .reg .pred p, q;\n"
      " setp.lt.f32 p, %4, 0f3FB8AA3B;\n setp.lt.f32 q, %5, 0f3FB8AA3B;\n"
      " selp.f32 %0, 0f3F800000, %6, p;\n selp.f32 %1, 0f3F800000, %7, q;\n"
      " selp.f32 %2, %8, %4, p;\n selp.f32 %3, %9, %5, q;\n}"
      : "=f"(N.x), "=f"(N.y), "=f"(D.x), "=f"(D.y)
      : "f"(y.x), "f"(y.y), "f"(Nd.x), "f"(Nd.y), "f"(gs.x), "f"(gs.y));
  const float2 den = __ffma2_rn(Zs, D, __fmul2_rn(m2e, N));
  R = make_float2(hw_rcp(den.x), hw_rcp(den.y));
}

// The same propagator for one line: G = N / (Zs D + m2e N), one reciprocal.
__device__ __forceinline__ float prop1(float y, float Zs, float m2e) {
  const float Nd = 1.0f - hw_ex2(-y);
  const float y2 = y * y;
  float t = fmaf(y2, -6.3553057516916001e-8f, 5.2910945025509696e-6f);
  t = fmaf(y2, t, -4.6253423887351317e-4f);
  t = fmaf(y2, t, 5.7762265046662109e-2f);
  const float gs = fmaf(y2, t, fmaf(y, 0.5f, 1.4426950408889634f));
  float N, D;
  asm("{\n .reg .pred p;\n setp.lt.f32 p, %2, 0f3FB8AA3B;\n"
      " selp.f32 %0, 0f3F800000, %3, p;\n selp.f32 %1, %4, %2, p;\n}"
      : "=f"(N), "=f"(D)
      : "f"(y), "f"(Nd), "f"(gs));
  return N * hw_rcp(fmaf(Zs, D, m2e * N));
}

// One FP32 row of angle nodes j0 .. j1-1 without the near-pole test: pairs
// of nodes in packed FP32 with the one-reciprocal propagator, an odd last
// node alone.  d=3: sum_j v_j G(|q+p|) at y_j = by + ty c_j.
__device__ __forceinline__ float d3_row_x2(const SmemLayout<float> &S, const KConst<float> &kc, Row32 Zt, int np,
                                           float by, float ty, int j0, int j1) {
  const float nm1 = (float)(np - 1);
  const float2 nm1v = make_float2(nm1, nm1), byv = make_float2(by, by), tyv = make_float2(ty, ty);
  const float2 m2v = make_float2(kc.m2, kc.m2);
  float2 rs = make_float2(0.0f, 0.0f);
  int j = j0;
  for (; j + 1 < j1; j += 2) {
    const float2 y = __ffma2_rn(tyv, make_float2(S.c1[j], S.c1[j + 1]), byv);
    const float2 Z = look2(Zt, y, kc.us, kc.uy1, nm1v);
    float2 N, R;
    prop2(y, Z, m2v, N, R);
    rs = __ffma2_rn(__fmul2_rn(make_float2(S.w1[j], S.w1[j + 1]), N), R, rs);
  }
  float t = rs.x + rs.y;
  if (j < j1) {
    const float y = fmaf(ty, S.c1[j], by);
    t = fmaf(S.w1[j], prop1(y, look(Zt, y, kc.us, kc.uy1, np), kc.m2), t);
  }
  return t;
}

// Finite T: sum_j v_j lam(j, s) G(j, s) of one K row from the (Z, lambda)
// node pairs of its stack row (interpolation weight form), om2s the row's
// scaled frequency^2 (mass term m^2 + Zs om2s per line).
__device__ __forceinline__ float ftk_row_x2(const SmemLayout<float> &S, const KConst<float> &kc, const float2 *zl,
                                            int np, int na1, float om2s, float by, float ty) {
  const float2 byv = make_float2(by, by), tyv = make_float2(ty, ty), omv = make_float2(om2s, om2s);
  const float2 m2v = make_float2(kc.m2, kc.m2);
  float2 rs = make_float2(0.0f, 0.0f);
  int j = 0;
  for (; j + 1 < na1; j += 2) {
    const float2 y = __ffma2_rn(tyv, make_float2(S.c1[j], S.c1[j + 1]), byv);
    int i0, i1;
    float w0, w1;
    lerp_pos(y.x, kc.us, kc.uy1, np, i0, w0);
    lerp_pos(y.y, kc.us, kc.uy1, np, i1, w1);
    const float2 a0 = zl[i0], b0 = zl[i0 + 1], a1 = zl[i1], b1 = zl[i1 + 1];
    const float2 Z = make_float2(fmaf(w0, b0.x - a0.x, a0.x), fmaf(w1, b1.x - a1.x, a1.x));
    const float2 L = make_float2(fmaf(w0, b0.y - a0.y, a0.y), fmaf(w1, b1.y - a1.y, a1.y));
    float2 N, R;
    prop2(y, Z, __ffma2_rn(Z, omv, m2v), N, R);
    rs = __ffma2_rn(__fmul2_rn(__fmul2_rn(make_float2(S.w1[j], S.w1[j + 1]), L), N), R, rs);
  }
  float t = rs.x + rs.y;
  if (j < na1) {
    const float y = fmaf(ty, S.c1[j], by);
    int i0;
    float w0;
    lerp_pos(y, kc.us, kc.uy1, np, i0, w0);
    const float2 a0 = zl[i0], b0 = zl[i0 + 1];
    const float Z = fmaf(w0, b0.x - a0.x, a0.x), L = fmaf(w0, b0.y - a0.y, a0.y);
    t = fmaf(S.w1[j] * L, prop1(y, Z, fmaf(Z, om2s, kc.m2)), t);
  }
  return t;
}

// d=3, T=0: row = (radial node o, block of jb angle nodes);
// sum_j v_j G(|q+p|)
template <typename T, bool POLE>
__device__ __forceinline__ RowAcc<T> d3_witem(const RhsArgs &a, const RhsArgs *sa, const SmemLayout<T> &S,
                                           const KConst<T> &kc, int e, int c, int lane) {
  const T us = kc.us, uy1 = kc.uy1, sy = kc.sy;
  const int np = a.n_pts, na1 = a.na1, jb = a.jb, nblk = (na1 + jb - 1) / jb;
  const auto Zt = tab_row(S, 0);
  const T p = (T)((e < a.n_ext_p) ? a.ext_pd[e] : 0.0);
  const int r0 = c * a.cr, r1 = min(r0 + a.cr, a.nr * nblk);
  RowAcc<T> acc;
  for (int rr = r0 + lane; rr < r1; rr += 32) {
    const int o = rr / nblk, j0 = (rr - o * nblk) * jb, j1 = min(j0 + jb, na1);
    const T q = radial_q<T>(a, o);
    // explicit FMAs: the single-flow and serving kernels must round alike
    const T by = fma(q, q, p * p) * sy, ty = (T)2 * q * p * sy;
    T rs = 0;
    if constexpr (sizeof(T) == 4 && !POLE) rs = d3_row_x2(S, kc, Zt, np, by, ty, j0, j1);
    else for (int j = j0; j < j1; ++j) {
      const T y = fma(ty, S.c1[j], by);   // sy |q+p|^2, >= 0 up to rounding; lookups clamp
      const T Z = look(Zt, y, us, uy1, np);
      auto pole = [&]() { return pole_d3(sa, e, o, j); };
      rs = fma(S.w1[j], inv_prop<POLE>(a, Z, y, (T)0, kc, pole), rs);
    }
    acc.add(radial_F<T>(a, o), rs);
  }
  return acc;
}

// finite-T lookups of Z and lambda at stack row srow: FP64 tables [table][row][pt];
// FP32 (Z, lambda) node pairs [row][pt] (+ one zero pair)
__device__ __forceinline__ void zl_lookup(const double *tab, const RhsArgs &a, int srow, int i0, double w, double &Z,
                                          double &L) {
  Z = lerp_at(tab + (size_t)srow * a.n_pts, i0, w);
  L = lerp_at(tab + ((size_t)a.n_stack + srow) * a.n_pts, i0, w);
}
__device__ __forceinline__ void zl_lookup(const float2 *tab, const RhsArgs &a, int srow, int i0, float w, float &Z,
                                          float &L) {
  const float2 *row = tab + (size_t)srow * a.n_pts;
  const float2 v0 = row[i0], v1 = row[i0 + 1];
  Z = fmaf(w, v1.x - v0.x, v0.x);
  L = fmaf(w, v1.y - v0.y, v0.y);
}

// finite T, factorised through the angle-integrated kernel K(p, q): the
// angular sum of a loop row depends on the shifted frequency index
// n' = n + m only through its stack row j (|n'| bosonic; n' or -n'-1
// fermionic) and that row's frequency^2, so
//   K[j][ip][r] = sum_c v_c lam(j, |q_r + p_ip|) G(j, |q_r + p_ip|)
// is evaluated once per (j, p, r), j = 0 .. N+M-1, and
//   I(m, p) = sum_n sum_r F(n, r) K[j(n + m)][p][r]
// is a contraction over loop frequencies and radial nodes (ft_contract).
// The same discrete sum as the direct loop over (m, n, r, c), with (N+M)
// instead of (2N+1) M angular sums per (p, r).
template <typename T, bool POLE>
__device__ __forceinline__ void ftk_rows(const RhsArgs &a, const RhsArgs *sa, const SmemLayout<T> &S,
                                         const KConst<T> &kc, int outer, int c, int lane,
                                         const T *q_loc = nullptr, const T *p_loc = nullptr) {
  const T us = kc.us, uy1 = kc.uy1, sy = kc.sy;
  const int np = a.n_pts, na1 = a.na1, nr = a.nr;
  const int jk = outer / a.n_ext_p, ip = outer - jk * a.n_ext_p;
  const int srow = min(jk, a.n_stack - 1);
  const T om = kc.twopiT * ((T)jk + (T)(a.stat ? 0.5 : 0.0));   // omega_j or nu_j
  const T om2s = om * om * kc.som;
  // p and q from the precompute's arrays, or (q_loc, p_loc) from the block's
  // own copies of the same values
  const T p = p_loc ? p_loc[ip] : (T)a.ext_pd[ip];
  T *K = (T *)a.kbuf + ((size_t)jk * a.n_ext_p + ip) * nr;
  const int r0 = c * a.cr, r1 = min(r0 + a.cr, nr);
  for (int r = r0 + lane; r < r1; r += 32) {
    const T q = q_loc ? q_loc[r] : radial_q<T>(a, r);
    const T by = fma(q, q, p * p) * sy, ty = (T)2 * q * p * sy;   // explicit FMAs, as in d3_witem
    T rs = 0;
    if constexpr (sizeof(T) == 4 && !POLE) rs = ftk_row_x2(S, kc, S.tab + (size_t)srow * np, np, na1, om2s, by, ty);
    else for (int j = 0; j < na1; ++j) {
      const T y = fma(ty, S.c1[j], by);
      int i0;
      T w, Z, Lv;
      lerp_pos(y, us, uy1, np, i0, w);
      zl_lookup(S.tab, a, srow, i0, w, Z, Lv);
      auto pole = [&]() { return pole_ftk(sa, ip, jk, r, j); };
      rs = fma(S.w1[j] * Lv, inv_prop<POLE>(a, Z, y, om2s, kc, pole), rs);
    }
    K[r] = rs;
  }
}

// Barrier of a group of threads of the block: the whole block (id 0), or the
// gsize threads of named barrier id (1..15).
__device__ __forceinline__ void group_sync(int id, int gsize) {
  if (id == 0) __syncthreads();
  else asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(gsize) : "memory");
}

// I(m, p) of external point e = (ip, m) from K and the radial factors, by a
// group of gsize threads (gtid = thread index in the group; the block with
// bar_id 0, else named barrier bar_id) in a fixed order: warp w of the group
// takes the frequency rows w, w + nw, ... (K row of the shifted frequency
// n + m, contiguous in r), four at a time, lane l the radial nodes l, l + 32,
// ... of each, accumulating in the precision's RowAcc; each warp reduces with
// its tree, thread 0 of the group adds the warp sums in order (valid there).
// Every thread of the group must call it; red holds gsize/32 doubles.

template <typename T>
__device__ __forceinline__ double ft_contract(const RhsArgs &a, int e, double *red, int gtid, int gsize, int bar_id) {
  const int nm = a.n_ext_ang, ip = e / nm, m = e - ip * nm, nr = a.nr;
  const int n_lo = -a.N - a.stat;
  const int lane = gtid & 31, nw = gsize >> 5;
  const T *K = (const T *)a.kbuf;
  auto krow = [&](int row) {   // K row of the shifted frequency of loop index row + n_lo
    return K + ((size_t)stack_index(a.stat, row + n_lo + m) * a.n_ext_p + ip) * nr;
  };
  RowAcc<T> acc;
  int row = gtid >> 5;
  // four rows at a time: their eight loads per node are in flight together
  for (; row + 3 * nw < a.nfreq; row += 4 * nw) {
    const T *K0 = krow(row), *K1 = krow(row + nw), *K2 = krow(row + 2 * nw), *K3 = krow(row + 3 * nw);
    const int o = row * nr, dn = nw * nr;   // radF rows of the four loop indices
    for (int r = lane; r < nr; r += 32) {
      const T k0 = __ldcg(K0 + r), k1 = __ldcg(K1 + r), k2 = __ldcg(K2 + r), k3 = __ldcg(K3 + r);
      const T f0 = radial_F<T>(a, o + r), f1 = radial_F<T>(a, o + dn + r);
      const T f2 = radial_F<T>(a, o + 2 * dn + r), f3 = radial_F<T>(a, o + 3 * dn + r);
      acc.add(f0, k0);
      acc.add(f1, k1);
      acc.add(f2, k2);
      acc.add(f3, k3);
    }
  }
  for (; row < a.nfreq; row += nw) {
    const T *Kr = krow(row);
    const int o = row * nr;
    for (int r = lane; r < nr; r += 32) acc.add(radial_F<T>(a, o + r), __ldcg(Kr + r));
  }
  const double w = acc.item_sum();
  if (lane == 0) red[gtid >> 5] = w;
  group_sync(bar_id, gsize);
  double t = 0.0;
  if (gtid == 0)
    for (int j = 0; j < nw; ++j) t += red[j];
  group_sync(bar_id, gsize);
  return t;
}

// D4_FULL three-point vertex lambda3(S0, a, b): the tables hold rows
// (ia, ib) of the log grid in S0 for uniform nodes of a and b on [-1, 1].
// For a vertex with legs k1, k2, k3 (sum 0; squared magnitudes s1, s2, s3):
// a = cosine between k1 and k2, b = (s1 - s2)/(s1 + s2), clamped to [-1, 1]
// with NaN to -1; linear between nodes in ln S0, a and b.  S0 enters through
// the table coordinate of y3 = (s1 + s2 + s3) sy with offset uy3 (lerp_pos).
// FP64 kernels take a = (s3 - s1 - s2)/(2 sqrt(s1 s2)) as the oracle does.
// In FP32 that form cancels when one leg is short (an error u p^2 divided by
// q p); the FP32 kernels take the cosine from the leg components instead
// (see d4_witem), which keeps its error near u.
__device__ __forceinline__ void shape_pos(double v, int m, int &i, double &w) {
  if (m < 2) {
    i = 0;
    w = 0.0;
    return;
  }
  v = v >= -1.0 ? (v <= 1.0 ? v : 1.0) : -1.0;
  const double u = 0.5 * (v + 1.0) * (m - 1);
  i = min((int)u, m - 2);
  w = u - i;
}
__device__ __forceinline__ void shape_pos(float v, int m, int &i, float &w) {
  if (m < 2) {
    i = 0;
    w = 0.0f;
    return;
  }
  float u1;  // (v + 1)/2 saturated to [0, 1], NaN to 0
  asm("fma.rn.sat.f32 %0, %1, 0f3F000000, 0f3F000000;" : "=f"(u1) : "f"(v));
  const float u = u1 * (float)(m - 1);
  i = min((int)u, m - 2);
  w = u - (float)i;
}
__device__ __forceinline__ double shape_a(double s1, double s2, double s3) {
  return (s3 - s1 - s2) / (2.0 * sqrt(s1 * s2));
}
__device__ __forceinline__ double shape_b(double s1, double s2) { return (s1 - s2) / (s1 + s2); }
__device__ __forceinline__ float shape_b(float s1, float s2) { return (s1 - s2) * hw_rcp(s1 + s2); }
// cosine between q and -(q + p) at |q+p|^2 = A2: (s3-s1-s2)/(2 sqrt(s1 s2)) in
// FP64; -(q + p c1)/|q + p| in FP32 (q.(q+p) = q (q + p c1), no cancellation)
__device__ __forceinline__ double va_shape_a(double, double, double, double q2, double A2, double p2) {
  return shape_a(q2, A2, p2);
}
__device__ __forceinline__ float va_shape_a(float q, float p, float c1, float, float A2, float) {
  return -fmaf(p, c1, q) * rsqrtf(A2);
}

__device__ __forceinline__ float lam3_full(const RhsArgs &a, Row32 L3, float y3, float us, float uy3, float va,
                                          float vb) {
  const int np = a.n_pts, na = a.n_va, nb = a.n_vb;
  int ia, ib;
  float wa, wb;
  const Pos32 ps = line_pos(y3, us, uy3, (float)(np - 1));
  shape_pos(va, na, ia, wa);
  shape_pos(vb, nb, ib, wb);
  const Row32 r00 = row32_at(L3, (ia * nb + ib) * np);
  const int db = nb > 1 ? np : 0, da = na > 1 ? nb * np : 0;
  const float v00 = line_at(r00, ps), v01 = line_at(row32_at(r00, db), ps);
  const float v10 = line_at(row32_at(r00, da), ps), v11 = line_at(row32_at(r00, da + db), ps);
  return (1.0f - wa) * ((1.0f - wb) * v00 + wb * v01) + wa * ((1.0f - wb) * v10 + wb * v11);
}
template <typename T, typename Tab>
__device__ __forceinline__ T lam3_full(const RhsArgs &a, const Tab *L3, T y3, T us, T uy3, T va, T vb) {
  const int np = a.n_pts, na = a.n_va, nb = a.n_vb;
  int i0, ia, ib;
  T w, wa, wb;
  lerp_pos(y3, us, uy3, np, i0, w);
  shape_pos(va, na, ia, wa);
  shape_pos(vb, nb, ib, wb);
  const Tab *r00 = L3 + (size_t)(ia * nb + ib) * np;
  const int db = nb > 1 ? np : 0, da = na > 1 ? nb * np : 0;
  const T v00 = lerp_at(r00, i0, w), v01 = lerp_at(r00 + db, i0, w);
  const T v10 = lerp_at(r00 + da, i0, w), v11 = lerp_at(r00 + da + db, i0, w);
  return ((T)1 - wa) * (((T)1 - wb) * v00 + wb * v01) + wa * (((T)1 - wb) * v10 + wb * v11);
}

// lambda3 from the FP32 cell polynomials: the cell index from the three
// normalised coordinates by the floor trick of line_pos (bit pattern of
// 1.5 2^23 + i), one address from the three biased indices, two 16-byte
// shared loads and the polynomial in four FMAs.  Saturation maps the shape
// variables to [0, 1] (NaN to 0) as shape_pos does; the last node of each
// axis is a cell of its own whose differences are zero.
struct Cell32 {
  unsigned base;  // shared address of the cells minus 32 x the bias of the three biased indices
  int nb, np;
  float Ns, Na, Nb;
};
__device__ __forceinline__ Cell32 cell32(const RhsArgs &a, const SmemLayout<float> &S) {
  constexpr unsigned kBias = 0x4B400000u;  // bit pattern of 1.5 2^23
  Cell32 C;
  C.nb = a.n_vb;
  C.np = a.n_pts;
  C.base = (unsigned)__cvta_generic_to_shared(S.tab + 2 * a.n_pts) -
           32u * kBias * (unsigned)((a.n_vb + 1) * a.n_pts + 1);
  C.Ns = (float)(a.n_pts - 1);
  C.Na = (float)(a.n_va - 1);
  C.Nb = (float)(a.n_vb - 1);
  return C;
}
__device__ __forceinline__ float cell_eval(unsigned addr, float us, float ua, float ub) {
  float4 A, B;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(A.x), "=f"(A.y), "=f"(A.z), "=f"(A.w) : "r"(addr));
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4+16];" : "=f"(B.x), "=f"(B.y), "=f"(B.z), "=f"(B.w) : "r"(addr));
  const float2 u2 = make_float2(us, us);
  const float2 P03 = __ffma2_rn(u2, make_float2(A.z, A.w), make_float2(A.x, A.y));   // c0 + c1 u_s, c3 + c5 u_s
  const float2 P27 = __ffma2_rn(u2, make_float2(B.z, B.w), make_float2(B.x, B.y));   // c2 + c4 u_s, c6 + c7 u_s
  const float2 t = __ffma2_rn(make_float2(ua, ua), P27, P03);   // the u_b^0 and u_b^1 parts
  return fmaf(ub, t.y, t.x);
}
__device__ __forceinline__ unsigned cell_addr(const Cell32 &C, float us, float ua, float ub) {
  const unsigned bs = __float_as_uint(__fmaf_rd(us, C.Ns, 12582912.0f));
  const unsigned ba = __float_as_uint(__fmaf_rd(ua, C.Na, 12582912.0f));
  const unsigned bb = __float_as_uint(__fmaf_rd(ub, C.Nb, 12582912.0f));
  return C.base + 32u * ((ba * (unsigned)C.nb + bb) * (unsigned)C.np + bs);
}
__device__ __forceinline__ float sat_half(float v) {  // (v + 1)/2 saturated to [0, 1], NaN to 0
  float u;
  asm("fma.rn.sat.f32 %0, %1, 0f3F000000, 0f3F000000;" : "=f"(u) : "f"(v));
  return u;
}
__device__ __forceinline__ float lam3_cell(const Cell32 &C, float y3, float us, float uy3, float va, float vb) {
  float u_s;
  asm("fma.rn.sat.f32 %0, %1, %2, %3;" : "=f"(u_s) : "f"(us), "f"(hw_lg2(y3)), "f"(uy3));
  const float u_a = sat_half(va), u_b = sat_half(vb);
  return cell_eval(cell_addr(C, u_s, u_a, u_b), u_s, u_a, u_b);
}

// sum_b w_b G(|q - p2|) lam3(.., b) lam3(.., c) of one (radial, first-angle)
// row of the three-point block in FP32 (arguments as in d4_witem); the even
// and odd nodes are summed separately and added at the end.
__device__ __forceinline__ float tp_sum_x2(const RhsArgs &a, const SmemLayout<float> &S, const KConst<float> &kc,
                                           Row32 Zt, Row32 L3, float b0, float t2y, float by, float sy_ab) {
  const float us = kc.us, uy1 = kc.uy1, uy3 = kc.uy3, nm1 = (float)(a.n_pts - 1);
  const float2 nm1v = make_float2(nm1, nm1), b0v = make_float2(b0, b0), nt2 = make_float2(-t2y, -t2y);
  const float2 byv = make_float2(by, by), sabv = make_float2(sy_ab, sy_ab), m2v = make_float2(kc.m2, kc.m2);
  float2 rs = make_float2(0.0f, 0.0f);
  const int npair = (a.na2 + 1) >> 1;
#pragma unroll 8   // independent pairs in flight: 8 % faster than no unrolling, 2 % than 4
  for (int j = 0; j < npair; ++j) {
    const float4 cw = S.cw4[j];
    const float2 By = __ffma2_rn(nt2, make_float2(cw.x, cw.y), b0v);   // sy |q - p2|^2
    const float2 ZB = look2(Zt, By, us, uy1, nm1v);
    float2 N, R;
    prop2(By, ZB, m2v, N, R);
    const float2 lb = look2(L3, __fadd2_rn(byv, By), us, uy3, nm1v);
    const float2 lc = look2(L3, __fadd2_rn(sabv, By), us, uy3, nm1v);
    const float2 P = __fmul2_rn(__fmul2_rn(__fmul2_rn(make_float2(cw.z, cw.w), N), R), lb);
    rs = __ffma2_rn(P, lc, rs);
  }
  return rs.x + rs.y;
}

// sum_b w_b G(|q - p2|) lam3(.., b) lam3(.., c) of one (radial, first-angle)
// row of the D4_FULL three-point block in FP32 with lambda3 cells (arguments
// as in d4_witem): the two vertex lookups of a node share their coordinate
// arithmetic in packed FP32 (FFMA2).  Shape variables from the leg components
// as in d4_witem's line-row branch.
template <bool POLE>
__device__ __forceinline__ float tp_full_cell(const RhsArgs &a, const RhsArgs *sa, const SmemLayout<float> &S,
                                              const KConst<float> &kc, int e, int r, int ia, float q, float q2,
                                              float A2, float Ay, float b0, float t2y, float by, float sy_ab,
                                              float qs1, float x1, float x2, float psp, float hc, float hs) {
  const Cell32 C = cell32(a, S);
  const Row32 Zt = tab_row(S, 0);
  const float us = kc.us, uy1 = kc.uy1, uy3 = kc.uy3;
  const float rA = hw_rsqrt(A2), qy = q2 * kc.sy, qs1sq = qs1 * qs1;
  const float2 magic = make_float2(12582912.0f, 12582912.0f);
  float rs = 0.0f;
  for (int b = 0; b < a.na2; ++b) {
    const float2 cw = S.cw2[b];
    const float By = fmaf(-t2y, cw.x, b0);   // sy |q - p2|^2
    const float ZB = look(Zt, By, us, uy1, a.n_pts);
    float GB;
    if constexpr (POLE) {
      auto pole_b = [&]() { return pole_d4<FFRG_MODEL_D4_FULL>(sa, e, r, ia, b); };
      GB = inv_prop<true>(a, ZB, By, 0.0f, kc, pole_b);
    } else {
      GB = prop1(By, ZB, kc.m2);
    }
    const float rB = hw_rsqrt(By * kc.isy);
    const float a_b = (fmaf(hs, cw.x, hc) - q) * rB;                        // cos(q, -(q - p2))
    const float y1 = qs1 * cw.x, y2 = y1 - psp, z2 = qs1sq * fmaf(-cw.x, cw.x, 1.0f);
    const float a_c = -fmaf(x1, x2, fmaf(y1, y2, z2)) * rA * rB;             // cos(q + p1, -(q - p2))
    const float db = qy + By, dc = Ay + By, rbc = hw_rcp(db * dc);
    const float b_b = (qy - By) * dc * rbc, b_c = (Ay - By) * db * rbc;
    // legs (q, -(q-p2), p2) and (q+p1, -(q-p2), -(p1+p2))
    float2 u_s;
    asm("fma.rn.sat.f32 %0, %1, %2, %3;" : "=f"(u_s.x) : "f"(us), "f"(hw_lg2(by + By)), "f"(uy3));
    asm("fma.rn.sat.f32 %0, %1, %2, %3;" : "=f"(u_s.y) : "f"(us), "f"(hw_lg2(sy_ab + By)), "f"(uy3));
    const float2 u_a = make_float2(sat_half(a_b), sat_half(a_c)), u_b = make_float2(sat_half(b_b), sat_half(b_c));
    const float2 ts = __ffma2_rd(u_s, make_float2(C.Ns, C.Ns), magic);
    const float2 ta = __ffma2_rd(u_a, make_float2(C.Na, C.Na), magic);
    const float2 tb = __ffma2_rd(u_b, make_float2(C.Nb, C.Nb), magic);
    const unsigned nb = (unsigned)C.nb, np = (unsigned)C.np;
    const unsigned ab = C.base + 32u * ((__float_as_uint(ta.x) * nb + __float_as_uint(tb.x)) * np + __float_as_uint(ts.x));
    const unsigned ac = C.base + 32u * ((__float_as_uint(ta.y) * nb + __float_as_uint(tb.y)) * np + __float_as_uint(ts.y));
    const float lb = cell_eval(ab, u_s.x, u_a.x, u_b.x), lc = cell_eval(ac, u_s.y, u_a.y, u_b.y);
    rs = fmaf(cw.y * GB, lb * lc, rs);
  }
  return rs;
}

// The same sum without a near-pole test, two second-angle nodes per step in
// packed FP32 (the node pairs of tp_sum_x2, an odd last node paired with
// itself at weight 0); the four vertex lookups of a step stay scalar.
__device__ __forceinline__ float tp_full_cell_x2(const RhsArgs &a, const SmemLayout<float> &S, const KConst<float> &kc,
                                                 float q, float q2, float A2, float Ay, float b0, float t2y, float by,
                                                 float sy_ab, float qs1, float x1, float x2, float psp, float hc,
                                                 float hs) {
  const Cell32 C = cell32(a, S);
  const Row32 Zt = tab_row(S, 0);
  const float us = kc.us, uy3 = kc.uy3, nm1 = (float)(a.n_pts - 1);
  const float nrA = -hw_rsqrt(A2), qy = q2 * kc.sy, qs1sq = qs1 * qs1, x12 = x1 * x2;
  const float2 magic = make_float2(12582912.0f, 12582912.0f);
  float2 rs = make_float2(0.0f, 0.0f);
  const int npair = (a.na2 + 1) >> 1;
  for (int j = 0; j < npair; ++j) {
    const float4 cw = S.cw4[j];
    const float2 c2 = make_float2(cw.x, cw.y);
    const float2 By = __ffma2_rn(make_float2(-t2y, -t2y), c2, make_float2(b0, b0));   // sy |q - p2|^2
    const float2 ZB = look2(Zt, By, us, kc.uy1, make_float2(nm1, nm1));
    float2 N, R;
    prop2(By, ZB, make_float2(kc.m2, kc.m2), N, R);
    const float2 B2 = __fmul2_rn(By, make_float2(kc.isy, kc.isy));
    const float2 rB = make_float2(hw_rsqrt(B2.x), hw_rsqrt(B2.y));
    // cos(q, -(q - p2)) and cos(q + p1, -(q - p2))
    const float2 a_b = __fmul2_rn(__ffma2_rn(make_float2(hs, hs), c2, make_float2(hc - q, hc - q)), rB);
    const float2 y1 = __fmul2_rn(make_float2(qs1, qs1), c2);
    const float2 z2 = __fmul2_rn(make_float2(qs1sq, qs1sq), __ffma2_rn(__fmul2_rn(c2, make_float2(-1.0f, -1.0f)), c2,
                                                                     make_float2(1.0f, 1.0f)));
    const float2 ac0 = __ffma2_rn(y1, __fadd2_rn(y1, make_float2(-psp, -psp)), __fadd2_rn(z2, make_float2(x12, x12)));
    const float2 a_c = __fmul2_rn(ac0, __fmul2_rn(rB, make_float2(nrA, nrA)));
    // b = (s1 - s2)/(s1 + s2) of both vertices from one reciprocal
    const float2 db = __fadd2_rn(make_float2(qy, qy), By), dc = __fadd2_rn(make_float2(Ay, Ay), By);
    const float2 P = __fmul2_rn(db, dc);
    const float2 rbc = make_float2(hw_rcp(P.x), hw_rcp(P.y));
    const float2 nBy = __fmul2_rn(By, make_float2(-1.0f, -1.0f));
    const float2 b_b = __fmul2_rn(__fmul2_rn(__fadd2_rn(make_float2(qy, qy), nBy), dc), rbc);
    const float2 b_c = __fmul2_rn(__fmul2_rn(__fadd2_rn(make_float2(Ay, Ay), nBy), db), rbc);
    const float2 yb = __fadd2_rn(make_float2(by, by), By), yc = __fadd2_rn(make_float2(sy_ab, sy_ab), By);
    float lb[2], lc[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float2 u_s;
      asm("fma.rn.sat.f32 %0, %1, %2, %3;" : "=f"(u_s.x) : "f"(us), "f"(hw_lg2(h ? yb.y : yb.x)), "f"(uy3));
      asm("fma.rn.sat.f32 %0, %1, %2, %3;" : "=f"(u_s.y) : "f"(us), "f"(hw_lg2(h ? yc.y : yc.x)), "f"(uy3));
      const float2 u_a = make_float2(sat_half(h ? a_b.y : a_b.x), sat_half(h ? a_c.y : a_c.x));
      const float2 u_b = make_float2(sat_half(h ? b_b.y : b_b.x), sat_half(h ? b_c.y : b_c.x));
      const float2 ts = __ffma2_rd(u_s, make_float2(C.Ns, C.Ns), magic);
      const float2 ta = __ffma2_rd(u_a, make_float2(C.Na, C.Na), magic);
      const float2 tb = __ffma2_rd(u_b, make_float2(C.Nb, C.Nb), magic);
      const unsigned nb = (unsigned)C.nb, np = (unsigned)C.np;
      const unsigned ab =
          C.base + 32u * ((__float_as_uint(ta.x) * nb + __float_as_uint(tb.x)) * np + __float_as_uint(ts.x));
      const unsigned ac =
          C.base + 32u * ((__float_as_uint(ta.y) * nb + __float_as_uint(tb.y)) * np + __float_as_uint(ts.y));
      lb[h] = cell_eval(ab, u_s.x, u_a.x, u_b.x);
      lc[h] = cell_eval(ac, u_s.y, u_a.y, u_b.y);
    }
    const float2 W = __fmul2_rn(__fmul2_rn(make_float2(cw.z, cw.w), N), R);
    rs = __ffma2_rn(__fmul2_rn(W, make_float2(lb[0], lb[1])), make_float2(lc[0], lc[1]), rs);
  }
  return rs.x + rs.y;
}

// d=4 vertex expansion: row = (radial node r, first-angle node ia), inner loop
// over the second-angle nodes for the three-point block.  FULL: the D4_FULL
// model (lambda3 on (S0, a, b); compact tables Z | lambda4 | lambda3 rows).
template <typename T, bool POLE, bool FULL = false, bool CELL = false>
__device__ __forceinline__ RowAcc<T> d4_witem(const RhsArgs &a, const RhsArgs *sa, const SmemLayout<T> &S,
                                           const KConst<T> &kc, int e, int c, int lane) {
  const T us = kc.us, sy = kc.sy;
  const int np = a.n_pts, np_ = a.n_ext_p, npsi = a.n_ext_ang, na1 = a.na1;
  const auto Zt = tab_row(S, 0), L3 = tab_row(S, (FULL ? 2 : 1) * np), L4 = tab_row(S, (FULL ? 1 : 2) * np);
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
  const T p = (T)pd, p2 = p * p;
  const T cpsi = (T)(block == 1 ? a.psi_x[jp] : 1.0), spsi = (T)(block == 1 ? a.psi_s[jp] : 0.0);
  const T C2 = (T)2 * p2 * ((T)1 + cpsi);
  const int o0 = c * a.cr, o1 = min(o0 + a.cr, a.nr);
  const int rows = (o1 - o0) * na1;
  const int dr = 32 / na1, dia = 32 % na1;  // row step of one lane in (r, ia)
  RowAcc<T> acc;
  int r = o0 + lane / na1, ia = lane % na1;
  for (int row = lane; row < rows; row += 32) {
    const T q = radial_q<T>(a, r), q2 = q * q, qp = q * p, c1 = S.c1[ia];
    const T A2 = q2 + p2 + (T)2 * qp * c1;   // >= 0 up to rounding; lookups clamp
    const T Ay = A2 * sy;
    const T ZA = look(Zt, Ay, us, kc.uy1, np);
    auto pole_a = [&]() { return pole_d4<FULL ? FFRG_MODEL_D4_FULL : FFRG_MODEL_D4_VERTEX>(sa, e, r, ia, -1); };
    const T GA = inv_prop<POLE>(a, ZA, Ay, (T)0, kc, pole_a);
    T v;
    if (block == 0) {
      const T l4 = look(L4, (q2 + p2) * sy, us, kc.uy2, np);
      T l3;
      if constexpr (CELL) l3 = lam3_cell(cell32(a, S), (q2 + A2 + p2) * sy, us, kc.uy3,
                                         va_shape_a(q, p, c1, q2, A2, p2), shape_b(q2, A2));
      else if constexpr (FULL) l3 = lam3_full(a, L3, (q2 + A2 + p2) * sy, us, kc.uy3, va_shape_a(q, p, c1, q2, A2, p2),
                                         shape_b(q2, A2));   // legs q, -(q+p), p
      else l3 = look(L3, (q2 + A2 + p2) * sy, us, kc.uy3, np);
      v = kc.sw2 * ((T)(-0.5) * l4 + l3 * l3 * GA);
    } else if (block == 2) {
      const T l4 = look(L4, (q2 + A2 + (T)2 * p2) * sy, us, kc.uy4, np);
      v = kc.sw2 * GA * l4 * l4;
    } else {
      const T uy1 = kc.uy1, uy3 = kc.uy3;
      T la;
      if constexpr (CELL)
        la = lam3_cell(cell32(a, S), (q2 + A2 + p2) * sy, us, uy3, va_shape_a(q, p, c1, q2, A2, p2),
                       shape_b(q2, A2));
      else if constexpr (FULL)
        la = lam3_full(a, L3, (q2 + A2 + p2) * sy, us, uy3, va_shape_a(q, p, c1, q2, A2, p2),
                       shape_b(q2, A2));   // legs q, -(q+p1), p1
      else la = look(L3, (q2 + A2 + p2) * sy, us, uy3, np);
      // components (e1 along p1, e2 in the p1-p2 plane): q = q (c1, s1 c2, s1 s2'),
      // p1 = p (1, 0, 0), p2 = p (cpsi, spsi, 0)
      [[maybe_unused]] const T qs1 = q * S.s1[ia], x1 = q * c1 + p, x2 = q * c1 - p * cpsi, psp = p * spsi;
      [[maybe_unused]] const T hc = p * cpsi * c1, hs = p * spsi * S.s1[ia];   // q^.p2 = hc + hs c2
      const T base = q2 + p2, t1 = (T)2 * qp * cpsi * c1, t2 = (T)2 * qp * spsi * S.s1[ia];
      const T by = base * sy, b0 = (base - t1) * sy, t2y = t2 * sy, sy_ab = (A2 + C2) * sy;
      T rs = 0;
      if constexpr (sizeof(T) == 4 && !FULL && !POLE) rs = tp_sum_x2(a, S, kc, Zt, L3, b0, t2y, by, sy_ab);
      else if constexpr (CELL && !POLE) rs = tp_full_cell_x2(a, S, kc, q, q2, A2, Ay, b0, t2y, by, sy_ab, qs1, x1, x2,
                                                             psp, hc, hs);
      else if constexpr (CELL) rs = tp_full_cell<POLE>(a, sa, S, kc, e, r, ia, q, q2, A2, Ay, b0, t2y, by, sy_ab, qs1, x1,
                                                       x2, psp, hc, hs);
      else for (int b = 0; b < a.na2; ++b) {
        const auto cw = S.cw2[b];
        const T By = b0 - t2y * cw.x;   // sy |q - p2|^2
        const T ZB = look(Zt, By, us, uy1, np);
        auto pole_b = [&]() { return pole_d4<FULL ? FFRG_MODEL_D4_FULL : FFRG_MODEL_D4_VERTEX>(sa, e, r, ia, b); };
        T GB;
        if constexpr (sizeof(T) == 4 && !POLE) GB = prop1(By, ZB, kc.m2);   // one reciprocal
        else GB = inv_prop<POLE>(a, ZB, By, (T)0, kc, pole_b);
        T lb, lc;
        if constexpr (FULL) {
          T a_b, a_c, b_b, b_c;
          if constexpr (sizeof(T) == 8) {   // FP64: the oracle's form
            const T B2 = By;                  // sy = 1
            a_b = shape_a(q2, B2, p2);
            a_c = shape_a(A2, B2, C2);
            b_b = shape_b(q2, By);
            b_c = shape_b(Ay, By);
          } else {                          // FP32: from the leg components
            const T B2 = By * kc.isy, rB = rsqrtf(B2);
            a_b = (fmaf(hs, cw.x, hc) - q) * rB;                     // cos(q, -(q - p2))
            const T y1 = qs1 * cw.x, y2 = y1 - psp, z2 = qs1 * qs1 * fmaf(-cw.x, cw.x, (T)1);
            a_c = -fmaf(x1, x2, fmaf(y1, y2, z2)) * rsqrtf(A2) * rB;  // cos(q + p1, -(q - p2))
            // both b = (s1 - s2)/(s1 + s2) from one reciprocal of the product of the denominators
            const T qy = q2 * sy, db = qy + By, dc = Ay + By, rbc = hw_rcp(db * dc);
            b_b = (qy - By) * dc * rbc;
            b_c = (Ay - By) * db * rbc;
          }
          lb = lam3_full(a, L3, by + By, us, uy3, a_b, b_b);   // legs q, -(q-p2), p2
          lc = lam3_full(a, L3, sy_ab + By, us, uy3, a_c, b_c);     // legs q+p1, -(q-p2), -(p1+p2)
        } else {
          lb = look(L3, by + By, us, uy3, np);
          lc = look(L3, sy_ab + By, us, uy3, np);
        }
        rs += cw.y * GB * lb * lc;
      }
      v = GA * la * rs;
    }
    acc.add(radial_F<T>(a, r), S.w1[ia] * v);
    r += dr;
    ia += dia;
    if (ia >= na1) {
      ia -= na1;
      ++r;
    }
  }
  return acc;
}

template <int MODEL, typename T, bool POLE>
__device__ __forceinline__ RowAcc<T> witem(const RhsArgs &a, const RhsArgs *sa, const SmemLayout<T> &S,
                                        const KConst<T> &kc, int e, int c, int lane) {
  if constexpr (MODEL == FFRG_MODEL_D3) return d3_witem<T, POLE>(a, sa, S, kc, e, c, lane);
  else if constexpr (MODEL == FFRG_MODEL_D4_VERTEX) return d4_witem<T, POLE>(a, sa, S, kc, e, c, lane);
  else if constexpr (MODEL == FFRG_MODEL_D4_FULL) return d4_witem<T, POLE, true>(a, sa, S, kc, e, c, lane);
  else if constexpr (MODEL == kModelD4FullCell) return d4_witem<float, POLE, true, true>(a, sa, S, kc, e, c, lane);
  else static_assert(MODEL != FFRG_MODEL_FINITE_T, "finite T runs through ftk_rows");
}

// warp sum in a fixed order (valid in lane 0)
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// The near-pole test can only fire with m^2 < 0 or a negative Z node (table
// 0, every stack row).  Block-wide: every thread of the CTA must call it.
// FP32 line rows do not hold node values, so the FP32 d=3 / d=4 kernels take
// the signs from the FP64 tables, where the Z rows come first (the FP32 value
// is the FP64 one times k^2 ln 2 > 0, rounded: the same sign).
template <typename T>
__device__ __forceinline__ bool pole_possible(const RhsArgs &a, const SmemLayout<T> &S, const KConst<T> &kc) {
  int neg = 0;
  const int nz = (a.model == FFRG_MODEL_D4_FULL ? 1 : a.n_stack) * a.n_pts;
  if (sizeof(T) == 4 && a.model != FFRG_MODEL_FINITE_T)
    for (int i = threadIdx.x; i < nz; i += blockDim.x) neg |= a.tab[i] < 0.0;
  else
    for (int i = threadIdx.x; i < nz; i += blockDim.x) neg |= table_value(S.tab[i]) < (T)0;
  return __syncthreads_or(neg) || kc.m2 < (T)0;
}

// Output of external point e from the sum s of its partials: diagram
// coefficient (d=4: 1, 3, 3/2 for the Z, lambda3, lambda4 blocks), overall
// normalisation, and the non-finite check into the status word.
__device__ __forceinline__ void write_output(const RhsArgs &a, int e, double s) {
  double coef = 1.0;
  if (is_d4(a.model)) {
    const int np_ = a.n_ext_p;
    if (e > np_ && e < np_ + 1 + np_ * a.n_ext_ang) coef = 3.0;
    else if (e >= np_ + 1 + np_ * a.n_ext_ang) coef = 1.5;
  }
  const double v = a.norm * coef * s;
  a.out[e] = v;
  if (!isfinite(v)) raise_status(a.status, kStatusNonFinite);
}

// Sum of the partials of one external point in a fixed order: lane l adds
// chunks l, l+32, ..., then the warp tree (valid in lane 0).  The single-flow
// and serving kernels share it, so both give bitwise the same outputs.
__device__ __forceinline__ double sum_partials(const RhsArgs &a, int e, int lane) {
  const double *pp = a.partial + (size_t)e * a.n_chunks;
  double t = 0.0;
  for (int j = lane; j < a.n_chunks; j += 32) t += __ldcg(pp + j);
  return warp_sum(t);
}

// Single-flow work loop: items from the device counter (d=4: the three-point
// block, 16x more work per item, first), outputs by the warp that completes
// an external point (fixed-order sum of its partials).
template <int MODEL, typename T, bool POLE>
__device__ __forceinline__ void item_loop(const RhsArgs &a, const RhsArgs *sa, const SmemLayout<T> &S,
                                          const KConst<T> &kc) {
  const int lane = threadIdx.x & 31;
  const int rot = is_d4(MODEL) || MODEL == kModelD4FullCell ? a.n_ext_p + 1 : 0;
  for (;;) {
    int d = 0;
    if (lane == 0) d = (int)atomicAdd(a.work_ctr, 1u);
    d = __shfl_sync(0xffffffffu, d, 0);
    if (d >= a.n_items) break;
    const int c = d % a.n_chunks, e = (d / a.n_chunks + rot) % a.n_ext;
    const double acc = witem<MODEL, T, POLE>(a, sa, S, kc, e, c, lane).item_sum();
    unsigned done = 0;
    if (lane == 0) {
      a.partial[(size_t)e * a.n_chunks + c] = acc;
      __threadfence();
      done = atomicAdd(a.ext_done + e, 1u);
    }
    done = __shfl_sync(0xffffffffu, done, 0);
    if (done == (unsigned)a.n_chunks - 1u) {
      __threadfence();
      const double t = sum_partials(a, e, lane);
      if (lane == 0) write_output(a, e, t);
    }
  }
}

template <int MODEL, typename T>
__global__ void __launch_bounds__(kThreads, MinBlocks<T>::value) rhs_main(RhsArgs a) {
  if (skipped(a)) {   // wait all the same: this kernel completes after its precompute
    pdl_wait();
    return;
  }
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t bar;
  __shared__ RhsArgs sa;  // for the out-of-line near-pole path
  if (threadIdx.x == 0) sa = a;
  SmemLayout<T> S(smem, a);
  if (!main_prologue<T>(a, S, &bar)) return;
  const KConst<T> kc = load_kconst<T>(a);
  const bool pole = pole_possible<T>(a, S, kc);
  if constexpr (MODEL == FFRG_MODEL_FINITE_T) {
    // K rows: items (stack row, |p|) x chunk of radial nodes from the counter
    const int lane = threadIdx.x & 31;
    for (;;) {
      int d = 0;
      if (lane == 0) d = (int)atomicAdd(a.work_ctr, 1u);
      d = __shfl_sync(0xffffffffu, d, 0);
      if (d >= a.n_items) break;
      const int outer = d / a.n_chunks, c = d - outer * a.n_chunks;
      if (pole) ftk_rows<T, true>(a, &sa, S, kc, outer, c, lane);
      else ftk_rows<T, false>(a, &sa, S, kc, outer, c, lane);
    }
  } else {
    if (pole) item_loop<MODEL, T, true>(a, &sa, S, kc);
    else item_loop<MODEL, T, false>(a, &sa, S, kc);
  }
}

// D4_FULL, mixed, lambda3 as cell polynomials: the cells take most of shared
// memory, so one CTA of 1024 threads per SM (the warps of four 256-thread CTAs)
__global__ void __launch_bounds__(kThreadsWide, 1) rhs_main_cell(RhsArgs a) {
  if (skipped(a)) {   // wait all the same: this kernel completes after its precompute
    pdl_wait();
    return;
  }
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t bar;
  __shared__ RhsArgs sa;  // for the out-of-line near-pole path
  if (threadIdx.x == 0) sa = a;
  SmemLayout<float> S(smem, a);
  if (!main_prologue<float>(a, S, &bar)) return;
  const KConst<float> kc = load_kconst<float>(a);
  const bool pole = pole_possible<float>(a, S, kc);
  if (pole) item_loop<kModelD4FullCell, float, true>(a, &sa, S, kc);
  else item_loop<kModelD4FullCell, float, false>(a, &sa, S, kc);
}

// finite T: outputs from K and the radial factors, one block per external point
template <typename T>
__global__ void __launch_bounds__(kThreads) ft_contract_kernel(RhsArgs a) {
  __shared__ double red[kThreads / 32];
  if (skipped(a)) return;
  const double t = ft_contract<T>(a, blockIdx.x, red, threadIdx.x, blockDim.x, 0);
  if (threadIdx.x == 0) write_output(a, blockIdx.x, t);
}

// Finite T, mixed, one flow: precompute, K rows and contraction in one
// cooperative launch (every CTA resident), so that the RHS pays one launch
// and one grid barrier instead of three kernels and two kernel boundaries.
// One 1024-thread CTA per SM: the same warps as four 256-thread CTAs, a
// quarter of the barrier arrivals and of the table copies.
// Phase 1: each CTA builds its inputs itself from the FP64 tables and rules
// (the FP32 (Z k^2 ln 2, lambda) pairs, the angle rule, q_r and p_i in
// shared memory; the FP32 scale constants come from the host), which is
// FP64 work once per SM, and its warps take K rows, except warp 1 of the
// last CTAs, which computes the radial factors F(n, r) of the contraction in
// warp units.  Phase 2, after the barrier: the outputs by 256-thread groups.
// The values are those of the three-launch path, bit for bit.
// Grid counters c[0..3]: K-row items, barrier arrivals (monotonic), arrivals
// before this launch, finished CTAs.  The last CTA to finish resets c[0] and
// c[3] and records c[1] in c[2]; since every CTA finishes (each wait is
// bounded), a launch whose barrier timed out still leaves the next launch's
// counters consistent.
// Single-launch finite-T RHS: shared memory of the FP32 layout (tables and
// angle rules), then q_r and p_i in FP32 (16-byte aligned regions).
__host__ __device__ inline size_t single_extra_offset(const RhsArgs &a) {
  const size_t ang32 = (size_t)a.na1 * 3 + (size_t)a.na2 * 2 + (size_t)4 * ((a.na2 + 1) / 2);
  return (((size_t)a.tab32_count * 8 + 15) & ~(size_t)15) + ((ang32 * 4 + 15) & ~(size_t)15);
}
__host__ __device__ inline size_t single_smem(const RhsArgs &a) {
  return single_extra_offset(a) + (size_t)4 * (((a.nr + 3) & ~3) + ((a.n_ext_p + 3) & ~3));
}

// Grid barrier in two halves: every CTA arrives (thread 0, after the block's
// writes), and waits later; a CTA may work between the two.
__device__ __forceinline__ void grid_arrive(unsigned *arrive) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(arrive, 1u);
  }
}
__device__ __forceinline__ bool grid_wait(const unsigned *arrive, unsigned target, unsigned *status, int *s_ok) {
  if (threadIdx.x == 0) {
    int ok = 1;
    const long long t0 = clock64();
    while ((int)(*(volatile const unsigned *)arrive - target) < 0) {
      if (clock64() - t0 > kWaitCycles) {
        ok = 0;
        raise_status(status, kStatusTimeout);
        break;
      }
    }
    __threadfence();
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

__global__ void __launch_bounds__(kThreadsWide, 1) ft_single_kernel(RhsArgs a) {
  if (skipped(a)) return;  // uniform over the grid: no counter is touched
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ RhsArgs sa;  // for the out-of-line near-pole path
  __shared__ int s_ok;
  __shared__ double red[kThreadsWide / 32];
  unsigned *cnt = a.fused_ctr;
  // arrivals before this launch: thread 0 alone waits at the barriers, so the
  // value stays in its register and the load overlaps the prologue
  unsigned base = 0;
  if (threadIdx.x == 0) {
    base = *(volatile unsigned *)(cnt + 2);
    sa = a;
  }
  const int lane = threadIdx.x & 31;
  // The block's own inputs, the values the precompute would store, from the
  // FP64 tables and rules (one CTA per SM, so this FP64 work is per SM): the
  // FP32 (Z k^2 ln 2, lambda) pairs, the angle rule, q_r and p_i, and the
  // near-pole test on the Z entries as they pass
  SmemLayout<float> S(smem, a);
  float *q_loc = (float *)(smem + single_extra_offset(a));
  float *p_loc = q_loc + ((a.nr + 3) & ~3);
  const double k = scale_k(a), kh = k * k * 0.6931471805599453094, L = a.qmax_over_k * k;
  const int z_count = a.n_stack * a.n_pts;
  int neg = 0;
  for (int i = threadIdx.x; i <= z_count; i += blockDim.x) {
    const float2 v = i < z_count ? make_float2((float)(kh * a.tab[i]), (float)a.tab[z_count + i])
                                 : make_float2(0.f, 0.f);
    S.tab[i] = v;
    neg |= v.x < 0.0f;
  }
  for (int r = threadIdx.x; r < a.nr; r += blockDim.x) q_loc[r] = (float)(L * a.rad_x[r]);
  for (int i = threadIdx.x; i < a.n_ext_p; i += blockDim.x) p_loc[i] = (float)ext_momentum(a, i);
  stage_angles<float, false>(a, S);   // finite T: no sqrt(1 - c^2)
  const KConst<float> kc = make_kconst<float>(a);   // the host's copy (plain calls only)
  const bool pole = __syncthreads_or(neg) || kc.m2 < 0.0f;
  bool ok = true;
  // The radial factors of the contraction: warp 1 of the last CTAs, one warp
  // unit each (FP64 work spread over SMs) instead of K rows, hidden behind
  // the K rows of the other warps; the grid has one warp more per unit.
  const bool radial_warp = (threadIdx.x >> 5) == 1 && gridDim.x - 1 - blockIdx.x < (unsigned)radial_units(a);
  if (radial_warp)
    for (int u = gridDim.x - 1 - blockIdx.x; u < radial_units(a); u += gridDim.x) radial_unit(a, u, lane);
  else
    for (;;) {
      int d = 0;
      if (lane == 0) d = (int)atomicAdd(cnt, 1u);
      d = __shfl_sync(0xffffffffu, d, 0);
      if (d >= a.n_items) break;
      const int outer = d / a.n_chunks, c = d - outer * a.n_chunks;
      if (pole) ftk_rows<float, true>(a, &sa, S, kc, outer, c, lane, q_loc, p_loc);
      else ftk_rows<float, false>(a, &sa, S, kc, outer, c, lane, q_loc, p_loc);
    }
  grid_arrive(cnt + 1);
  ok = grid_wait(cnt + 1, base + gridDim.x, a.status, &s_ok) && ok;
  // the outputs by 256-thread groups, four per CTA at once (named barriers
  // 1..4): the arithmetic order of ft_contract_kernel's blocks
  if (ok) {
    const int g = threadIdx.x / kThreads, ng = blockDim.x / kThreads, gtid = threadIdx.x - g * kThreads;
    for (int e = blockIdx.x * ng + g; e < a.n_ext; e += gridDim.x * ng) {
      const double t = ft_contract<float>(a, e, red + g * (kThreads / 32), gtid, kThreads, 1 + g);
      if (gtid == 0) write_output(a, e, t);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(cnt + 3, 1u) == gridDim.x - 1) {
      cnt[0] = 0u;
      cnt[2] = *(volatile unsigned *)(cnt + 1);
      cnt[3] = 0u;
      __threadfence();
    }
  }
}

// ---------------------------------------------------------------------------
constexpr size_t kMaxDynSmem = kMaxDynSmemBytes;

template <typename K>
static int persistent_grid(ffrg_ctx *ctx, K kernel, size_t smem, int items, int *grid, int threads = kThreads) {
  if (smem > kMaxDynSmem) {
    ctx->last_error = "dressing tables do not fit in shared memory";
    return FFRG_EINVAL;
  }
  int st = ensure_smem_limit(ctx, (const void *)kernel, smem);
  if (st) return st;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
  if (e != cudaSuccess) return set_cuda_error(ctx, e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
  if (per_sm < 1) {
    ctx->last_error = "RHS kernel cannot be resident";
    return FFRG_EINVAL;
  }
  // one warp-sized item per warp is the most a CTA can start with
  const int ctas = (items + threads / 32 - 1) / (threads / 32);
  *grid = std::max(1, std::min(ctas, per_sm * ctx->num_sms));
  return FFRG_OK;
}

// The single-launch finite-T RHS: every CTA of a cooperative launch is
// resident, so its grid barrier completes.  kNoSingleLaunch when the device
// cannot launch cooperatively (the caller then takes the three launches).
constexpr int kNoSingleLaunch = -100;
static int launch_ft_single(ffrg_ctx *ctx, Plan *pl, const RhsArgs &a, cudaStream_t s) {
  const size_t smem = single_smem(a);   // tables, rules, q_r and p_i of the block
  if (smem > kMaxDynSmem) return kNoSingleLaunch;
  if (pl->grid_single == 0) {
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, ctx->device);
    if (!coop) {
      pl->grid_single = -1;
    } else {
      // one warp per K-row item and one per radial unit (32 nodes x kRadN rows)
      const int units = ((a.nr + 31) / 32) * ((a.N + 1 + kRadN - 1) / kRadN);
      int st = persistent_grid(ctx, ft_single_kernel, smem, a.n_items + units, &pl->grid_single, kThreadsWide);
      if (st) return st;
    }
  }
  if (pl->grid_single < 0) return kNoSingleLaunch;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(pl->grid_single);
  cfg.blockDim = dim3(kThreadsWide);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cap);
  const bool prof = ctx->profiling && cap == cudaStreamCaptureStatusNone &&
                    ctx->prof_used * 2 + 1 < (int)ctx->prof_events.size();
  if (prof) cudaEventRecord(ctx->prof_events[2 * ctx->prof_used], s);
  cudaError_t e = cudaLaunchKernelEx(&cfg, ft_single_kernel, a);
  if (e == cudaErrorCooperativeLaunchTooLarge) {   // fewer SMs than the device reports (e.g. an MPS limit)
    (void)cudaGetLastError();
    pl->grid_single = -1;
    return kNoSingleLaunch;
  }
  if (prof) {
    cudaEventRecord(ctx->prof_events[2 * ctx->prof_used + 1], s);
    ctx->prof_used++;
  }
  return set_cuda_error(ctx, e, "single-launch finite-T RHS");
}

int precompute_blocks(const RhsArgs &a, int cap) {
  const int n_rt = (a.nr + kPreR - 1) / kPreR, n_nb = a.N / kPreN + 1;
  const int flat = std::max(std::max(a.tab_count, a.n_ext), a.n_ext_p);
  // blocks with per-radial work, then blocks for the scalar and flat work
  return std::max(1, std::min(n_rt * n_nb + (flat + kThreads - 1) / kThreads, cap));
}

int launch_precompute(ffrg_ctx *ctx, const RhsArgs &a, cudaStream_t s) {
  precompute_kernel<<<precompute_blocks(a, 4 * ctx->num_sms), kThreads, 0, s>>>(a);
  return set_cuda_error(ctx, cudaGetLastError(), "precompute launch");
}

int launch_rhs(ffrg_ctx *ctx, const Plan *pl_c, const RhsArgs &a_in, int precision, cudaStream_t s) {
  return launch_rhs_stages(ctx, pl_c, a_in, precision, s, true);
}

int launch_rhs_stages(ffrg_ctx *ctx, const Plan *pl_c, const RhsArgs &a_in, int precision, cudaStream_t s,
                      bool contract) {
  if (a_in.model == FFRG_MODEL_FINITE_T_4D) return launch_ft4(ctx, pl_c, a_in, precision, s);
  Plan *pl = const_cast<Plan *>(pl_c);
  const bool mixed = precision == FFRG_MIXED;
  RhsArgs a = a_in;  // forward geometry of this precision
  if (!mixed) {
    a.cr = pl->fcr64;
    a.n_chunks = pl->fn_chunks64;
    a.n_items = pl->fn_items64;
    a.jb = pl->fjb64;
  }
  int st;
  int &grid = mixed ? pl->grid32 : pl->grid64;
  size_t smem = mixed ? pl->smem32 : pl->smem64;
  a.tab_global = 0;
  if (!mixed && smem > kMaxDynSmem) {   // FP64 tables beyond shared memory: read from L2
    a.tab_global = 1;
    smem = pl->smem64g;
  }
  void (*kern)(RhsArgs) = nullptr;
  switch (a.model) {
  case FFRG_MODEL_D3: kern = mixed ? rhs_main<FFRG_MODEL_D3, float> : rhs_main<FFRG_MODEL_D3, double>; break;
  case FFRG_MODEL_D4_VERTEX:
    kern = mixed ? rhs_main<FFRG_MODEL_D4_VERTEX, float> : rhs_main<FFRG_MODEL_D4_VERTEX, double>;
    break;
  case FFRG_MODEL_D4_FULL:
    kern = mixed ? rhs_main<FFRG_MODEL_D4_FULL, float> : rhs_main<FFRG_MODEL_D4_FULL, double>;
    break;
  default: kern = mixed ? rhs_main<FFRG_MODEL_FINITE_T, float> : rhs_main<FFRG_MODEL_FINITE_T, double>; break;
  }
  int threads = kThreads;
  if (mixed && a.model == FFRG_MODEL_D4_FULL && a.l3cell) {
    kern = rhs_main_cell;
    threads = kThreadsWide;
  }
  if (!a.work_ctr || !a.radq32 || !a.ext_done || !a.kconst || (a.model == FFRG_MODEL_FINITE_T && !a.kbuf)) {
    ctx->last_error = "plan without work counters, FP32 radial nodes or constant block";
    return FFRG_EINVAL;
  }
  // the single launch pays where the K rows fill the GPU and the scale is a
  // host value: measured 45 -> 29 us for 4800 K-row items (N = 16, 576 ext),
  // but 3-4 us slower for the serving mix's few hundred items, and in flows
  // (k on the device: the FP32 constants would cost an FP64 chain per CTA)
  constexpr int kSingleLaunchItems = 152 * (kThreads / 32);
  if (mixed && a.model == FFRG_MODEL_FINITE_T && contract && a.fused_ctr && !a.k_dev && !a.m2_dev &&
      a.n_items >= kSingleLaunchItems) {
    st = launch_ft_single(ctx, pl, a, s);
    if (st != kNoSingleLaunch) return st;   // else the three launches below
  }
  if (grid == 0) {
    st = persistent_grid(ctx, kern, smem, a.n_items, &grid, threads);
    if (st) return st;
  }
  precompute_kernel<<<precompute_blocks(a, 4 * ctx->num_sms), kThreads, 0, s>>>(a);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cap);
  const bool prof = ctx->profiling && cap == cudaStreamCaptureStatusNone &&
                    ctx->prof_used * 2 + 1 < (int)ctx->prof_events.size();
  if (prof) cudaEventRecord(ctx->prof_events[2 * ctx->prof_used], s);
  // a programmatic dependent of the precompute kernel: its CTAs start while
  // the precompute runs (a profiling event in between makes it wait)
  cudaError_t le = launch_dependent(kern, dim3(grid), dim3(threads), smem, s, true, a);
  if (le != cudaSuccess) return set_cuda_error(ctx, le, "rhs launch");
  if (prof) {
    cudaEventRecord(ctx->prof_events[2 * ctx->prof_used + 1], s);
    ctx->prof_used++;
  }
  // d=3, d=4: the main kernel writes the outputs (last warp per external
  // point); finite T: the contraction of K with the radial factors
  if (a.model == FFRG_MODEL_FINITE_T && contract) {
    if (mixed) ft_contract_kernel<float><<<a.n_ext, kThreads, 0, s>>>(a);
    else ft_contract_kernel<double><<<a.n_ext, kThreads, 0, s>>>(a);
  }
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
  precompute_body(a);
}

// one block per external point blockIdx.x of flow blockIdx.y: finite T
// contracts K (the same function as the single-flow kernel), d=3 sums the
// item partials in warp 0
__global__ void __launch_bounds__(kThreads) batched_finalize_kernel(const RhsArgs *descs) {
  __shared__ double red[kThreads / 32];
  const RhsArgs &a = descs[blockIdx.y];
  const int e = blockIdx.x;
  if (skipped(a) || e >= a.n_ext) return;   // uniform over the block
  if (a.model == FFRG_MODEL_FINITE_T) {
    const double t = ft_contract<float>(a, e, red, threadIdx.x, blockDim.x, 0);
    if (threadIdx.x == 0) write_output(a, e, t);
  } else if (threadIdx.x < 32) {
    const double t = sum_partials(a, e, threadIdx.x);
    if (threadIdx.x == 0) write_output(a, e, t);
  }
}

// Each CTA takes a contiguous range of the combined item list holding an
// equal share of the estimated cost (cost[f] is cumulative at the flow
// boundaries, uniform per item within a flow), so that flows with longer
// rows do not leave other CTAs idle.  For each flow segment of its range the
// CTA copies the flow's descriptor and angle rules into shared memory (plain
// loads) and its FP32 tables (one bulk copy, mbarrier phase per segment); its
// warps then take the segment's warp-sized items.
__device__ __forceinline__ int item_at_cost(const int *start, const long long *cost, int n_fl, long long x) {
  int f = 0;
  while (f + 1 < n_fl && cost[f + 1] <= x) ++f;
  const int items = start[f + 1] - start[f];
  const long long w = cost[f + 1] - cost[f];
  if (w <= 0) return start[f];
  return start[f] + (int)min((long long)items, (x - cost[f]) * items / w);
}

template <int MODEL>
__global__ void __launch_bounds__(kThreads, 4)
    batched_main_kernel(const RhsArgs *descs, const int *flows, const int *start, const long long *cost, int n_fl) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ RhsArgs sa;
  __shared__ int skip;
  __shared__ uint64_t bar;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  mbar_init_once(&bar);
  unsigned parity = 0;
  const long long W = cost[n_fl];
  const int g0 = blockIdx.x == 0 ? 0 : item_at_cost(start, cost, n_fl, W * blockIdx.x / gridDim.x);
  const int g1 = blockIdx.x + 1 == gridDim.x ? start[n_fl]
                                             : item_at_cost(start, cost, n_fl, W * (blockIdx.x + 1) / gridDim.x);
  int f = 0;
  while (f < n_fl && start[f + 1] <= g0) ++f;
  for (; f < n_fl && start[f] < g1; ++f) {
    const int lo = max(g0, start[f]), hi = min(g1, start[f + 1]);
    if (lo >= hi) continue;
    __syncthreads();  // the previous segment's tables are no longer read
    if (threadIdx.x == 0) {
      sa = descs[flows[f]];
      skip = skipped(sa);
    }
    __syncthreads();
    if (skip) continue;
    SmemLayout<float> S(smem, sa);
    // the flow's FP32 tables by one bulk copy (up to ~150 KB for finite T)
    if (!stage_to_smem_phase<float2>(S.tab, sa.tab32, sa.tab32_count, &bar, parity, sa.status)) return;
    parity ^= 1u;
    stage_angles<float>(sa, S);
    __syncthreads();
    const KConst<float> kc = load_kconst<float>(sa);
    const bool pole = pole_possible<float>(sa, S, kc);
    for (int g = lo + warp; g < hi; g += nw) {
      const int item = g - start[f];
      const int e = item / sa.n_chunks, c = item - e * sa.n_chunks;
      if constexpr (MODEL == FFRG_MODEL_FINITE_T) {   // K rows (e: stack row x |p|)
        if (pole) ftk_rows<float, true>(sa, &sa, S, kc, e, c, lane);
        else ftk_rows<float, false>(sa, &sa, S, kc, e, c, lane);
      } else {
        const double acc = pole ? witem<MODEL, float, true>(sa, &sa, S, kc, e, c, lane).item_sum()
                                : witem<MODEL, float, false>(sa, &sa, S, kc, e, c, lane).item_sum();
        if (lane == 0) sa.partial[item] = acc;
      }
    }
  }
}

// resident CTAs per SM of the batched main kernel for a shared-memory size,
// memoised per (model, bytes, device): the serving scheduler asks for every
// flow of every launch set and every launch
template <int MODEL>
static int batched_occupancy(ffrg_ctx *ctx, size_t smem, int *per_sm) {
  static std::mutex mu;
  static std::map<std::tuple<int, size_t, int>, int> memo;
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = memo.find({MODEL, smem, ctx->device});
    if (it != memo.end()) {
      *per_sm = it->second;
      return FFRG_OK;
    }
  }
  void (*kern)(const RhsArgs *, const int *, const int *, const long long *, int) = batched_main_kernel<MODEL>;
  int st = ensure_smem_limit(ctx, (const void *)kern, smem);
  if (st) return st;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, kern, kThreads, smem);
  if (e != cudaSuccess || *per_sm < 1) return set_cuda_error(ctx, e ? e : cudaErrorInvalidConfiguration, "occupancy");
  std::lock_guard<std::mutex> lock(mu);
  memo[{MODEL, smem, ctx->device}] = *per_sm;
  return FFRG_OK;
}

int batched_ctas_per_sm(ffrg_ctx *ctx, int model, size_t smem) {
  int per_sm = 1;
  const int st = model == FFRG_MODEL_D3 ? batched_occupancy<FFRG_MODEL_D3>(ctx, smem, &per_sm)
                                        : batched_occupancy<FFRG_MODEL_FINITE_T>(ctx, smem, &per_sm);
  return st ? 1 : per_sm;
}

template <int MODEL>
static int launch_batched_main(ffrg_ctx *ctx, const RhsArgs *descs, const BatchGroup &G, cudaStream_t s) {
  if (G.n == 0 || G.items == 0) return FFRG_OK;
  int per_sm = 0;
  int st = batched_occupancy<MODEL>(ctx, G.smem, &per_sm);
  if (st) return st;
  const int ctas = (G.items + kThreads / 32 - 1) / (kThreads / 32);
  const int grid = std::max(1, std::min(ctas, per_sm * ctx->num_sms));
  batched_main_kernel<MODEL><<<grid, kThreads, G.smem, s>>>(descs, G.flows, G.start, G.cost, G.n);
  return FFRG_OK;
}

int launch_rhs_batched(ffrg_ctx *ctx, const BatchList &bl, cudaStream_t s) {
  if (bl.n_flows == 0) return FFRG_OK;
  batched_precompute_kernel<<<dim3(std::max(1, bl.max_pre), bl.n_flows), kThreads, 0, s>>>(bl.descs);
  int st = FFRG_OK;
  for (int g = 0; g < bl.n_groups && !st; ++g) {
    const BatchGroup &G = bl.groups[g];
    st = G.model == FFRG_MODEL_D3 ? launch_batched_main<FFRG_MODEL_D3>(ctx, bl.descs, G, s)
                                  : launch_batched_main<FFRG_MODEL_FINITE_T>(ctx, bl.descs, G, s);
  }
  if (st) return st;
  batched_finalize_kernel<<<dim3(std::max(1, bl.max_ext), bl.n_flows), kThreads, 0, s>>>(bl.descs);
  return set_cuda_error(ctx, cudaGetLastError(), "batched rhs launch");
}

}  // namespace ffrg
