// Finite T with a 4-dimensional regulator on a frequency domain that scales
// with k (Sec. 5.3.2 "Quadraturex0" integrators, efficient with 4D
// regulators; App. G external fermion legs at p0f = pi T exp(-k/(pi T))):
//
//   I(m, p) = pref lam^2 [T sum_n | int dq0/(2 pi)] int d^3q/(2 pi)^3
//             dR(Q) G(Q)^2 L(|Q|) L(|Q+P|) G(Q+P),   Q = (q0, q), P = (p0, p),
//
// R(Q) = Z(|Q|) k^2 r(|Q|^2/k^2), G(Q) = 1/(Z(|Q|)(|Q|^2 + k^2 r) + m^2),
// Z and L on one log grid in |Q|.  The frequency set depends on k: the loop
// Matsubara frequencies with |q0| <= qmax_over_k k while there are at most
// 2N+1 (+1 fermionic) of them, Gauss-Legendre nodes of the domain beyond.
// Three launches per RHS: the frequency set and radial nodes (one block), the
// loop factors F(f, r) = w_f w_r q_r^2 dR G^2 L at (q0_f, q_r) in FP64, and one
// block per external point summing F(f, r) times the angular sum of the
// shifted line over (f, r) in a fixed order.  The scale k is read on the
// device (a flow's stage scale), so every step of a flow sees its own
// frequency set.
#include <math.h>

#include "ffrg_internal.cuh"

namespace ffrg {

// kbuf layout of this model: [0, nfreq) frequencies, [nfreq, 2 nfreq) weights,
// [2 nfreq] the number of frequencies in use
__global__ void ft4_freq_kernel(RhsArgs a, int nfreq_max) {
  pdl_trigger();   // the factor kernel may start (it waits for these writes)
  double *kb = (double *)a.kbuf, *fq = kb, *fw = kb + nfreq_max;
  const double k = scale_k(a), L0 = a.qmax_over_k * k, T = a.T;
  const int cap = 2 * a.N + 1 + (a.stat ? 1 : 0);
  int count, Nk;
  if (a.stat) {
    const double x = L0 / (kPi * T);
    Nk = x < 1.0 ? -1 : (int)floor((x - 1.0) / 2.0);
    count = 2 * Nk + 2;
  } else {
    Nk = (int)floor(L0 / (2.0 * kPi * T));
    count = 2 * Nk + 1;
  }
  const bool sum = count <= cap;
  const int nf = sum ? count : a.na2;
  for (int f = threadIdx.x; f < nf; f += blockDim.x) {
    if (sum) {
      const int n = a.stat ? f - Nk - 1 : f - Nk;
      fq[f] = a.stat ? (2.0 * n + 1.0) * kPi * T : 2.0 * kPi * T * n;
      fw[f] = T;
    } else {
      fq[f] = L0 * a.a2_x[f];
      fw[f] = L0 * a.a2_w[f] / (2.0 * kPi);
    }
  }
  const double qs = a.qmax_over_k * k;
  for (int r = threadIdx.x; r < a.nr; r += blockDim.x) a.radq[r] = qs * a.rad_x[r];
  if (threadIdx.x == 0) kb[2 * nfreq_max] = (double)nf;
}

// F(f, r) = w_f w_r q^2 dR(Q) G(Q)^2 L(|Q|), |Q|^2 = q0_f^2 + q_r^2 (FP64; FP32 copy)
__global__ void ft4_factor_kernel(RhsArgs a, int nfreq_max) {
  pdl_trigger();   // the main kernel may start staging its tables
  pdl_wait();      // frequencies, weights and q_r of the frequency kernel
  const double *kb = (const double *)a.kbuf;
  const int nf = (int)kb[2 * nfreq_max];
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nf * a.nr) return;
  const int f = idx / a.nr, r = idx - f * a.nr;
  const double k = scale_k(a), k2 = k * k, inv_k2 = 1.0 / k2, m2 = mass2(a, k);
  const double q = a.radq[r], q0 = kb[f], Q2 = q0 * q0 + q * q;
  const double *Zt = a.tab, *Lt = a.tab + a.n_pts;
  const double Z = look(Zt, Q2, a.u_scale, a.u_off, a.n_pts);
  const double L = look(Lt, Q2, a.u_scale, a.u_off, a.n_pts);
  const double G = 1.0 / prop_den(a.reg, Z, 0.0, Q2, m2, k2, inv_k2);
  const double wr = a.qmax_over_k * k * a.rad_w[r];
  const double F = kb[nfreq_max + f] * wr * q * q * Z * k2 * reg_rdot(a.reg, Q2 * inv_k2) * G * G * L;
  a.radF[idx] = F;
  a.radF32[idx] = (float)F;
}

// angular sum of the shifted line at (q0 + p0, q, p): sum_c v_c L(|Q+P|) G(Q+P)
__device__ __forceinline__ double ft4_row(const RhsArgs &a, double sh2, double q, double p, double k2, double inv_k2,
                                          double m2) {
  const double *Zt = a.tab, *Lt = a.tab + a.n_pts;
  double rs = 0.0;
  for (int c = 0; c < a.na1; ++c) {
    const double QP2 = fmax(0.0, sh2 + fma(2.0 * q * p, a.a1_x[c], q * q + p * p));
    const double Z = look(Zt, QP2, a.u_scale, a.u_off, a.n_pts);
    const double L = look(Lt, QP2, a.u_scale, a.u_off, a.n_pts);
    rs = fma(a.a1_w[c] * L, 1.0 / prop_den(a.reg, Z, 0.0, QP2, m2, k2, inv_k2), rs);
  }
  return rs;
}

// FP32 angular sum (the mixed path) from shared memory: zl[i] = (Z_i, Z_{i+1}
// - Z_i, L_i, L_{i+1} - L_i) per node (the last node's differences 0), cw[c] =
// (c_c, v_c).  Propagator denominator Z k^2 h(x) + m^2 with h(x) = x + r(x) =
// x/(1 - e^-x) (exponential regulator; its Taylor series for x < 1/2, where
// 1 - e^-x cancels) or max(x, 1) (flat), hardware lg2/ex2/rcp.  A denominator that
// cancels more than half of its kinetic part (m^2 < 0 near the pole) is
// recomputed in FP64 from the FP64 tables.
__device__ __forceinline__ float ft4_row32(const RhsArgs &a, const float4 *zl, const float2 *cw, float sh2, float q,
                                           float p, float k2, float inv_k2, float m2, float us, float uo) {
  const int n = a.n_pts, na1 = a.na1;
  const float nm1 = (float)(n - 1);
  const float base = fmaf(q, q, fmaf(p, p, sh2)), tqp = 2.0f * q * p;
  float rs = 0.0f;
  for (int c = 0; c < na1; ++c) {
    const float2 cv = cw[c];
    const float QP2 = fmaxf(0.0f, fmaf(tqp, cv.x, base));
    float u = fminf(fmaxf(fmaf(us, hw_lg2(QP2), uo), 0.0f), nm1);   // NaN (QP2 = 0 -> -inf) saturates to 0
    const int i = min((int)u, n - 2);
    const float w = u - (float)i;
    const float4 t = zl[i];
    const float Z = fmaf(w, t.y, t.x), L = fmaf(w, t.w, t.z);
    const float x = QP2 * inv_k2;
    // G = 1/(kin + m^2), kin = Z k^2 h(x); for x >= 1/2 as d/(Z k^2 x + m^2 d),
    // d = 1 - e^-x >= 0.39 (the ex2 error, 2^-22.5, grows by at most 2.6x):
    // one reciprocal for regulator and propagator
    float num = 1.0f, kin, den;
    if (a.reg == FFRG_REG_LITIM) {
      kin = Z * k2 * fmaxf(x, 1.0f);
      den = kin + m2;
    } else if (x < 0.5f) {   // x/(1 - e^-x) = 1 + x/2 + x^2/12 - x^4/720 + x^6/30240 - ..., remainder < 4e-9
      const float x2 = x * x;
      kin = Z * k2 * fmaf(x2, fmaf(x2, fmaf(x2, 1.0f / 30240.0f, -1.0f / 720.0f), 1.0f / 12.0f), fmaf(x, 0.5f, 1.0f));
      den = kin + m2;
    } else {
      num = 1.0f - hw_ex2(-1.4426950408889634f * x);
      kin = Z * k2 * x;          // = the kinetic part times d
      den = fmaf(m2, num, kin);  // = d (kinetic part + m^2)
    }
    float g;
    if (m2 < 0.0f && den < 0.5f * kin) {
      const double QPd = (double)QP2;
      const double Zd = look(a.tab, QPd, a.u_scale, a.u_off, n);
      g = (float)(1.0 / prop_den(a.reg, Zd, 0.0, QPd, (double)m2, (double)k2, 1.0 / (double)k2));
    } else {
      g = num * hw_rcp(den);
    }
    rs = fmaf(cv.y * L, g, rs);
  }
  return rs;
}

// one block per external point e = (p, m): threads over the (f, r) terms,
// f major, in a fixed order; FP64 accumulation.  The FP32 kernel stages both
// tables and the angle rule in shared memory first.
template <typename T>
__global__ void __launch_bounds__(kThreads) ft4_main_kernel(RhsArgs a, int nfreq_max) {
  __shared__ double red[kThreads / 32];
  extern __shared__ __align__(16) unsigned char ft4_smem[];
  const int e = blockIdx.x, nm = a.n_ext_ang, ip = e / nm, m = e - ip * nm;
  const double *kb = (const double *)a.kbuf;
  const double k = scale_k(a), k2 = k * k, m2 = mass2(a, k);
  const double p = ext_momentum(a, ip);
  const double p0 = a.stat ? kPi * a.T * exp(-k / (kPi * a.T)) : 2.0 * kPi * a.T * m;
  float4 *zl = reinterpret_cast<float4 *>(ft4_smem);
  float2 *cw = reinterpret_cast<float2 *>(zl + a.n_pts);
  if (sizeof(T) == 4) {
    const double *Zt = a.tab, *Lt = a.tab + a.n_pts;
    for (int i = threadIdx.x; i < a.n_pts; i += blockDim.x) {
      const bool last = i + 1 >= a.n_pts;
      const double z0 = Zt[i], l0 = Lt[i];
      zl[i] = make_float4((float)z0, last ? 0.0f : (float)(Zt[i + 1] - z0), (float)l0,
                          last ? 0.0f : (float)(Lt[i + 1] - l0));
    }
    for (int c = threadIdx.x; c < a.na1; c += blockDim.x) cw[c] = make_float2((float)a.a1_x[c], (float)a.a1_w[c]);
    __syncthreads();
  }
  pdl_wait();   // the factor kernel's F(f, r) (and through it the frequency set)
  const int nf = (int)kb[2 * nfreq_max];
  const float us = (float)(a.u_scale * 0.69314718055994530942), uo = (float)a.u_off;
  double acc = 0.0;
  for (int i = threadIdx.x; i < nf * a.nr; i += blockDim.x) {
    const int f = i / a.nr, r = i - f * a.nr;
    const double sh = kb[f] + p0, q = a.radq[r];
    if (sizeof(T) == 8) {
      acc = fma(a.radF[i], ft4_row(a, sh * sh, q, p, k2, 1.0 / k2, m2), acc);
    } else {
      const float rs = ft4_row32(a, zl, cw, (float)(sh * sh), (float)q, (float)p, (float)k2, (float)(1.0 / k2),
                                 (float)m2, us, uo);
      acc = fma(a.radF[i], (double)rs, acc);
    }
  }
  const double t = block_sum(acc, red);
  if (threadIdx.x == 0) {
    const double v = a.norm * t;
    a.out[e] = v;
    if (!isfinite(v)) raise_status(a.status, kStatusNonFinite);
  }
}

int launch_ft4(ffrg_ctx *ctx, const Plan *pl, const RhsArgs &a, int precision, cudaStream_t s) {
  if (!a.kbuf || !a.radq || !a.radF || !a.radF32 || !a.a2_x) {
    ctx->last_error = "plan without the frequency buffer or radial factors";
    return FFRG_EINVAL;
  }
  const int nfreq = pl->nfreq;
  ft4_freq_kernel<<<1, kThreads, 0, s>>>(a, nfreq);
  const int terms = nfreq * pl->nr;
  cudaError_t e = launch_dependent(ft4_factor_kernel, dim3((terms + kThreads - 1) / kThreads), dim3(kThreads), 0, s,
                                   true, a, nfreq);
  if (e != cudaSuccess) return set_cuda_error(ctx, e, "finite-T 4D factor launch");
  const bool prof = ctx->profiling && ctx->prof_used * 2 + 1 < (int)ctx->prof_events.size();
  if (prof) cudaEventRecord(ctx->prof_events[2 * ctx->prof_used], s);
  if (precision == FFRG_MIXED) {
    const size_t smem = (size_t)pl->n_pts * sizeof(float4) + (size_t)pl->na1 * sizeof(float2);
    if (smem > 227 * 1024) {
      ctx->last_error = "tables and angle rule do not fit in shared memory";
      return FFRG_EINVAL;
    }
    int st = ensure_smem_limit(ctx, (const void *)ft4_main_kernel<float>, smem);
    if (st) return st;
    e = launch_dependent(ft4_main_kernel<float>, dim3(a.n_ext), dim3(kThreads), smem, s, true, a, nfreq);
  } else {
    e = launch_dependent(ft4_main_kernel<double>, dim3(a.n_ext), dim3(kThreads), 0, s, true, a, nfreq);
  }
  if (e != cudaSuccess) return set_cuda_error(ctx, e, "finite-T 4D launch");
  if (prof) {
    cudaEventRecord(ctx->prof_events[2 * ctx->prof_used + 1], s);
    ctx->prof_used++;
  }
  return set_cuda_error(ctx, cudaGetLastError(), "finite-T 4D launch");
}

}  // namespace ffrg
