// Internal declarations of the ffrg CUDA library (not part of the C ABI).
//
// Device-side pieces of the momentum-loop right-hand side (DiFfRG,
// arXiv:2412.13043): regulator shape and scale derivative (Sec. 5.3.1),
// log-grid table lookup (App. F interpolators), propagators with a
// Z-dressed regulator (App. G propagator form), and the argument block that
// every RHS kernel receives by value.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/ffrg.h"

namespace ffrg {

constexpr int kThreads = 256;          // threads per CTA of the RHS kernels
constexpr int kThreadsWide = 1024;     // the D4_FULL mixed kernel with lambda3 cells: one CTA per SM
constexpr size_t kMaxDynSmemBytes = 227 * 1024;   // dynamic shared memory of one block
constexpr unsigned kStatusNonFinite = 1u;
constexpr unsigned kStatusTimeout = 2u;
constexpr long long kWaitCycles = 4000000000LL;  // ~2 s at 2 GHz: bound of every device wait
constexpr double kPi = 3.141592653589793238462643383279502884;
constexpr int kMaxPts = 4096;
constexpr int kMaxNodes = 65536;

// ---------------------------------------------------------------------------
// Kernel argument block (passed by value).
// ---------------------------------------------------------------------------
// the two d=4 vertex-expansion models (1-D or 3-D three-point vertex)
__host__ __device__ inline bool is_d4(int model) {
  return model == FFRG_MODEL_D4_VERTEX || model == FFRG_MODEL_D4_FULL;
}

// bytes of the per-RHS constant block (FP32 and FP64 scale constants)
constexpr int kKConstBytes = 256;

// Scale-dependent constants of one RHS in a kernel precision (the FP32 and
// FP64 sets are described where the kernels use them).
template <typename T>
struct KConst {
  T k2, inv_k2, m2, us, uo, plim, sy, som;
  T uy1, uy2, uy3, uy4, twopiT, sw2;
  T isy;  // 1/sy
};

struct RhsArgs {
  int model, reg;
  int nr, na1, na2;
  int n_ext_p, n_ext_ang, N, include_p0, n_ext;
  int stat, nfreq;  // loop statistics (ffrg_statistics) and frequency rows: 2N+1 (bosonic), 2N+2 (fermionic)
  int n_tables, n_stack, n_pts, tab_count;
  int tab32_count; // float2 entries of the FP32 table layout
  int tabc_count;  // D4_FULL: doubles of the compact FP64 tables (0 otherwise)
  int n_va, n_vb;  // D4_FULL: vertex nodes in the shape variables a, b
  int l3cell;      // D4_FULL, mixed: lambda3 as FP32 cell polynomials (one 1024-thread CTA per SM)
  int cr;          // rows per work item (d=4: outer rows)
  int n_chunks;    // work items per external point
  int n_items;     // n_ext * n_chunks
  int jb;          // angle nodes per row (D3 / FINITE_T; rows = outer index x angle block)
  int tab_global;  // FP64 main kernels: tables read in place from global memory (L2), not staged,
                   // because they exceed shared memory; only the angle rules are staged
  double k, m2_over_k2, m2_shift, T;
  double p_min, p_ratio_step;  // p_i = p_min * exp(i * p_ratio_step)
  double qmax_over_k;
  double norm;                 // overall factor applied in finalize
  double u_scale, u_off;       // u = u_scale ln(s^2) + u_off
  double uoc[4];               // u_off - u_scale ln c, c = 1..4 (coordinate of S0^2 = sum of c squares / c)
  float us1f;                  // FP32 coordinate: u_scale ln 2 / (n_pts - 1) (multiplies log2)
  double uoc1[4];              // uoc[c-1] / (n_pts - 1)
  double us1;                  // u_scale / (n_pts - 1)
  double twopiT;               // 2 pi T
  double x_min2;               // x_min^2 (lookups below x_min return the first node)
  double sum_w2;               // sum of the second-angle weights (D4)
  KConst<float> kc_host;       // FP32 scale constants from the host (valid when kc_host_ok, k_dev and m2_dev null)
  int kc_host_ok;
  const double *tab;           // FP64 tables [n_tables][n_stack][n_pts]
  double *tabc;                // D4_FULL: compact FP64 tables [Z row | lambda4 row | lambda3 rows] (precompute)
  void *kbuf;                  // FINITE_T: K[j][ip][r], j < N + n_ext_ang, in the kernel precision (main kernel)
  float2 *tab32;               // FP32 tables (rows in line form, or finite-T (Z, lambda) pairs), precompute kernel
  const double *rad_x, *rad_w; // unit-interval GL rule on [0, 1]
  const double *a1_x, *a1_w;   // first angle rule
  const double *a2_x, *a2_w;   // second angle rule (D4)
  const double *psi_x;         // external angles cos(psi) (D4)
  const double *k_dev;         // optional device scale k (flow stages)
  const double *m2_dev;        // optional device m2_shift (feedback flows)
  const int *skip;             // optional device flag: when non-zero every kernel returns at once
  double *radD;                // optional: d radF / d Z(q) (adjoint)
  double *radF;                // per-(n, r) factor
  double *radq;                // per-r momentum q
  float *radq32;               // per-r momentum q in FP32
  float *radF32;               // radF in FP32 (mixed kernels)
  unsigned *work_ctr;          // optional: dynamic work-item counter, reset by the precompute kernel
  unsigned *fused_ctr;         // optional (finite T): four grid counters of the single-launch mixed RHS
  unsigned *ext_done;          // finished items per external point, reset likewise
  void *kconst;                // kKConstBytes: scale constants of the RHS, written by the precompute kernel
  double *ext_pd;              // per external |p| index: p_i (written by the precompute kernel)
  double *psi_s;               // per external angle: sin(psi) (D4)
  double *partial;             // [n_ext][n_chunks]
  double *out;                 // [n_ext]
  unsigned *status;
};

// ---------------------------------------------------------------------------
// Regulator r(x) = R / (Z k^2) and rdot(x) = k d_k R / (Z k^2), x = q^2/k^2.
// Exponential shape x/(e^x - 1) with dR-shape 2 x^2 e^{-x}/(1-e^{-x})^2;
// flat shape (1-x) Theta(1-x) with dR-shape 2 Theta(1-x).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double reg_r(int reg, double x) {
  if (reg == FFRG_REG_LITIM) return x < 1.0 ? 1.0 - x : 0.0;
  if (x > 700.0) return 0.0;
  if (x < 1e-100) return 1.0;
  return x / expm1(x);
}

__device__ __forceinline__ double reg_rdot(int reg, double x) {
  if (reg == FFRG_REG_LITIM) return x < 1.0 ? 2.0 : 0.0;
  if (x > 700.0) return 0.0;
  if (x < 1e-100) return 2.0;
  double em = expm1(-x);
  return 2.0 * x * x * exp(-x) / (em * em);
}

// Both shapes from one exponential: with em = e^{-x} - 1 (expm1, exact near 0),
// r = x e^{-x} / (1 - e^{-x}) = x/(e^x - 1) and rdot = 2 x^2 e^{-x}/(1 - e^{-x})^2.
__device__ __forceinline__ void reg_r_rdot(int reg, double x, double &r, double &rdot) {
  if (reg == FFRG_REG_LITIM) {
    r = x < 1.0 ? 1.0 - x : 0.0;
    rdot = x < 1.0 ? 2.0 : 0.0;
    return;
  }
  if (x > 700.0) {
    r = rdot = 0.0;
    return;
  }
  if (x < 1e-100) {
    r = 1.0;
    rdot = 2.0;
    return;
  }
  const double em = expm1(-x), inv = 1.0 / em, e = em + 1.0;
  r = -x * e * inv;
  rdot = 2.0 * x * x * e * inv * inv;
}

// Hardware special-function instructions (PTX ISA: lg2/ex2/rcp .approx.ftz.f32).
__device__ __forceinline__ float hw_lg2(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float hw_ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float hw_rsqrt(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
// Programmatic dependent launch: a kernel launched with
// launch_dependent() may start once every CTA of the kernel before it on the
// stream has called pdl_trigger() (or exited); pdl_wait() then holds it until
// that kernel has completed and its writes are visible.  In a kernel launched
// the ordinary way pdl_wait() returns at once.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ float hw_rcp(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// ---------------------------------------------------------------------------
// Log-grid lookup: u = (n-1) ln(s/x_min)/ln(x_max/x_min) = u_scale ln(s^2) + u_off,
// clamped to [0, n-1]; linear in the value between nodes.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void lerp_pos(double s2, double u_scale, double u_off, int n, int &i0, double &w) {
  double u = u_scale * log(s2) + u_off;
  u = fmin(fmax(u, 0.0), (double)(n - 1));
  int i = (int)u;
  i = min(i, n - 2);
  i0 = i;
  w = u - (double)i;
}

// FP32 coordinate, normalised: u1 = u / (n-1) = sat(u_scale1 log2(s^2) + u_off1)
// in one saturating FMA (the caller passes u_scale ln 2 / (n-1) and the
// offset divided by n-1).  s^2 <= 0 gives log2 = -inf or
// NaN, both saturated to 0 (the first node, as for s < x_min).  floor(u) comes
// from u1 (n-1) + 1.5*2^23 rounded towards -inf: the low mantissa bits of the
// sum hold floor(u), so no float<->int conversion is needed.  At u = n-1 this
// gives i0 = n-1, w = 0: the caller's table needs a readable entry after the
// last node (read with weight 0).  Line-form rows (below) use u1 itself.
__device__ __forceinline__ void lerp_pos(float s2, float u_scale1, float u_off1, int n, int &i0, float &w) {
  const float nm1 = (float)(n - 1);
  float u1;
  asm("fma.rn.sat.f32 %0, %1, %2, %3;" : "=f"(u1) : "f"(u_scale1), "f"(hw_lg2(s2)), "f"(u_off1));
  const float magic = 12582912.0f;
  const float t = __fmaf_rd(u1, nm1, magic);
  i0 = __float_as_int(t) - 0x4B400000;
  w = fmaf(u1, nm1, magic - t);
}

// FP32 table rows in line form (d=3, d=4): node i of a row of n nodes holds
// (x, y) = (T_i - i d_i, (n-1) d_i), d_i = T_{i+1} - T_i (0 at the last node),
// so that on [i, i+1] the linear interpolant is x + u1 y at the normalised
// coordinate u1 = u/(n-1): one FMA, no interpolation weight.  A row is
// addressed by its shared-memory byte address minus 8 x 0x4B400000 (mod 2^32,
// Row32): the bit pattern of the floor value t = 1.5 2^23 + i (lerp_pos)
// times 8 then added to it is the address of node i.
struct Row32 {
  unsigned b;
};
struct Pos32 {
  unsigned ib;  // bit pattern of t, times 8
  float u1;
};
__device__ __forceinline__ Row32 row32(const float2 *row) {
  return {(unsigned)__cvta_generic_to_shared(row) - 0x5A000000u};
}
__device__ __forceinline__ Row32 row32_at(Row32 r, int entries) { return {r.b + 8u * (unsigned)entries}; }
__device__ __forceinline__ Pos32 line_pos(float s2, float u_scale1, float u_off1, float nm1) {
  float u1;
  asm("fma.rn.sat.f32 %0, %1, %2, %3;" : "=f"(u1) : "f"(u_scale1), "f"(hw_lg2(s2)), "f"(u_off1));
  const float t = __fmaf_rd(u1, nm1, 12582912.0f);
  return {__float_as_uint(t) << 3, u1};
}
__device__ __forceinline__ float line_at(Row32 r, Pos32 p) {
  float x, y;
  asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(x), "=f"(y) : "r"(r.b + p.ib));
  return fmaf(p.u1, y, x);
}
// table lookup at s2 in the kernel precision: FP64 values, or an FP32 line row
__device__ __forceinline__ float look(Row32 r, float s2, float u_scale1, float u_off1, int n) {
  return line_at(r, line_pos(s2, u_scale1, u_off1, (float)(n - 1)));
}

template <typename T>
__device__ __forceinline__ T lerp_at(const T *tab, int i0, T w) {
  T a = tab[i0], b = tab[i0 + 1];
  return a + w * (b - a);
}

template <typename T>
__device__ __forceinline__ T lerp(const T *tab, T s2, T u_scale, T u_off, int n) {
  int i0;
  T w;
  lerp_pos(s2, u_scale, u_off, n, i0, w);
  return lerp_at(tab, i0, w);
}
__device__ __forceinline__ double look(const double *row, double s2, double u_scale, double u_off, int n) {
  return lerp(row, s2, u_scale, u_off, n);
}

// Propagator denominator Z (omega^2 + s^2 + k^2 r(s^2/k^2)) + m^2, FP64.
__device__ __forceinline__ double prop_den(int reg, double Z, double om2, double s2, double m2, double k2,
                                           double inv_k2) {
  return Z * (om2 + s2 + k2 * reg_r(reg, s2 * inv_k2)) + m2;
}

// Device-wide status word (sticky bits).
__device__ __forceinline__ void raise_status(unsigned *status, unsigned bit) {
  if (status) atomicOr(status, bit);
}

// ---------------------------------------------------------------------------
// TMA bulk staging (cp.async.bulk global -> shared, completion on an mbarrier)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}

// Stage `count` elements from global memory into shared memory.  The 16-byte
// aligned prefix goes through one bulk copy issued by thread 0; the rest (or
// everything, when the source is not 16-byte aligned) through plain loads.
// Every wait is bounded; on timeout the status word gets kStatusTimeout, the
// CTA waits once more (bounded) for its own copy in flight, and returns false.
template <typename T>
__device__ bool stage_to_smem(T *sdst, const T *gsrc, int count, uint64_t *bar, unsigned *status) {
  size_t bytes = (size_t)count * sizeof(T);
  uint32_t bulk = 0;
  if ((((uintptr_t)gsrc) & 15u) == 0 && (((uintptr_t)sdst) & 15u) == 0 && bytes < (1u << 20))
    bulk = (uint32_t)(bytes & ~(size_t)15);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (bulk) {
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bulk)
                   : "memory");
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
              smem_u32(sdst)),
          "l"(gsrc), "r"(bulk), "r"(smem_u32(bar))
          : "memory");
    } else {
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
    }
  }
  for (int i = (int)(bulk / sizeof(T)) + threadIdx.x; i < count; i += blockDim.x) sdst[i] = gsrc[i];
  bool ok = true;
  long long t0 = clock64();
  while (!mbar_try_wait(bar, 0)) {
    if (clock64() - t0 > kWaitCycles) {
      ok = false;
      break;
    }
  }
  if (!ok) {
    raise_status(status, kStatusTimeout);
    long long t1 = clock64();
    while (!mbar_try_wait(bar, 0) && clock64() - t1 < kWaitCycles) {
    }
  }
  int bad = __syncthreads_or(ok ? 0 : 1);
  return bad == 0;
}

// The same staging, repeated: a CTA that stages several inputs in turn (the
// serving kernel, one per flow segment) initialises `bar` once
// (mbar_init_once) and passes the parity of each staging (0, 1, 0, ...).
// Every thread calls it after a block barrier that ends all reads of the
// previous contents of sdst; the async-proxy fence orders those reads before
// the bulk copy's writes.
__device__ __forceinline__ void mbar_init_once(uint64_t *bar) {
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
}
template <typename T>
__device__ bool stage_to_smem_phase(T *sdst, const T *gsrc, int count, uint64_t *bar, unsigned parity,
                                    unsigned *status) {
  size_t bytes = (size_t)count * sizeof(T);
  uint32_t bulk = 0;
  if ((((uintptr_t)gsrc) & 15u) == 0 && (((uintptr_t)sdst) & 15u) == 0 && bytes < (1u << 20))
    bulk = (uint32_t)(bytes & ~(size_t)15);
  if (threadIdx.x == 0) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (bulk) {
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bulk)
                   : "memory");
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
              smem_u32(sdst)),
          "l"(gsrc), "r"(bulk), "r"(smem_u32(bar))
          : "memory");
    } else {
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
    }
  }
  for (int i = (int)(bulk / sizeof(T)) + threadIdx.x; i < count; i += blockDim.x) sdst[i] = gsrc[i];
  bool ok = true;
  long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > kWaitCycles) {
      ok = false;
      break;
    }
  }
  if (!ok) {
    raise_status(status, kStatusTimeout);
    long long t1 = clock64();
    while (!mbar_try_wait(bar, parity) && clock64() - t1 < kWaitCycles) {
    }
  }
  int bad = __syncthreads_or(ok ? 0 : 1);
  return bad == 0;
}

// ---------------------------------------------------------------------------
// Shared helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ double block_sum(double v, double *red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0) {
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
  }
  __syncthreads();
  return t;
}

__device__ __forceinline__ double scale_k(const RhsArgs &a) { return a.k_dev ? *a.k_dev : a.k; }
__device__ __forceinline__ double mass2(const RhsArgs &a, double k) {
  return a.m2_over_k2 * k * k + (a.m2_dev ? *a.m2_dev : a.m2_shift);
}

// The FP32 scale constants from the scale k and m^2 (a division and one log;
// the k-independent parts of the coordinates come from the host).  On the
// device this is FP64 work on one thread, slow on this part, so plain RHS
// calls take the host's copy (fill_args).  The FP32 coordinate offsets are
// formed in FP64 and rounded once (an error of a few FP32 ulps there would
// move lookups by ~1e-5 of a node).
__host__ __device__ inline KConst<float> kconst_f32(const RhsArgs &a, double kd, double m2d) {
  const double k2d = kd * kd, inv_k2d = 1.0 / k2d;
  KConst<float> c;
  c.k2 = (float)k2d;
  c.inv_k2 = (float)inv_k2d;
  c.m2 = (float)m2d;
  c.plim = -2.0f * c.m2;
  c.us = a.us1f;
  c.uo = (float)a.uoc1[0];
  c.sy = (float)(1.4426950408889634074 * inv_k2d);
  c.som = c.sy;  // 1/(k^2 ln 2) = log2(e)/k^2
  c.isy = (float)(0.6931471805599453094 * k2d);
  // coordinates taken in y = sy s^2: shift by -u_scale ln(sy) / (n-1)
  const double lnsy = 0.36651292058166432701 - log(k2d);  // ln(log2 e) - ln k^2
  c.uy1 = (float)(a.uoc1[0] - a.us1 * lnsy);
  c.uy2 = (float)(a.uoc1[1] - a.us1 * lnsy);
  c.uy3 = (float)(a.uoc1[2] - a.us1 * lnsy);
  c.uy4 = (float)(a.uoc1[3] - a.us1 * lnsy);
  c.twopiT = (float)a.twopiT;
  c.sw2 = (float)a.sum_w2;
  return c;
}

__device__ __forceinline__ double ext_momentum(const RhsArgs &a, int ip) {
  return a.p_min * exp((double)ip * a.p_ratio_step);
}

// ---------------------------------------------------------------------------
// Host-side objects.
// ---------------------------------------------------------------------------
struct Plan;

}  // namespace ffrg

struct ffrg_tables {
  ffrg_table_desc desc;
  double *dev;       // FP64 values
  size_t count;      // n_tables * n_stack * n_pts
  size_t bytes;      // allocated bytes (padded)
};

struct ffrg_ctx {
  int device;
  int num_sms;
  size_t budget;
  size_t used;
  unsigned *status_dev;     // sticky device status word
  unsigned *status_host;    // pinned mirror
  std::string last_error;
  std::map<std::vector<long long>, ffrg::Plan *> plans;
  std::vector<void *> owned;  // misc allocations freed at destroy
  void *server;  // ffrg::Server while serving
  int profiling;
  std::vector<cudaEvent_t> prof_events;  // start/stop pairs
  int prof_used;                         // pairs recorded
  // ffrg_flow's per-flow buffers (control block, stage state, stage
  // derivatives, raw RHS, feedback tables), pinned control-block mirror,
  // stream and event: kept between calls, grown when a flow needs more
  void *flow_dev = nullptr;
  size_t flow_cap = 0;
  // ffrg_rhs_host's device outputs, grown on demand
  void *host_out_dev = nullptr;
  size_t host_out_cap = 0;
  void *flow_host = nullptr;
  cudaStream_t flow_stream = nullptr;
  cudaEvent_t flow_ev = nullptr;
  // ffrg_ft_states scratch (operand slices, exact pass sums, scales), grown on demand
  void *states_dev = nullptr;
  size_t states_cap = 0;
  int states_chunks = 0;  // K ranges whose pass table the scratch holds (0: none)
};

namespace ffrg {

// Reusable launch plan for one problem shape: quadrature rules on the device,
// scratch buffers and the launch geometry.
struct Plan {
  std::vector<long long> key;
  int model;
  int nr, na1, na2, n_ext_ang, n_ext_p, N, include_p0, n_ext;
  int stat, nfreq;          // loop statistics and frequency rows (2N+1 bosonic, 2N+2 fermionic)
  int n_tables, n_stack, n_pts, tab_count;
  int cr, n_chunks, n_items, jb;  // block-sized work items (adjoint kernels)
  int fcr, fn_chunks, fn_items;   // warp-sized work items of the mixed forward kernels (and serving)
  int fjb;                        // angle nodes per forward row (D3 / FINITE_T)
  int fcr64, fn_chunks64, fn_items64, fjb64;  // the same for the FP64 forward kernels
  int tab32_count;                // float2 entries of the FP32 table layout
  int tabc_count, n_va, n_vb;     // D4_FULL: compact FP64 table doubles, vertex nodes
  int l3cell;                     // D4_FULL: the FP32 lambda3 cell layout fits in shared memory
  double *tabc;
  size_t kbuf_count;              // FINITE_T: entries of K (N + n_ext_ang) x n_ext_p x n_rad
  double *kbuf;
  int grid64, grid32;       // persistent grids (FP64 / mixed kernels)
  int grid_single;          // finite T, mixed: grid of the single-launch RHS (-1: not available)
  size_t smem64, smem32;    // dynamic shared memory bytes
  size_t smem64g;           // FP64 kernels with tables in global memory: angle rules only
  double *rad_x, *rad_w, *a1_x, *a1_w, *a2_x, *a2_w, *psi_x, *psi_w;
  double sum_w2;
  double *radF, *radq, *partial, *ext_pd, *psi_s;
  float *radq32, *radF32;
  unsigned *work_ctr, *ext_done;
  void *kconst;
  float2 *tab32;
  double *radD, *gpart;     // adjoint scratch (allocated on first use)
  double *jrows;            // Jacobian rows per work item (allocated on first use)
  int adj_grid;
  size_t adj_smem;
  std::vector<double> psi_w_host;
};

// Shape and launch geometry of a plan (no allocation): sizes from the problem
// and the table descriptor, and the grouping of angular rows into work items.
void plan_geometry(Plan *pl, const ffrg_problem *pb, const ffrg_table_desc *td);

// Raise a kernel's dynamic shared-memory limit to at least `bytes` (never
// lowers it: plans of different sizes share the kernel).
int ensure_smem_limit(ffrg_ctx *ctx, const void *func, size_t bytes);

// Several flows' RHS in one set of launches (serving).  Descriptors live in
// device memory; work items of the flows of one model are numbered
// consecutively (flow f owns items start[f] .. start[f+1]-1).
// Flows of one model whose shared-memory need allows the same number of
// resident CTAs per SM run in one main-kernel launch (a flow with large
// tables would otherwise set the occupancy of all).
struct BatchGroup {
  int model;
  const int *flows, *start;  // device: indices into descs, cumulative items (n + 1)
  const long long *cost;     // device: cumulative estimated cost at the flow boundaries (n + 1)
  int n, items;
  size_t smem;               // largest shared-memory need in the group (FP32 path)
};
constexpr int kMaxBatchGroups = 8;  // 2 models x 4 occupancy classes

struct BatchList {
  const RhsArgs *descs;          // [n_flows], device
  int n_flows;
  BatchGroup groups[kMaxBatchGroups];
  int n_groups;
  int max_ext, max_pre;          // largest n_ext and precompute block count among the flows
};
// resident CTAs per SM of the serving main kernel of `model` with `smem` bytes
int batched_ctas_per_sm(ffrg_ctx *ctx, int model, size_t smem);
int launch_rhs_batched(ffrg_ctx *ctx, const BatchList &bl, cudaStream_t s);

// Device control block and argument block of one DP5(4) flow.
struct FlowCtl {
  double t, dt, h, t0, t1, dt_min, dt_max, atol, rtol, end_tol, Lambda;
  double k_stage, m2_stage, err;
  long long steps, rejects, max_steps;
  int last_rejected, done, status, accepted;
};

struct FlowArgs {
  int ny, mode;       // mode: 0 frozen, 1 D3 feedback, 2 D4 feedback
  int n, npsi;        // table points / external angles (feedback)
  int tab_off, tab_len;
  double p_min, p_step;
  const double *psi_w;
  double *y, *ys, *K, *raw, *tabbuf;
  FlowCtl *ctl;
};

int launch_flow_batched_init(ffrg_ctx *ctx, const FlowArgs *fa, int n_flows, int max_ny, const BatchList &bl,
                             cudaStream_t s);
int launch_flow_batched_step(ffrg_ctx *ctx, const FlowArgs *fa, int n_flows, int max_ny, const BatchList &bl,
                             cudaStream_t s);

// Launch `kern` on `s`; with `early`, as a programmatic dependent of the
// kernel launched just before it (its CTAs may start while that kernel runs
// and must call pdl_wait() before reading what it writes).  Under stream
// capture the dependency becomes a programmatic edge of the graph (the flow
// steps: d=3 mixed flow 5.18 -> 4.67 ms).
template <typename... P, typename... A>
cudaError_t launch_dependent(void (*kern)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, bool early,
                             A &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = early ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<A &&>(args)...);
}

// helpers implemented in ffrg_api.cu
int set_cuda_error(ffrg_ctx *ctx, cudaError_t e, const char *what);
int dev_alloc(ffrg_ctx *ctx, void **p, size_t bytes);
void dev_free(ffrg_ctx *ctx, void *p, size_t bytes);
int validate_problem(const ffrg_problem *pb, const ffrg_table_desc *td);
int get_plan(ffrg_ctx *ctx, const ffrg_problem *pb, const ffrg_table_desc *td, Plan **out);
void fill_args(const Plan *pl, const ffrg_problem *pb, const ffrg_table_desc *td, const double *tab, double k,
               RhsArgs &a);
int host_gauss_legendre(int n, double a, double b, double *x, double *w);
int host_gauss_chebyshev2(int n, double *x, double *w);

// kernels launched from several translation units (ffrg_rhs.cu)
int launch_rhs(ffrg_ctx *ctx, const Plan *pl, const RhsArgs &a, int precision, cudaStream_t s);
// the finite-T model with a 4D regulator (frequency set, loop factors, one
// block per external point); launch_rhs dispatches to it
int launch_ft4(ffrg_ctx *ctx, const Plan *pl, const RhsArgs &a, int precision, cudaStream_t s);
// launch_rhs with the finite-T contraction optional: contract = false stops
// after the angle-integrated kernel K (plan kbuf, in the kernel precision)
int launch_rhs_stages(ffrg_ctx *ctx, const Plan *pl, const RhsArgs &a, int precision, cudaStream_t s,
                      bool contract);
int launch_precompute(ffrg_ctx *ctx, const RhsArgs &a, cudaStream_t s);
// blocks of the precompute kernel for one RHS (at most cap)
int precompute_blocks(const RhsArgs &a, int cap);
int launch_jacobian(ffrg_ctx *ctx, const ffrg_problem *pb, const ffrg_table_desc *td, const double *tab, double k,
                    double *J, cudaStream_t s);

}  // namespace ffrg
