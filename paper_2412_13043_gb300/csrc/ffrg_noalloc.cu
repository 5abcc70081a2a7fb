// ffrg_rhs_noalloc: the RHS of ffrg_rhs for callers that cannot allocate
// device memory.  It runs the same kernels (precompute, main, finite-T
// contraction) as ffrg_rhs, but all of its scratch -- quadrature rules, per-radial factors,
// partial sums, the FP32 table mirror and a status word -- lives in one
// file-scope device array of fixed size instead of cudaMalloc'd buffers.  No
// context, no cudaMalloc/cudaFree, no allocating library routine.
//
// The array belongs to every GPU that loads this library until the process
// exits.  Host code must not hand the array's name to a kernel: on the host it
// is only a stand-in for the symbol.  The device address is looked up once per
// device with cudaGetSymbolAddress (on the first call made with that device
// current) and passed to the kernels.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "ffrg_internal.cuh"

namespace ffrg {

constexpr size_t kNoallocScratchBytes = size_t(4) << 20;  // 4 MiB
constexpr int kNoallocMaxDevices = 64;

// Shared by every call of ffrg_rhs_noalloc on a device; keeps the last call's contents.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

static std::mutex g_noalloc_mu;
static unsigned char *g_noalloc_ptr[kNoallocMaxDevices];  // device address per device

static cudaError_t noalloc_scratch_for_current_device(int dev, unsigned char **out) {
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = (unsigned char *)p;
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}

// The call has no context whose status word a caller could read, so a
// bounded device wait that gave up (kStatusTimeout) is reported through the
// outputs: every entry becomes NaN, instead of keeping values that a CTA
// never wrote (the previous call's, or from stale scratch).
__global__ void noalloc_poison_on_timeout(const unsigned *status, double *out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && (*(volatile const unsigned *)status & kStatusTimeout)) out[i] = __longlong_as_double(-1ll);
}

// Bump allocator over the fixed array (256-byte aligned segments).
struct ScratchCarver {
  unsigned char *base;
  size_t used;
  template <typename T>
  T *take(size_t count) {
    size_t off = (used + 255) & ~(size_t)255;
    used = off + std::max<size_t>(count * sizeof(T), 16);
    return (T *)(base + off);
  }
};

}  // namespace ffrg

using namespace ffrg;

extern "C" int ffrg_rhs_noalloc(const ffrg_problem *pb, const ffrg_table_desc *td, const double *tables_dev,
                                double k, double *out_dev, int precision, void *stream) {
  if (!pb || !td || !tables_dev || !out_dev) return FFRG_EINVAL;
  if (!(k > 0.0) || !isfinite(k)) return FFRG_EINVAL;
  if (precision != FFRG_FP64 && precision != FFRG_MIXED) return FFRG_EINVAL;
  if (validate_problem(pb, td) != FFRG_OK) return FFRG_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FFRG_ECUDA;
  if (dev < 0 || dev >= kNoallocMaxDevices) return FFRG_EINVAL;
  unsigned char *base = nullptr;
  if (noalloc_scratch_for_current_device(dev, &base) != cudaSuccess) return FFRG_ECUDA;

  // Launch geometry: the same grouping of angular rows into work items as the
  // cached plans of ffrg_rhs use.
  Plan pl = Plan();
  plan_geometry(&pl, pb, td);

  // quadrature rules on the host
  std::vector<double> rx(pl.nr), rw(pl.nr), x1(pl.na1), w1(pl.na1), x2(pl.na2), w2(pl.na2);
  int npsi = std::max(1, pl.n_ext_ang);
  std::vector<double> xp(npsi), wp(npsi);
  host_gauss_legendre(pl.nr, 0.0, 1.0, rx.data(), rw.data());
  if (is_d4(pb->model)) host_gauss_chebyshev2(pl.na1, x1.data(), w1.data());
  else host_gauss_legendre(pl.na1, -1.0, 1.0, x1.data(), w1.data());
  host_gauss_legendre(pl.na2, -1.0, 1.0, x2.data(), w2.data());
  host_gauss_legendre(npsi, -1.0, 1.0, xp.data(), wp.data());
  pl.sum_w2 = 0.0;
  for (double v : w2) pl.sum_w2 += v;

  // carve the fixed array; reject problems that do not fit
  ScratchCarver sc{base, 0};
  unsigned *status = sc.take<unsigned>(4);
  pl.rad_x = sc.take<double>(pl.nr);
  pl.rad_w = sc.take<double>(pl.nr);
  pl.a1_x = sc.take<double>(pl.na1);
  pl.a1_w = sc.take<double>(pl.na1);
  pl.a2_x = sc.take<double>(pl.na2);
  pl.a2_w = sc.take<double>(pl.na2);
  pl.psi_x = sc.take<double>(npsi);
  pl.psi_w = sc.take<double>(npsi);
  pl.radF = sc.take<double>((size_t)pl.nr * pl.nfreq);
  pl.radq = sc.take<double>(pl.nr);
  pl.radq32 = sc.take<float>(pl.nr);
  pl.radF32 = sc.take<float>((size_t)pl.nr * pl.nfreq);
  pl.work_ctr = sc.take<unsigned>(4);
  pl.ext_done = sc.take<unsigned>(pl.n_ext);
  pl.kconst = sc.take<double>(kKConstBytes / sizeof(double));
  pl.ext_pd = sc.take<double>(pl.n_ext_p);
  pl.psi_s = sc.take<double>(npsi);
  pl.partial = sc.take<double>(std::max(pl.fn_items, pl.fn_items64));
  pl.tab32 = sc.take<float2>((size_t)pl.tab32_count);
  if (pl.tabc_count) pl.tabc = sc.take<double>((size_t)pl.tabc_count);
  if (pl.kbuf_count) pl.kbuf = sc.take<double>(pl.kbuf_count);
  if (sc.used > kNoallocScratchBytes) return FFRG_EINVAL;  // problem needs more than the 4 MiB scratch

  const size_t smem = precision == FFRG_MIXED ? pl.smem32 : pl.smem64;
  if (smem > 227 * 1024) return FFRG_EINVAL;

  cudaStream_t s = (cudaStream_t)stream;
  const size_t db = sizeof(double);
  cudaError_t e = cudaMemsetAsync(status, 0, 4 * sizeof(unsigned), s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(pl.rad_x, rx.data(), pl.nr * db, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(pl.rad_w, rw.data(), pl.nr * db, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(pl.a1_x, x1.data(), pl.na1 * db, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(pl.a1_w, w1.data(), pl.na1 * db, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(pl.a2_x, x2.data(), pl.na2 * db, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(pl.a2_w, w2.data(), pl.na2 * db, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(pl.psi_x, xp.data(), npsi * db, cudaMemcpyHostToDevice, s);
  // copies from pageable host memory return once the source has been staged,
  // so the host vectors may go out of scope afterwards
  if (e == cudaSuccess) e = cudaMemcpyAsync(pl.psi_w, wp.data(), npsi * db, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return FFRG_ECUDA;

  // a context-free stand-in for the launch helpers (no device memory behind it)
  ffrg_ctx lc;
  lc.device = dev;
  lc.budget = 0;
  lc.used = 0;
  lc.status_dev = status;
  lc.status_host = nullptr;
  lc.server = nullptr;
  lc.profiling = 0;
  lc.prof_used = 0;
  if (cudaDeviceGetAttribute(&lc.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return FFRG_ECUDA;
  pl.grid64 = 0;
  pl.grid32 = 0;
  RhsArgs a;
  fill_args(&pl, pb, td, tables_dev, k, a);
  a.fused_ctr = nullptr;   // the scratch holds no persistent grid counters: the three-launch finite-T path
  a.out = out_dev;
  a.status = status;
  int st = launch_rhs(&lc, &pl, a, precision, s);
  if (st != FFRG_OK) return st;
  noalloc_poison_on_timeout<<<(pl.n_ext + 255) / 256, 256, 0, s>>>(status, out_dev, pl.n_ext);
  return cudaGetLastError() == cudaSuccess ? FFRG_OK : FFRG_ECUDA;
}
