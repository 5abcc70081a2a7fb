// Finite-T sums over many loop-side states sharing one angle-integrated
// kernel K(p, q) (Sec. 5.3.2 momentum integrals; the finite-T RHS is the sum
// over loop frequencies n and radial nodes r of a loop-side factor F(n, r)
// times the angular sum of the shifted line, K[j(n+m)][p][r]):
//
//   out[s][e] = norm sum_{n, r} w_r q_r^2 F_s(n, r) K[j(n + m_e)][p_e][r]
//
// For S states this is one dense product A B^T with A[(m, p)][(n, r)] =
// K[j(n+m)][p][r] (n_ext x nfreq n_rad) and B[s][(n, r)] = w_r q_r^2 F_s(n, r).
// It runs on the tensor cores, FP64-faithful, by an Ozaki-type split:
//   - each row of A and of B is scaled by a power of two 2^-e so that its
//     largest magnitude is below 1, then cut into kSlices fixed-point slices
//     of kBits bits, x = sum_i x_i 2^(-kBits (i+1)), x_0 integer in
//     [-32, 32], x_i in [-16, 16]; the integers are exact in BF16;
//   - a slice pair (i, j) summed over at most 2^14 K-elements is an integer
//     below 2^24 in magnitude, exact in the FP32 tensor-memory accumulator
//     (ffrg_umma.cuh); every pair with i + j < kSlices is one pass;
//   - per output, the passes of one level i + j are added as integers
//     (exact), the levels in FP64 from the smallest, and the result scaled by
//     norm 2^(e_row + e_state - 2 kBits).
// The neglected levels and slice residuals are below ~2^-48 of
// max|A_row| max|B_s| per term.
#include <math.h>

#include <algorithm>
#include <vector>

#include "ffrg_internal.cuh"
#include "ffrg_umma.cuh"

namespace ffrg {

constexpr int kSlices = 10;
constexpr int kBits = 5;

struct StatesScratch {
  uint16_t *A, *B;
  float *part;
  int *e_row, *e_col;
  int4 *pass_tab;
};

// BF16 bits of a small integer held in a float (exact: at most 8 significant bits)
__device__ __forceinline__ uint16_t bf16_int(float v) { return (uint16_t)(__float_as_uint(v) >> 16); }

// |v| as an ordered integer (IEEE bit pattern without the sign)
__device__ __forceinline__ unsigned long long mag_bits(double v) {
  return (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull;
}

// exponent e with |x| < 2^e for every |x| whose bit pattern is at most m (0 for m = 0)
__device__ __forceinline__ int scale_exp_bits(unsigned long long m) {
  return m ? (int)(m >> 52) - 1022 : 0;
}

__device__ __forceinline__ unsigned long long block_max_bits(unsigned long long v, unsigned long long *red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  unsigned long long m = 0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = red[w] > m ? red[w] : m;
  __syncthreads();
  return m;
}

// X = round(v 2^(50 - e)) as an integer, |X| <= 2^50 for |v| < 2^e (integer
// operations on the IEEE fields; subnormal v gives 0)
__device__ __forceinline__ long long fixed50(double v, int e) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  const int E = (int)((u >> 52) & 0x7FF);
  if (E == 0) return 0;
  const long long M = (long long)((u & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull);
  const int sh = E - 1025 - e;           // v 2^(50-e) = M 2^sh
  long long X;
  if (sh >= 0) X = M << sh;
  else if (sh > -54) X = (M + (1ll << (-sh - 1))) >> (-sh);
  else X = 0;
  return (u >> 63) ? -X : X;
}

// slices of the 8 values v[0..7] (scale 2^-e) at K-elements 8g .. 8g + 7 of
// row `row` of a panel with tiles `th` rows high: x = sum_i a_i 2^(-5(i+1)),
// a_i = round of the remainder at weight 2^(45 - 5i) (shifts of X); one
// 16-byte core-matrix row per slice, slice arrays `slice_elems` apart
__device__ __forceinline__ void write_slices8(uint16_t *dst, size_t slice_elems, int k_tiles, int row, int th, int g,
                                              const double (&v)[8], int e) {
  const int col = 8 * g;
  const size_t off = ((size_t)(row / th) * k_tiles + col / umma::kBK) * (size_t)(th * umma::kBK) +
                     umma::tile_offset(row % th, col % umma::kBK, th);
  long long X[8];
#pragma unroll
  for (int h = 0; h < 8; ++h) X[h] = fixed50(v[h], e);
#pragma unroll
  for (int i = 0; i < kSlices; ++i) {
    const int w = kBits * (kSlices - 1 - i);
    uint32_t pk[4];
#pragma unroll
    for (int h = 0; h < 8; ++h) {
      long long a = X[h];
      if (w > 0) {
        a = (X[h] + (1ll << (w - 1))) >> w;
        X[h] -= a << w;
      }
      const uint32_t b = (uint32_t)bf16_int((float)(int)a);
      if (h & 1) pk[h >> 1] |= b << 16;
      else pk[h >> 1] = b;
    }
    *reinterpret_cast<uint4 *>(dst + (size_t)i * slice_elems + off) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
  }
}

struct SplitArgs {
  const void *K;          // angle-integrated kernel [N + M][n_p][n_rad], double or float
  int k_double;
  const double *F;        // states [S][nfreq][n_rad] (B split)
  const double *rad_x, *rad_w;  // unit radial rule on [0, 1]
  double qscale;          // k qmax: q_r = qscale x_r
  int n_p, nm, nr, nfreq, n_lo, stat, n_rows, n_cols, kdim, k_tiles;
  uint16_t *A, *B;
  int *e_row, *e_col;
  size_t a_slice, b_slice;  // elements per slice array
};

// one block per row of A (external point e = (p, m); padded rows are zero)
__global__ void __launch_bounds__(256) split_A_kernel(SplitArgs g) {
  __shared__ unsigned long long red[8];
  const int row = blockIdx.x;
  const int kpad = g.k_tiles * umma::kBK;
  const bool live = row < g.n_rows;
  const int ip = live ? row / g.nm : 0, m = live ? row % g.nm : 0;
  auto val = [&](int col) -> double {
    if (!live || col >= g.kdim) return 0.0;
    const int nrow = col / g.nr, r = col - nrow * g.nr;
    const int n = nrow + g.n_lo + m;
    const int j = g.stat ? (n >= 0 ? n : -n - 1) : abs(n);
    const size_t o = ((size_t)j * g.n_p + ip) * g.nr + r;
    return g.k_double ? ((const double *)g.K)[o] : (double)((const float *)g.K)[o];
  };
  unsigned long long mx = 0;
  for (int c = threadIdx.x; c < kpad; c += blockDim.x) {
    const unsigned long long b = mag_bits(val(c));
    mx = b > mx ? b : mx;
  }
  const int e = scale_exp_bits(block_max_bits(mx, red));
  if (threadIdx.x == 0) g.e_row[row] = e;
  for (int q = threadIdx.x; q < kpad / 8; q += blockDim.x) {
    double v[8];
#pragma unroll
    for (int h = 0; h < 8; ++h) v[h] = val(8 * q + h);
    write_slices8(g.A, g.a_slice, g.k_tiles, row, umma::kBM, q, v, e);
  }
}

// one block per state (padded states are zero); the state carries the radial
// weight and measure w_r q_r^2 (from the unit rule, staged per block)
__global__ void __launch_bounds__(256) split_B_kernel(SplitArgs g) {
  __shared__ unsigned long long red[8];
  extern __shared__ double wq[];   // [n_rad]: (k qmax)^3 w_r x_r^2
  const int s = blockIdx.x;
  const int kpad = g.k_tiles * umma::kBK;
  const bool live = s < g.n_cols;
  const double q3 = g.qscale * g.qscale * g.qscale;
  for (int r = threadIdx.x; r < g.nr; r += blockDim.x) wq[r] = q3 * g.rad_w[r] * g.rad_x[r] * g.rad_x[r];
  __syncthreads();
  auto val = [&](int col) -> double {
    if (!live || col >= g.kdim) return 0.0;
    return wq[col % g.nr] * g.F[(size_t)s * g.kdim + col];
  };
  unsigned long long mx = 0;
  for (int c = threadIdx.x; c < kpad; c += blockDim.x) {
    const unsigned long long b = mag_bits(val(c));
    mx = b > mx ? b : mx;
  }
  const int e = scale_exp_bits(block_max_bits(mx, red));
  if (threadIdx.x == 0) g.e_col[s] = e;
  for (int q = threadIdx.x; q < kpad / 8; q += blockDim.x) {
    double v[8];
#pragma unroll
    for (int h = 0; h < 8; ++h) v[h] = val(8 * q + h);
    write_slices8(g.B, g.b_slice, g.k_tiles, s, umma::kBN, q, v, e);
  }
}

struct CombineArgs {
  const float *part;     // [passes][rows_pad][cols_pad]
  const int *e_row, *e_col;
  double *out;           // [S][n_ext]
  unsigned *status;
  double norm;
  int n_rows, n_cols, rows_pad, cols_pad, n_chunks;
};

// pass index of slice pair (i, j) in level order: level l = i + j holds the
// pairs (0, l), (1, l - 1), ..., (l, 0)
__host__ __device__ inline int pair_index(int i, int j) {
  const int l = i + j;
  return l * (l + 1) / 2 + i;
}

// thread per output (state fastest): the passes of a level are exact
// integers (|sum| < 2^24 each, at most 10 x 12 of them per level: the sum
// fits a 32-bit integer for n_chunks <= 12); levels 0..6 are combined exactly
// in a 64-bit integer at weight 2^(30 - 5l), levels 7..9 and the scales in FP64
__global__ void __launch_bounds__(256) combine_kernel(CombineArgs g) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)g.n_rows * g.n_cols) return;
  const int e = (int)(t / g.n_cols), s = (int)(t % g.n_cols);
  const size_t plane = (size_t)g.rows_pad * g.cols_pad, at = (size_t)e * g.cols_pad + s;
  // the passes in pair_index order (level l = 0, 1, ...): all loads independent
  constexpr int kPairs = kSlices * (kSlices + 1) / 2;
  int lsum[kSlices];
#pragma unroll
  for (int l = 0; l < kSlices; ++l) lsum[l] = 0;
  for (int c = 0; c < g.n_chunks; ++c) {
    float v[kPairs];
#pragma unroll
    for (int p = 0; p < kPairs; ++p) v[p] = g.part[(size_t)(p * g.n_chunks + c) * plane + at];
#pragma unroll
    for (int l = 0, p = 0; l < kSlices; ++l)
#pragma unroll
      for (int i = 0; i <= l; ++i, ++p) lsum[l] += __float2int_rn(v[p]);
  }
  long long hi = 0;
  double tail = 0.0;
#pragma unroll
  for (int l = kSlices - 1; l >= 0; --l) {
    if (l > 6) tail += ldexp((double)lsum[l], -kBits * l);
    else hi += (long long)lsum[l] << (kBits * (6 - l));
  }
  const double acc = ldexp((double)hi, -30) + tail;
  const double v = g.norm * ldexp(acc, g.e_row[e] + g.e_col[s] - 2 * kBits);
  g.out[(size_t)s * g.n_rows + e] = v;
  if (!isfinite(v)) atomicOr(g.status, kStatusNonFinite);
}

}  // namespace ffrg

using namespace ffrg;

extern "C" int ffrg_ft_states(ffrg_ctx *ctx, const ffrg_problem *pb, const ffrg_tables *tables, double k,
                              int n_states, const double *F_dev, double *out_dev, int precision, void *stream) {
  if (!ctx || !pb || !tables || !F_dev || !out_dev) return FFRG_EINVAL;
  if (pb->model != FFRG_MODEL_FINITE_T || n_states < 1) return FFRG_EINVAL;
  if (!(k > 0.0) || !isfinite(k)) return FFRG_EINVAL;
  if (precision != FFRG_FP64 && precision != FFRG_MIXED) return FFRG_EINVAL;
  int st = validate_problem(pb, &tables->desc);
  if (st) return st;
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  Plan *pl = nullptr;
  st = get_plan(ctx, pb, &tables->desc, &pl);
  if (st) return st;

  // geometry of the product
  const int n_rows = pl->n_ext, kdim = pl->nfreq * pl->nr;
  const int m_tiles = (n_rows + umma::kBM - 1) / umma::kBM;
  const int n_tiles = (n_states + umma::kBN - 1) / umma::kBN;
  const int k_tiles = (kdim + umma::kBK - 1) / umma::kBK;
  const int kt_chunk = std::min(k_tiles, umma::kMaxExactK / umma::kBK);
  const int n_chunks = (k_tiles + kt_chunk - 1) / kt_chunk;
  if (n_chunks > 12) {   // level sums must fit 32-bit integers: nfreq n_rad <= 12 x 16384
    ctx->last_error = "ffrg_ft_states: more than 196608 (loop frequency, radial node) terms";
    return FFRG_EINVAL;
  }
  const int n_pairs = kSlices * (kSlices + 1) / 2;
  const int passes = n_pairs * n_chunks;
  const int rows_pad = m_tiles * umma::kBM, cols_pad = n_tiles * umma::kBN;
  const size_t a_slice = (size_t)rows_pad * k_tiles * umma::kBK, b_slice = (size_t)cols_pad * k_tiles * umma::kBK;

  // K in the requested precision (the finite-T RHS up to, not including, its contraction)
  RhsArgs a;
  fill_args(pl, pb, &tables->desc, tables->dev, k, a);
  a.out = out_dev;   // not written: no contraction
  a.status = ctx->status_dev;
  const int prof_on = ctx->profiling;   // the profiling events time the tensor-core kernel only
  ctx->profiling = 0;
  st = launch_rhs_stages(ctx, pl, a, precision, s, false);
  ctx->profiling = prof_on;
  if (st) return st;

  // scratch, kept by the context and grown on demand (256-byte segments):
  // pass table (room for 12 K ranges) | A slices | B slices | pass sums | scales
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t o_A = al((size_t)n_pairs * 12 * sizeof(int4));
  const size_t o_B = o_A + al(kSlices * a_slice * 2), o_part = o_B + al(kSlices * b_slice * 2);
  const size_t o_er = o_part + al((size_t)passes * rows_pad * cols_pad * 4);
  const size_t o_ec = o_er + al((size_t)rows_pad * 4);
  const size_t need = o_ec + al((size_t)cols_pad * 4);
  if (ctx->states_cap < need) {
    dev_free(ctx, ctx->states_dev, ctx->states_cap);
    ctx->states_dev = nullptr;
    ctx->states_cap = 0;
    ctx->states_chunks = 0;
    st = dev_alloc(ctx, &ctx->states_dev, need);
    if (st) return st;
    ctx->states_cap = need;
  }
  unsigned char *base = (unsigned char *)ctx->states_dev;
  StatesScratch sc{(uint16_t *)(base + o_A), (uint16_t *)(base + o_B), (float *)(base + o_part),
                   (int *)(base + o_er), (int *)(base + o_ec), (int4 *)base};
  if (ctx->states_chunks != n_chunks) {
    // the pass table, one slot per CTA z: slice pair (i, j), its output pass
    // (pair_index order, K ranges innermost) and K range.  Slots run in order
    // of i, so CTAs that run together read the same A slice (uploaded when the
    // number of K ranges changes)
    std::vector<int4> ij((size_t)passes);
    size_t z = 0;
    for (int i = 0; i < kSlices; ++i)
      for (int j = 0; i + j < kSlices; ++j)
        for (int c = 0; c < n_chunks; ++c) ij[z++] = make_int4(i, j, pair_index(i, j) * n_chunks + c, c);
    st = set_cuda_error(ctx, cudaMemcpyAsync(sc.pass_tab, ij.data(), ij.size() * sizeof(int4),
                                             cudaMemcpyHostToDevice, s), "ffrg_ft_states pass table");
    // from pageable memory: the copy must have read ij before it goes away
    if (!st) st = set_cuda_error(ctx, cudaStreamSynchronize(s), "ffrg_ft_states pass table");
    if (st) return st;
    ctx->states_chunks = n_chunks;
  }

  SplitArgs sg;
  sg.K = pl->kbuf;
  sg.k_double = precision == FFRG_FP64;
  sg.F = F_dev;
  sg.rad_x = pl->rad_x;
  sg.rad_w = pl->rad_w;
  sg.qscale = k * pb->qmax_over_k;
  sg.n_p = pl->n_ext_p;
  sg.nm = pl->n_ext_ang;
  sg.nr = pl->nr;
  sg.nfreq = pl->nfreq;
  sg.n_lo = -pl->N - pl->stat;
  sg.stat = pl->stat;
  sg.n_rows = n_rows;
  sg.n_cols = n_states;
  sg.kdim = kdim;
  sg.k_tiles = k_tiles;
  sg.A = sc.A;
  sg.B = sc.B;
  sg.e_row = sc.e_row;
  sg.e_col = sc.e_col;
  sg.a_slice = a_slice;
  sg.b_slice = b_slice;
  split_A_kernel<<<rows_pad, 256, 0, s>>>(sg);
  split_B_kernel<<<cols_pad, 256, (size_t)pl->nr * sizeof(double), s>>>(sg);

  st = ensure_smem_limit(ctx, (const void *)umma::slice_pair_gemm, umma::kSmemBytes);
  if (st) return st;
  umma::GemmArgs gg{sc.A, sc.B, sc.part, sc.pass_tab, m_tiles, n_tiles, k_tiles, kt_chunk, n_chunks,
                    ctx->status_dev};
  const bool prof = ctx->profiling && ctx->prof_used * 2 + 1 < (int)ctx->prof_events.size();
  if (prof) cudaEventRecord(ctx->prof_events[2 * ctx->prof_used], s);
  umma::slice_pair_gemm<<<dim3(n_tiles, m_tiles, passes), umma::kThreadsGemm, umma::kSmemBytes, s>>>(gg);
  if (prof) {
    cudaEventRecord(ctx->prof_events[2 * ctx->prof_used + 1], s);
    ctx->prof_used++;
  }

  CombineArgs cg{sc.part, sc.e_row, sc.e_col, out_dev, ctx->status_dev, a.norm, n_rows, n_states, rows_pad,
                 cols_pad, n_chunks};
  const long long n_out = (long long)n_rows * n_states;
  combine_kernel<<<(unsigned)((n_out + 255) / 256), 256, 0, s>>>(cg);
  return set_cuda_error(ctx, cudaGetLastError(), "ffrg_ft_states launch");
}
