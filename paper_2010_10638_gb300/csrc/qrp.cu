// K-c: Householder QR with column pivoting, truncated after k reflectors, FP64
// (Section III-D: A P = Q R with |r_11| >= |r_22| >= ...; H_j = I - 2 v v^T / v^T v,
// v = a + sign(a_1) ||a|| e_1, sign(0) = +1).  The paper runs this step on the CPU
// because each pivot choice depends on the column norms left by the previous
// reflector; on the GPU the sequential part is tiny and the bulk of every step is
// one streaming matrix-vector product over A.
//
// The matrix A is never modified.  After j reflectors the working matrix is kept
// implicitly as  A P - V F^T  (V: m x j reflectors, F: n x j, F[:, l] = tau_l *
// (P^T A^T v_l - F V^T v_l)), so every step reads A once (FP32 input is upcast
// exactly, accumulation is FP64).  Per step:
//   kernel A  rows of the updated pivot column -> V[:, j], partial ||.||^2;
//             the last block to finish forms the reflector (tau, beta, v_jj)
//   kernel B  partial sums of A^T v_j (2-D grid: row chunks x 64-column chunks)
//             and of V^T v_j; the last block reduces them in a fixed order, forms
//             F[:, j], row j of R, downdates the trailing column norms, extends the
//             compact-WY factor T, and picks and swaps in the next pivot
//   kernel R  only when a downdated norm lost too much to cancellation (it fell
//             below sqrt(eps) of its last exact value): exact recomputation of
//             those norms, then the pivot choice
// Q = H_1 ... H_k [I_k; 0] = [I_k; 0] - V T V[0:k, :]^T at the end.
// Ties in the pivot choice go to the lowest current column position.  A zero pivot
// column gives tau = 0 (H = I).  "Last block" = the block whose atomic ticket is the
// last one; it waits for nobody, so there is no spin anywhere.
#include <algorithm>
#include <cfloat>
#include <cstdlib>
#include <cstring>

#include "dfloat.cuh"
#include "internal.cuh"

namespace tk {

constexpr int kQThreads = 256;
constexpr int kQCols = 64;  // columns per block in the GEMV grid

struct QrpArgs {
  const void *A;
  int64_t m, n, lda;
  int k;
  double *V, *F, *part, *vn, *vref, *T, *M, *scal;
  int *perm, *flag, *iscal;
  unsigned *counter;
  int64_t *piv;
  double *rdiag;
  int row_chunks;  // grid.y of kernel B
  int64_t part_ld; // row stride of `part`
};

template <typename AT>
__device__ __forceinline__ double aload(const void *A, int64_t lda, int64_t i, int64_t c) {
  return (double)__ldg(static_cast<const AT *>(A) + i * lda + c);
}

__device__ __forceinline__ bool last_block(unsigned *counter, unsigned nblocks) {
  __shared__ bool is_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = (atomicAdd(counter, 1u) == nblocks - 1u);
  __syncthreads();
  if (is_last) __threadfence();
  return is_last;
}

__device__ __forceinline__ double block_sum(double v, double *sm) {
  sm[threadIdx.x] = v;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
    __syncthreads();
  }
  double r = sm[0];
  __syncthreads();
  return r;
}

// argmax of vn over positions [j0, n), lowest position on ties; then swap it into j0
// (perm, vn, vref and rows of F over the first j0 columns).  One block.
__device__ void choose_and_swap(const QrpArgs &a, int j0) {
  __shared__ double bv[kQThreads];
  __shared__ int bi[kQThreads];
  double best = -1.0;
  int bidx = INT_MAX;
  for (int64_t c = j0 + threadIdx.x; c < a.n; c += blockDim.x) {
    double v = __ldcg(a.vn + c);
    if (v > best) {  // strided ascending: first occurrence wins within the thread
      best = v;
      bidx = (int)c;
    }
  }
  bv[threadIdx.x] = best;
  bi[threadIdx.x] = bidx;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      double v2 = bv[threadIdx.x + o];
      int i2 = bi[threadIdx.x + o];
      if (v2 > bv[threadIdx.x] || (v2 == bv[threadIdx.x] && i2 < bi[threadIdx.x])) {
        bv[threadIdx.x] = v2;
        bi[threadIdx.x] = i2;
      }
    }
    __syncthreads();
  }
  const int p = bi[0];
  __syncthreads();
  if (p != j0 && p < a.n) {
    if (threadIdx.x == 0) {
      int t = a.perm[j0];
      a.perm[j0] = a.perm[p];
      a.perm[p] = t;
      double d = a.vn[j0];
      a.vn[j0] = a.vn[p];
      a.vn[p] = d;
      d = a.vref[j0];
      a.vref[j0] = a.vref[p];
      a.vref[p] = d;
    }
    for (int l = threadIdx.x; l < j0; l += blockDim.x) {
      double t = a.F[(int64_t)j0 * a.k + l];
      a.F[(int64_t)j0 * a.k + l] = a.F[(int64_t)p * a.k + l];
      a.F[(int64_t)p * a.k + l] = t;
    }
  }
  if (threadIdx.x == 0) a.iscal[0] = p;
  __syncthreads();
}

// ---- init: exact column norms, identity order, first pivot
template <typename AT>
__global__ void __launch_bounds__(kQThreads) qrp_init_kernel(QrpArgs a) {
  // grid: (column chunks, row chunks) as kernel B
  const int cl = threadIdx.x & (kQCols - 1), rl = threadIdx.x / kQCols;
  const int64_t c = (int64_t)blockIdx.x * kQCols + cl;
  const int64_t rows_per = (a.m + gridDim.y - 1) / gridDim.y;
  const int64_t r0 = (int64_t)blockIdx.y * rows_per, r1 = min(a.m, r0 + rows_per);
  __shared__ double sm[kQThreads];
  double s = 0.0;
  if (c < a.n)
    for (int64_t i = r0 + rl; i < r1; i += kQThreads / kQCols) {
      double v = aload<AT>(a.A, a.lda, i, c);
      s = fma(v, v, s);
    }
  sm[threadIdx.x] = s;
  __syncthreads();
  if (rl == 0 && c < a.n) {
    double t = 0.0;
    for (int q = 0; q < kQThreads / kQCols; ++q) t += sm[q * kQCols + cl];
    a.part[(int64_t)blockIdx.y * a.part_ld + c] = t;
  }
  if (!last_block(a.counter, gridDim.x * gridDim.y)) return;
  for (int64_t cc = threadIdx.x; cc < a.n; cc += blockDim.x) {
    double t = 0.0;
    for (int b = 0; b < (int)gridDim.y; ++b) t += __ldcg(a.part + (int64_t)b * a.part_ld + cc);
    a.vn[cc] = t;
    a.vref[cc] = t;
    a.perm[cc] = (int)cc;
    a.flag[cc] = 0;
  }
  for (int64_t q = threadIdx.x; q < (int64_t)a.k * a.k; q += blockDim.x) a.T[q] = 0.0;
  if (threadIdx.x == 0) a.iscal[1] = 0;
  __syncthreads();
  __threadfence_block();
  if (a.k > 0) choose_and_swap(a, 0);
  if (threadIdx.x == 0) *a.counter = 0u;
}

// ---- kernel A: updated pivot column rows -> V[:, j]; last block forms the reflector
template <typename AT>
__global__ void __launch_bounds__(kQThreads) qrp_col_kernel(QrpArgs a, int j) {
  __shared__ double sm[kQThreads];
  __shared__ double fj[64];
  const int64_t rows_per = (a.m + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = (int64_t)blockIdx.x * rows_per, r1 = min(a.m, r0 + rows_per);
  const int c0 = a.perm[j];
  double s = 0.0;
  for (int l0 = 0; l0 < max(j, 1); l0 += 64) {
    const int nl = min(64, j - l0);
    __syncthreads();
    if (threadIdx.x < nl) fj[threadIdx.x] = a.F[(int64_t)j * a.k + l0 + threadIdx.x];
    __syncthreads();
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
      double y = (l0 == 0) ? aload<AT>(a.A, a.lda, i, c0) : a.V[i * a.k + j];
      for (int l = 0; l < nl; ++l) y = fma(-a.V[i * a.k + l0 + l], fj[l], y);
      if (l0 + 64 >= j) {  // last chunk: final value
        y = (i >= j) ? y : 0.0;
        if (i >= j) s = fma(y, y, s);
      }
      a.V[i * a.k + j] = y;
    }
  }
  s = block_sum(s, sm);
  if (threadIdx.x == 0) a.part[blockIdx.x] = s;
  if (!last_block(a.counter, gridDim.x)) return;
  if (threadIdx.x == 0) {
    double a2 = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) a2 += __ldcg(a.part + b);
    const double alpha = sqrt(a2);
    const double x0 = __ldcg(a.V + (int64_t)j * a.k + j);
    double tau = 0.0, beta = 0.0;
    if (alpha > 0.0) {
      const double sg = (x0 < 0.0) ? -1.0 : 1.0;
      const double v0 = x0 + sg * alpha;
      a.V[(int64_t)j * a.k + j] = v0;
      tau = 2.0 / (2.0 * alpha * (alpha + fabs(x0)));
      beta = -sg * alpha;
    }
    a.scal[0] = tau;
    a.scal[1] = beta;
    if (a.rdiag) a.rdiag[j] = beta;
    if (a.piv) a.piv[j] = (int64_t)a.perm[j];
    *a.counter = 0u;
  }
}

// ---- kernel B: A^T v_j and V^T v_j partials; last block finishes step j
template <typename AT>
__global__ void __launch_bounds__(kQThreads) qrp_gemv_kernel(QrpArgs a, int j) {
  __shared__ double sm[kQThreads];
  const int cl = threadIdx.x & (kQCols - 1), rl = threadIdx.x / kQCols;
  constexpr int RL = kQThreads / kQCols;
  const int64_t c = (int64_t)blockIdx.x * kQCols + cl;
  const int64_t rows_per = (a.m + gridDim.y - 1) / gridDim.y;
  const int64_t r0 = max((int64_t)j, (int64_t)blockIdx.y * rows_per);
  const int64_t r1 = min(a.m, (int64_t)blockIdx.y * rows_per + rows_per);
  double s = 0.0;
  if (c < a.n)
    for (int64_t i = r0 + rl; i < r1; i += RL) s = fma(aload<AT>(a.A, a.lda, i, c), __ldcg(a.V + i * a.k + j), s);
  sm[threadIdx.x] = s;
  __syncthreads();
  if (rl == 0 && c < a.n) {
    double t = 0.0;
#pragma unroll
    for (int q = 0; q < RL; ++q) t += sm[q * kQCols + cl];
    a.part[(int64_t)blockIdx.y * a.part_ld + c] = t;
  }
  __syncthreads();  // sm is reused below
  // V^T v_j over this row chunk (column chunk 0 only)
  if (blockIdx.x == 0) {
    for (int l = 0; l < j; ++l) {
      double t = 0.0;
      for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x)
        t = fma(__ldcg(a.V + i * a.k + l), __ldcg(a.V + i * a.k + j), t);
      t = block_sum(t, sm);
      if (threadIdx.x == 0) a.part[(int64_t)blockIdx.y * a.part_ld + a.n + l] = t;
    }
  }
  if (!last_block(a.counter, gridDim.x * gridDim.y)) return;

  const int nrc = gridDim.y;
  const double tau = a.scal[0];
  const int k = a.k;
  __shared__ double u[64];
  __shared__ int nflag;
  if (threadIdx.x == 0) nflag = 0;
  // u_l = (V^T v_j)_l, l < j   (j < 64 is enforced by the host)
  for (int l = threadIdx.x; l < j; l += blockDim.x) {
    double t = 0.0;
    for (int b = 0; b < nrc; ++b) t += __ldcg(a.part + (int64_t)b * a.part_ld + a.n + l);
    u[l] = t;
  }
  __syncthreads();
  // T(0:j, j) = -tau T(0:j, 0:j) u(0:j), T(j, j) = tau
  for (int l = threadIdx.x; l < j; l += blockDim.x) {
    double t = 0.0;
    for (int q = l; q < j; ++q) t = fma(a.T[(int64_t)l * k + q], u[q], t);
    a.T[(int64_t)l * k + j] = -tau * t;
  }
  if (threadIdx.x == 0) a.T[(int64_t)j * k + j] = tau;
  const double tol = sqrt(DBL_EPSILON);
  for (int64_t cc = j + 1 + threadIdx.x; cc < a.n; cc += blockDim.x) {
    const int oc = a.perm[cc];
    double w = 0.0;
    for (int b = 0; b < nrc; ++b) w += __ldcg(a.part + (int64_t)b * a.part_ld + oc);
    double corr = 0.0;
    for (int l = 0; l < j; ++l) corr = fma(a.F[cc * k + l], u[l], corr);
    const double f = tau * (w - corr);
    a.F[cc * k + j] = f;
    double r = aload<AT>(a.A, a.lda, j, oc);
    for (int l = 0; l <= j; ++l) r = fma(-__ldcg(a.V + (int64_t)j * k + l), a.F[cc * k + l], r);
    double nv = a.vn[cc] - r * r;
    const double ref = a.vref[cc];
    if (ref > 0.0 && !(nv > tol * ref)) {  // cancellation: recompute exactly (kernel R)
      a.flag[cc] = 1;
      atomicAdd(&nflag, 1);
      nv = 0.0;
    } else if (!(nv > 0.0)) {
      nv = 0.0;  // an exactly zero column stays zero
    }
    a.vn[cc] = nv;
  }
  for (int64_t cc = threadIdx.x; cc <= j && cc < a.n; cc += blockDim.x) a.F[cc * k + j] = 0.0;
  __syncthreads();
  if (threadIdx.x == 0) a.iscal[1] = nflag;
  __syncthreads();
  if (nflag == 0 && j + 1 < k) choose_and_swap(a, j + 1);
  if (threadIdx.x == 0) *a.counter = 0u;
}

// ---- kernel R: exact norms of flagged columns (rare), then the pivot choice
template <typename AT>
__global__ void __launch_bounds__(kQThreads) qrp_renorm_kernel(QrpArgs a, int j) {
  if (a.iscal[1] == 0) return;  // uniform across the grid: written before this launch
  __shared__ double sm[kQThreads];
  const int64_t rows_per = (a.m + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = max((int64_t)j + 1, (int64_t)blockIdx.x * rows_per);
  const int64_t r1 = min(a.m, (int64_t)blockIdx.x * rows_per + rows_per);
  const int k = a.k;
  for (int64_t cc = j + 1; cc < a.n; ++cc) {
    if (!a.flag[cc]) continue;
    const int oc = a.perm[cc];
    double s = 0.0;
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
      double y = aload<AT>(a.A, a.lda, i, oc);
      for (int l = 0; l <= j; ++l) y = fma(-a.V[i * k + l], a.F[cc * k + l], y);
      s = fma(y, y, s);
    }
    s = block_sum(s, sm);
    if (threadIdx.x == 0) a.part[(int64_t)blockIdx.x * a.part_ld + cc] = s;
  }
  if (!last_block(a.counter, gridDim.x)) return;
  for (int64_t cc = j + 1 + threadIdx.x; cc < a.n; cc += blockDim.x) {
    if (!a.flag[cc]) continue;
    double t = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) t += __ldcg(a.part + (int64_t)b * a.part_ld + cc);
    a.vn[cc] = t;
    a.vref[cc] = t;
    a.flag[cc] = 0;
  }
  __syncthreads();
  if (threadIdx.x == 0) a.iscal[1] = 0;
  if (j + 1 < a.k) choose_and_swap(a, j + 1);
  if (threadIdx.x == 0) *a.counter = 0u;
}

// ---- Q = [I_k; 0] - V (T V[0:k, :]^T)
__global__ void qrp_m_kernel(QrpArgs a) {
  const int k = a.k;
  for (int q = threadIdx.x; q < k * k; q += blockDim.x) {
    const int l = q / k, cc = q % k;  // M[l, cc] = sum_p T[l, p] V[cc, p]  (p >= l, p <= cc)
    double t = 0.0;
    for (int p = l; p <= min(cc, k - 1); ++p) t = fma(a.T[(int64_t)l * k + p], a.V[(int64_t)cc * k + p], t);
    a.M[q] = t;
  }
}

__global__ void qrp_q_kernel(QrpArgs a, double *Q, int64_t ldq) {
  const int k = a.k;
  extern __shared__ double Ms[];
  for (int q = threadIdx.x; q < k * k; q += blockDim.x) Ms[q] = a.M[q];
  __syncthreads();
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < a.m * k;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / k;
    const int cc = (int)(idx % k);
    double t = (i == cc) ? 1.0 : 0.0;
    const int lmax = (int)min((int64_t)k - 1, i);  // V[i, l] = 0 for l > i
    for (int l = 0; l <= lmax; ++l) t = fma(-a.V[i * k + l], Ms[l * k + cc], t);
    Q[i * ldq + cc] = t;
  }
}

// ============================================================================ persistent form
// One cooperative launch runs all k steps.  Blocks own a contiguous range of rows for
// the row-parallel phases and a strided set of column positions for the column
// phases; two grid barriers separate the phases of a step:
//   A  rows of the updated pivot column y -> V[:, j], partial ||y||^2, then, on the
//      same rows, partial A^T y (all columns) and V^T y                 | barrier
//      every block forms tau, beta, v_jj from the same partials (identical values);
//      v_j differs from y only in row j, so A^T v_j = A^T y + (v_jj - y_jj) A[j, :]
//   C  per column: F[c, j], R[j, c], norm downdate (warp per column)   | barrier
//      [rare: exact recomputation of cancelled norms, two more barriers]
//      every block picks the next pivot from the same norms and swaps it in its own
//      shared-memory copy of the column order, so the swap needs no barrier.
// F, vn, vref and flag are indexed by original column, so nothing global is swapped.
// For FP32 input, A^T v accumulates exact FP32 products (a * v_hi split by FMA) in a
// double-float pair (TwoSum), flushed to FP64 every 256 rows; FP64 input uses DFMA.
// Data written by other blocks during the launch is read with ld.global.cg (L2).
// Every barrier wait is bounded; on a timeout the kernel records kErrTimeout, fills
// rdiag with NaN and returns.
constexpr int kPThreads = 512;
constexpr int kPWarps = kPThreads / 32;
constexpr int kPStage = 2048;  // rows of v staged in shared memory at a time
constexpr unsigned long long kSpinLimit = 1ull << 25;

struct PArgs {
  const void *A;
  int64_t m, n, lda;
  int k;
  double *V, *F, *part, *vn, *vref, *T, *Q;
  double *scal;  // [0]: y_jj of the current step, written by the block owning row j
  int64_t ldq;
  int *flag, *nflag;
  unsigned *bar;   // [0] arrivals, [1] generation, [2] abort flag (cleared per call)
  uint32_t *err;   // where a timeout is reported (the context's or the call's error word)
  int64_t *piv;
  double *rdiag;
  int64_t part_ld;
};

__device__ __forceinline__ bool grid_sync(const PArgs &a) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned *gen = a.bar + 1;
    const unsigned g0 = *gen;
    __threadfence();
    const unsigned t = atomicAdd(a.bar, 1u);
    if (t == gridDim.x - 1u) {
      atomicExch(a.bar, 0u);
      __threadfence();
      atomicAdd(a.bar + 1, 1u);
    } else {
      unsigned long long spins = 0;
      while (*gen == g0) {
        if (++spins > kSpinLimit) {
          atomicOr(a.bar + 2, 1u);
          atomicOr(a.err, kErrTimeout);
          break;
        }
        if ((spins & 1023u) == 0u && *(volatile unsigned *)(a.bar + 2)) break;  // another block gave up
        __nanosleep(64);
      }
    }
    __threadfence();
    ok = *(volatile unsigned *)(a.bar + 2) == 0u;
  }
  __syncthreads();
  return ok != 0;
}

__device__ __forceinline__ void timeout_exit(const PArgs &a) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const double qnan = __longlong_as_double(0x7ff8000000000000ll);
    if (a.rdiag)
      for (int j = 0; j < a.k; ++j) a.rdiag[j] = qnan;
    if (a.piv)
      for (int j = 0; j < a.k; ++j) a.piv[j] = -1;
    a.Q[0] = qnan;  // a factor with a NaN makes the failure visible downstream
  }
}

__device__ __forceinline__ double block_sum_p(double v, double *red) {
  red[threadIdx.x] = v;
  __syncthreads();
  for (int o = kPThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  const double r = red[0];
  __syncthreads();
  return r;
}

// Row-split, column-parallel reduction of sum_i f(A[i, c]) * v_i over this block's rows
// [r0, r1) for every column c; results to part[b * ld + c].  v_i (FP64) comes from
// vfun(i); with FP32 A it is split into hi/lo floats and accumulated in double-float.
template <typename AT, bool SQUARE, typename VF>
__device__ void colsum_rows(const PArgs &a, int64_t r0, int64_t r1, VF vfun, double *red, void *stage) {
  const int64_t n = a.n;
  int cw = 32;
  while (cw < n && cw < kPThreads) cw <<= 1;
  const int nrl = kPThreads / cw, cl = threadIdx.x % cw, rl = threadIdx.x / cw;
  for (int64_t c0 = 0; c0 < n; c0 += cw) {
    const int64_t c = c0 + cl;
    double acc = 0.0;
    for (int64_t s0 = r0; s0 < r1; s0 += kPStage) {
      const int64_t s1 = min(r1, s0 + kPStage);
      if (!SQUARE) {  // stage v for rows [s0, s1)
        __syncthreads();
        for (int64_t i = s0 + threadIdx.x; i < s1; i += kPThreads) {
          const double v = vfun(i);
          if constexpr (sizeof(AT) == 4) {
            const float h = (float)v;
            reinterpret_cast<float2 *>(stage)[i - s0] = make_float2(h, (float)(v - (double)h));
          } else {
            reinterpret_cast<double *>(stage)[i - s0] = v;
          }
        }
        __syncthreads();
      }
      if (c < n) {
        if constexpr (sizeof(AT) == 4) {
          const float *A = static_cast<const float *>(a.A);
          for (int64_t q0 = s0 + rl; q0 < s1; q0 += (int64_t)nrl * 256) {
            DF d;
            const int64_t q1 = min(s1, q0 + (int64_t)nrl * 256);
            for (int64_t i = q0; i < q1; i += nrl) {
              const float x = __ldg(A + i * a.lda + c);
              if (SQUARE) {
                df_fma(d, x, x, 0.f);
              } else {
                const float2 vv = reinterpret_cast<const float2 *>(stage)[i - s0];
                df_fma(d, x, vv.x, vv.y);
              }
            }
            acc += (double)d.hi + (double)d.lo;
          }
        } else {
          const double *A = static_cast<const double *>(a.A);
          for (int64_t i = s0 + rl; i < s1; i += nrl) {
            const double x = __ldg(A + i * a.lda + c);
            acc = fma(x, SQUARE ? x : reinterpret_cast<const double *>(stage)[i - s0], acc);
          }
        }
      }
    }
    __syncthreads();
    red[threadIdx.x] = acc;
    __syncthreads();
    if (rl == 0 && c < n) {
      double t = 0.0;
      for (int q = 0; q < nrl; ++q) t += red[q * cw + cl];
      a.part[(int64_t)blockIdx.x * a.part_ld + c] = t;
    }
  }
  __syncthreads();
}

// FP32 A with n % 4 == 0 and lda % 4 == 0: each thread owns four adjacent columns (one
// float4 per row) and issues 8 rows of loads before using them, so that enough bytes
// are in flight per SM to stream A at memory speed; four independent double-float
// accumulators per thread.  Same results layout as colsum_rows.
template <bool SQUARE, typename VF>
__device__ void colsum_rows_f32x4(const PArgs &a, int64_t r0, int64_t r1, VF vfun, double *red4, float2 *stage) {
  const int64_t nq = a.n / 4, ld4 = a.lda / 4;
  int cw = 8;
  while (cw < nq && cw < kPThreads) cw <<= 1;
  const int nrl = kPThreads / cw, cq = threadIdx.x % cw, rl = threadIdx.x / cw;
  const float4 *A4 = static_cast<const float4 *>(a.A);
  for (int64_t q0 = 0; q0 < nq; q0 += cw) {
    const int64_t qc = q0 + cq;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t s0 = r0; s0 < r1; s0 += kPStage) {
      const int64_t s1 = min(r1, s0 + kPStage);
      if (!SQUARE) {
        __syncthreads();
        for (int64_t i = s0 + threadIdx.x; i < s1; i += kPThreads) {
          const double v = vfun(i);
          const float h = (float)v;
          stage[i - s0] = make_float2(h, (float)(v - (double)h));
        }
        __syncthreads();
      }
      if (qc < nq) {
        const float4 *col = A4 + s0 * ld4 + qc;
        const int cnt = (int)(s1 - s0);
        for (int c0 = rl; c0 < cnt; c0 += nrl * 256) {  // flush the double-float pairs every 256 rows
          DF d0, d1, d2, d3;
          const int c1 = min(cnt, c0 + nrl * 256);
          int ii = c0;
          for (; ii + 7 * nrl < c1; ii += 8 * nrl) {
            float4 x[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) x[u] = __ldg(col + (int64_t)(ii + u * nrl) * ld4);
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              if (SQUARE) {
                df_fma(d0, x[u].x, x[u].x, 0.f);
                df_fma(d1, x[u].y, x[u].y, 0.f);
                df_fma(d2, x[u].z, x[u].z, 0.f);
                df_fma(d3, x[u].w, x[u].w, 0.f);
              } else {
                const float2 vv = stage[ii + u * nrl];
                df_fma(d0, x[u].x, vv.x, vv.y);
                df_fma(d1, x[u].y, vv.x, vv.y);
                df_fma(d2, x[u].z, vv.x, vv.y);
                df_fma(d3, x[u].w, vv.x, vv.y);
              }
            }
          }
          for (; ii < c1; ii += nrl) {
            const float4 x = __ldg(col + (int64_t)ii * ld4);
            const float2 vv = SQUARE ? make_float2(0.f, 0.f) : stage[ii];
            df_fma(d0, x.x, SQUARE ? x.x : vv.x, vv.y);
            df_fma(d1, x.y, SQUARE ? x.y : vv.x, vv.y);
            df_fma(d2, x.z, SQUARE ? x.z : vv.x, vv.y);
            df_fma(d3, x.w, SQUARE ? x.w : vv.x, vv.y);
          }
          acc[0] += (double)d0.hi + (double)d0.lo;
          acc[1] += (double)d1.hi + (double)d1.lo;
          acc[2] += (double)d2.hi + (double)d2.lo;
          acc[3] += (double)d3.hi + (double)d3.lo;
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) red4[q * kPThreads + threadIdx.x] = acc[q];
    __syncthreads();
    if (rl == 0 && qc < nq) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        double t = 0.0;
        for (int r = 0; r < nrl; ++r) t += red4[q * kPThreads + r * cw + cq];
        a.part[(int64_t)blockIdx.x * a.part_ld + 4 * qc + q] = t;
      }
    }
  }
  __syncthreads();
}

// sum over blocks of part[b * ld + col] by one warp (fixed order: lane-strided, then tree)
__device__ __forceinline__ double warp_part_sum(const PArgs &a, int64_t col) {
  const int lane = threadIdx.x & 31;
  double t = 0.0;
#pragma unroll 4
  for (int bb = lane; bb < (int)gridDim.x; bb += 32) t += __ldcg(a.part + (int64_t)bb * a.part_ld + col);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  return t;
}

template <typename AT>
__device__ __forceinline__ double aval(const PArgs &a, int64_t i, int64_t c) {
  return (double)__ldg(static_cast<const AT *>(a.A) + i * a.lda + c);
}

// argmax of vn over positions [j0, n) in this block's column order (lowest position on
// ties); swaps it into position j0 of perm_s.  Identical in every block.  Warp-level
// (value, position) reductions; wred / wredi hold one entry per warp.
__device__ void pick_pivot(const PArgs &a, int *perm_s, int j0, double *wred, int *wredi) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double best = -1.0;
  int bi = INT_MAX;
  for (int64_t pos = j0 + threadIdx.x; pos < a.n; pos += kPThreads) {
    const double v = __ldcg(a.vn + perm_s[pos]);
    if (v > best) {
      best = v;
      bi = (int)pos;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double v2 = __shfl_xor_sync(0xffffffffu, best, o);
    const int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
    if (v2 > best || (v2 == best && i2 < bi)) {
      best = v2;
      bi = i2;
    }
  }
  if (lane == 0) {
    wred[warp] = best;
    wredi[warp] = bi;
  }
  __syncthreads();
  if (warp == 0) {
    best = lane < kPWarps ? wred[lane] : -1.0;
    bi = lane < kPWarps ? wredi[lane] : INT_MAX;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double v2 = __shfl_xor_sync(0xffffffffu, best, o);
      const int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
      if (v2 > best || (v2 == best && i2 < bi)) {
        best = v2;
        bi = i2;
      }
    }
    if (lane == 0 && bi != j0 && bi < a.n) {
      const int t = perm_s[j0];
      perm_s[j0] = perm_s[bi];
      perm_s[bi] = t;
    }
  }
  __syncthreads();
}

// block sum through warp shuffles (fixed order); result in every thread
__device__ __forceinline__ double block_sum_w(double v, double *wred) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) wred[warp] = v;
  __syncthreads();
  double t = 0.0;
#pragma unroll
  for (int w = 0; w < kPWarps; ++w) t += wred[w];
  return t;
}

template <typename AT>
__global__ void __launch_bounds__(kPThreads) qrp_persistent_kernel(PArgs a) {
  extern __shared__ __align__(16) unsigned char psm[];
  __shared__ double red[kPThreads];
  __shared__ double red4[4 * kPThreads];
  __shared__ double wred[kPWarps];
  __shared__ int wredi[kPWarps];
  __shared__ double s_wp[kPWarps][64];  // per-warp partials of V^T y
  __shared__ double s_u[64];
  __shared__ double s_f[64];
  __shared__ double s_vj[64];
  __shared__ double s_v0, s_tau, s_dv;
  __shared__ int s_nflag;
  const int64_t n = a.n, m = a.m;
  const int k = a.k;
  int *perm_s = reinterpret_cast<int *>(psm);
  void *stage = psm + ((n * sizeof(int) + 15) & ~(size_t)15);
  const size_t stage_bytes = max((size_t)kPStage * 8, (size_t)k * k * sizeof(double));
  double *Ts = reinterpret_cast<double *>(static_cast<unsigned char *>(stage) +
                                          ((stage_bytes + 15) & ~(size_t)15));  // k x k, this block's T
  const int nb = gridDim.x, b = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t rows_per = (m + nb - 1) / nb;
  const int64_t r0 = min(m, (int64_t)b * rows_per), r1 = min(m, r0 + rows_per);
  const int64_t ld = a.part_ld;
  const int64_t gw = (int64_t)b * kPWarps + warp, nw = (int64_t)nb * kPWarps;
  const bool vec4 = sizeof(AT) == 4 && (n % 4) == 0 && (a.lda % 4) == 0 &&
                    (reinterpret_cast<uintptr_t>(a.A) % 16) == 0;

  // ---- initial column norms
  if (vec4)
    colsum_rows_f32x4<true>(a, r0, r1, [](int64_t) { return 0.0; }, red4, static_cast<float2 *>(stage));
  else
    colsum_rows<AT, true>(a, r0, r1, [](int64_t) { return 0.0; }, red, stage);
  for (int64_t c = threadIdx.x; c < n; c += kPThreads) perm_s[c] = (int)c;
  for (int q = threadIdx.x; q < k * k; q += kPThreads) Ts[q] = 0.0;
  if (b == 0)  // per-step counts of recomputed norms; stepped into only after later barriers
    for (int q = threadIdx.x; q < k; q += kPThreads) a.nflag[q] = 0;
  if (!grid_sync(a)) return timeout_exit(a);
  for (int64_t c = gw; c < n; c += nw) {
    const double t = warp_part_sum(a, c);
    if (lane == 0) {
      a.vn[c] = t;
      a.vref[c] = t;
      a.flag[c] = 0;
    }
  }
  if (!grid_sync(a)) return timeout_exit(a);
  pick_pivot(a, perm_s, 0, wred, wredi);

  const double tol = sqrt(DBL_EPSILON);
  for (int j = 0; j < k; ++j) {
    const int c0 = perm_s[j];
    // ---- A: pivot column rows y = A[:, c0] - V[:, :j] F[c0, :j]; partials of ||y||^2
    //      and of V^T y over rows > j (row j enters once v_jj is known)
    if (threadIdx.x < j) s_f[threadIdx.x] = __ldcg(a.F + (int64_t)c0 * k + threadIdx.x);
    __syncthreads();
    double s2 = 0.0;
    double pl[16];  // V[i, l] * y_i for l < min(j, 16), summed over this thread's rows
#pragma unroll
    for (int q = 0; q < 16; ++q) pl[q] = 0.0;
    for (int64_t i = r0 + threadIdx.x; i < r1; i += kPThreads) {
      double y = aval<AT>(a, i, c0);
      const double *vrow = a.V + i * k;
      if ((k & 1) == 0) {  // rows are 16-byte aligned: independent double2 loads
        const double2 *v2 = reinterpret_cast<const double2 *>(vrow);
        for (int l0 = 0; l0 < j; l0 += 16) {
          double2 buf[8];
#pragma unroll
          for (int q = 0; q < 8; ++q)
            if (l0 + 2 * q < j) buf[q] = __ldcg(v2 + (l0 >> 1) + q);
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            if (l0 + 2 * q < j) y = fma(-buf[q].x, s_f[l0 + 2 * q], y);
            if (l0 + 2 * q + 1 < j) y = fma(-buf[q].y, s_f[l0 + 2 * q + 1], y);
          }
        }
      } else {
#pragma unroll 8
        for (int l = 0; l < j; ++l) y = fma(-__ldcg(vrow + l), s_f[l], y);
      }
      y = (i >= j) ? y : 0.0;
      s2 = fma(y, y, s2);
      a.V[i * k + j] = y;
      if (i == j) a.scal[0] = y;  // x0 of the reflector, read by every block after the barrier
      if (i > j) {  // second pass over the (L1-resident) row: V[i, l] y_i for l < 16
        if ((k & 1) == 0) {
          const double2 *v2 = reinterpret_cast<const double2 *>(vrow);
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            if (2 * q < j) {
              const double2 v = __ldcg(v2 + q);
              pl[2 * q] = fma(v.x, y, pl[2 * q]);
              if (2 * q + 1 < j) pl[2 * q + 1] = fma(v.y, y, pl[2 * q + 1]);
            }
          }
        } else {
#pragma unroll
          for (int q = 0; q < 16; ++q)
            if (q < j) pl[q] = fma(__ldcg(vrow + q), y, pl[q]);
        }
      }
    }
    // ||y||^2 partial and V^T y partials (l < 16 from registers; l >= 16 reloaded)
    {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        if (q < j) {
          double t = pl[q];
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
          if (lane == 0) s_wp[warp][q] = t;
        }
      }
      for (int l = 16; l < j; ++l) {  // same rows as above: each thread reads the y it wrote
        double t = 0.0;
        for (int64_t i = r0 + threadIdx.x; i < r1; i += kPThreads)
          if (i > j) t = fma(__ldcg(a.V + i * k + l), __ldcg(a.V + i * k + j), t);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) s_wp[warp][l] = t;
      }
      if (lane == 0) wred[warp] = s2;
      __syncthreads();
      if (threadIdx.x < j || threadIdx.x == 63) {
        const int l = threadIdx.x;
        double t = 0.0;
        if (l == 63) {
          for (int w2 = 0; w2 < kPWarps; ++w2) t += wred[w2];
          a.part[(int64_t)b * ld + n + k] = t;
        } else {
          for (int w2 = 0; w2 < kPWarps; ++w2) t += s_wp[w2][l];
          a.part[(int64_t)b * ld + n + l] = t;
        }
      }
    }
    // ---- A^T y over this block's rows >= j (no barrier: v_j differs from y only in row j,
    //      whose term is added after the barrier as (v_jj - y_jj) A[j, :])
    {
      __syncthreads();  // this block's y rows (written above) are read back by the staging
      const int64_t rb0 = max(r0, (int64_t)j);
      auto yfun = [&](int64_t i) { return __ldcg(a.V + i * k + j); };
      if (vec4)
        colsum_rows_f32x4<false>(a, rb0, max(rb0, r1), yfun, red4, static_cast<float2 *>(stage));
      else
        colsum_rows<AT, false>(a, rb0, max(rb0, r1), yfun, red, stage);
    }
    if (!grid_sync(a)) return timeout_exit(a);
    // ---- reflector scalars, identically in every block (one warp)
    if (warp == 0) {
      const double x0 = __ldcg(a.scal);
      double t = 0.0;
#pragma unroll 4
      for (int bb = lane; bb < nb; bb += 32) t += __ldcg(a.part + (int64_t)bb * ld + n + k);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (lane == 0) {
        const double alpha = sqrt(t);
        double tau = 0.0, beta = 0.0, v0 = 0.0;
        if (alpha > 0.0) {
          const double sg = (x0 < 0.0) ? -1.0 : 1.0;
          v0 = x0 + sg * alpha;
          tau = 2.0 / (2.0 * alpha * (alpha + fabs(x0)));
          beta = -sg * alpha;
        }
        s_v0 = v0;
        s_tau = tau;
        s_dv = v0 - x0;
        if (b == 0) {
          if (a.rdiag) a.rdiag[j] = beta;
          if (a.piv) a.piv[j] = c0;
        }
      }
    }
    __syncthreads();
    const double v0 = s_v0, tau = s_tau, dv = s_dv;
    // ---- C: u = V^T v_j, this block's T, then F[:, j], row j of R, norm downdate
    // Row j of V gets v_jj only now: every block read x0 from it between the first two
    // barriers of this step, and until then only its owner used v_jj (from s_v0).
    if (threadIdx.x == 0 && j >= r0 && j < r1) a.V[(int64_t)j * k + j] = v0;
    {
      const double vj = (threadIdx.x < j) ? __ldcg(a.V + (int64_t)j * k + threadIdx.x) : 0.0;
      for (int l = warp; l < j; l += kPWarps) {
        const double t = warp_part_sum(a, n + l);
        if (lane == 0) s_u[l] = t;
      }
      if (threadIdx.x < j) s_vj[threadIdx.x] = vj;
      __syncthreads();
      if (threadIdx.x < j) s_u[threadIdx.x] = fma(s_vj[threadIdx.x], v0, s_u[threadIdx.x]);  // + V[j, l] v_jj
      __syncthreads();
      // T(0:j, j) = -tau T(0:j, 0:j) u, T(j, j) = tau
      if (threadIdx.x < j) {
        const int l = threadIdx.x;
        double t = 0.0;
        for (int q = l; q < j; ++q) t = fma(Ts[l * k + q], s_u[q], t);
        Ts[l * k + j] = -tau * t;
      }
      if (threadIdx.x == 0) Ts[j * k + j] = tau;
    }
    for (int64_t pos = j + 1 + gw; pos < n; pos += nw) {
      const int c = perm_s[pos];
      const double *frow = a.F + (int64_t)c * k;
      // every load of this column first (one round trip), then the arithmetic
      const double f0 = (lane < j) ? __ldcg(frow + lane) : 0.0;
      const double f1 = (lane + 32 < j) ? __ldcg(frow + lane + 32) : 0.0;
      const double ajc = aval<AT>(a, j, c);
      const double vnc = __ldcg(a.vn + c), ref = __ldcg(a.vref + c);
      const double w = fma(dv, ajc, warp_part_sum(a, c));  // A^T v = A^T y + (v_jj - y_jj) A[j, :]
      double corr = 0.0, rv = 0.0;
      if (lane < j) {
        corr = f0 * s_u[lane];
        rv = s_vj[lane] * f0;
      }
      if (lane + 32 < j) {
        corr = fma(f1, s_u[lane + 32], corr);
        rv = fma(s_vj[lane + 32], f1, rv);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        corr += __shfl_xor_sync(0xffffffffu, corr, o);
        rv += __shfl_xor_sync(0xffffffffu, rv, o);
      }
      if (lane == 0) {
        const double f = tau * (w - corr);
        a.F[(int64_t)c * k + j] = f;
        double r = ajc - rv;
        r = fma(-v0, f, r);
        double nv = vnc - r * r;
        if (ref > 0.0 && !(nv > tol * ref)) {
          a.flag[c] = 1;
          atomicAdd(a.nflag + j, 1);
          nv = 0.0;
        } else if (!(nv > 0.0)) {
          nv = 0.0;
        }
        a.vn[c] = nv;
      }
    }
    if (!grid_sync(a)) return timeout_exit(a);
    if (threadIdx.x == 0) s_nflag = *(volatile int *)(a.nflag + j);
    __syncthreads();
    if (s_nflag > 0) {  // exact recomputation of cancelled norms (uniform decision)
      const int64_t rr0 = max(r0, (int64_t)j + 1);
      for (int64_t pos = j + 1; pos < n; ++pos) {
        const int c = perm_s[pos];
        if (!__ldcg(a.flag + c)) continue;
        double t = 0.0;
        for (int64_t i = rr0 + threadIdx.x; i < r1; i += kPThreads) {
          double y = aval<AT>(a, i, c);
          for (int l = 0; l <= j; ++l) y = fma(-__ldcg(a.V + i * k + l), __ldcg(a.F + (int64_t)c * k + l), y);
          t = fma(y, y, t);
        }
        t = block_sum_w(t, wred);
        if (threadIdx.x == 0) a.part[(int64_t)b * ld + c] = t;
      }
      if (!grid_sync(a)) return timeout_exit(a);
      for (int64_t pos = j + 1 + gw; pos < n; pos += nw) {
        const int c = perm_s[pos];
        if (!__ldcg(a.flag + c)) continue;
        const double t = warp_part_sum(a, c);
        if (lane == 0) {
          a.vn[c] = t;
          a.vref[c] = t;
          a.flag[c] = 0;
        }
      }
      if (!grid_sync(a)) return timeout_exit(a);
    }
    if (j + 1 < k) pick_pivot(a, perm_s, j + 1, wred, wredi);
  }

  // ---- Q = [I_k; 0] - V (T V[0:k, :]^T), rows of this block (T from this block's copy)
  double *Ms = reinterpret_cast<double *>(stage);
  __syncthreads();
  for (int q = threadIdx.x; q < k * k; q += kPThreads) {
    const int l = q / k, cc = q % k;
    double t = 0.0;
    for (int p = l; p <= cc; ++p) t = fma(Ts[l * k + p], __ldcg(a.V + (int64_t)cc * k + p), t);
    Ms[q] = t;
  }
  __syncthreads();
  for (int64_t idx = r0 * k + threadIdx.x; idx < r1 * k; idx += kPThreads) {
    const int64_t i = idx / k;
    const int cc = (int)(idx % k);
    double t = (i == cc) ? 1.0 : 0.0;
    const int lmax = (int)min((int64_t)k - 1, i);
    for (int l = 0; l <= lmax; ++l) t = fma(-__ldcg(a.V + i * k + l), Ms[l * k + cc], t);
    a.Q[i * a.ldq + cc] = t;
  }
}

template <typename AT>
static bool qrp_persistent(const AT *A, int64_t m, int64_t n, int64_t lda, int k, double *Q, int64_t ldq,
                           int64_t *piv, double *rdiag, QrpWork *w, int nb_sms, cudaStream_t s, cudaError_t *err) {
  *err = cudaSuccess;
  if (n > 8192 || k > 64) return false;
  int dev = 0, coop = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) return false;
  const size_t perm_bytes = ((size_t)n * sizeof(int) + 15) & ~(size_t)15;
  const size_t stage_bytes = std::max<size_t>((size_t)kPStage * 8, (size_t)k * k * sizeof(double));
  const size_t smem = perm_bytes + ((stage_bytes + 15) & ~(size_t)15) + (size_t)k * k * sizeof(double);
  auto kern = qrp_persistent_kernel<AT>;
  // the 48 KB default bounds static + dynamic shared memory together: always opt in
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return false;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPThreads, smem) != cudaSuccess || per_sm < 1)
    return false;
  int64_t nb = std::min<int64_t>((int64_t)per_sm * nb_sms, (int64_t)nb_sms);
  nb = std::min<int64_t>(nb, std::max<int64_t>(1, (m * std::max<int64_t>(n, 1)) / 8192));
  nb = std::max<int64_t>(1, std::min<int64_t>(nb, m));
  PArgs a{};
  a.A = A;
  a.m = m;
  a.n = n;
  a.lda = lda;
  a.k = k;
  a.V = w->V;
  a.F = w->F;
  a.part = w->part;
  a.vn = w->vn;
  a.vref = w->vref;
  a.T = w->T;
  a.Q = Q;
  a.scal = w->scal;
  a.ldq = ldq;
  a.flag = w->flag;
  a.nflag = w->nflag;
  a.bar = w->bar;
  a.err = w->err_out ? w->err_out : w->bar + 2;
  a.piv = piv;
  a.rdiag = rdiag;
  a.part_ld = n + std::max(k, 1) + 8;
  if ((*err = cudaMemsetAsync(w->bar, 0, 3 * sizeof(unsigned), s)) != cudaSuccess) return true;
  void *args[] = {&a};
  *err = cudaLaunchCooperativeKernel((const void *)kern, dim3((unsigned)nb), dim3(kPThreads), args, smem, s);
  ::tk::count_launch();
  return true;
}

// ============================================================================ wait self-test
// One block polls a flag that nothing sets, with the bounded loop of the grid barrier
// above, and latches kErrTimeout when it gives up.  It exercises the timeout path of the
// library without any real wait going wrong.
__global__ void wait_selftest_kernel(const unsigned *flag, unsigned long long max_polls, uint32_t *err) {
  if (threadIdx.x != 0) return;
  volatile const unsigned *f = flag;
  unsigned long long polls = 0;
  while (*f == 0u) {
    if (++polls > max_polls) {
      atomicOr(err, kErrTimeout);
      return;
    }
    __nanosleep(100);
  }
}

tucker_status launch_wait_selftest(Ctx *c, unsigned long long max_polls, cudaStream_t s) {
  if (!c->qw.V) return TUCKER_ESTATE;
  unsigned *flag = reinterpret_cast<unsigned *>(c->qw.V) + (c->qw.bytes / sizeof(unsigned)) - 1;  // last word
  if (cudaMemsetAsync(flag, 0, sizeof(unsigned), s) != cudaSuccess) return TUCKER_ECUDA;
  wait_selftest_kernel<<<1, 32, 0, s>>>(flag, max_polls, c->d_err);
  ::tk::count_launch();
  return cudaGetLastError() == cudaSuccess ? TUCKER_OK : TUCKER_ECUDA;
}

// ---------------------------------------------------------------------------- host side
int qrp_blocks(int num_sms, int64_t m) {
  int64_t b = std::max<int64_t>(1, std::min<int64_t>((int64_t)num_sms, (m + 31) / 32));
  return (int)b;
}

static int row_chunks_for(int num_blocks_target, int64_t n, int64_t m) {
  const int64_t cchunks = (n + kQCols - 1) / kQCols;
  int64_t rc = std::max<int64_t>(1, num_blocks_target / std::max<int64_t>(cchunks, 1));
  rc = std::min<int64_t>(rc, std::max<int64_t>(1, (m + 15) / 16));
  return (int)rc;
}

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// nb = target number of blocks (typically the SM count)
size_t qrp_work_bytes(int64_t m, int64_t n, int k, int nb) {
  const int rc = row_chunks_for(2 * nb, n, m);
  const int64_t part_rows = std::max<int64_t>(std::max<int64_t>(rc, 2 * (int64_t)nb), 1);
  const int64_t part_ld = n + std::max(k, 1) + 8;
  size_t b = 0;
  b += align256(sizeof(double) * (size_t)std::max<int64_t>(m * k, 1));       // V
  b += align256(sizeof(double) * (size_t)std::max<int64_t>(n * k, 1));       // F
  b += align256(sizeof(double) * (size_t)(part_rows * part_ld));            // part
  b += 2 * align256(sizeof(double) * (size_t)std::max<int64_t>(n, 1));       // vn, vref
  b += 2 * align256(sizeof(int) * (size_t)std::max<int64_t>(n, 1));          // perm, flag
  b += 2 * align256(sizeof(double) * (size_t)std::max(k * k, 1));           // T, M
  b += align256(sizeof(double) * 16) + align256(sizeof(int) * 16) + align256(sizeof(unsigned) * 4);
  b += align256(sizeof(int) * 64) + align256(sizeof(unsigned) * 4);  // nflag, bar
  return b;
}

void qrp_bind_work(QrpWork *w, void *base, int64_t m, int64_t n, int k, int nb) {
  const int rc = row_chunks_for(2 * nb, n, m);
  const int64_t part_rows = std::max<int64_t>(std::max<int64_t>(rc, 2 * (int64_t)nb), 1);
  const int64_t part_ld = n + std::max(k, 1) + 8;
  char *p = static_cast<char *>(base);
  auto take = [&](size_t bytes) {
    char *r = p;
    p += align256(bytes);
    return r;
  };
  w->V = (double *)take(sizeof(double) * (size_t)std::max<int64_t>(m * k, 1));
  w->F = (double *)take(sizeof(double) * (size_t)std::max<int64_t>(n * k, 1));
  w->part = (double *)take(sizeof(double) * (size_t)(part_rows * part_ld));
  w->part_elems = (size_t)(part_rows * part_ld);
  w->vn = (double *)take(sizeof(double) * (size_t)std::max<int64_t>(n, 1));
  w->vref = (double *)take(sizeof(double) * (size_t)std::max<int64_t>(n, 1));
  w->perm = (int *)take(sizeof(int) * (size_t)std::max<int64_t>(n, 1));
  w->flag = (int *)take(sizeof(int) * (size_t)std::max<int64_t>(n, 1));
  w->T = (double *)take(sizeof(double) * (size_t)std::max(k * k, 1));
  w->M = (double *)take(sizeof(double) * (size_t)std::max(k * k, 1));
  w->scal = (double *)take(sizeof(double) * 16);
  w->iscal = (int *)take(sizeof(int) * 16);
  w->counter = (unsigned *)take(sizeof(unsigned) * 4);
  w->nflag = (int *)take(sizeof(int) * 64);
  w->bar = (unsigned *)take(sizeof(unsigned) * 4);
  w->err_out = w->bar + 2;
  w->bytes = (size_t)(p - static_cast<char *>(base));
}

template <typename AT>
static tucker_status qrp_run(const AT *A, int64_t m, int64_t n, int64_t lda, int k, double *Q, int64_t ldq,
                             int64_t *piv, double *rdiag, QrpWork *w, int nb, cudaStream_t s) {
  if (k == 0) return TUCKER_OK;
  if (k > 64) return TUCKER_ERANK;  // F rows are staged in 64-wide shared buffers
  // TUCKER_QRP_FORM=multi runs the multi-kernel form below for every shape (a test and
  // comparison switch); otherwise the single-launch forms are tried first
  const char *form = std::getenv("TUCKER_QRP_FORM");
  if (!(form && std::strcmp(form, "multi") == 0)) {
    cudaError_t e = cudaSuccess;
    if (qrp_cluster<AT>(A, m, n, lda, k, Q, ldq, piv, rdiag, w, s, &e))
      return e == cudaSuccess ? TUCKER_OK : TUCKER_ECUDA;
    if (e != cudaSuccess) return TUCKER_ECUDA;
    if (qrp_persistent<AT>(A, m, n, lda, k, Q, ldq, piv, rdiag, w, nb, s, &e))
      return e == cudaSuccess ? TUCKER_OK : TUCKER_ECUDA;
  }
  QrpArgs a{};
  a.A = A;
  a.m = m;
  a.n = n;
  a.lda = lda;
  a.k = k;
  a.V = w->V;
  a.F = w->F;
  a.part = w->part;
  a.vn = w->vn;
  a.vref = w->vref;
  a.T = w->T;
  a.M = w->M;
  a.scal = w->scal;
  a.perm = w->perm;
  a.flag = w->flag;
  a.iscal = w->iscal;
  a.counter = w->counter;
  a.piv = piv;
  a.rdiag = rdiag;
  a.row_chunks = row_chunks_for(2 * nb, n, m);
  a.part_ld = n + std::max(k, 1) + 8;
  const dim3 g2((unsigned)((n + kQCols - 1) / kQCols), (unsigned)a.row_chunks);
  const int nbA = qrp_blocks(nb, m);
  if (cudaMemsetAsync(w->counter, 0, sizeof(unsigned) * 4, s) != cudaSuccess) return TUCKER_ECUDA;
  if (cudaMemsetAsync(w->F, 0, sizeof(double) * (size_t)(n * k), s) != cudaSuccess) return TUCKER_ECUDA;
  qrp_init_kernel<AT><<<g2, kQThreads, 0, s>>>(a);
  ::tk::count_launch();
  for (int j = 0; j < k; ++j) {
    qrp_col_kernel<AT><<<nbA, kQThreads, 0, s>>>(a, j);
    ::tk::count_launch();
    qrp_gemv_kernel<AT><<<g2, kQThreads, 0, s>>>(a, j);
    ::tk::count_launch();
    qrp_renorm_kernel<AT><<<nbA, kQThreads, 0, s>>>(a, j);
    ::tk::count_launch();
  }
  qrp_m_kernel<<<1, 256, 0, s>>>(a);
  ::tk::count_launch();
  const int64_t qelems = m * k;
  const unsigned qb = (unsigned)std::max<int64_t>(1, std::min<int64_t>((qelems + 255) / 256, (int64_t)nb * 8));
  qrp_q_kernel<<<qb, 256, sizeof(double) * (size_t)k * k, s>>>(a, Q, ldq);
  ::tk::count_launch();
  return cudaGetLastError() == cudaSuccess ? TUCKER_OK : TUCKER_ECUDA;
}

tucker_status qrp_run_f64(const double *A, int64_t m, int64_t n, int64_t lda, int k, double *Q, int64_t ldq,
                          int64_t *piv, double *rdiag, QrpWork *w, int nb, cudaStream_t s) {
  return qrp_run<double>(A, m, n, lda, k, Q, ldq, piv, rdiag, w, nb, s);
}
tucker_status qrp_run_f32(const float *A, int64_t m, int64_t n, int64_t lda, int k, double *Q, int64_t ldq,
                          int64_t *piv, double *rdiag, QrpWork *w, int nb, cudaStream_t s) {
  return qrp_run<float>(A, m, n, lda, k, Q, ldq, piv, rdiag, w, nb, s);
}

// ---- Gram matrix S = Y Y^T (m x m) of an FP32 m x n matrix, FP64 accumulation
// (Section III-D, fat case).  Tiles of 32 x 32 outputs, 8 x 4 per thread... kept simple:
// one thread per output, K staged through shared memory.
__global__ void gram_kernel(const float *Y, int64_t m, int64_t n, double *S) {
  __shared__ float ta[32][33], tb[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
  const int64_t a0 = (int64_t)blockIdx.y * 32, b0 = (int64_t)blockIdx.x * 32;
  double acc[4] = {0, 0, 0, 0};
  for (int64_t c0 = 0; c0 < n; c0 += 32) {
    for (int r = ty; r < 32; r += 8) {
      ta[r][tx] = (a0 + r < m && c0 + tx < n) ? Y[(a0 + r) * n + c0 + tx] : 0.f;
      tb[r][tx] = (b0 + r < m && c0 + tx < n) ? Y[(b0 + r) * n + c0 + tx] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int q = 0; q < 32; ++q) {
      const double bv = (double)tb[tx][q];
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[r] = fma((double)ta[ty + 8 * r][q], bv, acc[r]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int64_t ia = a0 + ty + 8 * r, ib = b0 + tx;
    if (ia < m && ib < m) S[ia * m + ib] = acc[r];
  }
}

void gram_f32(const float *Y, int64_t m, int64_t n, double *S, cudaStream_t s) {
  const dim3 g((unsigned)((m + 31) / 32), (unsigned)((m + 31) / 32));
  gram_kernel<<<g, 256, 0, s>>>(Y, m, n, S);
  ::tk::count_launch();
}

}  // namespace tk
