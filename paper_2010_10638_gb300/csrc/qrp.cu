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
  const int64_t part_rows = std::max<int64_t>(std::max<int64_t>(rc, nb), 1);
  const int64_t part_ld = n + std::max(k, 1) + 8;
  size_t b = 0;
  b += align256(sizeof(double) * (size_t)std::max<int64_t>(m * k, 1));       // V
  b += align256(sizeof(double) * (size_t)std::max<int64_t>(n * k, 1));       // F
  b += align256(sizeof(double) * (size_t)(part_rows * part_ld));            // part
  b += 2 * align256(sizeof(double) * (size_t)std::max<int64_t>(n, 1));       // vn, vref
  b += 2 * align256(sizeof(int) * (size_t)std::max<int64_t>(n, 1));          // perm, flag
  b += 2 * align256(sizeof(double) * (size_t)std::max(k * k, 1));           // T, M
  b += align256(sizeof(double) * 16) + align256(sizeof(int) * 16) + align256(sizeof(unsigned) * 4);
  return b;
}

void qrp_bind_work(QrpWork *w, void *base, int64_t m, int64_t n, int k, int nb) {
  const int rc = row_chunks_for(2 * nb, n, m);
  const int64_t part_rows = std::max<int64_t>(std::max<int64_t>(rc, nb), 1);
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
  w->vn = (double *)take(sizeof(double) * (size_t)std::max<int64_t>(n, 1));
  w->vref = (double *)take(sizeof(double) * (size_t)std::max<int64_t>(n, 1));
  w->perm = (int *)take(sizeof(int) * (size_t)std::max<int64_t>(n, 1));
  w->flag = (int *)take(sizeof(int) * (size_t)std::max<int64_t>(n, 1));
  w->T = (double *)take(sizeof(double) * (size_t)std::max(k * k, 1));
  w->M = (double *)take(sizeof(double) * (size_t)std::max(k * k, 1));
  w->scal = (double *)take(sizeof(double) * 16);
  w->iscal = (int *)take(sizeof(int) * 16);
  w->counter = (unsigned *)take(sizeof(unsigned) * 4);
  w->bytes = (size_t)(p - static_cast<char *>(base));
}

template <typename AT>
static tucker_status qrp_run(const AT *A, int64_t m, int64_t n, int64_t lda, int k, double *Q, int64_t ldq,
                             int64_t *piv, double *rdiag, QrpWork *w, int nb, cudaStream_t s) {
  if (k == 0) return TUCKER_OK;
  if (k > 64) return TUCKER_ERANK;  // F rows are staged in 64-wide shared buffers
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
