/*
 * FP64 CPU oracle for sparse Tucker decomposition by HOOI with QR column pivoting
 * (Jiang, Zhang, Lin, Xing, Zhang, "Sparse Tucker Tensor Decomposition on a Hybrid
 * FPGA-CPU Platform", arXiv 2010.10638).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls this
 * file: only the tests, the smoke check and the bench's CPU-baseline leg use it.  It
 * shares no code, header, table or helper with the CUDA library.
 *
 * Every routine is a plain, slow restatement of the paper's definitions in double
 * precision: loops in the order the paper states them, no blocking, no fusion.
 *
 * Conventions (readings of the paper where it leaves the layout open):
 *   - indices are 0-based; tensors are given in COO form, coords[m*nnz + z] = i_m(z)
 *     (Section III-A, Table I);
 *   - factor U_m is I_m x R_m, row-major (Section III, Tucker model);
 *   - the columns of Y_(n) follow the Kronecker layout of Algorithm 4: the remaining
 *     modes in ascending order, the last one varying fastest;
 *   - the core tensor G is stored C-order [R_1]...[R_N] (last index fastest).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Number of Kronecker rows formed by orc_ttmc since the last reset.  Algorithm 2
 * forms one per nonzero per mode, so a run of T sweeps over an N-way tensor with
 * nnz nonzeros forms T*N*nnz of them (Section IV-C, the PMM tensor: 1,125). */
static int64_t g_kron_rows = 0;

int64_t orc_kron_count(void) { return g_kron_rows; }
void orc_kron_reset(void) { g_kron_rows = 0; }

/* ---------------------------------------------------------------------------
 * Duplicate coalescing.  A COO list may name the same coordinate twice; the
 * tensor it describes holds the sum of those values.  Sort by the full coordinate
 * (mode 0 most significant) and add equal neighbours in FP64.
 * ------------------------------------------------------------------------- */
static int g_cmp_order;
static const uint32_t *g_cmp_coords;
static int64_t g_cmp_nnz;

static int cmp_full_key(const void *pa, const void *pb) {
  int64_t a = *(const int64_t *)pa, b = *(const int64_t *)pb;
  for (int m = 0; m < g_cmp_order; ++m) {
    uint32_t ca = g_cmp_coords[(int64_t)m * g_cmp_nnz + a];
    uint32_t cb = g_cmp_coords[(int64_t)m * g_cmp_nnz + b];
    if (ca != cb) return ca < cb ? -1 : 1;
  }
  return a < b ? -1 : (a > b ? 1 : 0); /* stable: input position breaks ties */
}

/* out_coords holds order*nnz entries, out_vals nnz entries; returns the coalesced
 * count.  Input position order is kept among equal keys, so the FP64 sum of a
 * duplicate group is taken in input order. */
int64_t orc_coalesce(int order, int64_t nnz, const uint32_t *coords, const double *vals,
                     uint32_t *out_coords, double *out_vals) {
  int64_t *perm = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nnz > 0 ? nnz : 1));
  for (int64_t z = 0; z < nnz; ++z) perm[z] = z;
  g_cmp_order = order;
  g_cmp_coords = coords;
  g_cmp_nnz = nnz;
  qsort(perm, (size_t)nnz, sizeof(int64_t), cmp_full_key);
  int64_t out = 0;
  for (int64_t t = 0; t < nnz; ++t) {
    int64_t z = perm[t];
    int same = 0;
    if (out > 0) {
      same = 1;
      for (int m = 0; m < order; ++m)
        if (coords[(int64_t)m * nnz + z] != out_coords[(int64_t)m * nnz + out - 1]) {
          same = 0;
          break;
        }
    }
    if (same) {
      out_vals[out - 1] += vals[z];
    } else {
      for (int m = 0; m < order; ++m) out_coords[(int64_t)m * nnz + out] = coords[(int64_t)m * nnz + z];
      out_vals[out] = vals[z];
      ++out;
    }
  }
  free(perm);
  /* compact the SoA columns from stride nnz to stride out */
  if (out < nnz)
    for (int m = 1; m < order; ++m)
      memmove(out_coords + (int64_t)m * out, out_coords + (int64_t)m * nnz, sizeof(uint32_t) * (size_t)out);
  return out;
}

/* ---------------------------------------------------------------------------
 * Sparse TTMc, Algorithm 2 (inner loop) with the Kronecker row of Algorithm 4 /
 * the mode-1 example of Section III-C:
 *   Y_(n)(i_n, :) += x_z * [ kron_{t != n} U_t(i_t, :) ]   for every nonzero z.
 * The Kronecker row of the remaining modes is grown one mode at a time, ascending,
 * each new factor varying fastest: c[R_b * i + j] = a[i] * b[j].
 * Y is I_n x P_n row-major, P_n = prod_{m != n} R_m; it is overwritten.
 * ------------------------------------------------------------------------- */
void orc_ttmc(int order, const int64_t *dims, const int *ranks, int64_t nnz,
              const uint32_t *coords, const double *vals, int mode,
              const double *const *U, double *Y) {
  int64_t P = 1;
  for (int m = 0; m < order; ++m)
    if (m != mode) P *= ranks[m];
  memset(Y, 0, sizeof(double) * (size_t)(dims[mode] * P));
  double *kr = (double *)malloc(sizeof(double) * (size_t)P);
  double *tmp = (double *)malloc(sizeof(double) * (size_t)P);
  for (int64_t z = 0; z < nnz; ++z) {
    int64_t len = 1;
    kr[0] = 1.0;
    for (int m = 0; m < order; ++m) {
      if (m == mode) continue;
      const double *row = U[m] + (int64_t)coords[(int64_t)m * nnz + z] * ranks[m];
      for (int64_t i = 0; i < len; ++i)
        for (int j = 0; j < ranks[m]; ++j) tmp[(int64_t)ranks[m] * i + j] = kr[i] * row[j];
      len *= ranks[m];
      memcpy(kr, tmp, sizeof(double) * (size_t)len);
    }
    ++g_kron_rows;
    double x = vals[z];
    double *y = Y + (int64_t)coords[(int64_t)mode * nnz + z] * P;
    for (int64_t c = 0; c < P; ++c) y[c] += x * kr[c];
  }
  free(kr);
  free(tmp);
}

/* ---------------------------------------------------------------------------
 * Householder QR with column pivoting, Section III-D:  A P = Q R with
 * |r_11| >= |r_22| >= ...; H_j = I - 2 v v^T / (v^T v), v = a + sign(a_1) ||a|| e_1.
 * Truncated after k reflectors (HOOI only needs the leading R_n columns of Q).
 *
 * A is m x n with row stride lda (row-major).  On return
 *   Q     m x k row-major: Q = H_0 H_1 ... H_{k-1} [I_k; 0]
 *   piv   k original column indices, in the order they were chosen
 *   rdiag k diagonal entries r_jj of R.
 * At every step the column norms of the trailing block A[j:, j:] are recomputed
 * from scratch (no downdating); ties go to the smallest current column index;
 * sign(0) = +1; a zero pivot column gives H_j = I.
 * Returns 0, or -1 for k > min(m, n).
 * ------------------------------------------------------------------------- */
int orc_qrp(const double *A, int64_t m, int64_t n, int64_t lda, int k,
            double *Q, int64_t *piv, double *rdiag) {
  if (k < 0 || k > m || k > n) return -1;
  double *W = (double *)malloc(sizeof(double) * (size_t)(m * n + 1));
  for (int64_t i = 0; i < m; ++i)
    for (int64_t c = 0; c < n; ++c) W[i * n + c] = A[i * lda + c];
  int64_t *perm = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
  for (int64_t c = 0; c < n; ++c) perm[c] = c;
  double *V = (double *)calloc((size_t)(m * (k > 0 ? k : 1)), sizeof(double)); /* reflector j in column j */
  double *vtv = (double *)calloc((size_t)(k > 0 ? k : 1), sizeof(double));
  double *w = (double *)malloc(sizeof(double) * (size_t)(n + 1));

  for (int j = 0; j < k; ++j) {
    /* column norms of the trailing block, exactly */
    int64_t best = j;
    double best_nrm = -1.0;
    for (int64_t c = j; c < n; ++c) {
      double s = 0.0;
      for (int64_t i = j; i < m; ++i) s += W[i * n + c] * W[i * n + c];
      double nrm = sqrt(s);
      if (nrm > best_nrm) {
        best_nrm = nrm;
        best = c;
      }
    }
    /* swap columns j and best */
    if (best != j) {
      for (int64_t i = 0; i < m; ++i) {
        double t = W[i * n + j];
        W[i * n + j] = W[i * n + best];
        W[i * n + best] = t;
      }
      int64_t t = perm[j];
      perm[j] = perm[best];
      perm[best] = t;
    }
    piv[j] = perm[j];
    /* reflector from x = W[j:, j] */
    double alpha = 0.0;
    for (int64_t i = j; i < m; ++i) alpha += W[i * n + j] * W[i * n + j];
    alpha = sqrt(alpha);
    if (alpha == 0.0) { /* H_j = I */
      vtv[j] = 0.0;
      rdiag[j] = 0.0;
      continue;
    }
    double x0 = W[(int64_t)j * n + j];
    double sg = (x0 < 0.0) ? -1.0 : 1.0;
    for (int64_t i = j; i < m; ++i) V[i * k + j] = W[i * n + j];
    V[(int64_t)j * k + j] += sg * alpha;
    double s = 0.0;
    for (int64_t i = j; i < m; ++i) s += V[i * k + j] * V[i * k + j];
    vtv[j] = s;
    /* apply H_j to W[j:, j:]:  W <- W - (2/vtv) v (v^T W) */
    for (int64_t c = j; c < n; ++c) {
      double d = 0.0;
      for (int64_t i = j; i < m; ++i) d += V[i * k + j] * W[i * n + c];
      w[c] = 2.0 * d / s;
    }
    for (int64_t i = j; i < m; ++i)
      for (int64_t c = j; c < n; ++c) W[i * n + c] -= V[i * k + j] * w[c];
    rdiag[j] = W[(int64_t)j * n + j];
  }

  /* Q = H_0 ... H_{k-1} [I_k; 0]: start from the identity block, apply H_{k-1} first */
  for (int64_t i = 0; i < m; ++i)
    for (int c = 0; c < k; ++c) Q[i * k + c] = (i == c) ? 1.0 : 0.0;
  for (int j = k - 1; j >= 0; --j) {
    if (vtv[j] == 0.0) continue;
    for (int c = 0; c < k; ++c) {
      double d = 0.0;
      for (int64_t i = j; i < m; ++i) d += V[i * k + j] * Q[i * k + c];
      double f = 2.0 * d / vtv[j];
      for (int64_t i = j; i < m; ++i) Q[i * k + c] -= V[i * k + j] * f;
    }
  }
  free(W);
  free(perm);
  free(V);
  free(vtv);
  free(w);
  return 0;
}

/* Gram matrix S = Y Y^T (m x m) of an m x n row-major matrix: the square matrix on
 * which Section III-D runs QRP when Y_(n) is fat (n > m). */
void orc_gram(const double *Y, int64_t m, int64_t n, double *S) {
  for (int64_t a = 0; a < m; ++a)
    for (int64_t b = 0; b < m; ++b) {
      double s = 0.0;
      for (int64_t c = 0; c < n; ++c) s += Y[a * n + c] * Y[b * n + c];
      S[a * m + b] = s;
    }
}

/* ---------------------------------------------------------------------------
 * Core tensor, Section III-B (eq. ttm_ele / core_unfolded):
 *   G_(N) = U_N^T Y_(N),  G[r_1..r_{N-1}, r_N] = sum_i U_N(i, r_N) Y_(N)(i, c(r_1..r_{N-1})).
 * Y is I_N x P row-major (P = prod_{m<N} R_m), U_N is I_N x R_N; G is C-order with
 * r_N fastest, i.e. G[c * R_N + r_N].
 * ------------------------------------------------------------------------- */
void orc_core(int64_t I_N, int64_t P, int R_N, const double *Y, const double *U_N, double *G) {
  for (int64_t c = 0; c < P; ++c)
    for (int r = 0; r < R_N; ++r) {
      double s = 0.0;
      for (int64_t i = 0; i < I_N; ++i) s += U_N[i * R_N + r] * Y[i * P + c];
      G[c * R_N + r] = s;
    }
}

/* ---------------------------------------------------------------------------
 * Observed-entry loss and its gradients (the differentiation form):
 *   xhat_z = sum_r G[r] prod_m U_m(i_m(z), r_m),  e_z = xhat_z - x_z,
 *   L = 1/2 sum_z e_z^2,
 *   dL/dG = sum_z e_z kron_m U_m(i_m(z), :),
 *   dL/dU_n(i, r) = sum_{z : i_n(z) = i} e_z sum_{r' : r'_n = r} G[r'] prod_{m != n} U_m(i_m(z), r'_m).
 * Plain loops over every entry of the core for every nonzero.  G is C-order.
 * dU[m] is I_m x R_m; all outputs are overwritten.
 * ------------------------------------------------------------------------- */
void orc_loss_grad(int order, const int64_t *dims, const int *ranks, int64_t nnz,
                   const uint32_t *coords, const double *vals, const double *const *U,
                   const double *G, double *loss, double *const *dU, double *dG) {
  int64_t P = 1;
  for (int m = 0; m < order; ++m) P *= ranks[m];
  memset(dG, 0, sizeof(double) * (size_t)P);
  for (int m = 0; m < order; ++m) memset(dU[m], 0, sizeof(double) * (size_t)(dims[m] * ranks[m]));
  int r[16];
  double L = 0.0;
  for (int64_t z = 0; z < nnz; ++z) {
    /* forward: walk every multi-index r of the core */
    double xhat = 0.0;
    for (int m = 0; m < order; ++m) r[m] = 0;
    for (int64_t q = 0; q < P; ++q) {
      double prod = G[q];
      for (int m = 0; m < order; ++m) prod *= U[m][(int64_t)coords[(int64_t)m * nnz + z] * ranks[m] + r[m]];
      xhat += prod;
      for (int m = order - 1; m >= 0; --m) { /* advance r, last index fastest */
        if (++r[m] < ranks[m]) break;
        r[m] = 0;
      }
    }
    double e = xhat - vals[z];
    L += 0.5 * e * e;
    /* backward */
    for (int m = 0; m < order; ++m) r[m] = 0;
    for (int64_t q = 0; q < P; ++q) {
      double full = 1.0;
      for (int m = 0; m < order; ++m) full *= U[m][(int64_t)coords[(int64_t)m * nnz + z] * ranks[m] + r[m]];
      dG[q] += e * full;
      for (int n = 0; n < order; ++n) {
        double other = G[q];
        for (int m = 0; m < order; ++m)
          if (m != n) other *= U[m][(int64_t)coords[(int64_t)m * nnz + z] * ranks[m] + r[m]];
        dU[n][(int64_t)coords[(int64_t)n * nnz + z] * ranks[n] + r[n]] += e * other;
      }
      for (int m = order - 1; m >= 0; --m) {
        if (++r[m] < ranks[m]) break;
        r[m] = 0;
      }
    }
  }
  *loss = L;
}
