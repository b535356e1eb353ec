/*
 * The FP64 oracle's TTMc, QRP, Gram matrix and core tensor (tucker_oracle.c) split over
 * host threads by output column, for timing the oracle on all of a machine's cores.
 *
 * TEST INFRASTRUCTURE ONLY, like tucker_oracle.c: only the bench's CPU-baseline leg and
 * the tests call it; the product library never does.
 *
 * Nothing is reordered: every thread owns a range of output columns and computes each of
 * its entries with exactly the loops, operand order and summation order of the serial
 * routine (the Kronecker entry is grown ascending from 1.0 one factor at a time; sums run
 * over nonzeros, rows or columns in the serial order).  The results are therefore equal
 * bit for bit to the serial oracle's, which the CPU tests check.  POSIX threads only.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef void (*range_fn)(void *arg, int64_t lo, int64_t hi);

struct par_job {
  range_fn fn;
  void *arg;
  int64_t lo, hi;
};

static void *par_run(void *p) {
  struct par_job *j = (struct par_job *)p;
  if (j->lo < j->hi) j->fn(j->arg, j->lo, j->hi);
  return NULL;
}

/* fn(arg, lo, hi) over contiguous pieces of [0, n) on `threads` threads */
static void par_for(int threads, int64_t n, range_fn fn, void *arg) {
  if (threads < 1) threads = 1;
  if (threads > 256) threads = 256;
  if (threads == 1 || n < 2) {
    fn(arg, 0, n);
    return;
  }
  pthread_t tid[256];
  struct par_job job[256];
  int started[256];
  for (int t = 0; t < threads; ++t) {
    job[t].fn = fn;
    job[t].arg = arg;
    job[t].lo = n * t / threads;
    job[t].hi = n * (t + 1) / threads;
    started[t] = pthread_create(&tid[t], NULL, par_run, &job[t]) == 0;
    if (!started[t]) par_run(&job[t]);
  }
  for (int t = 0; t < threads; ++t)
    if (started[t]) pthread_join(tid[t], NULL);
}

/* ---------------------------------------------------------------- TTMc by columns */
struct ttmc_arg {
  int order, mode;
  const int *ranks;
  int64_t nnz, P;
  const uint32_t *coords;
  const double *vals;
  const double *const *U;
  double *Y;
  const int *digit;  /* [P][order]: rank index of each remaining mode in column c */
};

static void ttmc_cols(void *p, int64_t c0, int64_t c1) {
  const struct ttmc_arg *a = (const struct ttmc_arg *)p;
  for (int64_t z = 0; z < a->nnz; ++z) {
    double *y = a->Y + (int64_t)a->coords[(int64_t)a->mode * a->nnz + z] * a->P;
    for (int64_t c = c0; c < c1; ++c) {
      const int *digit = a->digit + c * a->order;
      double kr = 1.0;
      for (int m = 0; m < a->order; ++m) {
        if (m == a->mode) continue;
        kr = kr * a->U[m][(int64_t)a->coords[(int64_t)m * a->nnz + z] * a->ranks[m] + digit[m]];
      }
      y[c] += a->vals[z] * kr;
    }
  }
}

void orc_ttmc_par(int order, const int64_t *dims, const int *ranks, int64_t nnz, const uint32_t *coords,
                  const double *vals, int mode, const double *const *U, double *Y, int threads) {
  int64_t P = 1;
  for (int m = 0; m < order; ++m)
    if (m != mode) P *= ranks[m];
  memset(Y, 0, sizeof(double) * (size_t)(dims[mode] * P));
  /* digits of every column over the remaining modes, last one fastest (Algorithm 4) */
  const int64_t ndig = P * (int64_t)order;
  int *digit = (int *)malloc(sizeof(int) * (size_t)(ndig > 0 && ndig < ((int64_t)1 << 40) ? ndig : 1));
  if (!digit) return;
  for (int64_t c = 0; c < P; ++c) {
    int64_t rest = c;
    for (int m = order - 1; m >= 0; --m) {
      if (m == mode) continue;
      digit[c * order + m] = (int)(rest % ranks[m]);
      rest /= ranks[m];
    }
  }
  struct ttmc_arg a = {order, mode, ranks, nnz, P, coords, vals, U, Y, digit};
  par_for(threads, P, ttmc_cols, &a);
  free(digit);
}

/* ---------------------------------------------------------------- QRP by columns */
struct qrp_arg {
  int64_t m, n, j;
  int k;
  double *W, *V, *w, *nrm2, s;
  double *Q;
  const double *vtv;
};

static void qrp_norms(void *p, int64_t lo, int64_t hi) { /* columns j + lo .. j + hi */
  struct qrp_arg *a = (struct qrp_arg *)p;
  for (int64_t c = a->j + lo; c < a->j + hi; ++c) {
    double s = 0.0;
    for (int64_t i = a->j; i < a->m; ++i) s += a->W[i * a->n + c] * a->W[i * a->n + c];
    a->nrm2[c] = s;
  }
}

static void qrp_apply(void *p, int64_t lo, int64_t hi) {
  struct qrp_arg *a = (struct qrp_arg *)p;
  const int64_t j = a->j;
  for (int64_t c = j + lo; c < j + hi; ++c) {
    double d = 0.0;
    for (int64_t i = j; i < a->m; ++i) d += a->V[i * a->k + j] * a->W[i * a->n + c];
    a->w[c] = 2.0 * d / a->s;
  }
  for (int64_t i = j; i < a->m; ++i)
    for (int64_t c = j + lo; c < j + hi; ++c) a->W[i * a->n + c] -= a->V[i * a->k + j] * a->w[c];
}

static void qrp_form_q(void *p, int64_t lo, int64_t hi) { /* columns lo .. hi of Q */
  struct qrp_arg *a = (struct qrp_arg *)p;
  for (int j = a->k - 1; j >= 0; --j) {
    if (a->vtv[j] == 0.0) continue;
    for (int64_t c = lo; c < hi; ++c) {
      double d = 0.0;
      for (int64_t i = j; i < a->m; ++i) d += a->V[i * a->k + j] * a->Q[i * a->k + c];
      double f = 2.0 * d / a->vtv[j];
      for (int64_t i = j; i < a->m; ++i) a->Q[i * a->k + c] -= a->V[i * a->k + j] * f;
    }
  }
}

int orc_qrp_par(const double *A, int64_t m, int64_t n, int64_t lda, int k, double *Q, int64_t *piv, double *rdiag,
                int threads) {
  if (k < 0 || k > m || k > n) return -1;
  double *W = (double *)malloc(sizeof(double) * (size_t)(m * n + 1));
  for (int64_t i = 0; i < m; ++i)
    for (int64_t c = 0; c < n; ++c) W[i * n + c] = A[i * lda + c];
  int64_t *perm = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
  for (int64_t c = 0; c < n; ++c) perm[c] = c;
  double *V = (double *)calloc((size_t)(m * (k > 0 ? k : 1)), sizeof(double));
  double *vtv = (double *)calloc((size_t)(k > 0 ? k : 1), sizeof(double));
  double *w = (double *)malloc(sizeof(double) * (size_t)(n + 1));
  double *nrm2 = (double *)malloc(sizeof(double) * (size_t)(n + 1));
  struct qrp_arg a = {m, n, 0, k, W, V, w, nrm2, 0.0, Q, vtv};
  for (int j = 0; j < k; ++j) {
    a.j = j;
    par_for(threads, n - j, qrp_norms, &a);
    int64_t best = j;
    double best_nrm = -1.0;
    for (int64_t c = j; c < n; ++c) {
      double nrm = sqrt(nrm2[c]);
      if (nrm > best_nrm) {
        best_nrm = nrm;
        best = c;
      }
    }
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
    double alpha = 0.0;
    for (int64_t i = j; i < m; ++i) alpha += W[i * n + j] * W[i * n + j];
    alpha = sqrt(alpha);
    if (alpha == 0.0) {
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
    a.s = s;
    par_for(threads, n - j, qrp_apply, &a);
    rdiag[j] = W[(int64_t)j * n + j];
  }
  for (int64_t i = 0; i < m; ++i)
    for (int c = 0; c < k; ++c) Q[i * k + c] = (i == c) ? 1.0 : 0.0;
  par_for(threads, k, qrp_form_q, &a);
  free(W);
  free(perm);
  free(V);
  free(vtv);
  free(w);
  free(nrm2);
  return 0;
}

/* ---------------------------------------------------------------- Gram and core */
struct mat_arg {
  const double *Y, *U;
  int64_t m, n, P;
  int R;
  double *out;
};

static void gram_rows(void *p, int64_t lo, int64_t hi) {
  const struct mat_arg *a = (const struct mat_arg *)p;
  for (int64_t r = lo; r < hi; ++r)
    for (int64_t b = 0; b < a->m; ++b) {
      double s = 0.0;
      for (int64_t c = 0; c < a->n; ++c) s += a->Y[r * a->n + c] * a->Y[b * a->n + c];
      a->out[r * a->m + b] = s;
    }
}

void orc_gram_par(const double *Y, int64_t m, int64_t n, double *S, int threads) {
  struct mat_arg a = {Y, NULL, m, n, 0, 0, S};
  par_for(threads, m, gram_rows, &a);
}

static void core_cols(void *p, int64_t lo, int64_t hi) {
  const struct mat_arg *a = (const struct mat_arg *)p;
  for (int64_t c = lo; c < hi; ++c)
    for (int r = 0; r < a->R; ++r) {
      double s = 0.0;
      for (int64_t i = 0; i < a->m; ++i) s += a->U[i * a->R + r] * a->Y[i * a->P + c];
      a->out[c * a->R + r] = s;
    }
}

void orc_core_par(int64_t I_N, int64_t P, int R_N, const double *Y, const double *U_N, double *G, int threads) {
  struct mat_arg a = {Y, U_N, I_N, 0, P, R_N, G};
  par_for(threads, P, core_cols, &a);
}
