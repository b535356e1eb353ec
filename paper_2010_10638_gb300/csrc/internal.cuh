// Internal declarations shared by the translation units of libtucker.
// Not part of the public ABI (see include/tucker.h).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/tucker.h"

namespace tk {

constexpr int kMaxOrder = 8;
constexpr uint32_t kErrCoord = 1u;    // a coordinate >= its dimension
constexpr uint32_t kErrValue = 2u;    // a non-finite value
constexpr uint32_t kErrTimeout = 4u;  // a bounded device-side wait gave up
constexpr uint32_t kErrLaunch = 8u;   // a kernel found its launch shape different from its plan
constexpr uint32_t kErrCheck = 16u;   // checked build: an index fell outside its array

// Per-mode sorted copy of the nonzeros (a CSF root level over the non-empty slices)
// and the work-unit table of the TTMc kernel.
struct ModeCopy {
  int64_t I = 0;   // rows of Y_(n)
  int64_t P = 0;   // columns of Y_(n)
  int64_t S = 0;   // non-empty slices
  int nother = 0;  // N - 1
  int other[kMaxOrder] = {};           // remaining modes, ascending
  uint32_t *idx[kMaxOrder] = {};       // idx[t][e]: coordinate of mode other[t] of sorted nonzero e
  float *val = nullptr;                // value of sorted nonzero e
  uint32_t *sptr = nullptr;            // [S+1] first sorted position of each non-empty slice
  uint32_t *sid = nullptr;             // [S] row of Y_(n) of each non-empty slice
  uint32_t *empty = nullptr;           // [n_empty] rows with no nonzero
  int64_t n_empty = 0;
  int chunk = 0;                       // nominal nonzeros per work unit
  uint32_t *unit_e0 = nullptr;         // [n_units] first sorted position of each unit
  uint32_t *unit_k0 = nullptr;         // [n_units] slice containing that position
  int32_t *unit_slot = nullptr;        // [n_units] -1: whole slices -> Y; >= 0: partial row slot
  int64_t n_units = 0;
  uint32_t *long_k = nullptr;          // [n_long] slices longer than `chunk`
  uint32_t *long_u0 = nullptr;         // [n_long] their first unit (= first partial slot)
  uint32_t *long_np = nullptr;         // [n_long] their number of units
  int64_t n_long = 0;
  uint32_t *src = nullptr;             // [nnz] index in the coalesced order of sorted position e;
                                       // nullptr for a mode 1 copy in the coalesced order itself
  // Fiber level (order 3): within a slice, runs of nonzeros with the same index of the
  // middle remaining mode other[fmid_t], cut every kFiberCap nonzeros (with fmid_t = 1 the
  // copy is sorted by (i_n, i_other[1], i_other[0])).  Work units and long-slice tables over
  // fibers, as above over nonzeros.
  bool fib = false;
  int fmid_t = 0;                      // the middle (fiber) level is remaining mode other[fmid_t]
  int64_t F = 0;                       // fibers
  uint32_t *fptr = nullptr;            // [F+1] first sorted position of each fiber
  uint32_t *fmid = nullptr;            // [F] index of the first remaining mode of each fiber
  uint32_t *fsptr = nullptr;           // [S+1] first fiber of each non-empty slice
  uint32_t *fbits = nullptr;           // [Z/32 + 3] bit e: sorted position e starts a fiber (zero padded)
  uint32_t *unit_f0 = nullptr;         // [n_units] fiber containing the first position of each nonzero unit
  int fchunk = 0;
  uint32_t *funit_e0 = nullptr, *funit_k0 = nullptr;
  int32_t *funit_slot = nullptr;
  int64_t fn_units = 0;
  uint32_t *flong_k = nullptr, *flong_u0 = nullptr, *flong_np = nullptr;
  int64_t fn_long = 0;
};

constexpr int kFiberCap = 32;  // nonzeros per fiber at most (longer runs are cut)

// Workspace of the QR with column pivoting (one set, sized for the largest mode).
struct QrpWork {
  double *V = nullptr;       // m x k reflectors, V[i*k + j]
  double *F = nullptr;       // n x k, F[c*k + j]
  double *part = nullptr;    // nb x (n + k) block partial sums
  size_t part_elems = 0;     // doubles in `part`
  double *vn = nullptr;      // n trailing squared norms (current column order)
  double *vref = nullptr;    // n squared norms at their last exact computation
  int *perm = nullptr;       // n current column order (original indices)
  int *flag = nullptr;       // n columns whose norm must be recomputed
  double *T = nullptr;       // k x k triangular factor of the compact WY form
  double *M = nullptr;       // k x k, T * V[0:k, :]^T
  double *scal = nullptr;    // scalars: [0] tau, [1] beta, [2] v_jj, [3..] misc
  int *iscal = nullptr;      // int scalars: [0] pivot, [1] number of flagged columns, [2..3] counters
  unsigned *counter = nullptr;  // last-block counters
  int *nflag = nullptr;      // [64] per-step count of columns whose norm is recomputed
  unsigned *bar = nullptr;   // [4] grid barrier: arrivals, generation, error word, spare
  uint32_t *err_out = nullptr;  // where a timed-out barrier is reported (default &bar[2])
  // [n] column sums of squares of A given by the caller (FP32 A), or nullptr: the cluster
  // form then skips its own first pass over A and takes these as the initial norms
  const double *colsq = nullptr;
  size_t bytes = 0;
};

struct Ctx {
  int N = 0;
  int64_t dims[kMaxOrder] = {};
  int ranks[kMaxOrder] = {};
  uint32_t flags = 0;
  int64_t nnz_in = 0;
  int64_t nnz = 0;           // after coalescing
  double norm2 = 0.0;        // ||X||^2 over coalesced values
  int num_sms = 0;
  int device = 0;

  uint32_t *coords = nullptr;  // coalesced [N][nnz], sorted by the full key (mode 1 first)
  float *vals = nullptr;       // coalesced values (FP32 rounding of the FP64 sums)
  ModeCopy mode[kMaxOrder];

  double *U64[kMaxOrder] = {};        // FP64 master factors
  float *U32[kMaxOrder] = {};         // FP32 copies read by the TTMc
  __nv_bfloat16 *U16[kMaxOrder] = {}; // BF16 copies (TUCKER_F_BF16_FACTORS)
  // TMA descriptors of the BF16 copies (rows of one factor, one row per box) for the row
  // gathers of the pipelined BF16 TTMc; tm16_ok[m] false where none could be made
  CUtensorMap tm16[kMaxOrder] = {};
  bool tm16_ok[kMaxOrder] = {};

  float *Y = nullptr;          // TTMc output of the current mode (max I_n * P_n floats)
  float *carry = nullptr;      // partial rows of split slices (max n_units * P_n floats)
  float *fib_T = nullptr;      // fiber form: factor sums of the fibers (max F * R_last floats)
  uint32_t *fib_iota = nullptr;  // fiber form: 0, 1, ..., F-1 (max F)
  float *fib_ones = nullptr;   // fiber form: 1.0f (max F)
  double *gram = nullptr;      // Y Y^T for fat unfoldings
  double *gram_part = nullptr; // column-range partials of the tensor-core Gram matrix
  float2 *sq_part = nullptr;   // column sums of squares of Y_(n): [rows][P_n] double-float pairs,
                               // one row per pipelined TTMc block, then one per split slice
  int64_t sq_elems = 0;        // pairs in sq_part (with the reduction's chunk sums after the rows)
  unsigned *sq_cnt = nullptr;  // [8] arrival counters of the norm reduction (zero between launches)
  double *colsq = nullptr;     // [max P_n] column sums of squares of Y_(n), reduced from sq_part
  double *G = nullptr;         // core tensor of the last sweep
  double *fit_dev = nullptr;   // fit of the last sweep (device)
  double *norm_dev = nullptr;  // [0] ||X||^2, [1] ||G||^2
  double *core_part = nullptr; // block partials of the core GEMM
  unsigned *core_counter = nullptr;
  // adjoint workspaces (allocated by the first tucker_loss_grad)
  float *adj_e0 = nullptr;     // residuals in lexicographic order
  float *adj_en = nullptr;     // residuals in the order of one mode's copy
  float *adj_Y = nullptr;      // TTMc of the residual tensor (max I_n * P_n)
  float *adj_Q = nullptr;      // U_1 G_(1) (I_1 x P_1)
  float *adj_Gn = nullptr;     // one unfolding of G (prod R)
  double *adj_part = nullptr;  // loss partials
  float *adj_gpart = nullptr;  // split-K partials of dL/dG
  bool G_valid = false;
  int sweeps = 0;

  QrpWork qw;
  uint32_t *d_err = nullptr;   // latched device error bits

  bool profiling = false;      // record CUDA events around the phases of hooi_iter
  cudaEvent_t ev[2 * kMaxOrder + 2] = {};
  int n_ev = 0;

  // one HOOI sweep captured as a CUDA graph (tucker_hooi_graph), with the fit destination
  cudaGraphExec_t sweep_graph = nullptr;
  double *graph_fit = nullptr;
  uint64_t graph_kernels = 0;  // library kernels in one replay of the graph

  std::vector<void *> allocs;  // every device allocation, freed by tucker_free
  cudaStream_t astream = 0;    // the stream allocations and frees are ordered on (the current call's)
  std::string last_error;
};

// ---- instrumentation: kernels launched by this library (process-wide)
void count_launch();
uint64_t launches_so_far();
void count_launches(int64_t delta);  // graph replays add their kernels; captures remove theirs

// ---- allocation (host-side failure injection for tests: TUCKER_FAIL_ALLOC_AT=k fails the k-th)
cudaError_t dev_alloc(Ctx *c, void **p, size_t bytes);
void dev_free(Ctx *c, void *p);  // one of c's allocations, in the order of c->astream
template <typename T>
cudaError_t dev_alloc(Ctx *c, T **p, size_t count) {
  return dev_alloc(c, reinterpret_cast<void **>(p), count * sizeof(T));
}
void reset_alloc_counter();

// ---- scan (exclusive, uint32) over n elements; `tmp` must hold scan_tmp_elems(n) words
size_t scan_tmp_elems(int64_t n);
void exclusive_scan_u32(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *tmp, cudaStream_t s);

// ---- stable LSD radix sort of records of 32-bit words (radix.cu)
constexpr int kRadixMaxWords = kMaxOrder + 3;
struct RadixRecords {
  int nwords = 0;
  const uint32_t *in[kRadixMaxWords] = {};  // nullptr: the word is the record's input position
  uint32_t *out[kRadixMaxWords] = {};       // sorted words; must not alias `in`
};
struct RadixKey {
  int word;  // key word (least significant key first in the key list)
  int bits;  // its values are < 2^bits
};
int radix_bits(int64_t maxval);  // bits needed for values 0..maxval
size_t radix_scratch_bytes(int64_t n, int nwords, const RadixKey *keys, int nkeys);
// Sorts the n records by keys[nkeys-1], ..., keys[0] (most significant last), stable.
// Optionally validates words 0..nvalid-1 against valid_dims (device) and valid_vals for
// finiteness, setting bits of *err.  A look-back wait that gives up sets kErrTimeout.
// Returns 0, -1 (bad arguments) or -2 (a CUDA call failed).
int radix_sort_records(int64_t n, const RadixRecords &r, const RadixKey *keys, int nkeys, const int64_t *valid_dims,
                       int nvalid, const float *valid_vals, void *scratch, size_t scratch_bytes, uint32_t *err,
                       cudaStream_t s);
void iota_u32(uint32_t *out, int64_t n, cudaStream_t s);
// self-test of the bounded look-back: 0 and the error word in *err_out, or -2 (CUDA error)
int radix_selftest_wait(uint32_t polls, cudaStream_t s, uint32_t *err_out);

// ---- K-a: reorder (reorder.cu)
tucker_status build_sorted_copies(Ctx *c, const uint32_t *coords, const float *vals, cudaStream_t s);
// the library pool of `device` with one allocation made and freed (current device = device)
cudaError_t pool_warm(int device);
// load the kernels the initialisation launches (cudaFuncGetAttributes on each)
cudaError_t preload_radix_kernels();
cudaError_t preload_reorder_kernels();

// ---- K-b: TTMc (ttmc.cu)
tucker_status launch_ttmc(Ctx *c, int mode, float *Y, cudaStream_t s);
// launch_ttmc that also writes the column sums of squares of Y_(n) to colsq [P_n] where its
// pipelined FP32 form runs (*formed true), at no extra pass over Y; *formed false otherwise.
tucker_status launch_ttmc_norms(Ctx *c, int mode, float *Y, double *colsq, bool *formed, cudaStream_t s);
int64_t ttmc_pipe_blocks(int64_t units);  // blocks of a pipelined TTMc launch over `units` units
int32_t qrp_check_site();                 // checked build: first index check that failed (0: none); -1 otherwise
// TMA descriptors of the BF16 factor copies (host only; no device work)
void make_factor_maps(Ctx *c);
// 0, 1, ..., n-1 and n ones (the index and value streams of the fiber form's update pass)
void fill_iota_ones(uint32_t *iota, float *ones, int64_t n, cudaStream_t s);
// TTMc of mode `mode` with values `val` (in that mode's sorted order) and FP32 factors
// Uf[m] (indexed by mode; Uf[mode] unused) instead of the context's own.
tucker_status launch_ttmc_ex(Ctx *c, int mode, float *Y, const float *val, const float *const *Uf, cudaStream_t s);

// ---- K-c: QRP (qrp.cu)
size_t qrp_work_bytes(int64_t m, int64_t n, int k, int nb);
// standalone QRP calls keep their error word in the first bytes of their scratch
constexpr size_t kQrpErrWordBytes = 256;
tucker_status qrp_read_err_word(uint32_t *word, cudaStream_t s);
void qrp_bind_work(QrpWork *w, void *base, int64_t m, int64_t n, int k, int nb);
// A is m x n (row stride lda) of type float or double; writes Q (m x k, row stride ldq),
// piv (int64, may be null), rdiag (may be null).
// Cluster form of the QRP (qrp_cluster.cu): false when its shared-memory plan does not
// fit (the caller runs another form); *err reports a launch that was attempted and failed.
template <typename AT>
bool qrp_cluster(const AT *A, int64_t m, int64_t n, int64_t lda, int k, double *Q, int64_t ldq, int64_t *piv,
                 double *rdiag, QrpWork *w, cudaStream_t s, cudaError_t *err);
tucker_status qrp_run_f64(const double *A, int64_t m, int64_t n, int64_t lda, int k, double *Q, int64_t ldq,
                          int64_t *piv, double *rdiag, QrpWork *w, int nb, cudaStream_t s);
tucker_status qrp_run_f32(const float *A, int64_t m, int64_t n, int64_t lda, int k, double *Q, int64_t ldq,
                          int64_t *piv, double *rdiag, QrpWork *w, int nb, cudaStream_t s);
void gram_f32(const float *Y, int64_t m, int64_t n, double *S, cudaStream_t s);
// S = Y Y^T on the tensor cores where it fits (m <= 1024, c->gram_part allocated), else gram_f32
void launch_gram(Ctx *c, const float *Y, int64_t m, int64_t n, double *S, cudaStream_t s);
size_t gram_part_elems(int64_t m);  // partial buffer of launch_gram for an m x m Gram matrix (0: none)
int qrp_blocks(int num_sms, int64_t m);
tucker_status launch_wait_selftest(Ctx *c, unsigned long long max_polls, cudaStream_t s);

// ---- K-d: core tensor and fit (core.cu)
void launch_core(Ctx *c, const float *Y, const double *U, double *G, cudaStream_t s);
size_t core_part_elems(int num_sms, int64_t P, int R);

// ---- factor copies / misc (api.cu)
void refresh_factor_copies(Ctx *c, int mode, cudaStream_t s);

// ---- K-e: adjoint (adjoint.cu)
tucker_status launch_loss_grad(Ctx *c, const float *const *U, const float *G, double *loss, float *const *dU,
                               float *dG, cudaStream_t s);

}  // namespace tk

#define TK_CUDA(call)                                                     \
  do {                                                                    \
    cudaError_t e__ = (call);                                             \
    if (e__ != cudaSuccess) {                                             \
      c->last_error = std::string(#call) + ": " + cudaGetErrorString(e__); \
      return e__ == cudaErrorMemoryAllocation ? TUCKER_ENOMEM : TUCKER_ECUDA; \
    }                                                                     \
  } while (0)
