/*
 * libtucker: sparse Tucker decomposition by HOOI with QR column pivoting on one GPU
 * (sm_103a).  Method: Jiang, Zhang, Lin, Xing, Zhang, "Sparse Tucker Tensor
 * Decomposition on a Hybrid FPGA-CPU Platform", arXiv 2010.10638.
 *
 * C ABI.  No C++ or framework types cross it: plain pointers, sizes and a CUDA
 * stream passed as `void *` (a cudaStream_t; NULL is the legacy default stream).
 *
 * General conventions
 *   - Every call is asynchronous on `stream` unless stated otherwise.
 *   - A return value other than TUCKER_OK means that no output was written.
 *   - Errors that only the device can see (a coordinate out of range, a non-finite
 *     value, a bounded wait that gave up) are latched in a per-context device word
 *     and reported by the next call that synchronises (tucker_init,
 *     hooi_iter with a host fit pointer, tucker_sync_status).
 *   - No exception or longjmp crosses the ABI.  Calls on one context are not
 *     thread-safe; distinct contexts are independent.
 *   - Modes are 0-based.  Order N is 2..8.  Indices are 0-based uint32.
 *   - Matrices are row-major.  Factor U_m is I_m x R_m.  The mode-n TTMc output
 *     Y_(n) is I_n x P_n with P_n = prod_{m != n} R_m; its columns follow the
 *     Kronecker layout of Algorithm 4: the remaining modes in ascending order, the
 *     last one varying fastest.  The core tensor G is C-order [R_1]...[R_N].
 *   - The caller owns every pointer it passes.  A context owns its internal device
 *     copies (sorted nonzeros, factors, workspaces) until tucker_free.
 */
#ifndef TUCKER_H
#define TUCKER_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define TUCKER_API __attribute__((visibility("default")))
#else
#define TUCKER_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tucker_ctx tucker_ctx;

typedef enum {
  TUCKER_OK = 0,
  TUCKER_EINVAL = 1,   /* bad argument: null pointer, size, order, coordinate, value */
  TUCKER_ERANK = 2,    /* rank outside 1 <= R_n <= I_n (and R_n <= P_n for direct QRP) */
  TUCKER_ENOMEM = 3,   /* a device or host allocation failed; the context stays freeable */
  TUCKER_ECUDA = 4,    /* a CUDA runtime call failed (message in tucker_last_error) */
  TUCKER_ETIMEOUT = 5, /* a bounded device-side wait gave up */
  TUCKER_ESTATE = 6    /* call out of order (e.g. core tensor before any sweep) */
} tucker_status;

/* Flags for tucker_init. */
#define TUCKER_F_BF16_FACTORS 0x1u /* TTMc reads BF16 copies of the factors (FP32 accumulation) */
#define TUCKER_F_QRP_DIRECT 0x2u   /* fat Y_(n) (P_n > I_n): QRP on Y_(n) itself, not on Y Y^T */
#define TUCKER_F_HOST_INPUT 0x4u   /* coords, vals and U0 given to tucker_init are host pointers */
#define TUCKER_F_FIT_DEVICE 0x8u   /* hooi_iter writes the fit through a device pointer, no sync */
#define TUCKER_F_UNPIPELINED 0x20u /* FP32 TTMc without the one-tile-ahead register prefetch
                                      (same arithmetic, kept for comparison) */
#define TUCKER_F_TTMC_NORMS 0x40u /* hooi_iter: the QRP of Y_(n) takes its initial column norms
                                     from the pipelined FP32 TTMc, which forms them as it writes
                                     Y_(n) (ttmc_mode_norms), instead of its own first pass over
                                     Y_(n); same results to rounding, not faster on GB300 */

/*
 * tucker_lib_setup — optional one-time set-up of the library on a device: creates the
 * library's stream-ordered memory pool, makes its first allocation (a process's first use
 * of the stream-ordered allocator costs milliseconds), and loads the kernels that
 * tucker_init launches (under lazy module loading they would load at their first launch).
 * Without it the same happens on first use.  Safe to call again; leaves the calling
 * thread's current device unchanged.
 *   device  CUDA device ordinal
 * Returns TUCKER_OK, or TUCKER_ECUDA (no such device, or a CUDA call failed).
 */
TUCKER_API tucker_status tucker_lib_setup(int device);

/*
 * tucker_init — load a sparse tensor and prepare it for HOOI (Algorithm 2 input:
 * the sparse tensor X and the ranks R_1..R_N; COO storage, Section III-A).
 *
 *   out     receives the new context (set to NULL on failure)
 *   order   N, 2..8
 *   dims    host array [N]: I_1..I_N, each 1..2^31-1
 *   nnz     number of listed entries (>= 0; may be 0)
 *   coords  [N][nnz] uint32, structure-of-arrays (coords[m*nnz + z] is i_m of entry
 *           z), 0-based; device memory, or host with TUCKER_F_HOST_INPUT
 *   vals    [nnz] float; device, or host with TUCKER_F_HOST_INPUT
 *   ranks   host array [N]: R_1..R_N, 1 <= R_n <= min(I_n, 64), prod R_n <= 2^20
 *           (hooi_iter further needs R_n <= prod_{m != n} R_m unless Y_(n) is fat,
 *           and returns TUCKER_ERANK otherwise)
 *   U0      initial factors, the N matrices [I_m x R_m] (FP64, row-major) one after
 *           another; device, or host with TUCKER_F_HOST_INPUT.  U0 for mode 1 is
 *           never read (mode 1 is updated first).  NULL draws each U_m from a seeded
 *           N(0,1) and orthonormalises it by Householder QR on the device.
 *   seed    seed for the NULL-U0 case
 *   flags   TUCKER_F_* bits
 *
 * Entries naming the same coordinate are summed (FP64) into one nonzero; ||X||^2
 * is taken over the summed values.  For every mode the context builds a copy of the
 * nonzeros sorted by that mode's index (stable), the offsets of each non-empty
 * slice, and a table of work units of near-equal nonzero count.
 * Synchronises `stream` a few times (counts read back size the copies: the coalesced
 * nonzeros, then each mode's slices, units and fibers) and returns TUCKER_EINVAL for a
 * coordinate >= I_m or a non-finite value, TUCKER_ETIMEOUT if a bounded device-side wait
 * of the sort gave up (the context is not created).
 */
TUCKER_API tucker_status tucker_init(tucker_ctx **out, int order, const int64_t *dims, int64_t nnz,
                          const uint32_t *coords, const float *vals, const int *ranks,
                          const double *U0, uint64_t seed, uint32_t flags, void *stream);

/*
 * ttmc_mode — sparse tensor-times-matrix chain of one mode (Algorithm 2, inner loop;
 * Section III-C, eq. for Y_(1)):
 *     Y_(n)(i_n, :) = sum over nonzeros z in slice i_n of x_z * kron_{m != n} U_m(i_m(z), :)
 * using the context's current factors (FP32 copies, or BF16 with TUCKER_F_BF16_FACTORS).
 *   Y   device float [I_n x P_n], caller-owned, fully overwritten (empty slices -> 0)
 * Deterministic: no atomics; the same inputs give bitwise the same Y.
 */
TUCKER_API tucker_status ttmc_mode(tucker_ctx *c, int mode, float *Y, void *stream);

/*
 * ttmc_mode_norms — ttmc_mode, and the squared Euclidean norms of the columns of Y_(n)
 * (the initial pivot norms of the QRP of Y_(n), Section III-D) formed as Y_(n) is written,
 * without another pass over it; hooi_iter hands the same norms to its QRP.
 *     colsq(c) = sum over i of Y_(n)(i, c)^2, exact FP32 squares summed in double-float
 *                pairs within each block, then in a fixed order in FP64 (reproducible)
 *   Y      device float [I_n x P_n], as for ttmc_mode (16-byte aligned)
 *   colsq  device double [P_n], caller-owned, overwritten
 * TUCKER_EINVAL where the mode's TTMc does not run the pipelined FP32 form that forms
 * them (order 3, P_n <= 256, FP32 factors, not TUCKER_F_UNPIPELINED); Y is then written.
 */
TUCKER_API tucker_status ttmc_mode_norms(tucker_ctx *c, int mode, float *Y, double *colsq, void *stream);

/*
 * qrp_leading — Householder QR with column pivoting truncated after k reflectors
 * (Section III-D: A P = Q R, |r_11| >= |r_22| >= ..., H_j = I - 2 v v^T / (v^T v),
 * v = a + sign(a_1) ||a|| e_1 with sign(0) = +1).  Column norms are downdated after
 * each reflector and recomputed exactly when cancellation makes the downdate
 * unreliable; the pivot is the largest trailing norm, the lowest index on ties.
 *
 *   A      device double, m x n, row stride lda >= n (read only)
 *   k      number of reflectors, 0 <= k <= min(m, n)
 *   Q      device double [m x k], row-major: Q = H_1 ... H_k [I_k; 0]
 *   piv    device int64 [k]: original column index chosen at each step
 *   rdiag  device double [k]: diagonal r_jj of R
 *   work   device scratch of at least qrp_leading_work_bytes(m, n, k) bytes,
 *          256-byte aligned, caller-owned; contents on entry are ignored
 */
TUCKER_API tucker_status qrp_leading(const double *A, int64_t m, int64_t n, int64_t lda, int k, double *Q,
                          int64_t *piv, double *rdiag, void *work, size_t work_bytes, void *stream);
TUCKER_API size_t qrp_leading_work_bytes(int64_t m, int64_t n, int k);
/*
 * qrp_leading_sync_status — device-side outcome of the last qrp_leading that used `work`
 * (its first bytes hold that call's error word, cleared by each call).  Synchronises
 * `stream`, then returns TUCKER_ETIMEOUT if a bounded grid-wide wait gave up, TUCKER_ECUDA
 * if a kernel found its launch shape or shared memory different from its plan, TUCKER_OK
 * otherwise, and clears the word.  In both failure cases the call had written NaN into
 * rdiag[0..k) and Q[0] and -1 into piv[0..k) and left the rest of Q unspecified.
 */
TUCKER_API tucker_status qrp_leading_sync_status(void *work, void *stream);

/*
 * qrp_leading_noalloc — qrp_leading without caller-provided scratch, for callers that
 * cannot allocate device memory at all: a host program that hands all of its device
 * memory to another allocator when it starts, or a latency-bound loop that must never
 * call cudaMalloc/cudaFree (both can synchronise the whole device).  The paper has no
 * counterpart; the arithmetic, arguments and results are those of qrp_leading.
 *
 * The scratch is a fixed device array of qrp_leading_noalloc_max_bytes() bytes
 * (16 MiB) that every GPU loading this library holds until the process exits.  Sizes
 * with qrp_leading_work_bytes(m, n, k) above that limit return TUCKER_EINVAL.  No
 * device memory is allocated by the call.  The first call on a device looks up the
 * array's device address (once per device, with that device current); make that
 * first call before any stream capture.  The address is kept for the life of the
 * process, so cudaDeviceReset on a device after its first call is not supported.  All
 * calls share the array: whatever must start at zero is cleared by each call, and calls
 * that overlap on the GPU (different streams, or different host threads on one device)
 * race on it.
 */
TUCKER_API tucker_status qrp_leading_noalloc(const double *A, int64_t m, int64_t n, int64_t lda, int k,
                                             double *Q, int64_t *piv, double *rdiag, void *stream);
/* Device-side outcome of the last qrp_leading_noalloc on the current device, as
 * qrp_leading_sync_status (the error word sits at the start of the fixed array). */
TUCKER_API tucker_status qrp_leading_noalloc_sync_status(void *stream);
TUCKER_API size_t qrp_leading_noalloc_max_bytes(void);

/*
 * hooi_iter — one sweep of Algorithm 2: for n = 1..N, Y_(n) by ttmc_mode and
 * U_n <- the first R_n columns of Q from QRP of Y_(n) (of Y_(n) Y_(n)^T when
 * P_n > I_n, unless TUCKER_F_QRP_DIRECT); then the core G = Y_(N) x_N U_N^T and
 *     fit = 1 - sqrt(max(0, ||X||^2 - ||G||^2)) / ||X||.
 *   fit_out  host double (the call then synchronises `stream`), or a device double
 *            when the context was created with TUCKER_F_FIT_DEVICE; may be NULL
 */
TUCKER_API tucker_status hooi_iter(tucker_ctx *c, double *fit_out, void *stream);

/*
 * tucker_hooi_graph — `sweeps` sweeps of hooi_iter (Algorithm 2) replayed from a CUDA graph
 * of one sweep: the whole iteration (every mode's TTMc, QRP and factor refresh, the core
 * and the fit) is one graph launch, without per-kernel launch overhead or host work
 * between its kernels.  The results are those of hooi_iter, bit for bit.
 *   fit_out  device double: the fit of each sweep is written there (the last one remains);
 *            fixed at the first call (the graph writes to it)
 *   stream   a stream other than the legacy default stream (graph capture needs one)
 * The first call on a context runs one sweep as hooi_iter does (which also completes
 * every one-time set-up of the kernels), then captures the next sweep into a graph and
 * replays it for the remaining sweeps; later calls replay the graph.  TUCKER_EINVAL for a
 * NULL stream or fit pointer, or a fit pointer other than the first call's; errors of the
 * capture are TUCKER_ECUDA.  A later tucker_set_factor keeps the graph valid (it reads
 * the factors in place).
 */
TUCKER_API tucker_status tucker_hooi_graph(tucker_ctx *c, int sweeps, double *fit_out, void *stream);

/*
 * core_tensor — the core of the last sweep, G_(N) = U_N^T Y_(N) (Section III-B,
 * eqs. ttm_ele and core_unfolded).  G: device double [R_1 * ... * R_N], C-order.
 * TUCKER_ESTATE before the first hooi_iter or after tucker_set_factor.
 */
TUCKER_API tucker_status core_tensor(tucker_ctx *c, double *G, void *stream);

/* Current factor U_n (FP64 master copy), device double [I_n x R_n]. */
TUCKER_API tucker_status tucker_get_factor(tucker_ctx *c, int mode, double *U, void *stream);

/* Replace factor U_n (device double [I_n x R_n], or host with TUCKER_F_HOST_INPUT);
 * refreshes the FP32/BF16 copies that ttmc_mode reads. */
TUCKER_API tucker_status tucker_set_factor(tucker_ctx *c, int mode, const double *U, void *stream);

/*
 * tucker_loss_grad — observed-entry loss of a Tucker model and its adjoint:
 *     xhat_z = sum_r G[r] prod_m U_m(i_m(z), r_m),  e_z = xhat_z - x_z,
 *     L = 1/2 sum_z e_z^2,
 *     dL/dG = sum_z e_z kron_m U_m(i_m(z), :),
 *     dL/dU_n(i, :) = sum_{z in slice i of mode n} e_z (G_(n) kron_{m != n} U_m(i_m(z), :)^T)
 * over the context's (coalesced) nonzeros, in FP32; Kronecker rows are recomputed,
 * never stored.  The gradient of U_n is a TTMc of the residuals contracted with G_(n).
 *   U     host array of N device pointers, float [I_m x R_m]
 *   G     device float [prod R], C-order
 *   loss  device double [1]
 *   dU    host array of N device pointers, float [I_m x R_m], overwritten
 *   dG    device float [prod R], overwritten
 * Deterministic (fixed reduction trees, no atomics on values).
 */
TUCKER_API tucker_status tucker_loss_grad(tucker_ctx *c, const float *const *U, const float *G, double *loss,
                               float *const *dU, float *dG, void *stream);

/* Number of nonzeros after coalescing, and ||X||_F^2 (FP64). */
TUCKER_API int64_t tucker_nnz(const tucker_ctx *c);
TUCKER_API double tucker_norm2(const tucker_ctx *c);

/* Synchronise `stream` and report (then clear) the latched device error word. */
TUCKER_API tucker_status tucker_sync_status(tucker_ctx *c, void *stream);

/* Release every device and host resource of the context (NULL is a no-op).
 * Synchronises the context's internal work first. */
TUCKER_API void tucker_free(tucker_ctx *c);

/*
 * Instrumentation (no counterpart in the paper; used to report where a sweep spends
 * its time).  With profiling on, hooi_iter records CUDA events on its stream around
 * each phase; tucker_phase_times waits for the last event of the latest sweep and
 * writes 2N+1 durations in milliseconds: TTMc of mode 1, QRP (and factor copy) of
 * mode 1, ..., TTMc of mode N, QRP of mode N, core tensor + fit.  Returns the number
 * written, or -1 (profiling off, no complete sweep recorded, cap too small).
 */
TUCKER_API tucker_status tucker_set_profiling(tucker_ctx *c, int enable);
TUCKER_API int tucker_phase_times(tucker_ctx *c, float *ms, int cap);
/*
 * Layout of one mode's sorted copy (instrumentation; no counterpart in the paper).  Writes
 * up to `cap` int64 values to the host array `out`, in this order:
 *   [0] non-empty slices S        [1] nonzeros per work unit (chunk)   [2] work units
 *   [3] slices split over units   [4] 1 if the mode has a fiber level  [5] fibers F
 *   [6] fibers per fiber unit     [7] fiber units                      [8] slices split over fiber units
 *   [9] longest fiber (nonzeros)  [10] the middle remaining mode of the fiber level (0-based mode)
 * Returns the number written, or -1 for a bad context, mode or pointer.
 */
TUCKER_API int tucker_mode_info(const tucker_ctx *c, int mode, int64_t *out, int cap);

/*
 * Measured FP32 FMA throughput of the current device in TFLOP/s (instrumentation; no
 * counterpart in the paper): a grid of every SM's resident blocks runs `iters` x 128
 * independent FMAs per thread, timed with CUDA events on `stream` (synchronises it);
 * the best of three timed launches after one warm-up.  Returns -1 on a CUDA error.
 */
TUCKER_API double tucker_fp32_fma_tflops(int iters, void *stream);

/* Number of kernels libtucker has launched in this process, over all contexts. */
TUCKER_API uint64_t tucker_kernel_launches(void);

/*
 * tucker_check_site — for the checked build of the library (the cluster QRP compiled with
 * TUCKER_QRP_CHECKED: every index of its shared, distributed-shared and global arrays is
 * compared with the array's length; one outside is replaced by 0 and its site recorded,
 * and the launch's error word gets a check bit, so hooi_iter returns TUCKER_ECUDA and the
 * standalone QRP's status query TUCKER_ECUDA): the number of the first site whose index
 * fell outside, 0 when none did.  Synchronises the current device.  Returns -1 in the
 * normal build (no checks compiled in), -2 if a CUDA call failed.
 */
TUCKER_API int32_t tucker_check_site(void);

/*
 * Self-test of the bounded device-side waits (no counterpart in the paper): one block
 * polls a flag that nothing sets, with the bounded loop of the QRP grid barrier (at most
 * max_polls polls about 100 ns apart), gives up and latches the timeout bit in the
 * context's error word; the next tucker_sync_status returns TUCKER_ETIMEOUT and clears
 * it.  The context stays usable.
 */
TUCKER_API tucker_status tucker_selftest_wait(tucker_ctx *c, uint64_t max_polls, void *stream);

/*
 * Self-test of the initialisation sort's bounded look-back (no counterpart in the paper):
 * one sort pass over two tiles of 8192 words is launched with a single block that claims
 * the second tile, so the first tile's counts never appear; the block polls for them at
 * most max_polls times, gives up, stores nothing and latches the timeout bit.  Uses its
 * own small allocations on `stream` and synchronises it.
 * Returns TUCKER_ETIMEOUT when the wait gave up as designed, TUCKER_OK if it did not,
 * TUCKER_EINVAL for max_polls = 0 or above 2^22, TUCKER_ECUDA if a CUDA call failed.
 */
TUCKER_API tucker_status tucker_selftest_sort_wait(uint64_t max_polls, void *stream);

TUCKER_API const char *tucker_status_str(tucker_status s);
/* Text of the last error recorded on this context ("" if none); valid until the next call. */
TUCKER_API const char *tucker_last_error(const tucker_ctx *c);

#ifdef __cplusplus
}
#endif
#endif /* TUCKER_H */
