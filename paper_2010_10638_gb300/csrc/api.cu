// C-ABI entry points of libtucker (declared in include/tucker.h) and the HOOI driver
// of Algorithm 2.  Host code only orchestrates: every step of the method runs in the
// kernels of reorder.cu (K-a), ttmc.cu (K-b), qrp.cu (K-c), core.cu (K-d) and
// adjoint.cu (K-e).
#include <algorithm>
#include <atomic>
#include <cstring>
#include <new>

#include <nvtx3/nvToolsExt.h>

#include "internal.cuh"

using tk::Ctx;

struct tucker_ctx {
  Ctx c;
};

namespace tk {

// NVTX ranges on the host timeline (shown by Nsight tools; a few nanoseconds otherwise).
struct Range {
  explicit Range(const char *name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range &) = delete;
  Range &operator=(const Range &) = delete;
};
static const char *const kTtmcRange[kMaxOrder] = {"ttmc mode 0", "ttmc mode 1", "ttmc mode 2", "ttmc mode 3",
                                                  "ttmc mode 4", "ttmc mode 5", "ttmc mode 6", "ttmc mode 7"};
static const char *const kQrpRange[kMaxOrder] = {"qrp mode 0", "qrp mode 1", "qrp mode 2", "qrp mode 3",
                                                 "qrp mode 4", "qrp mode 5", "qrp mode 6", "qrp mode 7"};

static std::atomic<uint64_t> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
uint64_t launches_so_far() { return g_launches.load(std::memory_order_relaxed); }
void count_launches(int64_t delta) { g_launches.fetch_add((uint64_t)delta, std::memory_order_relaxed); }

__global__ void f64_to_f32_kernel(const double *in, int64_t n, float *out32, __nv_bfloat16 *out16) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = in[i];
    out32[i] = __double2float_rn(v);
    if (out16) out16[i] = __double2bfloat16(v);
  }
}

void refresh_factor_copies(Ctx *c, int m, cudaStream_t s) {
  const int64_t n = c->dims[m] * c->ranks[m];
  const unsigned b = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 4096));
  f64_to_f32_kernel<<<b, 256, 0, s>>>(c->U64[m], n, c->U32[m], c->U16[m]);
  ::tk::count_launch();
}

// SplitMix64 (Steele, Lea, Flood 2014) as a counter-based generator; Box-Muller for N(0,1).
__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void gaussian_kernel(uint64_t seed, int mode, int64_t n, double *out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t base = seed * 0x2545F4914F6CDD1Dull + ((uint64_t)mode << 48) + 2ull * (uint64_t)i;
    const double u1 = ((splitmix64(base) >> 11) + 1.0) * (1.0 / 9007199254740993.0);  // (0, 1]
    const double u2 = (splitmix64(base + 1) >> 11) * (1.0 / 9007199254740992.0);      // [0, 1)
    out[i] = sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
  }
}

// Error word of a standalone QRP call: synchronise, read, clear, map to a status.
tucker_status qrp_read_err_word(uint32_t *word, cudaStream_t s) {
  uint32_t bits = 0;
  if (cudaMemcpyAsync(&bits, word, sizeof(uint32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess) return TUCKER_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return TUCKER_ECUDA;
  if (!bits) return TUCKER_OK;
  if (cudaMemsetAsync(word, 0, sizeof(uint32_t), s) != cudaSuccess) return TUCKER_ECUDA;
  if (bits & kErrTimeout) return TUCKER_ETIMEOUT;
  return TUCKER_ECUDA;
}

static tucker_status check_err_word(Ctx *c, cudaStream_t s) {
  uint32_t bits = 0;
  TK_CUDA(cudaMemcpyAsync(&bits, c->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  TK_CUDA(cudaStreamSynchronize(s));
  if (bits) {
    TK_CUDA(cudaMemsetAsync(c->d_err, 0, sizeof(uint32_t), s));
    if (bits & kErrTimeout) {
      c->last_error = "a bounded device-side wait gave up";
      return TUCKER_ETIMEOUT;
    }
    if (bits & kErrLaunch) {
      c->last_error = "a kernel was launched in a shape other than the one it was planned for";
      return TUCKER_ECUDA;
    }
    if (bits & kErrCheck) {
      c->last_error = "checked build: an index fell outside its array (tucker_check_site names it)";
      return TUCKER_ECUDA;
    }
    c->last_error = "device-side input check failed";
    return TUCKER_EINVAL;
  }
  return TUCKER_OK;
}

static int qrp_n_cols(const Ctx *c, int n) {
  const int64_t I = c->dims[n], P = c->mode[n].P;
  const bool fat = P > I && !(c->flags & TUCKER_F_QRP_DIRECT);
  return (int)(fat ? I : P);
}

static tucker_status init_impl(Ctx *c, const uint32_t *coords, const float *vals, const double *U0, uint64_t seed,
                               cudaStream_t s) {
  const int N = c->N;
  c->astream = s;
  TK_CUDA(cudaGetDevice(&c->device));
  TK_CUDA(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device));
  TK_CUDA(dev_alloc(c, &c->d_err, 4));
  TK_CUDA(dev_alloc(c, &c->norm_dev, 2));
  TK_CUDA(dev_alloc(c, &c->fit_dev, 1));
  TK_CUDA(cudaMemsetAsync(c->d_err, 0, sizeof(uint32_t), s));

  // inputs on the device
  const uint32_t *dcoords = coords;
  const float *dvals = vals;
  uint32_t *stage_c = nullptr;
  float *stage_v = nullptr;
  const bool host = (c->flags & TUCKER_F_HOST_INPUT) != 0;
  if (host && c->nnz_in > 0) {
    TK_CUDA(dev_alloc(c, &stage_c, (size_t)c->nnz_in * N));
    TK_CUDA(dev_alloc(c, &stage_v, (size_t)c->nnz_in));
    TK_CUDA(cudaMemcpyAsync(stage_c, coords, sizeof(uint32_t) * (size_t)c->nnz_in * N, cudaMemcpyHostToDevice, s));
    TK_CUDA(cudaMemcpyAsync(stage_v, vals, sizeof(float) * (size_t)c->nnz_in, cudaMemcpyHostToDevice, s));
    dcoords = stage_c;
    dvals = stage_v;
  }
  tucker_status st = build_sorted_copies(c, dcoords, dvals, s);
  if (stage_c) {  // freed in stream order, after the sorts that read them
    dev_free(c, stage_c);
    dev_free(c, stage_v);
  }
  if (st != TUCKER_OK) return st;

  // buffers sized for the largest mode
  int64_t ymax = 1, carry_max = 1, gram_max = 1, Imax = 1, IRmax = 1;
  size_t qbytes = 256;
  for (int n = 0; n < N; ++n) {
    const ModeCopy &mc = c->mode[n];
    ymax = std::max(ymax, mc.I * mc.P);
    carry_max = std::max(carry_max, std::max(mc.n_units, mc.fn_units) * mc.P);
    Imax = std::max(Imax, mc.I);
    IRmax = std::max(IRmax, c->dims[n] * c->ranks[n]);
    const int ncols = qrp_n_cols(c, n);
    if (ncols == mc.I && mc.P > mc.I) gram_max = std::max(gram_max, mc.I * mc.I);
    qbytes = std::max(qbytes, qrp_work_bytes(mc.I, ncols, c->ranks[n], c->num_sms));
    // seeded initial factors run QRP on I_n x R_n
    qbytes = std::max(qbytes, qrp_work_bytes(mc.I, c->ranks[n], c->ranks[n], c->num_sms));
  }
  int64_t PR = 1;
  for (int n = 0; n < N; ++n) PR *= c->ranks[n];
  TK_CUDA(dev_alloc(c, &c->Y, (size_t)ymax));
  TK_CUDA(dev_alloc(c, &c->carry, (size_t)carry_max));
  {  // fiber form: factor sums, and the index / unit-value streams of its update pass
    int64_t fmax = 0, tmax = 0;
    for (int n = 0; n < N; ++n)
      if (c->mode[n].fib) {
        fmax = std::max(fmax, c->mode[n].F);
        const ModeCopy &mc = c->mode[n];  // t_f sums the remaining mode that is not the middle one
        tmax = std::max(tmax, mc.F * (int64_t)c->ranks[mc.other[1 - mc.fmid_t]]);
      }
    if (fmax > 0) {
      TK_CUDA(dev_alloc(c, &c->fib_T, (size_t)tmax));
      TK_CUDA(dev_alloc(c, &c->fib_iota, (size_t)fmax));
      TK_CUDA(dev_alloc(c, &c->fib_ones, (size_t)fmax));
      fill_iota_ones(c->fib_iota, c->fib_ones, fmax, s);
      TK_CUDA(cudaGetLastError());
    }
  }
  TK_CUDA(dev_alloc(c, &c->gram, (size_t)gram_max));
  {
    size_t gp = 0;
    for (int n = 0; n < N; ++n) {
      const ModeCopy &mc = c->mode[n];
      if (qrp_n_cols(c, n) == mc.I && mc.P > mc.I) gp = std::max(gp, gram_part_elems(mc.I));
    }
    if (gp) TK_CUDA(dev_alloc(c, &c->gram_part, gp));
  }
  {  // column sums of squares from the pipelined TTMc: one row per block, one per split slice
    int64_t rows = 0, pmax = 1;
    for (int n = 0; n < N; ++n) {
      const ModeCopy &mc = c->mode[n];
      int64_t r = std::max(ttmc_pipe_blocks(mc.n_units) + mc.n_long, ttmc_pipe_blocks(mc.fn_units) + mc.fn_long);
      r += (r + 63) / 64;  // the reduction's chunk sums (64 rows each)
      rows = std::max(rows, r * mc.P);
      pmax = std::max(pmax, mc.P);
    }
    TK_CUDA(dev_alloc(c, &c->sq_part, (size_t)std::max<int64_t>(rows, 1)));
    TK_CUDA(dev_alloc(c, &c->colsq, (size_t)pmax));
    TK_CUDA(dev_alloc(c, &c->sq_cnt, 8));
    TK_CUDA(cudaMemsetAsync(c->sq_cnt, 0, 8 * sizeof(unsigned), s));
    c->sq_elems = rows;
  }
  TK_CUDA(dev_alloc(c, &c->G, (size_t)PR));
  TK_CUDA(dev_alloc(c, &c->core_part, core_part_elems(c->num_sms, c->mode[N - 1].P, c->ranks[N - 1])));
  TK_CUDA(dev_alloc(c, &c->core_counter, 4));
  TK_CUDA(cudaMemsetAsync(c->core_counter, 0, 16, s));
  void *qbase = nullptr;
  TK_CUDA(dev_alloc(c, &qbase, qbytes));
  c->qw.V = static_cast<double *>(qbase);  // base pointer; bound per call
  c->qw.bytes = qbytes;

  // factors
  for (int m = 0; m < N; ++m) {
    const size_t n = (size_t)(c->dims[m] * c->ranks[m]);
    TK_CUDA(dev_alloc(c, &c->U64[m], n));
    TK_CUDA(dev_alloc(c, &c->U32[m], n));
    if (c->flags & TUCKER_F_BF16_FACTORS) TK_CUDA(dev_alloc(c, &c->U16[m], n));
  }
  if (U0) {
    size_t off = 0;
    for (int m = 0; m < N; ++m) {
      const size_t n = (size_t)(c->dims[m] * c->ranks[m]);
      TK_CUDA(cudaMemcpyAsync(c->U64[m], U0 + off, n * sizeof(double),
                              host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
      off += n;
    }
  } else {
    double *g = nullptr;
    TK_CUDA(dev_alloc(c, &g, (size_t)IRmax));
    for (int m = 0; m < N; ++m) {
      const int64_t n = c->dims[m] * c->ranks[m];
      gaussian_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, s>>>(seed, m, n, g);
      ::tk::count_launch();
      QrpWork w;
      qrp_bind_work(&w, c->qw.V, c->dims[m], c->ranks[m], c->ranks[m], c->num_sms);
      st = qrp_run_f64(g, c->dims[m], c->ranks[m], c->ranks[m], c->ranks[m], c->U64[m], c->ranks[m], nullptr,
                       nullptr, &w, c->num_sms, s);
      if (st != TUCKER_OK) return st;
    }
    dev_free(c, g);
  }
  for (int m = 0; m < N; ++m) refresh_factor_copies(c, m, s);
  if (c->flags & TUCKER_F_BF16_FACTORS) make_factor_maps(c);
  TK_CUDA(cudaGetLastError());
  TK_CUDA(cudaStreamSynchronize(s));
  c->astream = 0;  // the caller may destroy s; later allocations name their own stream
  return TUCKER_OK;
}

static tucker_status mark(Ctx *c, int i, cudaStream_t s) {
  if (!c->profiling) return TUCKER_OK;
  if (!c->ev[i]) TK_CUDA(cudaEventCreate(&c->ev[i]));
  TK_CUDA(cudaEventRecord(c->ev[i], s));
  c->n_ev = i + 1;
  return TUCKER_OK;
}

static tucker_status hooi_impl(Ctx *c, double *fit_out, cudaStream_t s) {
  const int N = c->N;
  for (int n = 0; n < N; ++n) {  // QRP takes k = R_n <= min(rows, columns) of the matrix it factors
    const int64_t I = c->dims[n], P = c->mode[n].P;
    const bool fat = P > I && !(c->flags & TUCKER_F_QRP_DIRECT);
    if (!fat && c->ranks[n] > P) {
      c->last_error = "HOOI needs R_n <= prod_{m != n} R_m for QRP of Y_(n)";
      return TUCKER_ERANK;
    }
  }
  Range sweep("hooi_iter");
  tucker_status st = mark(c, 0, s);
  if (st != TUCKER_OK) return st;
  for (int n = 0; n < N; ++n) {
    const ModeCopy &mc = c->mode[n];
    const int ncols = qrp_n_cols(c, n);
    const bool gram = ncols == mc.I && mc.P > mc.I;  // QRP of Y Y^T (fat Y_(n))
    // with TUCKER_F_TTMC_NORMS the QRP of Y itself takes its initial column norms from the
    // TTMc where that forms them
    const bool want_norms = !gram && (c->flags & TUCKER_F_TTMC_NORMS);
    bool norms = false;  // the TTMc left the column sums of squares of Y in c->colsq
    {
      Range r(kTtmcRange[n]);
      st = want_norms ? launch_ttmc_norms(c, n, c->Y, c->colsq, &norms, s) : launch_ttmc(c, n, c->Y, s);
    }
    if (st == TUCKER_OK) st = mark(c, 2 * n + 1, s);
    if (st != TUCKER_OK) return st;
    Range rq(kQrpRange[n]);
    const int k = c->ranks[n];
    QrpWork w;
    qrp_bind_work(&w, c->qw.V, mc.I, ncols, k, c->num_sms);
    w.err_out = c->d_err;  // a timed-out wait is reported by the next synchronising call
    if (gram) {
      launch_gram(c, c->Y, mc.I, mc.P, c->gram, s);
      st = qrp_run_f64(c->gram, mc.I, mc.I, mc.I, k, c->U64[n], k, nullptr, nullptr, &w, c->num_sms, s);
    } else {
      if (norms) w.colsq = c->colsq;
      st = qrp_run_f32(c->Y, mc.I, mc.P, mc.P, k, c->U64[n], k, nullptr, nullptr, &w, c->num_sms, s);
    }
    if (st != TUCKER_OK) return st;
    refresh_factor_copies(c, n, s);
    st = mark(c, 2 * n + 2, s);
    if (st != TUCKER_OK) return st;
  }
  {
    Range r("core + fit");
    launch_core(c, c->Y, c->U64[N - 1], c->G, s);
  }
  TK_CUDA(cudaGetLastError());
  st = mark(c, 2 * N + 1, s);
  if (st != TUCKER_OK) return st;
  c->G_valid = true;
  ++c->sweeps;
  if (fit_out) {
    if (c->flags & TUCKER_F_FIT_DEVICE) {
      TK_CUDA(cudaMemcpyAsync(fit_out, c->fit_dev, sizeof(double), cudaMemcpyDeviceToDevice, s));
    } else {
      TK_CUDA(cudaMemcpyAsync(fit_out, c->fit_dev, sizeof(double), cudaMemcpyDeviceToHost, s));
      return check_err_word(c, s);
    }
  }
  return TUCKER_OK;
}

// One sweep captured into a CUDA graph, replayed `sweeps` times.  hooi_impl with a device
// fit pointer makes no host synchronisation and allocates nothing, so it captures as is.
static tucker_status hooi_graph_impl(Ctx *c, int sweeps, double *fit_out, cudaStream_t s) {
  if (c->sweep_graph && fit_out != c->graph_fit) {
    c->last_error = "tucker_hooi_graph: the fit pointer differs from the one the graph was captured with";
    return TUCKER_EINVAL;
  }
  const uint32_t saved_flags = c->flags;
  const bool saved_prof = c->profiling;
  c->flags |= TUCKER_F_FIT_DEVICE;  // the fit goes to fit_out on the device inside the graph
  c->profiling = false;             // no event records inside the graph
  tucker_status st = TUCKER_OK;
  int done = 0;
  if (!c->sweep_graph) {
    if (sweeps > 0) {  // one eager sweep: it also completes every one-time set-up of the kernels
      st = hooi_impl(c, fit_out, s);
      ++done;
    }
    cudaGraph_t g = nullptr;
    if (st == TUCKER_OK) {
      cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        const uint64_t before = launches_so_far();
        const tucker_status cs = hooi_impl(c, fit_out, s);
        e = cudaStreamEndCapture(s, &g);
        // the captured launches did not run: count them on every replay instead
        c->graph_kernels = launches_so_far() - before;
        count_launches(-(int64_t)c->graph_kernels);
        if (cs != TUCKER_OK) st = cs;
      }
      if (st == TUCKER_OK && e == cudaSuccess) e = cudaGraphInstantiate(&c->sweep_graph, g, 0);
      if (g) cudaGraphDestroy(g);
      if (st == TUCKER_OK && e != cudaSuccess) {
        c->last_error = std::string("tucker_hooi_graph: capture of a sweep failed: ") + cudaGetErrorString(e);
        cudaGetLastError();
        c->sweep_graph = nullptr;
        st = TUCKER_ECUDA;
      }
      if (st == TUCKER_OK) {
        c->graph_fit = fit_out;
        --c->sweeps;  // the captured sweep did not run
      }
    }
  }
  for (; st == TUCKER_OK && done < sweeps; ++done) {
    const cudaError_t e = cudaGraphLaunch(c->sweep_graph, s);
    if (e != cudaSuccess) {
      c->last_error = std::string("cudaGraphLaunch: ") + cudaGetErrorString(e);
      st = TUCKER_ECUDA;
      break;
    }
    count_launches((int64_t)c->graph_kernels);
    ++c->sweeps;
  }
  if (st == TUCKER_OK && done > 0) c->G_valid = true;
  c->flags = saved_flags;
  c->profiling = saved_prof;
  return st;
}

}  // namespace tk

// ============================================================================ C ABI
extern "C" {

const char *tucker_status_str(tucker_status s) {
  switch (s) {
    case TUCKER_OK: return "ok";
    case TUCKER_EINVAL: return "invalid argument";
    case TUCKER_ERANK: return "rank out of range";
    case TUCKER_ENOMEM: return "out of memory";
    case TUCKER_ECUDA: return "CUDA error";
    case TUCKER_ETIMEOUT: return "device wait timed out";
    case TUCKER_ESTATE: return "call out of order";
  }
  return "unknown status";
}

const char *tucker_last_error(const tucker_ctx *c) { return c ? c->c.last_error.c_str() : ""; }

int64_t tucker_nnz(const tucker_ctx *c) { return c ? c->c.nnz : -1; }
double tucker_norm2(const tucker_ctx *c) { return c ? c->c.norm2 : 0.0; }

void tucker_free(tucker_ctx *c) {
  if (!c) return;
  cudaDeviceSynchronize();
  for (void *p : c->c.allocs) cudaFreeAsync(p, 0);  // back to the library's pool
  cudaStreamSynchronize(0);
  for (cudaEvent_t e : c->c.ev)
    if (e) cudaEventDestroy(e);
  if (c->c.sweep_graph) cudaGraphExecDestroy(c->c.sweep_graph);
  delete c;
}

tucker_status tucker_set_profiling(tucker_ctx *h, int enable) {
  if (!h) return TUCKER_EINVAL;
  h->c.profiling = enable != 0;
  h->c.n_ev = 0;
  return TUCKER_OK;
}

int tucker_phase_times(tucker_ctx *h, float *ms, int cap) {
  if (!h || !ms) return -1;
  Ctx *c = &h->c;
  const int want = 2 * c->N + 1;
  if (!c->profiling || c->n_ev != want + 1 || cap < want) return -1;
  if (cudaEventSynchronize(c->ev[want]) != cudaSuccess) return -1;
  for (int i = 0; i < want; ++i)
    if (cudaEventElapsedTime(&ms[i], c->ev[i], c->ev[i + 1]) != cudaSuccess) return -1;
  return want;
}

uint64_t tucker_kernel_launches(void) { return tk::g_launches.load(); }

int32_t tucker_check_site(void) { return tk::qrp_check_site(); }

int tucker_mode_info(const tucker_ctx *h, int mode, int64_t *out, int cap) {
  if (!h || !out || cap < 0 || mode < 0 || mode >= h->c.N) return -1;
  const tk::ModeCopy &mc = h->c.mode[mode];
  const int64_t v[] = {mc.S, mc.chunk, mc.n_units, mc.n_long, mc.fib ? 1 : 0, mc.F, mc.fchunk, mc.fn_units,
                       mc.fn_long, (int64_t)tk::kFiberCap, mc.fib ? (int64_t)mc.other[mc.fmid_t] : -1};
  const int n = std::min<int>(cap, (int)(sizeof(v) / sizeof(v[0])));
  for (int i = 0; i < n; ++i) out[i] = v[i];
  return n;
}

tucker_status tucker_selftest_sort_wait(uint64_t max_polls, void *stream) {
  if (max_polls == 0 || max_polls > (1ull << 22)) return TUCKER_EINVAL;
  uint32_t err = 0;
  if (tk::radix_selftest_wait((uint32_t)max_polls, static_cast<cudaStream_t>(stream), &err) != 0) {
    cudaGetLastError();
    return TUCKER_ECUDA;
  }
  return (err & tk::kErrTimeout) ? TUCKER_ETIMEOUT : TUCKER_OK;
}

tucker_status tucker_selftest_wait(tucker_ctx *h, uint64_t max_polls, void *stream) {
  if (!h) return TUCKER_EINVAL;
  return tk::launch_wait_selftest(&h->c, (unsigned long long)max_polls, static_cast<cudaStream_t>(stream));
}

tucker_status tucker_lib_setup(int device) {
  int old = 0, count = 0;
  if (cudaGetDevice(&old) != cudaSuccess || cudaGetDeviceCount(&count) != cudaSuccess) {
    cudaGetLastError();
    return TUCKER_ECUDA;
  }
  if (device < 0 || device >= count || cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return TUCKER_ECUDA;
  }
  cudaError_t e = tk::pool_warm(device);
  if (e == cudaSuccess) e = tk::preload_radix_kernels();
  if (e == cudaSuccess) e = tk::preload_reorder_kernels();
  if (e == cudaSuccess) {
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, tk::f64_to_f32_kernel);
  }
  cudaSetDevice(old);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return TUCKER_ECUDA;
  }
  return TUCKER_OK;
}

tucker_status tucker_init(tucker_ctx **out, int order, const int64_t *dims, int64_t nnz, const uint32_t *coords,
                          const float *vals, const int *ranks, const double *U0, uint64_t seed, uint32_t flags,
                          void *stream) {
  if (!out) return TUCKER_EINVAL;
  *out = nullptr;
  if (order < 2 || order > tk::kMaxOrder || !dims || !ranks || nnz < 0 || nnz > 0x7fffffffLL) return TUCKER_EINVAL;
  if (nnz > 0 && (!coords || !vals)) return TUCKER_EINVAL;
  int64_t PR = 1;
  for (int m = 0; m < order; ++m) {
    if (dims[m] < 1 || dims[m] > 0x7fffffffLL) return TUCKER_EINVAL;
    if (ranks[m] < 1 || ranks[m] > dims[m] || ranks[m] > 64) return TUCKER_ERANK;
    PR *= ranks[m];
    if (PR > (1 << 20)) return TUCKER_ERANK;
  }
  tucker_ctx *h = new (std::nothrow) tucker_ctx();
  if (!h) return TUCKER_ENOMEM;
  Ctx *c = &h->c;
  c->N = order;
  for (int m = 0; m < order; ++m) {
    c->dims[m] = dims[m];
    c->ranks[m] = ranks[m];
  }
  c->flags = flags;
  c->nnz_in = nnz;
  tk::reset_alloc_counter();
  tk::Range r("tucker_init");
  tucker_status st = tk::init_impl(c, coords, vals, U0, seed, static_cast<cudaStream_t>(stream));
  if (st != TUCKER_OK) {
    // keep the message for the caller through a temporary context? The context is
    // released; the status code carries the failure.
    tucker_free(h);
    return st;
  }
  *out = h;
  return TUCKER_OK;
}

tucker_status ttmc_mode(tucker_ctx *h, int mode, float *Y, void *stream) {
  if (!h || !Y || mode < 0 || mode >= h->c.N) return TUCKER_EINVAL;
  if (reinterpret_cast<uintptr_t>(Y) % 16) return TUCKER_EINVAL;
  tk::Range r("ttmc_mode");
  return tk::launch_ttmc(&h->c, mode, Y, static_cast<cudaStream_t>(stream));
}

tucker_status ttmc_mode_norms(tucker_ctx *h, int mode, float *Y, double *colsq, void *stream) {
  if (!h || !Y || !colsq || mode < 0 || mode >= h->c.N) return TUCKER_EINVAL;
  if (reinterpret_cast<uintptr_t>(Y) % 16) return TUCKER_EINVAL;
  tk::Range r("ttmc_mode_norms");
  bool formed = false;
  const tucker_status st = tk::launch_ttmc_norms(&h->c, mode, Y, colsq, &formed, static_cast<cudaStream_t>(stream));
  if (st != TUCKER_OK) return st;
  if (!formed) {
    h->c.last_error = "column norms are formed by the pipelined FP32 TTMc only (order 3, P_n <= 256)";
    return TUCKER_EINVAL;
  }
  return TUCKER_OK;
}

tucker_status hooi_iter(tucker_ctx *h, double *fit_out, void *stream) {
  if (!h) return TUCKER_EINVAL;
  return tk::hooi_impl(&h->c, fit_out, static_cast<cudaStream_t>(stream));
}

tucker_status tucker_hooi_graph(tucker_ctx *h, int sweeps, double *fit_out, void *stream) {
  if (!h || !fit_out || !stream || sweeps < 0) return TUCKER_EINVAL;
  tk::Range r("tucker_hooi_graph");
  return tk::hooi_graph_impl(&h->c, sweeps, fit_out, static_cast<cudaStream_t>(stream));
}

tucker_status core_tensor(tucker_ctx *h, double *G, void *stream) {
  if (!h || !G) return TUCKER_EINVAL;
  Ctx *c = &h->c;
  if (!c->G_valid) return TUCKER_ESTATE;
  int64_t PR = 1;
  for (int m = 0; m < c->N; ++m) PR *= c->ranks[m];
  TK_CUDA(cudaMemcpyAsync(G, c->G, sizeof(double) * (size_t)PR, cudaMemcpyDeviceToDevice,
                          static_cast<cudaStream_t>(stream)));
  return TUCKER_OK;
}

tucker_status tucker_get_factor(tucker_ctx *h, int mode, double *U, void *stream) {
  if (!h || !U || mode < 0 || mode >= h->c.N) return TUCKER_EINVAL;
  Ctx *c = &h->c;
  TK_CUDA(cudaMemcpyAsync(U, c->U64[mode], sizeof(double) * (size_t)(c->dims[mode] * c->ranks[mode]),
                          cudaMemcpyDeviceToDevice, static_cast<cudaStream_t>(stream)));
  return TUCKER_OK;
}

tucker_status tucker_set_factor(tucker_ctx *h, int mode, const double *U, void *stream) {
  if (!h || !U || mode < 0 || mode >= h->c.N) return TUCKER_EINVAL;
  Ctx *c = &h->c;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool host = (c->flags & TUCKER_F_HOST_INPUT) != 0;
  TK_CUDA(cudaMemcpyAsync(c->U64[mode], U, sizeof(double) * (size_t)(c->dims[mode] * c->ranks[mode]),
                          host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
  tk::refresh_factor_copies(c, mode, s);
  TK_CUDA(cudaGetLastError());
  c->G_valid = false;
  return TUCKER_OK;
}

tucker_status tucker_sync_status(tucker_ctx *h, void *stream) {
  if (!h) return TUCKER_EINVAL;
  return tk::check_err_word(&h->c, static_cast<cudaStream_t>(stream));
}

size_t qrp_leading_work_bytes(int64_t m, int64_t n, int k) {
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return tk::kQrpErrWordBytes + tk::qrp_work_bytes(m, n, k, sms);
}

tucker_status qrp_leading_sync_status(void *work, void *stream) {
  if (!work || reinterpret_cast<uintptr_t>(work) % 256) return TUCKER_EINVAL;
  return tk::qrp_read_err_word(static_cast<uint32_t *>(work), static_cast<cudaStream_t>(stream));
}

tucker_status qrp_leading(const double *A, int64_t m, int64_t n, int64_t lda, int k, double *Q, int64_t *piv,
                          double *rdiag, void *work, size_t work_bytes, void *stream) {
  if (m < 0 || n < 0 || lda < n || k < 0) return TUCKER_EINVAL;
  if (k > m || k > n) return TUCKER_ERANK;
  if (k > 64) return TUCKER_ERANK;
  if (k == 0) return TUCKER_OK;
  if (!A || !Q || !work) return TUCKER_EINVAL;
  if (reinterpret_cast<uintptr_t>(work) % 256) return TUCKER_EINVAL;
  if (work_bytes < qrp_leading_work_bytes(m, n, k)) return TUCKER_EINVAL;
  tk::Range r("qrp_leading");
  int dev = 0, sms = 1;
  if (cudaGetDevice(&dev) != cudaSuccess) return TUCKER_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return TUCKER_ECUDA;
  // the first bytes of the scratch hold the error word of this call (cleared here)
  uint32_t *errw = static_cast<uint32_t *>(work);
  if (cudaMemsetAsync(errw, 0, sizeof(uint32_t), static_cast<cudaStream_t>(stream)) != cudaSuccess) return TUCKER_ECUDA;
  tk::QrpWork w;
  tk::qrp_bind_work(&w, static_cast<char *>(work) + tk::kQrpErrWordBytes, m, n, k, sms);
  w.err_out = errw;
  return tk::qrp_run_f64(A, m, n, lda, k, Q, k, piv, rdiag, &w, sms, static_cast<cudaStream_t>(stream));
}

tucker_status tucker_loss_grad(tucker_ctx *h, const float *const *U, const float *G, double *loss, float *const *dU,
                               float *dG, void *stream) {
  if (!h || !U || !G || !loss || !dU || !dG) return TUCKER_EINVAL;
  for (int m = 0; m < h->c.N; ++m)
    if (!U[m] || !dU[m]) return TUCKER_EINVAL;
  tk::Range r("tucker_loss_grad");
  return tk::launch_loss_grad(&h->c, U, G, loss, dU, dG, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
