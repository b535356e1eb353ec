// qrp_leading_noalloc: the QR with column pivoting of qrp_leading with its scratch in a
// fixed, file-scope device array instead of caller-provided memory.  The paper has no
// counterpart; this entry point exists for callers that cannot allocate device memory
// at all (for example a host program whose device memory is handed in full to another
// allocator at start-up, or a latency-bound loop that must never call cudaMalloc /
// cudaFree, both of which can synchronise the whole device).
//
// The scratch is one static __device__ array of kStaticScratchBytes; every GPU that
// loads this library holds it until the process exits.  In host code its name is
// only a host-side stand-in, so the device address is looked up with
// cudaGetSymbolAddress once per device, with that device current, on the first call
// made on that device, and handed to the kernels as a plain pointer.  The address is
// cached for the life of the process: a cudaDeviceReset after the first call on a
// device unloads the module and makes the cached address stale, so it is not supported.
#include <mutex>

#include "internal.cuh"

namespace {

constexpr size_t kStaticScratchBytes = size_t(16) << 20;  // 16 MiB
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_qrp_scratch[kStaticScratchBytes];

std::mutex g_scratch_mu;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of g_qrp_scratch on the current device (looked up once per device).
tucker_status scratch_on_current_device(void **out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return TUCKER_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return TUCKER_ECUDA;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_qrp_scratch) != cudaSuccess || !p) return TUCKER_ECUDA;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return TUCKER_OK;
}

}  // namespace

extern "C" {

size_t qrp_leading_noalloc_max_bytes(void) { return kStaticScratchBytes; }

tucker_status qrp_leading_noalloc(const double *A, int64_t m, int64_t n, int64_t lda, int k, double *Q,
                                  int64_t *piv, double *rdiag, void *stream) {
  if (m < 0 || n < 0 || lda < n || k < 0) return TUCKER_EINVAL;
  if (k > m || k > n || k > 64) return TUCKER_ERANK;
  if (k == 0) return TUCKER_OK;
  if (!A || !Q) return TUCKER_EINVAL;
  if (qrp_leading_work_bytes(m, n, k) > kStaticScratchBytes) return TUCKER_EINVAL;  // beyond the fixed scratch
  int dev = 0, sms = 1;
  if (cudaGetDevice(&dev) != cudaSuccess) return TUCKER_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return TUCKER_ECUDA;
  void *scratch = nullptr;
  tucker_status st = scratch_on_current_device(&scratch);
  if (st != TUCKER_OK) return st;
  // The QRP clears the parts of its workspace that must start at zero (its block
  // counters, barrier words and F) at the start of every call, and this call clears its
  // error word (the array's first bytes), so stale contents left by an earlier call are
  // harmless; calls that overlap on the GPU share the array and race.
  uint32_t *errw = static_cast<uint32_t *>(scratch);
  if (cudaMemsetAsync(errw, 0, sizeof(uint32_t), static_cast<cudaStream_t>(stream)) != cudaSuccess) return TUCKER_ECUDA;
  tk::QrpWork w;
  tk::qrp_bind_work(&w, static_cast<char *>(scratch) + tk::kQrpErrWordBytes, m, n, k, sms);
  w.err_out = errw;
  return tk::qrp_run_f64(A, m, n, lda, k, Q, k, piv, rdiag, &w, sms, static_cast<cudaStream_t>(stream));
}

tucker_status qrp_leading_noalloc_sync_status(void *stream) {
  void *scratch = nullptr;
  tucker_status st = scratch_on_current_device(&scratch);
  if (st != TUCKER_OK) return st;
  return tk::qrp_read_err_word(static_cast<uint32_t *>(scratch), static_cast<cudaStream_t>(stream));
}

}  // extern "C"
