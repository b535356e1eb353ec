// K-a: input validation, duplicate coalescing and the per-mode sorted copies.
//
// The paper stores the sparse tensor in COO form (Section III-A, Table I) and runs the
// Kronecker accumulation of Algorithm 2 over its nonzeros.  On the GPU every mode gets
// its own copy of the nonzeros sorted by that mode's index, so that the nonzeros of a
// slice (one row of Y_(n)) are contiguous and can be reduced without atomics:
//   - LSD radix passes (8-bit digits, stable: histogram -> exclusive scan -> scatter
//     ranked with warp match) sort by the full coordinate, mode 1 most significant;
//   - equal neighbours are summed in FP64 (input order) into one nonzero;
//   - per mode: stable radix sort by i_n, gather of the other modes' indices and the
//     values (structure of arrays), offsets of the non-empty slices (a CSF root
//     level), the list of empty rows, and a table of work units of about `chunk`
//     nonzeros: runs of whole short slices, or pieces of a long slice whose partial
//     rows are combined by a second pass.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "internal.cuh"

namespace tk {

// ----------------------------------------------------------------------------- allocation
static int g_alloc_count = 0;
void reset_alloc_counter() { g_alloc_count = 0; }

// Device memory comes from one stream-ordered memory pool per device, owned by the
// library.  An initialisation allocates about a hundred buffers and frees its
// temporaries; with cudaMalloc / cudaFree that cost about 4 ms per initialisation of a
// 20M-nonzero tensor (cudaFree also synchronises the device).  Allocations and frees are
// ordered on the stream of the call that makes them (Ctx::astream); the pool keeps up to
// kPoolKeep bytes of freed memory for the next context and returns the rest to the
// device at the next synchronisation.
constexpr uint64_t kPoolKeep = 16ull << 30;
constexpr int kPoolDevs = 64;
static std::mutex g_pool_mu;
static cudaMemPool_t g_pool[kPoolDevs] = {};

static cudaError_t pool_for(int dev, cudaMemPool_t *out) {
  if (dev < 0 || dev >= kPoolDevs) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_pool_mu);
  if (!g_pool[dev]) {
    cudaMemPoolProps pp = {};
    pp.allocType = cudaMemAllocationTypePinned;
    pp.location.type = cudaMemLocationTypeDevice;
    pp.location.id = dev;
    cudaMemPool_t pool = nullptr;
    cudaError_t e = cudaMemPoolCreate(&pool, &pp);
    if (e != cudaSuccess) return e;
    uint64_t keep = kPoolKeep;
    e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    if (e != cudaSuccess) {
      cudaMemPoolDestroy(pool);
      return e;
    }
    g_pool[dev] = pool;
  }
  *out = g_pool[dev];
  return cudaSuccess;
}

cudaError_t dev_alloc(Ctx *c, void **p, size_t bytes) {
  *p = nullptr;
  ++g_alloc_count;
  const char *f = std::getenv("TUCKER_FAIL_ALLOC_AT");
  if (f && std::atoi(f) == g_alloc_count) return cudaErrorMemoryAllocation;
  if (bytes == 0) bytes = 256;
  cudaMemPool_t pool = nullptr;
  cudaError_t e = pool_for(c->device, &pool);
  if (e == cudaSuccess) e = cudaMallocFromPoolAsync(p, bytes, pool, c->astream);
  if (e == cudaSuccess) c->allocs.push_back(*p);
  else (void)cudaGetLastError();
  return e;
}

// frees p (one of c's allocations) in the order of c->astream
void dev_free(Ctx *c, void *p) {
  if (!p) return;
  auto it = std::find(c->allocs.begin(), c->allocs.end(), p);
  if (it != c->allocs.end()) c->allocs.erase(it);
  cudaFreeAsync(p, c->astream);
}

static void dev_release(Ctx *c, void *p) { dev_free(c, p); }

// ----------------------------------------------------------------------------- scan
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__global__ void __launch_bounds__(kScanThreads) scan_block_kernel(const uint32_t *in, uint32_t *out, int64_t n,
                                                                   uint32_t *block_sums) {
  __shared__ uint32_t warp_tot[32];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)tid * kScanItems;
  uint32_t v[kScanItems];
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = (base + i < n) ? in[base + i] : 0u;
    s += v[i];
  }
  uint32_t incl = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_tot[w] = incl;
  __syncthreads();
  if (w == 0) {
    uint32_t t = warp_tot[lane];
    uint32_t ti = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t u = __shfl_up_sync(0xffffffffu, ti, o);
      if (lane >= o) ti += u;
    }
    warp_tot[lane] = ti - t;  // exclusive prefix of warp totals
    if (lane == 31 && block_sums) block_sums[blockIdx.x] = ti;
  }
  __syncthreads();
  uint32_t run = warp_tot[w] + incl - s;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < n) out[base + i] = run;
    run += v[i];
  }
}

__global__ void scan_add_kernel(uint32_t *out, int64_t n, const uint32_t *block_off) {
  const uint32_t add = block_off[blockIdx.x];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  for (int i = threadIdx.x; i < kScanTile; i += blockDim.x)
    if (base + i < n) out[base + i] += add;
}

static int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

size_t scan_tmp_elems(int64_t n) {
  size_t t = 0;
  int64_t m = n;
  do {
    m = cdiv(m, kScanTile);
    t += (size_t)m + 1;
  } while (m > 1);
  return t + 1;
}

// exclusive scan; the grand total goes to *total (device) when total != nullptr
static void scan_rec(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *tmp, uint32_t *total, cudaStream_t s) {
  if (n <= 0) return;
  int64_t nb = cdiv(n, kScanTile);
  if (nb == 1) {
    scan_block_kernel<<<1, kScanThreads, 0, s>>>(in, out, n, total);
    ::tk::count_launch();
    return;
  }
  scan_block_kernel<<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, tmp);
  ::tk::count_launch();
  scan_rec(tmp, tmp, nb, tmp + nb + 1, total, s);
  scan_add_kernel<<<(unsigned)nb, 256, 0, s>>>(out, n, tmp);
  ::tk::count_launch();
}

void exclusive_scan_u32(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *tmp, cudaStream_t s) {
  scan_rec(in, out, n, tmp, nullptr, s);
}

static void exclusive_scan_total(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *tmp, uint32_t *total,
                                 cudaStream_t s) {
  scan_rec(in, out, n, tmp, total, s);
}

// ----------------------------------------------------------------------------- validation
__global__ void validate_kernel(int N, int64_t nnz, const uint32_t *coords, const float *vals, const int64_t *dims_in,
                                uint32_t *err) {
  __shared__ int64_t dims[kMaxOrder];
  if (threadIdx.x < N) dims[threadIdx.x] = dims_in[threadIdx.x];
  __syncthreads();
  uint32_t bits = 0;
  for (int64_t z = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; z < nnz; z += (int64_t)gridDim.x * blockDim.x) {
    for (int m = 0; m < N; ++m)
      if ((int64_t)coords[(int64_t)m * nnz + z] >= dims[m]) bits |= kErrCoord;
    if (!isfinite(vals[z])) bits |= kErrValue;
  }
  bits = __reduce_or_sync(0xffffffffu, bits);
  if ((threadIdx.x & 31) == 0 && bits) atomicOr(err, bits);
}

// ----------------------------------------------------------------------------- radix passes
constexpr int kRsThreads = 256;
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kRsPerWarp = 512;
constexpr int kRsTile = kRsWarps * kRsPerWarp;

// The keys of a sort are gathered once (key[perm[e]]) into a contiguous array and carried
// with the permutation through the passes, so every pass reads both coalesced; only the
// scatter writes go to data-dependent positions.
__global__ void gather_keys_kernel(const uint32_t *key, const uint32_t *perm, int64_t n, uint32_t *out) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = __ldg(key + perm[e]);
}

__global__ void __launch_bounds__(kRsThreads) radix_hist_kernel(const uint32_t *k, int64_t n, int shift,
                                                                uint32_t *hist) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kRsTile;
  for (int i = threadIdx.x; i < kRsTile; i += kRsThreads) {
    int64_t e = base + i;
    if (e < n) atomicAdd(&h[(k[e] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * gridDim.x + blockIdx.x] = h[threadIdx.x];
}

// One stable pass: element e (key kin[e], source pin[e], or e when pin is null) goes to
// position hist_off[digit, block] + (rank among this block's earlier elements of its
// digit); kout (skipped when null) receives the keys in the new order.
__global__ void __launch_bounds__(kRsThreads) radix_scatter_kernel(const uint32_t *kin, const uint32_t *pin,
                                                                   uint32_t *kout, uint32_t *pout, int64_t n,
                                                                   int shift, const uint32_t *hist_off) {
  __shared__ uint32_t wh[kRsWarps][256];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  for (int i = tid; i < kRsWarps * 256; i += kRsThreads) wh[i / 256][i % 256] = 0;
  __syncthreads();
  const int64_t wbase = (int64_t)blockIdx.x * kRsTile + (int64_t)w * kRsPerWarp;
  for (int st = 0; st < kRsPerWarp / 32; ++st) {
    int64_t e = wbase + st * 32 + lane;
    if (e < n) atomicAdd(&wh[w][(kin[e] >> shift) & 255u], 1u);
  }
  __syncthreads();
  {  // thread tid owns digit tid: running offset over the warps of this block
    uint32_t run = hist_off[(int64_t)tid * gridDim.x + blockIdx.x];
    for (int ww = 0; ww < kRsWarps; ++ww) {
      uint32_t cnt = wh[ww][tid];
      wh[ww][tid] = run;
      run += cnt;
    }
  }
  __syncthreads();
  const uint32_t lt = (1u << lane) - 1u;
  for (int st = 0; st < kRsPerWarp / 32; ++st) {
    int64_t e = wbase + st * 32 + lane;
    bool valid = e < n;
    uint32_t kk = 0, src = 0, d = 256u + lane;
    if (valid) {
      kk = kin[e];
      src = pin ? pin[e] : (uint32_t)e;
      d = (kk >> shift) & 255u;
    }
    uint32_t peers = __match_any_sync(0xffffffffu, d);
    uint32_t rank = __popc(peers & lt);
    uint32_t pos = valid ? wh[w][d] + rank : 0u;
    __syncwarp();
    if (valid && rank == 0) wh[w][d] += __popc(peers);
    __syncwarp();
    if (valid) {
      pout[pos] = src;
      if (kout) kout[pos] = kk;
    }
  }
}

static int bits_for(int64_t maxval) {
  int b = 0;
  while (b < 63 && (maxval >> b) > 0) ++b;
  return b;
}

// Stable sort of the permutation by key[perm[e]] (all bits of key < 2^bits).
// On return *perm points at the sorted permutation (one of pa / pb), or stays
// nullptr (identity) when no pass was needed.  ka / kb hold the carried keys.
static void radix_sort_perm(const uint32_t *key, int bits, int64_t n, uint32_t **perm, uint32_t *pa, uint32_t *pb,
                            uint32_t *ka, uint32_t *kb, uint32_t *hist, uint32_t *tmp, cudaStream_t s) {
  if (n <= 1 || bits <= 0) return;
  const int64_t nb = cdiv(n, kRsTile);
  const uint32_t *kin = key;
  if (*perm) {
    gather_keys_kernel<<<(unsigned)std::min<int64_t>(cdiv(n, 256), 65535LL * 8), 256, 0, s>>>(key, *perm, n, ka);
    ::tk::count_launch();
    kin = ka;
  }
  for (int shift = 0; shift < bits; shift += 8) {
    uint32_t *out = (*perm == pa) ? pb : pa;
    uint32_t *kout = shift + 8 < bits ? (kin == ka ? kb : ka) : nullptr;  // the last pass needs no keys
    radix_hist_kernel<<<(unsigned)nb, kRsThreads, 0, s>>>(kin, n, shift, hist);
    ::tk::count_launch();
    exclusive_scan_u32(hist, hist, 256 * nb, tmp, s);
    radix_scatter_kernel<<<(unsigned)nb, kRsThreads, 0, s>>>(kin, *perm, kout, out, n, shift, hist);
    ::tk::count_launch();
    *perm = out;
    kin = kout;
  }
}

// ----------------------------------------------------------------------------- coalescing
__global__ void mark_new_kernel(int N, int64_t n, const uint32_t *coords, const uint32_t *perm, uint32_t *flag) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    uint32_t f = 1;
    if (e > 0) {
      uint32_t a = perm ? perm[e] : (uint32_t)e, b = perm ? perm[e - 1] : (uint32_t)(e - 1);
      f = 0;
      for (int m = 0; m < N; ++m)
        if (coords[(int64_t)m * n + a] != coords[(int64_t)m * n + b]) {
          f = 1;
          break;
        }
    }
    flag[e] = f;
  }
}

// One thread per group of equal coordinates: FP64 sum in sorted (= input) order.
__global__ void coalesce_kernel(int N, int64_t n, const uint32_t *coords, const float *vals, const uint32_t *perm,
                                const uint32_t *flag, const uint32_t *uid, int64_t nout, uint32_t *out_coords,
                                float *out_vals, double *out_sq) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    if (!flag[e]) continue;
    const uint32_t u = uid[e];
    const uint32_t p = perm ? perm[e] : (uint32_t)e;
    for (int m = 0; m < N; ++m) out_coords[(int64_t)m * nout + u] = coords[(int64_t)m * n + p];
    double s = (double)vals[p];
    for (int64_t e2 = e + 1; e2 < n && !flag[e2]; ++e2) s += (double)vals[perm ? perm[e2] : (uint32_t)e2];
    out_vals[u] = (float)s;
    out_sq[u] = s * s;
  }
}

constexpr int kRedBlocks = 256;
__global__ void reduce_f64_partial(const double *in, int64_t n, double *part) {
  __shared__ double sm[256];
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s += in[i];
  sm[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sm[0];
}
__global__ void reduce_f64_final(const double *part, int np, double *out) {
  __shared__ double sm[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) s += part[i];
  sm[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sm[0];
}

// ----------------------------------------------------------------------------- per-mode copies
struct GatherArgs {
  int nother;
  const uint32_t *src[kMaxOrder];
  uint32_t *dst[kMaxOrder];
};

__global__ void gather_mode_kernel(int64_t n, const uint32_t *perm, GatherArgs g, const uint32_t *rowsrc,
                                   uint32_t *row, const float *vsrc, float *vdst) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t p = perm ? perm[e] : (uint32_t)e;
    row[e] = rowsrc[p];
    vdst[e] = vsrc[p];
    for (int t = 0; t < g.nother; ++t) g.dst[t][e] = g.src[t][p];
  }
}

__global__ void row_kernel(int64_t n, const uint32_t *perm, const uint32_t *rowsrc, uint32_t *row) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    row[e] = rowsrc[perm ? perm[e] : (uint32_t)e];
}

__global__ void iota_kernel(int64_t n, uint32_t *out) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = (uint32_t)e;
}

__global__ void slice_start_kernel(int64_t n, const uint32_t *row, uint32_t *flag) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    flag[e] = (e == 0 || row[e] != row[e - 1]) ? 1u : 0u;
}

__global__ void slice_write_kernel(int64_t n, const uint32_t *row, const uint32_t *flag, const uint32_t *kid,
                                   uint32_t *sptr, uint32_t *sid, uint32_t *present, int64_t S) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    if (flag[e]) {
      const uint32_t k = kid[e];
      sptr[k] = (uint32_t)e;
      sid[k] = row[e];
      present[row[e]] = 1u;
    }
    if (e == 0) sptr[S] = (uint32_t)n;
  }
}

__global__ void invert_flag_kernel(int64_t n, const uint32_t *present, uint32_t *absent) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    absent[i] = present[i] ? 0u : 1u;
}

__global__ void compact_kernel(int64_t n, const uint32_t *flag, const uint32_t *pos, uint32_t *out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (flag[i]) out[pos[i]] = (uint32_t)i;
}

// ---- fibers (order 3): runs of one slice with the same index of the first remaining
//      mode (the middle level of a CSF tree), cut every kFiberCap nonzeros
__global__ void fiber_flag_kernel(int64_t n, const uint32_t *row, const uint32_t *mid, uint32_t *flag) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    flag[e] = (e == 0 || row[e] != row[e - 1] || mid[e] != mid[e - 1]) ? 1u : 0u;
}

__global__ void fiber_nstart_kernel(int64_t n, const uint32_t *flag, const uint32_t *pos, uint32_t *nstart) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    if (flag[e]) nstart[pos[e]] = (uint32_t)e;
}

__global__ void fiber_cut_kernel(int64_t n, const uint32_t *flag, const uint32_t *pos, const uint32_t *nstart,
                                 uint32_t cap, uint32_t *cut) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t fid = pos[e] + flag[e] - 1u;  // the run that contains e
    cut[e] = (((uint32_t)e - nstart[fid]) % cap == 0u) ? 1u : 0u;
  }
}

__global__ void fiber_write_kernel(int64_t n, const uint32_t *cut, const uint32_t *cpos, const uint32_t *mid,
                                   uint32_t *fptr, uint32_t *fmid, int64_t F) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    if (cut[e]) {
      fptr[cpos[e]] = (uint32_t)e;
      fmid[cpos[e]] = mid[e];
    }
    if (e == 0) fptr[F] = (uint32_t)n;
  }
}

// bit e of words[e / 32]: position e starts a fiber (one warp per 32 positions)
__global__ void fiber_bits_kernel(int64_t n, const uint32_t *cut, uint32_t *words) {
  const int lane = threadIdx.x & 31;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e - lane < n; e += (int64_t)gridDim.x * blockDim.x) {
    const unsigned b = __ballot_sync(0xffffffffu, e < n && cut[e] != 0u);
    if (lane == 0) words[e >> 5] = b;
  }
}

// fiber containing the first position of each nonzero work unit
__global__ void unit_fiber_kernel(int64_t n_units, const uint32_t *unit_e0, const uint32_t *cut, const uint32_t *cpos,
                                  uint32_t *unit_f0) {
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n_units; u += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t e = unit_e0[u];
    unit_f0[u] = cpos[e] + cut[e] - 1u;
  }
}

__global__ void fiber_slices_kernel(int64_t S, const uint32_t *sptr, const uint32_t *cpos, uint32_t *fsptr,
                                    int64_t F) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < S; k += (int64_t)gridDim.x * blockDim.x) {
    fsptr[k] = cpos[sptr[k]];  // a slice start is always a fiber start
    if (k == 0) fsptr[S] = (uint32_t)F;
  }
}

// units contributed by each non-empty slice k: pieces of a long slice, or 1 for the
// first slice of a run of short slices (a new run starts at a long slice, after a long
// slice, and where the slice start crosses into a new multiple of `chunk`).
__global__ void unit_count_kernel(int64_t S, const uint32_t *sptr, uint32_t chunk, uint32_t *nu, uint32_t *islong) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < S; k += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t b = sptr[k], len = sptr[k + 1] - b;
    const bool lng = len > chunk;
    bool head = (k == 0) || lng;
    if (k > 0) {
      const uint32_t pb = sptr[k - 1], plen = b - pb;
      head = head || plen > chunk || (b / chunk) != (pb / chunk);
    }
    nu[k] = lng ? (len + chunk - 1) / chunk : (head ? 1u : 0u);
    islong[k] = lng ? 1u : 0u;
  }
}

__global__ void unit_write_kernel(int64_t S, const uint32_t *sptr, uint32_t chunk, const uint32_t *nu,
                                  const uint32_t *uoff, const uint32_t *islong, const uint32_t *lid,
                                  uint32_t *unit_e0, uint32_t *unit_k0, int32_t *unit_slot, uint32_t *long_k,
                                  uint32_t *long_u0, uint32_t *long_np) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < S; k += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t n = nu[k];
    if (n == 0) continue;
    const uint32_t u0 = uoff[k];
    if (islong[k]) {
      for (uint32_t p = 0; p < n; ++p) {
        unit_e0[u0 + p] = sptr[k] + p * chunk;
        unit_k0[u0 + p] = (uint32_t)k;
        unit_slot[u0 + p] = (int32_t)(u0 + p);
      }
      const uint32_t l = lid[k];
      long_k[l] = (uint32_t)k;
      long_u0[l] = u0;
      long_np[l] = n;
    } else {
      unit_e0[u0] = sptr[k];
      unit_k0[u0] = (uint32_t)k;
      unit_slot[u0] = -1;
    }
  }
}

static int pick_chunk(int64_t nnz, int num_sms) {
  const char *f = std::getenv("TUCKER_TTMC_CHUNK");
  if (f) {
    int v = std::atoi(f);
    if (v >= 32 && v <= (1 << 20) && (v % 32) == 0) return v;
  }
  int64_t target = nnz / ((int64_t)num_sms * 8);
  int chunk = 256;
  while (chunk < 2048 && (int64_t)chunk * 2 <= target) chunk *= 2;
  return chunk;
}

// RAII holder for temporaries of the build
struct Temps {
  Ctx *c;
  std::vector<void *> ptrs;
  explicit Temps(Ctx *cc) : c(cc) {}
  template <typename T>
  cudaError_t get(T **p, size_t count) {
    cudaError_t e = dev_alloc(c, p, count);
    if (e == cudaSuccess) ptrs.push_back(*p);
    return e;
  }
  ~Temps() {
    for (void *p : ptrs) dev_release(c, p);
  }
};

static unsigned grid_for(int64_t n, int threads = 256) {
  int64_t b = cdiv(n, threads);
  if (b < 1) b = 1;
  if (b > 65535LL * 8) b = 65535LL * 8;
  return (unsigned)b;
}

#define TK_TRY(call)                                                        \
  do {                                                                      \
    cudaError_t e__ = (call);                                               \
    if (e__ != cudaSuccess) {                                               \
      c->last_error = std::string(#call) + ": " + cudaGetErrorString(e__);  \
      return e__ == cudaErrorMemoryAllocation ? TUCKER_ENOMEM : TUCKER_ECUDA; \
    }                                                                       \
  } while (0)

static tucker_status read_u32(Ctx *c, const uint32_t *d, uint32_t *h, cudaStream_t s) {
  TK_TRY(cudaMemcpyAsync(h, d, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  TK_TRY(cudaStreamSynchronize(s));
  return TUCKER_OK;
}

// Work units over a slice table `ptr` ([S+1] offsets into positions: nonzeros or fibers).
struct UnitTables {
  uint32_t **e0, **k0, **long_k, **long_u0, **long_np;
  int32_t **slot;
  int64_t *n_units, *n_long;
};

static tucker_status build_units(Ctx *c, int64_t S, const uint32_t *ptr, int chunk, uint32_t *nu, uint32_t *islong,
                                 uint32_t *uoff, uint32_t *lid, uint32_t *stmp, uint32_t *d_small, UnitTables o,
                                 cudaStream_t s) {
  uint32_t nunits = 0, nlong = 0;
  if (S > 0) {
    unit_count_kernel<<<grid_for(S), 256, 0, s>>>(S, ptr, (uint32_t)chunk, nu, islong);
    ::tk::count_launch();
    exclusive_scan_total(nu, uoff, S, stmp, d_small + 2, s);
    exclusive_scan_total(islong, lid, S, stmp, d_small + 3, s);
    uint32_t h2[2];
    TK_TRY(cudaMemcpyAsync(h2, d_small + 2, 2 * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    TK_TRY(cudaStreamSynchronize(s));
    nunits = h2[0];
    nlong = h2[1];
  }
  *o.n_units = nunits;
  *o.n_long = nlong;
  TK_TRY(dev_alloc(c, o.e0, (size_t)std::max<uint32_t>(nunits, 1)));
  TK_TRY(dev_alloc(c, o.k0, (size_t)std::max<uint32_t>(nunits, 1)));
  TK_TRY(dev_alloc(c, o.slot, (size_t)std::max<uint32_t>(nunits, 1)));
  TK_TRY(dev_alloc(c, o.long_k, (size_t)std::max<uint32_t>(nlong, 1)));
  TK_TRY(dev_alloc(c, o.long_u0, (size_t)std::max<uint32_t>(nlong, 1)));
  TK_TRY(dev_alloc(c, o.long_np, (size_t)std::max<uint32_t>(nlong, 1)));
  if (S > 0) {
    unit_write_kernel<<<grid_for(S), 256, 0, s>>>(S, ptr, (uint32_t)chunk, nu, uoff, islong, lid, *o.e0, *o.k0,
                                                   *o.slot, *o.long_k, *o.long_u0, *o.long_np);
    ::tk::count_launch();
  }
  TK_TRY(cudaGetLastError());
  return TUCKER_OK;
}

// Whether mode copies of order-3 tensors get a fiber level (TUCKER_TTMC_FIBERS): "1"
// always, "0" never, otherwise when the fibers are at most kFiberShare of the nonzeros.
// The fiber form forms t_f once per nonzero and one rank-1 update per fiber, so it pays
// when fibers are long on average; on the 20M-nonzero skewed workload it ran faster than
// the nonzero form at 0.17 fibers per nonzero and slower at 0.42.
static int fiber_policy() {
  const char *f = std::getenv("TUCKER_TTMC_FIBERS");
  if (f && std::strcmp(f, "1") == 0) return 1;
  if (f && std::strcmp(f, "0") == 0) return 0;
  return -1;
}
constexpr double kFiberShare = 0.25;

tucker_status build_sorted_copies(Ctx *c, const uint32_t *coords_in, const float *vals_in, cudaStream_t s) {
  const int N = c->N;
  const int64_t n_in = c->nnz_in;
  Temps tmp(c);
  int64_t *d_dims = nullptr;
  uint32_t *d_small = nullptr;  // [0..7] totals read back to the host
  TK_TRY(tmp.get(&d_dims, kMaxOrder));
  TK_TRY(tmp.get(&d_small, 8));
  TK_TRY(cudaMemcpyAsync(d_dims, c->dims, sizeof(int64_t) * kMaxOrder, cudaMemcpyHostToDevice, s));
  TK_TRY(cudaMemsetAsync(c->d_err, 0, sizeof(uint32_t), s));

  // ---- validation
  if (n_in > 0) {
    validate_kernel<<<std::min<unsigned>(grid_for(n_in), (unsigned)c->num_sms * 8), 256, 0, s>>>(
        N, n_in, coords_in, vals_in, d_dims, c->d_err);
    ::tk::count_launch();
    TK_TRY(cudaGetLastError());
    uint32_t err = 0;
    tucker_status st = read_u32(c, c->d_err, &err, s);
    if (st != TUCKER_OK) return st;
    if (err) {
      c->last_error = (err & kErrCoord) ? "a coordinate is >= its dimension" : "a value is not finite";
      TK_TRY(cudaMemsetAsync(c->d_err, 0, sizeof(uint32_t), s));
      return TUCKER_EINVAL;
    }
  }

  // ---- scratch shared by all sorts
  const int64_t nmax = std::max<int64_t>(n_in, 1);
  const int64_t nb = cdiv(nmax, kRsTile);
  int64_t maxI = 1;
  for (int m = 0; m < N; ++m) maxI = std::max(maxI, c->dims[m]);
  const int64_t scan_n = std::max<int64_t>(std::max<int64_t>(256 * nb, nmax), maxI + 1);
  uint32_t *pa, *pb, *ka, *kb, *hist, *stmp, *flag, *pos;
  TK_TRY(tmp.get(&pa, nmax));
  TK_TRY(tmp.get(&pb, nmax));
  TK_TRY(tmp.get(&ka, nmax));
  TK_TRY(tmp.get(&kb, nmax));
  TK_TRY(tmp.get(&hist, 256 * nb));
  TK_TRY(tmp.get(&stmp, scan_tmp_elems(scan_n)));
  TK_TRY(tmp.get(&flag, std::max<int64_t>(nmax, maxI + 1)));
  TK_TRY(tmp.get(&pos, std::max<int64_t>(nmax, maxI + 1)));

  // ---- full-key sort: LSD over modes N..1, each mode's digits low to high
  uint32_t *perm = nullptr;
  for (int m = N - 1; m >= 0; --m)
    radix_sort_perm(coords_in + (int64_t)m * n_in, bits_for(c->dims[m] - 1), n_in, &perm, pa, pb, ka, kb, hist, stmp, s);
  TK_TRY(cudaGetLastError());

  // ---- coalesce duplicates
  uint32_t nout = 0;
  if (n_in > 0) {
    mark_new_kernel<<<grid_for(n_in), 256, 0, s>>>(N, n_in, coords_in, perm, flag);
    ::tk::count_launch();
    exclusive_scan_total(flag, pos, n_in, stmp, d_small, s);
    tucker_status st = read_u32(c, d_small, &nout, s);
    if (st != TUCKER_OK) return st;
  }
  c->nnz = nout;
  const int64_t Z = nout;
  TK_TRY(dev_alloc(c, &c->coords, (size_t)std::max<int64_t>(Z, 1) * N));
  TK_TRY(dev_alloc(c, &c->vals, (size_t)std::max<int64_t>(Z, 1)));
  double *sq = nullptr, *part = nullptr;
  TK_TRY(tmp.get(&sq, std::max<int64_t>(Z, 1)));
  TK_TRY(tmp.get(&part, kRedBlocks));
  c->norm2 = 0.0;
  if (n_in > 0) {
    coalesce_kernel<<<grid_for(n_in), 256, 0, s>>>(N, n_in, coords_in, vals_in, perm, flag, pos, Z, c->coords, c->vals,
                                                    sq);
    ::tk::count_launch();
    reduce_f64_partial<<<kRedBlocks, 256, 0, s>>>(sq, Z, part);
    ::tk::count_launch();
    reduce_f64_final<<<1, 256, 0, s>>>(part, kRedBlocks, c->norm_dev);
    ::tk::count_launch();
    TK_TRY(cudaGetLastError());
    TK_TRY(cudaMemcpyAsync(&c->norm2, c->norm_dev, sizeof(double), cudaMemcpyDeviceToHost, s));
    TK_TRY(cudaStreamSynchronize(s));
  } else {
    TK_TRY(cudaMemsetAsync(c->norm_dev, 0, sizeof(double), s));
  }

  // ---- per-mode sorted copies
  uint32_t *row = nullptr, *nu = nullptr, *islong = nullptr, *uoff = nullptr, *lid = nullptr;
  TK_TRY(tmp.get(&row, std::max<int64_t>(Z, 1)));
  TK_TRY(tmp.get(&nu, std::max<int64_t>(Z, 1) + 1));
  TK_TRY(tmp.get(&islong, std::max<int64_t>(Z, 1) + 1));
  TK_TRY(tmp.get(&uoff, std::max<int64_t>(Z, 1) + 1));
  TK_TRY(tmp.get(&lid, std::max<int64_t>(Z, 1) + 1));
  uint32_t fnat[kMaxOrder] = {};  // natural fiber counts, middle = first remaining mode
  uint32_t *fnstart = nullptr, *fcut = nullptr, *fcpos = nullptr;
  if (N == 3 && fiber_policy() != 0) {
    TK_TRY(tmp.get(&fnstart, std::max<int64_t>(Z, 1)));
    TK_TRY(tmp.get(&fcut, std::max<int64_t>(Z, 1)));
    TK_TRY(tmp.get(&fcpos, std::max<int64_t>(Z, 1)));
  }
  for (int n = 0; n < N; ++n) {
    ModeCopy &mc = c->mode[n];
    mc.I = c->dims[n];
    mc.nother = N - 1;
    mc.P = 1;
    int t = 0;
    for (int m = 0; m < N; ++m)
      if (m != n) {
        mc.other[t++] = m;
        mc.P *= c->ranks[m];
      }
    mc.chunk = pick_chunk(Z, c->num_sms);
    GatherArgs g{};
    g.nother = mc.nother;
    for (int q = 0; q < mc.nother; ++q) {
      TK_TRY(dev_alloc(c, &mc.idx[q], (size_t)std::max<int64_t>(Z, 1)));
      g.src[q] = c->coords + (int64_t)mc.other[q] * Z;
      g.dst[q] = mc.idx[q];
    }
    TK_TRY(dev_alloc(c, &mc.val, (size_t)std::max<int64_t>(Z, 1)));
    uint32_t *mperm = nullptr;  // mode 1: the lexicographic order is already sorted by i_1
    if (n > 0) radix_sort_perm(c->coords + (int64_t)n * Z, bits_for(mc.I - 1), Z, &mperm, pa, pb, ka, kb, hist, stmp, s);
    if (n > 0 && Z > 0) {
      TK_TRY(dev_alloc(c, &mc.src, (size_t)Z));
      if (mperm) {
        TK_TRY(cudaMemcpyAsync(mc.src, mperm, sizeof(uint32_t) * (size_t)Z, cudaMemcpyDeviceToDevice, s));
      } else {  // already in order (e.g. a single distinct index): identity
        iota_kernel<<<grid_for(Z), 256, 0, s>>>(Z, mc.src);
        ::tk::count_launch();
      }
    }
    uint32_t S = 0;
    if (Z > 0) {
      gather_mode_kernel<<<grid_for(Z), 256, 0, s>>>(Z, mperm, g, c->coords + (int64_t)n * Z, row, c->vals, mc.val);
      ::tk::count_launch();
      slice_start_kernel<<<grid_for(Z), 256, 0, s>>>(Z, row, flag);
      ::tk::count_launch();
      exclusive_scan_total(flag, pos, Z, stmp, d_small, s);
      tucker_status st = read_u32(c, d_small, &S, s);
      if (st != TUCKER_OK) return st;
    }
    mc.S = S;
    TK_TRY(dev_alloc(c, &mc.sptr, (size_t)S + 1));
    TK_TRY(dev_alloc(c, &mc.sid, (size_t)std::max<uint32_t>(S, 1)));
    uint32_t *present = nu;  // reuse: I_n + 1 <= ... not guaranteed, use dedicated buffer
    TK_TRY(tmp.get(&present, (size_t)mc.I + 1));
    TK_TRY(cudaMemsetAsync(present, 0, sizeof(uint32_t) * (size_t)mc.I, s));
    if (Z > 0) {
      slice_write_kernel<<<grid_for(Z), 256, 0, s>>>(Z, row, flag, pos, mc.sptr, mc.sid, present, S);
      ::tk::count_launch();
    } else {
      TK_TRY(cudaMemsetAsync(mc.sptr, 0, sizeof(uint32_t), s));
    }
    // empty rows
    invert_flag_kernel<<<grid_for(mc.I), 256, 0, s>>>(mc.I, present, flag);
    ::tk::count_launch();
    exclusive_scan_total(flag, pos, mc.I, stmp, d_small + 1, s);
    uint32_t ne = 0;
    tucker_status st = read_u32(c, d_small + 1, &ne, s);
    if (st != TUCKER_OK) return st;
    mc.n_empty = ne;
    TK_TRY(dev_alloc(c, &mc.empty, (size_t)std::max<uint32_t>(ne, 1)));
    if (ne) {
      compact_kernel<<<grid_for(mc.I), 256, 0, s>>>(mc.I, flag, pos, mc.empty);
      ::tk::count_launch();
    }
    // work units
    {
      UnitTables o{&mc.unit_e0, &mc.unit_k0, &mc.long_k, &mc.long_u0, &mc.long_np, &mc.unit_slot, &mc.n_units,
                   &mc.n_long};
      tucker_status st2 = build_units(c, S, mc.sptr, mc.chunk, nu, islong, uoff, lid, stmp, d_small, o, s);
      if (st2 != TUCKER_OK) return st2;
    }
    // natural fiber count with the first remaining mode as the middle level (order 3)
    if (N == 3 && Z > 0 && S > 0 && fiber_policy() != 0) {
      fiber_flag_kernel<<<grid_for(Z), 256, 0, s>>>(Z, row, mc.idx[0], flag);
      ::tk::count_launch();
      exclusive_scan_total(flag, pos, Z, stmp, d_small + 4, s);
      uint32_t fn = 0;
      tucker_status st2 = read_u32(c, d_small + 4, &fn, s);
      if (st2 != TUCKER_OK) return st2;
      fnat[n] = fn;
    }
  }

  // ---- fiber levels (order 3).  The middle level of mode n is its first remaining mode a,
  //      or its last one b when the copy of b is grouped by (i_b, i_n) and has at most 0.8
  //      as many (i_n, i_b) runs as mode n has (i_n, i_a) runs: then mode n's copy is
  //      re-sorted to (i_n, i_b, i_a) (slices and nonzero units are unchanged).
  const int fp = fiber_policy();
  for (int n = 0; n < N && N == 3 && Z > 0 && fp != 0; ++n) {
    ModeCopy &mc = c->mode[n];
    if (mc.S == 0) continue;
    const int b = mc.other[1];
    const bool alt = c->mode[b].other[0] == n && fnat[b] > 0 && (double)fnat[b] <= 0.8 * (double)fnat[n];
    uint32_t *perm = nullptr;
    if (alt) {  // stable sorts of the lexicographic list by i_b, then by i_n
      radix_sort_perm(c->coords + (int64_t)b * Z, bits_for(c->dims[b] - 1), Z, &perm, pa, pb, ka, kb, hist, stmp, s);
      radix_sort_perm(c->coords + (int64_t)n * Z, bits_for(mc.I - 1), Z, &perm, pa, pb, ka, kb, hist, stmp, s);
      if (!mc.src) TK_TRY(dev_alloc(c, &mc.src, (size_t)Z));
      if (perm) {
        TK_TRY(cudaMemcpyAsync(mc.src, perm, sizeof(uint32_t) * (size_t)Z, cudaMemcpyDeviceToDevice, s));
      } else {
        iota_kernel<<<grid_for(Z), 256, 0, s>>>(Z, mc.src);
        ::tk::count_launch();
      }
      GatherArgs g{};
      g.nother = mc.nother;
      for (int q = 0; q < mc.nother; ++q) {
        g.src[q] = c->coords + (int64_t)mc.other[q] * Z;
        g.dst[q] = mc.idx[q];
      }
      gather_mode_kernel<<<grid_for(Z), 256, 0, s>>>(Z, perm, g, c->coords + (int64_t)n * Z, row, c->vals, mc.val);
      ::tk::count_launch();
    } else {  // the rows of this mode's order
      row_kernel<<<grid_for(Z), 256, 0, s>>>(Z, mc.src, c->coords + (int64_t)n * Z, row);
      ::tk::count_launch();
    }
    const int ft = alt ? 1 : 0;
    const uint32_t *mid = mc.idx[ft];
    fiber_flag_kernel<<<grid_for(Z), 256, 0, s>>>(Z, row, mid, flag);
    ::tk::count_launch();
    exclusive_scan_total(flag, pos, Z, stmp, d_small + 4, s);
    fiber_nstart_kernel<<<grid_for(Z), 256, 0, s>>>(Z, flag, pos, fnstart);
    ::tk::count_launch();
    uint32_t cap = (uint32_t)kFiberCap;
    if (const char *fc = std::getenv("TUCKER_TTMC_FIBER_CAP")) {
      const int v = std::atoi(fc);
      if (v >= 1 && v <= kFiberCap) cap = (uint32_t)v;
    }
    fiber_cut_kernel<<<grid_for(Z), 256, 0, s>>>(Z, flag, pos, fnstart, cap, fcut);
    ::tk::count_launch();
    exclusive_scan_total(fcut, fcpos, Z, stmp, d_small + 5, s);
    uint32_t F = 0;
    tucker_status st2 = read_u32(c, d_small + 5, &F, s);
    if (st2 != TUCKER_OK) return st2;
    if (fp == 1 || (double)F <= kFiberShare * (double)Z) {
      mc.fib = true;
      mc.fmid_t = ft;
      mc.F = F;
      TK_TRY(dev_alloc(c, &mc.fptr, (size_t)F + 1));
      TK_TRY(dev_alloc(c, &mc.fmid, (size_t)std::max<uint32_t>(F, 1)));
      TK_TRY(dev_alloc(c, &mc.fsptr, (size_t)mc.S + 1));
      fiber_write_kernel<<<grid_for(Z), 256, 0, s>>>(Z, fcut, fcpos, mid, mc.fptr, mc.fmid, F);
      ::tk::count_launch();
      fiber_slices_kernel<<<grid_for(mc.S), 256, 0, s>>>(mc.S, mc.sptr, fcpos, mc.fsptr, F);
      ::tk::count_launch();
      {  // fiber starts as a bit mask over the sorted positions, three zero words past the end
        const int64_t nw = (Z + 31) / 32 + 3;
        TK_TRY(dev_alloc(c, &mc.fbits, (size_t)nw));
        TK_TRY(cudaMemsetAsync(mc.fbits, 0, sizeof(uint32_t) * (size_t)nw, s));
        fiber_bits_kernel<<<grid_for((Z + 31) / 32 * 32), 256, 0, s>>>(Z, fcut, mc.fbits);
        ::tk::count_launch();
        TK_TRY(dev_alloc(c, &mc.unit_f0, (size_t)std::max<int64_t>(mc.n_units, 1)));
        if (mc.n_units > 0) {
          unit_fiber_kernel<<<grid_for(mc.n_units), 256, 0, s>>>(mc.n_units, mc.unit_e0, fcut, fcpos, mc.unit_f0);
          ::tk::count_launch();
        }
      }
      TK_TRY(cudaGetLastError());
      // a fiber unit spans about as many nonzeros as a nonzero unit (a fiber costs its
      // nonzeros plus one rank-1 update), in multiples of 32 fibers
      {
        const double per = (double)mc.chunk * (double)F / (double)Z;
        int fc = (int)(per / 32.0) * 32;
        mc.fchunk = std::max(64, std::min(2048, fc));
        const char *f = std::getenv("TUCKER_TTMC_FCHUNK");
        if (f) {
          const int v = std::atoi(f);
          if (v >= 32 && v <= (1 << 20) && (v % 32) == 0) mc.fchunk = v;
        }
      }
      UnitTables o{&mc.funit_e0, &mc.funit_k0, &mc.flong_k, &mc.flong_u0, &mc.flong_np, &mc.funit_slot,
                   &mc.fn_units, &mc.fn_long};
      st2 = build_units(c, mc.S, mc.fsptr, mc.fchunk, nu, islong, uoff, lid, stmp, d_small, o, s);
      if (st2 != TUCKER_OK) return st2;
    } else if (alt) {  // keep the re-sorted copy: the nonzero form does not depend on the order
      mc.fmid_t = 0;
    }
  }
  TK_TRY(cudaStreamSynchronize(s));
  return TUCKER_OK;
}

}  // namespace tk
