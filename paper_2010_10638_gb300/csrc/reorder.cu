// K-a: input validation, duplicate coalescing and the per-mode sorted copies.
//
// The paper stores the sparse tensor in COO form (Section III-A, Table I) and runs the
// Kronecker accumulation of Algorithm 2 over its nonzeros.  On the GPU every mode gets
// its own copy of the nonzeros sorted by that mode's index, so that the nonzeros of a
// slice (one row of Y_(n)) are contiguous and can be reduced without atomics:
//   - a stable radix sort of whole records (radix.cu) by the full coordinate, mode 1 most
//     significant, validating every coordinate and value on the way;
//   - equal neighbours are summed in FP64 (input order) into one nonzero;
//   - per mode: a stable radix sort of the coalesced records by i_n (the other modes'
//     indices, the value and the source position carried: structure of arrays), offsets
//     of the non-empty slices (a CSF root level), the list of empty rows, and a table of
//     work units of about `chunk` nonzeros: runs of whole short slices, or pieces of a
//     long slice whose partial rows are combined by a second pass;
//   - order 3: a fiber level (runs of one slice with one middle index, cut every
//     kFiberCap nonzeros) where fibers are few enough to pay.
// Positions where something starts (a group, a slice, a run) are numbered by per-tile
// counts, one block's prefix over the tiles, and a pass that writes the compacted lists.
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

cudaError_t pool_warm(int device) {
  cudaMemPool_t pool = nullptr;
  cudaError_t e = pool_for(device, &pool);
  if (e != cudaSuccess) return e;
  cudaStream_t s = nullptr;
  e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e != cudaSuccess) return e;
  void *p = nullptr;
  e = cudaMallocFromPoolAsync(&p, 1 << 20, pool, s);
  if (e == cudaSuccess) e = cudaFreeAsync(p, s);
  const cudaError_t e2 = cudaStreamSynchronize(s);
  cudaStreamDestroy(s);
  return e != cudaSuccess ? e : e2;
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

// ----------------------------------------------------------------------------- compaction
// Positions e of a sorted list where a predicate holds (a new nonzero, a new slice, a new
// fiber), numbered in order, in three launches and without flag or position arrays:
// per-tile counts, one block's exclusive prefix over the tiles, and a pass that evaluates the
// predicate again and hands (e, rank) to a writer.  A tile is 8192 positions: warp w of the
// block takes positions [512 w, 512 w + 512) of it in 16 steps of 32.
constexpr int kCpThreads = 512;
constexpr int kCpWarps = kCpThreads / 32;
constexpr int kCpSteps = 16;
constexpr int kCpTile = kCpWarps * kCpSteps * 32;

static int64_t cp_tiles(int64_t n) { return std::max<int64_t>(cdiv(n, kCpTile), 1); }

// Bit j of the result: the lane's position e0 + 32 j differs in word w from the position
// before it (positions >= n give 0).  The 16 loads are issued together; the previous
// position's word comes from the neighbour lane (lane 0 loads its own).
__device__ __forceinline__ uint32_t word_diff(const uint32_t *w, int64_t n, int64_t e0, int lane) {
  uint32_t c[kCpSteps], pl[kCpSteps];
#pragma unroll
  for (int j = 0; j < kCpSteps; ++j) {
    const int64_t e = e0 + j * 32;
    c[j] = e < n ? __ldg(w + e) : 0u;
  }
  if (lane == 0) {
#pragma unroll
    for (int j = 0; j < kCpSteps; ++j) {
      const int64_t e = e0 + j * 32;
      pl[j] = (e > 0 && e < n) ? __ldg(w + e - 1) : 0u;
    }
  }
  uint32_t diff = 0;
#pragma unroll
  for (int j = 0; j < kCpSteps; ++j) {
    uint32_t p = __shfl_up_sync(0xffffffffu, c[j], 1);
    if (lane == 0) p = pl[j];
    if (c[j] != p) diff |= 1u << j;
  }
  return diff;
}

// A position starts a run when it is the first, when one of the words differs from the
// previous position, or when its bit in `bits` is set.
struct ChangePred {
  int nw;
  int64_t n;
  const uint32_t *w[kMaxOrder];
  const uint32_t *bits;  // nullptr: none
};

// ballots of the 16 steps of this lane's warp: bit l of bal[j] = position e0 - lane + l + 32 j
// starts a run
__device__ __forceinline__ void change_ballots(const ChangePred &p, int64_t e0, int lane, uint32_t *bal) {
  uint32_t diff = 0;
  for (int m = 0; m < p.nw; ++m) diff |= word_diff(p.w[m], p.n, e0, lane);
  if (p.bits) {
#pragma unroll
    for (int j = 0; j < kCpSteps; ++j) {
      const int64_t e = e0 + j * 32;
      if (e < p.n && ((__ldg(p.bits + (e >> 5)) >> (e & 31)) & 1u)) diff |= 1u << j;
    }
  }
#pragma unroll
  for (int j = 0; j < kCpSteps; ++j) {
    const int64_t e = e0 + j * 32;
    bal[j] = __ballot_sync(0xffffffffu, e < p.n && (e == 0 || ((diff >> j) & 1u)));
  }
}

__global__ void __launch_bounds__(kCpThreads) tile_count_kernel(ChangePred pred, uint32_t *counts) {
  __shared__ uint32_t ws[kCpWarps];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t e0 = (int64_t)blockIdx.x * kCpTile + w * (kCpSteps * 32) + lane;
  uint32_t bal[kCpSteps];
  change_ballots(pred, e0, lane, bal);
  uint32_t c = 0;
#pragma unroll
  for (int j = 0; j < kCpSteps; ++j) c += (uint32_t)__popc(bal[j]);
  if (lane == 0) ws[w] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int i = 0; i < kCpWarps; ++i) t += ws[i];
    counts[blockIdx.x] = t;
  }
}

// one block of 1024 threads: exclusive prefix of the tile counts, and their total
__global__ void __launch_bounds__(1024) tile_prefix_kernel(const uint32_t *counts, int64_t nt, uint32_t *prefix,
                                                           uint32_t *total) {
  __shared__ uint32_t wsum[32];
  __shared__ uint32_t carry;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t c0 = 0; c0 < nt; c0 += 1024) {
    const int64_t i = c0 + threadIdx.x;
    const uint32_t v = i < nt ? counts[i] : 0u;
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
      const uint32_t x = wsum[lane];
      uint32_t xi = x;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, xi, o);
        if (lane >= o) xi += t;
      }
      wsum[lane] = xi - x;
    }
    __syncthreads();
    const uint32_t excl = carry + wsum[w] + incl - v;
    if (i < nt) prefix[i] = excl;
    __syncthreads();
    if (threadIdx.x == 1023) carry = excl + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

// Rank of the first run start of this warp in the whole list (bal[j] as from change_ballots);
// the rank of the lane's position at step j is that plus the run starts before it.
__device__ __forceinline__ uint32_t warp_rank0(const uint32_t *bal, const uint32_t *prefix, uint32_t *woff, int lane,
                                               int w) {
  uint32_t wc = 0;
#pragma unroll
  for (int j = 0; j < kCpSteps; ++j) wc += (uint32_t)__popc(bal[j]);
  if (lane == 0) woff[w] = wc;
  __syncthreads();
  if (w == 0) {
    const uint32_t x = lane < kCpWarps ? woff[lane] : 0u;
    uint32_t xi = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, xi, o);
      if (lane >= o) xi += t;
    }
    if (lane < kCpWarps) woff[lane] = xi - x;
  }
  __syncthreads();
  return prefix[blockIdx.x] + woff[w];
}

// hands every run start, with its rank, to the writer; sent[*sent_idx] = sent_val afterwards
// when sent != nullptr (a list's end marker)
template <class W>
__global__ void __launch_bounds__(kCpThreads) tile_compact_kernel(ChangePred pred, const uint32_t *prefix, W wr,
                                                                  uint32_t *sent, const uint32_t *sent_idx,
                                                                  uint32_t sent_val) {
  __shared__ uint32_t woff[kCpWarps];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t e0 = (int64_t)blockIdx.x * kCpTile + w * (kCpSteps * 32) + lane;
  uint32_t bal[kCpSteps];
  change_ballots(pred, e0, lane, bal);
  uint32_t r = warp_rank0(bal, prefix, woff, lane, w);
  const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
  for (int j = 0; j < kCpSteps; ++j) {
    if ((bal[j] >> lane) & 1u) wr(e0 + j * 32, r + (uint32_t)__popc(bal[j] & lt));
    r += (uint32_t)__popc(bal[j]);
  }
  if (sent && blockIdx.x == 0 && threadIdx.x == 0) sent[*sent_idx] = sent_val;
}

// One group of equal coordinates -> one nonzero at its rank: FP64 sum of its values in sorted
// (= input, the sort being stable) order; the squares of the sums, per tile, into part[tile].
// Coordinate m of sorted position e is pred.w[m][e]; a run start of pred is a group head.
__global__ void __launch_bounds__(kCpThreads, 1) coalesce_write_kernel(ChangePred pred, const float *vals,
                                                                   const uint32_t *prefix, int64_t nout,
                                                                   uint32_t *out_coords, float *out_vals,
                                                                   double *part) {
  __shared__ uint32_t woff[kCpWarps];
  __shared__ double wsq[kCpWarps];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t e0 = (int64_t)blockIdx.x * kCpTile + w * (kCpSteps * 32) + lane;
  const int64_t n = pred.n;
  uint32_t bal[kCpSteps];
  change_ballots(pred, e0, lane, bal);
  const uint32_t r0 = warp_rank0(bal, prefix, woff, lane, w);
  const uint32_t lt = (1u << lane) - 1u;
  for (int m = 0; m < pred.nw; ++m) {
    uint32_t c[kCpSteps];
#pragma unroll
    for (int j = 0; j < kCpSteps; ++j) c[j] = (e0 + j * 32 < n) ? __ldg(pred.w[m] + e0 + j * 32) : 0u;
    uint32_t r = r0;
#pragma unroll
    for (int j = 0; j < kCpSteps; ++j) {
      if ((bal[j] >> lane) & 1u) out_coords[(int64_t)m * nout + r + (uint32_t)__popc(bal[j] & lt)] = c[j];
      r += (uint32_t)__popc(bal[j]);
    }
  }
  float v[kCpSteps];
#pragma unroll
  for (int j = 0; j < kCpSteps; ++j) v[j] = (e0 + j * 32 < n) ? __ldg(vals + e0 + j * 32) : 0.0f;
  double acc = 0.0;
  uint32_t r = r0;
#pragma unroll
  for (int j = 0; j < kCpSteps; ++j) {
    const uint32_t rank = r + (uint32_t)__popc(bal[j] & lt);
    r += (uint32_t)__popc(bal[j]);
    if ((bal[j] >> lane) & 1u) {
      const int64_t e = e0 + j * 32;
      double sum = (double)v[j];
      // the next position starts a group when its bit says so (lane 31 of the warp's last
      // step looks at the positions after it directly)
      bool next_head;
      if (lane < 31) next_head = (bal[j] >> (lane + 1)) & 1u;
      else if (j + 1 < kCpSteps) next_head = bal[j + 1] & 1u;
      else next_head = false;
      if (e + 1 < n && !next_head) {
        for (int64_t e2 = e + 1; e2 < n; ++e2) {
          bool same = true;
          for (int m = 0; m < pred.nw; ++m) same = same && (pred.w[m][e2] == pred.w[m][e2 - 1]);
          if (!same) break;
          sum += (double)__ldg(vals + e2);
        }
      }
      out_vals[rank] = (float)sum;
      acc += sum * sum;
    }
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) wsq[w] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < kCpWarps; ++i) t += wsq[i];
    part[blockIdx.x] = t;
  }
}

struct SliceWrite {
  const uint32_t *row;
  uint32_t *sptr, *sid, *present;
  __device__ void operator()(int64_t e, uint32_t k) const {
    const uint32_t i = __ldg(row + e);
    sptr[k] = (uint32_t)e;
    sid[k] = i;
    present[i] = 1u;
  }
};

struct StartWrite {
  uint32_t *start;
  __device__ void operator()(int64_t e, uint32_t k) const { start[k] = (uint32_t)e; }
};

__global__ void reduce_f64_final(const double *part, int64_t np, double *out) {
  __shared__ double sm[256];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < np; i += blockDim.x) s += part[i];
  sm[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sm[0];
}

// ----------------------------------------------------------------------------- per-mode copies
__global__ void invert_flag_kernel(int64_t n, const uint32_t *present, uint32_t *absent) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    absent[i] = present[i] ? 0u : 1u;
}

__global__ void compact_kernel(int64_t n, const uint32_t *flag, const uint32_t *pos, uint32_t *out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (flag[i]) out[pos[i]] = (uint32_t)i;
}

// Slice starts per tile; with mid != nullptr also the runs of equal (row, mid) pairs, added
// to *runs.
__global__ void __launch_bounds__(kCpThreads) slice_count_kernel(int64_t n, const uint32_t *row,
                                                                 const uint32_t *mid, uint32_t *counts,
                                                                 uint32_t *runs) {
  __shared__ uint32_t ws[kCpWarps], wr[kCpWarps];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t e0 = (int64_t)blockIdx.x * kCpTile + w * (kCpSteps * 32) + lane;
  const uint32_t dr = word_diff(row, n, e0, lane);
  const uint32_t dm = mid ? word_diff(mid, n, e0, lane) : 0u;
  uint32_t cs = 0, cr = 0;
#pragma unroll
  for (int j = 0; j < kCpSteps; ++j) {
    const int64_t e = e0 + j * 32;
    const bool valid = e < n;
    const bool ns = valid && (e == 0 || ((dr >> j) & 1u));
    cs += (uint32_t)__popc(__ballot_sync(0xffffffffu, ns));
    cr += (uint32_t)__popc(__ballot_sync(0xffffffffu, ns || (valid && ((dm >> j) & 1u))));
  }
  if (lane == 0) {
    ws[w] = cs;
    wr[w] = cr;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0, u = 0;
    for (int i = 0; i < kCpWarps; ++i) {
      t += ws[i];
      u += wr[i];
    }
    counts[blockIdx.x] = t;
    if (mid && u) atomicAdd(runs, u);
  }
}

// ---- fibers (order 3): runs of one slice with one index of the middle mode (the middle
//      level of a CSF tree), cut every `cap` nonzeros.  Run r starts at rstart[r]
//      (rstart[nrun] = n); it becomes ceil(len / cap) fibers, the first at poff[r].
__global__ void slice_bits_kernel(int64_t S, const uint32_t *sptr, uint32_t *bits) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < S; k += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t e = sptr[k];
    atomicOr(bits + (e >> 5), 1u << (e & 31));
  }
}

__global__ void run_pieces_kernel(int64_t nrun, const uint32_t *rstart, uint32_t cap, uint32_t *pieces) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nrun; r += (int64_t)gridDim.x * blockDim.x)
    pieces[r] = (rstart[r + 1] - rstart[r] + cap - 1) / cap;
}

// fiber starts, middle indices and the start bit mask of every run's first kRunPieces
// fibers (fptr[F] = n); runs with more pieces are listed for fiber_emit_long_kernel
constexpr uint32_t kRunPieces = 32;
__global__ void fiber_emit_kernel(int64_t nrun, const uint32_t *rstart, const uint32_t *poff, const uint32_t *mid,
                                  uint32_t cap, uint32_t *fptr, uint32_t *fmid, uint32_t *fbits, uint32_t *long_list,
                                  uint32_t *long_count, uint32_t F, uint32_t n) {
  if (blockIdx.x == 0 && threadIdx.x == 0) fptr[F] = n;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nrun; r += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t s0 = rstart[r], len = rstart[r + 1] - s0, f0 = poff[r], m = mid[s0];
    const uint32_t np = (len + cap - 1) / cap;
    for (uint32_t p = 0; p < np && p < kRunPieces; ++p) {
      const uint32_t e = s0 + p * cap;
      fptr[f0 + p] = e;
      fmid[f0 + p] = m;
      atomicOr(fbits + (e >> 5), 1u << (e & 31));
    }
    if (np > kRunPieces) long_list[atomicAdd(long_count, 1u)] = (uint32_t)r;
  }
}

// the remaining fibers of the long runs, one block per run at a time
__global__ void fiber_emit_long_kernel(const uint32_t *long_list, const uint32_t *long_count, const uint32_t *rstart,
                                       const uint32_t *poff, const uint32_t *mid, uint32_t cap, uint32_t *fptr,
                                       uint32_t *fmid, uint32_t *fbits) {
  const uint32_t nl = *long_count;
  for (uint32_t i = blockIdx.x; i < nl; i += gridDim.x) {
    const uint32_t r = long_list[i];
    const uint32_t s0 = rstart[r], len = rstart[r + 1] - s0, f0 = poff[r], m = mid[s0];
    const uint32_t np = (len + cap - 1) / cap;
    for (uint32_t p = kRunPieces + threadIdx.x; p < np; p += blockDim.x) {
      const uint32_t e = s0 + p * cap;
      fptr[f0 + p] = e;
      fmid[f0 + p] = m;
      atomicOr(fbits + (e >> 5), 1u << (e & 31));
    }
  }
}

// largest f < F with fptr[f] <= e (fptr ascending, fptr[0] = 0 <= e)
__device__ __forceinline__ uint32_t fiber_of(const uint32_t *fptr, uint32_t F, uint32_t e) {
  uint32_t lo = 0, hi = F;  // fptr[lo] <= e < fptr[hi] (fptr[F] = n)
  while (hi - lo > 1) {
    const uint32_t mid = lo + (hi - lo) / 2;
    if (fptr[mid] <= e) lo = mid;
    else hi = mid;
  }
  return lo;
}

// first fiber of every slice (a slice start is a fiber start), fsptr[S] = F
__global__ void fiber_slices_kernel(int64_t S, const uint32_t *sptr, const uint32_t *fptr, uint32_t F,
                                    uint32_t *fsptr) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < S; k += (int64_t)gridDim.x * blockDim.x) {
    fsptr[k] = fiber_of(fptr, F, sptr[k]);
    if (k == 0) fsptr[S] = F;
  }
}

// fiber containing the first position of each nonzero work unit
__global__ void unit_fiber_kernel(int64_t n_units, const uint32_t *unit_e0, const uint32_t *fptr, uint32_t F,
                                  uint32_t *unit_f0) {
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n_units; u += (int64_t)gridDim.x * blockDim.x)
    unit_f0[u] = fiber_of(fptr, F, unit_e0[u]);
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
    if (islong[k]) {  // its pieces: unit_long_kernel
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

// the units of the long slices, one block per slice at a time
__global__ void unit_long_kernel(int64_t n_long, const uint32_t *long_k, const uint32_t *long_u0,
                                 const uint32_t *long_np, const uint32_t *sptr, uint32_t chunk, uint32_t *unit_e0,
                                 uint32_t *unit_k0, int32_t *unit_slot) {
  for (int64_t l = blockIdx.x; l < n_long; l += gridDim.x) {
    const uint32_t k = long_k[l], u0 = long_u0[l], np = long_np[l], e0 = sptr[k];
    for (uint32_t p = threadIdx.x; p < np; p += blockDim.x) {
      unit_e0[u0 + p] = e0 + p * chunk;
      unit_k0[u0 + p] = k;
      unit_slot[u0 + p] = (int32_t)(u0 + p);
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
    if (nlong > 0) {
      unit_long_kernel<<<(unsigned)std::min<uint32_t>(nlong, (uint32_t)c->num_sms * 4), 256, 0, s>>>(
          nlong, *o.long_k, *o.long_u0, *o.long_np, ptr, (uint32_t)chunk, *o.e0, *o.k0, *o.slot);
      ::tk::count_launch();
    }
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

cudaError_t preload_reorder_kernels() {
  cudaFuncAttributes fa;
  cudaError_t e = cudaSuccess;
  const void *k[] = {
      reinterpret_cast<const void *>(scan_block_kernel),
      reinterpret_cast<const void *>(scan_add_kernel),
      reinterpret_cast<const void *>(tile_count_kernel),
      reinterpret_cast<const void *>(tile_prefix_kernel),
      reinterpret_cast<const void *>(tile_compact_kernel<SliceWrite>),
      reinterpret_cast<const void *>(tile_compact_kernel<StartWrite>),
      reinterpret_cast<const void *>(coalesce_write_kernel),
      reinterpret_cast<const void *>(reduce_f64_final),
      reinterpret_cast<const void *>(invert_flag_kernel),
      reinterpret_cast<const void *>(compact_kernel),
      reinterpret_cast<const void *>(slice_count_kernel),
      reinterpret_cast<const void *>(slice_bits_kernel),
      reinterpret_cast<const void *>(run_pieces_kernel),
      reinterpret_cast<const void *>(fiber_emit_kernel),
      reinterpret_cast<const void *>(fiber_emit_long_kernel),
      reinterpret_cast<const void *>(fiber_slices_kernel),
      reinterpret_cast<const void *>(unit_fiber_kernel),
      reinterpret_cast<const void *>(unit_count_kernel),
      reinterpret_cast<const void *>(unit_write_kernel),
      reinterpret_cast<const void *>(unit_long_kernel),
  };
  for (const void *f : k)
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, f);
  return e;
}

// Reads a device total and the error word in one synchronisation; a set error bit ends the
// initialisation (the sorted words may be wrong and must not be used as indices).
static tucker_status read_checked(Ctx *c, const uint32_t *d, uint32_t *h, cudaStream_t s) {
  uint32_t err = 0;
  TK_TRY(cudaMemcpyAsync(h, d, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  TK_TRY(cudaMemcpyAsync(&err, c->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  TK_TRY(cudaStreamSynchronize(s));
  if (err) {
    TK_TRY(cudaMemsetAsync(c->d_err, 0, sizeof(uint32_t), s));
    if (err & kErrTimeout) {
      c->last_error = "a bounded wait of the radix sort gave up";
      return TUCKER_ETIMEOUT;
    }
    c->last_error = (err & kErrCoord) ? "a coordinate is >= its dimension" : "a value is not finite";
    return TUCKER_EINVAL;
  }
  return TUCKER_OK;
}

static tucker_status sort_records(Ctx *c, int64_t n, const RadixRecords &r, const RadixKey *keys, int nkeys,
                                  const int64_t *dims, int nvalid, const float *vals, void *scratch, size_t bytes,
                                  cudaStream_t s) {
  const int rc = radix_sort_records(n, r, keys, nkeys, dims, nvalid, vals, scratch, bytes, c->d_err, s);
  if (rc == -1) {
    c->last_error = "radix sort: bad plan";
    return TUCKER_EINVAL;
  }
  TK_TRY(cudaGetLastError());
  if (rc != 0) {
    c->last_error = "radix sort: a CUDA call failed";
    return TUCKER_ECUDA;
  }
  return TUCKER_OK;
}

tucker_status build_sorted_copies(Ctx *c, const uint32_t *coords_in, const float *vals_in, cudaStream_t s) {
  const int N = c->N;
  const int64_t n_in = c->nnz_in;
  Temps tmp(c);
  int64_t *d_dims = nullptr;
  uint32_t *d_small = nullptr;  // [0..15] totals read back to the host
  TK_TRY(tmp.get(&d_dims, kMaxOrder));
  TK_TRY(tmp.get(&d_small, 16));
  TK_TRY(cudaMemcpyAsync(d_dims, c->dims, sizeof(int64_t) * kMaxOrder, cudaMemcpyHostToDevice, s));
  TK_TRY(cudaMemsetAsync(c->d_err, 0, sizeof(uint32_t), s));
  TK_TRY(cudaMemsetAsync(d_small, 0, sizeof(uint32_t) * 16, s));

  const int64_t nmax = std::max<int64_t>(n_in, 1);
  int64_t maxI = 1;
  for (int m = 0; m < N; ++m) maxI = std::max(maxI, c->dims[m]);

  // ---- sort plans: the full key (mode 1 most significant; every coordinate and the value
  //      carried) and the per-mode keys (index, the other coordinates, value, source position).
  //      With fiber levels (order 3) the full key of mode 1 orders its other two modes with the
  //      smaller one first: that one is likely to be mode 1's better middle level (fewer
  //      runs), and then mode 1's copy needs no second sort.  The copies of modes 2 and 3 are
  //      the same either way (each is a stable sort by its own index).
  const int fp = (N == 3) ? fiber_policy() : 0;
  const int mid0 = (fp != 0 && c->dims[2] < c->dims[1]) ? 2 : 1;  // mode 1's middle in this order
  RadixKey fkeys[kMaxOrder];
  for (int k = 0; k < N; ++k) fkeys[k] = RadixKey{N - 1 - k, radix_bits(c->dims[N - 1 - k] - 1)};
  if (N == 3 && mid0 == 2) {  // key (i_1, i_3, i_2)
    fkeys[0] = RadixKey{1, radix_bits(c->dims[1] - 1)};
    fkeys[1] = RadixKey{2, radix_bits(c->dims[2] - 1)};
  }
  size_t sbytes = radix_scratch_bytes(n_in, N + 1, fkeys, N);
  for (int m = 0; m < N; ++m) {
    const RadixKey mk{0, radix_bits(c->dims[m] - 1)};
    sbytes = std::max(sbytes, radix_scratch_bytes(n_in, N + 2, &mk, 1));
  }
  // the fiber levels' temporaries share the scratch: run starts, pieces, offsets, long runs
  if (N == 3) sbytes = std::max(sbytes, sizeof(uint32_t) * (4 * (size_t)nmax + 8) + 4096);
  void *scratch = nullptr;
  TK_TRY(tmp.get(reinterpret_cast<uint8_t **>(&scratch), sbytes));
  const int64_t ntiles = cp_tiles(nmax);
  uint32_t *stmp, *flag, *pos, *present, *counts, *prefix;
  TK_TRY(tmp.get(&stmp, scan_tmp_elems(std::max<int64_t>(nmax, maxI + 1))));
  TK_TRY(tmp.get(&flag, maxI + 1));
  TK_TRY(tmp.get(&pos, maxI + 1));
  TK_TRY(tmp.get(&present, maxI + 1));
  TK_TRY(tmp.get(&counts, ntiles));
  TK_TRY(tmp.get(&prefix, ntiles));

  // ---- full-key sort (+ validation of every coordinate and value)
  uint32_t *fs = nullptr;  // sorted words: coordinates 0..N-1, then the values
  TK_TRY(tmp.get(&fs, (size_t)nmax * (N + 1)));
  uint32_t nout = 0;
  ChangePred head{};  // groups of equal coordinates in the sorted words
  head.nw = N;
  head.n = n_in;
  for (int m = 0; m < N; ++m) head.w[m] = fs + (int64_t)m * n_in;
  if (n_in > 0) {
    RadixRecords fr;
    fr.nwords = N + 1;
    for (int m = 0; m < N; ++m) fr.in[m] = coords_in + (int64_t)m * n_in;
    fr.in[N] = reinterpret_cast<const uint32_t *>(vals_in);
    for (int q = 0; q <= N; ++q) fr.out[q] = fs + (int64_t)q * n_in;
    tucker_status st = sort_records(c, n_in, fr, fkeys, N, d_dims, N, vals_in, scratch, sbytes, s);
    if (st != TUCKER_OK) return st;
    // ---- coalesce duplicates: count the groups of equal coordinates
    tile_count_kernel<<<(unsigned)cp_tiles(n_in), kCpThreads, 0, s>>>(head, counts);
    ::tk::count_launch();
    tile_prefix_kernel<<<1, 1024, 0, s>>>(counts, cp_tiles(n_in), prefix, d_small);
    ::tk::count_launch();
    st = read_checked(c, d_small, &nout, s);  // also the validation and the sort's waits
    if (st != TUCKER_OK) return st;
  }
  c->nnz = nout;
  const int64_t Z = nout;
  TK_TRY(dev_alloc(c, &c->coords, (size_t)std::max<int64_t>(Z, 1) * N));
  TK_TRY(dev_alloc(c, &c->vals, (size_t)std::max<int64_t>(Z, 1)));
  c->norm2 = 0.0;
  if (n_in > 0) {
    double *part = nullptr;
    TK_TRY(tmp.get(&part, cp_tiles(n_in)));
    coalesce_write_kernel<<<(unsigned)cp_tiles(n_in), kCpThreads, 0, s>>>(
        head, reinterpret_cast<const float *>(fs + (int64_t)N * n_in), prefix, Z, c->coords, c->vals, part);
    ::tk::count_launch();
    reduce_f64_final<<<1, 256, 0, s>>>(part, cp_tiles(n_in), c->norm_dev);
    ::tk::count_launch();
    TK_TRY(cudaGetLastError());
    TK_TRY(cudaMemcpyAsync(&c->norm2, c->norm_dev, sizeof(double), cudaMemcpyDeviceToHost, s));
  } else {
    TK_TRY(cudaMemsetAsync(c->norm_dev, 0, sizeof(double), s));
  }

  // ---- per-mode sorted copies
  uint32_t *nu = nullptr, *islong = nullptr, *uoff = nullptr, *lid = nullptr;  // per slice
  TK_TRY(tmp.get(&nu, maxI + 1));
  TK_TRY(tmp.get(&islong, maxI + 1));
  TK_TRY(tmp.get(&uoff, maxI + 1));
  TK_TRY(tmp.get(&lid, maxI + 1));
  const uint32_t *rows[kMaxOrder] = {};  // sorted index of each mode's copy, while it is held
  uint32_t *rowbuf = nullptr, *rowbuf2 = nullptr;  // the sorted modes' indices (with fiber
  TK_TRY(tmp.get(&rowbuf, (size_t)std::max<int64_t>(Z, 1)));  // levels modes 2 and 3 keep theirs)
  if (N == 3 && fp != 0) TK_TRY(tmp.get(&rowbuf2, (size_t)std::max<int64_t>(Z, 1)));
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
    if (n == 0) {  // the lexicographic order is already sorted by i_1: mode 1 reads the
                   // coalesced arrays themselves (read-only after the initialisation)
      rows[0] = c->coords;
      for (int q = 0; q < mc.nother; ++q) mc.idx[q] = c->coords + (int64_t)mc.other[q] * Z;
      mc.val = c->vals;
    } else {
      for (int q = 0; q < mc.nother; ++q) TK_TRY(dev_alloc(c, &mc.idx[q], (size_t)std::max<int64_t>(Z, 1)));
      TK_TRY(dev_alloc(c, &mc.val, (size_t)std::max<int64_t>(Z, 1)));
    }
    uint32_t *rb = (rowbuf2 && n == 2) ? rowbuf2 : rowbuf;
    if (n > 0 && Z > 0) {
      for (int m = 1; m < n; ++m)
        if (rows[m] == rb) rows[m] = nullptr;  // overwritten below
      TK_TRY(dev_alloc(c, &mc.src, (size_t)Z));
      RadixRecords mr;
      mr.nwords = N + 2;
      mr.in[0] = c->coords + (int64_t)n * Z;
      mr.out[0] = rb;
      for (int q = 0; q < mc.nother; ++q) {
        mr.in[1 + q] = c->coords + (int64_t)mc.other[q] * Z;
        mr.out[1 + q] = mc.idx[q];
      }
      mr.in[N] = reinterpret_cast<const uint32_t *>(c->vals);
      mr.out[N] = reinterpret_cast<uint32_t *>(mc.val);
      mr.in[N + 1] = nullptr;  // source position in the lexicographic order
      mr.out[N + 1] = mc.src;
      const RadixKey mk{0, radix_bits(mc.I - 1)};
      tucker_status st = sort_records(c, Z, mr, &mk, 1, nullptr, 0, nullptr, scratch, sbytes, s);
      if (st != TUCKER_OK) return st;
      rows[n] = rb;
    }
    const uint32_t *row = rows[n];
    // slices: count, then sptr / sid / present written directly
    uint32_t S = 0;
    ChangePred rp{};
    rp.nw = 1;
    rp.n = Z;
    rp.w[0] = row;
    if (Z > 0) {  // modes 2, 3 (order 3): with the runs of (i_n, i_1) pairs
      slice_count_kernel<<<(unsigned)cp_tiles(Z), kCpThreads, 0, s>>>(Z, row, (fp != 0 && n > 0) ? mc.idx[0] : nullptr,
                                                                      counts, d_small + 8 + n);
      ::tk::count_launch();
      tile_prefix_kernel<<<1, 1024, 0, s>>>(counts, cp_tiles(Z), prefix, d_small);
      ::tk::count_launch();
      tucker_status st = read_checked(c, d_small, &S, s);  // also before rows are used as indices
      if (st != TUCKER_OK) return st;
    }
    mc.S = S;
    TK_TRY(dev_alloc(c, &mc.sptr, (size_t)S + 1));
    TK_TRY(dev_alloc(c, &mc.sid, (size_t)std::max<uint32_t>(S, 1)));
    TK_TRY(cudaMemsetAsync(present, 0, sizeof(uint32_t) * (size_t)mc.I, s));
    if (Z > 0) {
      const SliceWrite sw{row, mc.sptr, mc.sid, present};
      tile_compact_kernel<<<(unsigned)cp_tiles(Z), kCpThreads, 0, s>>>(rp, prefix, sw, mc.sptr, d_small, (uint32_t)Z);
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
  }
  uint32_t fnat[kMaxOrder] = {};  // modes 2, 3: runs of (i_n, i_1) = distinct (i_1, i_n) pairs
  if (fp != 0 && Z > 0) {
    TK_TRY(cudaMemcpyAsync(fnat, d_small + 8, sizeof(uint32_t) * N, cudaMemcpyDeviceToHost, s));
    TK_TRY(cudaStreamSynchronize(s));
  }

  // ---- fiber levels (order 3).  The middle level of modes 2 and 3 is mode 1.  That of mode
  //      1 is mode 3 when it has at most 0.8 times as many distinct (i_1, i_3) pairs as
  //      (i_1, i_2) pairs, else mode 2; when that is not the middle of mode 1's copy, the copy
  //      is re-sorted by a stable sort of the chosen mode's copy by i_1 (slices and nonzero
  //      units are unchanged).
  //      The temporaries live in the sort scratch: a re-sort runs before its mode's fiber
  //      level is built, and in stream order after the previous mode's was.
  uint32_t *rstart = static_cast<uint32_t *>(scratch);  // [nrun + 1] run starts
  uint32_t *pieces = rstart + (Z + 1);                   // [nrun] fibers per run
  uint32_t *poff = pieces + Z;                           // [nrun] first fiber of each run
  uint32_t *long_list = poff + Z;                        // [nrun] runs of more than kRunPieces fibers
  uint32_t *sbits = nullptr;                             // slice starts as a bit mask
  uint32_t cap = (uint32_t)kFiberCap;
  if (const char *fc = std::getenv("TUCKER_TTMC_FIBER_CAP")) {
    const int v = std::atoi(fc);
    if (v >= 1 && v <= kFiberCap) cap = (uint32_t)v;
  }
  if (N == 3 && Z > 0 && fp != 0) TK_TRY(tmp.get(&sbits, (size_t)(Z / 32 + 2)));
  for (int n = 0; n < N && N == 3 && Z > 0 && fp != 0; ++n) {
    ModeCopy &mc = c->mode[n];
    if (mc.S == 0) continue;
    int mid_mode = mc.other[0];  // modes 2, 3: mode 1
    bool resorted = false;
    if (n == 0) {
      mid_mode = (fnat[1] > 0 && fnat[2] > 0 && (double)fnat[2] <= 0.8 * (double)fnat[1]) ? 2 : 1;
      if (mid_mode != mid0 && rows[mid_mode] && c->mode[mid_mode].src) {
        // (i_1, i_p, i_r) from the copy of p = mid_mode, grouped by (i_p, i_1, i_r)
        const ModeCopy &mb = c->mode[mid_mode];
        for (int q = 0; q < mc.nother; ++q) TK_TRY(dev_alloc(c, &mc.idx[q], (size_t)Z));
        TK_TRY(dev_alloc(c, &mc.val, (size_t)Z));
        TK_TRY(dev_alloc(c, &mc.src, (size_t)Z));
        uint32_t *keys_out = nullptr;  // the sorted i_1 is not kept
        TK_TRY(tmp.get(&keys_out, (size_t)Z));
        RadixRecords ar;
        ar.nwords = 5;
        ar.in[0] = mb.idx[0];  // i_1: the key
        ar.out[0] = keys_out;
        ar.in[1] = rows[mid_mode];  // i_p
        ar.out[1] = mc.idx[mid_mode - 1];
        ar.in[2] = mb.idx[1];  // i_r
        ar.out[2] = mc.idx[2 - mid_mode];
        ar.in[3] = reinterpret_cast<const uint32_t *>(mb.val);
        ar.out[3] = reinterpret_cast<uint32_t *>(mc.val);
        ar.in[4] = mb.src;
        ar.out[4] = mc.src;
        const RadixKey ak{0, radix_bits(mc.I - 1)};
        tucker_status st = sort_records(c, Z, ar, &ak, 1, nullptr, 0, nullptr, scratch, sbytes, s);
        if (st != TUCKER_OK) return st;
        dev_release(c, keys_out);
        tmp.ptrs.pop_back();
        resorted = true;
      } else if (mid_mode != mid0) {
        mid_mode = mid0;
      }
    }
    const int ft = mid_mode == mc.other[0] ? 0 : 1;
    const uint32_t *mid = mc.idx[ft];
    // runs of (slice, middle index): slice starts as a bit mask, then the runs' starts
    TK_TRY(cudaMemsetAsync(sbits, 0, sizeof(uint32_t) * (size_t)(Z / 32 + 2), s));
    slice_bits_kernel<<<grid_for(mc.S), 256, 0, s>>>(mc.S, mc.sptr, sbits);
    ::tk::count_launch();
    ChangePred rp{};
    rp.nw = 1;
    rp.n = Z;
    rp.w[0] = mid;
    rp.bits = sbits;
    tile_count_kernel<<<(unsigned)cp_tiles(Z), kCpThreads, 0, s>>>(rp, counts);
    ::tk::count_launch();
    tile_prefix_kernel<<<1, 1024, 0, s>>>(counts, cp_tiles(Z), prefix, d_small + 4);
    ::tk::count_launch();
    tile_compact_kernel<<<(unsigned)cp_tiles(Z), kCpThreads, 0, s>>>(rp, prefix, StartWrite{rstart}, rstart,
                                                                      d_small + 4, (uint32_t)Z);
    ::tk::count_launch();
    uint32_t nrun = 0;
    tucker_status st2 = read_checked(c, d_small + 4, &nrun, s);
    if (st2 != TUCKER_OK) return st2;
    // fibers: runs cut every `cap` nonzeros
    run_pieces_kernel<<<grid_for(nrun), 256, 0, s>>>(nrun, rstart, cap, pieces);
    ::tk::count_launch();
    exclusive_scan_total(pieces, poff, nrun, stmp, d_small + 5, s);
    uint32_t F = 0;
    st2 = read_checked(c, d_small + 5, &F, s);
    if (st2 != TUCKER_OK) return st2;
    if (fp == 1 || (double)F <= kFiberShare * (double)Z) {
      mc.fib = true;
      mc.fmid_t = ft;
      mc.F = F;
      TK_TRY(dev_alloc(c, &mc.fptr, (size_t)F + 1));
      TK_TRY(dev_alloc(c, &mc.fmid, (size_t)std::max<uint32_t>(F, 1)));
      TK_TRY(dev_alloc(c, &mc.fsptr, (size_t)mc.S + 1));
      // fiber starts as a bit mask over the sorted positions, three zero words past the end
      const int64_t nw = (Z + 31) / 32 + 3;
      TK_TRY(dev_alloc(c, &mc.fbits, (size_t)nw));
      TK_TRY(cudaMemsetAsync(mc.fbits, 0, sizeof(uint32_t) * (size_t)nw, s));
      TK_TRY(cudaMemsetAsync(d_small + 6, 0, sizeof(uint32_t), s));
      fiber_emit_kernel<<<std::min<unsigned>(grid_for(nrun), (unsigned)c->num_sms * 8), 256, 0, s>>>(
          nrun, rstart, poff, mid, cap, mc.fptr, mc.fmid, mc.fbits, long_list, d_small + 6, F, (uint32_t)Z);
      ::tk::count_launch();
      fiber_emit_long_kernel<<<(unsigned)c->num_sms * 2, 256, 0, s>>>(long_list, d_small + 6, rstart, poff, mid, cap,
                                                                      mc.fptr, mc.fmid, mc.fbits);
      ::tk::count_launch();
      fiber_slices_kernel<<<grid_for(mc.S), 256, 0, s>>>(mc.S, mc.sptr, mc.fptr, F, mc.fsptr);
      ::tk::count_launch();
      TK_TRY(dev_alloc(c, &mc.unit_f0, (size_t)std::max<int64_t>(mc.n_units, 1)));
      if (mc.n_units > 0) {
        unit_fiber_kernel<<<grid_for(mc.n_units), 256, 0, s>>>(mc.n_units, mc.unit_e0, mc.fptr, F, mc.unit_f0);
        ::tk::count_launch();
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
    } else {  // the nonzero form does not depend on the order within a slice
      mc.fmid_t = 0;
      (void)resorted;
    }
  }
  TK_TRY(cudaStreamSynchronize(s));
  return TUCKER_OK;
}

}  // namespace tk
