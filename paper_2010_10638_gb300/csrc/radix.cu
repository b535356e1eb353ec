// Stable LSD radix sort of records held as structure-of-arrays of 32-bit words (the
// coordinates, values and source positions of the nonzeros; Section III-A's COO list),
// used by the initialisation to build the sorted copies of the tensor.
//
// A record is carried whole through every pass, so no pass reads through a permutation:
//   1. one histogram kernel counts the first pass's digits and optionally validates the
//      input; every pass counts the next pass's digits while it moves the records (a digit's
//      global count does not depend on the order of the records);
//   2. one kernel per pass: each block claims the next tile of 8192 records and ranks them
//      by digit (peer lanes of equal digit found by one ballot per digit bit; stable),
//      publishes its digit counts, finds the counts of all earlier tiles by a decoupled
//      look-back over a per-tile status word, and writes every word of the tile out in
//      digit order through shared memory, so that the stores of a warp fall into a few
//      contiguous runs.
// Look-back waits are bounded: a block that gives up sets kErrTimeout in the error word,
// publishes a (wrong) prefix so that later tiles do not wait on it, and writes nothing; every
// store is also checked against n.  Callers read the error word before using the sorted
// words as indices.
#include <algorithm>

#include "internal.cuh"

namespace tk {

constexpr int kRxThreads = 512;
constexpr int kRxWarps = kRxThreads / 32;
constexpr int kRxSteps = 16;                         // 32-record steps per warp
constexpr int kRxTile = kRxWarps * kRxSteps * 32;    // 8192 records per tile
constexpr int kRxBins = 256;                         // digits of at most 8 bits
constexpr int kRxMaxPasses = 4 * kMaxOrder + 4;
constexpr uint64_t kRxFlagAgg = 1ull << 32;          // status: this tile's own counts
constexpr uint64_t kRxFlagPre = 2ull << 32;          // status: inclusive prefix over tiles
constexpr uint32_t kRxSpin = 1u << 22;               // polls of one status word at most

// Lanes of the warp whose digit equals this lane's (bits-wide digits), among `active`:
// one ballot per digit bit.
__device__ __forceinline__ uint32_t rx_peers(uint32_t d, int bits, uint32_t active) {
  uint32_t m = active;
  for (int b = 0; b < bits; ++b) {
    const uint32_t x = __ballot_sync(0xffffffffu, (d >> b) & 1u);
    m &= ((d >> b) & 1u) ? x : ~x;
  }
  return m;
}

struct RxPass {
  int word, shift, bits;
};

struct RxHistWord {
  int word;   // the word read
  int np;     // passes keyed on it (0: read for validation only)
  int p0;     // index of its first pass
  int shift[4], bits[4];
};

struct RxHistArgs {
  int64_t n;
  int npass, nkw;
  RxHistWord kw[kRadixMaxWords];
  const uint32_t *src[kRadixMaxWords];  // the words
  const int64_t *dims;                  // validation: word w must be < dims[w] (w < nvalid)
  int nvalid;
  const float *vals;                    // validation: finite (nullptr: none)
  uint32_t *hist;                       // [npass][256], zeroed by the caller
  uint32_t *err;
};

constexpr int kRxHistThreads = 512;
constexpr int kRxHistItems = 8;  // records per thread per round: their loads are in flight together

// Digit counts of every pass; with validation, coordinates >= their dimension and
// non-finite values set bits of *err (digits are masked, so the sort stays in bounds).
// Equal digits of a warp are counted once by their lowest lane (ballot match), so skewed
// digits cause no shared-memory atomic conflicts.
__global__ void __launch_bounds__(kRxHistThreads) rx_hist_kernel(RxHistArgs a) {
  extern __shared__ uint32_t sh[];  // [npass][256]
  __shared__ int64_t dims[kRadixMaxWords];
  for (int i = threadIdx.x; i < a.npass * kRxBins; i += blockDim.x) sh[i] = 0;
  if (threadIdx.x < a.nvalid) dims[threadIdx.x] = a.dims[threadIdx.x];
  __syncthreads();
  uint32_t bad = 0;
  const int lane = threadIdx.x & 31;
  const int64_t round = (int64_t)kRxHistThreads * kRxHistItems;
  // rounds are block-uniform, so every lane of a warp reaches each match
  for (int64_t r0 = (int64_t)blockIdx.x * round; r0 < a.n; r0 += (int64_t)gridDim.x * round) {
    const int64_t e0 = r0 + threadIdx.x;
    for (int q = 0; q < a.nkw; ++q) {
      const uint32_t *src = a.src[a.kw[q].word];
      uint32_t k[kRxHistItems];
#pragma unroll
      for (int j = 0; j < kRxHistItems; ++j) {
        const int64_t e = e0 + (int64_t)j * kRxHistThreads;
        k[j] = e < a.n ? __ldg(src + e) : 0u;
      }
      const int np = a.kw[q].np, p0 = a.kw[q].p0, wq = a.kw[q].word;
#pragma unroll
      for (int j = 0; j < kRxHistItems; ++j) {
        const bool valid = e0 + (int64_t)j * kRxHistThreads < a.n;
        const uint32_t active = __ballot_sync(0xffffffffu, valid);
        for (int p = 0; p < np; ++p) {
          const int bits = a.kw[q].bits[p];
          const uint32_t d = (k[j] >> a.kw[q].shift[p]) & ((1u << bits) - 1u);
          const uint32_t peers = rx_peers(d, bits, active);
          if (valid && lane == __ffs(peers) - 1) atomicAdd(&sh[(p0 + p) * kRxBins + d], (uint32_t)__popc(peers));
        }
        if (valid && wq < a.nvalid && (int64_t)k[j] >= dims[wq]) bad |= kErrCoord;
      }
    }
    if (a.vals) {
      float v[kRxHistItems];
#pragma unroll
      for (int j = 0; j < kRxHistItems; ++j) {
        const int64_t e = e0 + (int64_t)j * kRxHistThreads;
        v[j] = e < a.n ? __ldg(a.vals + e) : 0.0f;
      }
#pragma unroll
      for (int j = 0; j < kRxHistItems; ++j)
        if (!isfinite(v[j])) bad |= kErrValue;
    }
  }
  bad = __reduce_or_sync(0xffffffffu, bad);
  if (lane == 0 && bad) atomicOr(a.err, bad);
  __syncthreads();
  for (int i = threadIdx.x; i < a.npass * kRxBins; i += blockDim.x)
    if (sh[i]) atomicAdd(&a.hist[i], sh[i]);
}

struct RxPassArgs {
  int64_t n;
  int nwords, key_word, shift, bits;
  const uint32_t *in[kRadixMaxWords];  // nullptr: the word is the record's input position
  uint32_t *out[kRadixMaxWords];
  const uint32_t *hist;                // [256] global digit counts of this pass
  uint32_t *next_hist;                 // [256] counts of the next pass's digits (nullptr: last pass)
  int next_word, next_shift, next_bits;
  unsigned long long *status;          // [tiles][256], zeroed
  uint32_t *tile_ctr;                  // zeroed
  uint32_t *err;
  uint32_t spin;                       // polls of one status word at most
};

__device__ __forceinline__ unsigned long long rx_load(const unsigned long long *p) {
  return *reinterpret_cast<const volatile unsigned long long *>(p);
}
__device__ __forceinline__ void rx_store(unsigned long long *p, unsigned long long v) {
  *reinterpret_cast<volatile unsigned long long *>(p) = v;
}

struct RxSmem {
  uint32_t wcnt[kRxWarps][kRxBins];  // per-warp digit counts, then the warp's offset in the tile bucket
  uint32_t tstart[kRxBins];          // first local position of each digit
  uint32_t gbase[kRxBins];           // global position of that first record
  uint32_t buf[kRxTile];             // one word of the tile, by local position
  uint32_t gidx[kRxTile];            // local position -> global position
  uint32_t nh[kRxBins];               // this tile's counts of the next pass's digits
  uint32_t wsum[kRxWarps];
  uint32_t tile;
  uint32_t bad;
};

__global__ void __launch_bounds__(kRxThreads, 2) rx_pass_kernel(RxPassArgs a) {
  extern __shared__ __align__(16) unsigned char rx_raw[];
  RxSmem &sm = *reinterpret_cast<RxSmem *>(rx_raw);
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const uint32_t nbins = 1u << a.bits, mask = nbins - 1u;
  if (tid == 0) {
    sm.tile = atomicAdd(a.tile_ctr, 1u);  // tiles are claimed in launch order: earlier tiles never wait on later ones
    sm.bad = 0;
  }
  for (int i = tid; i < kRxWarps * kRxBins; i += kRxThreads) (&sm.wcnt[0][0])[i] = 0;
  if (tid < kRxBins) sm.nh[tid] = 0;
  __syncthreads();
  const uint32_t tile = sm.tile;
  const int64_t base = (int64_t)tile * kRxTile;
  const int cnt = (int)std::min<int64_t>(kRxTile, a.n - base);
  const uint32_t lt = (1u << lane) - 1u;
  const int wbase = w * (kRxSteps * 32) + lane;  // tile index of this thread's step 0

  // ---- keys (all loads in flight at once); warp w holds tile indices [w*512, (w+1)*512),
  //      step j the 32 indices from w*512 + 32 j.  The rank of a record among the records of
  //      its digit in its warp (stable) is kept, two 16-bit ranks per register.
  uint32_t kv[kRxSteps];
  const uint32_t *kin = a.in[a.key_word];
#pragma unroll
  for (int j = 0; j < kRxSteps; ++j) kv[j] = (wbase + j * 32 < cnt) ? __ldg(kin + base + wbase + j * 32) : 0u;
  uint32_t rk[kRxSteps / 2];
#pragma unroll
  for (int j = 0; j < kRxSteps; ++j) {
    const bool valid = wbase + j * 32 < cnt;
    const uint32_t d = (kv[j] >> a.shift) & mask;
    const uint32_t peers = rx_peers(d, a.bits, __ballot_sync(0xffffffffu, valid));
    uint32_t r = 0;
    if (valid) r = sm.wcnt[w][d] + (uint32_t)__popc(peers & lt);
    __syncwarp();
    if (valid && lane == __ffs(peers) - 1) sm.wcnt[w][d] += (uint32_t)__popc(peers);
    __syncwarp();
    if (j & 1) rk[j >> 1] |= r << 16;
    else rk[j >> 1] = r;
  }
  __syncthreads();

  // ---- tile counts, per-warp offsets, local bucket starts
  uint32_t tot = 0;
  if (tid < kRxBins) {
    for (int ww = 0; ww < kRxWarps; ++ww) {
      const uint32_t c = sm.wcnt[ww][tid];
      sm.wcnt[ww][tid] = tot;
      tot += c;
    }
    if ((uint32_t)tid < nbins)
      rx_store(a.status + (int64_t)tile * kRxBins + tid, (tile == 0 ? kRxFlagPre : kRxFlagAgg) | tot);
  }
  // exclusive scan of the tile counts over the digits (threads 0..255 = warps 0..7)
  uint32_t incl = tot;
  if (tid < kRxBins) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) sm.wsum[w] = incl;
  }
  // global bucket starts of this pass, scanned the same way (threads 256..511)
  uint32_t gh = (tid >= kRxBins && (uint32_t)(tid - kRxBins) < nbins) ? __ldg(a.hist + tid - kRxBins) : 0u;
  uint32_t gincl = gh;
  if (tid >= kRxBins) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, gincl, o);
      if (lane >= o) gincl += t;
    }
    if (lane == 31) sm.wsum[w] = gincl;  // warps 8..15
  }
  __syncthreads();
  if (tid < kRxBins) {
    uint32_t off = 0;
    for (int ww = 0; ww < w; ++ww) off += sm.wsum[ww];
    sm.tstart[tid] = off + incl - tot;
  } else {
    uint32_t off = 0;
    for (int ww = kRxWarps / 2; ww < w; ++ww) off += sm.wsum[ww];
    sm.gbase[tid - kRxBins] = off + gincl - gh;  // exclusive: records of smaller digits
  }
  __syncthreads();

  // ---- look-back over earlier tiles (one thread per digit)
  if (tid < kRxBins && (uint32_t)tid < nbins && tile > 0) {
    uint32_t excl = 0;
    bool ok = true;
    for (int64_t t = (int64_t)tile - 1; t >= 0;) {
      unsigned long long v = rx_load(a.status + t * kRxBins + tid);
      uint32_t polls = 0;
      while ((v >> 32) == 0ull) {
        if (++polls >= a.spin) break;
        if (polls > 64) __nanosleep(128);
        v = rx_load(a.status + t * kRxBins + tid);
      }
      if ((v >> 32) == 0ull) {
        ok = false;
        break;
      }
      excl += (uint32_t)v;
      if ((v >> 32) == (kRxFlagPre >> 32)) break;
      --t;
    }
    rx_store(a.status + (int64_t)tile * kRxBins + tid, kRxFlagPre | (uint32_t)(excl + tot));
    if (!ok) {
      atomicOr(a.err, kErrTimeout);
      sm.bad = 1;
    }
    sm.gbase[tid] += excl;
  }
  __syncthreads();
  if (sm.bad) return;

  // ---- local position of every record (replacing its warp rank) and the global position
  //      of every local position
#pragma unroll
  for (int j = 0; j < kRxSteps; ++j) {
    const bool valid = wbase + j * 32 < cnt;
    const uint32_t d = (kv[j] >> a.shift) & mask;
    const uint32_t r = (j & 1) ? (rk[j >> 1] >> 16) : (rk[j >> 1] & 0xffffu);
    uint32_t lp = 0;
    if (valid) {
      const uint32_t off = sm.wcnt[w][d] + r;  // rank among the tile's records of digit d
      lp = sm.tstart[d] + off;
      sm.gidx[lp] = sm.gbase[d] + off;
    }
    if (j & 1) rk[j >> 1] = (rk[j >> 1] & 0xffffu) | (lp << 16);
    else rk[j >> 1] = (rk[j >> 1] & 0xffff0000u) | lp;
  }

  // ---- every word of the tile, out in digit order: registers -> shared memory at the
  //      local position -> global memory in local order.  The key word goes first (its
  //      values are in registers); the next word's loads are issued before the stores.
  auto load_word = [&](int q, uint32_t *v) {
    const uint32_t *src = a.in[q];
    if (src) {
#pragma unroll
      for (int j = 0; j < kRxSteps; ++j) v[j] = (wbase + j * 32 < cnt) ? __ldg(src + base + wbase + j * 32) : 0u;
    } else {
#pragma unroll
      for (int j = 0; j < kRxSteps; ++j) v[j] = (uint32_t)(base + wbase + j * 32);
    }
  };
  uint32_t v[kRxSteps];
#pragma unroll
  for (int j = 0; j < kRxSteps; ++j) v[j] = kv[j];
  for (int t = 0; t < a.nwords; ++t) {
    const int q = t == 0 ? a.key_word : (t <= a.key_word ? t - 1 : t);
    if (a.next_hist && q == a.next_word) {  // the next pass's digit histogram (order-free)
      const uint32_t nmask = (1u << a.next_bits) - 1u;
#pragma unroll
      for (int j = 0; j < kRxSteps; ++j) {
        const bool valid = wbase + j * 32 < cnt;
        const uint32_t d = (v[j] >> a.next_shift) & nmask;
        const uint32_t peers = rx_peers(d, a.next_bits, __ballot_sync(0xffffffffu, valid));
        if (valid && lane == __ffs(peers) - 1) atomicAdd(&sm.nh[d], (uint32_t)__popc(peers));
      }
    }
#pragma unroll
    for (int j = 0; j < kRxSteps; ++j)
      if (wbase + j * 32 < cnt) sm.buf[(j & 1) ? (rk[j >> 1] >> 16) : (rk[j >> 1] & 0xffffu)] = v[j];
    __syncthreads();  // buf and gidx complete
    if (t + 1 < a.nwords) load_word(t + 1 <= a.key_word ? t : t + 1, v);
    uint32_t *dst = a.out[q];
#pragma unroll 4
    for (int p = tid; p < cnt; p += kRxThreads) {
      const uint32_t g = sm.gidx[p];
      if (g < (uint64_t)a.n) dst[g] = sm.buf[p];
    }
    __syncthreads();
  }
  if (a.next_hist && tid < kRxBins && sm.nh[tid]) atomicAdd(a.next_hist + tid, sm.nh[tid]);
}

static int64_t rx_cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

int radix_bits(int64_t maxval) {
  int b = 0;
  while (b < 63 && (maxval >> b) > 0) ++b;
  return b;
}

static int rx_plan(const RadixKey *keys, int nkeys, RxPass *pass) {
  int np = 0;
  for (int k = 0; k < nkeys; ++k) {
    const int b = keys[k].bits;
    if (b <= 0) continue;
    const int passes = (b + 7) / 8;
    const int width = (b + passes - 1) / passes;
    for (int p = 0, sh = 0; p < passes; ++p, sh += width) {
      if (np >= kRxMaxPasses) return -1;
      pass[np++] = RxPass{keys[k].word, sh, std::min(width, b - sh)};
    }
  }
  return np;
}

size_t radix_scratch_bytes(int64_t n, int nwords, const RadixKey *keys, int nkeys) {
  RxPass pass[kRxMaxPasses];
  const int np = rx_plan(keys, nkeys, pass);
  if (np < 0) return 0;
  const int64_t tiles = std::max<int64_t>(rx_cdiv(n, kRxTile), 1);
  size_t b = 0;
  b += sizeof(unsigned long long) * (size_t)(np * tiles * kRxBins);  // status
  b += sizeof(uint32_t) * (size_t)(np * kRxBins + np + 64);           // histograms + tile counters
  const int sets = np >= 2 ? 1 : 0;  // ping-pong partner of the output words
  b += sizeof(uint32_t) * (size_t)(sets * nwords * std::max<int64_t>(n, 1)) + 256 * (size_t)(nwords + 4);
  return b;
}

static inline uint8_t *rx_align(uint8_t *p) {
  return reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(p) + 255) & ~uintptr_t(255));
}

int radix_sort_records(int64_t n, const RadixRecords &r, const RadixKey *keys, int nkeys, const int64_t *valid_dims,
                       int nvalid, const float *valid_vals, void *scratch, size_t scratch_bytes, uint32_t *err,
                       cudaStream_t s) {
  RxPass pass[kRxMaxPasses];
  const int np = rx_plan(keys, nkeys, pass);
  if (np < 0 || r.nwords < 1 || r.nwords > kRadixMaxWords || nvalid > r.nwords) return -1;
  for (int k = 0; k < np; ++k)
    if (pass[k].word < 0 || pass[k].word >= r.nwords || !r.in[pass[k].word]) return -1;
  for (int q = 0; q < nvalid; ++q)
    if (!r.in[q]) return -1;
  if (scratch_bytes < radix_scratch_bytes(n, r.nwords, keys, nkeys)) return -1;
  const int64_t tiles = std::max<int64_t>(rx_cdiv(n, kRxTile), 1);
  uint8_t *p = rx_align(static_cast<uint8_t *>(scratch));
  auto *status = reinterpret_cast<unsigned long long *>(p);
  p = rx_align(p + sizeof(unsigned long long) * (size_t)(np * tiles * kRxBins));
  auto *hist = reinterpret_cast<uint32_t *>(p);
  uint32_t *ctr = hist + np * kRxBins;
  const size_t zero_bytes = (reinterpret_cast<uint8_t *>(ctr + np) - static_cast<uint8_t *>(scratch));
  p = rx_align(reinterpret_cast<uint8_t *>(ctr + np));
  uint32_t *tmpw[kRadixMaxWords] = {};  // passes alternate between these and the outputs
  if (np >= 2)
    for (int q = 0; q < r.nwords; ++q) {
      tmpw[q] = reinterpret_cast<uint32_t *>(p);
      p = rx_align(p + sizeof(uint32_t) * (size_t)std::max<int64_t>(n, 1));
    }
  if (cudaMemsetAsync(scratch, 0, zero_bytes, s) != cudaSuccess) return -2;

  // histograms of every pass (+ validation), one read of each word involved
  if (n > 0 && (np > 0 || nvalid > 0 || valid_vals)) {
    // only the first pass's digits: every pass counts the digits of the next one
    RxHistArgs h{};
    h.n = n;
    h.npass = np > 0 ? 1 : 0;
    for (int q = 0; q < r.nwords; ++q) h.src[q] = r.in[q];
    for (int q = 0; q < r.nwords; ++q) {
      RxHistWord hw{};
      hw.word = q;
      if (np > 0 && pass[0].word == q) {
        hw.np = 1;
        hw.shift[0] = pass[0].shift;
        hw.bits[0] = pass[0].bits;
      }
      if (hw.np > 0 || q < nvalid) h.kw[h.nkw++] = hw;
    }
    h.dims = valid_dims;
    h.nvalid = nvalid;
    h.vals = valid_vals;
    h.hist = hist;
    h.err = err;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t rounds = rx_cdiv(n, (int64_t)kRxHistThreads * kRxHistItems);
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>(rounds, (int64_t)sms * 4));
    rx_hist_kernel<<<blocks, kRxHistThreads, sizeof(uint32_t) * h.npass * kRxBins, s>>>(h);
    ::tk::count_launch();
  }
  if (np == 0) {  // nothing to sort: copy
    for (int q = 0; q < r.nwords; ++q) {
      if (r.in[q]) {
        if (cudaMemcpyAsync(r.out[q], r.in[q], sizeof(uint32_t) * (size_t)n, cudaMemcpyDeviceToDevice, s) !=
            cudaSuccess)
          return -2;
      } else {
        iota_u32(r.out[q], n, s);
      }
    }
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
  }
  if (cudaFuncSetAttribute(rx_pass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(RxSmem)) !=
      cudaSuccess)
    return -2;
  const uint32_t *cur[kRadixMaxWords];
  for (int q = 0; q < r.nwords; ++q) cur[q] = r.in[q];
  for (int k = 0; k < np; ++k) {
    RxPassArgs a{};
    a.n = n;
    a.nwords = r.nwords;
    a.key_word = pass[k].word;
    a.shift = pass[k].shift;
    a.bits = pass[k].bits;
    const bool to_out = ((np - 1 - k) % 2) == 0;  // the last pass writes the outputs
    for (int q = 0; q < r.nwords; ++q) {
      a.in[q] = cur[q];
      a.out[q] = to_out ? r.out[q] : tmpw[q];
    }
    a.hist = hist + k * kRxBins;
    if (k + 1 < np) {
      a.next_hist = hist + (k + 1) * kRxBins;
      a.next_word = pass[k + 1].word;
      a.next_shift = pass[k + 1].shift;
      a.next_bits = pass[k + 1].bits;
    }
    a.status = status + (int64_t)k * tiles * kRxBins;
    a.tile_ctr = ctr + k;
    a.err = err;
    a.spin = kRxSpin;
    if (n > 0) {
      rx_pass_kernel<<<(unsigned)tiles, kRxThreads, sizeof(RxSmem), s>>>(a);
      ::tk::count_launch();
    }
    for (int q = 0; q < r.nwords; ++q) cur[q] = a.out[q];
  }
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

__global__ void rx_iota_kernel(uint32_t *out, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = (uint32_t)e;
}

// One pass over two tiles run by a single block that claims the second tile (the tile
// counter starts at 1): its look-back waits for counts that never come, gives up after
// `polls` polls and stores nothing.  Returns the error word (kErrTimeout expected).
int radix_selftest_wait(uint32_t polls, cudaStream_t s, uint32_t *err_out) {
  const int64_t n = 2 * (int64_t)kRxTile;
  uint32_t *words = nullptr;  // in [n], out [n], hist [256], counter, error word
  unsigned long long *status = nullptr;
  if (cudaMallocAsync(reinterpret_cast<void **>(&words), sizeof(uint32_t) * (size_t)(2 * n + kRxBins + 2), s) !=
      cudaSuccess)
    return -2;
  if (cudaMallocAsync(reinterpret_cast<void **>(&status), sizeof(unsigned long long) * 2 * kRxBins, s) != cudaSuccess) {
    cudaFreeAsync(words, s);
    return -2;
  }
  uint32_t *in = words, *out = words + n, *hist = words + 2 * n, *ctr = hist + kRxBins, *err = ctr + 1;
  const uint32_t one = 1u;
  cudaError_t e = cudaMemsetAsync(words, 0, sizeof(uint32_t) * (size_t)(2 * n + kRxBins + 2), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(unsigned long long) * 2 * kRxBins, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ctr, &one, sizeof(uint32_t), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(rx_pass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(RxSmem));
  if (e == cudaSuccess) {
    RxPassArgs a{};
    a.n = n;
    a.nwords = 1;
    a.key_word = 0;
    a.shift = 0;
    a.bits = 8;
    a.in[0] = in;
    a.out[0] = out;
    a.hist = hist;
    a.status = status;
    a.tile_ctr = ctr;
    a.err = err;
    a.spin = polls;
    rx_pass_kernel<<<1, kRxThreads, sizeof(RxSmem), s>>>(a);
    e = cudaGetLastError();
  }
  *err_out = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(err_out, err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(status, s);
  cudaFreeAsync(words, s);
  const cudaError_t e2 = cudaStreamSynchronize(s);
  return (e == cudaSuccess && e2 == cudaSuccess) ? 0 : -2;
}

cudaError_t preload_radix_kernels() {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, rx_hist_kernel);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, rx_pass_kernel);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, rx_iota_kernel);
  return e;
}

void iota_u32(uint32_t *out, int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  rx_iota_kernel<<<(unsigned)std::min<int64_t>(rx_cdiv(n, 256), 65535LL * 8), 256, 0, s>>>(out, n);
  ::tk::count_launch();
}

}  // namespace tk
