// K-d: core tensor of one HOOI sweep and the fit (Section III-B, eqs. ttm_ele and
// core_unfolded:  G_(N) = U_N^T Y_(N),  G[c, r] = sum_i U_N(i, r) Y_(N)(i, c)).
// Y_(N) is the FP32 TTMc output of the last mode (I_N x P), U_N the FP64 factor
// (I_N x R).  Two forms: on the tensor cores (core_tc_kernel, exact fixed-point slices,
// below) with a separate reduction of the row ranges (core_reduce_kernel), and an FP64
// SIMT form (core_kernel: split over rows of Y into chunks, each block owns a 16 x 16 tile
// of (column c, rank r) outputs for one row chunk and accumulates in FP64).  Both write G
// (C-order, r fastest), ||G||^2 and fit = 1 - sqrt(max(0, ||X||^2 - ||G||^2)) / ||X||,
// adding the row ranges' partials in a fixed order.
#include <algorithm>
#include <cstdlib>

#include "internal.cuh"

namespace tk {

constexpr int kCoreRows = 64;  // rows of Y per chunk staged at once

__global__ void __launch_bounds__(256) core_kernel(const float *Y, const double *U, int64_t I, int64_t P, int R,
                                                   int rows_per_chunk, double *part, unsigned *counter, double *G,
                                                   const double *norm_x2, double *norm_g2, double *fit) {
  __shared__ float ys[kCoreRows][17];
  __shared__ double us[kCoreRows][17];
  const int tc = threadIdx.x & 15, tr = threadIdx.x >> 4;
  const int64_t c = (int64_t)blockIdx.x * 16 + tc;
  const int r = blockIdx.y * 16 + tr;
  const int64_t i_begin = (int64_t)blockIdx.z * rows_per_chunk;
  const int64_t i_end = std::min<int64_t>(I, i_begin + rows_per_chunk);
  double acc = 0.0;
  for (int64_t i0 = i_begin; i0 < i_end; i0 += kCoreRows) {
    for (int q = threadIdx.x; q < kCoreRows * 16; q += blockDim.x) {
      const int ri = q / 16, cc = q % 16;
      const int64_t i = i0 + ri;
      const int64_t col = (int64_t)blockIdx.x * 16 + cc;
      const int rr = blockIdx.y * 16 + cc;
      ys[ri][cc] = (i < i_end && col < P) ? Y[i * P + col] : 0.f;
      us[ri][cc] = (i < i_end && rr < R) ? U[i * R + rr] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int ri = 0; ri < kCoreRows; ++ri) acc = fma(us[ri][tr], (double)ys[ri][tc], acc);
    __syncthreads();
  }
  const int64_t PR = P * R;
  if (c < P && r < R) part[(int64_t)blockIdx.z * PR + c * R + r] = acc;

  // last block: reduce chunks, ||G||^2, fit
  __shared__ bool is_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = atomicAdd(counter, 1u) == gridDim.x * gridDim.y * gridDim.z - 1u;
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  __shared__ double red[256];
  double g2 = 0.0;
  for (int64_t q = threadIdx.x; q < PR; q += blockDim.x) {
    double t = 0.0;
    for (int z = 0; z < (int)gridDim.z; ++z) t += __ldcg(part + (int64_t)z * PR + q);
    G[q] = t;
    g2 = fma(t, t, g2);
  }
  red[threadIdx.x] = g2;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double gx = red[0];
    const double nx = *norm_x2;
    *norm_g2 = gx;
    *fit = (nx > 0.0) ? 1.0 - sqrt(fmax(0.0, nx - gx)) / sqrt(nx) : 1.0;
    *counter = 0u;
  }
}

// ---------------------------------------------------------------- tensor-core form
// The same G on the 5th-generation tensor cores: G as a P x R matrix is Y_(N)^T U_N, so one
// CTA computes a tile of 128 columns c of Y (the MMA's M) by all ranks r (N = R rounded up
// to 16) over a range of at most 128 rows i of Y (the K of the product), 16 rows at a time.
//
// Fixed-point slices (an Ozaki-type split): each column of Y over the CTA's rows, and each
// column of U_N (FP64), gets a shared power of two 2^E above its largest magnitude, and
// every value v is written as 2^(E-8) (m_0 + m_1 2^-8 + m_2 2^-16 + m_3 2^-24) with integer
// slices |m_0| <= 256, |m_s| <= 128 (rounded to nearest, remainders exact in FP64; the
// part below the last slice, under 2^(E-33), is dropped).  The slices are exact in BF16.
// For every pair of slices (a, b) one tcgen05.mma kind::f16 adds m_a(Y) m_b(U) over 16 rows
// into the FP32 tensor-memory accumulator of level a + b.  A product is at most 2^16, and a
// level's sum over at most 128 rows stays below 2^24, so every accumulator holds an exact
// integer: the FP32 accumulation never rounds, whatever the tensor core's rounding rule.
// At the end each level is read with tcgen05.ld and added into FP64 with its scale
// 2^(E_c + E_r - 16 - 8 level).  The result differs from the exact G of the FP32 Y and FP64
// U only by the dropped parts (relative ~2^-33 of the columns' largest entries) and the FP64
// additions of the levels and row ranges.  Operands are staged K-major in the no-swizzle
// canonical layout (8-row x 16-byte core matrices) in two buffers: the slices of chunk j + 1
// are written while the products of chunk j run.  The last CTA adds the partials of every row
// range in order, as core_kernel does.
constexpr int kTcM = 128;   // columns of Y per tile (MMA M)
constexpr int kTcK = 16;    // rows of Y per staged chunk (one MMA of K = 16 per slice pair)
constexpr int kTcKC = kTcK * 2 / 16;  // core-matrix columns (16 bytes) along K per chunk
constexpr int kTcRows = 128;  // rows of Y per CTA at most: keeps every level sum below 2^24
constexpr int kTcSlices = 4;  // 8-bit slices per value
constexpr int kTcLevels = 5;  // slice pairs a + b <= 4 (the three pairs above add under 2^-40 of a product)
constexpr unsigned long long kTcSpin = 1ull << 22;

__host__ __device__ constexpr uint32_t tc_tmem_cols(int np) {
  uint32_t c = 32;
  while (c < (uint32_t)(kTcLevels * np)) c <<= 1;
  return c;
}
__host__ __device__ constexpr size_t tc_rows_bytes(int rows, int np) {  // the CTA's rows of Y and U_N
  return ((size_t)rows * kTcM * 4 + (size_t)rows * np * 8 + 127) / 128 * 128;
}
__host__ __device__ constexpr size_t tc_smem_bytes(int rows, int np) {
  return tc_rows_bytes(rows, np) + (size_t)2 * kTcSlices * (kTcM + np) * kTcK * 2 + 128;  // + two slice buffers
}

__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of this architecture; base offset 0, no swizzle
  return d;
}
// The four integer slices of an FP32 y against 2^e (|y| < 2^e; 2^(8 - e) = sc1 sc2, two
// factors so that neither overflows when the column holds only subnormal values), each
// exact in BF16.  FP32 arithmetic, all exact: t = y 2^(8 - e) has at most 24 significant
// bits below 2^8, and |t - rint(t)| <= 1/2 keeps its bits.
__device__ __forceinline__ void slices_f32(float y, float sc1, float sc2, __nv_bfloat16 *out, int stride) {
  float t = (y * sc1) * sc2;
#pragma unroll
  for (int q = 0; q < kTcSlices; ++q) {
    const float m = rintf(t);
    out[q * stride] = __float2bfloat16_rn(m);
    t = (t - m) * 256.0f;
  }
}
// The four slices of an FP64 u against 2^e (|u| < 2^e): x = u 2^(32 - e) rounded to the
// nearest integer (ties to even), |x| <= 2^32, in balanced base-256 digits
// x = m_0 2^24 + m_1 2^16 + m_2 2^8 + m_3 with |m_s| <= 128 for s >= 1, hence |m_0| <= 256.
// Integer arithmetic on the bits of u (the FP64 pipe is narrow on this part).
__device__ __forceinline__ void slices_f64(double u, int e, __nv_bfloat16 *out, int stride) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(u);
  const int ex = (int)((bits >> 52) & 0x7ff);
  unsigned long long mant = bits & 0xFFFFFFFFFFFFFull;
  int sh;  // u = mant 2^(ex - 1075) with the hidden bit; x = u 2^(32 - e) = mant 2^-sh
  if (ex == 0) {
    sh = 1042 + e;  // subnormal: u = mant 2^-1074
  } else {
    mant |= 1ull << 52;
    sh = 1043 + e - ex;
  }
  unsigned long long qv = 0;  // sh >= 21 since |u| < 2^e; above 63 the value rounds to 0
  if (sh < 64) {
    const unsigned long long half = 1ull << (sh - 1), rem = mant & ((1ull << sh) - 1ull);
    qv = mant >> sh;
    if (rem > half || (rem == half && (qv & 1ull))) ++qv;
  }
  long long x = (bits >> 63) ? -(long long)qv : (long long)qv;
  int m[kTcSlices];
#pragma unroll
  for (int q = kTcSlices - 1; q > 0; --q) {
    const int d = (int)(((x + 128) & 255) - 128);
    m[q] = d;
    x = (x - d) >> 8;
  }
  m[0] = (int)x;
#pragma unroll
  for (int q = 0; q < kTcSlices; ++q) out[q * stride] = __int2bfloat16_rn(m[q]);
}
// exponent e with |x| < 2^e (0 for x = 0) of a finite FP32 / FP64 magnitude given by its bits
// (the exponent field, or the leading zeros of a subnormal's fraction): integer arithmetic
__device__ __forceinline__ int above_exp_f32(uint32_t b) {
  const int ef = (int)(b >> 23);
  if (ef) return ef - 126;
  return b ? -149 + 32 - __clz((int)b) : 0;
}
__device__ __forceinline__ int above_exp_f64(unsigned long long b) {
  const int ef = (int)(b >> 52);
  if (ef) return ef - 1022;
  return b ? -1074 + 64 - __clzll((long long)b) : 0;
}
// 2^k as a double for -1022 <= k <= 1023 (built from its bits)
__device__ __forceinline__ double pow2d(int k) { return __longlong_as_double((long long)(1023 + k) << 52); }
// element (row, k) of a K-major 16-bit operand tile with kTcKC core columns per 8-row group
__device__ __forceinline__ int kmaj16(int row, int k) {
  return ((row >> 3) * kTcKC + (k >> 3)) * 64 + (row & 7) * 8 + (k & 7);
}
// bounded wait for completion `parity` of an mbarrier; false if it gave up
__device__ __forceinline__ bool tc_wait(uint32_t bar, uint32_t parity) {
  for (unsigned long long it = 0; it < kTcSpin; ++it) {
    uint32_t d;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(d)
        : "r"(bar), "r"(parity)
        : "memory");
    if (d) return true;
    if (it > 32) __nanosleep(64);
  }
  return false;
}

template <int NP>  // N of the MMA: R rounded up to 16
__global__ void __launch_bounds__(128) core_tc_kernel(const float *Y, const double *U, int64_t I, int64_t P, int R,
                                                      int rows_per_split, double *part, uint32_t *err) {
  static_assert(NP % 16 == 0 && NP >= 16 && NP <= 64, "N of the MMA");
  constexpr uint32_t kCols = tc_tmem_cols(NP);  // tensor-memory columns: kTcLevels accumulators of NP
  constexpr int kASlice = kTcM * kTcK, kBSlice = NP * kTcK;  // BF16 elements per slice tile
  extern __shared__ unsigned char tc_raw[];
  unsigned char *base = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(tc_raw) + 127) & ~static_cast<uintptr_t>(127));
  const int rcap = rows_per_split;  // a multiple of kTcK, at most kTcRows
  float *sY = reinterpret_cast<float *>(base);                              // [rcap][kTcM]
  double *sU = reinterpret_cast<double *>(base + (size_t)rcap * kTcM * 4);  // [rcap][NP]
  __nv_bfloat16 *sA = reinterpret_cast<__nv_bfloat16 *>(base + tc_rows_bytes(rcap, NP));
  __nv_bfloat16 *sB = sA + 2 * kTcSlices * kASlice;  // sA: [2][kTcSlices][kASlice], sB: [2][kTcSlices][kBSlice]
  __shared__ __align__(8) unsigned long long bar[2];
  __shared__ uint32_t tbase;
  __shared__ int s_ok;
  __shared__ int s_eu[NP];
  const int tid = threadIdx.x, warp = tid >> 5;
  const int64_t c0 = (int64_t)blockIdx.x * kTcM;
  const int64_t i_begin = (int64_t)blockIdx.y * rows_per_split;
  const int64_t i_end = min(I, i_begin + rows_per_split);
  uint32_t sb[2];
  sb[0] = (uint32_t)__cvta_generic_to_shared(&bar[0]);
  sb[1] = (uint32_t)__cvta_generic_to_shared(&bar[1]);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sb[0]) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sb[1]) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_ok = 1;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(&tbase)),
                 "r"(kCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // the CTA's rows of Y (thread t: column c0 + t) and of U_N into shared memory, loads in flight
  // together; then the shared exponents of the columns
  const int64_t c = c0 + tid;
  const int nrows = (int)(i_end - i_begin);
#pragma unroll 16
  for (int i = 0; i < rcap; ++i)
    sY[i * kTcM + tid] = (i < nrows && c < P) ? __ldg(Y + (i_begin + i) * P + c) : 0.f;
  for (int q = tid; q < rcap * NP; q += 128) {
    const int i = q / NP, n = q % NP;
    sU[q] = (i < nrows && n < R) ? __ldg(U + (i_begin + i) * R + n) : 0.0;
  }
  __syncthreads();
  // (the magnitudes of finite values order like their bit patterns without the sign)
  uint32_t ybits = 0;
  for (int i = 0; i < nrows; ++i) ybits = max(ybits, __float_as_uint(sY[i * kTcM + tid]) & 0x7fffffffu);
  const int ec = above_exp_f32(ybits);
  const int ysh = 8 - ec, ysh1 = min(ysh, 120);
  const float ysc1 = __int_as_float((127 + ysh1) << 23), ysc2 = __int_as_float((127 + ysh - ysh1) << 23);
  for (int n = tid; n < NP; n += 128) {
    unsigned long long ub = 0;
    for (int i = 0; i < nrows; ++i)
      ub = max(ub, (unsigned long long)__double_as_longlong(sU[i * NP + n]) & 0x7FFFFFFFFFFFFFFFull);
    s_eu[n] = above_exp_f64(ub);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tbase;
  // D f32, A and B bf16, both K-major, N >> 3, M >> 4
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NP >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);
  const uint32_t lbo = 128, sbo = kTcKC * 128;  // K-adjacent core matrices, 8-row groups
  const uint32_t aS = (uint32_t)__cvta_generic_to_shared(sA), bS = (uint32_t)__cvta_generic_to_shared(sB);
  const int nchunks = (int)((i_end - i_begin + kTcK - 1) / kTcK);
  bool ok = true;
  int issued = 0;  // chunks whose products were issued
  for (int j = 0; j < nchunks && ok; ++j) {
    const int b = j & 1;
    if (j >= 2) ok = tc_wait(sb[b], (uint32_t)(((j >> 1) - 1) & 1));  // the products that read this buffer
    ok = __syncthreads_and(ok ? 1 : 0) != 0;
    if (!ok) break;
    __nv_bfloat16 *a = sA + (size_t)b * kTcSlices * kASlice;
    __nv_bfloat16 *bb = sB + (size_t)b * kTcSlices * kBSlice;
#pragma unroll 4
    for (int k = 0; k < kTcK; ++k)
      slices_f32(sY[(j * kTcK + k) * kTcM + tid], ysc1, ysc2, a + kmaj16(tid, k), kASlice);
    for (int q = tid; q < NP * kTcK; q += 128) {
      const int n = q % NP, k = q / NP;
      slices_f64(sU[(j * kTcK + k) * NP + n], s_eu[n], bb + kmaj16(n, k), kBSlice);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0) {
      const uint32_t aB = aS + (uint32_t)(b * kTcSlices * kASlice * 2), bB = bS + (uint32_t)(b * kTcSlices * kBSlice * 2);
#pragma unroll
      for (int L = 0; L < kTcLevels; ++L) {
        const int s0 = L < kTcSlices ? 0 : L - (kTcSlices - 1);
        const int s1 = L < kTcSlices ? L : kTcSlices - 1;  // pairs (a, L - a), both below kTcSlices
        for (int sa = s0; sa <= s1; ++sa) {
          const int sbk = L - sa;
          const uint64_t ad = umma_desc(aB + (uint32_t)(sa * kASlice * 2), lbo, sbo);
          const uint64_t bd = umma_desc(bB + (uint32_t)(sbk * kBSlice * 2), lbo, sbo);
          const uint32_t acc = (j > 0 || sa != s0) ? 1u : 0u;
          asm volatile(
              "{ .reg .pred p; setp.ne.u32 p, %4, 0; tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }" ::"r"(
                  tmem + (uint32_t)(L * NP)),
              "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
              : "memory");
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(sb[b])
                   : "memory");
    }
    issued = j + 1;
  }
  // the last products of both buffers (bounded; on a give-up the products still in flight get
  // the same bounded time to end before the memory is freed)
  if (tid == 0) {
    bool done = ok;
    for (int b = 0; b < 2; ++b) {
      const int jl = (issued - 1 - b) >= 0 ? ((issued - 1 - b) & ~1) + b : -1;  // last chunk issued in buffer b
      if (jl >= 0) done = tc_wait(sb[b], (uint32_t)((jl >> 1) & 1)) && done;
    }
    if (!done) {
      atomicOr(err, kErrTimeout);
      s_ok = 0;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  // the levels are exact integers below 2^24: X = sum_L A_L 2^(8 (4 - L)) is exact in 64 bits;
  // then one conversion and one scaling by 2^(E_c + E_r - 16 - 32) (two factors: no overflow)
  long long accx[NP];
#pragma unroll
  for (int q = 0; q < NP; ++q) accx[q] = 0;
  if (s_ok && nchunks > 0) {
#pragma unroll
    for (int L = 0; L < kTcLevels; ++L)
#pragma unroll
      for (int n0 = 0; n0 < NP; n0 += 16) {
        uint32_t v[16];
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(L * NP + n0);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int q = 0; q < 16; ++q)
          accx[n0 + q] += (long long)__float2int_rn(__uint_as_float(v[q])) << (8 * (kTcLevels - 1 - L));
      }
  }
  double accd[NP];
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    const int sh = ec + s_eu[q] - 16 - 8 * (kTcLevels - 1);
    const int sh1 = min(max(sh, -1000), 1000);  // two exact factors when |sh| is out of range
    accd[q] = ((double)accx[q] * pow2d(sh1)) * pow2d(sh - sh1);
  }
  // warp w holds tensor-memory lanes 32w .. 32w + 31 = columns c0 + 32w + lane (= c: tid)
  const int64_t PR = P * R;
  if (c < P)
#pragma unroll
    for (int q = 0; q < NP; ++q)
      if (q < R) part[(int64_t)blockIdx.y * PR + c * R + q] = s_ok ? accd[q] : __longlong_as_double(0x7ff8000000000000ll);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
}

// G[q] = the partials of every row range added in order (q = c R + r), ||G||^2 from per-block
// sums added by the last block in a fixed tree order, and the fit.
constexpr int kRedT = 64;
__global__ void __launch_bounds__(kRedT) core_reduce_kernel(const double *part, int nz, int64_t PR, double *G,
                                                           double *bsum, unsigned *counter, const double *norm_x2,
                                                           double *norm_g2, double *fit) {
  __shared__ double red[kRedT];
  __shared__ bool is_last;
  const int64_t q = (int64_t)blockIdx.x * kRedT + threadIdx.x;
  double g2 = 0.0;
  if (q < PR) {
    double t = 0.0;
    int z = 0;
    for (; z + 8 <= nz; z += 8) {  // eight loads in flight, added in order
      double v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = __ldcg(part + (int64_t)(z + u) * PR + q);
#pragma unroll
      for (int u = 0; u < 8; ++u) t += v[u];
    }
    for (; z < nz; ++z) t += __ldcg(part + (int64_t)z * PR + q);
    G[q] = t;
    g2 = t * t;
  }
  red[threadIdx.x] = g2;
  __syncthreads();
  for (int o = kRedT / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    bsum[blockIdx.x] = red[0];
    __threadfence();
    is_last = atomicAdd(counter, 1u) == gridDim.x - 1u;
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  double gb = 0.0;  // block sums b = t, t + kRedT, ... then a tree over the threads
  for (unsigned b = threadIdx.x; b < gridDim.x; b += kRedT) gb += __ldcg(bsum + b);
  red[threadIdx.x] = gb;
  __syncthreads();
  for (int o = kRedT / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double gx = red[0];
    const double nx = *norm_x2;
    *norm_g2 = gx;
    *fit = (nx > 0.0) ? 1.0 - sqrt(fmax(0.0, nx - gx)) / sqrt(nx) : 1.0;
    *counter = 0u;
  }
}

static bool core_on_tensor_cores();

// ---------------------------------------------------------------- Gram matrix on the tensor cores
// S = Y Y^T (m x m) of an FP32 m x n matrix, for the fat unfoldings of Section III-D, with
// the exact fixed-point slices of the core: one CTA computes a 128 x 64 tile of S (rows i
// of Y as the MMA's M, rows j as its N) over a range of columns c (the K), 128 columns at
// a time.  For each 128-column block every row of Y gets a shared power of two over the
// block, the slices' level sums are exact integers in tensor memory (products <= 2^16, at
// most 128 columns), and after each block they are combined in 64-bit integers and added,
// scaled, into FP64 registers.  The column ranges are added in a fixed order afterwards.
constexpr int kGmM = 128;           // rows i per tile (MMA M)
constexpr int kGmN = 64;            // rows j per tile (MMA N)
constexpr int kGmCols = 128;        // columns per exact block
constexpr int kGmLd = kGmCols + 1;  // shared-memory row stride of the staged block (no bank conflicts)
constexpr int kGramMaxRows = 1024;  // larger Gram matrices use the FP64 form
constexpr int kGramMaxRanges = 8;   // column ranges (partial sets)

__host__ __device__ constexpr size_t gm_smem_bytes() {
  return (size_t)(kGmM + kGmN) * kGmLd * 4                                // the rows' column block
         + (size_t)2 * kTcSlices * (kGmM + kGmN) * kTcK * 2 + 128;        // two slice buffers
}

__global__ void __launch_bounds__(128) gram_tc_kernel(const float *Y, int64_t m, int64_t n, int64_t cols_per_range,
                                                      double *part, uint32_t *err) {
  constexpr uint32_t kCols = tc_tmem_cols(kGmN);
  constexpr int kASlice = kGmM * kTcK, kBSlice = kGmN * kTcK;
  extern __shared__ unsigned char gm_raw[];
  unsigned char *base = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(gm_raw) + 127) & ~static_cast<uintptr_t>(127));
  float *sYa = reinterpret_cast<float *>(base);  // [kGmM][kGmLd]: rows i of the block
  float *sYb = sYa + kGmM * kGmLd;               // [kGmN][kGmLd]: rows j
  __nv_bfloat16 *sA = reinterpret_cast<__nv_bfloat16 *>(
      base + ((size_t)(kGmM + kGmN) * kGmLd * 4 + 127) / 128 * 128);
  __nv_bfloat16 *sB = sA + 2 * kTcSlices * kASlice;
  __shared__ __align__(8) unsigned long long bar[2];
  __shared__ uint32_t tbase;
  __shared__ int s_ok;
  __shared__ int s_eb[kGmN];
  __shared__ float s_bsc[2][kGmN];
  const int tid = threadIdx.x, warp = tid >> 5;
  const int64_t i0 = (int64_t)blockIdx.x * kGmM, j0 = (int64_t)blockIdx.y * kGmN;
  const int64_t c_begin = (int64_t)blockIdx.z * cols_per_range;
  const int64_t c_end = min(n, c_begin + cols_per_range);
  uint32_t sb[2];
  sb[0] = (uint32_t)__cvta_generic_to_shared(&bar[0]);
  sb[1] = (uint32_t)__cvta_generic_to_shared(&bar[1]);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sb[0]) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sb[1]) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_ok = 1;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(&tbase)),
                 "r"(kCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tbase;
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kGmN >> 3) << 17) | ((uint32_t)(kGmM >> 4) << 24);
  const uint32_t lbo = 128, sbo = kTcKC * 128;
  const uint32_t aS = (uint32_t)__cvta_generic_to_shared(sA), bS = (uint32_t)__cvta_generic_to_shared(sB);
  const int64_t ri = i0 + tid;  // this thread's row i (TMEM lane)
  double accd[kGmN];
#pragma unroll
  for (int q = 0; q < kGmN; ++q) accd[q] = 0.0;
  bool ok = true;
  int phase[2] = {0, 0};  // completions waited for, per buffer
  int issued[2] = {0, 0};  // products issued, per buffer
  int jglob = 0;           // chunk counter over all blocks (buffer = jglob & 1)
  for (int64_t cb = c_begin; cb < c_end && ok; cb += kGmCols) {
    const int ncb = (int)min((int64_t)kGmCols, c_end - cb);
    const int nch = (ncb + kTcK - 1) / kTcK;
    // the block's columns of rows i and rows j, zero-padded (coalesced along the rows)
#pragma unroll 8
    for (int q = tid; q < kGmM * kGmCols; q += 128) {
      const int r = q / kGmCols, k = q % kGmCols;
      const int64_t rr = i0 + r;
      sYa[r * kGmLd + k] = (rr < m && k < ncb) ? __ldg(Y + rr * n + cb + k) : 0.f;
    }
#pragma unroll 8
    for (int q = tid; q < kGmN * kGmCols; q += 128) {
      const int r = q / kGmCols, k = q % kGmCols;
      const int64_t rj = j0 + r;
      sYb[r * kGmLd + k] = (rj < m && k < ncb) ? __ldg(Y + rj * n + cb + k) : 0.f;
    }
    __syncthreads();
    uint32_t abits = 0;
    for (int k = 0; k < ncb; ++k) abits = max(abits, __float_as_uint(sYa[tid * kGmLd + k]) & 0x7fffffffu);
    const int ea = above_exp_f32(abits);
    const int ash = 8 - ea, ash1 = min(ash, 120);
    const float asc1 = __int_as_float((127 + ash1) << 23), asc2 = __int_as_float((127 + ash - ash1) << 23);
    if (tid < kGmN) {
      uint32_t bbits = 0;
      for (int k = 0; k < ncb; ++k) bbits = max(bbits, __float_as_uint(sYb[tid * kGmLd + k]) & 0x7fffffffu);
      const int eb = above_exp_f32(bbits), bsh = 8 - eb, bsh1 = min(bsh, 120);
      s_eb[tid] = eb;
      s_bsc[0][tid] = __int_as_float((127 + bsh1) << 23);
      s_bsc[1][tid] = __int_as_float((127 + bsh - bsh1) << 23);
    }
    __syncthreads();
    for (int j = 0; j < nch && ok; ++j, ++jglob) {
      const int b = jglob & 1;
      if (issued[b] > phase[b]) {  // the products that last read this buffer
        ok = tc_wait(sb[b], (uint32_t)(phase[b] & 1));
        ++phase[b];
      }
      ok = __syncthreads_and(ok ? 1 : 0) != 0;
      if (!ok) break;
      __nv_bfloat16 *a = sA + (size_t)b * kTcSlices * kASlice;
      __nv_bfloat16 *bb = sB + (size_t)b * kTcSlices * kBSlice;
#pragma unroll 4
      for (int k = 0; k < kTcK; ++k) slices_f32(sYa[tid * kGmLd + j * kTcK + k], asc1, asc2, a + kmaj16(tid, k), kASlice);
      for (int q = tid; q < kGmN * kTcK; q += 128) {
        const int r = q / kTcK, k = q % kTcK;
        slices_f32(sYb[r * kGmLd + j * kTcK + k], s_bsc[0][r], s_bsc[1][r], bb + kmaj16(r, k), kBSlice);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (tid == 0) {
        const uint32_t aB = aS + (uint32_t)(b * kTcSlices * kASlice * 2), bB = bS + (uint32_t)(b * kTcSlices * kBSlice * 2);
#pragma unroll
        for (int L = 0; L < kTcLevels; ++L) {
          const int s0 = L < kTcSlices ? 0 : L - (kTcSlices - 1);
          const int s1 = L < kTcSlices ? L : kTcSlices - 1;
          for (int sa = s0; sa <= s1; ++sa) {
            const uint64_t ad = umma_desc(aB + (uint32_t)(sa * kASlice * 2), lbo, sbo);
            const uint64_t bd = umma_desc(bB + (uint32_t)((L - sa) * kBSlice * 2), lbo, sbo);
            const uint32_t acc = (j > 0 || sa != s0) ? 1u : 0u;  // a fresh accumulation per block
            asm volatile(
                "{ .reg .pred p; setp.ne.u32 p, %4, 0; tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }" ::"r"(
                    tmem + (uint32_t)(L * kGmN)),
                "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                : "memory");
          }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(sb[b])
                     : "memory");
      }
      ++issued[b];
    }
    // this block's products complete (both buffers), then its levels into FP64
    for (int b = 0; b < 2 && ok; ++b)
      while (issued[b] > phase[b] && ok) {
        ok = tc_wait(sb[b], (uint32_t)(phase[b] & 1));
        ++phase[b];
      }
    ok = __syncthreads_and(ok ? 1 : 0) != 0;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!ok) break;
#pragma unroll
    for (int n0 = 0; n0 < kGmN; n0 += 16) {  // 16 columns of j at a time: five levels, then FP64
      long long accx[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) accx[q] = 0;
#pragma unroll
      for (int L = 0; L < kTcLevels; ++L) {
        uint32_t v[16];
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(L * kGmN + n0);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int q = 0; q < 16; ++q)
          accx[q] += (long long)__float2int_rn(__uint_as_float(v[q])) << (8 * (kTcLevels - 1 - L));
      }
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int sh = ea + s_eb[n0 + q] - 16 - 8 * (kTcLevels - 1);
        const int sh1 = min(max(sh, -1000), 1000);
        accd[n0 + q] += ((double)accx[q] * pow2d(sh1)) * pow2d(sh - sh1);
      }
    }
    // every warp has read the levels (and s_eb) before the next block overwrites them
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }
  if (!ok && tid == 0) {  // give products still in flight (bounded) time to end, then record
    for (int b = 0; b < 2; ++b)
      while (issued[b] > phase[b]) {
        tc_wait(sb[b], (uint32_t)(phase[b] & 1));
        ++phase[b];
      }
    atomicOr(err, kErrTimeout);
    s_ok = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (ri < m)
#pragma unroll
    for (int q = 0; q < kGmN; ++q)
      if (j0 + q < m)
        part[(int64_t)blockIdx.z * m * m + ri * m + j0 + q] = s_ok ? accd[q] : __longlong_as_double(0x7ff8000000000000ll);
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
}

// S[q] = the column ranges' partials added in order
__global__ void gram_reduce_kernel(const double *part, int nr, int64_t mm, double *S) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < mm; q += (int64_t)gridDim.x * blockDim.x) {
    double t = 0.0;
    for (int r = 0; r < nr; ++r) t += __ldcg(part + (int64_t)r * mm + q);
    S[q] = t;
  }
}

size_t gram_part_elems(int64_t m) {
  return (m > 0 && m <= kGramMaxRows) ? (size_t)kGramMaxRanges * (size_t)(m * m) : 0;
}

void launch_gram(Ctx *c, const float *Y, int64_t m, int64_t n, double *S, cudaStream_t s) {
  if (!core_on_tensor_cores() || !c->gram_part || m > kGramMaxRows || m < 1 || n < 1) {
    gram_f32(Y, m, n, S, s);
    return;
  }
  const int64_t ti = (m + kGmM - 1) / kGmM, tj = (m + kGmN - 1) / kGmN;
  // column ranges: enough CTAs to reach about 2 x SMs, at most kGramMaxRanges, at least 32 columns each
  int64_t nr = std::max<int64_t>(1, std::min<int64_t>((2 * (int64_t)c->num_sms) / (ti * tj), kGramMaxRanges));
  nr = std::min<int64_t>(nr, std::max<int64_t>(1, n / 32));
  const int64_t cpr = (n + nr - 1) / nr;
  nr = (n + cpr - 1) / cpr;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cap);
  if (cap == cudaStreamCaptureStatusNone)
    cudaFuncSetAttribute(gram_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gm_smem_bytes());
  gram_tc_kernel<<<dim3((unsigned)ti, (unsigned)tj, (unsigned)nr), 128, gm_smem_bytes(), s>>>(Y, m, n, cpr,
                                                                                           c->gram_part, c->d_err);
  ::tk::count_launch();
  const int64_t mm = m * m;
  gram_reduce_kernel<<<(unsigned)std::min<int64_t>((mm + 255) / 256, 4096), 256, 0, s>>>(c->gram_part, (int)nr, mm, S);
  ::tk::count_launch();
}

// The core runs on the tensor cores (core_tc_kernel + core_reduce_kernel) where R <= 64 and
// the row ranges fit the partial buffer; TUCKER_CORE_TC=0 selects the FP64 SIMT form
// (core_kernel) instead.  Both agree to FP64 rounding: on the 1M-nonzero Zipf workload
// (fit 0.84) the fits of ten sweeps differ by at most 7e-10.
static bool core_on_tensor_cores() {
  const char *e = std::getenv("TUCKER_CORE_TC");
  return !(e && e[0] == '0');
}

static int core_chunks(int num_sms, int64_t I, int64_t P, int R) {
  const int64_t tiles = ((P + 15) / 16) * ((R + 15) / 16);
  int64_t z = std::max<int64_t>(1, (2 * (int64_t)num_sms) / std::max<int64_t>(tiles, 1));
  z = std::min<int64_t>(z, std::max<int64_t>(1, (I + kCoreRows - 1) / kCoreRows));
  return (int)z;
}

size_t core_part_elems(int num_sms, int64_t P, int R) {
  // enough for the largest chunk count any mode can ask for
  return (size_t)P * R * (size_t)std::max(1, 2 * num_sms);
}

static void launch_core_fp64(Ctx *c, const float *Y, const double *U, double *G, cudaStream_t s);

template <int NP>
static void launch_core_tc(Ctx *c, const float *Y, const double *U, int64_t I, int64_t P, int R, int rows, dim3 grid,
                           double *G, cudaStream_t s) {
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cap);  // the attribute is set by the eager launches before any capture
  if (cap == cudaStreamCaptureStatusNone)
    cudaFuncSetAttribute(core_tc_kernel<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)tc_smem_bytes(kTcRows, NP));
  core_tc_kernel<NP><<<grid, 128, tc_smem_bytes(rows, NP), s>>>(Y, U, I, P, R, rows, c->core_part, c->d_err);
  ::tk::count_launch();
  const int64_t PR = P * R;
  double *bsum = c->core_part + (int64_t)(2 * c->num_sms - 1) * PR;  // after the largest partial set
  core_reduce_kernel<<<(unsigned)((PR + kRedT - 1) / kRedT), kRedT, 0, s>>>(
      c->core_part, (int)grid.y, PR, G, bsum, c->core_counter, c->norm_dev, c->norm_dev + 1, c->fit_dev);
  ::tk::count_launch();
}

void launch_core(Ctx *c, const float *Y, const double *U, double *G, cudaStream_t s) {
  const int N = c->N;
  const int64_t I = c->dims[N - 1];
  const int64_t P = c->mode[N - 1].P;
  const int R = c->ranks[N - 1];
  if (R <= 64 && I > 0 && core_on_tensor_cores()) {
    // tensor-core form: tiles of 128 columns; row ranges of 32 to 128 rows (whole chunks of
    // 16), as many as give about 2 x SMs CTAs; the partial buffer holds 2 x SMs - 1 ranges
    // (its last slot holds the reduction's block sums)
    const int64_t tiles = (P + kTcM - 1) / kTcM;
    const int64_t zmax = 2 * (int64_t)c->num_sms - 1;
    int64_t rows = (I + std::max<int64_t>(1, zmax / tiles) - 1) / std::max<int64_t>(1, zmax / tiles);
    rows = std::min<int64_t>(kTcRows, std::max<int64_t>(32, (rows + kTcK - 1) / kTcK * kTcK));
    const int64_t z = (I + rows - 1) / rows;
    if (z > zmax) return launch_core_fp64(c, Y, U, G, s);  // partials would not fit
    const dim3 grid((unsigned)tiles, (unsigned)z);
    if (R <= 16) launch_core_tc<16>(c, Y, U, I, P, R, (int)rows, grid, G, s);
    else if (R <= 32) launch_core_tc<32>(c, Y, U, I, P, R, (int)rows, grid, G, s);
    else if (R <= 48) launch_core_tc<48>(c, Y, U, I, P, R, (int)rows, grid, G, s);
    else launch_core_tc<64>(c, Y, U, I, P, R, (int)rows, grid, G, s);
    return;
  }
  launch_core_fp64(c, Y, U, G, s);
}

static void launch_core_fp64(Ctx *c, const float *Y, const double *U, double *G, cudaStream_t s) {
  const int N = c->N;
  const int64_t I = c->dims[N - 1];
  const int64_t P = c->mode[N - 1].P;
  const int R = c->ranks[N - 1];
  const int z = core_chunks(c->num_sms, I, P, R);
  const int rows_per_chunk = (int)((I + z - 1) / z);
  const dim3 grid((unsigned)((P + 15) / 16), (unsigned)((R + 15) / 16), (unsigned)z);
  core_kernel<<<grid, 256, 0, s>>>(Y, U, I, P, R, rows_per_chunk, c->core_part, c->core_counter, G, c->norm_dev,
                                   c->norm_dev + 1, c->fit_dev);
  ::tk::count_launch();
}

}  // namespace tk
