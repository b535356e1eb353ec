// K-d: core tensor of one HOOI sweep and the fit (Section III-B, eqs. ttm_ele and
// core_unfolded:  G_(N) = U_N^T Y_(N),  G[c, r] = sum_i U_N(i, r) Y_(N)(i, c)).
// Y_(N) is the FP32 TTMc output of the last mode (I_N x P), U_N the FP64 factor
// (I_N x R).  Split over rows of Y into chunks; each block owns a 16 x 16 tile of
// (column c, rank r) outputs for one row chunk and accumulates in FP64; the last
// block to finish sums the chunk partials in chunk order, writes G (C-order, r
// fastest), ||G||^2 and fit = 1 - sqrt(max(0, ||X||^2 - ||G||^2)) / ||X||.
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
// Each FP32 input is split exactly into three BF16 pieces, y = y0 + y1 + y2 (8 + 8 + 8
// significant bits), and the six tcgen05.mma kind::f16 products y_a u_b with a + b <= 2,
// smallest first, accumulate in FP32 in tensor memory; every product of two BF16 pieces is
// exact in FP32 and the three dropped ones are about 2^-23 of a product.  After each 16 rows
// the tile is read with tcgen05.ld and added into FP64 registers, so a tensor-memory
// accumulation spans six products.  Operands are staged K-major in the no-swizzle canonical
// layout (8-row x 16-byte core matrices; the descriptor's leading offset steps along K, its
// stride offset along M or N).  The FP64 tiles are written as partials; the last CTA adds
// the partials of every row range in order, as core_kernel does.
constexpr int kTcM = 128;   // columns of Y per tile (MMA M)
constexpr int kTcK = 16;    // rows of Y per staged chunk (one MMA of K = 16 per product)
constexpr int kTcKC = kTcK * 2 / 16;  // core-matrix columns (16 bytes) along K per chunk
constexpr int kTcRows = 128;  // rows of Y per CTA at most (its FP32 accumulation length)
constexpr unsigned long long kTcSpin = 1ull << 22;

__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of this architecture; base offset 0, no swizzle
  return d;
}
// y = p0 + p1 + p2 exactly (round-to-nearest pieces; every residual is exact in FP32)
__device__ __forceinline__ void bf16_split3(float v, __nv_bfloat16 &p0, __nv_bfloat16 &p1, __nv_bfloat16 &p2) {
  p0 = __float2bfloat16_rn(v);
  const float r1 = v - __bfloat162float(p0);
  p1 = __float2bfloat16_rn(r1);
  const float r2 = r1 - __bfloat162float(p1);
  p2 = __float2bfloat16_rn(r2);
}
// element (row, k) of a K-major 16-bit operand tile with kTcKC core columns per 8-row group
__device__ __forceinline__ int kmaj16(int row, int k) {
  return ((row >> 3) * kTcKC + (k >> 3)) * 64 + (row & 7) * 8 + (k & 7);
}

template <int NP>  // N of the MMA: R rounded up to 16
__global__ void __launch_bounds__(128) core_tc_kernel(const float *Y, const float *U, int64_t I, int64_t P, int R,
                                                      int rows_per_split, double *part, unsigned *counter, double *G,
                                                      const double *norm_x2, double *norm_g2, double *fit,
                                                      uint32_t *err) {
  static_assert(NP % 16 == 0 && NP >= 16 && NP <= 64, "N of the MMA");
  constexpr uint32_t kCols = NP <= 32 ? 32u : 64u;  // tensor-memory columns (a power of two >= 32)
  __shared__ __align__(1024) __nv_bfloat16 sA[3][kTcM * kTcK];
  __shared__ __align__(1024) __nv_bfloat16 sB[3][NP * kTcK];
  __shared__ __align__(8) unsigned long long bar;
  __shared__ uint32_t tbase;
  __shared__ int s_ok;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t c0 = (int64_t)blockIdx.x * kTcM;
  const int64_t i_begin = (int64_t)blockIdx.y * rows_per_split;
  const int64_t i_end = min(I, i_begin + rows_per_split);
  const uint32_t sb = (uint32_t)__cvta_generic_to_shared(&bar);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sb) : "memory");
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
  // D f32, A and B bf16, both K-major, N >> 3, M >> 4
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NP >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);
  const uint32_t lbo = 128, sbo = kTcKC * 128;  // K-adjacent core matrices, 8-row groups
  uint32_t aS[3], bS[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    aS[q] = (uint32_t)__cvta_generic_to_shared(sA[q]);
    bS[q] = (uint32_t)__cvta_generic_to_shared(sB[q]);
  }
  double accd[NP];
#pragma unroll
  for (int q = 0; q < NP; ++q) accd[q] = 0.0;
  int chunk = 0;
  bool ok = true;
  for (int64_t i0 = i_begin; i0 < i_end && ok; i0 += kTcK, ++chunk) {
    // stage: thread t owns column c0 + t of Y (coalesced rows), all rows of the chunk
    const int64_t c = c0 + tid;
    for (int k = 0; k < kTcK; ++k) {
      const int64_t i = i0 + k;
      const float v = (i < i_end && c < P) ? __ldg(Y + i * P + c) : 0.f;
      const int o = kmaj16(tid, k);
      bf16_split3(v, sA[0][o], sA[1][o], sA[2][o]);
    }
    for (int q = tid; q < NP * kTcK; q += 128) {
      const int n = q % NP, k = q / NP;
      const int64_t i = i0 + k;
      const float v = (i < i_end && n < R) ? __ldg(U + i * R + n) : 0.f;
      const int o = kmaj16(n, k);
      bf16_split3(v, sB[0][o], sB[1][o], sB[2][o]);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0) {
      // pieces a + b <= 2, the smallest products first into a fresh accumulator
      constexpr int pa[6] = {2, 1, 0, 1, 0, 0}, pb[6] = {0, 1, 2, 0, 1, 0};
#pragma unroll
      for (int st = 0; st < kTcK / 16; ++st) {  // 16 BF16 values of K per instruction: two core columns
        const uint32_t off = (uint32_t)st * 2u * 128u;
#pragma unroll
        for (int t = 0; t < 6; ++t) {
          const uint64_t ad = umma_desc(aS[pa[t]] + off, lbo, sbo), bd = umma_desc(bS[pb[t]] + off, lbo, sbo);
          const uint32_t acc = (st > 0 || t > 0) ? 1u : 0u;
          asm volatile(
              "{ .reg .pred p; setp.ne.u32 p, %4, 0; tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }" ::"r"(
                  tmem),
              "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
              : "memory");
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(sb) : "memory");
    }
    // the MMAs have read the operands (and written D) before the next chunk is staged
    bool done = false;
    for (unsigned long long it = 0; it < kTcSpin && !done; ++it) {
      uint32_t d;
      asm volatile(
          "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
          : "=r"(d)
          : "r"(sb), "r"((unsigned)(chunk & 1))
          : "memory");
      done = d != 0;
      if (!done && it > 32) __nanosleep(64);
    }
    ok = __syncthreads_and(done ? 1 : 0) != 0;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {  // this chunk's FP32 tile into the thread's FP64 row of the result
#pragma unroll
      for (int n0 = 0; n0 < NP; n0 += 16) {
        uint32_t v[16];
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)n0;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int q = 0; q < 16; ++q) accd[n0 + q] += (double)__uint_as_float(v[q]);
      }
      // every warp has read the accumulator before the next chunk's first product overwrites it
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
  }
  if (!ok) {  // record; give the products still in flight (bounded) time to end before the memory is freed
    if (tid == 0) {
      atomicOr(err, kErrTimeout);
      s_ok = 0;
      for (unsigned long long it = 0; it < kTcSpin; ++it) {
        uint32_t d;
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
            : "=r"(d)
            : "r"(sb), "r"((unsigned)((chunk - 1) & 1))
            : "memory");
        if (d) break;
        __nanosleep(64);
      }
    }
  }
  __syncthreads();
  // read the tile (warp w holds tensor-memory lanes 32w .. 32w + 31 = columns c0 + 32w + lane)
  const int64_t PR = P * R;
  const int64_t c = c0 + warp * 32 + lane;
  if (c < P)
#pragma unroll
    for (int q = 0; q < NP; ++q)
      if (q < R) part[(int64_t)blockIdx.y * PR + c * R + q] = s_ok ? accd[q] : __longlong_as_double(0x7ff8000000000000ll);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");

  // last block: partials of every row range in order, ||G||^2, fit
  __shared__ bool is_last;
  __threadfence();
  __syncthreads();
  if (tid == 0) is_last = atomicAdd(counter, 1u) == gridDim.x * gridDim.y - 1u;
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  __shared__ double red[128];
  double g2 = 0.0;
  for (int64_t q = tid; q < PR; q += 128) {
    double t = 0.0;
    for (int z = 0; z < (int)gridDim.y; ++z) t += __ldcg(part + (int64_t)z * PR + q);
    G[q] = t;
    g2 = fma(t, t, g2);
  }
  red[tid] = g2;
  __syncthreads();
  for (int o = 64; o > 0; o >>= 1) {
    if (tid < o) red[tid] += red[tid + o];
    __syncthreads();
  }
  if (tid == 0) {
    const double gx = red[0];
    const double nx = *norm_x2;
    *norm_g2 = gx;
    *fit = (nx > 0.0) ? 1.0 - sqrt(fmax(0.0, nx - gx)) / sqrt(nx) : 1.0;
    *counter = 0u;
  }
}

// TUCKER_CORE_TC=1 runs the core on the tensor cores (core_tc_kernel) where R <= 64.
// It is not the default: the tensor cores accumulate in FP32 with a directed rounding, so
// even with every 16 rows moved into FP64 the core is FP32-accurate (relative error about
// 3e-7 on the 1M-nonzero Zipf workload), and where the fit is high that is amplified:
// there (fit 0.84) the fit came out 1.5e-6 to 1.8e-6 low against the FP64 oracle, above the
// 1e-6 bar that core_kernel's FP64 accumulation meets.  Measured and tested as an option.
static bool core_on_tensor_cores() {
  const char *e = std::getenv("TUCKER_CORE_TC");
  return e && e[0] == '1';
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

void launch_core(Ctx *c, const float *Y, const double *U, double *G, cudaStream_t s) {
  const int N = c->N;
  const int64_t I = c->dims[N - 1];
  const int64_t P = c->mode[N - 1].P;
  const int R = c->ranks[N - 1];
  if (R <= 64 && I > 0 && core_on_tensor_cores()) {
    // tensor-core form: tiles of 128 columns, rows split so that about 2 x SMs CTAs run,
    // each over at least 4 chunks of 32 rows; the partial buffer holds 2 x SMs tiles
    const int64_t tiles = (P + kTcM - 1) / kTcM;
    int64_t z = std::max<int64_t>(1, (I + kTcRows - 1) / kTcRows);  // at most 128 rows per CTA
    if (z > 2 * (int64_t)c->num_sms) return launch_core_fp64(c, Y, U, G, s);  // partials would not fit
    const int rows = (int)((I + z - 1) / z);
    const dim3 grid((unsigned)tiles, (unsigned)z);
    const float *U32 = c->U32[N - 1];
    double *ng = c->norm_dev + 1;
#define TK_CORE_TC(NP_)                                                                                            \
  core_tc_kernel<NP_><<<grid, 128, 0, s>>>(Y, U32, I, P, R, rows, c->core_part, c->core_counter, G, c->norm_dev, ng, \
                                          c->fit_dev, c->d_err)
    if (R <= 16) TK_CORE_TC(16);
    else if (R <= 32) TK_CORE_TC(32);
    else if (R <= 48) TK_CORE_TC(48);
    else TK_CORE_TC(64);
#undef TK_CORE_TC
    ::tk::count_launch();
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
