// K-b: sparse TTMc of one mode (Algorithm 2 inner loop; Section III-C):
//     Y_(n)(i_n, :) = sum_{z in slice i_n} x_z * kron_{m != n} U_m(i_m(z), :)
//
// GPU design.  The remaining modes are split into a "left" group (all but the last,
// Kronecker length PL) and the last mode (length RB), so that one nonzero contributes
// the rank-1 block (x_z a_z) b_z^T of a PL x RB row, with a_z the Kronecker of the left
// rows (Algorithm 4 layout: c = ra * RB + rb, last mode fastest).  One warp owns one
// work unit of consecutive sorted nonzeros (a run of whole slices, or a piece of a long
// slice).  Per tile of 32 nonzeros the warp
//   1. loads indices and values coalesced (lane = position) and finds the slice of every
//      position from 32 slice offsets with one OR-reduction (no per-nonzero row index
//      is stored);
//   2. gathers the factor rows with 16-byte vector loads into shared memory, scaling
//      the left Kronecker row by x_z;
//   3. accumulates each slice segment in registers: the warp is cut into NG groups of
//      G lanes, each lane owns a TA x TB block of the row, the groups take alternate
//      nonzeros and are merged by warp shuffles when the segment closes;
//   4. writes the finished row to Y_(n) (or, for a piece of a long slice, to a partial
//      row that a second kernel sums in piece order).
// No global atomics: every output element has one writer, so Y is bitwise reproducible.
#include <algorithm>
#include <cstdlib>

#include "dfloat.cuh"
#include "internal.cuh"

namespace tk {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kTtmcWarps = 8;

struct TtmcParams {
  const uint32_t *idx[kMaxOrder];  // sorted coordinates of the remaining modes (ascending)
  const void *U[kMaxOrder];        // their factors (float or bf16), row-major I_m x R_m
  int R[kMaxOrder];                // their ranks
  int nother;
  const float *val;
  const uint32_t *sptr;
  const uint32_t *sid;
  uint32_t S;
  const uint32_t *unit_e0;
  const uint32_t *unit_k0;
  const int32_t *unit_slot;
  int64_t n_units;
  uint32_t Z;
  float *Y;
  float *carry;
  int64_t P;
  uint32_t *err;         // the context's error word (bounded waits that gave up)
  const uint32_t *fptr;  // fiber form: [F+1] first nonzero of each fiber (positions above are fibers)
  const uint32_t *fmid;  // fiber form: [F] index of the first remaining mode of each fiber
  float2 *sq_part;       // pipelined form: [blocks][P] column sums of squares of the whole rows each
                         // block wrote (double-float pairs), nullptr: not formed
};

// Slice structure of the tile [e, e + nt) of sorted positions, kb = slice of position e.
struct TileSlices {
  uint32_t starts;     // bit p: a new slice starts at position p of the tile (p >= 1)
  uint32_t kp;         // slice index of position `lane`
  bool end_is_start;   // position e + nt starts a new slice (or is the end of all nonzeros)
  uint32_t kb_next;    // slice of position e + nt
};

__device__ __forceinline__ TileSlices tile_slices(const uint32_t *__restrict__ sptr, uint32_t S, uint32_t kb,
                                                  uint32_t e, int nt, int lane) {
  const uint32_t k = kb + 1u + (uint32_t)lane;
  const uint32_t bound = (k <= S) ? __ldg(sptr + k) : 0xffffffffu;
  const uint32_t q = bound - e;  // >= 1: slice kb contains e
  uint32_t starts = __reduce_or_sync(kFull, q < 32u ? (1u << q) : 0u);
  starts &= (nt >= 32) ? kFull : ((1u << nt) - 1u);
  TileSlices t;
  t.starts = starts;
  t.kp = kb + __popc(starts & ((2u << lane) - 1u));
  t.end_is_start = __any_sync(kFull, q == (uint32_t)nt);
  t.kb_next = kb + __popc(__ballot_sync(kFull, q <= (uint32_t)nt));
  return t;
}

template <typename FT>
struct Ld;
template <>
struct Ld<float> {
  static __device__ __forceinline__ float4 v4(const float *row, int c) {
    return __ldg(reinterpret_cast<const float4 *>(row + c));
  }
  static __device__ __forceinline__ float s(const float *row, int c) { return __ldg(row + c); }
};
template <>
struct Ld<__nv_bfloat16> {
  static __device__ __forceinline__ float4 v4(const __nv_bfloat16 *row, int c) {
    uint2 raw = __ldg(reinterpret_cast<const uint2 *>(row + c));
    float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&raw.x));
    float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&raw.y));
    return make_float4(a.x, a.y, b.x, b.y);
  }
  static __device__ __forceinline__ float s(const __nv_bfloat16 *row, int c) { return __bfloat162float(row[c]); }
};

template <int T>
__device__ __forceinline__ void lds(const float *p, float (&v)[T]) {
  if constexpr (T % 4 == 0) {
#pragma unroll
    for (int i = 0; i < T; i += 4) {
      float4 q = *reinterpret_cast<const float4 *>(p + i);
      v[i] = q.x;
      v[i + 1] = q.y;
      v[i + 2] = q.z;
      v[i + 3] = q.w;
    }
  } else if constexpr (T % 2 == 0) {
#pragma unroll
    for (int i = 0; i < T; i += 2) {
      float2 q = *reinterpret_cast<const float2 *>(p + i);
      v[i] = q.x;
      v[i + 1] = q.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < T; ++i) v[i] = p[i];
  }
}

// NL = number of left modes (0, 1 or 2); PL = product of their ranks; RB = rank of the
// last remaining mode.  Requires RB % 4 == 0, and for NL == 2 the second left rank % 4 == 0.
template <int NL, int PL, int RB, int TA, int TB, typename FT>
__global__ void __launch_bounds__(kTtmcWarps * 32) ttmc_fast_kernel(const TtmcParams p) {
  constexpr int G = (PL / TA) * (RB / TB);  // lanes per group
  constexpr int NG = 32 / G;                // groups per warp
  static_assert(G * NG == 32, "group size must divide the warp");
  static_assert(RB % 4 == 0, "last rank must be a multiple of 4");
  extern __shared__ float4 smem_f4[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float *xa = reinterpret_cast<float *>(smem_f4) + w * 32 * (PL + RB);
  float *bb = xa + 32 * PL;
  const int64_t u = (int64_t)blockIdx.x * kTtmcWarps + w;
  if (u >= p.n_units) return;

  const FT *UB = static_cast<const FT *>(p.U[NL]);
  const uint32_t *idxB = p.idx[NL];
  uint32_t e = __ldg(p.unit_e0 + u);
  const uint32_t e_end = (u + 1 < p.n_units) ? __ldg(p.unit_e0 + u + 1) : p.Z;
  uint32_t kb = __ldg(p.unit_k0 + u);
  const int slot = __ldg(p.unit_slot + u);

  const int g = lane / G, j = lane % G;
  const int ra0 = (j / (RB / TB)) * TA, rb0 = (j % (RB / TB)) * TB;
  float acc[TA][TB];
#pragma unroll
  for (int a = 0; a < TA; ++a)
#pragma unroll
    for (int b = 0; b < TB; ++b) acc[a][b] = 0.f;

  while (e < e_end) {
    const int nt = (int)min(32u, e_end - e);
    const TileSlices ts = tile_slices(p.sptr, p.S, kb, e, nt, lane);

    float x = 0.f;
    uint32_t i0 = 0, i1 = 0, ib = 0;
    if (lane < nt) {
      x = __ldg(p.val + e + lane);
      ib = __ldg(idxB + e + lane);
      if constexpr (NL >= 1) i0 = __ldg(p.idx[0] + e + lane);
      if constexpr (NL >= 2) i1 = __ldg(p.idx[1] + e + lane);
    }
    __syncwarp();
    // ---- stage x * kron(left rows) and the last-mode rows
    if constexpr (NL == 0) {
      xa[lane] = x;
    } else if constexpr (NL == 1) {
      const FT *U0 = static_cast<const FT *>(p.U[0]);
#pragma unroll
      for (int it = lane; it < 32 * (PL / 4); it += 32) {
        const int t = it / (PL / 4), c = (it % (PL / 4)) * 4;
        const float xt = __shfl_sync(kFull, x, t);
        const uint32_t r = __shfl_sync(kFull, i0, t);
        float4 v = Ld<FT>::v4(U0 + (size_t)r * PL, c);
        v.x *= xt;
        v.y *= xt;
        v.z *= xt;
        v.w *= xt;
        *reinterpret_cast<float4 *>(xa + t * PL + c) = v;
      }
    } else {
      const FT *U0 = static_cast<const FT *>(p.U[0]);
      const FT *U1 = static_cast<const FT *>(p.U[1]);
      const int R1 = p.R[1], R0 = p.R[0];
#pragma unroll 4
      for (int it = lane; it < 32 * (PL / 4); it += 32) {
        const int t = it / (PL / 4), c = (it % (PL / 4)) * 4;
        const float xt = __shfl_sync(kFull, x, t);
        const uint32_t r0 = __shfl_sync(kFull, i0, t);
        const uint32_t r1 = __shfl_sync(kFull, i1, t);
        const int a0 = c / R1, a1 = c - a0 * R1;
        const float s0 = xt * Ld<FT>::s(U0 + (size_t)r0 * R0, a0);
        float4 v = Ld<FT>::v4(U1 + (size_t)r1 * R1, a1);
        v.x *= s0;
        v.y *= s0;
        v.z *= s0;
        v.w *= s0;
        *reinterpret_cast<float4 *>(xa + t * PL + c) = v;
      }
    }
#pragma unroll
    for (int it = lane; it < 32 * (RB / 4); it += 32) {
      const int t = it / (RB / 4), c = (it % (RB / 4)) * 4;
      const uint32_t r = __shfl_sync(kFull, ib, t);
      *reinterpret_cast<float4 *>(bb + t * RB + c) = Ld<FT>::v4(UB + (size_t)r * RB, c);
    }
    __syncwarp();

    // ---- segments of equal slice inside the tile
    uint32_t segs = ts.starts | 1u;
    while (segs) {
      const int p0 = __ffs(segs) - 1;
      segs &= segs - 1u;
      const int p1 = segs ? (__ffs(segs) - 1) : nt;
      int q = p0 + g;
      auto step = [&](int qq) {
        float av[TA], bv[TB];
        lds<TA>(xa + qq * PL + ra0, av);
        lds<TB>(bb + qq * RB + rb0, bv);
#pragma unroll
        for (int a = 0; a < TA; ++a)
#pragma unroll
          for (int b = 0; b < TB; ++b) acc[a][b] = fmaf(av[a], bv[b], acc[a][b]);
      };
      for (; q + NG < p1; q += 2 * NG) {
        step(q);
        step(q + NG);
      }
      if (q < p1) step(q);
      const bool flush = (p1 < nt) || ts.end_is_start || (e + (uint32_t)nt == e_end);
      if (flush) {
#pragma unroll
        for (int o = G; o < 32; o <<= 1)
#pragma unroll
          for (int a = 0; a < TA; ++a)
#pragma unroll
            for (int b = 0; b < TB; ++b) acc[a][b] += __shfl_xor_sync(kFull, acc[a][b], o);
        const uint32_t kseg = __shfl_sync(kFull, ts.kp, p0);
        if (g == 0) {
          float *dst = (slot >= 0) ? p.carry + (size_t)slot * p.P : p.Y + (size_t)__ldg(p.sid + kseg) * p.P;
#pragma unroll
          for (int a = 0; a < TA; ++a) {
            float *d = dst + (size_t)(ra0 + a) * RB + rb0;
            if constexpr (TB % 4 == 0) {
#pragma unroll
              for (int b = 0; b < TB; b += 4)
                *reinterpret_cast<float4 *>(d + b) = make_float4(acc[a][b], acc[a][b + 1], acc[a][b + 2], acc[a][b + 3]);
            } else {
#pragma unroll
              for (int b = 0; b < TB; ++b) d[b] = acc[a][b];
            }
          }
        }
#pragma unroll
        for (int a = 0; a < TA; ++a)
#pragma unroll
          for (int b = 0; b < TB; ++b) acc[a][b] = 0.f;
      }
    }
    kb = ts.kb_next;
    e += (uint32_t)nt;
    __syncwarp();
  }
}

// ============================================================================ pipelined form
// s += (x.x + x.y): TwoSum of the high parts, every rounding error into the low part
__device__ __forceinline__ void sq_add(DF &s, float2 x) {
  const float t = s.hi + x.x, bp = t - s.hi;
  s.lo += ((s.hi - (t - bp)) + (x.x - bp)) + x.y;
  s.hi = t;
}

// The arithmetic of ttmc_fast_kernel (order 3: one left mode) with the global latency of
// each tile shortened: the slice offsets, indices and values of tile t+1 are loaded into
// registers while tile t is staged and computed, so a tile waits on one round trip (the
// L1-cached factor-row gathers) instead of three chained ones.
// SQ form of the pipelined TTMc, after a warp's last tile: the rows it wrote whole (slices
// kfirst .. kfirst + nrows - 1), read back through L2 (lane l: columns CPL l .. CPL l + CPL - 1),
// their exact squares summed in double-float pairs into the warp's staging area (warp w's
// at smem + w * ws floats).  The last warp of the block to arrive adds the eight warps'
// pairs in warp order to sq_part[block]: no block barrier, so warps without a unit leave early.
template <int P>
__device__ __forceinline__ void sq_rows_finish(const TtmcParams &p, float *smem, int ws, uint32_t kfirst,
                                               uint32_t nrows, unsigned *arrived) {
  constexpr int CPL = P / 32;
  static_assert(CPL % 2 == 0, "column pairs per lane");
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  DF q[CPL];
  __syncwarp();  // this warp's rows of Y are visible to all its lanes
#pragma unroll 1
  for (uint32_t r = 0; r < nrows; ++r) {
    const float2 *y = reinterpret_cast<const float2 *>(p.Y + (size_t)__ldg(p.sid + kfirst + r) * P + lane * CPL);
    float2 v[CPL / 2];
#pragma unroll
    for (int c = 0; c < CPL / 2; ++c) v[c] = __ldcg(y + c);
#pragma unroll
    for (int c = 0; c < CPL / 2; ++c) {
      df_fma(q[2 * c], v[c].x, v[c].x, 0.f);
      df_fma(q[2 * c + 1], v[c].y, v[c].y, 0.f);
    }
  }
  float2 *mine = reinterpret_cast<float2 *>(smem + w * ws);  // the tiles are done: the area is free
#pragma unroll
  for (int c = 0; c < CPL; ++c) mine[lane * CPL + c] = make_float2(q[c].hi, q[c].lo);
  __syncwarp();  // the warp's pairs are written ...
  unsigned before = 0;
  if (lane == 0) {
    __threadfence_block();  // ... and ordered before its arrival
    before = atomicAdd(arrived, 1u);
    if (before == kTtmcWarps - 1) __threadfence_block();  // every arrival's pairs before the reads
  }
  before = __shfl_sync(0xffffffffu, before, 0);  // (and the warp's lanes after lane 0's fence)
  if (before != kTtmcWarps - 1) return;
  for (int c = lane; c < P; c += 32) {
    DF t;
    for (int ww = 0; ww < kTtmcWarps; ++ww) sq_add(t, reinterpret_cast<const float2 *>(smem + ww * ws)[c]);
    p.sq_part[(size_t)blockIdx.x * P + c] = make_float2(t.hi, t.lo);
  }
}

template <int PL, int RB, int TA, int TB, bool SQ>
__device__ __forceinline__ void ttmc_pipe_body(const TtmcParams &p) {
  constexpr int G = (PL / TA) * (RB / TB);
  constexpr int NG = 32 / G;
  static_assert(G * NG == 32, "group size must divide the warp");
  static_assert(PL % 4 == 0 && RB % 4 == 0, "16-byte row pieces");
  static_assert(!SQ || PL * RB * 2 <= 32 * (PL + RB), "SQ: a warp's pairs fit its staging area");
  extern __shared__ float4 smem_f4[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float *xa = reinterpret_cast<float *>(smem_f4) + w * 32 * (PL + RB);
  float *bb = xa + 32 * PL;
  // SQ: a unit with slot < 0 holds whole slices only, the consecutive slices from its first,
  // kfirst, to the one that starts where it ends (kb after its last tile); their rows'
  // squares are summed after the last tile
  uint32_t kfirst = 0, nrows = 0;
  __shared__ unsigned s_sq_arrived;  // SQ: warps whose pairs are in their staging areas
  if constexpr (SQ) {
    if (threadIdx.x == 0) s_sq_arrived = 0u;
    __syncthreads();
  }
  const int64_t u = (int64_t)blockIdx.x * kTtmcWarps + w;
  if (u >= p.n_units) {
    if constexpr (SQ) sq_rows_finish<PL * RB>(p, reinterpret_cast<float *>(smem_f4), 32 * (PL + RB), 0u, 0u, &s_sq_arrived);
    return;
  }
  {
  const float *UA = static_cast<const float *>(p.U[0]);
  const float *UB = static_cast<const float *>(p.U[1]);
  const uint32_t *idxA = p.idx[0];
  const uint32_t *idxB = p.idx[1];
  const uint32_t e0 = __ldg(p.unit_e0 + u);
  const uint32_t e_end = (u + 1 < p.n_units) ? __ldg(p.unit_e0 + u + 1) : p.Z;
  const int slot = __ldg(p.unit_slot + u);
  const int ntiles = (int)((e_end - e0 + 31u) / 32u);
  const int g = lane / G, j = lane % G;
  const int ra0 = (j / (RB / TB)) * TA, rb0 = (j % (RB / TB)) * TB;
  float acc[TA][TB];
#pragma unroll
  for (int a = 0; a < TA; ++a)
#pragma unroll
    for (int b = 0; b < TB; ++b) acc[a][b] = 0.f;

  uint32_t kb = __ldg(p.unit_k0 + u);
  uint32_t bound = (kb + 1u + lane <= p.S) ? __ldg(p.sptr + kb + 1u + lane) : 0xffffffffu;
  float x = 0.f;
  uint32_t ia = 0u, ib = 0u;
  if (e0 + lane < e_end) {
    x = __ldg(p.val + e0 + lane);
    ia = __ldg(idxA + e0 + lane);
    ib = __ldg(idxB + e0 + lane);
  }
  for (int t = 0; t < ntiles; ++t) {
    const uint32_t e = e0 + 32u * (uint32_t)t;
    const int nt = (int)min(32u, e_end - e);
    const uint32_t q = bound - e;
    uint32_t starts = __reduce_or_sync(kFull, q < 32u ? (1u << q) : 0u);
    starts &= (nt >= 32) ? kFull : ((1u << nt) - 1u);
    const uint32_t kp = kb + __popc(starts & ((2u << lane) - 1u));
    const bool end_is_start = __any_sync(kFull, q == (uint32_t)nt);
    const uint32_t kb_next = kb + __popc(__ballot_sync(kFull, q <= (uint32_t)nt));
    // loads of tile t+1 (consumed next iteration)
    const uint32_t bound_next = (kb_next + 1u + lane <= p.S) ? __ldg(p.sptr + kb_next + 1u + lane) : 0xffffffffu;
    float xn = 0.f;
    uint32_t ian = 0u, ibn = 0u;
    const uint32_t posn = e + 32u + (uint32_t)lane;
    if (posn < e_end) {
      xn = __ldg(p.val + posn);
      ian = __ldg(idxA + posn);
      ibn = __ldg(idxB + posn);
    }
    // stage tile t: x * left rows, last-mode rows
#pragma unroll
    for (int it = lane; it < 32 * (PL / 4); it += 32) {
      const int tt = it / (PL / 4), c = (it % (PL / 4)) * 4;
      const float xt = __shfl_sync(kFull, x, tt);
      const uint32_t r = __shfl_sync(kFull, ia, tt);
      float4 v = __ldg(reinterpret_cast<const float4 *>(UA + (size_t)r * PL + c));
      v.x *= xt;
      v.y *= xt;
      v.z *= xt;
      v.w *= xt;
      *reinterpret_cast<float4 *>(xa + tt * PL + c) = v;
    }
#pragma unroll
    for (int it = lane; it < 32 * (RB / 4); it += 32) {
      const int tt = it / (RB / 4), c = (it % (RB / 4)) * 4;
      const uint32_t r = __shfl_sync(kFull, ib, tt);
      *reinterpret_cast<float4 *>(bb + tt * RB + c) = __ldg(reinterpret_cast<const float4 *>(UB + (size_t)r * RB + c));
    }
    __syncwarp();
    uint32_t segs = starts | 1u;
    while (segs) {
      const int p0 = __ffs(segs) - 1;
      segs &= segs - 1u;
      const int p1 = segs ? (__ffs(segs) - 1) : nt;
      int qq = p0 + g;
      auto step = [&](int r) {
        float av[TA], bv[TB];
        lds<TA>(xa + r * PL + ra0, av);
        lds<TB>(bb + r * RB + rb0, bv);
#pragma unroll
        for (int a = 0; a < TA; ++a)
#pragma unroll
          for (int b = 0; b < TB; ++b) acc[a][b] = fmaf(av[a], bv[b], acc[a][b]);
      };
      for (; qq + NG < p1; qq += 2 * NG) {
        step(qq);
        step(qq + NG);
      }
      if (qq < p1) step(qq);
      const bool flush = (p1 < nt) || end_is_start || (e + (uint32_t)nt == e_end);
      if (flush) {
#pragma unroll
        for (int o = G; o < 32; o <<= 1)
#pragma unroll
          for (int a = 0; a < TA; ++a)
#pragma unroll
            for (int b = 0; b < TB; ++b) acc[a][b] += __shfl_xor_sync(kFull, acc[a][b], o);
        const uint32_t kseg = __shfl_sync(kFull, kp, p0);
        if (g == 0) {
          float *dst = (slot >= 0) ? p.carry + (size_t)slot * p.P : p.Y + (size_t)__ldg(p.sid + kseg) * p.P;
#pragma unroll
          for (int a = 0; a < TA; ++a) {
            float *d = dst + (size_t)(ra0 + a) * RB + rb0;
#pragma unroll
            for (int b = 0; b < TB; b += 4)
              *reinterpret_cast<float4 *>(d + b) = make_float4(acc[a][b], acc[a][b + 1], acc[a][b + 2], acc[a][b + 3]);
          }
        }
#pragma unroll
        for (int a = 0; a < TA; ++a)
#pragma unroll
          for (int b = 0; b < TB; ++b) acc[a][b] = 0.f;
      }
    }
    __syncwarp();
    kb = kb_next;
    bound = bound_next;
    x = xn;
    ia = ian;
    ib = ibn;
  }
  if constexpr (SQ) {  // the unit's index and tables are read again: nothing more stays live
    const int64_t uu = (int64_t)blockIdx.x * kTtmcWarps + (threadIdx.x >> 5);
    if (__ldg(p.unit_slot + uu) < 0) {
      kfirst = __ldg(p.unit_k0 + uu);
      nrows = kb - kfirst;
    }
  }
  }
  if constexpr (SQ) {
    sq_rows_finish<PL * RB>(p, reinterpret_cast<float *>(smem_f4), 32 * (PL + RB), kfirst, nrows, &s_sq_arrived);
  }
}

template <int PL, int RB, int TA, int TB>
__global__ void __launch_bounds__(kTtmcWarps * 32) ttmc_pipe_kernel(const TtmcParams p) {
  ttmc_pipe_body<PL, RB, TA, TB, false>(p);
}

// The same, also forming the column sums of squares of the rows it writes (p.sq_part, one
// row of P pairs per block); held to 64 registers, the occupancy of the plain form.
template <int PL, int RB, int TA, int TB>
__global__ void __launch_bounds__(kTtmcWarps * 32, 4) ttmc_pipe_sq_kernel(const TtmcParams p) {
  ttmc_pipe_body<PL, RB, TA, TB, true>(p);
}

// ============================================================================ fiber form
// Order 3 with a fiber level (Section III-C, CSF): within a slice, the nonzeros that
// share the index i_a of the first remaining mode form a fiber f (cut every kFiberCap
// nonzeros); the slice row is the sum over its fibers of U_a(i_a(f), :) (x) t_f with
//     t_f = sum over the nonzeros of f of x_z U_b(i_b(z), :),
// so the RB-term sum is formed once per nonzero and the PL x RB rank-1 update once per
// fiber.  Two passes over fiber work units:
//   1. ttmc_fibsum_kernel writes t_f for every fiber (below);
//   2. the nonzero form's pipelined kernel runs over the fibers as if they were nonzeros,
//      with index stream fmid (rows of U_a), value 1 and the t_f rows as its last-mode rows
//      (an identity index into t), so slices, split slices and the fixup are shared.
//
// Pass 1: one warp per run of `fpw` fibers (any run of whole fibers will do: t_f does not
// depend on slices).  One fiber per group of QL = RB/4 lanes (lane q of the group owns the
// column quad t_f[4q, 4q+4)), 32/QL fibers of the warp side by side; a group adds its
// fiber's positions in order (fibers are at most kFiberCap long), with the values, indices
// and factor rows of four positions in flight at a time; with four or more lanes per fiber
// the values and indices of the four positions are loaded once (one position per lane) and
// shared by shuffles within the group.  One fixed order: t is reproducible.
template <int RB>
__global__ void __launch_bounds__(kTtmcWarps * 32) ttmc_fibsum_kernel(const TtmcParams p, float *__restrict__ T,
                                                                     int64_t fpw) {
  constexpr int QL = RB / 4;   // lanes per fiber
  constexpr int FG = 32 / QL;  // fibers side by side in a warp
  static_assert(RB % 4 == 0 && 32 % QL == 0, "RB in {4, 8, 16, 32}");
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t u = (int64_t)blockIdx.x * kTtmcWarps + w;  // this warp's fibers: [u fpw, u fpw + fpw)
  if (u * fpw >= (int64_t)p.Z) return;
  const float4 *UB4 = static_cast<const float4 *>(p.U[1]);
  const uint32_t *idxB = p.idx[1];
  const int g = lane / QL, q = lane % QL;
  const uint32_t f_begin = (uint32_t)(u * fpw);
  const uint32_t f_end = (uint32_t)min((int64_t)p.Z, u * fpw + fpw);
  float4 *T4 = reinterpret_cast<float4 *>(T);
  for (uint32_t fr = f_begin; fr < f_end; fr += FG) {
    const uint32_t f = fr + (uint32_t)g;
    if (f >= f_end) continue;
    const uint32_t zs = __ldg(p.fptr + f), ze = __ldg(p.fptr + f + 1);
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (uint32_t z = zs; z < ze; z += 4u) {
      float xv[4];
      uint32_t iv[4];
      if constexpr (QL >= 4) {
        // lane q < 4 of the group loads position z + q; the group's lanes (all on this
        // fiber, so all in this loop) take the four values and indices by shuffle
        const unsigned gmask = ((QL == 32) ? 0xffffffffu : ((1u << QL) - 1u)) << (g * QL);
        const uint32_t zq = z + (uint32_t)q;
        float xm = 0.f;
        uint32_t im = 0u;
        if (q < 4 && zq < ze) {
          xm = __ldg(p.val + zq);
          im = __ldg(idxB + zq);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          xv[k] = __shfl_sync(gmask, xm, k, QL);
          iv[k] = __shfl_sync(gmask, im, k, QL);
        }
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const bool in = z + (uint32_t)k < ze;
          xv[k] = in ? __ldg(p.val + z + k) : 0.f;
          iv[k] = in ? __ldg(idxB + z + k) : 0u;
        }
      }
      float4 r[4];
#pragma unroll
      for (int k = 0; k < 4; ++k)
        r[k] = (z + (uint32_t)k < ze) ? __ldg(UB4 + (size_t)iv[k] * QL + q) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        acc.x = fmaf(xv[k], r[k].x, acc.x);
        acc.y = fmaf(xv[k], r[k].y, acc.y);
        acc.z = fmaf(xv[k], r[k].z, acc.z);
        acc.w = fmaf(xv[k], r[k].w, acc.w);
      }
    }
    T4[(size_t)f * QL + q] = acc;
  }
}

// ============================================================================ fused fiber form
// Both levels of the fiber form in one kernel, the fiber sums never leaving the chip.
// One warp per nonzero work unit [z0, z1) (the nonzero form's units: runs of whole slices of
// about `chunk` nonzeros, or one piece of a longer slice).  A fiber cut by a piece boundary
// is a fiber of each piece: both pieces belong to one long slice, whose partial rows the
// fixup kernel adds, and the fiber's rank-1 update is linear in its sum.
//   Level 1, per window of kWin consecutive nonzeros: lane (block pb, quad q) adds
//     x_z U_s(i_s(z), 4q..4q+3) over the PB positions of its block in order (U_s: the
//     factor of the summed mode; rows gathered coalesced, QL lanes per row), closing the
//     fibers that start and end inside the block; the pieces before a block's first fiber
//     start and after its last are joined across blocks by a shuffle scan of the maps
//     "A -> A + lead" (no start) and "A -> trail" (a start), applied to the fiber carried
//     over from the previous window.  Fiber starts come from a per-position bit mask.
//     Finished t_f go to a per-warp ring in shared memory (kRing rows).
//   Level 2, whenever 32 finished fibers wait (and at the unit's end): the pipelined
//     kernel's tile over fibers: rows U_m(fmid(f)) of the middle mode gathered, rows t_f
//     from the ring, a TA x TB block of the slice row per lane, NG groups merged by
//     shuffles where a slice closes, rows written to Y (or to a partial-row slot).
// MIDA: the middle mode is the first remaining mode (Y column = r_mid * RS + r_sum);
// otherwise it is the last one (Y column = r_sum * RM + r_mid).  Fixed orders: Y is
// reproducible bit for bit.
constexpr int kFibWarps = 4;

struct FiberParams {
  const float *val;      // [Z] values, in the copy's order
  const uint32_t *isum;  // [Z] index of the summed mode
  const void *Usum;      // its factor (float or bf16), I x RS
  const void *Umid;      // factor of the middle mode, I x RM
  const uint32_t *fptr;  // [F+1]
  const uint32_t *fmid;  // [F]
  const uint32_t *fbits; // fiber starts, one bit per position (zero padded)
  const uint32_t *fsptr; // [S+1] first fiber of each non-empty slice
  const uint32_t *sid;   // [S]
  uint32_t S, F, Z;
  const uint32_t *unit_e0;  // [n_units] first position of each unit
  const uint32_t *unit_f0;  // [n_units] fiber containing it
  const uint32_t *unit_k0;  // [n_units] slice containing it
  const int32_t *unit_slot;
  int64_t n_units;
  float *Y;
  float *carry;
  int64_t P;
};

template <typename FT>
__device__ __forceinline__ float4 row4(const FT *U, uint32_t r, int R, int c) {
  return Ld<FT>::v4(U + (size_t)r * R, c);
}

constexpr int kWinDefault = 64;  // nonzeros per level-1 window

// 64 bits of the start mask beginning at position z
__device__ __forceinline__ uint64_t start_bits64(const uint32_t *__restrict__ fbits, uint32_t z) {
  const uint32_t w = z >> 5, sh = z & 31u;
  const uint32_t a = __ldg(fbits + w), b = __ldg(fbits + w + 1), c = __ldg(fbits + w + 2);
  const uint32_t lo = __funnelshift_r(a, b, sh), hi = __funnelshift_r(b, c, sh);
  return ((uint64_t)hi << 32) | lo;
}

template <int RM, int RS, int TA, int TB, bool MIDA, typename FT, int kWin = 64, int MINB = 1>
__global__ void __launch_bounds__(kFibWarps * 32, MINB) ttmc_fiber_kernel(const FiberParams p) {
  constexpr int kRing = 2 * kWin;  // ring rows: < 32 waiting + at most kWin + 1 finished per window
  constexpr int PL = MIDA ? RM : RS, RB = MIDA ? RS : RM;
  constexpr int G = (PL / TA) * (RB / TB);
  constexpr int NG = 32 / G;
  static_assert(G * NG == 32, "group size must divide the warp");
  static_assert(RM % 4 == 0 && RS % 4 == 0, "16-byte row pieces");
  constexpr int QL = RS / 4;          // lanes per summed-mode row
  constexpr int PG = 32 / QL;         // position blocks per window
  constexpr int PB = kWin / PG;       // positions per block
  static_assert(QL * PG == 32 && PB * PG == kWin && PG <= 32, "window layout");
  constexpr int WARP_FLOATS = kRing * RS + 32 * RM + 2 * (kWin + 32);
  // window entry of position t, one spare entry per block so that the blocks' reads fall in
  // distinct banks
  auto xsi = [](int t) { return t + t / PB; };
  extern __shared__ float4 smem_f4[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float *ring = reinterpret_cast<float *>(smem_f4) + (size_t)w * WARP_FLOATS;
  float *stage = ring + kRing * RS;                                 // 32 gathered middle-mode rows
  uint2 *xs = reinterpret_cast<uint2 *>(stage + 32 * RM);           // window values and indices
  float4 *ring4 = reinterpret_cast<float4 *>(ring);
  const int64_t u = (int64_t)blockIdx.x * kFibWarps + w;
  if (u >= p.n_units) return;
  const FT *US = static_cast<const FT *>(p.Usum);
  const FT *UM = static_cast<const FT *>(p.Umid);
  const uint32_t f0 = __ldg(p.unit_f0 + u);
  const uint32_t z0 = __ldg(p.unit_e0 + u);
  const uint32_t z1 = (u + 1 < p.n_units) ? __ldg(p.unit_e0 + u + 1) : p.Z;
  // one past the unit's last fiber (the next unit may begin inside it)
  const uint32_t f1 = (u + 1 < p.n_units)
                          ? __ldg(p.unit_f0 + u + 1) + (((__ldg(p.fbits + (z1 >> 5)) >> (z1 & 31u)) & 1u) ? 0u : 1u)
                          : p.F;
  const int slot = __ldg(p.unit_slot + u);
  const int q = lane % QL, pb = lane / QL, P0 = pb * PB;
  const int g = lane / G, j = lane % G;
  const int ra0 = (j / (RB / TB)) * TA, rb0 = (j % (RB / TB)) * TB;
  auto ring_slot = [&](uint32_t f) { return (int)((f - f0) & (uint32_t)(kRing - 1)); };

  float acc[TA][TB];
#pragma unroll
  for (int a = 0; a < TA; ++a)
#pragma unroll
    for (int b = 0; b < TB; ++b) acc[a][b] = 0.f;
  uint32_t kb2 = __ldg(p.unit_k0 + u);  // slice of fiber fdone
  uint32_t fdone = f0;                  // level 2 has consumed fibers [f0, fdone)
  uint32_t fcur = f0;                   // fiber open at the end of the last window
  float4 carry = make_float4(0.f, 0.f, 0.f, 0.f);

  // level 2 over the finished fibers [fdone, fdone + nt)
  auto level2 = [&](int nt) {
    const uint32_t e = fdone;
    const uint32_t bound = (kb2 + 1u + lane <= p.S) ? __ldg(p.fsptr + kb2 + 1u + lane) : 0xffffffffu;
    const uint32_t fm = (lane < nt) ? __ldg(p.fmid + e + lane) : 0u;
    const uint32_t qd = bound - e;
    uint32_t starts = __reduce_or_sync(kFull, qd < 32u ? (1u << qd) : 0u);
    starts &= (nt >= 32) ? kFull : ((1u << nt) - 1u);
    const uint32_t kp = kb2 + __popc(starts & ((2u << lane) - 1u));
    const bool end_is_start = __any_sync(kFull, qd == (uint32_t)nt);
    const uint32_t kb_next = kb2 + __popc(__ballot_sync(kFull, qd <= (uint32_t)nt));
#pragma unroll
    for (int it = lane; it < 32 * (RM / 4); it += 32) {
      const int tt = it / (RM / 4), c = (it % (RM / 4)) * 4;
      const uint32_t r = __shfl_sync(kFull, fm, tt);
      if (tt < nt) *reinterpret_cast<float4 *>(stage + tt * RM + c) = row4(UM, r, RM, c);
    }
    __syncwarp();
    const int rbase = ring_slot(e);
    auto arow = [&](int r) -> const float * {
      if constexpr (MIDA) return stage + r * RM;
      else return ring + ((rbase + r) & (kRing - 1)) * RS;
    };
    auto brow = [&](int r) -> const float * {
      if constexpr (MIDA) return ring + ((rbase + r) & (kRing - 1)) * RS;
      else return stage + r * RM;
    };
    uint32_t segs = starts | 1u;
    while (segs) {
      const int p0 = __ffs(segs) - 1;
      segs &= segs - 1u;
      const int p1 = segs ? (__ffs(segs) - 1) : nt;
      int qq = p0 + g;
      auto step = [&](int r) {
        float av[TA], bv[TB];
        lds<TA>(arow(r) + ra0, av);
        lds<TB>(brow(r) + rb0, bv);
#pragma unroll
        for (int a = 0; a < TA; ++a)
#pragma unroll
          for (int b = 0; b < TB; ++b) acc[a][b] = fmaf(av[a], bv[b], acc[a][b]);
      };
      for (; qq + NG < p1; qq += 2 * NG) {
        step(qq);
        step(qq + NG);
      }
      if (qq < p1) step(qq);
      const bool flush = (p1 < nt) || end_is_start || (e + (uint32_t)nt == f1);
      if (flush) {
#pragma unroll
        for (int o = G; o < 32; o <<= 1)
#pragma unroll
          for (int a = 0; a < TA; ++a)
#pragma unroll
            for (int b = 0; b < TB; ++b) acc[a][b] += __shfl_xor_sync(kFull, acc[a][b], o);
        const uint32_t kseg = __shfl_sync(kFull, kp, p0);
        if (g == 0) {
          float *dst = (slot >= 0) ? p.carry + (size_t)slot * p.P : p.Y + (size_t)__ldg(p.sid + kseg) * p.P;
#pragma unroll
          for (int a = 0; a < TA; ++a) {
            float *d = dst + (size_t)(ra0 + a) * RB + rb0;
#pragma unroll
            for (int b = 0; b < TB; b += 4)
              *reinterpret_cast<float4 *>(d + b) = make_float4(acc[a][b], acc[a][b + 1], acc[a][b + 2], acc[a][b + 3]);
          }
        }
#pragma unroll
        for (int a = 0; a < TA; ++a)
#pragma unroll
          for (int b = 0; b < TB; ++b) acc[a][b] = 0.f;
      }
    }
    __syncwarp();
    kb2 = kb_next;
    fdone += (uint32_t)nt;
  };

  // level 1: window loads one window ahead
  float xr[kWin / 32];
  uint32_t ir[kWin / 32];
#pragma unroll
  for (int jj = 0; jj < kWin / 32; ++jj) {
    const uint32_t pos = z0 + 32u * jj + lane;
    xr[jj] = (pos < z1) ? __ldg(p.val + pos) : 0.f;
    ir[jj] = (pos < z1) ? __ldg(p.isum + pos) : 0u;
  }
  for (uint32_t z = z0; z < z1; z += kWin) {
    const int nt = (int)min((uint32_t)kWin, z1 - z);
#pragma unroll
    for (int jj = 0; jj < kWin / 32; ++jj) xs[xsi(32 * jj + lane)] = make_uint2(__float_as_uint(xr[jj]), ir[jj]);
    uint64_t starts = start_bits64(p.fbits, z);
    starts &= (nt >= 64) ? ~0ull : ((1ull << nt) - 1ull);
    if (z != z0 && (starts & 1ull)) {  // the fiber carried in ended at z - 1
      if (pb == 0) ring4[ring_slot(fcur) * QL + q] = carry;
      ++fcur;
      carry = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    starts &= ~1ull;
#pragma unroll
    for (int jj = 0; jj < kWin / 32; ++jj) {  // next window
      const uint32_t pos = z + kWin + 32u * jj + lane;
      xr[jj] = (pos < z1) ? __ldg(p.val + pos) : 0.f;
      ir[jj] = (pos < z1) ? __ldg(p.isum + pos) : 0u;
    }
    __syncwarp();
    float xv[PB];
    float4 r[PB];
#pragma unroll
    for (int i = 0; i < PB; ++i) {
      const uint2 e2 = xs[xsi(P0 + i)];
      xv[i] = __uint_as_float(e2.x);
      r[i] = (P0 + i < nt) ? row4(US, e2.y, RS, 4 * q) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    auto fiber_of = [&](int s) { return fcur + (uint32_t)__popcll(starts & ((2ull << s) - 1ull)); };
    // local pass: lead piece, fibers inside the block, trail piece
    float4 a4 = make_float4(0.f, 0.f, 0.f, 0.f), lead = a4;
    bool seen = false;
#pragma unroll
    for (int i = 0; i < PB; ++i) {
      if ((starts >> (P0 + i)) & 1ull) {  // the fiber at P0 + i - 1 ends
        if (seen)
          ring4[ring_slot(fiber_of(P0 + i - 1)) * QL + q] = a4;
        else
          lead = a4;
        seen = true;
        a4 = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      a4.x = fmaf(xv[i], r[i].x, a4.x);
      a4.y = fmaf(xv[i], r[i].y, a4.y);
      a4.z = fmaf(xv[i], r[i].z, a4.z);
      a4.w = fmaf(xv[i], r[i].w, a4.w);
    }
    if (!seen) lead = a4;
    // block map: A -> (seen ? 0 : A) + (seen ? trail : lead); inclusive scan over blocks
    bool cz = seen;
    float4 cb = seen ? a4 : lead;
#pragma unroll
    for (int d = 1; d < PG; d <<= 1) {
      const bool ez = __shfl_up_sync(kFull, (int)cz, d * QL) != 0;
      float4 eb;
      eb.x = __shfl_up_sync(kFull, cb.x, d * QL);
      eb.y = __shfl_up_sync(kFull, cb.y, d * QL);
      eb.z = __shfl_up_sync(kFull, cb.z, d * QL);
      eb.w = __shfl_up_sync(kFull, cb.w, d * QL);
      if (pb >= d && !cz) {
        cz = ez;
        cb.x = eb.x + cb.x;
        cb.y = eb.y + cb.y;
        cb.z = eb.z + cb.z;
        cb.w = eb.w + cb.w;
      }
    }
    // open fiber entering this block = (composition of the blocks before it)(carry)
    const bool pz = __shfl_up_sync(kFull, (int)cz, QL) != 0;
    float4 pbv;
    pbv.x = __shfl_up_sync(kFull, cb.x, QL);
    pbv.y = __shfl_up_sync(kFull, cb.y, QL);
    pbv.z = __shfl_up_sync(kFull, cb.z, QL);
    pbv.w = __shfl_up_sync(kFull, cb.w, QL);
    float4 open = carry;
    if (pb > 0) {
      if (pz) {
        open = pbv;
      } else {
        open.x = carry.x + pbv.x;
        open.y = carry.y + pbv.y;
        open.z = carry.z + pbv.z;
        open.w = carry.w + pbv.w;
      }
    }
    if (seen) {  // the open fiber ends at this block's first start
      const uint64_t bm = ((PB >= 64) ? ~0ull : (((1ull << PB) - 1ull) << P0));
      const int s0 = __ffsll((long long)(starts & bm)) - 1;
      ring4[ring_slot(fiber_of(s0 - 1)) * QL + q] =
          make_float4(open.x + lead.x, open.y + lead.y, open.z + lead.z, open.w + lead.w);
    }
    // the fiber open at the end of the window: the last block's composition applied to carry
    const int last = PG - 1;
    const bool lz = __shfl_sync(kFull, (int)cz, last * QL + q) != 0;
    float4 fin;
    fin.x = __shfl_sync(kFull, cb.x, last * QL + q);
    fin.y = __shfl_sync(kFull, cb.y, last * QL + q);
    fin.z = __shfl_sync(kFull, cb.z, last * QL + q);
    fin.w = __shfl_sync(kFull, cb.w, last * QL + q);
    if (!lz) {
      fin.x = carry.x + fin.x;
      fin.y = carry.y + fin.y;
      fin.z = carry.z + fin.z;
      fin.w = carry.w + fin.w;
    }
    carry = fin;
    fcur += (uint32_t)__popcll(starts);
    const bool unit_end = (z + (uint32_t)nt == z1);
    if (unit_end) {  // the last fiber of the unit ends here
      if (pb == 0) ring4[ring_slot(fcur) * QL + q] = carry;
      ++fcur;
    }
    __syncwarp();
    while (fcur - fdone >= 32u) level2(32);
    if (unit_end && fcur > fdone) level2((int)(fcur - fdone));
  }
}

template <int RM, int RS, int TA, int TB, bool MIDA, typename FT, int kWin = kWinDefault, int MINB = 4>
static cudaError_t run_fiber(const FiberParams &p, cudaStream_t s) {
  const size_t smem = (size_t)kFibWarps * (2 * kWin * RS + 32 * RM + 2 * (kWin + 32)) * sizeof(float);
  auto kern = ttmc_fiber_kernel<RM, RS, TA, TB, MIDA, FT, kWin, MINB>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const unsigned blocks = (unsigned)((p.n_units + kFibWarps - 1) / kFibWarps);
  kern<<<blocks, kFibWarps * 32, smem, s>>>(p);
  ::tk::count_launch();
  return cudaGetLastError();
}

// Fused fiber form for order-3 shapes (middle rank RM, summed rank RS).
template <typename FT>
static bool dispatch_fiber(const FiberParams &p, int RM, int RS, bool mida, cudaStream_t s, cudaError_t *err) {
#define TK_FIB(RM_, RS_, TA_, TB_)                                                                        \
  if (RM == RM_ && RS == RS_) {                                                                           \
    *err = mida ? run_fiber<RM_, RS_, TA_, TB_, true, FT>(p, s) : run_fiber<RM_, RS_, TA_, TB_, false, FT>(p, s); \
    return true;                                                                                          \
  }
  TK_FIB(16, 16, 4, 4)
  TK_FIB(8, 8, 2, 4)
  TK_FIB(32, 32, 8, 4)
  TK_FIB(16, 8, 4, 4)
  TK_FIB(8, 16, 4, 4)
#undef TK_FIB
  return false;
}

__global__ void fill_iota_ones_kernel(uint32_t *iota, float *ones, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    iota[i] = (uint32_t)i;
    ones[i] = 1.0f;
  }
}

void fill_iota_ones(uint32_t *iota, float *ones, int64_t n, cudaStream_t s) {
  const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 65535));
  fill_iota_ones_kernel<<<blocks, 256, 0, s>>>(iota, ones, n);
  ::tk::count_launch();
}

// ============================================================================ tensor-core form
// The contribution of one slice is the small GEMM  Y_i (PL x RB) = A_i^T B_i  with
// A_i = [x_z a_z] and B_i = [b_z] over its nonzeros z (K = slice length).  PL = 16 k
// rows fit the m16n8 tiles of mma.sync exactly, so a warp runs the slice segments of its
// tile through m16n8k16 BF16 products with K = the segment's nonzeros (rows outside the
// segment masked to zero), FP32 accumulation: the BF16-factor form.  Accumulators stay in
// the MMA C fragments while a segment continues across tiles.
__device__ __forceinline__ uint32_t pack_bf16(float lo_k, float hi_k) {
  uint32_t r;  // lower 16 bits hold the element with the lower k index
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi_k), "f"(lo_k));
  return r;
}
__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// BF16-factor form with ldmatrix fragments.  Staging (lane = nonzero of the tile): the
// left Kronecker row times x_z is formed in FP32 from the BF16 factor rows and rounded to
// BF16; the last-mode row is copied as is.  Both are stored k-major ([nonzero][rank],
// 48-byte or 16-byte-multiple padded rows), so that ldmatrix .trans hands each lane its
// m16n8k16 A and B fragments directly; nonzeros outside the current slice segment are
// masked in the A fragment (BF16 halves zeroed).  Slice offsets, indices and values of
// tile t+1 are prefetched into registers while tile t is processed.
__device__ __forceinline__ void ldsm_x4_trans(uint32_t (&r)[4], const void *row_addr) {
  const uint32_t sa = (uint32_t)__cvta_generic_to_shared(row_addr);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(sa));
}
__device__ __forceinline__ void ldsm_x2_trans(uint32_t &r0, uint32_t &r1, const void *row_addr) {
  const uint32_t sa = (uint32_t)__cvta_generic_to_shared(row_addr);
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n" : "=r"(r0), "=r"(r1) : "r"(sa));
}
__host__ __device__ constexpr int bf16_stride(int v) {  // row stride (elements): 16-byte rows, 16 (mod 64) bytes
  return ((v * 2 + 15) / 16 * 16 % 128 == 16 || (v * 2 + 15) / 16 * 16 % 128 == 48 ||
          (v * 2 + 15) / 16 * 16 % 128 == 80 || (v * 2 + 15) / 16 * 16 % 128 == 112)
             ? (v * 2 + 15) / 16 * 8
             : (v * 2 + 15) / 16 * 8 + 8;
}

template <int NL, int PL, int RB>
__global__ void __launch_bounds__(kTtmcWarps * 32) ttmc_bf16_kernel(const TtmcParams p) {
  static_assert(PL % 16 == 0 && RB % 8 == 0, "mma tiles");
  constexpr int MT = PL / 16, NT = RB / 8;
  constexpr int SA = bf16_stride(PL), SB = bf16_stride(RB);  // in BF16 elements
  constexpr int ROWS = 48;                                   // 32 nonzeros + a 16-row zero tail
  extern __shared__ float4 smem_f4[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __nv_bfloat16 *As = reinterpret_cast<__nv_bfloat16 *>(smem_f4) + (size_t)w * ROWS * (SA + SB);
  __nv_bfloat16 *Bs = As + ROWS * SA;
  const int64_t u = (int64_t)blockIdx.x * kTtmcWarps + w;
  if (u >= p.n_units) return;
  const __nv_bfloat16 *UA0 = static_cast<const __nv_bfloat16 *>(p.U[0]);
  const __nv_bfloat16 *UA1 = static_cast<const __nv_bfloat16 *>(p.U[1]);
  const __nv_bfloat16 *UB = static_cast<const __nv_bfloat16 *>(p.U[NL]);
  const uint32_t e0 = __ldg(p.unit_e0 + u);
  const uint32_t e_end = (u + 1 < p.n_units) ? __ldg(p.unit_e0 + u + 1) : p.Z;
  const int slot = __ldg(p.unit_slot + u);
  const int ntiles = (int)((e_end - e0 + 31u) / 32u);
  const int g = lane >> 2, t4 = lane & 3;
  for (int q = lane; q < 16 * SA; q += 32) As[32 * SA + q] = __float2bfloat16(0.f);
  for (int q = lane; q < 16 * SB; q += 32) Bs[32 * SB + q] = __float2bfloat16(0.f);
  float acc[MT][NT][4];
#pragma unroll
  for (int i = 0; i < MT; ++i)
#pragma unroll
    for (int jn = 0; jn < NT; ++jn)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][jn][q] = 0.f;

  uint32_t kb = __ldg(p.unit_k0 + u);
  uint32_t bound = (kb + 1u + lane <= p.S) ? __ldg(p.sptr + kb + 1u + lane) : 0xffffffffu;
  float x = 0.f;
  uint32_t i0 = 0u, i1 = 0u, ib = 0u;
  if (e0 + lane < e_end) {
    x = __ldg(p.val + e0 + lane);
    i0 = __ldg(p.idx[0] + e0 + lane);
    if constexpr (NL == 2) i1 = __ldg(p.idx[1] + e0 + lane);
    ib = __ldg(p.idx[NL] + e0 + lane);
  }
  for (int t = 0; t < ntiles; ++t) {
    const uint32_t e = e0 + 32u * (uint32_t)t;
    const int nt = (int)min(32u, e_end - e);
    const uint32_t q = bound - e;
    uint32_t starts = __reduce_or_sync(kFull, q < 32u ? (1u << q) : 0u);
    starts &= (nt >= 32) ? kFull : ((1u << nt) - 1u);
    const uint32_t kp = kb + __popc(starts & ((2u << lane) - 1u));
    const bool end_is_start = __any_sync(kFull, q == (uint32_t)nt);
    const uint32_t kb_next = kb + __popc(__ballot_sync(kFull, q <= (uint32_t)nt));
    const uint32_t bound_next = (kb_next + 1u + lane <= p.S) ? __ldg(p.sptr + kb_next + 1u + lane) : 0xffffffffu;
    float xn = 0.f;
    uint32_t i0n = 0u, i1n = 0u, ibn = 0u;
    const uint32_t posn = e + 32u + (uint32_t)lane;
    if (posn < e_end) {
      xn = __ldg(p.val + posn);
      i0n = __ldg(p.idx[0] + posn);
      if constexpr (NL == 2) i1n = __ldg(p.idx[1] + posn);
      ibn = __ldg(p.idx[NL] + posn);
    }
    // ---- staging.  16-byte pieces: consecutive lanes take consecutive pieces of one row,
    // so a row's pieces share one L1 request.
    {
      if constexpr (NL == 1) {
        constexpr int PA = PL / 8;  // pieces per row
#pragma unroll
        for (int it = lane; it < 32 * PA; it += 32) {
          const int tt = it / PA, c = it % PA;
          const float xt = __shfl_sync(kFull, x, tt);
          const uint32_t r = __shfl_sync(kFull, i0, tt);
          uint4 v = __ldg(reinterpret_cast<const uint4 *>(UA0 + (size_t)r * PL) + c);
          __nv_bfloat162 *h = reinterpret_cast<__nv_bfloat162 *>(&v);
#pragma unroll
          for (int qq = 0; qq < 4; ++qq) {
            const float2 f = __bfloat1622float2(h[qq]);
            h[qq] = __floats2bfloat162_rn(f.x * xt, f.y * xt);
          }
          *reinterpret_cast<uint4 *>(As + tt * SA + 8 * c) = v;
        }
      } else {
        __nv_bfloat16 *arow = As + lane * SA;
        const int R0 = p.R[0], R1 = p.R[1];
        const __nv_bfloat16 *ra = UA0 + (size_t)i0 * R0;
        const __nv_bfloat16 *rb = UA1 + (size_t)i1 * R1;
        for (int a0 = 0; a0 < R0; ++a0) {
          const float s0 = x * __bfloat162float(ra[a0]);
          for (int a1 = 0; a1 < R1; a1 += 2) {
            const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(rb + a1));
            *reinterpret_cast<__nv_bfloat162 *>(arow + a0 * R1 + a1) = __floats2bfloat162_rn(s0 * f.x, s0 * f.y);
          }
        }
      }
      constexpr int PB = RB / 8;
#pragma unroll
      for (int it = lane; it < 32 * PB; it += 32) {
        const int tt = it / PB, c = it % PB;
        const uint32_t r = __shfl_sync(kFull, ib, tt);
        *reinterpret_cast<uint4 *>(Bs + tt * SB + 8 * c) = __ldg(reinterpret_cast<const uint4 *>(UB + (size_t)r * RB) + c);
      }
    }
    __syncwarp();
    uint32_t segs = starts | 1u;
    while (segs) {
      const int p0 = __ffs(segs) - 1;
      segs &= segs - 1u;
      const int p1 = segs ? (__ffs(segs) - 1) : nt;
      for (int ks = p0; ks < p1; ks += 16) {
        // masks of the BF16 halves by nonzero index: k = ks + 2 t4 (+1), ks + 8 + 2 t4 (+1)
        const int k0 = ks + 2 * t4, k8 = k0 + 8;
        const uint32_t m0 = (k0 < p1 ? 0x0000ffffu : 0u) | (k0 + 1 < p1 ? 0xffff0000u : 0u);
        const uint32_t m8 = (k8 < p1 ? 0x0000ffffu : 0u) | (k8 + 1 < p1 ? 0xffff0000u : 0u);
        const int mrow = lane & 7, msel = lane >> 3;  // ldmatrix: lanes 8j..8j+7 address matrix j
        uint32_t bfr[NT][2];
#pragma unroll
        for (int nq = 0; nq < NT; nq += 2) {
          if (nq + 1 < NT) {
            // matrices: (k 0-7, n nq*8), (k 8-15, n nq*8), (k 0-7, n nq*8+8), (k 8-15, n nq*8+8)
            const int kr = ks + mrow + ((msel & 1) ? 8 : 0);
            const int nc = nq * 8 + ((msel & 2) ? 8 : 0);
            uint32_t r[4];
            ldsm_x4_trans(r, Bs + kr * SB + nc);
            bfr[nq][0] = r[0];
            bfr[nq][1] = r[1];
            bfr[nq + 1][0] = r[2];
            bfr[nq + 1][1] = r[3];
          } else {
            const int kr = ks + mrow + ((msel & 1) ? 8 : 0);
            ldsm_x2_trans(bfr[nq][0], bfr[nq][1], Bs + kr * SB + nq * 8);
          }
        }
#pragma unroll
        for (int mt = 0; mt < MT; ++mt) {
          // matrices: (k 0-7, m), (k 0-7, m+8), (k 8-15, m), (k 8-15, m+8) -> a0 a1 a2 a3
          const int kr = ks + mrow + ((msel & 2) ? 8 : 0);
          const int mc = mt * 16 + ((msel & 1) ? 8 : 0);
          uint32_t a[4];
          ldsm_x4_trans(a, As + kr * SA + mc);
          a[0] &= m0;
          a[1] &= m0;
          a[2] &= m8;
          a[3] &= m8;
#pragma unroll
          for (int nq = 0; nq < NT; ++nq) mma_bf16(acc[mt][nq], a, bfr[nq][0], bfr[nq][1]);
        }
      }
      const bool flush = (p1 < nt) || end_is_start || (e + (uint32_t)nt == e_end);
      if (flush) {
        const uint32_t kseg = __shfl_sync(kFull, kp, p0);
        float *dst = (slot >= 0) ? p.carry + (size_t)slot * p.P : p.Y + (size_t)__ldg(p.sid + kseg) * p.P;
#pragma unroll
        for (int mt = 0; mt < MT; ++mt)
#pragma unroll
          for (int nq = 0; nq < NT; ++nq) {
            const int row = mt * 16 + g, col = nq * 8 + 2 * t4;
            *reinterpret_cast<float2 *>(dst + (size_t)row * RB + col) = make_float2(acc[mt][nq][0], acc[mt][nq][1]);
            *reinterpret_cast<float2 *>(dst + (size_t)(row + 8) * RB + col) =
                make_float2(acc[mt][nq][2], acc[mt][nq][3]);
            acc[mt][nq][0] = acc[mt][nq][1] = acc[mt][nq][2] = acc[mt][nq][3] = 0.f;
          }
      }
    }
    __syncwarp();
    kb = kb_next;
    bound = bound_next;
    x = xn;
    i0 = i0n;
    i1 = i1n;
    ib = ibn;
  }
}

// ============================================================================ TMA-fed BF16 form
// The arithmetic of ttmc_bf16_kernel (order 3, ranks 16 x 16) with the factor rows brought
// into shared memory by the tensor memory accelerator instead of by the warp's own loads:
// each warp keeps a ring of kTmaStages tiles (32 nonzeros each); for every tile, sixteen
// lanes issue one cp.async.bulk.tensor gather4 each (four rows of U_a or U_b of 32 bytes),
// completing on the stage's mbarrier.  The rows of tile t + kTmaStages are requested as
// soon as tile t has been consumed, so a warp has up to kTmaStages tiles of gathers in
// flight and holds none of them in registers.  The value x_z is applied to the A
// fragments after ldmatrix, in FP32 and rounded to BF16 as the staging of ttmc_bf16_kernel
// does, so both kernels give the same Y bit for bit.  Every wait is bounded; a warp whose
// wait gives up records kErrTimeout, waits (bounded) for its copies in flight and leaves.
constexpr int kTmaWarps = 4;
constexpr int kTmaStages = 4;
constexpr int kTmaRows = 48;                       // 32 rows per tile + 16 zero rows read past the tile
constexpr unsigned long long kTmaSpin = 1ull << 22;  // polls of an mbarrier before a wait gives up

__device__ __forceinline__ void mbar_init(uint32_t bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, unsigned parity) {
  uint32_t done;
  asm volatile(
      "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}
// bounded wait for the phase with the given parity; false when it gave up
__device__ __forceinline__ bool mbar_wait(uint32_t bar, unsigned parity) {
  for (unsigned long long i = 0; i < kTmaSpin; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if (i > 64) __nanosleep(32);
  }
  return false;
}
// four rows r0..r3 of a row-major factor (one box = one row) to dst (4 x row bytes)
__device__ __forceinline__ void tma_gather4(uint32_t dst, const CUtensorMap *tm, uint32_t r0, uint32_t r1,
                                            uint32_t r2, uint32_t r3, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cta.global.tile::gather4.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
      "%4, %5, %6}], [%7];" ::"r"(dst),
      "l"(tm), "r"(0), "r"(r0), "r"(r1), "r"(r2), "r"(r3), "r"(bar)
      : "memory");
}

template <int PL, int RB>
__global__ void __launch_bounds__(kTmaWarps * 32) ttmc_bf16_tma_kernel(const TtmcParams p,
                                                                       const __grid_constant__ CUtensorMap tmA,
                                                                       const __grid_constant__ CUtensorMap tmB) {
  static_assert(PL == 16 && RB == 16, "one gather4 box per 32-byte row");
  constexpr int MT = PL / 16, NT = RB / 8;
  constexpr int STAGE = kTmaRows * (PL + RB);  // BF16 elements per stage
  constexpr unsigned TX = 32u * (PL + RB) * 2u;  // bytes a stage receives
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __nv_bfloat16 *ring = reinterpret_cast<__nv_bfloat16 *>(smem_raw) + (size_t)w * kTmaStages * STAGE;
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem_raw + (size_t)kTmaWarps * kTmaStages * STAGE * 2) + w * kTmaStages;
  const int64_t u = (int64_t)blockIdx.x * kTmaWarps + w;
  if (u >= p.n_units) return;
  const uint32_t e0 = __ldg(p.unit_e0 + u);
  const uint32_t e_end = (u + 1 < p.n_units) ? __ldg(p.unit_e0 + u + 1) : p.Z;
  const int slot = __ldg(p.unit_slot + u);
  const int ntiles = (int)((e_end - e0 + 31u) / 32u);
  const int g = lane >> 2, t4 = lane & 3;
  auto As = [&](int st) { return ring + st * STAGE; };
  auto Bs = [&](int st) { return ring + st * STAGE + kTmaRows * PL; };
  auto bar = [&](int st) { return (uint32_t)__cvta_generic_to_shared(bars + st); };
  // zero tails (never written by the copies), barriers
  for (int st = 0; st < kTmaStages; ++st) {
    for (int q = lane; q < 16 * PL; q += 32) As(st)[32 * PL + q] = __float2bfloat16(0.f);
    for (int q = lane; q < 16 * RB; q += 32) Bs(st)[32 * RB + q] = __float2bfloat16(0.f);
  }
  if (lane == 0)
    for (int st = 0; st < kTmaStages; ++st) mbar_init(bar(st), 1u);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncwarp();

  // requests the rows of tile tt into stage st (indices of its positions, lane = position)
  auto issue = [&](int tt, uint32_t ia, uint32_t ib) {
    const int st = tt % kTmaStages;
    if (lane == 0) mbar_expect_tx(bar(st), TX);
    __syncwarp();
    const int q = lane & 7;  // lanes q and 8 + q request rows 4q .. 4q + 3 of U_a and U_b
    const uint32_t a0 = __shfl_sync(kFull, ia, 4 * q), a1 = __shfl_sync(kFull, ia, 4 * q + 1);
    const uint32_t a2 = __shfl_sync(kFull, ia, 4 * q + 2), a3 = __shfl_sync(kFull, ia, 4 * q + 3);
    const uint32_t b0 = __shfl_sync(kFull, ib, 4 * q), b1 = __shfl_sync(kFull, ib, 4 * q + 1);
    const uint32_t b2 = __shfl_sync(kFull, ib, 4 * q + 2), b3 = __shfl_sync(kFull, ib, 4 * q + 3);
    if (lane < 8) {
      tma_gather4((uint32_t)__cvta_generic_to_shared(As(st) + 4 * q * PL), &tmA, a0, a1, a2, a3, bar(st));
    } else if (lane < 16) {
      tma_gather4((uint32_t)__cvta_generic_to_shared(Bs(st) + 4 * q * RB), &tmB, b0, b1, b2, b3, bar(st));
    }
  };
  // indices of tile tt (positions past the unit read row 0, a valid row, and are masked)
  auto tile_idx = [&](int tt, uint32_t &ia, uint32_t &ib) {
    const uint32_t pos = e0 + 32u * (uint32_t)tt + (uint32_t)lane;
    ia = (pos < e_end) ? __ldg(p.idx[0] + pos) : 0u;
    ib = (pos < e_end) ? __ldg(p.idx[1] + pos) : 0u;
  };
  const int pro = ntiles < kTmaStages ? ntiles : kTmaStages;
  for (int tt = 0; tt < pro; ++tt) {
    uint32_t ia, ib;
    tile_idx(tt, ia, ib);
    issue(tt, ia, ib);
  }

  float acc[MT][NT][4];
#pragma unroll
  for (int i = 0; i < MT; ++i)
#pragma unroll
    for (int jn = 0; jn < NT; ++jn)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][jn][q] = 0.f;
  uint32_t kb = __ldg(p.unit_k0 + u);
  uint32_t bound = (kb + 1u + lane <= p.S) ? __ldg(p.sptr + kb + 1u + lane) : 0xffffffffu;
  float x = (e0 + lane < e_end) ? __ldg(p.val + e0 + lane) : 0.f;
  int failed_at = -1;
  for (int t = 0; t < ntiles; ++t) {
    const int st = t % kTmaStages;
    const uint32_t e = e0 + 32u * (uint32_t)t;
    const int nt = (int)min(32u, e_end - e);
    const uint32_t q = bound - e;
    uint32_t starts = __reduce_or_sync(kFull, q < 32u ? (1u << q) : 0u);
    starts &= (nt >= 32) ? kFull : ((1u << nt) - 1u);
    const uint32_t kp = kb + __popc(starts & ((2u << lane) - 1u));
    const bool end_is_start = __any_sync(kFull, q == (uint32_t)nt);
    const uint32_t kb_next = kb + __popc(__ballot_sync(kFull, q <= (uint32_t)nt));
    // loads of the next tile's slice offsets and values, and of the indices of the tile
    // whose rows are requested after this one is consumed
    const uint32_t bound_next = (kb_next + 1u + lane <= p.S) ? __ldg(p.sptr + kb_next + 1u + lane) : 0xffffffffu;
    const uint32_t posn = e + 32u + (uint32_t)lane;
    const float xn = (posn < e_end) ? __ldg(p.val + posn) : 0.f;
    uint32_t ia_f = 0u, ib_f = 0u;
    if (t + kTmaStages < ntiles) tile_idx(t + kTmaStages, ia_f, ib_f);
    if (!__all_sync(kFull, mbar_wait(bar(st), (unsigned)((t / kTmaStages) & 1)))) {
      failed_at = t;
      break;
    }
    const __nv_bfloat16 *A = As(st), *B = Bs(st);
    uint32_t segs = starts | 1u;
    while (segs) {
      const int p0 = __ffs(segs) - 1;
      segs &= segs - 1u;
      const int p1 = segs ? (__ffs(segs) - 1) : nt;
      for (int ks = p0; ks < p1; ks += 16) {
        const int k0 = ks + 2 * t4, k8 = k0 + 8;
        const float x0 = __shfl_sync(kFull, x, k0 & 31), x1 = __shfl_sync(kFull, x, (k0 + 1) & 31);
        const float x8 = __shfl_sync(kFull, x, k8 & 31), x9 = __shfl_sync(kFull, x, (k8 + 1) & 31);
        const uint32_t m0 = (k0 < p1 ? 0x0000ffffu : 0u) | (k0 + 1 < p1 ? 0xffff0000u : 0u);
        const uint32_t m8 = (k8 < p1 ? 0x0000ffffu : 0u) | (k8 + 1 < p1 ? 0xffff0000u : 0u);
        const int mrow = lane & 7, msel = lane >> 3;
        uint32_t bfr[NT][2];
#pragma unroll
        for (int nq = 0; nq < NT; nq += 2) {
          const int kr = ks + mrow + ((msel & 1) ? 8 : 0);
          const int nc = nq * 8 + ((msel & 2) ? 8 : 0);
          uint32_t r[4];
          ldsm_x4_trans(r, B + kr * RB + nc);
          bfr[nq][0] = r[0];
          bfr[nq][1] = r[1];
          bfr[nq + 1][0] = r[2];
          bfr[nq + 1][1] = r[3];
        }
#pragma unroll
        for (int mt = 0; mt < MT; ++mt) {
          const int kr = ks + mrow + ((msel & 2) ? 8 : 0);
          const int mc = mt * 16 + ((msel & 1) ? 8 : 0);
          uint32_t a[4];
          ldsm_x4_trans(a, A + kr * PL + mc);
          // x_z on the A fragments: a0, a1 hold nonzeros k0, k0 + 1; a2, a3 hold k8, k8 + 1
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&a[r]));
            const float lo = (r < 2) ? x0 : x8, hi = (r < 2) ? x1 : x9;
            const __nv_bfloat162 h = __floats2bfloat162_rn(f.x * lo, f.y * hi);
            a[r] = *reinterpret_cast<const uint32_t *>(&h);
          }
          a[0] &= m0;
          a[1] &= m0;
          a[2] &= m8;
          a[3] &= m8;
#pragma unroll
          for (int nq = 0; nq < NT; ++nq) mma_bf16(acc[mt][nq], a, bfr[nq][0], bfr[nq][1]);
        }
      }
      const bool flush = (p1 < nt) || end_is_start || (e + (uint32_t)nt == e_end);
      if (flush) {
        const uint32_t kseg = __shfl_sync(kFull, kp, p0);
        float *dst = (slot >= 0) ? p.carry + (size_t)slot * p.P : p.Y + (size_t)__ldg(p.sid + kseg) * p.P;
#pragma unroll
        for (int mt = 0; mt < MT; ++mt)
#pragma unroll
          for (int nq = 0; nq < NT; ++nq) {
            const int row = mt * 16 + g, col = nq * 8 + 2 * t4;
            *reinterpret_cast<float2 *>(dst + (size_t)row * RB + col) = make_float2(acc[mt][nq][0], acc[mt][nq][1]);
            *reinterpret_cast<float2 *>(dst + (size_t)(row + 8) * RB + col) =
                make_float2(acc[mt][nq][2], acc[mt][nq][3]);
            acc[mt][nq][0] = acc[mt][nq][1] = acc[mt][nq][2] = acc[mt][nq][3] = 0.f;
          }
      }
    }
    __syncwarp();  // every lane has read stage st
    if (t + kTmaStages < ntiles) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(t + kTmaStages, ia_f, ib_f);
    }
    kb = kb_next;
    bound = bound_next;
    x = xn;
  }
  if (failed_at >= 0) {  // record, then let the copies still in flight land before the warp leaves
    if (lane == 0) atomicOr(p.err, kErrTimeout);
    // tiles failed_at .. failed_at + S - 1 (below ntiles) were requested and not consumed:
    // one outstanding phase per stage
    for (int tt = failed_at; tt < failed_at + kTmaStages && tt < ntiles; ++tt)
      mbar_wait(bar(tt % kTmaStages), (unsigned)((tt / kTmaStages) & 1));
  }
}

// Any shape: each lane owns CPL columns of a block of 32*CPL columns (grid.y), and
// forms its Kronecker entries directly from the factor rows (cached loads).
template <int CPL, typename FT>
__global__ void __launch_bounds__(kTtmcWarps * 32) ttmc_generic_kernel(const TtmcParams p) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t u = (int64_t)blockIdx.x * kTtmcWarps + w;
  if (u >= p.n_units) return;
  const int nother = p.nother;
  // column decode
  int rr[CPL][kMaxOrder];
  bool own[CPL];
  int64_t col[CPL];
#pragma unroll
  for (int s = 0; s < CPL; ++s) {
    col[s] = (int64_t)blockIdx.y * 32 * CPL + lane + 32 * s;
    own[s] = col[s] < p.P;
    int64_t cc = own[s] ? col[s] : 0;
    for (int t = kMaxOrder - 1; t >= 0; --t) {
      if (t < nother) {
        rr[s][t] = (int)(cc % p.R[t]);
        cc /= p.R[t];
      } else {
        rr[s][t] = 0;
      }
    }
  }
  uint32_t e = __ldg(p.unit_e0 + u);
  const uint32_t e_end = (u + 1 < p.n_units) ? __ldg(p.unit_e0 + u + 1) : p.Z;
  uint32_t kb = __ldg(p.unit_k0 + u);
  const int slot = __ldg(p.unit_slot + u);
  float acc[CPL];
#pragma unroll
  for (int s = 0; s < CPL; ++s) acc[s] = 0.f;
  while (e < e_end) {
    const int nt = (int)min(32u, e_end - e);
    const TileSlices ts = tile_slices(p.sptr, p.S, kb, e, nt, lane);
    float x = 0.f;
    uint32_t id[kMaxOrder];
#pragma unroll
    for (int t = 0; t < kMaxOrder; ++t) id[t] = 0;
    if (lane < nt) {
      x = __ldg(p.val + e + lane);
      for (int t = 0; t < nother; ++t) id[t] = __ldg(p.idx[t] + e + lane);
    }
    uint32_t segs = ts.starts | 1u;
    while (segs) {
      const int p0 = __ffs(segs) - 1;
      segs &= segs - 1u;
      const int p1 = segs ? (__ffs(segs) - 1) : nt;
      for (int q = p0; q < p1; ++q) {
        const float xq = __shfl_sync(kFull, x, q);
        uint32_t iq[kMaxOrder];
#pragma unroll
        for (int t = 0; t < kMaxOrder; ++t) iq[t] = __shfl_sync(kFull, id[t], q);
#pragma unroll
        for (int s = 0; s < CPL; ++s) {
          float v = xq;
          for (int t = 0; t < nother; ++t)
            v *= Ld<FT>::s(static_cast<const FT *>(p.U[t]) + (size_t)iq[t] * p.R[t], rr[s][t]);
          acc[s] += v;
        }
      }
      const bool flush = (p1 < nt) || ts.end_is_start || (e + (uint32_t)nt == e_end);
      if (flush) {
        const uint32_t kseg = __shfl_sync(kFull, ts.kp, p0);
        float *dst = (slot >= 0) ? p.carry + (size_t)slot * p.P : p.Y + (size_t)__ldg(p.sid + kseg) * p.P;
#pragma unroll
        for (int s = 0; s < CPL; ++s) {
          if (own[s]) dst[col[s]] = acc[s];
          acc[s] = 0.f;
        }
      }
    }
    kb = ts.kb_next;
    e += (uint32_t)nt;
  }
}

// Rows of slices split over several units: block (l, c) sums the partial rows of long
// slice l for columns [32c, 32c + 32).  Warp w adds the pieces w, w + 8, ... (four loads in
// flight), then the eight warp sums are added in warp order: a fixed order, so Y is
// reproducible, and a slice cut into thousands of pieces is summed by many blocks.  With
// `sq` given, the exact square of each finished entry goes to sq[l * P + c] as a pair.
constexpr int kFixWarps = 8;
__global__ void __launch_bounds__(kFixWarps * 32) ttmc_fixup_kernel(const uint32_t *long_k, const uint32_t *long_u0,
                                                                     const uint32_t *long_np, const uint32_t *sid,
                                                                     const float *carry, float *Y, int64_t P,
                                                                     float2 *sq) {
  __shared__ float part[kFixWarps][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t l = blockIdx.x, c = (int64_t)blockIdx.y * 32 + lane;
  const uint32_t row = __ldg(sid + __ldg(long_k + l)), u0 = __ldg(long_u0 + l), np = __ldg(long_np + l);
  float s = 0.f;
  if (c < P) {
    const float *base = carry + (size_t)u0 * P + c;
    uint32_t q = (uint32_t)warp;
    for (; q + 3u * kFixWarps < np; q += 4u * kFixWarps) {
      float v[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) v[k] = __ldcg(base + (size_t)(q + k * kFixWarps) * P);
#pragma unroll
      for (int k = 0; k < 4; ++k) s += v[k];
    }
    for (; q < np; q += kFixWarps) s += __ldcg(base + (size_t)q * P);
  }
  part[warp][lane] = s;
  __syncthreads();
  if (warp == 0 && c < P) {
    float t = part[0][lane];
#pragma unroll
    for (int k = 1; k < kFixWarps; ++k) t += part[k][lane];
    Y[(size_t)row * P + c] = t;
    if (sq) {
      const float t2 = t * t;
      sq[(size_t)l * P + c] = make_float2(t2, fmaf(t, t, -t2));
    }
  }
}

static void launch_fixup(const uint32_t *long_k, const uint32_t *long_u0, const uint32_t *long_np, int64_t n_long,
                         const uint32_t *sid, const float *carry, float *Y, int64_t P, cudaStream_t s,
                         float2 *sq = nullptr) {
  const dim3 grid((unsigned)n_long, (unsigned)((P + 31) / 32));
  ttmc_fixup_kernel<<<grid, kFixWarps * 32, 0, s>>>(long_k, long_u0, long_np, sid, carry, Y, P, sq);
  ::tk::count_launch();
}

// Column sums of squares of Y_(n) from the pairs of the pipelined TTMc and the fixup
// (`rows` rows of P pairs), in two levels within one launch.  Block (g, h) adds rows
// [64h, 64h + 64) of columns [32g, 32g + 32): warp w the rows 64h + w, 64h + w + 8, ...
// (all eight loads in flight), then the warp sums in warp order, to chunk[h].  The last
// block of column group g to finish (a counter, which that block resets) adds the chunks
// in order and the warps' sums in FP64.  A fixed order: the norms are reproducible.
constexpr int kSqRows = 64, kSqW = 8;
__global__ void __launch_bounds__(kSqW * 32) ttmc_colsq_kernel(const float2 *part, int64_t rows, int64_t P,
                                                               float2 *chunk, unsigned *cnt, double *colsq) {
  __shared__ float2 ws[kSqW][32];
  __shared__ int last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t c = (int64_t)blockIdx.x * 32 + lane;
  const int64_t r0 = (int64_t)blockIdx.y * kSqRows + warp;
  DF t;
  if (c < P) {
    float2 v[kSqRows / kSqW];
#pragma unroll
    for (int u = 0; u < kSqRows / kSqW; ++u) {
      const int64_t r = r0 + u * kSqW;
      v[u] = r < rows ? __ldcg(part + (size_t)r * P + c) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < kSqRows / kSqW; ++u) sq_add(t, v[u]);
  }
  ws[warp][lane] = make_float2(t.hi, t.lo);
  __syncthreads();
  if (warp == 0) {
    DF b;
    for (int w = 0; w < kSqW; ++w) sq_add(b, ws[w][lane]);
    if (c < P) chunk[(size_t)blockIdx.y * P + c] = make_float2(b.hi, b.lo);
    __threadfence();  // the chunk is visible before the counter says so
  }
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(cnt + blockIdx.x, 1u) == gridDim.y - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  const int nch = (int)gridDim.y;
  DF f;
  if (c < P) {
    int h = warp;
    for (; h + 3 * kSqW < nch; h += 4 * kSqW) {
      float2 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = __ldcg(chunk + (size_t)(h + u * kSqW) * P + c);
#pragma unroll
      for (int u = 0; u < 4; ++u) sq_add(f, v[u]);
    }
    for (; h < nch; h += kSqW) sq_add(f, __ldcg(chunk + (size_t)h * P + c));
  }
  ws[warp][lane] = make_float2(f.hi, f.lo);
  __syncthreads();
  if (warp == 0 && c < P) {
    double v = 0.0;
    for (int w = 0; w < kSqW; ++w) v += (double)ws[w][lane].x + (double)ws[w][lane].y;
    colsq[c] = v;
  }
  if (threadIdx.x == 0) cnt[blockIdx.x] = 0u;  // ready for the next launch
}

// rows of pairs in `part`, then the chunk sums after them (sq_elems covers both)
static int64_t colsq_chunks(int64_t rows) { return (rows + kSqRows - 1) / kSqRows; }

static void launch_colsq(float2 *part, int64_t rows, int64_t P, unsigned *cnt, double *colsq, cudaStream_t s) {
  const dim3 grid((unsigned)((P + 31) / 32), (unsigned)colsq_chunks(rows));
  ttmc_colsq_kernel<<<grid, kSqW * 32, 0, s>>>(part, rows, P, part + (size_t)rows * P, cnt, colsq);
  ::tk::count_launch();
}

__global__ void ttmc_zero_rows_kernel(const uint32_t *rows, int64_t n, float *Y, int64_t P) {
  for (int64_t r = blockIdx.x; r < n; r += gridDim.x) {
    float *y = Y + (size_t)rows[r] * P;
    for (int64_t c = threadIdx.x; c < P; c += blockDim.x) y[c] = 0.f;
  }
}

template <int NL, int PL, int RB, int TA, int TB, typename FT>
static cudaError_t run_fast(const TtmcParams &p, cudaStream_t s) {
  const size_t smem = (size_t)kTtmcWarps * 32 * (PL + RB) * sizeof(float);
  auto kern = ttmc_fast_kernel<NL, PL, RB, TA, TB, FT>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const unsigned blocks = (unsigned)((p.n_units + kTtmcWarps - 1) / kTtmcWarps);
  kern<<<blocks, kTtmcWarps * 32, smem, s>>>(p);
  ::tk::count_launch();
  return cudaGetLastError();
}

template <int NL, int PL, int RB>
static cudaError_t run_bf16(const TtmcParams &p, cudaStream_t s) {
  const size_t smem = (size_t)kTtmcWarps * 48 * (bf16_stride(PL) + bf16_stride(RB)) * sizeof(__nv_bfloat16);
  auto kern = ttmc_bf16_kernel<NL, PL, RB>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const unsigned blocks = (unsigned)((p.n_units + kTtmcWarps - 1) / kTtmcWarps);
  kern<<<blocks, kTtmcWarps * 32, smem, s>>>(p);
  ::tk::count_launch();
  return cudaGetLastError();
}

template <int PL, int RB>
static cudaError_t run_bf16_tma(const TtmcParams &p, const CUtensorMap &tmA, const CUtensorMap &tmB, cudaStream_t s) {
  const size_t smem = (size_t)kTmaWarps * kTmaStages * (kTmaRows * (PL + RB) * 2 + sizeof(uint64_t));
  auto kern = ttmc_bf16_tma_kernel<PL, RB>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const unsigned blocks = (unsigned)((p.n_units + kTmaWarps - 1) / kTmaWarps);
  kern<<<blocks, kTmaWarps * 32, smem, s>>>(p, tmA, tmB);
  ::tk::count_launch();
  return cudaGetLastError();
}

// TUCKER_TTMC_TMA=1 runs the BF16 form on ttmc_bf16_tma_kernel (rows gathered by the TMA).
// Same Y bit for bit, but slower on the 20M-nonzero skewed workload (0.59 / 0.92 / 0.90 ms
// against 0.34 / 0.24 / 0.29 ms per mode): a tile of 32 nonzeros needs 16 gather4 requests
// of 128 bytes, and the copy engine completes one such request per ~28 SM cycles, well
// below the rate at which the warps' own 16-byte loads bring the same rows.  Kept opt-in.
static bool tma_rows() {
  const char *e = std::getenv("TUCKER_TTMC_TMA");
  return e && e[0] == '1';
}

// BF16-factor dispatch (shapes with PL % 16 == 0 and RB % 8 == 0).
static bool dispatch_bf16(const TtmcParams &p, cudaStream_t s, cudaError_t *err) {
  const int no = p.nother;
  const int RB = p.R[no - 1];
#define TK_MMA(NL_, PL_, RB_)                \
  {                                          \
    *err = run_bf16<NL_, PL_, RB_>(p, s);    \
    return true;                             \
  }
  if (no == 2) {
    const int PL = p.R[0];
    if (PL == 16 && RB == 16) TK_MMA(1, 16, 16)
    if (PL == 16 && RB == 8) TK_MMA(1, 16, 8)
    if (PL == 32 && RB == 32) TK_MMA(1, 32, 32)
  } else if (no == 3 && p.R[1] % 4 == 0) {
    const int PL = p.R[0] * p.R[1];
    if (PL == 64 && RB == 8) TK_MMA(2, 64, 8)
    if (PL == 64 && RB == 16) TK_MMA(2, 64, 16)
  }
#undef TK_MMA
  return false;
}

template <int PL, int RB, int TA, int TB>
static cudaError_t run_pipe(const TtmcParams &p, cudaStream_t s) {
  // the norm-forming kernel (p.sq_part given) exists where the pairs stay small: P_n <= 256
  constexpr bool kSqShape = PL * RB <= 256;
  if (p.sq_part && !kSqShape) return cudaErrorInvalidValue;
  const size_t smem = (size_t)kTtmcWarps * 32 * (PL + RB) * sizeof(float);
  auto kern = ttmc_pipe_kernel<PL, RB, TA, TB>;
  if constexpr (kSqShape)
    if (p.sq_part) kern = ttmc_pipe_sq_kernel<PL, RB, TA, TB>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const unsigned blocks = (unsigned)ttmc_pipe_blocks(p.n_units);
  kern<<<blocks, kTtmcWarps * 32, smem, s>>>(p);
  ::tk::count_launch();
  return cudaGetLastError();
}

template <int RB>
static cudaError_t run_fibsum(const TtmcParams &p, float *T, int64_t nnz, cudaStream_t s) {
  // two rounds of side-by-side fibers per warp (16 fibers for RB = 16: measured best on the
  // skewed 20M-nonzero workload against 8, 24, 32, 64, 128; short warps balance the
  // Zipf-skewed fiber lengths)
  const int64_t F = std::max<int64_t>(p.Z, 1);
  (void)nnz;
  int64_t fpw = 2 * (32 / (RB / 4));
  if (const char *e = std::getenv("TUCKER_FIBSUM_FPW")) fpw = std::max<int64_t>(4, std::atoll(e) / 4 * 4);
  const int64_t warps = (F + fpw - 1) / fpw;
  const unsigned blocks = (unsigned)((warps + kTtmcWarps - 1) / kTtmcWarps);
  ttmc_fibsum_kernel<RB><<<blocks, kTtmcWarps * 32, 0, s>>>(p, T, fpw);
  ::tk::count_launch();
  return cudaGetLastError();
}

// Fiber sums for the shapes the update pass covers (order 3, RB in {8, 16, 32}).
static bool dispatch_fibsum(const TtmcParams &p, float *T, int64_t nnz, cudaStream_t s, cudaError_t *err) {
  if (p.nother != 2) return false;
  const int RB = p.R[1];
  if (RB == 16) *err = run_fibsum<16>(p, T, nnz, s);
  else if (RB == 8) *err = run_fibsum<8>(p, T, nnz, s);
  else if (RB == 32) *err = run_fibsum<32>(p, T, nnz, s);
  else return false;
  return true;
}

static bool dispatch_pipe(const TtmcParams &p, cudaStream_t s, cudaError_t *err);

int64_t ttmc_pipe_blocks(int64_t units) { return (units + kTtmcWarps - 1) / kTtmcWarps; }

// shapes (first rank, last rank) of the pipelined kernel below
static bool pipe_shape(int PL, int RB) {
  return (PL == 16 && RB == 16) || (PL == 8 && RB == 8) || (PL == 32 && RB == 32) || (PL == 16 && RB == 8) ||
         (PL == 8 && RB == 16);
}

// Pipelined FP32 dispatch (order 3, row-aligned factors).
static bool dispatch_pipe(const TtmcParams &p, cudaStream_t s, cudaError_t *err) {
  if (p.nother != 2) return false;
  const int PL = p.R[0], RB = p.R[1];
#define TK_PIPE(PL_, RB_, TA_, TB_)                   \
  {                                                   \
    *err = run_pipe<PL_, RB_, TA_, TB_>(p, s);        \
    return true;                                      \
  }
  if (PL == 16 && RB == 16) TK_PIPE(16, 16, 4, 4)
  if (PL == 8 && RB == 8) TK_PIPE(8, 8, 2, 4)
  if (PL == 32 && RB == 32) TK_PIPE(32, 32, 8, 4)
  if (PL == 16 && RB == 8) TK_PIPE(16, 8, 4, 4)
  if (PL == 8 && RB == 16) TK_PIPE(8, 16, 4, 4)
#undef TK_PIPE
  return false;
}

template <typename FT>
static cudaError_t run_generic(const TtmcParams &p, cudaStream_t s) {
  constexpr int CPL = 4;
  const unsigned blocks = (unsigned)((p.n_units + kTtmcWarps - 1) / kTtmcWarps);
  const unsigned cols = (unsigned)((p.P + 32 * CPL - 1) / (32 * CPL));
  ttmc_generic_kernel<CPL, FT><<<dim3(blocks, cols), kTtmcWarps * 32, 0, s>>>(p);
  ::tk::count_launch();
  return cudaGetLastError();
}

// Shape dispatch.  Returns false when no specialised kernel covers the shape.
template <typename FT>
static bool dispatch_fast(const TtmcParams &p, cudaStream_t s, cudaError_t *err) {
  const int no = p.nother;
  const int RB = p.R[no - 1];
#define TK_FAST(NL_, PL_, RB_, TA_, TB_)                   \
  {                                                        \
    *err = run_fast<NL_, PL_, RB_, TA_, TB_, FT>(p, s);    \
    return true;                                           \
  }
  if (no == 1) {
    if (RB == 16) TK_FAST(0, 1, 16, 1, 4)
    if (RB == 32) TK_FAST(0, 1, 32, 1, 4)
    if (RB == 8) TK_FAST(0, 1, 8, 1, 4)
  } else if (no == 2) {
    const int PL = p.R[0];
    if (PL == 16 && RB == 16) TK_FAST(1, 16, 16, 4, 4)
    if (PL == 8 && RB == 8) TK_FAST(1, 8, 8, 2, 4)
    if (PL == 32 && RB == 32) TK_FAST(1, 32, 32, 8, 4)
    if (PL == 16 && RB == 8) TK_FAST(1, 16, 8, 4, 4)
    if (PL == 8 && RB == 16) TK_FAST(1, 8, 16, 4, 4)
  } else if (no == 3) {
    const int PL = p.R[0] * p.R[1];
    if (p.R[1] % 4 == 0) {
      if (PL == 64 && RB == 8) TK_FAST(2, 64, 8, 4, 4)
      if (PL == 64 && RB == 16) TK_FAST(2, 64, 16, 8, 4)
      if (PL == 16 && RB == 4) TK_FAST(2, 16, 4, 2, 4)
    }
  }
#undef TK_FAST
  return false;
}

// TUCKER_TTMC_FUSED=1 selects the fused fiber kernel instead of the two-pass fiber form.
// Measured on the 20M-nonzero skewed workload it ran at best level with the two passes
// (0.55 / 0.42 ms against 0.42 / 0.435 ms on its two fiber modes): both levels wait on
// factor-row gathers, and holding the fiber ring and both levels' registers leaves fewer
// resident warps to hide them.  It is kept as an opt-in form: it moves no t_f through HBM.
static bool fused_fibers() {
  const char *e = std::getenv("TUCKER_TTMC_FUSED");
  return e && e[0] == '1';
}

// With `colsq` given, the pipelined FP32 forms also write the column sums of squares of Y
// there (*norms true); every other form leaves *norms false.
static tucker_status ttmc_impl(Ctx *c, int mode, float *Y, const float *val, const float *const *Uf,
                               cudaStream_t s, double *colsq = nullptr, bool *norms = nullptr) {
  const ModeCopy &mc = c->mode[mode];
  if (norms) *norms = false;
  // per-block pairs of P columns for each of the 8 warps: formed where that stays small
  const bool want_sq = colsq && norms && c->sq_part && c->sq_cnt && mc.P <= 256;
  const bool bf16 = !Uf && (c->flags & TUCKER_F_BF16_FACTORS) != 0;
  TtmcParams p{};
  p.nother = mc.nother;
  for (int t = 0; t < mc.nother; ++t) {
    const int m = mc.other[t];
    p.idx[t] = mc.idx[t];
    p.U[t] = Uf ? static_cast<const void *>(Uf[m])
                : bf16 ? static_cast<const void *>(c->U16[m]) : static_cast<const void *>(c->U32[m]);
    p.R[t] = c->ranks[m];
  }
  p.val = val ? val : mc.val;
  p.sptr = mc.sptr;
  p.sid = mc.sid;
  p.S = (uint32_t)mc.S;
  p.unit_e0 = mc.unit_e0;
  p.unit_k0 = mc.unit_k0;
  p.unit_slot = mc.unit_slot;
  p.n_units = mc.n_units;
  p.Z = (uint32_t)c->nnz;
  p.Y = Y;
  p.carry = c->carry;
  p.P = mc.P;
  p.err = c->d_err;
  // A fiber level, opt-in fused kernel (fiber sums kept on chip), FP32 or BF16 factors
  if (!(c->flags & TUCKER_F_UNPIPELINED) && mc.fib && mc.n_units > 0 && mc.unit_f0 &&
      p.nother == 2 && fused_fibers()) {
    const int ft = mc.fmid_t;
    FiberParams f{};
    f.val = p.val;
    f.isum = mc.idx[1 - ft];
    f.Usum = p.U[1 - ft];
    f.Umid = p.U[ft];
    f.fptr = mc.fptr;
    f.fmid = mc.fmid;
    f.fbits = mc.fbits;
    f.fsptr = mc.fsptr;
    f.sid = mc.sid;
    f.S = (uint32_t)mc.S;
    f.F = (uint32_t)mc.F;
    f.Z = (uint32_t)c->nnz;
    f.unit_e0 = mc.unit_e0;
    f.unit_f0 = mc.unit_f0;
    f.unit_k0 = mc.unit_k0;
    f.unit_slot = mc.unit_slot;
    f.n_units = mc.n_units;
    f.Y = Y;
    f.carry = c->carry;
    f.P = mc.P;
    cudaError_t err = cudaSuccess;
    const bool done = bf16 ? dispatch_fiber<__nv_bfloat16>(f, p.R[ft], p.R[1 - ft], ft == 0, s, &err)
                           : dispatch_fiber<float>(f, p.R[ft], p.R[1 - ft], ft == 0, s, &err);
    if (done) {
      TK_CUDA(err);
      if (mc.n_long > 0) launch_fixup(mc.long_k, mc.long_u0, mc.long_np, mc.n_long, mc.sid, c->carry, Y, mc.P, s);
      if (mc.n_empty > 0) {
        ttmc_zero_rows_kernel<<<(unsigned)std::min<int64_t>(mc.n_empty, 65535), 256, 0, s>>>(mc.empty, mc.n_empty,
                                                                                            Y, mc.P);
        ::tk::count_launch();
      }
      TK_CUDA(cudaGetLastError());
      return TUCKER_OK;
    }
  }
  // FP32 factors with a fiber level, two passes: fiber sums to HBM, then the pipelined
  // update over fibers
  if (!bf16 && !(c->flags & TUCKER_F_UNPIPELINED) && mc.fib && mc.fn_units > 0 && c->fib_T &&
      p.nother == 2 && pipe_shape(p.R[0], p.R[1])) {
    TtmcParams q = p;
    q.sptr = mc.fsptr;
    q.unit_e0 = mc.funit_e0;
    q.unit_k0 = mc.funit_k0;
    q.unit_slot = mc.funit_slot;
    q.n_units = mc.fn_units;
    q.Z = (uint32_t)mc.F;
    q.fptr = mc.fptr;
    q.fmid = mc.fmid;
    cudaError_t err = cudaSuccess;
    const int ft = mc.fmid_t;  // middle level: remaining mode other[ft]; t_f sums other[1 - ft]
    TtmcParams qs = q;         // the fiber-sum pass reads the summed mode as its "last" mode
    qs.idx[1] = q.idx[1 - ft];
    qs.U[1] = q.U[1 - ft];
    qs.R[1] = q.R[1 - ft];
    if (dispatch_fibsum(qs, c->fib_T, c->nnz, s, &err)) {
      TK_CUDA(err);
      TtmcParams r = q;  // the fibers as nonzeros, value 1: rows t_f and the middle mode's rows
      r.idx[ft] = mc.fmid;
      r.idx[1 - ft] = c->fib_iota;
      r.U[1 - ft] = c->fib_T;
      r.val = c->fib_ones;
      const int64_t nb = ttmc_pipe_blocks(r.n_units);
      const bool sq = want_sq && (nb + mc.fn_long + colsq_chunks(nb + mc.fn_long)) * mc.P <= c->sq_elems;
      if (sq) r.sq_part = c->sq_part;
      dispatch_pipe(r, s, &err);  // covers the shape (checked above)
      TK_CUDA(err);
      if (mc.fn_long > 0)
        launch_fixup(mc.flong_k, mc.flong_u0, mc.flong_np, mc.fn_long, mc.sid, c->carry, Y, mc.P, s,
                     sq ? c->sq_part + nb * mc.P : nullptr);
      if (sq) {
        launch_colsq(c->sq_part, nb + mc.fn_long, mc.P, c->sq_cnt, colsq, s);
        *norms = true;
      }
      if (mc.n_empty > 0) {
        ttmc_zero_rows_kernel<<<(unsigned)std::min<int64_t>(mc.n_empty, 65535), 256, 0, s>>>(mc.empty, mc.n_empty,
                                                                                            Y, mc.P);
        ::tk::count_launch();
      }
      TK_CUDA(cudaGetLastError());
      return TUCKER_OK;
    }
  }
  int64_t sq_rows = 0;      // rows of pairs the pipelined form left (0: none)
  float2 *sq_fix = nullptr;  // where the fixup puts the squares of the split slices' rows
  if (mc.n_units > 0) {
    cudaError_t err = cudaSuccess;
    bool done = false;
    if (bf16) {  // the BF16-factor form runs on the tensor cores
      if (p.nother == 2 && p.R[0] == 16 && p.R[1] == 16 && c->tm16_ok[mc.other[0]] && c->tm16_ok[mc.other[1]] &&
          tma_rows()) {  // rows gathered by the TMA into a ring of tiles
        err = run_bf16_tma<16, 16>(p, c->tm16[mc.other[0]], c->tm16[mc.other[1]], s);
        done = true;
      } else {
        done = dispatch_bf16(p, s, &err);
      }
    } else if (!(c->flags & TUCKER_F_UNPIPELINED)) {
      const int64_t nb = ttmc_pipe_blocks(p.n_units);
      const bool sq = want_sq && pipe_shape(p.R[0], p.R[1]) && p.nother == 2 &&
                      (nb + mc.n_long + colsq_chunks(nb + mc.n_long)) * mc.P <= c->sq_elems;
      if (sq) p.sq_part = c->sq_part;
      done = dispatch_pipe(p, s, &err);
      if (done && sq) {
        sq_rows = nb + mc.n_long;
        sq_fix = c->sq_part + nb * mc.P;
      }
      p.sq_part = nullptr;
    }
    if (!done) done = bf16 ? dispatch_fast<__nv_bfloat16>(p, s, &err) : dispatch_fast<float>(p, s, &err);
    if (!done) err = bf16 ? run_generic<__nv_bfloat16>(p, s) : run_generic<float>(p, s);
    TK_CUDA(err);
  }
  if (mc.n_long > 0) {
    launch_fixup(mc.long_k, mc.long_u0, mc.long_np, mc.n_long, mc.sid, c->carry, Y, mc.P, s, sq_fix);
    TK_CUDA(cudaGetLastError());
  }
  if (sq_rows > 0) {
    launch_colsq(c->sq_part, sq_rows, mc.P, c->sq_cnt, colsq, s);
    TK_CUDA(cudaGetLastError());
    *norms = true;
  }
  if (mc.n_empty > 0) {
    ttmc_zero_rows_kernel<<<(unsigned)std::min<int64_t>(mc.n_empty, 65535), 256, 0, s>>>(mc.empty, mc.n_empty, Y,
                                                                                        mc.P);
    ::tk::count_launch();
    TK_CUDA(cudaGetLastError());
  }
  return TUCKER_OK;
}

// TMA descriptors of the BF16 factor copies: a 2-D tensor I_m x R_m (rows of R_m * 2 bytes),
// one row per box, so that a gather4 copy fetches four rows.  Built with the driver's
// cuTensorMapEncodeTiled, looked up through the runtime (no link against the driver).
void make_factor_maps(Ctx *c) {
  using EncodeFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  void *fn = nullptr;
  cudaDriverEntryPointQueryResult q{};
  for (int m = 0; m < c->N; ++m) c->tm16_ok[m] = false;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !fn) {
    cudaGetLastError();
    return;
  }
  auto encode = reinterpret_cast<EncodeFn>(fn);
  for (int m = 0; m < c->N; ++m) {
    const int R = c->ranks[m];
    if (!c->U16[m] || (R * 2) % 16 != 0 || c->dims[m] > 0xffffffffLL) continue;
    const cuuint64_t dims[2] = {(cuuint64_t)R, (cuuint64_t)c->dims[m]};
    const cuuint64_t strides[1] = {(cuuint64_t)R * 2};
    const cuuint32_t box[2] = {(cuuint32_t)R, 1};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = encode(&c->tm16[m], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, c->U16[m], dims, strides, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    c->tm16_ok[m] = (r == CUDA_SUCCESS);
  }
}

tucker_status launch_ttmc(Ctx *c, int mode, float *Y, cudaStream_t s) {
  return ttmc_impl(c, mode, Y, nullptr, nullptr, s);
}

tucker_status launch_ttmc_norms(Ctx *c, int mode, float *Y, double *colsq, bool *formed, cudaStream_t s) {
  return ttmc_impl(c, mode, Y, nullptr, nullptr, s, colsq, formed);
}

tucker_status launch_ttmc_ex(Ctx *c, int mode, float *Y, const float *val, const float *const *Uf, cudaStream_t s) {
  return ttmc_impl(c, mode, Y, val, Uf, s);
}

}  // namespace tk
