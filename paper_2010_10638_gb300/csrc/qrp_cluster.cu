// K-c, cluster form: the Householder QR with column pivoting of qrp.cu (Section III-D;
// same implicit update A P - V F^T, same reflector, norm-downdate and pivot rules) run
// with one grid-wide synchronisation per reflector.
//
// Rows of A are split over all blocks of one launch; columns are split over the S
// blocks of each thread-block cluster (block `rank` owns the columns c = rank mod S),
// and every cluster repeats the same column work.  Each block keeps in shared memory
// its rows of V, the F rows, norms and flags of its columns, the column order, T, the
// top k x k corner of V, and as many of its rows of A as fit.  A step j is
//   rows     y = A[:, p] - V F[p, :]^T on this block's rows (F[p, :] read from the
//            owning block's shared memory); partial sums of A^T y, V^T y, ||y||^2,
//            and from the block owning row j, y_jj and V[j, :j]
//   reduce   the partial vectors of a cluster are added through distributed shared
//            memory; with several clusters one slice per block goes to global memory,
//            the clusters meet at one bounded counter barrier, and every block adds
//            the cluster sums it needs (its columns and the scalars) in cluster order
//   columns  the reflector (tau, beta, v_jj), F[:, j], row j of R and the norm
//            downdates of this block's columns
//   pivot    each block proposes the largest remaining norm of its columns; after one
//            cluster barrier every block takes the best proposal (lowest position on
//            ties), so all copies of the column order stay identical.
// A^T v_j is A^T y + (v_jj - y_jj) A[j, :] (v_j differs from y only in row j), so the
// pass over A starts before the reflector is known.  FP32 A: the column norms are exact
// products summed in double-float pairs (dfloat.cuh); A^T y is summed around power-of-two
// offsets chosen from those norms (off_fma), eight FP32 operations per product with the
// rounding residuals kept; each column's sum is converted to FP64 once.  FP64 A: FMA.
// The FP64 pipe is narrow on this GPU, so FP64 work is kept to what the method needs
// and is not issued for idle lanes in long loops.  Downdated norms that lose more than
// sqrt(eps) of their last exact value are recomputed exactly (rare).
#include <cooperative_groups.h>

#include <algorithm>
#include <cfloat>
#include <climits>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <type_traits>

#include "dfloat.cuh"
#include "internal.cuh"

namespace cg = cooperative_groups;

namespace tk {
namespace {

constexpr int kCT = 512;  // threads per block, one block per SM
constexpr int kCW = kCT / 32;
constexpr unsigned long long kCSpin = 1ull << 25;  // polls before a barrier wait gives up
// During a reflector step the first kColT threads form A^T y (FP32 pipe) while the last
// kCT - kColT threads form V^T y and ||y||^2 (FP64 pipe), each group with its own barrier.
constexpr int kColT = 448;
constexpr int64_t kQfDfRows = 128;  // rows per block from which Q is formed in double-float sums
constexpr int kAuxT = kCT - kColT;
// the auxiliary warps keep their V^T y partials in red4[kCT, kCT + 64) and their ||y||^2
// sums from red4[kCT + 64] on: at most two of them (448 / 64 measured fastest of 480 / 32
// and 448 / 64)
static_assert(kAuxT == 32 || kAuxT == 64, "one or two auxiliary warps");

// Threads per row of A in the FP32 column sums (one column quad per thread): the power of
// two from 8 up to the number of quads nq, at most nt; the remaining threads form nt / cw
// row lanes.  The norm pass and the A^T y passes use the same layout, so a thread keeps the
// same rows and columns in both.
__host__ __device__ inline int quad_cw(int64_t nq, int nt) {
  int cw = 8;
  while (cw < nq && cw * 2 <= nt) cw <<= 1;
  return cw;
}

// barrier of the first NT threads of the block (all of them: __syncthreads)
template <int NT>
__device__ __forceinline__ void group_sync() {
  if constexpr (NT == kCT)
    __syncthreads();
  else
    asm volatile("bar.sync 1, %0;\n" ::"r"(NT) : "memory");
}

struct CArgs {
  const void *A;
  int64_t m, n, lda;
  int k;
  int L;          // partial-vector length n + 2k + 2
  int nclusters;  // clusters in the launch
  int cluster;    // blocks per cluster the shared-memory plan was made for
  int vec4;       // FP32 A read as float4 (n % 4 == 0, lda % 4 == 0, 16-byte aligned)
  int64_t rows_per;     // rows of A per block
  int64_t rows_cached;  // leading rows of each block's range kept in shared memory
  double *slots;        // [2][nclusters][L] cluster sums (alternating buffers)
  unsigned *bar;        // [0] arrival count, [2] abort flag
  uint32_t *err;        // where a timed-out wait is reported
  double *Q;
  int64_t ldq;
  int64_t *piv;
  double *rdiag;
  const double *colsq;  // [n] column sums of squares of A given by the caller (FP32 A read as
                        // float4 only), or nullptr: the first pass over A forms them
};

// Checked build (TUCKER_QRP_CHECKED): QX(i, len, site) is i when 0 <= i < len; otherwise it
// records the site and gives 0, so that the access stays inside its array.  Each block
// reports a recorded site through the launch's error word (kErrCheck) as it leaves.  In
// the normal build QX(i, len, site) is i itself and nothing else changes.
#ifdef TUCKER_QRP_CHECKED
__device__ unsigned g_qc_site;  // first site whose index fell outside its array (0: none)
__device__ __forceinline__ int64_t qc_index(int64_t i, int64_t len, unsigned site) {
  if (i >= 0 && i < len) return i;
  atomicCAS(&g_qc_site, 0u, site);
  return 0;
}
#define QX(i, len, site) qc_index((int64_t)(i), (int64_t)(len), (site))
__device__ __forceinline__ void qc_report(uint32_t *err) {
  if (threadIdx.x == 0 && *(volatile unsigned *)&g_qc_site) atomicOr(err, kErrCheck);
}
#else
#define QX(i, len, site) (i)
__device__ __forceinline__ void qc_report(uint32_t *) {}
#endif

// Dynamic shared memory of one block; the same arithmetic on host and device.
struct CLayout {
  size_t Fo, vno, vrefo, ajo, svo, svs, flago, doneo, red, Ts, Vt, Ms, su, Vs, red4, cscr, nat, ys, perm, posof, cand,
      As, total;
  int kp;      // row stride of Vs in doubles (odd: rows fall in different banks)
  int64_t no;  // columns per block, rounded up
};

__host__ __device__ inline size_t c16(size_t b) { return (b + 15) & ~(size_t)15; }

__host__ __device__ inline CLayout clayout(int64_t n, int k, int L, int S, int64_t rows_per, int64_t rows_cached,
                                           int esize) {
  CLayout l{};
  l.kp = k | 1;
  l.no = (n + S - 1) / S;
  const size_t no = (size_t)l.no;
  size_t o = 0;
  l.Fo = o;    o += c16(sizeof(double) * (size_t)k * no);  // F of this block's columns: Fo[l * no + lc]
  l.vno = o;   o += c16(sizeof(double) * no);
  l.vrefo = o; o += c16(sizeof(double) * no);
  l.ajo = o;   o += c16(sizeof(double) * no);              // A[j, c] of this block's columns
  l.svo = o;   o += c16(sizeof(double) * no);              // reduced A^T y of this block's columns
  l.svs = o;   o += c16(sizeof(double) * (size_t)(2 * k + 2));  // reduced scalars
  l.flago = o; o += c16(sizeof(int) * no);
  l.doneo = o; o += c16(sizeof(int) * no);
  l.red = o;   o += c16(sizeof(double) * 2 * (size_t)L);  // this block's partials, two buffers
  l.Ts = o;    o += c16(sizeof(double) * (size_t)k * k);
  l.Vt = o;    o += c16(sizeof(double) * (size_t)k * k);  // V[0:k, 0:k]
  l.Ms = o;    o += c16(sizeof(double) * (size_t)k * k);
  l.su = o;    o += c16(sizeof(double) * 64);
  l.Vs = o;    o += c16(sizeof(double) * (size_t)rows_per * l.kp);  // this block's rows of V
  l.red4 = o;  o += c16(sizeof(double) * 2 * kCT);        // reduction scratch (8 KB)
  l.cscr = o;  // column-sum scratch: 2 x kCT doubles, or 4 x kColT double-float pairs
  o += c16(sizeof(double) * 2 * kCT > sizeof(float) * 8 * kColT ? sizeof(double) * 2 * kCT : sizeof(float) * 8 * kColT);
  l.nat = o;   // FP32 A: per thread and column quad, bounds on the norms of its pieces of 4 columns
  if (esize == 4 && n % 4 == 0) {
    const int64_t nq = n / 4, cw = quad_cw(nq, kColT);
    o += c16(sizeof(float) * 4 * (size_t)kColT * (size_t)((nq + cw - 1) / cw));
  }
  l.ys = o;    o += c16(sizeof(double) * (size_t)rows_per);  // y per row (float2 or double)
  l.perm = o;  o += c16(sizeof(int) * (size_t)n);
  l.posof = o; o += c16(sizeof(int) * (size_t)n);
  l.cand = o;  o += 32;                                    // pivot proposal: key, position, any flag
  l.As = o;    o += c16((size_t)esize * (size_t)rows_cached * (size_t)n);
  l.total = o;
  return l;
}

// global -> shared copies without a register round trip (completed by cp.async.wait_all)
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
template <typename T>
__device__ __forceinline__ void cp_async_elem(T *dst, const T *src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  if constexpr (sizeof(T) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}

// double-float addition a += b (TwoSum of the high parts, then renormalisation)
__device__ __forceinline__ void df_add(DF &a, const DF b) {
  const float s = a.hi + b.hi;
  const float bp = s - a.hi;
  float e = (a.hi - (s - bp)) + (b.hi - bp);
  e += a.lo + b.lo;
  a.hi = s + e;
  a.lo = e - (a.hi - s);
}

// Entries of the reductions' partial vectors.  FP32 A: double-float pairs (x = hi,
// y = lo), so that their sums over the blocks of a cluster and over the clusters run on
// the FP32 pipe (the FP64 pipe issues one warp instruction per 16 cycles per SM here),
// with about 2^-48 relative error per addition; each needed entry is converted to FP64
// once at the end.  FP64 A (values of any FP64 magnitude): FP64.
__device__ __forceinline__ float2 df2_of(double v) {
  const float h = __double2float_rn(v);
  return make_float2(h, __double2float_rn(v - (double)h));
}
__device__ __forceinline__ double df2_val(float2 p) { return (double)p.x + (double)p.y; }
__device__ __forceinline__ float2 df2_add(float2 a, float2 b) {
  DF x;
  x.hi = a.x;
  x.lo = a.y;
  DF y;
  y.hi = b.x;
  y.lo = b.y;
  df_add(x, y);
  return make_float2(x.hi, x.lo);
}

// t -= (v.x + v.y) (m.x + m.y): the product of the high parts exactly (FMA residual), the
// cross terms by FMA, the low-low term dropped (2^-48 of the product); TwoSum of the high parts
__device__ __forceinline__ void df_sub_prod(DF &t, float2 v, float2 m) {
  const float p = v.x * m.x;
  float e = fmaf(v.x, m.x, -p);
  e = fmaf(v.x, m.y, e);
  e = fmaf(v.y, m.x, e);
  const float s = t.hi - p;
  const float bp = s - t.hi;
  const float err = (t.hi - (s - bp)) - (p + bp);
  t.hi = s;
  t.lo += err - e;
}

// FP32 -> FP64 without the FP64 pipe: the same sign, the exponent rebiased (+896), the
// mantissa shifted up 29 bits; exact for normal numbers (zero, subnormals, inf and NaN
// take the conversion instruction)
__device__ __forceinline__ double f2d_exact(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned e = (b >> 23) & 0xffu;
  if (e == 0u || e == 0xffu) return (double)f;
  const unsigned long long d = ((unsigned long long)(b & 0x80000000u) << 32) |
                               ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)(b & 0x7fffffu) << 29);
  return __longlong_as_double((long long)d);
}

template <typename PT>
struct Part;
template <>
struct Part<float2> {
  static __device__ __forceinline__ float2 of(double v) { return df2_of(v); }
  static __device__ __forceinline__ double val(float2 p) { return df2_val(p); }
  static __device__ __forceinline__ float2 add(float2 a, float2 b) { return df2_add(a, b); }
  static __device__ __forceinline__ float2 zero() { return make_float2(0.f, 0.f); }
};
template <>
struct Part<double> {
  static __device__ __forceinline__ double of(double v) { return v; }
  static __device__ __forceinline__ double val(double p) { return p; }
  static __device__ __forceinline__ double add(double a, double b) { return a + b; }
  static __device__ __forceinline__ double zero() { return 0.0; }
};
template <typename AT>
using PartT = typename std::conditional<sizeof(AT) == 4, float2, double>::type;

// Ordering key of a squared norm (>= 0): its bit pattern without the sign (so -0 = 0);
// NaN gets -1 and is never preferred.  Integer compares keep argmax off the FP64 pipe.
__device__ __forceinline__ long long norm_key(double v) {
  const long long b = __double_as_longlong(v) & 0x7fffffffffffffffll;
  return b > 0x7ff0000000000000ll ? -1ll : b;
}

// Bounded counter barrier of the clusters' leading threads: every arrival adds one
// (release); a leader waits until the count reaches target = calls so far x clusters.
__device__ bool leaders_barrier(const CArgs &a, unsigned target) {
  asm volatile("red.release.gpu.global.add.u32 [%0], 1;\n" ::"l"(a.bar) : "memory");
  unsigned long long spins = 0;
  while (true) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(a.bar) : "memory");
    if (v >= target) break;
    if (++spins > kCSpin) {
      atomicOr(a.bar + 2, 1u);
      atomicOr(a.err, kErrTimeout);
      break;
    }
    if ((spins & 255u) == 0u && *(volatile unsigned *)(a.bar + 2)) break;  // another cluster gave up
    __nanosleep(20);
  }
  return *(volatile unsigned *)(a.bar + 2) == 0u;
}

// Pairwise sum of 16 values in a fixed tree ((x0 + x1) + (x2 + x3)) + ...: depth 4
// instead of a 15-long chain of dependent FP64 additions.
__device__ __forceinline__ double tree16(double (&x)[16]) {
#pragma unroll
  for (int w = 1; w < 16; w <<= 1)
#pragma unroll
    for (int i = 0; i < 16; i += 2 * w) x[i] += x[i + w];
  return x[0];
}

// the same tree over partial-vector entries
template <int NS, typename PT>
__device__ __forceinline__ PT ptree(PT (&x)[NS]) {
#pragma unroll
  for (int w = 1; w < NS; w <<= 1)
#pragma unroll
    for (int i = 0; i < NS; i += 2 * w) x[i] = Part<PT>::add(x[i], x[i + w]);
  return x[0];
}

template <int NS, typename PT>
__device__ __forceinline__ PT peer_tree(cg::cluster_group &cl, PT *mine, int q) {
  PT x[NS];
#pragma unroll
  for (int r = 0; r < NS; ++r) x[r] = cl.map_shared_rank(mine, (unsigned)r)[q];
  return ptree<NS>(x);
}

// sum over the S blocks of the cluster (S a power of two, at most 16) of entry q of
// their vectors `mine` (shared memory), in a fixed tree over the ranks; all S loads are
// issued before the additions
template <typename PT>
__device__ __forceinline__ PT peer_sum(cg::cluster_group &cl, PT *mine, unsigned S, int q) {
  switch (S) {
    case 16: return peer_tree<16, PT>(cl, mine, q);
    case 8: return peer_tree<8, PT>(cl, mine, q);
    case 4: return peer_tree<4, PT>(cl, mine, q);
    case 2: return peer_tree<2, PT>(cl, mine, q);
    default: return mine[q];
  }
}

struct Team {
  unsigned S, rank;
  int nown;        // columns owned by this block
  unsigned epoch;  // grid-wide reductions so far
};

// Sums of the blocks' partial vectors `mine` (L double-float pairs each, shared memory),
// in the same order in every block: entries of this block's columns into svo, the scalar
// entries n .. L-1 into svs (FP64).  `scratch` holds ceil(clusters / 16) x (entries
// needed) pairs.  False when a wait timed out (then no block reads a peer's memory any more).
template <typename PT>
__device__ bool allreduce(const CArgs &a, cg::cluster_group &cl, Team &tm, PT *mine, double *svo, double *svs,
                          int par, int *s_ok, PT *scratch) {
  const int L = a.L, n = (int)a.n, ns = 2 * a.k + 2, need = tm.nown + ns;
  auto entry = [&](int t) { return t < tm.nown ? (int)tm.rank + (int)tm.S * t : n + (t - tm.nown); };
  auto store = [&](int t, double v) {
    if (t < tm.nown)
      svo[t] = v;
    else
      svs[t - tm.nown] = v;
  };
  cl.sync();  // every block of the cluster has written its partials
  if (a.nclusters == 1) {
    for (int t = threadIdx.x; t < need; t += kCT) store(t, Part<PT>::val(peer_sum(cl, mine, tm.S, QX(entry(t), L, 1))));
    __syncthreads();
    return true;  // `mine` alternates between two buffers: the next write cannot race these reads
  }
  const int cid = (int)(blockIdx.x / tm.S);
  PT *slot = reinterpret_cast<PT *>(a.slots) + ((size_t)par * a.nclusters + cid) * L;
  const int per = (int)((L + tm.S - 1) / tm.S);
  const int q0 = (int)tm.rank * per, q1 = min(L, q0 + per);
  bool wrote = false;
  for (int q = q0 + threadIdx.x; q < q1; q += kCT) {
    slot[q] = peer_sum(cl, mine, tm.S, QX(q, L, 2));
    wrote = true;
  }
  if (wrote) __threadfence();
  cl.sync();  // the cluster's sum is stored
  tm.epoch += 1;
  if (tm.rank == 0 && threadIdx.x == 0) *s_ok = leaders_barrier(a, tm.epoch * (unsigned)a.nclusters) ? 1 : 0;
  cl.sync();  // the leader passed the barrier (or gave up)
  const int ok = *cl.map_shared_rank(s_ok, 0);
  if (!ok) {
    cl.sync();  // nobody reads rank 0's flag once it may have left
    return false;
  }
  // the cluster sums this block needs: thread (entry t, chunk h) adds the clusters
  // 16h .. 16h+15 of entry t in a fixed tree (one round trip for all of them), then the
  // chunk sums of each entry are added in chunk order
  const PT *base = reinterpret_cast<const PT *>(a.slots) + (size_t)par * a.nclusters * L;
  const int nch = (a.nclusters + 15) / 16;
  for (int idx = threadIdx.x; idx < need * nch; idx += kCT) {
    const int t = idx % need, h = idx / need, q = entry(t);
    PT x[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int cc = 16 * h + u;
      x[u] = (cc < a.nclusters) ? __ldcg(base + (size_t)cc * L + QX(q, L, 3)) : Part<PT>::zero();
    }
    scratch[idx] = ptree<16>(x);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < need; t += kCT) {
    PT sum = scratch[t];
    for (int h = 1; h < nch; ++h) sum = Part<PT>::add(sum, scratch[h * need + t]);
    store(t, Part<PT>::val(sum));
  }
  __syncthreads();
  return true;
}

// Rows [s0, s1) (local indices) of four adjacent columns into double-float sums.
template <bool GLOBAL, bool SQUARE>
__device__ __forceinline__ void seg4(const float4 *base, int64_t stride4, int64_t s0, int64_t s1, int rl, int nrl,
                                     const float2 *y2, DF &d0, DF &d1, DF &d2, DF &d3) {
  int64_t ii = s0 + rl;
  for (; ii + 7 * nrl < s1; ii += 8 * nrl) {
    float4 x[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const float4 *p = base + (ii + u * nrl) * stride4;
      x[u] = GLOBAL ? __ldg(p) : *p;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      if (SQUARE) {
        df_fma(d0, x[u].x, x[u].x, 0.f);
        df_fma(d1, x[u].y, x[u].y, 0.f);
        df_fma(d2, x[u].z, x[u].z, 0.f);
        df_fma(d3, x[u].w, x[u].w, 0.f);
      } else {
        const float2 vv = y2[ii + u * nrl];
        df_fma(d0, x[u].x, vv.x, vv.y);
        df_fma(d1, x[u].y, vv.x, vv.y);
        df_fma(d2, x[u].z, vv.x, vv.y);
        df_fma(d3, x[u].w, vv.x, vv.y);
      }
    }
  }
  for (; ii < s1; ii += nrl) {
    const float4 *p = base + ii * stride4;
    const float4 x = GLOBAL ? __ldg(p) : *p;
    if (SQUARE) {
      df_fma(d0, x.x, x.x, 0.f);
      df_fma(d1, x.y, x.y, 0.f);
      df_fma(d2, x.z, x.z, 0.f);
      df_fma(d3, x.w, x.w, 0.f);
    } else {
      const float2 vv = y2[ii];
      df_fma(d0, x.x, vv.x, vv.y);
      df_fma(d1, x.y, vv.x, vv.y);
      df_fma(d2, x.z, vv.x, vv.y);
      df_fma(d3, x.w, vv.x, vv.y);
    }
  }
}

// Offset accumulation of sum_i a_i (bh_i + bl_i) (FP32 a, FP64 y split into bh + bl), used
// for A^T y.  With B >= |every partial sum of a_i bh_i| and s1 a power of two > 2B, the
// running sum hi = s1 + (partial) stays in [s1/2, 3 s1/2]: every hi is a multiple of
// ulp(s1/2), so hi - t below is exact, and t = fma(a, bh, hi) rounds a_i bh_i onto that grid
// with residual r = a_i bh_i + hi - t (computed by a second FMA, to 2^-24 of |r|).  The
// residuals (each below 2^-24 s1) are summed exactly the same way around a second power of
// two s2 (Fast2Sum against a much larger addend), and only the residuals of that sum and
// the bl terms (2^-24 below the bh terms) are summed in plain FP32.  Eight FP32 operations
// per product instead of the twelve of a double-float sum; the error stays at about
// 2^-49 s1 per product.  B comes from Cauchy-Schwarz: ||a|| ||bh|| over the thread's rows.
struct OffAcc {
  float hi, mid, lo;
};

__device__ __forceinline__ void off_fma(OffAcc &s, float a, float bh, float bl) {
  const float t = fmaf(a, bh, s.hi);
  const float r = fmaf(a, bh, s.hi - t);
  const float t2 = s.mid + r;
  const float r2 = r + (s.mid - t2);
  s.lo = fmaf(a, bl, s.lo + r2);
  s.hi = t;
  s.mid = t2;
}

// s1: the power of two in (2 nb, 4 nb] (biased exponent + 2), kept inside the normal range
__device__ __forceinline__ float off_s1(float nb) {
  int e = (int)((__float_as_uint(nb) >> 23) & 0xffu) + 2;
  e = e < 1 ? 1 : (e > 254 ? 254 : e);
  return __uint_as_float((unsigned)e << 23);
}

// s2 for at most 2^lk residuals, each below 2^-24 s1: 4 times their largest possible sum
__device__ __forceinline__ float off_s2(float s1, int lk) {
  int e = (int)(__float_as_uint(s1) >> 23) - 22 + lk;
  e = e < 1 ? 1 : e;
  return __uint_as_float((unsigned)e << 23);
}

// Rows [s0, s1) (local indices, step nrl from s0 + rl) of four adjacent columns, eight
// rows per batch with all loads issued first (in this kernel's register budget, deeper
// batches keep more loads in flight: measured faster than four).  Row offsets are 32-bit:
// a block's rows times the row stride stay far below 2^31.
template <bool GLOBAL>
__device__ __forceinline__ void seg4_off(const float4 *base, int stride4, int s0, int s1, int rl, int nrl,
                                         const float2 *y2, OffAcc (&d)[4]) {
  int ii = s0 + rl;
  for (; ii + 7 * nrl < s1; ii += 8 * nrl) {
    float4 x[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const float4 *p = base + (ii + u * nrl) * stride4;
      x[u] = GLOBAL ? __ldg(p) : *p;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const float2 vv = y2[ii + u * nrl];
      off_fma(d[0], x[u].x, vv.x, vv.y);
      off_fma(d[1], x[u].y, vv.x, vv.y);
      off_fma(d[2], x[u].z, vv.x, vv.y);
      off_fma(d[3], x[u].w, vv.x, vv.y);
    }
  }
  for (; ii < s1; ii += nrl) {
    const float4 *p = base + ii * stride4;
    const float4 x = GLOBAL ? __ldg(p) : *p;
    const float2 vv = y2[ii];
    off_fma(d[0], x.x, vv.x, vv.y);
    off_fma(d[1], x.y, vv.x, vv.y);
    off_fma(d[2], x.z, vv.x, vv.y);
    off_fma(d[3], x.w, vv.x, vv.y);
  }
}

__device__ __forceinline__ DF df_of(float2 p) {
  DF d;
  d.hi = p.x;
  d.lo = p.y;
  return d;
}

// out[c], c < n (a double-float pair): sum over local rows li in [l0, nrows) of
// A[r0 + li, c] * y_li (SQUARE:
// A[r0 + li, c]^2).  Rows li < ncache come from the shared copy As (row stride n).
// Run by the first NT threads (NT a multiple of 32); `scratch` holds 2 * NT doubles (and,
// for FP32 A read as float4, 4 * NT double-float pairs).  FP32 A read as float4: the SQUARE
// pass stores in `nat` each thread's bound on the norms of its pieces of its 4 columns
// (quad layout of quad_cw), and the other passes use the offset accumulation with those
// bounds; their partial sums are added over the row lanes in one round, the threads of
// row lane c adding column c of every quad.
template <typename AT, bool SQUARE, int NT>
__device__ void ccolsum(const CArgs &a, const AT *As, int64_t ncache, int64_t r0, int64_t l0, int64_t nrows,
                        const void *ys, void *scratch, float *nat, PartT<AT> *out) {
  const int64_t n = a.n;
  const AT *A = static_cast<const AT *>(a.A);
  l0 = min(l0, nrows);
  if constexpr (sizeof(AT) == 4) {
    float2 *red = static_cast<float2 *>(scratch);
    const float2 *y2 = static_cast<const float2 *>(ys);
    if (a.vec4) {
      const int64_t nq = n / 4, ld4 = a.lda / 4, sn4 = n / 4;
      const int cw = quad_cw(nq, NT);
      const int nrl = NT / cw, cq = threadIdx.x % cw, rl = threadIdx.x / cw;
      const bool act = rl < nrl;  // NT need not be a multiple of cw
      float4 *nat4 = reinterpret_cast<float4 *>(nat);
      constexpr float kMargin = 1.0f + 1.0f / 256.0f;  // covers the FP32 rounding of the bounds
      if constexpr (SQUARE) {
        for (int64_t q0 = 0, it = 0; q0 < nq; q0 += cw, ++it) {
          const int64_t qc = q0 + cq;
          DF d[4];
          if (act && qc < nq) {
            seg4<false, true>(reinterpret_cast<const float4 *>(As) + qc, sn4, l0, min(nrows, ncache), rl, nrl, y2,
                              d[0], d[1], d[2], d[3]);
            seg4<true, true>(reinterpret_cast<const float4 *>(A) + r0 * ld4 + qc, ld4, max(l0, ncache), nrows, rl,
                             nrl, y2, d[0], d[1], d[2], d[3]);
          }
          if (nat && act)
            nat4[QX(it * NT + threadIdx.x, ((nq + cw - 1) / cw) * NT, 4)] = make_float4(sqrtf(fmaxf(d[0].hi, 0.f)) * kMargin, sqrtf(fmaxf(d[1].hi, 0.f)) * kMargin,
                                                      sqrtf(fmaxf(d[2].hi, 0.f)) * kMargin, sqrtf(fmaxf(d[3].hi, 0.f)) * kMargin);
#pragma unroll
          for (int h = 0; h < 2; ++h) {  // two columns of the four at a time through the scratch
            group_sync<NT>();
            red[threadIdx.x] = make_float2(d[2 * h].hi, d[2 * h].lo);
            red[NT + threadIdx.x] = make_float2(d[2 * h + 1].hi, d[2 * h + 1].lo);
            group_sync<NT>();
            if (rl == 0 && qc < nq) {
#pragma unroll
              for (int q = 0; q < 2; ++q) {
                DF t = d[2 * h + q];
                for (int r = 1; r < nrl; ++r) df_add(t, df_of(red[q * NT + r * cw + cq]));
                out[4 * qc + 2 * h + q] = make_float2(t.hi, t.lo);
              }
            }
          }
        }
      } else {
        // this thread's ||bh|| over its rows, and the number of rows it sums (for s2)
        float ny2 = 0.f;
        if (act) {  // eight independent sums: a single dependent chain costs a load latency per row
          float e8[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
          int li = (int)l0 + rl;
          for (; li + 7 * nrl < (int)nrows; li += 8 * nrl)
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              const float h = y2[li + u * nrl].x;
              e8[u] = fmaf(h, h, e8[u]);
            }
          for (; li < (int)nrows; li += nrl) {
            const float h = y2[li].x;
            e8[0] = fmaf(h, h, e8[0]);
          }
          ny2 = ((e8[0] + e8[1]) + (e8[2] + e8[3])) + ((e8[4] + e8[5]) + (e8[6] + e8[7]));
        }
        const float sy = sqrtf(ny2) * kMargin;
        const int lk = 64 - __clzll((nrows - l0 + nrl - 1) / nrl + 1);  // 2^lk > rows per thread
        for (int64_t q0 = 0, it = 0; q0 < nq; q0 += cw, ++it) {
          const int64_t qc = q0 + cq;
          const bool mine = act && qc < nq;
          const float4 nb = mine ? nat4[QX(it * NT + threadIdx.x, ((nq + cw - 1) / cw) * NT, 5)] : make_float4(0.f, 0.f, 0.f, 0.f);
          const float s1[4] = {off_s1(nb.x * sy), off_s1(nb.y * sy), off_s1(nb.z * sy), off_s1(nb.w * sy)};
          OffAcc d[4];
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            d[c].hi = s1[c];
            d[c].mid = off_s2(s1[c], lk);
            d[c].lo = 0.f;
          }
          if (mine) {
            seg4_off<false>(reinterpret_cast<const float4 *>(As) + qc, (int)sn4, (int)l0, (int)min(nrows, ncache), rl,
                            nrl, y2, d);
            seg4_off<true>(reinterpret_cast<const float4 *>(A) + r0 * ld4 + qc, (int)ld4, (int)max(l0, ncache),
                           (int)nrows, rl, nrl, y2, d);
          }
          if (it > 0) group_sync<NT>();  // the previous chunk's sums are read (the first: the caller's barrier)
#pragma unroll
          for (int c = 0; c < 4; ++c)  // hi - s1 and mid - s2 are exact (Sterbenz)
            red[c * NT + threadIdx.x] = make_float2(d[c].hi - s1[c], (d[c].mid - off_s2(s1[c], lk)) + d[c].lo);
          group_sync<NT>();
          if (act && qc < nq) {
            for (int c = rl; c < 4; c += nrl) {
              DF t = df_of(red[c * NT + cq]);
              for (int r = 1; r < nrl; ++r) df_add(t, df_of(red[c * NT + r * cw + cq]));
              out[4 * qc + c] = make_float2(t.hi, t.lo);
            }
          }
        }
      }
      group_sync<NT>();
      return;
    }
    int cw = 32;
    while (cw < n && cw * 2 <= NT) cw <<= 1;  // cw <= NT
    const int nrl = NT / cw, cl = threadIdx.x % cw, rl = threadIdx.x / cw;
    const bool act = rl < nrl;
    for (int64_t c0 = 0; c0 < n; c0 += cw) {
      const int64_t c = c0 + cl;
      DF d;
      if (act && c < n) {
        for (int64_t li = l0 + rl; li < nrows; li += nrl) {
          const float x = li < ncache ? (float)As[li * n + c] : (float)__ldg(A + (r0 + li) * a.lda + c);
          if (SQUARE) {
            df_fma(d, x, x, 0.f);
          } else {
            const float2 vv = y2[li];
            df_fma(d, x, vv.x, vv.y);
          }
        }
      }
      group_sync<NT>();
      red[threadIdx.x] = make_float2(d.hi, d.lo);
      group_sync<NT>();
      if (rl == 0 && c < n) {
        DF t = d;
        for (int r = 1; r < nrl; ++r) df_add(t, df_of(red[r * cw + cl]));
        out[c] = make_float2(t.hi, t.lo);
      }
    }
    group_sync<NT>();
  } else {
    double *red = static_cast<double *>(scratch);
    const double *yd = static_cast<const double *>(ys);
    int cw = 32;
    while (cw < n && cw * 2 <= NT) cw <<= 1;  // cw <= NT
    const int nrl = NT / cw, cl = threadIdx.x % cw, rl = threadIdx.x / cw;
    const bool act = rl < nrl;
    for (int64_t c0 = 0; c0 < n; c0 += cw) {
      const int64_t c = c0 + cl;
      double acc = 0.0;
      if (act && c < n) {
        for (int64_t li = l0 + rl; li < nrows; li += nrl) {
          const double x = li < ncache ? (double)As[li * n + c] : (double)__ldg(A + (r0 + li) * a.lda + c);
          acc = fma(x, SQUARE ? x : yd[li], acc);
        }
      }
      group_sync<NT>();
      red[threadIdx.x] = acc;
      group_sync<NT>();
      if (rl == 0 && c < n) {
        double t = acc;
        for (int r = 1; r < nrl; ++r) t += red[r * cw + cl];
        out[c] = t;
      }
    }
    group_sync<NT>();
  }
}

// The pivot for position j0: every block proposes its largest remaining norm (lowest
// position on ties), one cluster barrier, then every block takes the best proposal and
// swaps it into position j0.  When some block holds a norm flagged for exact
// recomputation nothing is swapped and true is returned (the same answer in every
// block).  The cluster barrier also publishes this step's F rows to the peers.
// The norm bounds of the A^T y passes (layout of ccolsum's SQUARE pass) when the caller
// gives the column sums of squares: each thread's pieces of its four columns are bounded by
// the whole columns' norms.  Those are valid bounds, looser than the pieces' own norms by
// about the square root of the number of pieces of a column, and so is each pass's offset.
template <int NT>
__device__ void nat_from_colsq(const CArgs &a, float *nat) {
  const int64_t nq = a.n / 4;
  const int cw = quad_cw(nq, NT);
  const int nrl = NT / cw, cq = threadIdx.x % cw, rl = threadIdx.x / cw;
  if (rl >= nrl) return;
  float4 *nat4 = reinterpret_cast<float4 *>(nat);
  constexpr float kMargin = 1.0f + 1.0f / 256.0f;  // covers the FP32 rounding of the bounds
  for (int64_t q0 = 0, it = 0; q0 < nq; q0 += cw, ++it) {
    const int64_t qc = q0 + cq;
    if (qc >= nq) continue;  // no pass reads these
    const double *cs = a.colsq + QX(4 * qc, a.n - 3, 6);
    nat4[QX(it * NT + threadIdx.x, ((nq + cw - 1) / cw) * NT, 7)] =
        make_float4(sqrtf((float)cs[0]) * kMargin, sqrtf((float)cs[1]) * kMargin, sqrtf((float)cs[2]) * kMargin,
                    sqrtf((float)cs[3]) * kMargin);
  }
}

__device__ bool choose_pivot(cg::cluster_group &cl, const Team &tm, int j0, int64_t n, const double *vno,
                             const int *flago, int *doneo, int *perm, int *posof, unsigned long long *cand,
                             int *s_res) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (warp == 0) {
    long long best = -1;
    int bp = INT_MAX, anyf = 0;
    for (int lc = lane; lc < tm.nown; lc += 32) {
      anyf |= flago[lc];
      if (doneo[lc]) continue;
      const long long key = norm_key(vno[lc]);
      const int p = posof[tm.rank + tm.S * lc];
      if (key > best || (key == best && key >= 0 && p < bp)) {
        best = key;
        bp = p;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const long long k2 = __shfl_xor_sync(0xffffffffu, best, o);
      const int p2 = __shfl_xor_sync(0xffffffffu, bp, o);
      if (k2 > best || (k2 == best && p2 < bp)) {
        best = k2;
        bp = p2;
      }
      anyf |= __shfl_xor_sync(0xffffffffu, anyf, o);
    }
    if (lane == 0) {
      cand[0] = (unsigned long long)best;
      cand[1] = (unsigned long long)(unsigned)bp;
      cand[2] = (unsigned long long)anyf;
    }
  }
  cl.sync();
  if (warp == 0) {
    long long best = -1;
    int bp = INT_MAX, anyf = 0;
    if (lane < (int)tm.S) {
      const unsigned long long *pc = cl.map_shared_rank(cand, (unsigned)lane);
      best = (long long)pc[0];
      bp = (int)(unsigned)pc[1];
      anyf = (int)pc[2];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const long long k2 = __shfl_xor_sync(0xffffffffu, best, o);
      const int p2 = __shfl_xor_sync(0xffffffffu, bp, o);
      if (k2 > best || (k2 == best && p2 < bp)) {
        best = k2;
        bp = p2;
      }
      anyf |= __shfl_xor_sync(0xffffffffu, anyf, o);
    }
    if (lane == 0) {
      if (!anyf && bp != INT_MAX && bp < n) {
        const int cj = perm[j0], cb = perm[bp];
        perm[j0] = cb;
        perm[bp] = cj;
        posof[cb] = j0;
        posof[cj] = bp;
        if (cb % (int)tm.S == (int)tm.rank) doneo[cb / (int)tm.S] = 1;
      }
      *s_res = anyf;
    }
  }
  __syncthreads();
  return *s_res != 0;
}

__device__ void cbail(const CArgs &a) {
  qc_report(a.err);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const double qnan = __longlong_as_double(0x7ff8000000000000ll);
    if (a.rdiag)
      for (int j = 0; j < a.k; ++j) a.rdiag[j] = qnan;
    if (a.piv)
      for (int j = 0; j < a.k; ++j) a.piv[j] = -1;
    a.Q[0] = qnan;  // a factor with a NaN makes the failure visible downstream
  }
}

template <typename AT>
__global__ void __launch_bounds__(kCT, 1) qrp_cluster_kernel(CArgs a) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ double s_f[64];  // F[p, 0:j] of the current pivot column
  __shared__ double s_sc[4];  // v_jj, tau, v_jj - y_jj
  __shared__ int s_ok, s_res;
  cg::cluster_group cl = cg::this_cluster();
  Team tm;
  tm.S = cl.num_blocks();
  tm.rank = cl.block_rank();
  tm.epoch = 0;
  // The shared-memory carve-up below depends on the cluster shape and must fit the launch's
  // dynamic shared memory: a launch whose shape or size differs from the plan (the same in
  // every block) reports an error and touches nothing else.
  if ((int)tm.S != a.cluster || (int)gridDim.x != a.cluster * a.nclusters) {
    if (threadIdx.x == 0) atomicOr(a.err, kErrLaunch);
    return cbail(a);
  }
  const int64_t n = a.n, m = a.m;
  const int k = a.k, L = a.L;
  const CLayout lay = clayout(n, k, L, (int)tm.S, a.rows_per, a.rows_cached, (int)sizeof(AT));
  {  // the carve-up must fit the dynamic shared memory this launch actually has
    unsigned dyn;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
    if ((size_t)lay.total > (size_t)dyn) {
      if (threadIdx.x == 0) atomicOr(a.err, kErrLaunch);
      return cbail(a);
    }
  }
  tm.nown = (int)((n - (int64_t)tm.rank + tm.S - 1) / tm.S);
  const int64_t no = lay.no;
  double *Fo = reinterpret_cast<double *>(sm + lay.Fo);
  double *vno = reinterpret_cast<double *>(sm + lay.vno);
  double *vrefo = reinterpret_cast<double *>(sm + lay.vrefo);
  double *ajo = reinterpret_cast<double *>(sm + lay.ajo);
  double *svo = reinterpret_cast<double *>(sm + lay.svo);
  double *svs = reinterpret_cast<double *>(sm + lay.svs);
  int *flago = reinterpret_cast<int *>(sm + lay.flago);
  int *doneo = reinterpret_cast<int *>(sm + lay.doneo);
  using PT = PartT<AT>;  // entries of the partial vectors
  double *red = reinterpret_cast<double *>(sm + lay.red);
  double *Ts = reinterpret_cast<double *>(sm + lay.Ts);
  double *Vt = reinterpret_cast<double *>(sm + lay.Vt);
  double *Ms = reinterpret_cast<double *>(sm + lay.Ms);
  double *su = reinterpret_cast<double *>(sm + lay.su);
  double *Vs = reinterpret_cast<double *>(sm + lay.Vs);
  double *red4 = reinterpret_cast<double *>(sm + lay.red4);
  double *cscr = reinterpret_cast<double *>(sm + lay.cscr);
  float *nat = reinterpret_cast<float *>(sm + lay.nat);
  void *ys = sm + lay.ys;
  int *perm = reinterpret_cast<int *>(sm + lay.perm);
  int *posof = reinterpret_cast<int *>(sm + lay.posof);
  unsigned long long *cand = reinterpret_cast<unsigned long long *>(sm + lay.cand);
  AT *As = reinterpret_cast<AT *>(sm + lay.As);
  const int kp = lay.kp;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t r0 = min(m, (int64_t)blockIdx.x * a.rows_per), r1 = min(m, r0 + a.rows_per);
  const int64_t nrows = r1 - r0, ncache = min(nrows, a.rows_cached);
  const AT *A = static_cast<const AT *>(a.A);
  int par = 0;

  // ---- set-up: this block's cached rows of A (asynchronous copies, all in flight at
  //      once), identity column order, zero T, V corner and column flags
  if (sizeof(AT) == 4 && a.vec4) {
    const int64_t n4 = n / 4;
    for (int64_t li = 0; li < ncache; ++li)
      for (int64_t c4 = tid; c4 < n4; c4 += kCT) cp_async16(As + li * n + 4 * c4, A + (r0 + li) * a.lda + 4 * c4);
  } else {
    for (int64_t li = 0; li < ncache; ++li)
      for (int64_t c = tid; c < n; c += kCT) cp_async_elem(As + li * n + c, A + (r0 + li) * a.lda + c);
  }
  for (int64_t c = tid; c < n; c += kCT) {
    perm[c] = (int)c;
    posof[c] = (int)c;
  }
  for (int lc = tid; lc < tm.nown; lc += kCT) {
    flago[lc] = 0;
    doneo[lc] = 0;
  }
  for (int q = tid; q < k * k; q += kCT) {
    Ts[q] = 0.0;
    Vt[q] = 0.0;
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  __syncthreads();

  // ---- initial column norms and the first pivot
  if (a.colsq) {  // given by the caller: no pass over A, no reduction
    if (tid < kColT) nat_from_colsq<kColT>(a, nat);
    for (int lc = tid; lc < tm.nown; lc += kCT) {
      const double v = a.colsq[QX(tm.rank + tm.S * lc, n, 8)];
      vno[lc] = v;
      vrefo[lc] = v;
    }
    __syncthreads();
    choose_pivot(cl, tm, 0, n, vno, flago, doneo, perm, posof, cand, &s_res);
  } else {
    PT *rp = reinterpret_cast<PT *>(red) + (size_t)par * L;
    if (tid < kColT)  // the layout of the A^T y passes, which use the norm bounds it leaves in nat
      ccolsum<AT, true, kColT>(a, As, ncache, r0, 0, nrows, ys, cscr, nat, rp);
    for (int q = (int)n + tid; q < L; q += kCT) rp[q] = Part<PT>::zero();
    __syncthreads();
    if (!allreduce(a, cl, tm, rp, svo, svs, par, &s_ok, reinterpret_cast<PT *>(red4))) return cbail(a);
    par ^= 1;
    for (int lc = tid; lc < tm.nown; lc += kCT) {
      vno[lc] = svo[lc];
      vrefo[lc] = svo[lc];
    }
    __syncthreads();
    choose_pivot(cl, tm, 0, n, vno, flago, doneo, perm, posof, cand, &s_res);
  }

  const double tol = sqrt(DBL_EPSILON);
  for (int j = 0; j < k; ++j) {
    const int c0 = (int)QX(perm[j], n, 9);
    const bool owner = j >= r0 && j < r1;
    if (tid < j) {  // F[c0, :j] from the block that owns column c0
      const double *pF = cl.map_shared_rank(Fo, (unsigned)QX(c0 % (int)tm.S, tm.S, 10));
      s_f[QX(tid, 64, 11)] = pF[QX((int64_t)tid * no + c0 / (int)tm.S, (int64_t)k * no, 12)];
    }
    for (int lc = tid; lc < tm.nown; lc += kCT)  // A[j, :] of this block's columns, used after the reduction
      ajo[QX(lc, no, 13)] = (double)__ldg(A + QX((int64_t)j * a.lda + tm.rank + (int64_t)tm.S * lc, m * a.lda, 14));
    __syncthreads();
    // ---- rows: y = A[:, c0] - V[:, :j] F[c0, :j]^T (zero above row j)
    double s2 = 0.0;
    for (int64_t li = tid; li < nrows; li += kCT) {
      const int64_t i = r0 + li;
      double *vr = Vs + QX(li * kp, a.rows_per * kp, 15);
      if (i < j) {
        vr[QX(j, kp, 16)] = 0.0;
        if constexpr (sizeof(AT) == 4)
          reinterpret_cast<float2 *>(a.Q)[QX(i * a.ldq + j, m * a.ldq, 17)] = make_float2(0.f, 0.f);
        continue;
      }
      double y = li < ncache ? (double)As[QX(li * n + c0, a.rows_cached * n, 18)]
                             : (double)__ldg(A + QX(i * a.lda + c0, m * a.lda, 19));
      for (int l = 0; l < j; ++l) y = fma(-vr[l], s_f[l], y);
      vr[QX(j, kp, 16)] = y;
      s2 = fma(y, y, s2);
      if constexpr (sizeof(AT) == 4) {
        const float h = (float)y;
        const float2 yp = make_float2(h, (float)(y - (double)h));
        static_cast<float2 *>(ys)[QX(li, a.rows_per, 20)] = yp;
        reinterpret_cast<float2 *>(a.Q)[QX(i * a.ldq + j, m * a.ldq, 17)] = yp;  // V[i, j] as a pair, for the Q formation
      } else {
        static_cast<double *>(ys)[QX(li, a.rows_per, 20)] = y;
      }
    }
    PT *rp = reinterpret_cast<PT *>(red) + (size_t)par * L;
    red4[tid] = s2;
    __syncthreads();
    if (tid < kColT) {
      // A^T y over this block's rows from row j on (FP32 pipe)
      ccolsum<AT, false, kColT>(a, As, ncache, r0, max((int64_t)0, (int64_t)j - r0), nrows, ys, cscr, nat, rp);
    } else {
      // meanwhile, on the FP64 pipe: V^T y over this block's rows below row j (j < 32), lanes =
      // (row group g, column l) with the group width P the power of two >= j; ||y||^2; row j of V
      const int aw = warp - kColT / 32, at = tid - kColT;  // auxiliary warp 0 .. kAuxT/32 - 1
      constexpr int kAuxW = kAuxT / 32;
      if (j > 0) {
        const int P = j <= 1 ? 1 : j <= 2 ? 2 : j <= 4 ? 4 : j <= 8 ? 8 : j <= 16 ? 16 : 32;
        const int G = 32 / P, g = lane / P, l = lane % P;
        double u = 0.0;
        const int64_t lo = max((int64_t)0, (int64_t)j + 1 - r0);
        for (int64_t li = lo + (int64_t)aw * G + g; li < nrows; li += (int64_t)kAuxW * G) {
          const double *vr = Vs + QX(li * kp, a.rows_per * kp, 21);
          if (l < j) u = fma(vr[l], vr[j], u);
        }
        for (int o = P; o < 32; o <<= 1) u += __shfl_xor_sync(0xffffffffu, u, o);
        if (g == 0) red4[QX(kCT + aw * 32 + l, 2 * kCT, 22)] = u;  // [0, kCT) holds the ||y||^2 partials
      }
      // ||y||^2: a tree over each thread's kCT / kAuxT partials, then over the lanes and warps
      double x[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) x[q] = (q < kCT / kAuxT) ? red4[q * kAuxT + at] : 0.0;
      double s = tree16(x);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) red4[kCT + 64 + aw] = s;
      asm volatile("bar.sync 2, %0;\n" ::"r"(kAuxT) : "memory");
      if (at == 0) {
        double tt = red4[kCT + 64];
        for (int w2 = 1; w2 < kAuxW; ++w2) tt += red4[kCT + 64 + w2];
        rp[QX(n + k, L, 23)] = Part<PT>::of(tt);
        rp[QX(n + k + 1, L, 23)] = Part<PT>::of(owner ? Vs[QX((j - r0) * kp + j, a.rows_per * kp, 24)] : 0.0);
      }
      for (int q = at; q < k; q += kAuxT) {
        double tt = 0.0;
        if (q < j) {
          tt = red4[kCT + q];
          for (int w2 = 1; w2 < kAuxW; ++w2) tt += red4[kCT + w2 * 32 + q];
        }
        rp[QX(n + q, L, 23)] = Part<PT>::of(tt);
        rp[QX(n + k + 2 + q, L, 23)] = Part<PT>::of((owner && q < j) ? Vs[QX((j - r0) * kp + q, a.rows_per * kp, 24)] : 0.0);
      }
    }
    __syncthreads();
    if (!allreduce(a, cl, tm, rp, svo, svs, par, &s_ok, reinterpret_cast<PT *>(red4))) return cbail(a);
    par ^= 1;

    // ---- reflector (thread 0) while the column threads form the dot products that do not
    //      depend on it: with u_l = s_l + V[j, l] v_jj (s_l = sum below row j),
    //      F[c, :j] u = F[c, :j] s + v_jj (F[c, :j] V[j, :j]^T)
    if (tid == 0) {
      const double x0 = svs[k + 1];
      const double alpha = sqrt(svs[k]);
      double tau = 0.0, beta = 0.0, v0 = 0.0;
      if (alpha > 0.0) {
        const double sg = (x0 < 0.0) ? -1.0 : 1.0;
        v0 = x0 + sg * alpha;
        tau = 2.0 / (2.0 * alpha * (alpha + fabs(x0)));
        beta = -sg * alpha;
      }
      s_sc[0] = v0;
      s_sc[1] = tau;
      s_sc[2] = v0 - x0;
      Vt[QX(j * k + j, k * k, 25)] = v0;
      if (owner) {
        Vs[QX((j - r0) * kp + j, a.rows_per * kp, 24)] = v0;
        if constexpr (sizeof(AT) == 4) reinterpret_cast<float2 *>(a.Q)[QX((int64_t)j * a.ldq + j, m * a.ldq, 17)] = df2_of(v0);
      }
      if (blockIdx.x == 0) {
        if (a.rdiag) a.rdiag[j] = beta;
        if (a.piv) a.piv[j] = c0;
      }
    }
    const int lc = tid - 64;  // warps 2..: this block's columns (at most kCT - 64 of them)
    const bool colt = lc >= 0 && lc < tm.nown && !doneo[lc];
    double cs0 = 0.0, cs1 = 0.0, cv0 = 0.0, cv1 = 0.0;
    if (colt) {
      int l = 0;
      for (; l + 1 < j; l += 2) {  // two independent chains each
        const double f0 = Fo[QX((int64_t)l * no + lc, (int64_t)k * no, 26)], f1 = Fo[QX((int64_t)(l + 1) * no + lc, (int64_t)k * no, 26)];
        cs0 = fma(f0, svs[l], cs0);
        cs1 = fma(f1, svs[l + 1], cs1);
        cv0 = fma(svs[QX(k + 2 + l, 2 * k + 2, 27)], f0, cv0);
        cv1 = fma(svs[QX(k + 2 + l + 1, 2 * k + 2, 27)], f1, cv1);
      }
      if (l < j) {
        const double f0 = Fo[(int64_t)l * no + lc];
        cs0 = fma(f0, svs[l], cs0);
        cv0 = fma(svs[k + 2 + l], f0, cv0);
      }
    }
    __syncthreads();
    const double v0 = s_sc[0], tau = s_sc[1], dv = s_sc[2];
    if (tid < j) {
      const double vj = svs[k + 2 + tid];
      Vt[j * k + tid] = vj;
      su[tid] = fma(vj, v0, svs[tid]);  // V[:, l]^T v_j = sum below row j + V[j, l] v_jj
    }
    __syncthreads();
    if (tid < j) {  // T(0:j, j) = -tau T(0:j, 0:j) u (two chains)
      double t0 = 0.0, t1 = 0.0;
      int q = tid;
      for (; q + 1 < j; q += 2) {
        t0 = fma(Ts[tid * k + q], su[q], t0);
        t1 = fma(Ts[tid * k + q + 1], su[q + 1], t1);
      }
      if (q < j) t0 = fma(Ts[tid * k + q], su[q], t0);
      Ts[tid * k + j] = -tau * (t0 + t1);
    }
    if (tid == 0) Ts[j * k + j] = tau;
    if (colt) {
      const double ajc = ajo[lc];
      const double w = fma(dv, ajc, svo[lc]);  // A^T v = A^T y + (v_jj - y_jj) A[j, :]
      const double rv = cv0 + cv1;             // F[c, :j] V[j, :j]^T
      const double corr = fma(v0, rv, cs0 + cs1);
      const double f = tau * (w - corr);
      Fo[QX((int64_t)j * no + lc, (int64_t)k * no, 26)] = f;
      double r = ajc - rv;
      r = fma(-v0, f, r);
      double nv = vno[lc] - r * r;
      const double ref = vrefo[lc];
      if (ref > 0.0 && !(nv > tol * ref)) {
        flago[lc] = 1;
        nv = 0.0;
      } else if (!(nv > 0.0)) {
        nv = 0.0;
      }
      vno[lc] = nv;
    }
    __syncthreads();
    if (j + 1 < k && choose_pivot(cl, tm, j + 1, n, vno, flago, doneo, perm, posof, cand, &s_res)) {
      // exact norms of the flagged columns of the whole cluster (rare)
      PT *rq = reinterpret_cast<PT *>(red) + (size_t)par * L;
      for (int q = tid; q < L; q += kCT) rq[q] = Part<PT>::zero();
      __syncthreads();
      for (unsigned q = 0; q < tm.S; ++q) {
        const int *pf = cl.map_shared_rank(flago, (unsigned)QX(q, tm.S, 28));
        const double *pF = cl.map_shared_rank(Fo, (unsigned)QX(q, tm.S, 28));
        const int nq = (int)((n - (int64_t)q + tm.S - 1) / tm.S);
        for (int lc = 0; lc < nq; ++lc) {
          if (!pf[QX(lc, no, 29)]) continue;
          const int64_t c = q + (int64_t)tm.S * lc;
          if (tid <= j) s_f[QX(tid, 64, 11)] = pF[QX((int64_t)tid * no + lc, (int64_t)k * no, 30)];
          __syncthreads();
          double t = 0.0;
          for (int64_t li = max((int64_t)0, (int64_t)j + 1 - r0) + tid; li < nrows; li += kCT) {
            double y = li < ncache ? (double)As[QX(li * n + c, a.rows_cached * n, 31)]
                                   : (double)__ldg(A + QX((r0 + li) * a.lda + c, m * a.lda, 32));
            const double *vr = Vs + QX(li * kp, a.rows_per * kp, 33);
            for (int l = 0; l <= j; ++l) y = fma(-vr[l], s_f[l], y);
            t = fma(y, y, t);
          }
          red4[tid] = t;
          __syncthreads();
          if (warp == 0) {
            double u = 0.0;
#pragma unroll
            for (int w = 0; w < kCW; ++w) u += red4[w * 32 + lane];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) u += __shfl_xor_sync(0xffffffffu, u, o);
            if (lane == 0) rq[QX(c, L, 34)] = Part<PT>::of(u);
          }
          __syncthreads();
        }
      }
      if (!allreduce(a, cl, tm, rq, svo, svs, par, &s_ok, reinterpret_cast<PT *>(red4))) return cbail(a);
      par ^= 1;
      for (int lc = tid; lc < tm.nown; lc += kCT) {
        if (flago[lc]) {
          vno[lc] = svo[lc];
          vrefo[lc] = svo[lc];
          flago[lc] = 0;
        }
      }
      __syncthreads();
      choose_pivot(cl, tm, j + 1, n, vno, flago, doneo, perm, posof, cand, &s_res);
    }
  }

  // ---- Q = [I_k; 0] - V (T V[0:k, :]^T) on this block's rows
  for (int q = tid; q < k * k; q += kCT) {
    const int l = q / k, cc = q % k;
    double t = 0.0;
    for (int p = l; p <= cc; ++p) t = fma(Ts[l * k + p], Vt[cc * k + p], t);
    Ms[q] = t;
  }
  __syncthreads();
  // FP32 A with many rows per block: the double-float formation below; with few (the
  // 1,000 x 256 unfolding: 63 rows per block) its set-up costs more than it saves, and the
  // FP64 formation from V's FP64 copy runs instead (2 us less measured there)
  bool df_q = false;
  if constexpr (sizeof(AT) == 4) df_q = a.rows_per >= kQfDfRows;
  if (df_q) {
    // FP32 A: V's entries were kept as double-float pairs in Q's slots during the steps;
    // they replace the FP64 copy in shared memory (no longer needed), M is split in place,
    // and each entry of Q is a double-float sum on the FP32 pipe (about 2^-47 relative),
    // converted to FP64 with one FP64 addition: 16 FP64 operations per row instead of
    // k^2 = 256 FMAs, on a pipe that issues one warp instruction per 16 cycles per SM.
    float2 *Vsf = reinterpret_cast<float2 *>(Vs);
    float2 *Mf = reinterpret_cast<float2 *>(Ms);
    const float2 *Qf = reinterpret_cast<const float2 *>(a.Q);
    const int64_t tot = nrows * k;
    for (int64_t b0 = tid; b0 < tot; b0 += 8 * kCT) {  // eight loads in flight per thread, then the stores
      float2 v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int64_t idx = b0 + (int64_t)u * kCT;
        if (idx < tot) v[u] = Qf[QX((r0 + idx / k) * a.ldq + idx % k, m * a.ldq, 35)];
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int64_t idx = b0 + (int64_t)u * kCT;
        if (idx < tot) Vsf[QX((idx / k) * kp + idx % k, a.rows_per * kp, 36)] = v[u];
      }
    }
    for (int q = tid; q < k * k; q += kCT) Mf[q] = df2_of(Ms[q]);  // each slot read, then rewritten, by one thread
    __syncthreads();
    for (int64_t idx = tid; idx < nrows * k; idx += kCT) {
      const int64_t li = idx / k, i = r0 + li;
      const int cc = (int)(idx % k);
      DF t;
      t.hi = (i == cc) ? 1.f : 0.f;
      t.lo = 0.f;
      const int lmax = (int)min((int64_t)k - 1, i);
      const float2 *vr = Vsf + QX(li * kp, a.rows_per * kp, 37);
      for (int l = 0; l <= lmax; ++l) df_sub_prod(t, vr[l], Mf[l * k + cc]);
      a.Q[QX(i * a.ldq + cc, m * a.ldq, 38)] = f2d_exact(t.hi) + f2d_exact(t.lo);
    }
  } else {
    for (int64_t idx = tid; idx < nrows * k; idx += kCT) {
      const int64_t li = idx / k, i = r0 + li;
      const int cc = (int)(idx % k);
      double t = (i == cc) ? 1.0 : 0.0;
      const int lmax = (int)min((int64_t)k - 1, i);
      const double *vr = Vs + QX(li * kp, a.rows_per * kp, 37);
      for (int l = 0; l <= lmax; ++l) t = fma(-vr[l], Ms[l * k + cc], t);
      a.Q[QX(i * a.ldq + cc, m * a.ldq, 38)] = t;
    }
  }
  qc_report(a.err);
  cl.sync();  // no block leaves while a peer may still read its shared memory
}

// ---- host side: per-device limits, cached
struct DevInfo {
  bool init = false;
  int smem_dyn = 0;          // dynamic shared memory one block may use
  int max_clusters[5] = {};  // for cluster sizes 16, 8, 4, 2, 1 (one block per SM)
  bool coop_cluster_ok = true;
};
constexpr int kSizes[5] = {16, 8, 4, 2, 1};
constexpr int kMaxDev = 64;
std::mutex g_mu;
DevInfo g_info[2][kMaxDev];  // [FP32 A, FP64 A]

template <typename AT>
bool dev_info(int dev, DevInfo **out) {
  if (dev < 0 || dev >= kMaxDev) return false;
  std::lock_guard<std::mutex> lock(g_mu);
  DevInfo &d = g_info[sizeof(AT) == 8][dev];
  if (!d.init) {
    int optin = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return false;
    auto kern = qrp_cluster_kernel<AT>;
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess) return false;
    const int dyn = optin - (int)fa.sharedSizeBytes;
    if (dyn <= 0) return false;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn) != cudaSuccess) return false;
    const bool big_ok = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess;
    cudaGetLastError();
    for (int si = 0; si < 5; ++si) {
      const int S = kSizes[si];
      d.max_clusters[si] = 0;
      if (S > 8 && !big_ok) continue;
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = (unsigned)S;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.gridDim = dim3((unsigned)S);
      cfg.blockDim = dim3(kCT);
      cfg.dynamicSmemBytes = (size_t)dyn;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int nc = 0;
      if (cudaOccupancyMaxActiveClusters(&nc, kern, &cfg) == cudaSuccess) d.max_clusters[si] = nc;
      cudaGetLastError();
    }
    d.smem_dyn = dyn;
    d.init = true;
  }
  *out = &d;
  return true;
}

const char *qrp_form_env() {
  const char *e = std::getenv("TUCKER_QRP_FORM");
  return e ? e : "";
}

}  // namespace

// Checked build: the first site whose index fell outside its array (0: none), read after
// synchronising the device; -1 in the normal build (no checks compiled in).
int32_t qrp_check_site() {
#ifdef TUCKER_QRP_CHECKED
  unsigned site = 0;
  if (cudaDeviceSynchronize() != cudaSuccess) return -2;
  if (cudaMemcpyFromSymbol(&site, g_qc_site, sizeof(site)) != cudaSuccess) return -2;
  return (int32_t)site;
#else
  return -1;
#endif
}

// Runs the cluster form when its shared-memory plan fits; false = not applicable
// (the caller runs another form).  *err reports a failed launch that was attempted.
template <typename AT>
bool qrp_cluster(const AT *A, int64_t m, int64_t n, int64_t lda, int k, double *Q, int64_t ldq, int64_t *piv,
                 double *rdiag, QrpWork *w, cudaStream_t s, cudaError_t *err) {
  *err = cudaSuccess;
  if (std::strcmp(qrp_form_env(), "persistent") == 0 || std::strcmp(qrp_form_env(), "multi") == 0) return false;
  if (k < 1 || k > 32 || m < 1 || n < 1 || n > (1 << 20)) return false;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  DevInfo *d = nullptr;
  if (!dev_info<AT>(dev, &d)) return false;
  const int L = (int)n + 2 * k + 2;
  const int es = (int)sizeof(AT);
  const size_t avail = (size_t)d->smem_dyn;
  int S = 0, C = 0;
  int64_t rows_per = 0, rows_cached = 0;
  auto need = [&](int s_, int64_t rp, int64_t rc) { return clayout(n, k, L, s_, rp, rc, es).total; };
  // a block's columns are handled by threads 64 .. kCT-1, one column each
  auto cols_fit = [&](int s_) { return (n + s_ - 1) / s_ <= (int64_t)(kCT - 64); };
  // one cluster holding all of A in shared memory: no grid-wide barrier
  for (int si = 0; si < 2 && !S; ++si) {
    if (d->max_clusters[si] < 1 || !cols_fit(kSizes[si])) continue;
    const int64_t rp = (m + kSizes[si] - 1) / kSizes[si];
    if (need(kSizes[si], rp, rp) <= avail) {
      S = kSizes[si];
      C = 1;
      rows_per = rows_cached = rp;
    }
  }
  if (!S) {
    if (!d->coop_cluster_ok) return false;
    // every block adds up C cluster sums per step: take the largest cluster size that
    // keeps at least 90% of the blocks that fit with any size
    int gmax = 0;
    for (int si = 1; si < 4; ++si) gmax = std::max(gmax, kSizes[si] * d->max_clusters[si]);
    if (gmax < 2) return false;
    for (int si = 1; si < 4 && !S; ++si) {
      if (10 * kSizes[si] * d->max_clusters[si] >= 9 * gmax && cols_fit(kSizes[si])) {
        S = kSizes[si];
        C = d->max_clusters[si];
      }
    }
    rows_per = (m + (int64_t)S * C - 1) / ((int64_t)S * C);
    const size_t base = need(S, rows_per, 0);
    if (base > avail) return false;
    rows_cached = std::min<int64_t>(rows_per, (int64_t)((avail - base) / ((size_t)n * es + 16)));
    while (rows_cached > 0 && need(S, rows_per, rows_cached) > avail) --rows_cached;
  }
  const size_t smem = need(S, rows_per, rows_cached);
  if (C > 1 && 2 * (size_t)C * L > w->part_elems) return false;  // the cluster sums live in `part`
  if ((int64_t)((C + 15) / 16) * ((n + S - 1) / S + 2 * k + 2) > 2 * kCT) return false;  // chunk sums: scratch

  CArgs a{};
  a.A = A;
  a.m = m;
  a.n = n;
  a.lda = lda;
  a.k = k;
  a.L = L;
  a.nclusters = C;
  a.cluster = S;
  // (the float4 column sums index a block's rows with 32-bit offsets)
  a.vec4 = (es == 4 && n % 4 == 0 && lda % 4 == 0 && (reinterpret_cast<uintptr_t>(A) % 16) == 0 &&
            rows_per * (lda / 4 + 1) < ((int64_t)1 << 31))
               ? 1
               : 0;
  a.rows_per = rows_per;
  a.rows_cached = rows_cached;
  a.slots = w->part;
  a.bar = w->bar;
  a.err = w->err_out ? w->err_out : w->bar + 2;
  a.Q = Q;
  a.ldq = ldq;
  a.piv = piv;
  a.rdiag = rdiag;
  a.colsq = (es == 4 && a.vec4) ? w->colsq : nullptr;
  if (C > 1 && (*err = cudaMemsetAsync(w->bar, 0, 3 * sizeof(unsigned), s)) != cudaSuccess) return true;

  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)S;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  int nat = 1;
  if (C > 1) {  // the clusters wait on one another: all of them must be resident
    at[1].id = cudaLaunchAttributeCooperative;
    at[1].val.cooperative = 1;
    nat = 2;
  }
  cfg.gridDim = dim3((unsigned)(S * C));
  cfg.blockDim = dim3(kCT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = at;
  cfg.numAttrs = nat;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, qrp_cluster_kernel<AT>, a);
  if (e != cudaSuccess) {
    cudaGetLastError();  // a configuration error is not sticky
    if (C > 1) {
      std::lock_guard<std::mutex> lock(g_mu);
      d->coop_cluster_ok = false;
    }
    return false;
  }
  ::tk::count_launch();
  return true;
}

template bool qrp_cluster<float>(const float *, int64_t, int64_t, int64_t, int, double *, int64_t, int64_t *,
                                 double *, QrpWork *, cudaStream_t, cudaError_t *);
template bool qrp_cluster<double>(const double *, int64_t, int64_t, int64_t, int, double *, int64_t, int64_t *,
                                  double *, QrpWork *, cudaStream_t, cudaError_t *);

}  // namespace tk
