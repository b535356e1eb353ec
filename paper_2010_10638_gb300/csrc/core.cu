// K-d: core tensor of one HOOI sweep and the fit (Section III-B, eqs. ttm_ele and
// core_unfolded:  G_(N) = U_N^T Y_(N),  G[c, r] = sum_i U_N(i, r) Y_(N)(i, c)).
// Y_(N) is the FP32 TTMc output of the last mode (I_N x P), U_N the FP64 factor
// (I_N x R).  Split over rows of Y into chunks; each block owns a 16 x 16 tile of
// (column c, rank r) outputs for one row chunk and accumulates in FP64; the last
// block to finish sums the chunk partials in chunk order, writes G (C-order, r
// fastest), ||G||^2 and fit = 1 - sqrt(max(0, ||X||^2 - ||G||^2)) / ||X||.
#include <algorithm>

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

void launch_core(Ctx *c, const float *Y, const double *U, double *G, cudaStream_t s) {
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
