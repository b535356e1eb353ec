// K-e: observed-entry loss of a Tucker model and its adjoint (the differentiation form
// of the sparse TTMc of Algorithm 2):
//     xhat_z = sum_r G[r] prod_m U_m(i_m(z), r_m),   e_z = xhat_z - x_z,   L = 1/2 sum_z e_z^2.
// With E the sparse tensor of residuals e_z at the observed coordinates,
//     dL/dU_n = TTMc_n(E) G_(n)^T          (TTMc_n as in Algorithm 2, values e_z)
//     dL/dG_(1) = U_1^T TTMc_1(E)          (the core-tensor contraction of Section III-B)
// and the forward pass needs only one row of Q = U_1 G_(1) per slice:
//     xhat_z = < Q(i_1(z), :), kron_{m > 1} U_m(i_m(z), :) >.
// So the adjoint is: one small dense product (Q), one pass over the nonzeros for the
// residuals and the loss, then for every mode a TTMc of the residuals (the kernel of
// ttmc.cu, fed with the caller's FP32 factors) and two small dense contractions.
// Kronecker rows are recomputed, never stored; every reduction has a fixed order.
#include <algorithm>

#include "internal.cuh"

namespace tk {

constexpr int kAdjRedBlocks = 304;  // fixed grid of the loss reduction (determinism)

// Q[i, c] = sum_r U1[i, r] G[r * P + c]    (U1: I x R1, G as R1 x P)
__global__ void adj_q_kernel(const float *U1, const float *G, int64_t I, int R1, int64_t P, float *Q) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < I * P;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / P, c = idx % P;
    float t = 0.f;
    for (int r = 0; r < R1; ++r) t = fmaf(U1[i * R1 + r], G[(int64_t)r * P + c], t);
    Q[idx] = t;
  }
}

struct AdjFwd {
  int N;
  int64_t Z;
  const uint32_t *coords;  // [N][Z] lexicographic
  const float *vals;
  const float *U[kMaxOrder];
  int R[kMaxOrder];
  const float *Q;
  int64_t P;  // P_1 = prod_{m >= 1} R_m
  float *e;
  double *part;
};

// One thread per nonzero (lexicographic order): xhat = <Q(i_1,:), kron_{m>1} U_m(i_m,:)>
// walked with an odometer over the Kronecker index (last mode fastest).
__global__ void __launch_bounds__(256) adj_forward_kernel(AdjFwd a) {
  __shared__ double red[256];
  double sq = 0.0;
  const int N = a.N;
  for (int64_t z = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; z < a.Z; z += (int64_t)gridDim.x * blockDim.x) {
    const float *q = a.Q + (int64_t)a.coords[z] * a.P;
    const float *row[kMaxOrder];
    for (int m = 1; m < N; ++m) row[m] = a.U[m] + (int64_t)a.coords[(int64_t)m * a.Z + z] * a.R[m];
    float xhat = 0.f;
    if (N == 2) {
      for (int r = 0; r < a.R[1]; ++r) xhat = fmaf(q[r], row[1][r], xhat);
    } else {
      int r[kMaxOrder];
      float pref[kMaxOrder + 1];
      for (int m = 1; m < N; ++m) r[m] = 0;
      pref[1] = 1.f;
      for (int m = 1; m < N - 1; ++m) pref[m + 1] = pref[m] * row[m][0];
      const int Rl = a.R[N - 1];
      const float *rl = row[N - 1];
      for (int64_t c0 = 0; c0 < a.P; c0 += Rl) {
        const float pp = pref[N - 1];
        float t = 0.f;
        for (int x = 0; x < Rl; ++x) t = fmaf(q[c0 + x], rl[x], t);
        xhat = fmaf(pp, t, xhat);
        // advance modes N-2 .. 1
        int m = N - 2;
        while (m >= 1) {
          if (++r[m] < a.R[m]) break;
          r[m] = 0;
          --m;
        }
        if (m < 1) break;
        for (int t2 = m; t2 < N - 1; ++t2) pref[t2 + 1] = pref[t2] * row[t2][r[t2]];
      }
    }
    const float e = xhat - a.vals[z];
    a.e[z] = e;
    sq = fma((double)e, (double)e, sq);
  }
  red[threadIdx.x] = sq;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) a.part[blockIdx.x] = red[0];
}

__global__ void adj_loss_kernel(const double *part, int np, double *loss) {
  __shared__ double red[256];
  double t = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) t += part[i];
  red[threadIdx.x] = t;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = 0.5 * red[0];
}

__global__ void adj_gather_kernel(int64_t Z, const uint32_t *src, const float *e0, float *en) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < Z; p += (int64_t)gridDim.x * blockDim.x)
    en[p] = e0[src[p]];
}

struct Unfold {
  int N, n;
  int R[kMaxOrder];
};

// Gn[r_n, c] = G[r_1, ..., r_N] with c the remaining indices in ascending mode order,
// last fastest (the column order of Y_(n)).
__global__ void adj_unfold_kernel(Unfold u, const float *G, int64_t PR, float *Gn) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < PR; idx += (int64_t)gridDim.x * blockDim.x) {
    // decode the C-order index of G
    int64_t t = idx;
    int r[kMaxOrder];
    for (int m = u.N - 1; m >= 0; --m) {
      r[m] = (int)(t % u.R[m]);
      t /= u.R[m];
    }
    int64_t c = 0;
    for (int m = 0; m < u.N; ++m)
      if (m != u.n) c = c * u.R[m] + r[m];
    const int64_t P = PR / u.R[u.n];
    Gn[(int64_t)r[u.n] * P + c] = G[idx];
  }
}

// dU[i, r] = sum_c Y[i, c] Gn[r, c]
__global__ void adj_du_kernel(const float *Y, const float *Gn, int64_t I, int64_t P, int R, float *dU) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < I * R;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / R;
    const int r = (int)(idx % R);
    const float *y = Y + i * P;
    const float *g = Gn + (int64_t)r * P;
    float t = 0.f;
    for (int64_t c = 0; c < P; ++c) t = fmaf(y[c], g[c], t);
    dU[idx] = t;
  }
}

// split-K partials of dG[r, c] = sum_i U1[i, r] Y[i, c]  (outputs r*P + c)
__global__ void adj_dg_partial_kernel(const float *U1, const float *Y, int64_t I, int R, int64_t P, int rows_per,
                                      float *gpart) {
  const int64_t out = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (out >= (int64_t)R * P) return;
  const int r = (int)(out / P);
  const int64_t c = out % P;
  const int64_t i0 = (int64_t)blockIdx.y * rows_per, i1 = std::min<int64_t>(I, i0 + rows_per);
  float t = 0.f;
  for (int64_t i = i0; i < i1; ++i) t = fmaf(U1[i * R + r], Y[i * P + c], t);
  gpart[(int64_t)blockIdx.y * R * P + out] = t;
}

__global__ void adj_dg_reduce_kernel(const float *gpart, int chunks, int64_t RP, float *dG) {
  for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < RP; o += (int64_t)gridDim.x * blockDim.x) {
    float t = 0.f;
    for (int q = 0; q < chunks; ++q) t += gpart[(int64_t)q * RP + o];
    dG[o] = t;
  }
}

static unsigned blocks_for(int64_t n, int64_t cap = 65535LL * 8) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, cap));
}

tucker_status launch_loss_grad(Ctx *c, const float *const *U, const float *G, double *loss, float *const *dU,
                               float *dG, cudaStream_t s) {
  const int N = c->N;
  const int64_t Z = c->nnz;
  int64_t PR = 1, ymax = 1;
  for (int m = 0; m < N; ++m) PR *= c->ranks[m];
  for (int m = 0; m < N; ++m) ymax = std::max(ymax, c->mode[m].I * c->mode[m].P);
  const int64_t I1 = c->dims[0], P1 = c->mode[0].P;
  const int R1 = c->ranks[0];
  const int chunks = (int)std::max<int64_t>(1, std::min<int64_t>(64, (I1 + 255) / 256));
  if (!c->adj_e0) {  // first call: buffers allocated in the order of s, ready for any stream after the sync
    c->astream = s;
    TK_CUDA(dev_alloc(c, &c->adj_e0, (size_t)std::max<int64_t>(Z, 1)));
    TK_CUDA(dev_alloc(c, &c->adj_en, (size_t)std::max<int64_t>(Z, 1)));
    TK_CUDA(dev_alloc(c, &c->adj_Y, (size_t)ymax));
    TK_CUDA(dev_alloc(c, &c->adj_Q, (size_t)(I1 * P1)));
    TK_CUDA(dev_alloc(c, &c->adj_Gn, (size_t)PR));
    TK_CUDA(dev_alloc(c, &c->adj_part, (size_t)kAdjRedBlocks));
    TK_CUDA(dev_alloc(c, &c->adj_gpart, (size_t)(64 * PR)));
    TK_CUDA(cudaStreamSynchronize(s));
    c->astream = 0;
  }
  // (1) Q = U_1 G_(1)
  adj_q_kernel<<<blocks_for(I1 * P1), 256, 0, s>>>(U[0], G, I1, R1, P1, c->adj_Q);
  ::tk::count_launch();
  // (2) residuals and the loss
  AdjFwd f{};
  f.N = N;
  f.Z = Z;
  f.coords = c->coords;
  f.vals = c->vals;
  for (int m = 0; m < N; ++m) {
    f.U[m] = U[m];
    f.R[m] = c->ranks[m];
  }
  f.Q = c->adj_Q;
  f.P = P1;
  f.e = c->adj_e0;
  f.part = c->adj_part;
  adj_forward_kernel<<<kAdjRedBlocks, 256, 0, s>>>(f);
  ::tk::count_launch();
  adj_loss_kernel<<<1, 256, 0, s>>>(c->adj_part, kAdjRedBlocks, loss);
  ::tk::count_launch();
  // (3) per mode: TTMc of the residuals, then dU_n and (mode 1) dG
  for (int n = 0; n < N; ++n) {
    const ModeCopy &mc = c->mode[n];
    const float *en = c->adj_e0;
    if (mc.src && Z > 0) {  // this mode's order is not the lexicographic one
      adj_gather_kernel<<<blocks_for(Z, 4096), 256, 0, s>>>(Z, mc.src, c->adj_e0, c->adj_en);
      ::tk::count_launch();
      en = c->adj_en;
    }
    tucker_status st = launch_ttmc_ex(c, n, c->adj_Y, en, U, s);
    if (st != TUCKER_OK) return st;
    Unfold uf{};
    uf.N = N;
    uf.n = n;
    for (int m = 0; m < N; ++m) uf.R[m] = c->ranks[m];
    adj_unfold_kernel<<<blocks_for(PR), 256, 0, s>>>(uf, G, PR, c->adj_Gn);
    ::tk::count_launch();
    adj_du_kernel<<<blocks_for(mc.I * c->ranks[n]), 256, 0, s>>>(c->adj_Y, c->adj_Gn, mc.I, mc.P, c->ranks[n], dU[n]);
    ::tk::count_launch();
    if (n == 0) {
      const int rows_per = (int)((I1 + chunks - 1) / chunks);
      adj_dg_partial_kernel<<<dim3((unsigned)((R1 * P1 + 255) / 256), (unsigned)chunks), 256, 0, s>>>(
          U[0], c->adj_Y, I1, R1, P1, rows_per, c->adj_gpart);
      ::tk::count_launch();
      adj_dg_reduce_kernel<<<blocks_for(PR), 256, 0, s>>>(c->adj_gpart, chunks, PR, dG);
      ::tk::count_launch();
    }
  }
  TK_CUDA(cudaGetLastError());
  return TUCKER_OK;
}

}  // namespace tk
