// Adjoint of the assembly (gradients).  For a scalar L of the spectrum with
// dL = tr(Gamma dH) (Gamma Hermitian: x x^dagger for an exciton energy by Hellmann-Feynman),
//   dL/dW(q)_mu,nu = -(1/N_k) sum_k1 sum_ijab Gamma_(k2,j,b),(k1,i,a) M_vv(k1,q)^mu_ij M_cc(k1,q)^nu_ab
// (the direct term of Eq. W_LRI is the only place W enters), then the adjoint of
// W(q) = sum_R w_R W(R) e^{-i q.R} gives dL/dW_mu,nu(R) = w_R Re sum_q e^{-i q.R} dL/dW(q)_mu,nu,
// and the E_c - E_v diagonal (Eq. Hamiltonian) gives dL/dE^QP.  The pair projections are
// recomputed one q-slab at a time, never stored for all pairs; everything is FP64 for an FP64
// context.  A split-precision context runs the slab loop from its FP32 pair table with FP32
// sums (k_split.cu:split_adjoint_slabs; its error is the split forward's own) and the same
// FP64 Fourier adjoint and diagonal.
#include <algorithm>

#include "bse_internal.cuh"

namespace {

__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

constexpr int PCH = 64;  // nu chunk

// U[qq][k1][i][j][nu] = sum_ab Gamma[(k2,j,b),(k1,i,a)] M_cc[qq][k1][a][b][nu]
__global__ void __launch_bounds__(256) k_adj_phi_mc(const double2 *__restrict__ Gamma, const double2 *__restrict__ Mc,
                                                    int nv, int nc, int naux, int n1, int n2, int n3, int q0,
                                                    const int *__restrict__ qlist, long long dim,
                                                    double2 *__restrict__ U) {
  extern __shared__ double2 sa[];
  const int nk = n1 * n2 * n3;
  const int k1 = blockIdx.x, qq = blockIdx.y, q = qlist[q0 + qq];
  const int k2 = kdiff(k1, q, n1, n2, n3);
  const int nvv = nv * nv, ncc = nc * nc, nvc = nv * nc;
  double2 *phi = sa;                 // [nvv][ncc]
  double2 *mcs = sa + nvv * ncc;     // [ncc][PCH]
  for (int e = threadIdx.x; e < nvv * ncc; e += blockDim.x) {
    const int ij = e / ncc, ab = e % ncc;
    const int i = ij / nv, j = ij % nv, a = ab / nc, b = ab % nc;
    phi[e] = Gamma[((long long)k2 * nvc + j * nc + b) * dim + (long long)k1 * nvc + i * nc + a];
  }
  const double2 *Mk = Mc + ((long long)qq * nk + k1) * ncc * naux;
  double2 *Uk = U + ((long long)qq * nk + k1) * nvv * naux;
  for (int n0 = 0; n0 < naux; n0 += PCH) {
    const int nn = min(PCH, naux - n0);
    __syncthreads();
    for (int e = threadIdx.x; e < ncc * PCH; e += blockDim.x) {
      const int ab = e / PCH, u = e % PCH;
      mcs[e] = u < nn ? Mk[(long long)ab * naux + n0 + u] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nvv * PCH; e += blockDim.x) {
      const int ij = e / PCH, u = e % PCH;
      if (u >= nn) continue;
      double2 acc = make_double2(0.0, 0.0);
      for (int ab = 0; ab < ncc; ab++) {
        const double2 t = zmul(phi[ij * ncc + ab], mcs[ab * PCH + u]);
        acc.x += t.x;
        acc.y += t.y;
      }
      Uk[(long long)ij * naux + n0 + u] = acc;
    }
  }
}

// C[qlist[q0+b]] (C[b] when qlist is null) = alpha A[b]^T B[b]: A, B row-major [K x M],
// [K x N]; C [M x N].
__global__ void __launch_bounds__(256) k_zgemm_tn(int M, int N, int K, const double2 *__restrict__ A, long long sA,
                                                  const double2 *__restrict__ B, long long sB, double2 *__restrict__ C,
                                                  long long sC, const int *__restrict__ cidx, int q0, double alpha) {
  __shared__ double2 As[16][64];
  __shared__ double2 Bs[16][64];
  const int bz = blockIdx.z;
  A += bz * sA;
  B += bz * sB;
  C += (long long)(cidx ? cidx[q0 + bz] : bz) * sC;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int row0 = blockIdx.y * 64, col0 = blockIdx.x * 64;
  double2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; i++)
#pragma unroll
    for (int j = 0; j < 4; j++) acc[i][j] = make_double2(0, 0);
  for (int k0 = 0; k0 < K; k0 += 16) {
    for (int e = threadIdx.x; e < 1024; e += 256) {
      const int kk = e / 64, r = e % 64, gk = k0 + kk;
      As[kk][r] = (gk < K && row0 + r < M) ? A[(long long)gk * M + row0 + r] : make_double2(0, 0);
      Bs[kk][r] = (gk < K && col0 + r < N) ? B[(long long)gk * N + col0 + r] : make_double2(0, 0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; kk++) {
      double2 a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; i++) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; j++) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) {
          acc[i][j].x = fma(a[i].x, b[j].x, fma(-a[i].y, b[j].y, acc[i][j].x));
          acc[i][j].y = fma(a[i].x, b[j].y, fma(a[i].y, b[j].x, acc[i][j].y));
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; i++)
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const int r = row0 + ty + 16 * i, cc = col0 + tx + 16 * j;
      if (r < M && cc < N) C[(long long)r * N + cc] = make_double2(alpha * acc[i][j].x, alpha * acc[i][j].y);
    }
}

constexpr int FTR = 4, FTQ = 256;

// dW[r][e] = w_r Re sum_q e^{-2 pi i q.R_r} A[q][e]
__global__ void k_adj_ft(const double2 *__restrict__ Aq, const int *__restrict__ RW, const double *__restrict__ wRW,
                         int nRW, long long nn, int n1, int n2, int n3, double *__restrict__ dW) {
  __shared__ double2 ph[FTR][FTQ];
  const int nk = n1 * n2 * n3;
  const int r0 = blockIdx.y * FTR;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double acc[FTR] = {0.0, 0.0, 0.0, 0.0};
  for (int qb = 0; qb < nk; qb += FTQ) {
    __syncthreads();
    for (int t = threadIdx.x; t < FTR * FTQ; t += blockDim.x) {
      const int rr = t / FTQ, qq = t % FTQ, r = r0 + rr, q = qb + qq;
      double2 v = make_double2(0.0, 0.0);
      if (r < nRW && q < nk) {
        const int m1 = q / (n2 * n3), m2 = (q / n3) % n2, m3 = q % n3;
        long long p = (long long)m1 * RW[3 * r] * n2 * n3 + (long long)m2 * RW[3 * r + 1] * n1 * n3 +
                      (long long)m3 * RW[3 * r + 2] * n1 * n2;
        p %= nk;
        if (p < 0) p += nk;
        double s, c;
        sincospi(2.0 * (double)p / (double)nk, &s, &c);
        v = make_double2(c, -s);
      }
      ph[rr][qq] = v;
    }
    __syncthreads();
    if (e < nn) {
      const int qn = min(FTQ, nk - qb);
      for (int qq = 0; qq < qn; qq++) {
        const double2 a = Aq[(long long)(qb + qq) * nn + e];
#pragma unroll
        for (int rr = 0; rr < FTR; rr++) acc[rr] += ph[rr][qq].x * a.x - ph[rr][qq].y * a.y;
      }
    }
  }
  if (e < nn)
#pragma unroll
    for (int rr = 0; rr < FTR; rr++)
      if (r0 + rr < nRW) dW[(long long)(r0 + rr) * nn + e] = wRW[r0 + rr] * acc[rr];
}

// de[k][n] from the diagonal of Gamma.  Valence n at k enters the pairs at k; conduction n
// at k enters the pairs at k - Q (= kdiff(k, qQ)), whose conduction point is k.
__global__ void k_adj_diag(const double2 *__restrict__ Gamma, long long dim, int n1, int n2, int n3, int qQ,
                           int nv, int nc, double *__restrict__ de) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int nb = nv + nc, nk = n1 * n2 * n3;
  if (t >= nk * nb) return;
  const int k = t / nb, n = t % nb;
  const int kp = n < nv ? k : kdiff(k, qQ, n1, n2, n3);
  double s = 0.0;
  if (n < nv) {
    for (int a = 0; a < nc; a++) {
      const long long r = ((long long)k * nv + n) * nc + a;
      s -= Gamma[r * dim + r].x;
    }
  } else {
    for (int i = 0; i < nv; i++) {
      const long long r = ((long long)kp * nv + i) * nc + (n - nv);
      s += Gamma[r * dim + r].x;
    }
  }
  de[t] = s;
}

// Gamma = sum_s g_s x_s x_s^dagger
__global__ void k_seed_lowrank(const double2 *__restrict__ X, const double *__restrict__ g, int r, long long dim,
                               double2 *__restrict__ Gamma) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= dim * dim) return;
  const long long row = e / dim, col = e % dim;
  double2 acc = make_double2(0.0, 0.0);
  for (int s = 0; s < r; s++) {
    const double2 a = X[(long long)s * dim + row], b = X[(long long)s * dim + col];
    acc.x += g[s] * (a.x * b.x + a.y * b.y);
    acc.y += g[s] * (a.y * b.x - a.x * b.y);
  }
  Gamma[e] = acc;
}

}  // namespace

bse_status adjoint_workspace(bse_ctx *c) {
  if (!c->Aq) {
    if (cudaMalloc((void **)&c->Aq, sizeof(double2) * (size_t)c->nk * c->naux_tot * c->naux_tot) != cudaSuccess) {
      cudaGetLastError();
      c->Aq = nullptr;
      return bse_fail(c, BSE_ENOMEM, "adjoint: workspace allocation failed");
    }
  }
  if (!c->Mv && c->precision == BSE_FP64) {  // the split precisions use their own slab buffers
    const size_t per_q = (size_t)c->nk * (2 * c->nv * c->nv + c->nc * c->nc) * c->naux_tot * sizeof(double2);
    const size_t budget = (size_t)768 << 20;
    c->slab = (int)std::max<size_t>(1, std::min<size_t>((size_t)c->nk, budget / std::max<size_t>(per_q, 1)));
    c->slab = std::min(c->slab, 65535);
    const size_t nvv = (size_t)c->slab * c->nk * c->nv * c->nv * c->naux_tot;
    const size_t ncc = (size_t)c->slab * c->nk * c->nc * c->nc * c->naux_tot;
    if (cudaMalloc((void **)&c->Mv, sizeof(double2) * nvv) != cudaSuccess ||
        cudaMalloc((void **)&c->T, sizeof(double2) * nvv) != cudaSuccess ||
        cudaMalloc((void **)&c->Mc, sizeof(double2) * ncc) != cudaSuccess) {
      cudaGetLastError();
      return bse_fail(c, BSE_ENOMEM, "adjoint: slab allocation failed");
    }
  }
  return BSE_OK;
}

bse_status run_adjoint(bse_ctx *c, const double2 *Gamma, double *dW_R, double *de_qp) {
  bse_status s = adjoint_workspace(c);
  if (s != BSE_OK) return s;
  const int na = c->naux_tot;
  const long long rows = (long long)c->nk * c->nv * c->nv;
  if (c->precision != BSE_FP64) {  // the split precisions: FP32 slabs from their pair table
    s = split_adjoint_slabs(c, Gamma);
    if (s != BSE_OK) return s;
  }
  for (int q0 = 0; c->precision == BSE_FP64 && q0 < c->nk; q0 += c->slab) {
    const int nq = std::min(c->slab, c->nk - q0);
    s = launch_project_slab_fp64(c, q0, nq, c->d_qall);
    if (s != BSE_OK) return s;
    const size_t sm = sizeof(double2) * (c->nv * c->nv * c->nc * c->nc + c->nc * c->nc * PCH);
    if (sm > 48 * 1024) cudaFuncSetAttribute(k_adj_phi_mc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_adj_phi_mc<<<dim3(c->nk, nq), 256, sm, c->stream>>>(Gamma, c->Mc, c->nv, c->nc, na, c->mesh[0], c->mesh[1],
                                                          c->mesh[2], q0, c->d_qall, c->dim, c->T);
    dim3 grid((na + 63) / 64, (na + 63) / 64, nq);
    k_zgemm_tn<<<grid, 256, 0, c->stream>>>(na, na, (int)rows, c->Mv, rows * na, c->T, rows * na, c->Aq,
                                            (long long)na * na, c->d_qall, q0, -1.0 / c->nk);
    bse_count_launch(2);
    s = bse_check_launch(c, "adjoint slab");
    if (s != BSE_OK) return s;
  }
  const long long nn = (long long)na * na;
  k_adj_ft<<<dim3((unsigned)((nn + 255) / 256), (c->n_RW + FTR - 1) / FTR), 256, 0, c->stream>>>(
      c->Aq, c->d_R_W, c->d_w_RW, c->n_RW, nn, c->mesh[0], c->mesh[1], c->mesh[2], dW_R);
  k_adj_diag<<<(c->nk * c->nb + 255) / 256, 256, 0, c->stream>>>(Gamma, c->dim, c->mesh[0], c->mesh[1],
                                                                  c->mesh[2], c->qQ, c->nv, c->nc, de_qp);
  bse_count_launch(2);
  return bse_check_launch(c, "adjoint transform");
}

bse_status run_seed_lowrank(bse_ctx *c, const double2 *X, const double *g, int r, double2 *Gamma) {
  const long long n = c->dim * c->dim;
  k_seed_lowrank<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(X, g, r, c->dim, Gamma);
  bse_count_launch();
  return bse_check_launch(c, "adjoint seed");
}

// C = alpha A^T B for one pair of row-major complex matrices A [K x M], B [K x N]; C [M x N].
bse_status launch_zgemm_tn(bse_ctx *c, int M, int N, int K, const double2 *A, const double2 *B, double2 *C,
                           double alpha) {
  dim3 grid((N + 63) / 64, (M + 63) / 64, 1);
  if (grid.y > 65535) return bse_fail(c, BSE_EINVAL, "zgemm_tn grid too large");
  k_zgemm_tn<<<grid, 256, 0, c->stream>>>(M, N, K, A, 0, B, 0, C, 0, nullptr, 0, alpha);
  bse_count_launch();
  return bse_check_launch(c, "zgemm_tn");
}
