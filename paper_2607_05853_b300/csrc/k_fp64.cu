// FP64 CUDA-core kernels of the BSE assembly (the plain FP64 GPU path) and the per-k
// stage shared by every precision.
//
//  k_interp_W        W(q) = sum_R w_R W(R) exp(-i q.R)      (R-sum of Eq. W_LRI, §III.B)
//  k_half_transform  Y^mu_sn(k) = sum_t [sum_R C^mu_st(R) exp(i k.R)] c^k_tn, s on atom(mu)
//  k_exchange_X      X[(k,i,a)]^mu = C~^mu_{a k+Q, i k}                     (§III.A)
//  k_project_slab    M_vv(k1,q)^mu_ij = C~^mu_{j k2, i k1},
//                    M_cc(k1,q)^mu_ab = C~^mu_{a k1+Q, b k2+Q}, k2 = k1 - q (§III.A)
//  (Q is the exciton momentum, 0 for the optical Hamiltonian; the pair (k, i, a) holds
//   valence i at k and conduction a at k + Q)
//  k_zgemm_nn        batched complex GEMM  C = A B (row-major), used for T = M_vv W(q)
//                    and P = X V(0)
//  k_project_cv_slab coupling block B (full BSE): M1(k1,q)^mu_bi = C~^mu_{b k2, i k1},
//                    M2(k1,q)^mu_aj = C~^mu_{a k1, j k2}                    (§II.C, §III.A)
//  k_g2_coupling     B block = (alpha X V X^T - T1 M2^T)/N_k with T1 = M1 W(q); B = B^T
//  k_g2_write        H block = (alpha X V X^dagger - T M_cc^T)/N_k + diagonal, V = V(0) at
//                    Q = 0 and sum_R w_R Vbar(R) e^{+iQ.R} otherwise
//                    (Eq. Hamiltonian with the kernels of Eq. W_LRI)
//
// With C^mu_st(R) real the second term of the KS-basis coefficient is a conjugate of the
// first:  C~^mu_{m k', n k} = F(k',k)_mn + conj(F(k,k')_nm),
//         F^mu(k',k)_mn = sum_{s on atom(mu)} conj(c^{k'}_sm) Y^mu_sn(k),
// so one table Y serves both terms (§III.A, C(-k) = conj C(k) for real C(R)).
#include "bse_internal.cuh"

namespace {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {  // conj(a) * b
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) {
  return make_double2(a.x + b.x, a.y + b.y);
}
__device__ __forceinline__ double2 conjd(double2 a) { return make_double2(a.x, -a.y); }

constexpr int QB = 4;  // q values per interp block

// out[q - q_first] for the transfers q = q_first .. q_first + n_q - 1.
__global__ void k_interp_W(const double *__restrict__ WR, const int *__restrict__ RW,
                           const double *__restrict__ wRW, int nRW, int naux, int n1, int n2,
                           int n3, int q_first, int n_q, double2 *__restrict__ out) {
  extern __shared__ double2 ph[];  // [QB][nRW]
  const int nk = q_first + n_q;
  const int q0 = q_first + blockIdx.y * QB;
  for (int t = threadIdx.x; t < QB * nRW; t += blockDim.x) {
    int qq = t / nRW, r = t % nRW, q = q0 + qq;
    double2 v = make_double2(0.0, 0.0);
    if (q < nk) {
      double2 e = phase_qR(q, RW + 3 * r, n1, n2, n3);
      v = make_double2(e.x * wRW[r], e.y * wRW[r]);
    }
    ph[t] = v;
  }
  __syncthreads();
  const long long nn = (long long)naux * naux;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nn;
       e += (long long)gridDim.x * blockDim.x) {
    double2 acc[QB];
#pragma unroll
    for (int j = 0; j < QB; j++) acc[j] = make_double2(0.0, 0.0);
    for (int r = 0; r < nRW; r++) {
      double w = WR[r * nn + e];
#pragma unroll
      for (int j = 0; j < QB; j++) {
        acc[j].x = fma(ph[j * nRW + r].x, w, acc[j].x);
        acc[j].y = fma(ph[j * nRW + r].y, w, acc[j].y);
      }
    }
#pragma unroll
    for (int j = 0; j < QB; j++)
      if (q0 + j < nk) out[(long long)(q0 + j - q_first) * nn + e] = acc[j];
  }
}

constexpr int TCH = 16;  // t-chunk of the half transform

// One block per (s, k): Y[k][s_loc][n][mu] for mu on atom(s).
__global__ void k_half_transform(const double *__restrict__ CR, const int *__restrict__ RC,
                                 int nRC, const double2 *__restrict__ ck, int nao_tot, int nb,
                                 int naux, int nao_max, const int *__restrict__ ao_start,
                                 const int *__restrict__ aux_start, const int *__restrict__ nauxA,
                                 int n_atoms, int n1, int n2, int n3, double o1, double o2,
                                 double o3, double2 *__restrict__ Y) {
  extern __shared__ double2 sm[];
  const int s = blockIdx.x, k = blockIdx.y;
  int A = 0;
  while (A + 1 < n_atoms && ao_start[A + 1] <= s) A++;
  const int s_loc = s - ao_start[A], mu0 = aux_start[A], nmu = nauxA[A];
  double2 *phs = sm;                      // [nRC]
  double2 *cks = phs + nRC;               // [nao_tot][nb]
  double2 *Ckc = cks + nao_tot * nb;      // [TCH][nmu]
  double2 *Yacc = Ckc + TCH * nmu;        // [nb][nmu]
  for (int r = threadIdx.x; r < nRC; r += blockDim.x)
    phs[r] = phase_kR(k, RC + 3 * r, n1, n2, n3, o1, o2, o3);
  for (int e = threadIdx.x; e < nao_tot * nb; e += blockDim.x)
    cks[e] = ck[(long long)k * nao_tot * nb + e];
  for (int e = threadIdx.x; e < nb * nmu; e += blockDim.x) Yacc[e] = make_double2(0.0, 0.0);
  __syncthreads();
  const long long sR = (long long)nao_tot * nao_tot * naux;
  for (int t0 = 0; t0 < nao_tot; t0 += TCH) {
    for (int e = threadIdx.x; e < TCH * nmu; e += blockDim.x) {
      int tt = e / nmu, mu = e % nmu, t = t0 + tt;
      double2 acc = make_double2(0.0, 0.0);
      if (t < nao_tot) {
        const double *src = CR + ((long long)s * nao_tot + t) * naux + mu0 + mu;
        for (int r = 0; r < nRC; r++) {
          double v = src[r * sR];
          acc.x = fma(phs[r].x, v, acc.x);
          acc.y = fma(phs[r].y, v, acc.y);
        }
      }
      Ckc[e] = acc;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nb * nmu; e += blockDim.x) {
      int n = e / nmu, mu = e % nmu;
      double2 acc = Yacc[e];
      int tmax = min(TCH, nao_tot - t0);
      for (int tt = 0; tt < tmax; tt++) acc = cadd(acc, cmul(Ckc[tt * nmu + mu], cks[(t0 + tt) * nb + n]));
      Yacc[e] = acc;
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < nb * nmu; e += blockDim.x) {
    int n = e / nmu, mu = e % nmu;
    Y[(((long long)k * nao_max + s_loc) * nb + n) * naux + mu0 + mu] = Yacc[e];
  }
}

// X[k][i][a][mu] = C~^mu_{a k+Q, i k} = F(k+Q,k)_{(nv+a) i} + conj(F(k,k+Q)_{i (nv+a)})
// (k + Q = kdiff(k, qmQ); Q = 0 gives the optical pairs).
__global__ void k_exchange_X(const double2 *__restrict__ Y, const double2 *__restrict__ ck,
                             int nao_tot, int nb, int nv, int nc, int naux, int nao_max,
                             const int *__restrict__ aux_atom, const int *__restrict__ ao_start,
                             const int *__restrict__ naoA, int n1, int n2, int n3, int qmQ,
                             double2 *__restrict__ X) {
  const int k = blockIdx.y, kq = kdiff(k, qmQ, n1, n2, n3);
  const int mu = blockIdx.x * blockDim.x + threadIdx.x;
  if (mu >= naux) return;
  const int A = aux_atom[mu], ao0 = ao_start[A], na = naoA[A];
  const double2 *c = ck + (long long)k * nao_tot * nb;
  const double2 *cq = ck + (long long)kq * nao_tot * nb;
  const double2 *Yk = Y + (long long)k * nao_max * nb * naux;
  const double2 *Yq = Y + (long long)kq * nao_max * nb * naux;
  for (int i = 0; i < nv; i++)
    for (int a = 0; a < nc; a++) {
      double2 f1 = make_double2(0, 0), f2 = make_double2(0, 0);
      for (int s = 0; s < na; s++) {
        f1 = cadd(f1, cmulc(cq[(ao0 + s) * nb + nv + a], Yk[((long long)s * nb + i) * naux + mu]));
        f2 = cadd(f2, cmulc(c[(ao0 + s) * nb + i], Yq[((long long)s * nb + nv + a) * naux + mu]));
      }
      X[(((long long)k * nv + i) * nc + a) * naux + mu] = cadd(f1, conjd(f2));
    }
}

constexpr int MAXB = 8;

// grid: x = nmu_chunks * (nv + nc), y = k1, z = q - q0.  Row r < nv -> M_vv row i (bands at
// k1, k2), else M_cc row a = r - nv (bands at k1 + Q, k2 + Q; k + Q = kdiff(k, qmQ)).
__global__ void k_project_slab(const double2 *__restrict__ Y, const double2 *__restrict__ ck,
                               int nao_tot, int nb, int nv, int nc, int naux, int nao_max,
                               const int *__restrict__ aux_atom, const int *__restrict__ ao_start,
                               const int *__restrict__ naoA, int n1, int n2, int n3, int qmQ, int q0,
                               const int *__restrict__ qlist, double2 *__restrict__ Mv,
                               double2 *__restrict__ Mc) {
  extern __shared__ double2 sc[];  // c1 [nao][nb], c2 [nao][nb]
  const int nk = n1 * n2 * n3;
  const int nchunk = (naux + blockDim.x - 1) / blockDim.x;
  const int row = blockIdx.x / nchunk;
  const int mu = (blockIdx.x % nchunk) * blockDim.x + threadIdx.x;
  const int k1 = blockIdx.y, qq = blockIdx.z, q = qlist[q0 + qq];
  const int k2 = kdiff(k1, q, n1, n2, n3);
  const int p1 = row < nv ? k1 : kdiff(k1, qmQ, n1, n2, n3);
  const int p2 = row < nv ? k2 : kdiff(k2, qmQ, n1, n2, n3);
  double2 *c1 = sc, *c2 = sc + nao_tot * nb;
  for (int e = threadIdx.x; e < nao_tot * nb; e += blockDim.x) {
    c1[e] = ck[(long long)p1 * nao_tot * nb + e];
    c2[e] = ck[(long long)p2 * nao_tot * nb + e];
  }
  __syncthreads();
  if (mu >= naux) return;
  const int A = aux_atom[mu], ao0 = ao_start[A], na = naoA[A];
  const double2 *Y1 = Y + (long long)p1 * nao_max * nb * naux + mu;
  const double2 *Y2 = Y + (long long)p2 * nao_max * nb * naux + mu;
  double2 acc1[MAXB], acc2[MAXB];
#pragma unroll
  for (int j = 0; j < MAXB; j++) acc1[j] = acc2[j] = make_double2(0, 0);
  if (row < nv) {
    const int i = row;
    for (int s = 0; s < na; s++) {
      const double2 y1 = Y1[((long long)s * nb + i) * naux];
      const double2 ci = c1[(ao0 + s) * nb + i];
#pragma unroll
      for (int j = 0; j < MAXB; j++)
        if (j < nv) {
          acc1[j] = cadd(acc1[j], cmulc(c2[(ao0 + s) * nb + j], y1));
          acc2[j] = cadd(acc2[j], cmulc(ci, Y2[((long long)s * nb + j) * naux]));
        }
    }
    double2 *out = Mv + ((((long long)qq * nk + k1) * nv + i) * nv) * naux + mu;
#pragma unroll
    for (int j = 0; j < MAXB; j++)
      if (j < nv) out[(long long)j * naux] = cadd(acc1[j], conjd(acc2[j]));
  } else {
    const int a = row - nv;
    for (int s = 0; s < na; s++) {
      const double2 y1 = Y1[((long long)s * nb + nv + a) * naux];
      const double2 ca = c1[(ao0 + s) * nb + nv + a];
#pragma unroll
      for (int b = 0; b < MAXB; b++)
        if (b < nc) {
          acc1[b] = cadd(acc1[b], cmulc(ca, Y2[((long long)s * nb + nv + b) * naux]));
          acc2[b] = cadd(acc2[b], cmulc(c2[(ao0 + s) * nb + nv + b], y1));
        }
    }
    double2 *out = Mc + ((((long long)qq * nk + k1) * nc + a) * nc) * naux + mu;
#pragma unroll
    for (int b = 0; b < MAXB; b++)
      if (b < nc) out[(long long)b * naux] = cadd(acc1[b], conjd(acc2[b]));
  }
}

// Conduction-valence projections of one q-slab for the coupling block.  grid: x = nmu_chunks *
// 2 nc, y = k1, z = q - q0.  Row r < nc -> M1 row b = r (columns i), else M2 row a = r - nc
// (columns j).  With F as above:
//   M1[b][i] = F(k2,k1)_{(nv+b) i} + conj(F(k1,k2)_{i (nv+b)}),
//   M2[a][j] = F(k1,k2)_{(nv+a) j} + conj(F(k2,k1)_{j (nv+a)}).
__global__ void k_project_cv_slab(const double2 *__restrict__ Y, const double2 *__restrict__ ck,
                                  int nao_tot, int nb, int nv, int nc, int naux, int nao_max,
                                  const int *__restrict__ aux_atom, const int *__restrict__ ao_start,
                                  const int *__restrict__ naoA, int n1, int n2, int n3, int q0,
                                  const int *__restrict__ qlist, double2 *__restrict__ M1,
                                  double2 *__restrict__ M2) {
  extern __shared__ double2 sc[];  // c1 [nao][nb], c2 [nao][nb]
  const int nk = n1 * n2 * n3;
  const int nchunk = (naux + blockDim.x - 1) / blockDim.x;
  const int row = blockIdx.x / nchunk;
  const int mu = (blockIdx.x % nchunk) * blockDim.x + threadIdx.x;
  const int k1 = blockIdx.y, qq = blockIdx.z, q = qlist[q0 + qq];
  const int k2 = kdiff(k1, q, n1, n2, n3);
  double2 *c1 = sc, *c2 = sc + nao_tot * nb;
  for (int e = threadIdx.x; e < nao_tot * nb; e += blockDim.x) {
    c1[e] = ck[(long long)k1 * nao_tot * nb + e];
    c2[e] = ck[(long long)k2 * nao_tot * nb + e];
  }
  __syncthreads();
  if (mu >= naux) return;
  const int A = aux_atom[mu], ao0 = ao_start[A], na = naoA[A];
  const double2 *Y1 = Y + (long long)k1 * nao_max * nb * naux + mu;
  const double2 *Y2 = Y + (long long)k2 * nao_max * nb * naux + mu;
  const bool first = row < nc;
  const int cb = nv + (first ? row : row - nc);            // the conduction band of this row
  // first: bra conduction at k2, valence kets at k1; else bra conduction at k1, kets at k2
  const double2 *cc = first ? c2 : c1, *cvv = first ? c1 : c2;
  const double2 *Yv = first ? Y1 : Y2, *Yc = first ? Y2 : Y1;
  double2 acc1[MAXB], acc2[MAXB];
#pragma unroll
  for (int j = 0; j < MAXB; j++) acc1[j] = acc2[j] = make_double2(0, 0);
  for (int s = 0; s < na; s++) {
    const double2 cs = cc[(ao0 + s) * nb + cb];
    const double2 yc = Yc[((long long)s * nb + cb) * naux];
#pragma unroll
    for (int j = 0; j < MAXB; j++)
      if (j < nv) {
        acc1[j] = cadd(acc1[j], cmulc(cs, Yv[((long long)s * nb + j) * naux]));
        acc2[j] = cadd(acc2[j], cmulc(cvv[(ao0 + s) * nb + j], yc));
      }
  }
  double2 *out = (first ? M1 : M2) + ((((long long)qq * nk + k1) * nc + (cb - nv)) * nv) * naux + mu;
#pragma unroll
  for (int j = 0; j < MAXB; j++)
    if (j < nv) out[(long long)j * naux] = cadd(acc1[j], conjd(acc2[j]));
}

// Batched row-major complex GEMM C = A B, 64x64 tiles, 4x4 complex outputs per thread.
__global__ void __launch_bounds__(256) k_zgemm_nn(int M, int N, int K, const double2 *__restrict__ A,
                                                  int lda, long long sA, const double2 *__restrict__ B,
                                                  int ldb, long long sB, double2 *__restrict__ C,
                                                  int ldc, long long sC, const int *__restrict__ bidx) {
  __shared__ double2 As[16][64];
  __shared__ double2 Bs[16][64];
  const int bz = blockIdx.z;
  A += bz * sA;
  B += (bidx ? bidx[bz] : bz) * sB;
  C += bz * sC;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int row0 = blockIdx.y * 64, col0 = blockIdx.x * 64;
  double2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; i++)
#pragma unroll
    for (int j = 0; j < 4; j++) acc[i][j] = make_double2(0, 0);
  for (int k0 = 0; k0 < K; k0 += 16) {
    for (int e = threadIdx.x; e < 1024; e += 256) {
      int r = e / 16, kk = e % 16, gr = row0 + r, gk = k0 + kk;
      As[kk][r] = (gr < M && gk < K) ? A[(long long)gr * lda + gk] : make_double2(0, 0);
      int kb = e / 64, cc = e % 64, gkb = k0 + kb, gc = col0 + cc;
      Bs[kb][cc] = (gkb < K && gc < N) ? B[(long long)gkb * ldb + gc] : make_double2(0, 0);
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
      int r = row0 + ty + 16 * i, cc = col0 + tx + 16 * j;
      if (r < M && cc < N) C[(long long)r * ldc + cc] = acc[i][j];
    }
}

constexpr int G2CH = 16;  // nu chunk staged in shared memory

// One block per pair (k1, q): writes the nvc x nvc block of H at rows k1, columns k2.
__global__ void __launch_bounds__(256) k_g2_write(const double2 *__restrict__ T, const double2 *__restrict__ Mc,
                                                  const double2 *__restrict__ P, const double2 *__restrict__ X,
                                                  const double *__restrict__ eqp, int nv, int nc, int naux,
                                                  int n1, int n2, int n3, int qmQ, int q0,
                                                  const int *__restrict__ qlist, double alpha, long long dim,
                                                  double2 *__restrict__ H) {
  extern __shared__ double2 sm[];
  const int nk = n1 * n2 * n3;
  const int k1 = blockIdx.x, qq = blockIdx.y, q = qlist[q0 + qq];
  const int k2 = kdiff(k1, q, n1, n2, n3);
  const bool mirror = !q_self_conjugate(q, n1, n2, n3);
  const int nvc = nv * nc, nvv = nv * nv, ncc = nc * nc, nb = nv + nc;
  double2 *sT = sm, *sM = sT + nvv * G2CH, *sP = sM + ncc * G2CH, *sX = sP + nvc * G2CH;
  const double2 *Tk = T + ((long long)qq * nk + k1) * nvv * naux;
  const double2 *Mk = Mc + ((long long)qq * nk + k1) * ncc * naux;
  const double2 *Pk = P + (long long)k1 * nvc * naux;
  const double2 *Xk = X + (long long)k2 * nvc * naux;
  const int nout = nvc * nvc;
  constexpr int MAXO = 16;  // nvc <= 64 -> at most 16 outputs per thread
  double2 ad[MAXO], ax[MAXO];
#pragma unroll
  for (int t = 0; t < MAXO; t++) ad[t] = ax[t] = make_double2(0, 0);
  for (int n0 = 0; n0 < naux; n0 += G2CH) {
    const int nn = min(G2CH, naux - n0);
    for (int e = threadIdx.x; e < (nvv + ncc + 2 * nvc) * G2CH; e += blockDim.x) {
      int r = e / G2CH, u = e % G2CH;
      double2 v = make_double2(0, 0);
      if (u < nn) {
        if (r < nvv) v = Tk[(long long)r * naux + n0 + u];
        else if (r < nvv + ncc) v = Mk[(long long)(r - nvv) * naux + n0 + u];
        else if (r < nvv + ncc + nvc) v = Pk[(long long)(r - nvv - ncc) * naux + n0 + u];
        else v = Xk[(long long)(r - nvv - ncc - nvc) * naux + n0 + u];
      }
      sm[e] = v;
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < MAXO; t++) {
      int o = threadIdx.x + t * blockDim.x;
      if (o < nout) {
        int ia = o / nvc, jb = o % nvc;
        int i = ia / nc, a = ia % nc, j = jb / nc, b = jb % nc;
        const double2 *pt = sT + (i * nv + j) * G2CH, *pm = sM + (a * nc + b) * G2CH;
        const double2 *pp = sP + ia * G2CH, *px = sX + jb * G2CH;
        for (int u = 0; u < nn; u++) {
          ad[t] = cadd(ad[t], cmul(pt[u], pm[u]));
          ax[t] = cadd(ax[t], cmul(pp[u], conjd(px[u])));
        }
      }
    }
    __syncthreads();
  }
  const double inv = 1.0 / nk;
#pragma unroll
  for (int t = 0; t < MAXO; t++) {
    int o = threadIdx.x + t * blockDim.x;
    if (o < nout) {
      int ia = o / nvc, jb = o % nvc;
      int i = ia / nc, a = ia % nc;
      double2 h = make_double2((alpha * ax[t].x - ad[t].x) * inv, (alpha * ax[t].y - ad[t].y) * inv);
      if (q == 0 && ia == jb)
        h.x += eqp[(long long)kdiff(k1, qmQ, n1, n2, n3) * nb + nv + a] - eqp[(long long)k1 * nb + i];
      H[((long long)k1 * nvc + ia) * dim + (long long)k2 * nvc + jb] = h;
      if (mirror) H[((long long)k2 * nvc + jb) * dim + (long long)k1 * nvc + ia] = conjd(h);
    }
  }
}

// One block per pair (k1, q): the nvc x nvc block of B at rows k1, columns k2 = k1 - q,
// B[(k1,i,a),(k2,j,b)] = (alpha sum_mu P[(k1,i,a)] X[(k2,j,b)] - sum_nu T1[(b,i)] M2[(a,j)]) / N_k,
// and its transpose at (k2, k1) (B is symmetric).
__global__ void __launch_bounds__(256) k_g2_coupling(const double2 *__restrict__ T1, const double2 *__restrict__ M2,
                                                     const double2 *__restrict__ P, const double2 *__restrict__ X,
                                                     int nv, int nc, int naux, int n1, int n2, int n3, int q0,
                                                     const int *__restrict__ qlist, double alpha, long long dim,
                                                     double2 *__restrict__ B) {
  extern __shared__ double2 sm[];
  const int nk = n1 * n2 * n3;
  const int k1 = blockIdx.x, qq = blockIdx.y, q = qlist[q0 + qq];
  const int k2 = kdiff(k1, q, n1, n2, n3);
  const bool mirror = !q_self_conjugate(q, n1, n2, n3);
  const int nvc = nv * nc;
  double2 *sT = sm, *sM = sT + nvc * G2CH, *sP = sM + nvc * G2CH, *sX = sP + nvc * G2CH;
  const double2 *Tk = T1 + ((long long)qq * nk + k1) * nvc * naux;
  const double2 *Mk = M2 + ((long long)qq * nk + k1) * nvc * naux;
  const double2 *Pk = P + (long long)k1 * nvc * naux;
  const double2 *Xk = X + (long long)k2 * nvc * naux;
  const int nout = nvc * nvc;
  constexpr int MAXO = 16;  // nvc <= 64 -> at most 16 outputs per thread
  double2 ad[MAXO], ax[MAXO];
#pragma unroll
  for (int t = 0; t < MAXO; t++) ad[t] = ax[t] = make_double2(0, 0);
  for (int n0 = 0; n0 < naux; n0 += G2CH) {
    const int nn = min(G2CH, naux - n0);
    for (int e = threadIdx.x; e < 4 * nvc * G2CH; e += blockDim.x) {
      const int r = e / G2CH, u = e % G2CH, part = r / nvc, rr = r % nvc;
      double2 v = make_double2(0, 0);
      if (u < nn) {
        const double2 *src = part == 0 ? Tk : part == 1 ? Mk : part == 2 ? Pk : Xk;
        v = src[(long long)rr * naux + n0 + u];
      }
      sm[e] = v;
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < MAXO; t++) {
      const int o = threadIdx.x + t * blockDim.x;
      if (o < nout) {
        const int ia = o / nvc, jb = o % nvc;
        const int i = ia / nc, a = ia % nc, j = jb / nc, b = jb % nc;
        const double2 *pt = sT + (b * nv + i) * G2CH, *pm = sM + (a * nv + j) * G2CH;
        const double2 *pp = sP + ia * G2CH, *px = sX + jb * G2CH;
        for (int u = 0; u < nn; u++) {
          ad[t] = cadd(ad[t], cmul(pt[u], pm[u]));
          ax[t] = cadd(ax[t], cmul(pp[u], px[u]));
        }
      }
    }
    __syncthreads();
  }
  const double inv = 1.0 / nk;
#pragma unroll
  for (int t = 0; t < MAXO; t++) {
    const int o = threadIdx.x + t * blockDim.x;
    if (o < nout) {
      const int ia = o / nvc, jb = o % nvc;
      const double2 h = make_double2((alpha * ax[t].x - ad[t].x) * inv, (alpha * ax[t].y - ad[t].y) * inv);
      B[((long long)k1 * nvc + ia) * dim + (long long)k2 * nvc + jb] = h;
      if (mirror) B[((long long)k2 * nvc + jb) * dim + (long long)k1 * nvc + ia] = h;
    }
  }
}

}  // namespace

// ------------------------------------------------------------------------------ launchers
bse_status launch_interp_W_fp64(bse_ctx *c, const double *W_R, double2 *out, int q_first, int n_q) {
  if (n_q < 0) n_q = c->nk - q_first;
  if (q_first < 0 || n_q < 1 || q_first + n_q > c->nk) return bse_fail(c, BSE_EINVAL, "interp: bad q range");
  const long long nn = (long long)c->naux_tot * c->naux_tot;
  dim3 grid((unsigned)std::min<long long>((nn + 255) / 256, 1024), (n_q + QB - 1) / QB);
  size_t sm = sizeof(double2) * QB * c->n_RW;
  bse_prof_begin(c, BSE_KP_INTERP);
  k_interp_W<<<grid, 256, sm, c->stream>>>(W_R, c->d_R_W, c->d_w_RW, c->n_RW, c->naux_tot,
                                           c->mesh[0], c->mesh[1], c->mesh[2], q_first, n_q, out);
  bse_prof_end(c, BSE_KP_INTERP);
  bse_count_launch();
  return bse_check_launch(c, "interp_W");
}

bse_status launch_half_transform_fp64(bse_ctx *c, const double *C_R) {
  int maxmu = 0;
  for (int a : c->naux) maxmu = std::max(maxmu, a);
  size_t sm = sizeof(double2) * (c->n_RC + c->nao_tot * c->nb + TCH * maxmu + c->nb * maxmu);
  if (sm > 200 * 1024) return bse_fail(c, BSE_EINVAL, "half transform: basis too large for one block");
  if (sm > 48 * 1024)
    cudaFuncSetAttribute(k_half_transform, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  dim3 grid(c->nao_tot, c->nk);
  bse_prof_begin(c, BSE_KP_HALF);
  k_half_transform<<<grid, 256, sm, c->stream>>>(C_R, c->d_R_C, c->n_RC, c->ck, c->nao_tot, c->nb,
                                                 c->naux_tot, c->nao_max, c->d_ao_start,
                                                 c->d_aux_start, c->d_naux, c->n_atoms, c->mesh[0],
                                                 c->mesh[1], c->mesh[2], c->koff[0], c->koff[1],
                                                 c->koff[2], c->Y);
  bse_prof_end(c, BSE_KP_HALF);
  bse_count_launch();
  return bse_check_launch(c, "half_transform");
}

bse_status launch_exchange_factors_fp64(bse_ctx *c) {
  dim3 grid((c->naux_tot + 127) / 128, c->nk);
  k_exchange_X<<<grid, 128, 0, c->stream>>>(c->Y, c->ck, c->nao_tot, c->nb, c->nv, c->nc,
                                            c->naux_tot, c->nao_max, c->d_aux_atom, c->d_ao_start,
                                            c->d_nao, c->mesh[0], c->mesh[1], c->mesh[2], c->qmQ, c->X);
  bse_count_launch();
  return bse_check_launch(c, "exchange_X");
}

bse_status launch_zgemm_fp64(bse_ctx *c, int M, int N, int K, const double2 *A, int lda, long long sA,
                             const double2 *B, int ldb, long long sB, double2 *C, int ldc,
                             long long sC, int batch, int prof_id, const int *bidx) {
  dim3 grid((N + 63) / 64, (M + 63) / 64, batch);
  if (grid.y > 65535 || batch > 65535) return bse_fail(c, BSE_EINVAL, "zgemm grid too large");
  if (prof_id >= 0) bse_prof_begin(c, prof_id);
  k_zgemm_nn<<<grid, 256, 0, c->stream>>>(M, N, K, A, lda, sA, B, ldb, sB, C, ldc, sC, bidx);
  if (prof_id >= 0) bse_prof_end(c, prof_id);
  bse_count_launch();
  return bse_check_launch(c, "zgemm");
}

bse_status launch_project_slab_fp64(bse_ctx *c, int q0, int nq, const int *qlist) {
  const int nchunk = (c->naux_tot + 127) / 128;
  dim3 grid(nchunk * (c->nv + c->nc), c->nk, nq);
  size_t sm = sizeof(double2) * 2 * c->nao_tot * c->nb;
  if (sm > 48 * 1024) return bse_fail(c, BSE_EINVAL, "project: N_ao * (nv + nc) too large");
  bse_prof_begin(c, BSE_KP_PROJECT);
  k_project_slab<<<grid, 128, sm, c->stream>>>(c->Y, c->ck, c->nao_tot, c->nb, c->nv, c->nc,
                                               c->naux_tot, c->nao_max, c->d_aux_atom, c->d_ao_start,
                                               c->d_nao, c->mesh[0], c->mesh[1], c->mesh[2], c->qmQ,
                                               q0, qlist, c->Mv, c->Mc);
  bse_prof_end(c, BSE_KP_PROJECT);
  bse_count_launch();
  return bse_check_launch(c, "project_slab");
}

bse_status launch_g2_write_fp64(bse_ctx *c, int q0, int nq, double2 *H) {
  dim3 grid(c->nk, nq);
  size_t sm = sizeof(double2) * (c->nv * c->nv + c->nc * c->nc + 2 * c->nvc) * G2CH;
  if (sm > 48 * 1024) cudaFuncSetAttribute(k_g2_write, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  bse_prof_begin(c, BSE_KP_G2);
  k_g2_write<<<grid, 256, sm, c->stream>>>(c->T, c->Mc, c->P, c->X, c->eqp, c->nv, c->nc,
                                           c->naux_tot, c->mesh[0], c->mesh[1], c->mesh[2], c->qmQ, q0,
                                           c->d_qplus, c->alpha, c->dim, H);
  bse_prof_end(c, BSE_KP_G2);
  bse_count_launch();
  return bse_check_launch(c, "g2_write");
}

bse_status launch_project_cv_slab_fp64(bse_ctx *c, int q0, int nq, const int *qlist, double2 *M1, double2 *M2) {
  const int nchunk = (c->naux_tot + 127) / 128;
  dim3 grid(nchunk * 2 * c->nc, c->nk, nq);
  size_t sm = sizeof(double2) * 2 * c->nao_tot * c->nb;
  if (sm > 48 * 1024) return bse_fail(c, BSE_EINVAL, "project: N_ao * (nv + nc) too large");
  bse_prof_begin(c, BSE_KP_PROJECT);
  k_project_cv_slab<<<grid, 128, sm, c->stream>>>(c->Y, c->ck, c->nao_tot, c->nb, c->nv, c->nc, c->naux_tot,
                                                  c->nao_max, c->d_aux_atom, c->d_ao_start, c->d_nao, c->mesh[0],
                                                  c->mesh[1], c->mesh[2], q0, qlist, M1, M2);
  bse_prof_end(c, BSE_KP_PROJECT);
  bse_count_launch();
  return bse_check_launch(c, "project_cv_slab");
}

bse_status launch_g2_coupling_fp64(bse_ctx *c, int q0, int nq, const double2 *T1, const double2 *M2, double2 *B) {
  dim3 grid(c->nk, nq);
  size_t sm = sizeof(double2) * 4 * c->nvc * G2CH;
  if (sm > 48 * 1024) cudaFuncSetAttribute(k_g2_coupling, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  bse_prof_begin(c, BSE_KP_G2);
  k_g2_coupling<<<grid, 256, sm, c->stream>>>(T1, M2, c->P, c->X, c->nv, c->nc, c->naux_tot, c->mesh[0], c->mesh[1],
                                              c->mesh[2], q0, c->d_qplus, c->alpha, c->dim, B);
  bse_prof_end(c, BSE_KP_G2);
  bse_count_launch();
  return bse_check_launch(c, "g2_coupling");
}
