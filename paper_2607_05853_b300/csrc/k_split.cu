// Split-precision assembly of H (BSE_BF16X3 / X2 / X1, BSE_TF32X2): the bulk complex
// contractions run on tcgen05 tensor cores with bf16 (or tf32) operand pieces and FP32
// accumulation; phases and the E_c - E_v diagonal stay FP64; H is stored as complex64 (or
// complex128 on request).
//
// Per q-slab (q = k1 - k2, §III.A Eq. W_LRI):
//   k_proj32      M_vv(k1,q) and M_cc(k1,q) in FP32 from Y (F(k',k) + conj F(k,k')^T),
//                 M_vv written as bf16 pieces (the GEMM A operand), M_cc as FP32;
//   k_tc_zgemm    T = M_vv W(q) on tensor cores (B operand: bf16 pieces of W(q)^T);
//   k_g2_32       H block += -(1/N_k) T M_cc^T (+ diagonal, FP64), FP32 per pair.
// Before the slabs, the exchange term alpha/N_k (X V) conj(X)^T is one tensor-core GEMM
// that writes every element of H (V = V(0) at exciton momentum Q = 0, else the complex
// sum_R w_R Vbar(R) e^{+iQ.R}).  At Q != 0 the per-k tables are relabelled once (valence
// columns of k, conduction columns of k + Q; k_shift_tables) and the kernels run unchanged.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <array>
#include <map>
#include <mutex>
#include <tuple>
#include <cstring>
#include <functional>
#include <vector>

#include "bse_internal.cuh"
#include "tc_direct.cuh"
#include "tc_direct_ns.cuh"
#include "tc_gemm.cuh"

namespace {

constexpr int TC_BN = 160;                       // default N tile (and the exchange's)
constexpr int TC_BN_CAND[4] = {64, 96, 128, 160};  // N tiles the autotuner may pick for T = M_vv W(q)

struct SplitWS {
  int np = 3, pp = 6;
  int kmem = 0, kchunks = 0;
  int nq = 1, rows = 0;
  bool tf32 = false;             // pieces are tf32 values in FP32 words (two per value)
  int pbytes = 2;                // bytes per piece element (2 bf16, 4 tf32)
  // piece buffers (PP = 2 x pieces planes, elements of pbytes bytes)
  void *Wp = nullptr;            // [nk][PP][naux][kmem]   B[nu][mu] = W(q)[mu][nu]
  void *Ap = nullptr;            // [nq][PP][rows][kmem]   M_vv pieces
  float2 *Mc32 = nullptr;        // [nq][nk][nc*nc][naux], or [nq][nk][naux_pad][nc*nc] for the fused kernel
  float2 *T32 = nullptr;         // [nq][naux][rows]  (column nu of T = M_vv W(q) is contiguous)
  float2 *Y32 = nullptr;         // [nk][nao_max][nb][naux]
  void *Pp = nullptr;            // [PP][dim][kmem]        pieces of X V
  void *Xp = nullptr;            // [PP][dim][kmem]        pieces of conj(X)
  CUtensorMap tmA_g1, tmB_g1, tmA_x, tmB_x;
  int bn_g1 = TC_BN;             // N tile of the M_vv W(q) GEMM (autotuned)
  int proj_bs = 0;               // threads per block of the register-blocked projection (autotuned; 0 = default)
  // fused direct term (T = M_vv W(q) and T M_cc^T in one kernel, T kept in tensor memory):
  // used when N_aux fits one N tile and the window has a register-blocked projection
  bool fused = false;
  int bn_d = 0;                  // N tile of the fused kernel (>= N_aux)
  int naux_pad = 0;              // M_cc row length (multiple of 16) in the fused layout
  int pairs_d = 0, nui_d = 0;    // pairs per tile; M_cc columns per ring item
  CUtensorMap tmB_d, tmM_d;      // W pieces with the fused N tile; M_cc {nu, ab, (q, k1)} per item
  // the fused kernel with T's columns in two halves (k_tc_direct_ns): N_aux in (80, 160],
  // Nc <= 4 and pairs x Nc^2 <= 128 (a 16-column M_cc slice in 16 KB)
  bool nsplit = false;
  CUtensorMap tmB_dh, tmM_dh;    // W pieces with 80-row boxes; M_cc with 16-column boxes
  // FP32 per-k stage
  float2 *PHQ = nullptr;         // [nk][n_RW]  w_R e^{-i q.R}
  float2 *PHK = nullptr;         // [nk][n_RC]  e^{+i k.R}
  float *WR32T = nullptr;        // [n_RW][nu][mu]
  float *CR32 = nullptr;         // [n_RC][nao][nao][naux]
  float2 *V032 = nullptr;        // [naux][naux] exchange interaction V (V(0) real at Q = 0)
  // exciton momentum Q != 0: the per-k tables relabelled so that the pairs at k read their
  // valence columns at k and their conduction columns at k + Q (allocated on first use)
  bool shifted = false;
  float2 *Y32q = nullptr, *ck32q = nullptr;
  double2 *ckq = nullptr;
  double *eqpq = nullptr;
  float2 *ck32 = nullptr;        // [nk][nao][nb]
  float2 *X32 = nullptr;         // [dim][naux]  exchange factors
  // coupling block B of the full BSE (allocated on first use)
  int nqB = 0, rowsB = 0;        // q per slab; rows (k1, b, i) of M1 per q
  void *ApB = nullptr;           // [nqB][PP][rowsB][kmem]  M1 pieces
  void *XpB = nullptr;           // [PP][dim][kmem]         pieces of X (no conjugate)
  float2 *McB = nullptr;         // [nqB][nk][nc*nv][naux]   M2
  float2 *TB = nullptr;          // [nqB][naux][rowsB]       T1 = M1 W(q)
  CUtensorMap tmA_B, tmB_xB;
  // matrix-free products (allocated on first use): per-slab partial vectors and exchange sums
  double2 *mf_fwd = nullptr, *mf_bwd = nullptr;  // [3][nq][nk][nvc]
  double2 *mf_zp = nullptr;                      // [3][nchunk][naux] partial X^dagger x
  double2 *mf_z2 = nullptr;                      // [3][naux]         V X^dagger x
  // adjoint (allocated on first use): M_vv of a slab of transfers in plain FP32, two planes
  float *adjMv = nullptr;                        // [nq][2][rows][kmem]
  int mf_nch = 0;
};

SplitWS *ws(bse_ctx *c) { return (SplitWS *)c->tc; }

// x ~ p0 + p1 + p2, each a bf16 (round to nearest), residuals formed exactly in the
// source precision.
template <class R>
__device__ __forceinline__ void split_pieces(R x, int np, __nv_bfloat16 *p) {
  __nv_bfloat16 h = __float2bfloat16_rn((float)x);
  p[0] = h;
  if (np > 1) {
    R r = x - (R)__bfloat162float(h);
    __nv_bfloat16 m = __float2bfloat16_rn((float)r);
    p[1] = m;
    if (np > 2) {
      R r2 = r - (R)__bfloat162float(m);
      p[2] = __float2bfloat16_rn((float)r2);
    }
  }
}

// A tensor-core operand as planes of pieces, [piece * 2 + (re, im)][...]: bf16 pieces (np of
// them, split_pieces) or, with tf32 = 1, two tf32 pieces in FP32 words (x ~ tf32(x) +
// tf32(x - tf32(x)), the residual exact in the source precision); tf32 = 2 (with np = 1): the
// plain FP32 value in two planes (re, im), for the adjoint's CUDA-core GEMM.  Offsets and plane
// pitches count elements of the piece type.
struct PieceBuf {
  void *p;
  int np;
  int tf32;
  template <class R>
  __device__ __forceinline__ void put(long long plane, long long off, R re, R im) const {
    if (tf32 == 2) {
      float *b = static_cast<float *>(p) + off;
      b[0] = (float)re;
      b[plane] = (float)im;
    } else if (tf32) {
      float *b = static_cast<float *>(p) + off;
      const float hr = tc::tf32_rna((float)re), hi = tc::tf32_rna((float)im);
      b[0] = hr;
      b[plane] = hi;
      b[2 * plane] = tc::tf32_rna((float)(re - (R)hr));
      b[3 * plane] = tc::tf32_rna((float)(im - (R)hi));
    } else {
      __nv_bfloat16 pr[3], pi[3];
      split_pieces<R>(re, np, pr);
      split_pieces<R>(im, np, pi);
      __nv_bfloat16 *b = static_cast<__nv_bfloat16 *>(p) + off;
#pragma unroll
      for (int k = 0; k < 3; k++) {
        if (k >= np) break;
        b[(2 * k) * plane] = pr[k];
        b[(2 * k + 1) * plane] = pi[k];
      }
    }
  }
};

PieceBuf pieces(const SplitWS *w, void *p) { return PieceBuf{p, w->np, w->tf32 ? 1 : 0}; }

// ---- FP32 per-k stage (split precisions): phases in FP64, sums in FP32 -------------------
// The products feed bf16 pieces whose sum carries ~2^-24 relative precision, so FP32 sums
// lose nothing that the tensor-core path keeps, and B300's FP32 rate is ~60x its FP64 rate.

// PHQ[q][r] = w_R e^{-2 pi i q.R} and PHK[k][r] = e^{+2 pi i k.R}, reduced exactly in FP64
__global__ void k_phase_tables(const int *__restrict__ RW, const double *__restrict__ wRW, int nRW,
                               const int *__restrict__ RC, int nRC, int n1, int n2, int n3, double o1, double o2,
                               double o3, float2 *__restrict__ PHQ, float2 *__restrict__ PHK) {
  const long long nk = (long long)n1 * n2 * n3;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < nk * nRW) {
    const int q = (int)(e / nRW), r = (int)(e % nRW);
    const double2 d = phase_qR(q, RW + 3 * r, n1, n2, n3);
    PHQ[e] = make_float2((float)(d.x * wRW[r]), (float)(d.y * wRW[r]));
  } else if (e < nk * (nRW + nRC)) {
    const long long e2 = e - nk * nRW;
    const int k = (int)(e2 / nRC), r = (int)(e2 % nRC);
    const double2 d = phase_kR(k, RC + 3 * r, n1, n2, n3, o1, o2, o3);
    PHK[e2] = make_float2((float)d.x, (float)d.y);
  }
}

// WR32T[r][nu][mu] = W_R[r][mu][nu]
__global__ void k_wr_f32t(const double *__restrict__ WR, int nRW, int naux, float *__restrict__ WR32T) {
  const long long nn = (long long)naux * naux;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nn * nRW) return;
  const long long r = e / nn, rem = e % nn;
  const int mu = (int)(rem / naux), nu = (int)(rem % naux);
  WR32T[r * nn + (long long)nu * naux + mu] = (float)WR[e];
}

__global__ void k_d2f(const double *__restrict__ src, long long n, float *__restrict__ dst) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    dst[e] = (float)src[e];
}

// W(q) = sum_R w_R e^{-i q.R} W(R) (R-sum of Eq. W_LRI) for IQB transfers per block, written
// straight as the bf16 pieces of the tensor-core operand B[nu][mu] = W(q)[mu][nu] and, when
// asked, as complex128 W(q)[mu][nu].
constexpr int IQB = 16;
__global__ void __launch_bounds__(256) k_interp_W32(const float *__restrict__ WR32T, const float2 *__restrict__ PHQ,
                                                    int nRW, int naux, int nk, int kmem, PieceBuf Wp,
                                                    double2 *__restrict__ Wq_out) {
  extern __shared__ float2 phs[];  // [IQB][nRW]
  const int q0 = blockIdx.y * IQB;
  for (int t = threadIdx.x; t < IQB * nRW; t += blockDim.x) {
    const int qq = t / nRW, r = t % nRW;
    phs[t] = q0 + qq < nk ? PHQ[(long long)(q0 + qq) * nRW + r] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const long long nn = (long long)naux * naux;
  const long long plane = (long long)naux * kmem;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nn; e += (long long)gridDim.x * blockDim.x) {
    float2 acc[IQB];
#pragma unroll
    for (int j = 0; j < IQB; j++) acc[j] = make_float2(0.f, 0.f);
    for (int r = 0; r < nRW; r++) {
      const float w = WR32T[r * nn + e];
#pragma unroll
      for (int j = 0; j < IQB; j++) {
        acc[j].x = fmaf(phs[j * nRW + r].x, w, acc[j].x);
        acc[j].y = fmaf(phs[j * nRW + r].y, w, acc[j].y);
      }
    }
    const int nu = (int)(e / naux), mu = (int)(e % naux);
#pragma unroll
    for (int j = 0; j < IQB; j++) {
      const int q = q0 + j;
      if (q >= nk) break;
      Wp.put<float>(plane, (long long)q * 2 * Wp.np * plane + (long long)nu * kmem + mu, acc[j].x, acc[j].y);
      if (Wq_out) Wq_out[(long long)q * nn + (long long)mu * naux + nu] = make_double2(acc[j].x, acc[j].y);
    }
  }
}

constexpr int TCH32 = 16;  // t-chunk of the half transform

// One block per (s, k): Y32[k][s_loc][n][mu] = sum_t [sum_R C^mu_st(R) e^{ik.R}] c^k_tn, mu on atom(s).
__global__ void k_half_transform32(const float *__restrict__ CR, const float2 *__restrict__ PHK, int nRC,
                                   const float2 *__restrict__ ck, int nao_tot, int nb, int naux, int nao_max,
                                   const int *__restrict__ ao_start, const int *__restrict__ aux_start,
                                   const int *__restrict__ nauxA, int n_atoms, float2 *__restrict__ Y) {
  extern __shared__ float2 sh[];
  const int s = blockIdx.x, k = blockIdx.y;
  int A = 0;
  while (A + 1 < n_atoms && ao_start[A + 1] <= s) A++;
  const int s_loc = s - ao_start[A], mu0 = aux_start[A], nmu = nauxA[A];
  float2 *phs = sh;                       // [nRC]
  float2 *cks = phs + nRC;                // [nao_tot][nb]
  float2 *Ckc = cks + nao_tot * nb;       // [TCH32][nmu]
  float2 *Yacc = Ckc + TCH32 * nmu;       // [nb][nmu]
  for (int r = threadIdx.x; r < nRC; r += blockDim.x) phs[r] = PHK[(long long)k * nRC + r];
  for (int e = threadIdx.x; e < nao_tot * nb; e += blockDim.x) cks[e] = ck[(long long)k * nao_tot * nb + e];
  for (int e = threadIdx.x; e < nb * nmu; e += blockDim.x) Yacc[e] = make_float2(0.f, 0.f);
  __syncthreads();
  const long long sR = (long long)nao_tot * nao_tot * naux;
  for (int t0 = 0; t0 < nao_tot; t0 += TCH32) {
    for (int e = threadIdx.x; e < TCH32 * nmu; e += blockDim.x) {
      const int tt = e / nmu, mu = e % nmu, t = t0 + tt;
      float2 acc = make_float2(0.f, 0.f);
      if (t < nao_tot) {
        const float *src = CR + ((long long)s * nao_tot + t) * naux + mu0 + mu;
        for (int r = 0; r < nRC; r++) {
          const float v = src[r * sR];
          acc.x = fmaf(phs[r].x, v, acc.x);
          acc.y = fmaf(phs[r].y, v, acc.y);
        }
      }
      Ckc[e] = acc;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nb * nmu; e += blockDim.x) {
      const int n = e / nmu, mu = e % nmu;
      float2 acc = Yacc[e];
      const int tmax = min(TCH32, nao_tot - t0);
      for (int tt = 0; tt < tmax; tt++) {
        const float2 a = Ckc[tt * nmu + mu], b = cks[(t0 + tt) * nb + n];
        acc.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x));
        acc.y = fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y));
      }
      Yacc[e] = acc;
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < nb * nmu; e += blockDim.x) {
    const int n = e / nmu, mu = e % nmu;
    Y[(((long long)k * nao_max + s_loc) * nb + n) * naux + mu0 + mu] = Yacc[e];
  }
}

// X[(k,i,a)][mu] = C~^mu_{a k, i k} = F(k,k)_{(nv+a) i} + conj(F(k,k)_{i (nv+a)}) in FP32,
// also written as the bf16 pieces of conj(X) (operand B of the exchange GEMM).
__global__ void k_exchange_X32(const float2 *__restrict__ Y, const float2 *__restrict__ ck, int nao_tot, int nb,
                               int nv, int nc, int naux, int nao_max, const int *__restrict__ aux_atom,
                               const int *__restrict__ ao_start, const int *__restrict__ naoA, long long dim,
                               int kmem, float2 *__restrict__ X, PieceBuf Xp) {
  const int k = blockIdx.y;
  const int mu = blockIdx.x * blockDim.x + threadIdx.x;
  if (mu >= naux) return;
  const int A = aux_atom[mu], ao0 = ao_start[A], na = naoA[A];
  const float2 *c = ck + (long long)k * nao_tot * nb;
  const float2 *Yk = Y + (long long)k * nao_max * nb * naux;
  const long long plane = dim * kmem;
  for (int i = 0; i < nv; i++)
    for (int a = 0; a < nc; a++) {
      float2 f1 = make_float2(0.f, 0.f), f2 = make_float2(0.f, 0.f);
      for (int s = 0; s < na; s++) {
        const float2 ca = c[(ao0 + s) * nb + nv + a], y1 = Yk[((long long)s * nb + i) * naux + mu];
        const float2 ci = c[(ao0 + s) * nb + i], y2 = Yk[((long long)s * nb + nv + a) * naux + mu];
        f1.x = fmaf(ca.x, y1.x, fmaf(ca.y, y1.y, f1.x));   // conj(ca) y1
        f1.y = fmaf(ca.x, y1.y, fmaf(-ca.y, y1.x, f1.y));
        f2.x = fmaf(ci.x, y2.x, fmaf(ci.y, y2.y, f2.x));   // conj(ci) y2
        f2.y = fmaf(ci.x, y2.y, fmaf(-ci.y, y2.x, f2.y));
      }
      const float2 x = make_float2(f1.x + f2.x, f1.y - f2.y);
      const long long r = ((long long)k * nv + i) * nc + a;
      X[r * naux + mu] = x;
      Xp.put<float>(plane, r * kmem + mu, x.x, -x.y);
    }
}

// P = X V in FP32, 64 x 64 tiles, written as bf16 pieces (operand A of the exchange GEMM).
// V is V(0), real, at Q = 0 (CPLX = false reads only its real parts) and the complex
// Hermitian sum_R w_R Vbar(R) e^{+iQ.R} otherwise.
template <bool CPLX>
__global__ void __launch_bounds__(256) k_xv0_pieces(int M, int N, const float2 *__restrict__ X,
                                                    const float2 *__restrict__ V0, int kmem, PieceBuf Pp) {
  __shared__ float2 As[16][64];
  __shared__ float2 Bs[16][64];
  const int K = N;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int row0 = blockIdx.y * 64, col0 = blockIdx.x * 64;
  float2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; i++)
#pragma unroll
    for (int j = 0; j < 4; j++) acc[i][j] = make_float2(0.f, 0.f);
  for (int k0 = 0; k0 < K; k0 += 16) {
    for (int e = threadIdx.x; e < 1024; e += 256) {
      const int r = e / 16, kk = e % 16, gr = row0 + r, gk = k0 + kk;
      As[kk][r] = (gr < M && gk < K) ? X[(long long)gr * K + gk] : make_float2(0.f, 0.f);
      const int kb = e / 64, cc = e % 64, gkb = k0 + kb, gc = col0 + cc;
      Bs[kb][cc] = (gkb < K && gc < N) ? V0[(long long)gkb * N + gc] : make_float2(0.f, 0.f);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; kk++) {
      float2 a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; i++) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; j++) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) {
          acc[i][j].x = fmaf(a[i].x, b[j].x, acc[i][j].x);
          acc[i][j].y = fmaf(a[i].y, b[j].x, acc[i][j].y);
          if (CPLX) {
            acc[i][j].x = fmaf(-a[i].y, b[j].y, acc[i][j].x);
            acc[i][j].y = fmaf(a[i].x, b[j].y, acc[i][j].y);
          }
        }
    }
    __syncthreads();
  }
  const long long plane = (long long)M * kmem;
#pragma unroll
  for (int i = 0; i < 4; i++)
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const int r = row0 + ty + 16 * i, cc = col0 + tx + 16 * j;
      if (r >= M || cc >= N) continue;
      Pp.put<float>(plane, (long long)r * kmem + cc, acc[i][j].x, acc[i][j].y);
    }
}

// Exciton momentum Q (pairs: valence at k, conduction at k + Q): relabel the per-k tables so
// that entry k holds the valence columns of k and the conduction columns of k + Q
// (= kdiff(k, qmQ)).  Every Q = 0 formula of the exchange factors, pair projections and
// diagonal then gives the Q blocks (the C~ of §III.A taken at the pair's own points).
__global__ void k_shift_tables(const float2 *__restrict__ Y, const double2 *__restrict__ ck,
                               const double *__restrict__ eqp, int nao_max, int nao_tot, int nb, int nv, int naux,
                               int n1, int n2, int n3, int qmQ, float2 *__restrict__ Yq, double2 *__restrict__ ckq,
                               float2 *__restrict__ ck32q, double *__restrict__ eqpq) {
  const int nk = n1 * n2 * n3;
  const long long ny = (long long)nk * nao_max * nb * naux, nc_ = (long long)nk * nao_tot * nb;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < ny; e += stride) {
    const long long r = e / naux;                       // row (k, s, n)
    const int n = (int)(r % nb), k = (int)(r / ((long long)nao_max * nb));
    const int src = n < nv ? k : kdiff(k, qmQ, n1, n2, n3);
    Yq[e] = Y[e + (long long)(src - k) * nao_max * nb * naux];
  }
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nc_; e += stride) {
    const int n = (int)(e % nb), k = (int)(e / ((long long)nao_tot * nb));
    const int src = n < nv ? k : kdiff(k, qmQ, n1, n2, n3);
    const double2 v = ck[e + (long long)(src - k) * nao_tot * nb];
    ckq[e] = v;
    ck32q[e] = make_float2((float)v.x, (float)v.y);
  }
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < (long long)nk * nb; e += stride) {
    const int n = (int)(e % nb), k = (int)(e / nb);
    const int src = n < nv ? k : kdiff(k, qmQ, n1, n2, n3);
    eqpq[e] = eqp[(long long)src * nb + n];
  }
}

__global__ void k_to_f32(const double2 *__restrict__ src, long long n, float2 *__restrict__ dst) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = make_float2((float)src[i].x, (float)src[i].y);
}

__device__ __forceinline__ float2 fcmulc(float2 a, float2 b) {  // conj(a) * b
  return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

constexpr int MAXB = 8;

// FP32 pair projection of one q-slab.  grid: x = nmu_chunks*(nv+nc), y = q - q0, z = k1.
__global__ void k_proj32(const float2 *__restrict__ Y, const double2 *__restrict__ ck, int nao_tot, int nb, int nv,
                         int nc, int naux, int nao_max, const int *__restrict__ aux_atom,
                         const int *__restrict__ ao_start, const int *__restrict__ naoA, int n1, int n2, int n3,
                         int q0, const int *__restrict__ qlist, int rows, int kmem, PieceBuf Ap,
                         float2 *__restrict__ Mc) {
  extern __shared__ float2 scf[];
  const int nk = n1 * n2 * n3;
  const int nchunk = (naux + blockDim.x - 1) / blockDim.x;
  const int row = blockIdx.x / nchunk;
  const int mu = (blockIdx.x % nchunk) * blockDim.x + threadIdx.x;
  const int qq = blockIdx.y, q = qlist[q0 + qq], k1 = blockIdx.z;
  const int k2 = kdiff(k1, q, n1, n2, n3);
  float2 *c1 = scf, *c2 = scf + nao_tot * nb;
  for (int e = threadIdx.x; e < nao_tot * nb; e += blockDim.x) {
    const double2 a = ck[(long long)k1 * nao_tot * nb + e], b = ck[(long long)k2 * nao_tot * nb + e];
    c1[e] = make_float2((float)a.x, (float)a.y);
    c2[e] = make_float2((float)b.x, (float)b.y);
  }
  __syncthreads();
  if (mu >= naux) return;
  const int A = aux_atom[mu], ao0 = ao_start[A], na = naoA[A];
  const float2 *Y1 = Y + (long long)k1 * nao_max * nb * naux + mu;
  const float2 *Y2 = Y + (long long)k2 * nao_max * nb * naux + mu;
  float2 acc1[MAXB], acc2[MAXB];
#pragma unroll
  for (int j = 0; j < MAXB; j++) acc1[j] = acc2[j] = make_float2(0.f, 0.f);
  if (row < nv) {
    const int i = row;
    for (int s = 0; s < na; s++) {
      const float2 y1 = Y1[((long long)s * nb + i) * naux];
      const float2 ci = c1[(ao0 + s) * nb + i];
#pragma unroll
      for (int j = 0; j < MAXB; j++)
        if (j < nv) {
          const float2 t1 = fcmulc(c2[(ao0 + s) * nb + j], y1);
          const float2 t2 = fcmulc(ci, Y2[((long long)s * nb + j) * naux]);
          acc1[j].x += t1.x; acc1[j].y += t1.y;
          acc2[j].x += t2.x; acc2[j].y += t2.y;
        }
    }
    const long long plane = (long long)rows * kmem;
    const long long out = (long long)qq * 2 * Ap.np * plane + (long long)(k1 * nv + i) * nv * kmem + mu;
#pragma unroll
    for (int j = 0; j < MAXB; j++)
      if (j < nv) Ap.put<float>(plane, out + (long long)j * kmem, acc1[j].x + acc2[j].x, acc1[j].y - acc2[j].y);
  } else {
    const int a = row - nv;
    for (int s = 0; s < na; s++) {
      const float2 y1 = Y1[((long long)s * nb + nv + a) * naux];
      const float2 ca = c1[(ao0 + s) * nb + nv + a];
#pragma unroll
      for (int b = 0; b < MAXB; b++)
        if (b < nc) {
          const float2 t1 = fcmulc(ca, Y2[((long long)s * nb + nv + b) * naux]);
          const float2 t2 = fcmulc(c2[(ao0 + s) * nb + nv + b], y1);
          acc1[b].x += t1.x; acc1[b].y += t1.y;
          acc2[b].x += t2.x; acc2[b].y += t2.y;
        }
    }
    float2 *out = Mc + ((((long long)qq * nk + k1) * nc + a) * nc) * naux + mu;
#pragma unroll
    for (int b = 0; b < MAXB; b++)
      if (b < nc) out[(long long)b * naux] = make_float2(acc1[b].x + acc2[b].x, acc1[b].y - acc2[b].y);
  }
}

// Conduction-valence projections of one q-slab for the coupling block (FP32).  grid: x =
// nmu_chunks * 2 nc, y = q - q0, z = k1.  Row r < nc: M1 row b = r, C~_{b k2, i k1} for the
// valence i, written as bf16 pieces (GEMM operand A, row (k1, b, i)); else M2 row a = r - nc,
// C~_{a k1, j k2}, FP32 (row (k1, a, j)).  F as in k_proj32.
__global__ void k_proj_cv32(const float2 *__restrict__ Y, const double2 *__restrict__ ck, int nao_tot, int nb, int nv,
                            int nc, int naux, int nao_max, const int *__restrict__ aux_atom,
                            const int *__restrict__ ao_start, const int *__restrict__ naoA, int n1, int n2, int n3,
                            int q0, const int *__restrict__ qlist, int rowsB, int kmem, PieceBuf Ap,
                            float2 *__restrict__ M2) {
  extern __shared__ float2 scf[];
  const int nk = n1 * n2 * n3;
  const int nchunk = (naux + blockDim.x - 1) / blockDim.x;
  const int row = blockIdx.x / nchunk;
  const int mu = (blockIdx.x % nchunk) * blockDim.x + threadIdx.x;
  const int qq = blockIdx.y, q = qlist[q0 + qq], k1 = blockIdx.z;
  const int k2 = kdiff(k1, q, n1, n2, n3);
  float2 *c1 = scf, *c2 = scf + nao_tot * nb;
  for (int e = threadIdx.x; e < nao_tot * nb; e += blockDim.x) {
    const double2 a = ck[(long long)k1 * nao_tot * nb + e], b = ck[(long long)k2 * nao_tot * nb + e];
    c1[e] = make_float2((float)a.x, (float)a.y);
    c2[e] = make_float2((float)b.x, (float)b.y);
  }
  __syncthreads();
  if (mu >= naux) return;
  const int A = aux_atom[mu], ao0 = ao_start[A], na = naoA[A];
  const float2 *Y1 = Y + (long long)k1 * nao_max * nb * naux + mu;
  const float2 *Y2 = Y + (long long)k2 * nao_max * nb * naux + mu;
  const bool first = row < nc;
  const int cb = nv + (first ? row : row - nc);
  const float2 *cc = first ? c2 : c1, *cv = first ? c1 : c2;   // bra conduction, valence kets
  const float2 *Yv = first ? Y1 : Y2, *Yc = first ? Y2 : Y1;
  float2 acc1[MAXB], acc2[MAXB];
#pragma unroll
  for (int j = 0; j < MAXB; j++) acc1[j] = acc2[j] = make_float2(0.f, 0.f);
  for (int s = 0; s < na; s++) {
    const float2 cs = cc[(ao0 + s) * nb + cb];
    const float2 yc = Yc[((long long)s * nb + cb) * naux];
#pragma unroll
    for (int j = 0; j < MAXB; j++)
      if (j < nv) {
        const float2 t1 = fcmulc(cs, Yv[((long long)s * nb + j) * naux]);
        const float2 t2 = fcmulc(cv[(ao0 + s) * nb + j], yc);
        acc1[j].x += t1.x; acc1[j].y += t1.y;
        acc2[j].x += t2.x; acc2[j].y += t2.y;
      }
  }
  if (first) {
    const long long plane = (long long)rowsB * kmem;
    const long long out = (long long)qq * 2 * Ap.np * plane + ((long long)(k1 * nc + row) * nv) * kmem + mu;
#pragma unroll
    for (int j = 0; j < MAXB; j++)
      if (j < nv) Ap.put<float>(plane, out + (long long)j * kmem, acc1[j].x + acc2[j].x, acc1[j].y - acc2[j].y);
  } else {
    float2 *out = M2 + ((((long long)qq * nk + k1) * nc + (row - nc)) * nv) * naux + mu;
#pragma unroll
    for (int j = 0; j < MAXB; j++)
      if (j < nv) out[(long long)j * naux] = make_float2(acc1[j].x + acc2[j].x, acc1[j].y - acc2[j].y);
  }
}

// dst[pp][r][k] pieces of src [rows][naux] (FP32 complex, no conjugate).
__global__ void k_pieces_f32(const float2 *__restrict__ src, long long rows, int naux, int kmem, PieceBuf dst) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows * naux) return;
  const long long r = e / naux;
  const int k = (int)(e % naux);
  const float2 v = src[e];
  dst.put<float>(rows * kmem, r * kmem + k, v.x, v.y);
}

// ---- matrix-free products H x (no H stored) ---------------------------------------------
// The exchange part (alpha/N_k) X V X^dagger x in three small passes, the diagonal, and per
// q-slab the direct blocks D = -(1/N_k) T M_cc^T formed as for H and applied at once.
constexpr int MF_RB = 128;  // rows of X per partial of X^dagger x

// zp[p][chunk][mu] = sum over the chunk's rows r of conj(X[r][mu]) x[p][r]
__global__ void k_mf_xh(const float2 *__restrict__ X, long long dim, int naux, const double2 *__restrict__ x,
                        long long xs, int nch, double2 *__restrict__ zp) {
  const int ch = blockIdx.x, p = blockIdx.y;
  const long long r0 = (long long)ch * MF_RB, r1 = min(dim, r0 + MF_RB);
  for (int mu = threadIdx.x; mu < naux; mu += blockDim.x) {
    double sr = 0.0, si = 0.0;
    for (long long r = r0; r < r1; r++) {
      const float2 a = X[r * naux + mu];
      const double2 v = x[p * xs + r];
      sr += (double)a.x * v.x + (double)a.y * v.y;
      si += (double)a.x * v.y - (double)a.y * v.x;
    }
    zp[((long long)p * nch + ch) * naux + mu] = make_double2(sr, si);
  }
}

// z2[p][mu] = sum_nu V[mu][nu] z[p][nu], z[p][nu] = sum_chunk zp[p][chunk][nu]
__global__ void k_mf_zv(const double2 *__restrict__ zp, int nch, int naux, const float2 *__restrict__ V,
                        double2 *__restrict__ z2) {
  extern __shared__ double2 zs[];
  const int p = blockIdx.x;
  for (int nu = threadIdx.x; nu < naux; nu += blockDim.x) {
    double sr = 0.0, si = 0.0;
    for (int ch = 0; ch < nch; ch++) {
      const double2 v = zp[((long long)p * nch + ch) * naux + nu];
      sr += v.x;
      si += v.y;
    }
    zs[nu] = make_double2(sr, si);
  }
  __syncthreads();
  for (int mu = threadIdx.x; mu < naux; mu += blockDim.x) {
    double sr = 0.0, si = 0.0;
    for (int nu = 0; nu < naux; nu++) {
      const float2 v = V[(long long)mu * naux + nu];
      const double2 z = zs[nu];
      sr += (double)v.x * z.x - (double)v.y * z.y;
      si += (double)v.x * z.y + (double)v.y * z.x;
    }
    z2[(long long)p * naux + mu] = make_double2(sr, si);
  }
}

// W[p][r] = (E_c - E_v)[r] x[p][r] + (alpha/N_k) sum_mu X[r][mu] z2[p][mu]  (a warp per row)
__global__ void k_mf_xv(const float2 *__restrict__ X, long long dim, int naux, const double2 *__restrict__ z2,
                        const double *__restrict__ eqp, int nv, int nc, double scale, const double2 *__restrict__ x,
                        long long xs, int n_pol, double2 *__restrict__ W) {
  const long long r = (long long)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x % 32;
  if (r >= dim) return;
  const int nvc = nv * nc, nb = nv + nc;
  const long long k = r / nvc;
  const int ia = (int)(r % nvc), i = ia / nc, a = ia % nc;
  const double de = eqp[k * nb + nv + a] - eqp[k * nb + i];
  for (int p = 0; p < n_pol; p++) {
    double sr = 0.0, si = 0.0;
    for (int mu = lane; mu < naux; mu += 32) {
      const float2 xv = X[r * naux + mu];
      const double2 z = z2[(long long)p * naux + mu];
      sr += (double)xv.x * z.x - (double)xv.y * z.y;
      si += (double)xv.x * z.y + (double)xv.y * z.x;
    }
    for (int o = 16; o > 0; o >>= 1) {
      sr += __shfl_xor_sync(0xffffffffu, sr, o);
      si += __shfl_xor_sync(0xffffffffu, si, o);
    }
    if (lane == 0) {
      const double2 v = x[p * xs + r];
      W[(long long)p * dim + r] = make_double2(de * v.x + scale * sr, de * v.y + scale * si);
    }
  }
}

constexpr int G2CH = 32;

// Direct blocks of one q-slab applied without storing them.  Per pair (k1, q): D[ia][jb] =
// -(1/N_k) sum_nu T[(k1,i,j)][nu] M_cc[(k1,a,b)][nu] in shared memory (as k_g2_32 forms it),
// then fwd[p][qq][k1] = D x[p][k2] and, for a block with a mirror (q != -q),
// bwd[p][qq][k2] = D^dagger x[p][k1] (else 0).
__global__ void __launch_bounds__(256) k_g2mv_32(const float2 *__restrict__ T, const float2 *__restrict__ Mc,
                                                 int nv, int nc, int naux, int n1, int n2, int n3, int q0,
                                                 const int *__restrict__ qlist, int rows, const double2 *__restrict__ x,
                                                 long long xs, int n_pol, int nqs, double2 *__restrict__ fwd,
                                                 double2 *__restrict__ bwd) {
  extern __shared__ float2 sg[];
  const int nk = n1 * n2 * n3;
  const int k1 = blockIdx.x, qq = blockIdx.y, q = qlist[q0 + qq];
  const int k2 = kdiff(k1, q, n1, n2, n3);
  const bool mirror = !q_self_conjugate(q, n1, n2, n3);
  const int nvc = nv * nc, nvv = nv * nv, ncc = nc * nc;
  float2 *sT = sg, *sM = sT + nvv * G2CH, *sD = sM + ncc * G2CH;
  const float2 *Tq = T + (long long)qq * rows * naux + (long long)k1 * nvv;
  const float2 *Mk = Mc + ((long long)qq * nk + k1) * ncc * naux;
  const int nout = nvc * nvc;
  constexpr int MAXO = 16;
  float2 ad[MAXO];
#pragma unroll
  for (int t = 0; t < MAXO; t++) ad[t] = make_float2(0.f, 0.f);
  for (int n0 = 0; n0 < naux; n0 += G2CH) {
    const int nn = min(G2CH, naux - n0);
    for (int e = threadIdx.x; e < (nvv + ncc) * G2CH; e += blockDim.x) {
      const int r = e / G2CH, u = e % G2CH;
      float2 v = make_float2(0.f, 0.f);
      if (u < nn) v = r < nvv ? Tq[(long long)(n0 + u) * rows + r] : Mk[(long long)(r - nvv) * naux + n0 + u];
      sg[e] = v;
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < MAXO; t++) {
      const int o = threadIdx.x + t * blockDim.x;
      if (o < nout) {
        const int ia = o / nvc, jb = o % nvc;
        const int i = ia / nc, a = ia % nc, j = jb / nc, b = jb % nc;
        const float2 *pt = sT + (i * nv + j) * G2CH, *pm = sM + (a * nc + b) * G2CH;
        float xr = ad[t].x, xi = ad[t].y;
        for (int u = 0; u < nn; u++) {
          xr = fmaf(pt[u].x, pm[u].x, fmaf(-pt[u].y, pm[u].y, xr));
          xi = fmaf(pt[u].x, pm[u].y, fmaf(pt[u].y, pm[u].x, xi));
        }
        ad[t] = make_float2(xr, xi);
      }
    }
    __syncthreads();
  }
  const float inv = 1.0f / nk;
#pragma unroll
  for (int t = 0; t < MAXO; t++) {
    const int o = threadIdx.x + t * blockDim.x;
    if (o < nout) sD[o] = make_float2(-inv * ad[t].x, -inv * ad[t].y);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 2 * n_pol * nvc; e += blockDim.x) {
    const int side = e / (n_pol * nvc), p = (e / nvc) % n_pol, r = e % nvc;
    double sr = 0.0, si = 0.0;
    if (side == 0) {  // row ia = r of D times x[k2]
      const double2 *xv = x + p * xs + (long long)k2 * nvc;
      for (int jb = 0; jb < nvc; jb++) {
        const float2 d = sD[r * nvc + jb];
        const double2 v = xv[jb];
        sr += (double)d.x * v.x - (double)d.y * v.y;
        si += (double)d.x * v.y + (double)d.y * v.x;
      }
      fwd[(((long long)p * nqs + qq) * nk + k1) * nvc + r] = make_double2(sr, si);
    } else {          // column jb = r of D, conjugated, times x[k1]
      if (mirror) {
        const double2 *xv = x + p * xs + (long long)k1 * nvc;
        for (int ia = 0; ia < nvc; ia++) {
          const float2 d = sD[ia * nvc + r];
          const double2 v = xv[ia];
          sr += (double)d.x * v.x + (double)d.y * v.y;
          si += (double)d.x * v.y - (double)d.y * v.x;
        }
      }
      bwd[(((long long)p * nqs + qq) * nk + k2) * nvc + r] = make_double2(sr, si);
    }
  }
}

// W[p][k nvc + r] += sum over the slab's nq transfers of fwd + bwd (fixed order)
__global__ void k_mf_reduce(const double2 *__restrict__ fwd, const double2 *__restrict__ bwd, int nq, int nqs,
                            int nk, int nvc, int n_pol, double2 *__restrict__ W) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long per = (long long)nk * nvc;
  if (e >= n_pol * per) return;
  const int p = (int)(e / per);
  const long long kr = e % per;
  double2 acc = W[e];
  for (int qq = 0; qq < nq; qq++) {
    const double2 f = fwd[((long long)p * nqs + qq) * per + kr], b = bwd[((long long)p * nqs + qq) * per + kr];
    acc.x += f.x + b.x;
    acc.y += f.y + b.y;
  }
  W[e] = acc;
}

// hmax[0] = 2 max |E| over the band window (scale of the early-stop threshold)
__global__ void k_mf_hmax(const double *__restrict__ eqp, long long n, double *__restrict__ hmax) {
  __shared__ double red[256];
  double m = 0.0;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, fabs(eqp[i]));
  red[threadIdx.x] = m;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) hmax[0] = 2.0 * red[0];
}

// B block (k1, k2 = k1 - q) += -(1/N_k) sum_nu T1[(k1,b,i)][nu] M2[(k1,a,j)][nu], and the same
// value at the transposed position (k2, k1) (B is symmetric).  T1 [q][nu][rowsB].
__global__ void __launch_bounds__(256) k_g2c_32(const float2 *__restrict__ T, const float2 *__restrict__ M2, int nv,
                                                int nc, int naux, int n1, int n2, int n3, int q0,
                                                const int *__restrict__ qlist, int rowsB, long long dim,
                                                float2 *__restrict__ B) {
  extern __shared__ float2 sg[];
  const int nk = n1 * n2 * n3;
  const int k1 = blockIdx.x, qq = blockIdx.y, q = qlist[q0 + qq];
  const int k2 = kdiff(k1, q, n1, n2, n3);
  const bool mirror = !q_self_conjugate(q, n1, n2, n3);
  const int nvc = nv * nc;
  float2 *sT = sg, *sM = sT + nvc * G2CH;
  const float2 *Tq = T + (long long)qq * rowsB * naux + (long long)k1 * nvc;
  const float2 *Mk = M2 + ((long long)qq * nk + k1) * nvc * naux;
  const int nout = nvc * nvc;
  constexpr int MAXO = 16;
  float2 ad[MAXO];
#pragma unroll
  for (int t = 0; t < MAXO; t++) ad[t] = make_float2(0.f, 0.f);
  for (int n0 = 0; n0 < naux; n0 += G2CH) {
    const int nn = min(G2CH, naux - n0);
    for (int e = threadIdx.x; e < 2 * nvc * G2CH; e += blockDim.x) {
      const int r = e / G2CH, u = e % G2CH;
      float2 v = make_float2(0.f, 0.f);
      if (u < nn) v = r < nvc ? Tq[(long long)(n0 + u) * rowsB + r] : Mk[(long long)(r - nvc) * naux + n0 + u];
      sg[e] = v;
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < MAXO; t++) {
      const int o = threadIdx.x + t * blockDim.x;
      if (o < nout) {
        const int ia = o / nvc, jb = o % nvc;
        const int i = ia / nc, a = ia % nc, j = jb / nc, b = jb % nc;
        const float2 *pt = sT + (b * nv + i) * G2CH, *pm = sM + (a * nv + j) * G2CH;
        float xr = ad[t].x, xi = ad[t].y;
        for (int u = 0; u < nn; u++) {
          xr = fmaf(pt[u].x, pm[u].x, fmaf(-pt[u].y, pm[u].y, xr));
          xi = fmaf(pt[u].x, pm[u].y, fmaf(pt[u].y, pm[u].x, xi));
        }
        ad[t] = make_float2(xr, xi);
      }
    }
    __syncthreads();
  }
  const float inv = 1.0f / nk;
#pragma unroll
  for (int t = 0; t < MAXO; t++) {
    const int o = threadIdx.x + t * blockDim.x;
    if (o < nout) {
      const int ia = o / nvc, jb = o % nvc;
      float2 *hp = B + ((long long)k1 * nvc + ia) * dim + (long long)k2 * nvc + jb;
      const float2 hx = *hp;
      *hp = make_float2(fmaf(-inv, ad[t].x, hx.x), fmaf(-inv, ad[t].y, hx.y));
      if (mirror) {
        float2 *hm = B + ((long long)k2 * nvc + jb) * dim + (long long)k1 * nvc + ia;
        const float2 mx = *hm;
        *hm = make_float2(fmaf(-inv, ad[t].x, mx.x), fmaf(-inv, ad[t].y, mx.y));
      }
    }
  }
}

// H block (k1, k2 = k1 - q) += -(1/N_k) sum_nu T[(k1,i,j)][nu] M_cc[(k1,a,b)][nu] (+ diagonal).
__global__ void __launch_bounds__(256) k_g2_32(const float2 *__restrict__ T, const float2 *__restrict__ Mc,
                                               const double *__restrict__ eqp, int nv, int nc, int naux, int n1,
                                               int n2, int n3, int q0, const int *__restrict__ qlist, int rows,
                                               long long dim, float2 *__restrict__ H, double2 *__restrict__ H64) {
  extern __shared__ float2 sg[];
  const int nk = n1 * n2 * n3;
  const int k1 = blockIdx.x, qq = blockIdx.y, q = qlist[q0 + qq];
  const int k2 = kdiff(k1, q, n1, n2, n3);
  const bool mirror = !q_self_conjugate(q, n1, n2, n3);
  const int nvc = nv * nc, nvv = nv * nv, ncc = nc * nc, nb = nv + nc;
  float2 *sT = sg, *sM = sT + nvv * G2CH;
  const float2 *Tq = T + (long long)qq * rows * naux + (long long)k1 * nvv;  // T[q][nu][row]
  const float2 *Mk = Mc + ((long long)qq * nk + k1) * ncc * naux;
  const int nout = nvc * nvc;
  constexpr int MAXO = 16;
  float2 ad[MAXO];
#pragma unroll
  for (int t = 0; t < MAXO; t++) ad[t] = make_float2(0.f, 0.f);
  for (int n0 = 0; n0 < naux; n0 += G2CH) {
    const int nn = min(G2CH, naux - n0);
    for (int e = threadIdx.x; e < (nvv + ncc) * G2CH; e += blockDim.x) {
      const int r = e / G2CH, u = e % G2CH;
      float2 v = make_float2(0.f, 0.f);
      if (u < nn) v = r < nvv ? Tq[(long long)(n0 + u) * rows + r] : Mk[(long long)(r - nvv) * naux + n0 + u];
      sg[e] = v;
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < MAXO; t++) {
      const int o = threadIdx.x + t * blockDim.x;
      if (o < nout) {
        const int ia = o / nvc, jb = o % nvc;
        const int i = ia / nc, a = ia % nc, j = jb / nc, b = jb % nc;
        const float2 *pt = sT + (i * nv + j) * G2CH, *pm = sM + (a * nc + b) * G2CH;
        float xr = ad[t].x, xi = ad[t].y;
        for (int u = 0; u < nn; u++) {
          xr = fmaf(pt[u].x, pm[u].x, fmaf(-pt[u].y, pm[u].y, xr));
          xi = fmaf(pt[u].x, pm[u].y, fmaf(pt[u].y, pm[u].x, xi));
        }
        ad[t] = make_float2(xr, xi);
      }
    }
    __syncthreads();
  }
  const double inv = 1.0 / nk;
  const float invf = (float)inv;
#pragma unroll
  for (int t = 0; t < MAXO; t++) {
    const int o = threadIdx.x + t * blockDim.x;
    if (o < nout) {
      const int ia = o / nvc, jb = o % nvc;
      const int i = ia / nc, a = ia % nc;
      const long long ih = ((long long)k1 * nvc + ia) * dim + (long long)k2 * nvc + jb;
      const long long im = ((long long)k2 * nvc + jb) * dim + (long long)k1 * nvc + ia;
      if (H64) {  // complex128 H: the contribution and the diagonal added in FP64
        double2 hv = H64[ih];
        hv.x -= inv * (double)ad[t].x;
        hv.y -= inv * (double)ad[t].y;
        if (q == 0 && ia == jb) hv.x += eqp[(long long)k1 * nb + nv + a] - eqp[(long long)k1 * nb + i];
        H64[ih] = hv;
        if (mirror) {
          double2 mv = H64[im];
          mv.x -= inv * (double)ad[t].x;
          mv.y += inv * (double)ad[t].y;
          H64[im] = mv;
        }
        continue;
      }
      float2 *hp = H + ih;
      const float2 hx = *hp;
      float2 hv = make_float2(fmaf(-invf, ad[t].x, hx.x), fmaf(-invf, ad[t].y, hx.y));
      if (q == 0 && ia == jb)  // the diagonal sums in FP64 (one element per row)
        hv.x = (float)((double)hx.x - inv * (double)ad[t].x + eqp[(long long)k1 * nb + nv + a] -
                       eqp[(long long)k1 * nb + i]);
      *hp = hv;
      if (mirror) {  // block (k2, k1) gets the conjugate of the direct contribution
        float2 *hm = H + im;
        const float2 mx = *hm;
        *hm = make_float2(fmaf(-invf, ad[t].x, mx.x), fmaf(invf, ad[t].y, mx.y));
      }
    }
  }
}


// Register-blocked projection: one thread per ABF mu of one pair computes every M_vv and
// M_cc element of that mu; both LRI terms go into one accumulator,
//   M_vv[i][j] = sum_s conj(c2_sj) Y1_si + c1_si conj(Y2_sj),
//   M_cc[a][b] = sum_s conj(c1_sa) Y2_sb + c2_sb conj(Y1_sa)   (band indices in the window).
// M_cc is written [q][k1][a b][nu] with rows of naux (mc_pad = 0) or of mc_pad (> naux, for the
// fused kernel's tensor map) elements; the stores of one (a, b) over a warp's mu coalesce.
// grid: x = q - q0, y = k1; block: mu chunk (blockDim >= 32), loop over mu.
template <int NV, int NC>
__device__ __forceinline__ void proj_t_body(const float2 *__restrict__ Y, const double2 *__restrict__ ck, int nao_tot,
                                            int naux, int nao_max, const int *__restrict__ aux_atom,
                                            const int *__restrict__ ao_start, const int *__restrict__ naoA, int n1,
                                            int n2, int n3, int q0, const int *__restrict__ qlist, int rows,
                                            int kmem, PieceBuf Ap, float2 *__restrict__ Mc, int mc_pad, int qq,
                                            int k1) {
  constexpr int NB = NV + NC;
  extern __shared__ float2 scf[];
  const int nk = n1 * n2 * n3;
  const int q = qlist[q0 + qq];
  const int k2 = kdiff(k1, q, n1, n2, n3);
  float2 *c1 = scf, *c2 = scf + nao_tot * NB;
  for (int e = threadIdx.x; e < nao_tot * NB; e += blockDim.x) {
    const double2 a = ck[(long long)k1 * nao_tot * NB + e], b = ck[(long long)k2 * nao_tot * NB + e];
    c1[e] = make_float2((float)a.x, (float)a.y);
    c2[e] = make_float2((float)b.x, (float)b.y);
  }
  __syncthreads();
  const long long plane = (long long)rows * kmem;
  const int mrow = mc_pad ? mc_pad : naux;  // M_cc row length
  for (int mu = threadIdx.x; mu < naux; mu += blockDim.x) {
    const int A = aux_atom[mu], ao0 = ao_start[A], na = naoA[A];
    const float2 *Y1 = Y + (long long)k1 * nao_max * NB * naux + mu;
    const float2 *Y2 = Y + (long long)k2 * nao_max * NB * naux + mu;
    float2 mv[NV][NV], mc[NC][NC];
#pragma unroll
    for (int i = 0; i < NV; i++)
#pragma unroll
      for (int j = 0; j < NV; j++) mv[i][j] = make_float2(0.f, 0.f);
#pragma unroll
    for (int a = 0; a < NC; a++)
#pragma unroll
      for (int b = 0; b < NC; b++) mc[a][b] = make_float2(0.f, 0.f);
    for (int s = 0; s < na; s++) {
      float2 y1[NB], y2[NB];
#pragma unroll
      for (int n = 0; n < NB; n++) {
        y1[n] = Y1[((long long)s * NB + n) * naux];
        y2[n] = Y2[((long long)s * NB + n) * naux];
      }
      const float2 *cs1 = c1 + (ao0 + s) * NB, *cs2 = c2 + (ao0 + s) * NB;
#pragma unroll
      for (int i = 0; i < NV; i++) {
        const float2 a1 = cs1[i];
#pragma unroll
        for (int j = 0; j < NV; j++) {
          const float2 b2 = cs2[j];
          // conj(b2) y1[i] + a1 conj(y2[j])
          float xr = mv[i][j].x, xi = mv[i][j].y;
          xr = fmaf(b2.x, y1[i].x, fmaf(b2.y, y1[i].y, xr));
          xi = fmaf(b2.x, y1[i].y, fmaf(-b2.y, y1[i].x, xi));
          xr = fmaf(a1.x, y2[j].x, fmaf(a1.y, y2[j].y, xr));
          xi = fmaf(a1.y, y2[j].x, fmaf(-a1.x, y2[j].y, xi));
          mv[i][j] = make_float2(xr, xi);
        }
      }
#pragma unroll
      for (int a = 0; a < NC; a++) {
        const float2 a1 = cs1[NV + a];
#pragma unroll
        for (int b = 0; b < NC; b++) {
          const float2 b2 = cs2[NV + b];
          // conj(a1) y2[b] + b2 conj(y1[a])
          float xr = mc[a][b].x, xi = mc[a][b].y;
          xr = fmaf(a1.x, y2[NV + b].x, fmaf(a1.y, y2[NV + b].y, xr));
          xi = fmaf(a1.x, y2[NV + b].y, fmaf(-a1.y, y2[NV + b].x, xi));
          xr = fmaf(b2.x, y1[NV + a].x, fmaf(b2.y, y1[NV + a].y, xr));
          xi = fmaf(b2.y, y1[NV + a].x, fmaf(-b2.x, y1[NV + a].y, xi));
          mc[a][b] = make_float2(xr, xi);
        }
      }
    }
    const long long out = (long long)qq * 2 * Ap.np * plane + (long long)k1 * NV * NV * kmem + mu;
#pragma unroll
    for (int i = 0; i < NV; i++)
#pragma unroll
      for (int j = 0; j < NV; j++)
        Ap.put<float>(plane, out + (long long)(i * NV + j) * kmem, mv[i][j].x, mv[i][j].y);
    float2 *mo = Mc + (((long long)qq * nk + k1) * NC * NC) * mrow + mu;
#pragma unroll
    for (int a = 0; a < NC; a++)
#pragma unroll
      for (int b = 0; b < NC; b++) mo[(long long)(a * NC + b) * mrow] = mc[a][b];
  }
}

template <int NV, int NC>
__global__ void __launch_bounds__(160) k_proj32_t(const float2 *__restrict__ Y, const double2 *__restrict__ ck,
                                                  int nao_tot, int naux, int nao_max,
                                                  const int *__restrict__ aux_atom, const int *__restrict__ ao_start,
                                                  const int *__restrict__ naoA, int n1, int n2, int n3, int q0,
                                                  const int *__restrict__ qlist, int rows, int kmem, PieceBuf Ap,
                                                  float2 *__restrict__ Mc, int mc_pad) {
  proj_t_body<NV, NC>(Y, ck, nao_tot, naux, nao_max, aux_atom, ao_start, naoA, n1, n2, n3, q0, qlist, rows, kmem, Ap,
                      Mc, mc_pad, blockIdx.x, blockIdx.y);
}

// The projections of several systems' q-slabs in one launch (the batched assembly's work
// list): group g owns blocks blk0[g] .. blk0[g + 1] - 1, block b of a group being the pair
// block (qq = b % nq, k1 = b / nq) of that system's slab.
constexpr int MAXPG = 16;
struct ProjGroup {
  const float2 *Y;
  const double2 *ck;
  int nao_tot, naux, nao_max;
  const int *aux_atom, *ao_start, *naoA;
  int n1, n2, n3, q0;
  const int *qlist;
  int rows, kmem;
  PieceBuf Ap;
  float2 *Mc;
  int mc_pad, nq;
};
struct ProjGroups {
  ProjGroup g[MAXPG];
  long long blk0[MAXPG + 1];
  int n;
};

template <int NV, int NC>
__global__ void __launch_bounds__(160) k_proj32_t_grouped(const __grid_constant__ ProjGroups G) {
  int g = 0;
  const long long b = blockIdx.x;
  while (g + 1 < G.n && b >= G.blk0[g + 1]) g++;
  const ProjGroup a = G.g[g];
  const long long lb = b - G.blk0[g];
  proj_t_body<NV, NC>(a.Y, a.ck, a.nao_tot, a.naux, a.nao_max, a.aux_atom, a.ao_start, a.naoA, a.n1, a.n2, a.n3, a.q0,
                      a.qlist, a.rows, a.kmem, a.Ap, a.Mc, a.mc_pad, (int)(lb % a.nq), (int)(lb / a.nq));
}

// Second contraction per pair: the pair's T rows (R consecutive elements per column nu of the
// column-major T) and M_cc rows (C x N_aux, contiguous) are copied to shared memory in one
// vectorised asynchronous sweep; thread
// (r, c) then owns the 2x2 outputs rows (i,j) in {2r, 2r+1}, columns (a,b) in {2c, 2c+1}
// of D = T M_cc^T.  H gets D's contribution at (k1, k2) and its conjugate at (k2, k1).
template <int NV, int NC>
__device__ __forceinline__ void g2_t_body(const float2 *__restrict__ T, const float2 *__restrict__ Mc,
                                          const double *__restrict__ eqp, int naux, int n1, int n2, int n3, int q0,
                                          const int *__restrict__ qlist, int rows, long long dim,
                                          float2 *__restrict__ H, double2 *__restrict__ H64, int k1, int qq) {
  constexpr int R = NV * NV, C = NC * NC, TR = (R + 1) / 2, TCC = (C + 1) / 2, NVC = NV * NC, NB = NV + NC;
  extern __shared__ float2 sg2[];
  float2 *sT = sg2, *sM = sg2 + R * naux;
  const int nk = n1 * n2 * n3;
  const int q = qlist[q0 + qq];
  const int k2 = kdiff(k1, q, n1, n2, n3);
  const bool mirror = !q_self_conjugate(q, n1, n2, n3);
  static_assert(R % 2 == 0, "the pair's T rows are copied in 16-byte pieces");
  const float2 *Tq = T + (long long)qq * rows * naux + (long long)k1 * R;  // T[q][nu][row]
  const float2 *Mk = Mc + ((long long)qq * nk + k1) * C * naux;
  // asynchronous 16-byte global->shared copies: every load of the sweep is in flight at once.
  // sT[nu][r] holds the pair's R rows of T per column nu (R consecutive elements in memory).
  {
    float4 *st4 = reinterpret_cast<float4 *>(sT);
    for (int e = threadIdx.x; e < naux * (R / 2); e += blockDim.x) {
      const int nu = e / (R / 2), h = e % (R / 2);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(tc::smem_u32(st4 + e)),
                   "l"(reinterpret_cast<const float4 *>(Tq + (long long)nu * rows) + h)
                   : "memory");
    }
  }
  if ((naux & 1) == 0) {
    const float4 *m4 = reinterpret_cast<const float4 *>(Mk);
    float4 *sm4 = reinterpret_cast<float4 *>(sM);
    for (int e = threadIdx.x; e < C * naux / 2; e += blockDim.x)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(tc::smem_u32(sm4 + e)), "l"(m4 + e) : "memory");
  } else {
    for (int e = threadIdx.x; e < C * naux; e += blockDim.x) sM[e] = Mk[e];
  }
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
  __syncthreads();
  const double inv = 1.0 / nk;
  const float invf = (float)inv;
  for (int w = threadIdx.x; w < TR * TCC; w += blockDim.x) {
    const int tr = w / TCC, tc = w % TCC;
    const int r0 = 2 * tr, r1 = min(2 * tr + 1, R - 1), m0 = 2 * tc, m1 = min(2 * tc + 1, C - 1);
    const float2 *pt0 = sT + r0, *pt1 = sT + r1, *pm0 = sM + m0 * naux, *pm1 = sM + m1 * naux;
    float2 acc[2][2];
#pragma unroll
    for (int x = 0; x < 2; x++)
#pragma unroll
      for (int y = 0; y < 2; y++) acc[x][y] = make_float2(0.f, 0.f);
    for (int u = 0; u < naux; u++) {
      const float2 tt[2] = {pt0[u * R], pt1[u * R]}, mm[2] = {pm0[u], pm1[u]};
#pragma unroll
      for (int x = 0; x < 2; x++)
#pragma unroll
        for (int y = 0; y < 2; y++) {
          acc[x][y].x = fmaf(tt[x].x, mm[y].x, fmaf(-tt[x].y, mm[y].y, acc[x][y].x));
          acc[x][y].y = fmaf(tt[x].x, mm[y].y, fmaf(tt[x].y, mm[y].x, acc[x][y].y));
        }
    }
#pragma unroll
    for (int x = 0; x < 2; x++)
#pragma unroll
      for (int y = 0; y < 2; y++) {
        const int ij = 2 * tr + x, ab = 2 * tc + y;
        if (ij >= R || ab >= C) continue;
        const int i = ij / NV, j = ij % NV, a = ab / NC, b = ab % NC;
        const int ia = i * NC + a, jb = j * NC + b;
        const long long ih = ((long long)k1 * NVC + ia) * dim + (long long)k2 * NVC + jb;
        const long long im = ((long long)k2 * NVC + jb) * dim + (long long)k1 * NVC + ia;
        if (H64) {  // complex128 H: the contribution and the diagonal added in FP64
          double2 hv = H64[ih];
          hv.x -= inv * (double)acc[x][y].x;
          hv.y -= inv * (double)acc[x][y].y;
          if (q == 0 && ia == jb) hv.x += eqp[(long long)k1 * NB + NV + a] - eqp[(long long)k1 * NB + i];
          H64[ih] = hv;
          if (mirror) {
            double2 mv = H64[im];
            mv.x -= inv * (double)acc[x][y].x;
            mv.y += inv * (double)acc[x][y].y;
            H64[im] = mv;
          }
          continue;
        }
        float2 *hp = H + ih;
        const float2 hx = *hp;
        float2 hv = make_float2(fmaf(-invf, acc[x][y].x, hx.x), fmaf(-invf, acc[x][y].y, hx.y));
        if (q == 0 && ia == jb)  // the diagonal sums in FP64 (one element per row)
          hv.x = (float)((double)hx.x - inv * (double)acc[x][y].x + eqp[(long long)k1 * NB + NV + a] -
                         eqp[(long long)k1 * NB + i]);
        *hp = hv;
        if (mirror) {
          float2 *hm = H + im;
          const float2 mx = *hm;
          *hm = make_float2(fmaf(-invf, acc[x][y].x, mx.x), fmaf(invf, acc[x][y].y, mx.y));
        }
      }
  }
}

template <int NV, int NC>
__global__ void __launch_bounds__(256) k_g2_32_t(const float2 *__restrict__ T, const float2 *__restrict__ Mc,
                                                 const double *__restrict__ eqp, int naux, int n1, int n2, int n3,
                                                 int q0, const int *__restrict__ qlist, int rows, long long dim,
                                                 float2 *__restrict__ H, double2 *__restrict__ H64) {
  g2_t_body<NV, NC>(T, Mc, eqp, naux, n1, n2, n3, q0, qlist, rows, dim, H, H64, blockIdx.x, blockIdx.y);
}

// The second contractions of several systems' q-slabs in one launch (the batched assembly's
// work list): group g owns blocks blk0[g] .. blk0[g + 1] - 1, block b being the pair block
// (k1 = b % nk, qq = b / nk) of that system's slab.
struct G2Group {
  const float2 *T, *Mc;
  const double *eqp;
  int naux, n1, n2, n3, q0;
  const int *qlist;
  int rows;
  long long dim;
  float2 *H;
  double2 *H64;
};
struct G2Groups {
  G2Group g[MAXPG];
  long long blk0[MAXPG + 1];
  int n;
};

template <int NV, int NC>
__global__ void __launch_bounds__(256) k_g2_32_t_grouped(const __grid_constant__ G2Groups G) {
  int g = 0;
  const long long b = blockIdx.x;
  while (g + 1 < G.n && b >= G.blk0[g + 1]) g++;
  const G2Group a = G.g[g];
  const int nk = a.n1 * a.n2 * a.n3;
  const long long lb = b - G.blk0[g];
  g2_t_body<NV, NC>(a.T, a.Mc, a.eqp, a.naux, a.n1, a.n2, a.n3, a.q0, a.qlist, a.rows, a.dim, a.H, a.H64,
                    (int)(lb % nk), (int)(lb / nk));
}

// Matrix-free form of k_g2_32_t: the pair's block D = -(1/N_k) T M_cc^T is formed the same way
// (the pair's rows staged by asynchronous copies, 2 x 2 register blocks) and applied as soon as
// it is formed: its rows to x[k2] (fwd[p][qq][k1]) and, for a mirrored transfer, D^dagger to
// x[k1] (bwd[p][qq][k2]), as k_g2mv_32 does with the generic blocking.
template <int NV, int NC>
__global__ void __launch_bounds__(256) k_g2mv_32_t(const float2 *__restrict__ T, const float2 *__restrict__ Mc,
                                                   int naux, int n1, int n2, int n3, int q0,
                                                   const int *__restrict__ qlist, int rows,
                                                   const double2 *__restrict__ x, long long xs, int n_pol, int nqs,
                                                   double2 *__restrict__ fwd, double2 *__restrict__ bwd) {
  constexpr int R = NV * NV, C = NC * NC, TR = (R + 1) / 2, TCC = (C + 1) / 2, NVC = NV * NC;
  extern __shared__ float2 sg2[];
  float2 *sT = sg2, *sM = sg2 + R * naux, *sD = sM + C * naux;
  const int nk = n1 * n2 * n3;
  const int k1 = blockIdx.x, qq = blockIdx.y, q = qlist[q0 + qq];
  const int k2 = kdiff(k1, q, n1, n2, n3);
  const bool mirror = !q_self_conjugate(q, n1, n2, n3);
  static_assert(R % 2 == 0, "the pair's T rows are copied in 16-byte pieces");
  const float2 *Tq = T + (long long)qq * rows * naux + (long long)k1 * R;
  const float2 *Mk = Mc + ((long long)qq * nk + k1) * C * naux;
  {
    float4 *st4 = reinterpret_cast<float4 *>(sT);
    for (int e = threadIdx.x; e < naux * (R / 2); e += blockDim.x) {
      const int nu = e / (R / 2), h = e % (R / 2);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(tc::smem_u32(st4 + e)),
                   "l"(reinterpret_cast<const float4 *>(Tq + (long long)nu * rows) + h)
                   : "memory");
    }
  }
  if ((naux & 1) == 0) {
    const float4 *m4 = reinterpret_cast<const float4 *>(Mk);
    float4 *sm4 = reinterpret_cast<float4 *>(sM);
    for (int e = threadIdx.x; e < C * naux / 2; e += blockDim.x)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(tc::smem_u32(sm4 + e)), "l"(m4 + e) : "memory");
  } else {
    for (int e = threadIdx.x; e < C * naux; e += blockDim.x) sM[e] = Mk[e];
  }
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
  __syncthreads();
  const float invf = 1.0f / nk;
  for (int w = threadIdx.x; w < TR * TCC; w += blockDim.x) {
    const int tr = w / TCC, tc = w % TCC;
    const int r0 = 2 * tr, r1 = min(2 * tr + 1, R - 1), m0 = 2 * tc, m1 = min(2 * tc + 1, C - 1);
    const float2 *pt0 = sT + r0, *pt1 = sT + r1, *pm0 = sM + m0 * naux, *pm1 = sM + m1 * naux;
    float2 acc[2][2];
#pragma unroll
    for (int a = 0; a < 2; a++)
#pragma unroll
      for (int b = 0; b < 2; b++) acc[a][b] = make_float2(0.f, 0.f);
    for (int u = 0; u < naux; u++) {
      const float2 tt[2] = {pt0[u * R], pt1[u * R]}, mm[2] = {pm0[u], pm1[u]};
#pragma unroll
      for (int a = 0; a < 2; a++)
#pragma unroll
        for (int b = 0; b < 2; b++) {
          acc[a][b].x = fmaf(tt[a].x, mm[b].x, fmaf(-tt[a].y, mm[b].y, acc[a][b].x));
          acc[a][b].y = fmaf(tt[a].x, mm[b].y, fmaf(tt[a].y, mm[b].x, acc[a][b].y));
        }
    }
#pragma unroll
    for (int a = 0; a < 2; a++)
#pragma unroll
      for (int b = 0; b < 2; b++) {
        const int ij = 2 * tr + a, ab = 2 * tc + b;
        if (ij >= R || ab >= C) continue;
        const int i = ij / NV, j = ij % NV, ca = ab / NC, cb = ab % NC;
        sD[(i * NC + ca) * NVC + j * NC + cb] = make_float2(-invf * acc[a][b].x, -invf * acc[a][b].y);
      }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 2 * n_pol * NVC; e += blockDim.x) {
    const int side = e / (n_pol * NVC), p = (e / NVC) % n_pol, r = e % NVC;
    double sr = 0.0, si = 0.0;
    if (side == 0) {  // row ia = r of D times x[k2]
      const double2 *xv = x + p * xs + (long long)k2 * NVC;
#pragma unroll 4
      for (int jb = 0; jb < NVC; jb++) {
        const float2 d = sD[r * NVC + jb];
        const double2 v = xv[jb];
        sr += (double)d.x * v.x - (double)d.y * v.y;
        si += (double)d.x * v.y + (double)d.y * v.x;
      }
      fwd[(((long long)p * nqs + qq) * nk + k1) * NVC + r] = make_double2(sr, si);
    } else {          // column jb = r of D, conjugated, times x[k1]
      if (mirror) {
        const double2 *xv = x + p * xs + (long long)k1 * NVC;
#pragma unroll 4
        for (int ia = 0; ia < NVC; ia++) {
          const float2 d = sD[ia * NVC + r];
          const double2 v = xv[ia];
          sr += (double)d.x * v.x + (double)d.y * v.y;
          si += (double)d.x * v.y - (double)d.y * v.x;
        }
      }
      bwd[(((long long)p * nqs + qq) * nk + k2) * NVC + r] = make_double2(sr, si);
    }
  }
}

// Register-blocked conduction-valence projections for the coupling block (windows with Nv, Nc
// in {2, 4, 6}): per mu the bands of k1 and k2 are loaded once and
//   M1[b][i] = sum_s conj(c2_s,nv+b) y1_s,i + c1_s,i conj(y2_s,nv+b)   (C~_{b k2, i k1}),
//   M2[a][j] = sum_s conj(c1_s,nv+a) y2_s,j + c2_s,j conj(y1_s,nv+a)   (C~_{a k1, j k2}),
// M1 written as bf16 pieces (GEMM operand, row (k1, b, i)), M2 in FP32 (row (k1, a, j)).
// grid: x = q - q0, y = k1; block: mu chunk, loop over mu.
template <int NV, int NC>
__global__ void __launch_bounds__(160) k_proj_cv32_t(const float2 *__restrict__ Y, const double2 *__restrict__ ck,
                                                     int nao_tot, int naux, int nao_max,
                                                     const int *__restrict__ aux_atom, const int *__restrict__ ao_start,
                                                     const int *__restrict__ naoA, int n1, int n2, int n3, int q0,
                                                     const int *__restrict__ qlist, int rowsB, int kmem, PieceBuf Ap,
                                                     float2 *__restrict__ M2) {
  constexpr int NB = NV + NC, NVC = NV * NC;
  extern __shared__ float2 scf[];
  const int nk = n1 * n2 * n3;
  const int qq = blockIdx.x, q = qlist[q0 + qq], k1 = blockIdx.y;
  const int k2 = kdiff(k1, q, n1, n2, n3);
  float2 *c1 = scf, *c2 = scf + nao_tot * NB;
  for (int e = threadIdx.x; e < nao_tot * NB; e += blockDim.x) {
    const double2 a = ck[(long long)k1 * nao_tot * NB + e], b = ck[(long long)k2 * nao_tot * NB + e];
    c1[e] = make_float2((float)a.x, (float)a.y);
    c2[e] = make_float2((float)b.x, (float)b.y);
  }
  __syncthreads();
  const long long plane = (long long)rowsB * kmem;
  for (int mu = threadIdx.x; mu < naux; mu += blockDim.x) {
    const int A = aux_atom[mu], ao0 = ao_start[A], na = naoA[A];
    const float2 *Y1 = Y + (long long)k1 * nao_max * NB * naux + mu;
    const float2 *Y2 = Y + (long long)k2 * nao_max * NB * naux + mu;
    float2 m1[NC][NV], m2[NC][NV];
#pragma unroll
    for (int b = 0; b < NC; b++)
#pragma unroll
      for (int i = 0; i < NV; i++) m1[b][i] = m2[b][i] = make_float2(0.f, 0.f);
    for (int s = 0; s < na; s++) {
      float2 y1[NB], y2[NB];
#pragma unroll
      for (int n = 0; n < NB; n++) {
        y1[n] = Y1[((long long)s * NB + n) * naux];
        y2[n] = Y2[((long long)s * NB + n) * naux];
      }
      const float2 *cs1 = c1 + (ao0 + s) * NB, *cs2 = c2 + (ao0 + s) * NB;
#pragma unroll
      for (int b = 0; b < NC; b++) {
        const float2 cb2 = cs2[NV + b], cb1 = cs1[NV + b];
#pragma unroll
        for (int i = 0; i < NV; i++) {
          const float2 ci1 = cs1[i], ci2 = cs2[i];
          // m1[b][i] += conj(cb2) y1[i] + ci1 conj(y2[NV+b])
          float xr = m1[b][i].x, xi = m1[b][i].y;
          xr = fmaf(cb2.x, y1[i].x, fmaf(cb2.y, y1[i].y, xr));
          xi = fmaf(cb2.x, y1[i].y, fmaf(-cb2.y, y1[i].x, xi));
          xr = fmaf(ci1.x, y2[NV + b].x, fmaf(ci1.y, y2[NV + b].y, xr));
          xi = fmaf(ci1.y, y2[NV + b].x, fmaf(-ci1.x, y2[NV + b].y, xi));
          m1[b][i] = make_float2(xr, xi);
          // m2[b][i] (= M2[a = b][j = i]) += conj(cb1) y2[i] + ci2 conj(y1[NV+b])
          xr = m2[b][i].x;
          xi = m2[b][i].y;
          xr = fmaf(cb1.x, y2[i].x, fmaf(cb1.y, y2[i].y, xr));
          xi = fmaf(cb1.x, y2[i].y, fmaf(-cb1.y, y2[i].x, xi));
          xr = fmaf(ci2.x, y1[NV + b].x, fmaf(ci2.y, y1[NV + b].y, xr));
          xi = fmaf(ci2.y, y1[NV + b].x, fmaf(-ci2.x, y1[NV + b].y, xi));
          m2[b][i] = make_float2(xr, xi);
        }
      }
    }
    const long long out = (long long)qq * 2 * Ap.np * plane + (long long)k1 * NVC * kmem + mu;
#pragma unroll
    for (int b = 0; b < NC; b++)
#pragma unroll
      for (int i = 0; i < NV; i++)
        Ap.put<float>(plane, out + (long long)(b * NV + i) * kmem, m1[b][i].x, m1[b][i].y);
    float2 *mo = M2 + (((long long)qq * nk + k1) * NVC) * naux + mu;
#pragma unroll
    for (int a = 0; a < NC; a++)
#pragma unroll
      for (int j = 0; j < NV; j++) mo[(long long)(a * NV + j) * naux] = m2[a][j];
  }
}

// Register-blocked coupling block writer: the pair's NVC rows of T1 ((b, i), consecutive per
// column nu) and of M2 ((a, j)) copied to shared memory in one asynchronous sweep; a thread
// owns 2 x 2 products T1 row x M2 row and adds -(1/N_k) of each to B at (k1, i, a; k2, j, b)
// and, for a block with a mirror, the same value at the transposed position.
template <int NV, int NC>
__global__ void __launch_bounds__(256) k_g2c_32_t(const float2 *__restrict__ T, const float2 *__restrict__ M2,
                                                  int naux, int n1, int n2, int n3, int q0,
                                                  const int *__restrict__ qlist, int rowsB, long long dim,
                                                  float2 *__restrict__ B) {
  constexpr int R = NV * NC, TR = (R + 1) / 2, NVC = NV * NC;
  extern __shared__ float2 sg2[];
  float2 *sT = sg2, *sM = sg2 + R * naux;
  const int nk = n1 * n2 * n3;
  const int k1 = blockIdx.x, qq = blockIdx.y, q = qlist[q0 + qq];
  const int k2 = kdiff(k1, q, n1, n2, n3);
  const bool mirror = !q_self_conjugate(q, n1, n2, n3);
  static_assert(R % 2 == 0, "the pair's T1 rows are copied in 16-byte pieces");
  const float2 *Tq = T + (long long)qq * rowsB * naux + (long long)k1 * R;  // T1[q][nu][row]
  const float2 *Mk = M2 + ((long long)qq * nk + k1) * R * naux;
  {
    float4 *st4 = reinterpret_cast<float4 *>(sT);
    for (int e = threadIdx.x; e < naux * (R / 2); e += blockDim.x) {
      const int nu = e / (R / 2), h = e % (R / 2);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(tc::smem_u32(st4 + e)),
                   "l"(reinterpret_cast<const float4 *>(Tq + (long long)nu * rowsB) + h)
                   : "memory");
    }
  }
  if ((naux & 1) == 0) {
    const float4 *m4 = reinterpret_cast<const float4 *>(Mk);
    float4 *sm4 = reinterpret_cast<float4 *>(sM);
    for (int e = threadIdx.x; e < R * naux / 2; e += blockDim.x)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(tc::smem_u32(sm4 + e)), "l"(m4 + e) : "memory");
  } else {
    for (int e = threadIdx.x; e < R * naux; e += blockDim.x) sM[e] = Mk[e];
  }
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
  __syncthreads();
  const float invf = 1.0f / nk;
  for (int w = threadIdx.x; w < TR * TR; w += blockDim.x) {
    const int tr = w / TR, tm = w % TR;
    const int r0 = 2 * tr, r1 = min(2 * tr + 1, R - 1), m0 = 2 * tm, m1 = min(2 * tm + 1, R - 1);
    const float2 *pt0 = sT + r0, *pt1 = sT + r1, *pm0 = sM + m0 * naux, *pm1 = sM + m1 * naux;
    float2 acc[2][2];
#pragma unroll
    for (int x = 0; x < 2; x++)
#pragma unroll
      for (int y = 0; y < 2; y++) acc[x][y] = make_float2(0.f, 0.f);
    for (int u = 0; u < naux; u++) {
      const float2 tt[2] = {pt0[u * R], pt1[u * R]}, mm[2] = {pm0[u], pm1[u]};
#pragma unroll
      for (int x = 0; x < 2; x++)
#pragma unroll
        for (int y = 0; y < 2; y++) {
          acc[x][y].x = fmaf(tt[x].x, mm[y].x, fmaf(-tt[x].y, mm[y].y, acc[x][y].x));
          acc[x][y].y = fmaf(tt[x].x, mm[y].y, fmaf(tt[x].y, mm[y].x, acc[x][y].y));
        }
    }
#pragma unroll
    for (int x = 0; x < 2; x++)
#pragma unroll
      for (int y = 0; y < 2; y++) {
        const int bi = 2 * tr + x, aj = 2 * tm + y;   // T1 row (b, i), M2 row (a, j)
        if (bi >= R || aj >= R) continue;
        const int b = bi / NV, i = bi % NV, a = aj / NV, j = aj % NV;
        const int ia = i * NC + a, jb = j * NC + b;
        float2 *hp = B + ((long long)k1 * NVC + ia) * dim + (long long)k2 * NVC + jb;
        const float2 hx = *hp;
        *hp = make_float2(fmaf(-invf, acc[x][y].x, hx.x), fmaf(-invf, acc[x][y].y, hx.y));
        if (mirror) {
          float2 *hm = B + ((long long)k2 * NVC + jb) * dim + (long long)k1 * NVC + ia;
          const float2 mx = *hm;
          *hm = make_float2(fmaf(-invf, acc[x][y].x, mx.x), fmaf(-invf, acc[x][y].y, mx.y));
        }
      }
  }
}

bool alloc(void **p, size_t bytes) {
  if (cudaMalloc(p, bytes) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return false;
  }
  return true;
}

// The per-k tables the slabs read: relabelled at exciton momentum Q != 0, the originals at Q = 0.
const float2 *y_tab(const SplitWS *w) { return w->shifted ? w->Y32q : w->Y32; }
const double2 *ck_tab(const bse_ctx *c, const SplitWS *w) { return w->shifted ? w->ckq : c->ck; }
const double *e_tab(const bse_ctx *c, const SplitWS *w) { return w->shifted ? w->eqpq : c->eqp; }

template <int NV, int NC>
void launch_proj_fast(bse_ctx *c, SplitWS *w, int q0, int nq, int mc_pad) {
  const int na = c->naux_tot;
  const int bs = w->proj_bs ? w->proj_bs : std::min(160, (na + 31) / 32 * 32);
  const size_t sm = sizeof(float2) * 2 * c->nao_tot * (NV + NC);
  k_proj32_t<NV, NC><<<dim3(nq, c->nk), bs, sm, c->stream>>>(y_tab(w), ck_tab(c, w), c->nao_tot, na, c->nao_max, c->d_aux_atom,
                                                             c->d_ao_start, c->d_nao, c->mesh[0], c->mesh[1],
                                                             c->mesh[2], q0, c->d_qplus, w->rows, w->kmem,
                                                             pieces(w, w->Ap), w->Mc32, mc_pad);
}

template <int NV, int NC>
bool launch_g2_fast(bse_ctx *c, SplitWS *w, int q0, int nq, float2 *H) {
  double2 *H64 = c->h64 ? reinterpret_cast<double2 *>(H) : nullptr;
  if (H64) H = nullptr;
  constexpr int threads = ((NV * NV + 1) / 2) * ((NC * NC + 1) / 2);
  const int bs = std::max(128, std::min(256, (threads + 31) / 32 * 32));
  const size_t sm = sizeof(float2) * (size_t)(NV * NV + NC * NC) * c->naux_tot;
  if (sm > 200 * 1024) return false;  // the pair's rows do not fit: generic chunked kernel
  k_g2_32_t<NV, NC><<<dim3(c->nk, nq), bs, sm, c->stream>>>(w->T32, w->Mc32, e_tab(c, w), c->naux_tot, c->mesh[0],
                                                           c->mesh[1], c->mesh[2], q0, c->d_qplus, w->rows, c->dim, H,
                                                           H64);
  return true;
}

// The register-blocked matrix-free second contraction for windows with Nv, Nc in {2, 4, 6};
// false means the caller runs the generic k_g2mv_32.
template <int NV, int NC>
bool launch_g2mv_t(bse_ctx *c, SplitWS *w, int q0, int nq, const double2 *x, long long xs, int n_pol) {
  constexpr int threads = ((NV * NV + 1) / 2) * ((NC * NC + 1) / 2);
  const int bs = std::max(128, std::min(256, (threads + 31) / 32 * 32));
  const size_t sm = sizeof(float2) * ((size_t)(NV * NV + NC * NC) * c->naux_tot + (size_t)(NV * NC) * (NV * NC));
  if (sm > 200 * 1024) return false;
  k_g2mv_32_t<NV, NC><<<dim3(c->nk, nq), bs, sm, c->stream>>>(w->T32, w->Mc32, c->naux_tot, c->mesh[0], c->mesh[1],
                                                             c->mesh[2], q0, c->d_qplus, w->rows, x, xs, n_pol, w->nq,
                                                             w->mf_fwd, w->mf_bwd);
  return true;
}

bool fast_g2mv(bse_ctx *c, SplitWS *w, int q0, int nq, const double2 *x, long long xs, int n_pol) {
#define BSE_FAST_MV(NV, NC) \
  if (c->nv == NV && c->nc == NC) return launch_g2mv_t<NV, NC>(c, w, q0, nq, x, xs, n_pol);
  BSE_FAST_MV(2, 2) BSE_FAST_MV(2, 4) BSE_FAST_MV(2, 6) BSE_FAST_MV(4, 2) BSE_FAST_MV(4, 4) BSE_FAST_MV(4, 6)
  BSE_FAST_MV(6, 2) BSE_FAST_MV(6, 4) BSE_FAST_MV(6, 6)
#undef BSE_FAST_MV
  return false;
}

// Dispatch the register-blocked kernels for windows with Nv, Nc in {2, 4, 6}; false means
// the caller falls back to the generic kernels.
// mc_pad > 0: the projection writes M_cc in the fused kernel's layout.
bool fast_pair_kernels(bse_ctx *c, SplitWS *w, int q0, int nq, float2 *H, bool proj, int mc_pad = 0) {
#define BSE_FAST(NV, NC)                                                       \
  if (c->nv == NV && c->nc == NC) {                                            \
    if (proj) {                                                                \
      launch_proj_fast<NV, NC>(c, w, q0, nq, mc_pad);                          \
      return true;                                                             \
    }                                                                          \
    return launch_g2_fast<NV, NC>(c, w, q0, nq, H);                            \
  }
  BSE_FAST(2, 2) BSE_FAST(2, 4) BSE_FAST(2, 6) BSE_FAST(4, 2) BSE_FAST(4, 4) BSE_FAST(4, 6)
  BSE_FAST(6, 2) BSE_FAST(6, 4) BSE_FAST(6, 6)
#undef BSE_FAST
  return false;
}

// The register-blocked coupling-block kernels for windows with Nv, Nc in {2, 4, 6}; false
// means the caller runs the generic ones.
template <int NV, int NC>
bool launch_cv_fast(bse_ctx *c, SplitWS *w, int q0, int nq, float2 *B, bool proj) {
  const int na = c->naux_tot;
  if (proj) {
    const int bs = std::min(160, (na + 31) / 32 * 32);
    const size_t sm = sizeof(float2) * 2 * c->nao_tot * (NV + NC);
    k_proj_cv32_t<NV, NC><<<dim3(nq, c->nk), bs, sm, c->stream>>>(
        y_tab(w), ck_tab(c, w), c->nao_tot, na, c->nao_max, c->d_aux_atom, c->d_ao_start, c->d_nao, c->mesh[0],
        c->mesh[1], c->mesh[2], q0, c->d_qplus, w->rowsB, w->kmem, pieces(w, w->ApB), w->McB);
    return true;
  }
  constexpr int threads = ((NV * NC + 1) / 2) * ((NV * NC + 1) / 2);
  const int bs = std::max(128, std::min(256, (threads + 31) / 32 * 32));
  const size_t sm = sizeof(float2) * (size_t)(2 * NV * NC) * na;
  if (sm > 200 * 1024) return false;
  k_g2c_32_t<NV, NC><<<dim3(c->nk, nq), bs, sm, c->stream>>>(w->TB, w->McB, na, c->mesh[0], c->mesh[1], c->mesh[2],
                                                            q0, c->d_qplus, w->rowsB, c->dim, B);
  return true;
}

bool fast_cv_kernels(bse_ctx *c, SplitWS *w, int q0, int nq, float2 *B, bool proj) {
#define BSE_FAST_CV(NV, NC) \
  if (c->nv == NV && c->nc == NC) return launch_cv_fast<NV, NC>(c, w, q0, nq, B, proj);
  BSE_FAST_CV(2, 2) BSE_FAST_CV(2, 4) BSE_FAST_CV(2, 6) BSE_FAST_CV(4, 2) BSE_FAST_CV(4, 4) BSE_FAST_CV(4, 6)
  BSE_FAST_CV(6, 2) BSE_FAST_CV(6, 4) BSE_FAST_CV(6, 6)
#undef BSE_FAST_CV
  return false;
}

// ---- tensor maps ------------------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

// 3-D tensor of pieces {K = k_extent, rows, planes} with row pitch kmem elements: bf16, or FP32
// words holding tf32 pieces (tf32); the box is one 64-byte row of K by box_rows rows.
bool make_map(CUtensorMap *m, void *base, int k_extent, long long rows, long long planes, int kmem, int box_rows,
              bool tf32) {
  auto fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t eb = tf32 ? 4 : 2;
  cuuint64_t dims[3] = {(cuuint64_t)k_extent, (cuuint64_t)rows, (cuuint64_t)planes};
  cuuint64_t strides[2] = {(cuuint64_t)kmem * eb, (cuuint64_t)rows * kmem * eb};
  cuuint32_t box[3] = {(cuuint32_t)(tf32 ? tcg::BK_TF32 : tcg::BK), (cuuint32_t)box_rows, 1};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = fn(m, tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides,
                  box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// 3-D tensor of 8-byte elements (complex64 values copied bit for bit) {x, y, z} with row pitch
// x_pitch and plane pitch y * x_pitch elements, box {bx, by, bz}: M_cc of a slab for the fused
// kernel, {nu, (a, b), (q, k1)}.
bool make_map_c64_3d(CUtensorMap *m, void *base, long long x, long long y, long long z, long long x_pitch, int bx,
                     int by, int bz) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[3] = {(cuuint64_t)x, (cuuint64_t)y, (cuuint64_t)z};
  cuuint64_t strides[2] = {(cuuint64_t)x_pitch * 8, (cuuint64_t)(y * x_pitch) * 8};
  cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <int NP, int BN, bool TF>
bse_status launch_tc(bse_ctx *c, const CUtensorMap &A, const CUtensorMap &B, const tcg::Args &args, dim3 grid,
                     int prof_id) {
  using Cf = tcg::Cfg<NP, BN>;
  tcg::Groups<1> G;
  G.A[0] = A;
  G.B[0] = B;
  G.a[0] = args;
  G.a[0].tiles_n = (int)grid.x;
  G.a[0].tiles_m = (int)grid.y;
  G.a[0].tiles_b = (int)grid.z;
  const long long total = (long long)grid.x * grid.y * grid.z;
  G.tile0[0] = 0;
  G.tile0[1] = total;
  G.n = 1;
  const int ctas = (int)std::min<long long>(total, c->n_sm);
  bse_prof_begin(c, prof_id);
  tcg::k_tc_zgemm<NP, BN, TF><<<ctas, 192, Cf::SMEM, c->stream>>>(G);
  bse_prof_end(c, prof_id);
  bse_count_launch();
  return bse_check_launch(c, "tc_zgemm");
}

template <int NP, bool TF = false>
bse_status launch_tc_bn(bse_ctx *c, int bn, const CUtensorMap &A, const CUtensorMap &B, const tcg::Args &args,
                        dim3 grid, int prof_id) {
  switch (bn) {
    case 64: return launch_tc<NP, 64, TF>(c, A, B, args, grid, prof_id);
    case 96: return launch_tc<NP, 96, TF>(c, A, B, args, grid, prof_id);
    case 128: return launch_tc<NP, 128, TF>(c, A, B, args, grid, prof_id);
    default: return launch_tc<NP, 160, TF>(c, A, B, args, grid, prof_id);
  }
}

// The context's piece kind picks the instantiation: tf32 pieces (two of them) or np bf16 pieces.
bse_status launch_tc_np(bse_ctx *c, int np, int bn, const CUtensorMap &A, const CUtensorMap &B,
                        const tcg::Args &args, dim3 grid, int prof_id) {
  if (ws(c)->tf32) return launch_tc_bn<2, true>(c, bn, A, B, args, grid, prof_id);
  if (np == 3) return launch_tc_bn<3>(c, bn, A, B, args, grid, prof_id);
  if (np == 2) return launch_tc_bn<2>(c, bn, A, B, args, grid, prof_id);
  return launch_tc_bn<1>(c, bn, A, B, args, grid, prof_id);
}

// ---- fused direct term -------------------------------------------------------------------
template <int NP, int BN, int NC, bool TF, bool MF = false>
bse_status launch_direct_t(bse_ctx *c, SplitWS *w, const tcd::DArgs &a, int prof_id) {
  using Cf = tcd::DCfg<NP, BN>;
  const long long total = (long long)a.tiles_m * a.tiles_b;
  const int ctas = (int)std::min<long long>(total, c->n_sm);
  tcd::DGroups<1> G;
  G.A[0] = w->tmA_g1;
  G.B[0] = w->tmB_d;
  G.M[0] = w->tmM_d;
  G.a[0] = a;
  G.tile0[0] = 0;
  G.tile0[1] = total;
  G.n = 1;
  if constexpr (BN == 160 && !MF && NC <= 4) {
    if (w->nsplit) {  // T's columns in two halves, the epilogue of one under the MMAs of the next
      G.B[0] = w->tmB_dh;
      G.M[0] = w->tmM_dh;
      bse_prof_begin(c, prof_id);
      tcd::k_tc_direct_ns<NP, NC, TF><<<ctas, tcd::NS_THREADS, tcd::NsCfg<NP>::SMEM, c->stream>>>(G);
      bse_prof_end(c, prof_id);
      bse_count_launch();
      return bse_check_launch(c, "tc_direct_ns");
    }
  }
  bse_prof_begin(c, prof_id);
  tcd::k_tc_direct<NP, BN, NC, TF, 1, MF><<<ctas, tcd::THREADS, Cf::SMEM, c->stream>>>(G);
  bse_prof_end(c, prof_id);
  bse_count_launch();
  return bse_check_launch(c, "tc_direct");
}

template <int NP, int BN, bool TF, bool MF = false>
bse_status launch_direct_nc(bse_ctx *c, SplitWS *w, const tcd::DArgs &a, int prof_id) {
  switch (c->nc) {
    case 2: return launch_direct_t<NP, BN, 2, TF, MF>(c, w, a, prof_id);
    case 4: return launch_direct_t<NP, BN, 4, TF, MF>(c, w, a, prof_id);
    default: return launch_direct_t<NP, BN, 6, TF, MF>(c, w, a, prof_id);
  }
}

// N tiles of the fused kernel: T's N_aux columns in one tile (two ring stages of bf16x3 pieces
// fit up to 160 columns), so the fused path takes N_aux <= 160.
template <int NP, bool TF = false, bool MF = false>
bse_status launch_direct_bn(bse_ctx *c, SplitWS *w, const tcd::DArgs &a, int prof_id) {
  if (w->bn_d == 64) return launch_direct_nc<NP, 64, TF, MF>(c, w, a, prof_id);
  return launch_direct_nc<NP, 160, TF, MF>(c, w, a, prof_id);
}

bse_status launch_direct(bse_ctx *c, SplitWS *w, const tcd::DArgs &a, int prof_id) {
  if (w->tf32) return launch_direct_bn<2, true>(c, w, a, prof_id);
  if (w->np == 3) return launch_direct_bn<3>(c, w, a, prof_id);
  if (w->np == 2) return launch_direct_bn<2>(c, w, a, prof_id);
  return launch_direct_bn<1>(c, w, a, prof_id);
}

// The matrix-free form of the fused kernel (a.x, a.fwd, a.bwd set; Nv = 2 or 4).
bse_status launch_direct_mf(bse_ctx *c, SplitWS *w, const tcd::DArgs &a, int prof_id) {
  if (w->tf32) return launch_direct_bn<2, true, true>(c, w, a, prof_id);
  if (w->np == 3) return launch_direct_bn<3, false, true>(c, w, a, prof_id);
  if (w->np == 2) return launch_direct_bn<2, false, true>(c, w, a, prof_id);
  return launch_direct_bn<1, false, true>(c, w, a, prof_id);
}

// Ring stage bytes of the fused kernel (operand pieces of one K chunk).
int direct_stage_bytes(int np, int bn) { return 2 * np * (tcg::A_TILE + bn * tcg::ROWB); }

// Shared-memory size attributes of every tensor-core instantiation, set once (outside any
// stream capture).
template <int NP, int BN, bool TF = false>
void set_attr() {
  cudaFuncSetAttribute(tcg::k_tc_zgemm<NP, BN, TF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       tcg::Cfg<NP, BN>::SMEM);
}
template <int NV, int NC>
void set_g2_attr() {
  cudaFuncSetAttribute(k_g2_32_t<NV, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_g2mv_32_t<NV, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_g2c_32_t<NV, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}
template <int NP, int BN, bool TF = false>
void set_direct_attr() {
  constexpr int sm = tcd::DCfg<NP, BN>::SMEM;
  cudaFuncSetAttribute(tcd::k_tc_direct<NP, BN, 2, TF>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  cudaFuncSetAttribute(tcd::k_tc_direct<NP, BN, 4, TF>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  cudaFuncSetAttribute(tcd::k_tc_direct<NP, BN, 6, TF>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  cudaFuncSetAttribute(tcd::k_tc_direct<NP, BN, 2, TF, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  cudaFuncSetAttribute(tcd::k_tc_direct<NP, BN, 4, TF, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  cudaFuncSetAttribute(tcd::k_tc_direct<NP, BN, 6, TF, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if constexpr (BN == 160) {
    constexpr int sn = tcd::NsCfg<NP>::SMEM;
    cudaFuncSetAttribute(tcd::k_tc_direct_ns<NP, 2, TF>, cudaFuncAttributeMaxDynamicSharedMemorySize, sn);
    cudaFuncSetAttribute(tcd::k_tc_direct_ns<NP, 4, TF>, cudaFuncAttributeMaxDynamicSharedMemorySize, sn);
  }
}
void set_all_attrs_now() {
  set_direct_attr<1, 64>(); set_direct_attr<1, 160>();
  set_direct_attr<2, 64>(); set_direct_attr<2, 160>();
  set_direct_attr<3, 64>(); set_direct_attr<3, 160>();
  set_g2_attr<2, 2>(); set_g2_attr<2, 4>(); set_g2_attr<2, 6>(); set_g2_attr<4, 2>(); set_g2_attr<4, 4>();
  set_g2_attr<4, 6>(); set_g2_attr<6, 2>(); set_g2_attr<6, 4>(); set_g2_attr<6, 6>();
  set_attr<1, 64>(); set_attr<1, 96>(); set_attr<1, 128>(); set_attr<1, 160>();
  set_attr<2, 64>(); set_attr<2, 96>(); set_attr<2, 128>(); set_attr<2, 160>();
  set_attr<3, 64>(); set_attr<3, 96>(); set_attr<3, 128>(); set_attr<3, 160>();
  set_direct_attr<2, 64, true>(); set_direct_attr<2, 160, true>();
  set_attr<2, 64, true>(); set_attr<2, 96, true>(); set_attr<2, 128, true>(); set_attr<2, 160, true>();
}
void set_all_attrs(const bse_ctx *c) { bse_once_per_device(c, BSE_ONCE_SPLIT, set_all_attrs_now); }

}  // namespace

bse_status split_setup(bse_ctx *c) {
  SplitWS *w = new SplitWS();
  c->tc = w;
  w->tf32 = c->precision == BSE_TF32X2;
  w->pbytes = w->tf32 ? 4 : 2;
  w->np = c->precision == BSE_BF16X3 ? 3 : (c->precision == BSE_BF16X2 || w->tf32) ? 2 : 1;
  w->pp = 2 * w->np;
  const int na = c->naux_tot;
  w->kmem = (na + 7) / 8 * 8;
  const int bk = w->tf32 ? tcg::BK_TF32 : tcg::BK;
  w->kchunks = (na + bk - 1) / bk;
  w->rows = c->nk * c->nv * c->nv;
  // fused direct term: a window with register-blocked projections and T's columns in one tile
  const bool win = (c->nv == 2 || c->nv == 4 || c->nv == 6) && (c->nc == 2 || c->nc == 4 || c->nc == 6);
  w->fused = win && na <= 160;
  w->naux_pad = (na + 15) / 16 * 16;
  if (w->fused) {
    w->bn_d = na <= 64 ? 64 : 160;
    const int ncc = c->nc * c->nc, rpp = c->nv * c->nv;
    const long long stage = direct_stage_bytes(w->np, w->bn_d);
    w->pairs_d = 128 / rpp;
    w->nui_d = (int)(stage / ((long long)w->pairs_d * ncc * 8)) / 16 * 16;
    if (w->nui_d < 16) {  // wide conduction windows on Nv = 2: fewer pairs per tile
      w->pairs_d = (int)(stage / (16LL * ncc * 8));
      w->nui_d = 16;
    }
    w->nui_d = std::min(w->nui_d, w->naux_pad);
    w->nsplit = w->bn_d == 160 && na > tcd::NS_HALF && c->nc <= 4 && w->pairs_d * ncc <= 128;
  }
  const size_t pb = (size_t)w->pbytes;
  const size_t per_q = (size_t)w->pp * w->rows * w->kmem * pb + (size_t)c->nk * c->nc * c->nc * w->naux_pad * 8 +
                       (size_t)w->rows * na * 8;
  const size_t budget = (size_t)1536 << 20;
  w->nq = (int)std::max<size_t>(1, std::min<size_t>((size_t)c->nk, budget / std::max<size_t>(per_q, 1)));
  w->nq = std::min(w->nq, 65535);
  if (c->mesh[2] > 1 && w->nq >= c->mesh[2]) w->nq = w->nq / c->mesh[2] * c->mesh[2];  // whole q-lines
  const size_t nn = (size_t)na * na;
  const size_t dimz = (size_t)c->dim;
  if (!alloc((void **)&w->PHQ, (size_t)c->nk * c->n_RW * sizeof(float2)) ||
      !alloc((void **)&w->PHK, (size_t)c->nk * c->n_RC * sizeof(float2)) ||
      !alloc((void **)&w->WR32T, (size_t)c->n_RW * nn * sizeof(float)) ||
      !alloc((void **)&w->CR32, (size_t)c->n_RC * c->nao_tot * c->nao_tot * na * sizeof(float)) ||
      !alloc((void **)&w->V032, nn * sizeof(float2)) ||
      !alloc((void **)&w->ck32, (size_t)c->nk * c->nao_tot * c->nb * sizeof(float2)) ||
      !alloc((void **)&w->X32, dimz * na * sizeof(float2)) ||
      !alloc((void **)&w->Wp, (size_t)c->nk * w->pp * na * w->kmem * pb) ||
      !alloc((void **)&w->Ap, (size_t)w->nq * w->pp * w->rows * w->kmem * pb) ||
      !alloc((void **)&w->Mc32, (size_t)w->nq * c->nk * c->nc * c->nc * w->naux_pad * 8) ||
      !alloc((void **)&w->T32, (size_t)w->nq * w->rows * na * 8) ||
      !alloc((void **)&w->Y32, (size_t)c->nk * c->nao_max * c->nb * na * 8) ||
      !alloc((void **)&w->Pp, (size_t)w->pp * dimz * w->kmem * pb) ||
      !alloc((void **)&w->Xp, (size_t)w->pp * dimz * w->kmem * pb))
    return bse_fail(c, BSE_ENOMEM, "split workspace allocation failed");
  cudaMemset(w->Wp, 0, (size_t)c->nk * w->pp * na * w->kmem * pb);
  cudaMemset(w->Ap, 0, (size_t)w->nq * w->pp * w->rows * w->kmem * pb);
  cudaMemset(w->Mc32, 0, (size_t)w->nq * c->nk * c->nc * c->nc * w->naux_pad * 8);
  cudaMemset(w->Pp, 0, (size_t)w->pp * dimz * w->kmem * pb);
  cudaMemset(w->Xp, 0, (size_t)w->pp * dimz * w->kmem * pb);
  {
    const long long nph = (long long)c->nk * (c->n_RW + c->n_RC);
    k_phase_tables<<<(unsigned)((nph + 255) / 256), 256, 0, c->stream>>>(
        c->d_R_W, c->d_w_RW, c->n_RW, c->d_R_C, c->n_RC, c->mesh[0], c->mesh[1], c->mesh[2], c->koff[0],
        c->koff[1], c->koff[2], w->PHQ, w->PHK);
    bse_count_launch();
  }
  set_all_attrs(c);
  const bool tf = w->tf32;
  bool ok = make_map(&w->tmA_g1, w->Ap, na, w->rows, (long long)w->pp * w->nq, w->kmem, tcg::BM, tf) &&
            make_map(&w->tmB_g1, w->Wp, na, na, (long long)w->pp * c->nk, w->kmem, w->bn_g1, tf) &&
            (!w->fused || make_map(&w->tmB_d, w->Wp, na, na, (long long)w->pp * c->nk, w->kmem, w->bn_d, tf)) &&
            (!w->fused || make_map_c64_3d(&w->tmM_d, w->Mc32, w->naux_pad, (long long)c->nc * c->nc,
                                          (long long)w->nq * c->nk, w->naux_pad, w->nui_d, c->nc * c->nc,
                                          w->pairs_d)) &&
            (!w->nsplit ||
             (make_map(&w->tmB_dh, w->Wp, na, na, (long long)w->pp * c->nk, w->kmem, tcd::NS_HALF, tf) &&
              make_map_c64_3d(&w->tmM_dh, w->Mc32, w->naux_pad, (long long)c->nc * c->nc, (long long)w->nq * c->nk,
                              w->naux_pad, tcd::NS_MC_COLS, c->nc * c->nc, w->pairs_d))) &&
            make_map(&w->tmA_x, w->Pp, na, c->dim, w->pp, w->kmem, tcg::BM, tf) &&
            make_map(&w->tmB_x, w->Xp, na, c->dim, w->pp, w->kmem, TC_BN, tf);
  if (!ok) return bse_fail(c, BSE_ECUDA, "tensor map encoding failed");
  if (cudaGetLastError() != cudaSuccess) return bse_fail(c, BSE_ECUDA, "split workspace initialisation failed");
  return BSE_OK;
}

void split_free(bse_ctx *c) {
  SplitWS *w = ws(c);
  if (!w) return;
  void *ptrs[] = {w->Wp, w->Ap, w->Mc32, w->T32, w->Y32, w->Pp, w->Xp, w->PHQ, w->PHK, w->WR32T, w->CR32, w->V032,
                  w->ck32, w->X32, w->Y32q, w->ck32q, w->ckq, w->eqpq, w->ApB, w->XpB, w->McB, w->TB,
                  w->mf_fwd, w->mf_bwd, w->mf_zp, w->mf_z2, w->adjMv};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  delete w;
  c->tc = nullptr;
}

bse_status split_interp_W(bse_ctx *c, const double *W_R, double2 *Wq_out) {
  SplitWS *w = ws(c);
  const int na = c->naux_tot;
  const long long nn = (long long)na * na;
  k_wr_f32t<<<(unsigned)((nn * c->n_RW + 255) / 256), 256, 0, c->stream>>>(W_R, c->n_RW, na, w->WR32T);
  const size_t sm = sizeof(float2) * IQB * c->n_RW;
  if (sm > 48 * 1024 &&
      cudaFuncSetAttribute(k_interp_W32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
    return bse_fail(c, BSE_EINVAL, "interp_W: too many W(R) images for one block");
  dim3 grid((unsigned)std::min<long long>((nn + 255) / 256, 1024), (c->nk + IQB - 1) / IQB);
  bse_prof_begin(c, BSE_KP_INTERP);
  k_interp_W32<<<grid, 256, sm, c->stream>>>(w->WR32T, w->PHQ, c->n_RW, na, c->nk, w->kmem, pieces(w, w->Wp),
                                              Wq_out);
  bse_prof_end(c, BSE_KP_INTERP);
  bse_count_launch(2);
  return bse_check_launch(c, "split interp_W");
}

// Per-k stage in FP32: Y, the exchange factors X (+ pieces of conj X) and P = X V (pieces).
bse_status split_project(bse_ctx *c, const double *C_R) {
  SplitWS *w = ws(c);
  const int na = c->naux_tot;
  const long long ncr = (long long)c->n_RC * c->nao_tot * c->nao_tot * na;
  const long long nck = (long long)c->nk * c->nao_tot * c->nb * 2;
  k_d2f<<<(unsigned)std::min<long long>((ncr + 255) / 256, 8192), 256, 0, c->stream>>>(C_R, ncr, w->CR32);
  k_d2f<<<(unsigned)std::min<long long>((nck + 255) / 256, 8192), 256, 0, c->stream>>>((const double *)c->ck, nck,
                                                                                        (float *)w->ck32);
  int maxmu = 0;
  for (int a : c->naux) maxmu = std::max(maxmu, a);
  const size_t sm = sizeof(float2) * (c->n_RC + c->nao_tot * c->nb + TCH32 * maxmu + c->nb * maxmu);
  if (sm > 200 * 1024) return bse_fail(c, BSE_EINVAL, "half transform: basis too large for one block");
  if (sm > 48 * 1024)
    cudaFuncSetAttribute(k_half_transform32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  bse_prof_begin(c, BSE_KP_HALF);
  k_half_transform32<<<dim3(c->nao_tot, c->nk), 256, sm, c->stream>>>(
      w->CR32, w->PHK, c->n_RC, w->ck32, c->nao_tot, c->nb, na, c->nao_max, c->d_ao_start, c->d_aux_start,
      c->d_naux, c->n_atoms, w->Y32);
  bse_prof_end(c, BSE_KP_HALF);
  w->shifted = c->qmQ != 0;
  if (w->shifted) {
    const size_t ny = (size_t)c->nk * c->nao_max * c->nb * na, nckq = (size_t)c->nk * c->nao_tot * c->nb;
    if (!w->Y32q && (!alloc((void **)&w->Y32q, ny * sizeof(float2)) ||
                     !alloc((void **)&w->ckq, nckq * sizeof(double2)) ||
                     !alloc((void **)&w->ck32q, nckq * sizeof(float2)) ||
                     !alloc((void **)&w->eqpq, (size_t)c->nk * c->nb * sizeof(double))))
      return bse_fail(c, BSE_ENOMEM, "finite momentum: relabelled per-k tables do not fit");
    k_shift_tables<<<c->n_sm * 8, 256, 0, c->stream>>>(w->Y32, c->ck, c->eqp, c->nao_max, c->nao_tot, c->nb, c->nv,
                                                        na, c->mesh[0], c->mesh[1], c->mesh[2], c->qmQ, w->Y32q,
                                                        w->ckq, w->ck32q, w->eqpq);
    bse_count_launch();
  }
  k_exchange_X32<<<dim3((na + 127) / 128, c->nk), 128, 0, c->stream>>>(
      w->shifted ? w->Y32q : w->Y32, w->shifted ? w->ck32q : w->ck32, c->nao_tot, c->nb, c->nv, c->nc, na,
      c->nao_max, c->d_aux_atom, c->d_ao_start, c->d_nao, c->dim, w->kmem, w->X32, pieces(w, w->Xp));
  const long long nn = (long long)na * na;
  k_to_f32<<<(unsigned)((nn + 255) / 256), 256, 0, c->stream>>>(c->V0c, nn, w->V032);
  dim3 g((na + 63) / 64, (unsigned)((c->dim + 63) / 64));
  if (g.y > 65535) return bse_fail(c, BSE_EINVAL, "exchange factors: dim too large for the P grid");
  if (c->vx_from_R)
    k_xv0_pieces<true><<<g, 256, 0, c->stream>>>((int)c->dim, na, w->X32, w->V032, w->kmem, pieces(w, w->Pp));
  else
    k_xv0_pieces<false><<<g, 256, 0, c->stream>>>((int)c->dim, na, w->X32, w->V032, w->kmem, pieces(w, w->Pp));
  bse_count_launch(6);
  return bse_check_launch(c, "split project");
}

namespace {

// ---- the assembly's stages (one system) ----------------------------------------------------
// The exchange GEMM: H = alpha/N_k (X V) conj(X)^T, writing every element.
void exchange_gemm(const bse_ctx *c, const SplitWS *w, float2 *H, tcg::Args &a, dim3 &grid) {
  a = tcg::Args{};
  a.rows = (int)c->dim;
  a.n_valid = (int)c->dim;
  a.k_chunks = w->kchunks;
  a.scale = (float)(c->alpha / c->nk);
  // the exchange block is Hermitian: element (r, c) is stored as conj at (c, r), so a lane's
  // row index runs along memory and the stores coalesce
  a.out = H;
  a.out64 = c->h64 ? 1 : 0;
  a.ld_row = 1;
  a.ld_col = c->dim;
  a.conj_out = 1;
  a.out_bstride = 0;
  a.b_batch_planes = 0;
  a.b_base = 0;
  a.qlist = nullptr;
  a.err = c->d_err;
  grid = dim3((unsigned)((c->dim + TC_BN - 1) / TC_BN), (unsigned)((c->dim + tcg::BM - 1) / tcg::BM), 1);
}

// The pair projections of q-slab [q0, q0 + nq) (M_cc in the fused layout on the fused path).
bse_status slab_project(bse_ctx *c, SplitWS *w, int q0, int nq, float2 *H) {
  const int na = c->naux_tot;
  bse_prof_begin(c, BSE_KP_PROJECT);
  if (w->fused) {
    fast_pair_kernels(c, w, q0, nq, H, true, w->naux_pad);
  } else if (!fast_pair_kernels(c, w, q0, nq, H, true)) {
    const int nchunk = (na + 127) / 128;
    dim3 grid(nchunk * (c->nv + c->nc), nq, c->nk);
    size_t sm = sizeof(float2) * 2 * c->nao_tot * c->nb;
    k_proj32<<<grid, 128, sm, c->stream>>>(y_tab(w), ck_tab(c, w), c->nao_tot, c->nb, c->nv, c->nc, na, c->nao_max,
                                           c->d_aux_atom, c->d_ao_start, c->d_nao, c->mesh[0], c->mesh[1],
                                           c->mesh[2], q0, c->d_qplus, w->rows, w->kmem, pieces(w, w->Ap), w->Mc32);
  }
  bse_prof_end(c, BSE_KP_PROJECT);
  bse_count_launch();
  return bse_check_launch(c, "proj32");
}

// Fused path: T = M_vv W(q) and H += -T M_cc^T / N_k for the slab in one kernel.
void direct_args(const bse_ctx *c, const SplitWS *w, int q0, int nq, float2 *H, tcd::DArgs &a) {
  a = tcd::DArgs{};
  a.nv = c->nv;
  a.pairs = w->pairs_d;
  a.rows = w->rows;
  a.tiles_m = (c->nk + w->pairs_d - 1) / w->pairs_d;
  a.tiles_b = nq;
  a.k_chunks = w->kchunks;
  a.naux = c->naux_tot;
  a.naux_pad = w->naux_pad;
  a.nui = w->nui_d;
  a.n_mitems = (w->naux_pad + w->nui_d - 1) / w->nui_d;
  a.Mc = w->Mc32;
  a.qlist = c->d_qplus;
  a.b_base = q0;
  a.n1 = c->mesh[0];
  a.n2 = c->mesh[1];
  a.n3 = c->mesh[2];
  a.eqp = e_tab(c, w);
  a.dim = c->dim;
  a.H = c->h64 ? nullptr : H;
  a.H64 = c->h64 ? reinterpret_cast<double2 *>(H) : nullptr;
  a.err = c->d_err;
}

bse_status slab_direct(bse_ctx *c, SplitWS *w, int q0, int nq, float2 *H) {
  tcd::DArgs a;
  direct_args(c, w, q0, nq, H, a);
  return launch_direct(c, w, a, BSE_KP_G1);
}

// Unfused path, first contraction: T = M_vv W(q) (tensor cores) for the slab.
void slab_g1(const bse_ctx *c, const SplitWS *w, int q0, int nq, tcg::Args &a, dim3 &grid) {
  const int na = c->naux_tot;
  a = tcg::Args{};
  a.rows = w->rows;
  a.n_valid = na;
  a.k_chunks = w->kchunks;
  a.scale = 1.0f;
  a.out = w->T32;
  a.ld_row = 1;
  a.ld_col = w->rows;
  a.out_bstride = (long long)w->rows * na;
  a.b_batch_planes = 1;
  a.b_base = q0;
  a.qlist = c->d_qplus;
  a.err = c->d_err;
  grid = dim3((unsigned)((na + w->bn_g1 - 1) / w->bn_g1), (unsigned)((w->rows + tcg::BM - 1) / tcg::BM), nq);
}

// Unfused path, second contraction: H block += -(1/N_k) T M_cc^T (+ the diagonal).
bse_status slab_g2(bse_ctx *c, SplitWS *w, int q0, int nq, float2 *H) {
  const int na = c->naux_tot;
  dim3 grid(c->nk, nq);
  size_t sm = sizeof(float2) * (c->nv * c->nv + c->nc * c->nc) * G2CH;
  bse_prof_begin(c, BSE_KP_G2);
  if (!fast_pair_kernels(c, w, q0, nq, H, false))
    k_g2_32<<<grid, 256, sm, c->stream>>>(w->T32, w->Mc32, e_tab(c, w), c->nv, c->nc, na, c->mesh[0], c->mesh[1],
                                          c->mesh[2], q0, c->d_qplus, w->rows, c->dim, c->h64 ? nullptr : H,
                                          c->h64 ? reinterpret_cast<double2 *>(H) : nullptr);
  bse_prof_end(c, BSE_KP_G2);
  bse_count_launch();
  return bse_check_launch(c, "g2_32");
}

}  // namespace

bse_status split_assemble(bse_ctx *c, void *Hv) {
  SplitWS *w = ws(c);
  float2 *H = (float2 *)Hv;
  {
    tcg::Args a;
    dim3 grid;
    exchange_gemm(c, w, H, a, grid);
    bse_status s = launch_tc_np(c, w->np, TC_BN, w->tmA_x, w->tmB_x, a, grid, BSE_KP_EXCH);
    if (s != BSE_OK) return s;
  }
  const int nqp = (int)c->qplus.size();
  for (int q0 = 0; q0 < nqp; q0 += w->nq) {
    const int nq = std::min(w->nq, nqp - q0);
    bse_status s = slab_project(c, w, q0, nq, H);
    if (s == BSE_OK) {
      if (w->fused) {
        s = slab_direct(c, w, q0, nq, H);
      } else {
        tcg::Args a;
        dim3 grid;
        slab_g1(c, w, q0, nq, a, grid);
        s = launch_tc_np(c, w->np, w->bn_g1, w->tmA_g1, w->tmB_g1, a, grid, BSE_KP_G1);
        if (s == BSE_OK) s = slab_g2(c, w, q0, nq, H);
      }
    }
    if (s != BSE_OK) return s;
  }
  return BSE_OK;
}

namespace {

// ---- batched assembly of several systems as a work list ----------------------------------
// One grouped tensor-core launch per step and N tile: every (system, q-slab) GEMM of the step
// is a group of the launch's work list (Groups), so the persistent CTAs stream the tiles of
// all of them (smallest system first) instead of one launch per system.
constexpr int MAXG = 16;
struct GemmItem {
  const CUtensorMap *A, *B;
  tcg::Args a;
  dim3 grid;
};

template <int NP, int BN, bool TF>
bse_status launch_grouped_t(bse_ctx *c, const std::vector<GemmItem> &items, int prof_id) {
  using Cf = tcg::Cfg<NP, BN>;
  for (size_t i0 = 0; i0 < items.size(); i0 += MAXG) {
    const int n = (int)std::min<size_t>(MAXG, items.size() - i0);
    tcg::Groups<MAXG> G;
    long long t0 = 0;
    for (int g = 0; g < n; g++) {
      const GemmItem &it = items[i0 + g];
      G.A[g] = *it.A;
      G.B[g] = *it.B;
      G.a[g] = it.a;
      G.a[g].tiles_n = (int)it.grid.x;
      G.a[g].tiles_m = (int)it.grid.y;
      G.a[g].tiles_b = (int)it.grid.z;
      G.tile0[g] = t0;
      t0 += (long long)it.grid.x * it.grid.y * it.grid.z;
    }
    for (int g = n; g <= MAXG; g++) G.tile0[g] = t0;
    G.n = n;
    if (t0 == 0) continue;
    const int ctas = (int)std::min<long long>(t0, c->n_sm);
    bse_prof_begin(c, prof_id);
    tcg::k_tc_zgemm<NP, BN, TF, MAXG><<<ctas, 192, Cf::SMEM, c->stream>>>(G);
    bse_prof_end(c, prof_id);
    bse_count_launch();
    const bse_status s = bse_check_launch(c, "tc_zgemm (grouped)");
    if (s != BSE_OK) return s;
  }
  return BSE_OK;
}

template <int NP, bool TF>
bse_status launch_grouped_bn(bse_ctx *c, int bn, const std::vector<GemmItem> &items, int prof_id) {
  switch (bn) {
    case 64: return launch_grouped_t<NP, 64, TF>(c, items, prof_id);
    case 96: return launch_grouped_t<NP, 96, TF>(c, items, prof_id);
    case 128: return launch_grouped_t<NP, 128, TF>(c, items, prof_id);
    default: return launch_grouped_t<NP, 160, TF>(c, items, prof_id);
  }
}

bse_status launch_grouped(bse_ctx *c, const SplitWS *w, int bn, const std::vector<GemmItem> &items, int prof_id) {
  if (items.empty()) return BSE_OK;
  if (w->tf32) return launch_grouped_bn<2, true>(c, bn, items, prof_id);
  if (w->np == 3) return launch_grouped_bn<3, false>(c, bn, items, prof_id);
  if (w->np == 2) return launch_grouped_bn<2, false>(c, bn, items, prof_id);
  return launch_grouped_bn<1, false>(c, bn, items, prof_id);
}

template <int NP, bool TF>
void set_grouped_attr() {
  cudaFuncSetAttribute(tcg::k_tc_zgemm<NP, 64, TF, MAXG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       tcg::Cfg<NP, 64>::SMEM);
  cudaFuncSetAttribute(tcg::k_tc_zgemm<NP, 96, TF, MAXG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       tcg::Cfg<NP, 96>::SMEM);
  cudaFuncSetAttribute(tcg::k_tc_zgemm<NP, 128, TF, MAXG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       tcg::Cfg<NP, 128>::SMEM);
  cudaFuncSetAttribute(tcg::k_tc_zgemm<NP, 160, TF, MAXG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       tcg::Cfg<NP, 160>::SMEM);
}
template <int NP, bool TF>
void set_grouped_direct_attr() {
  cudaFuncSetAttribute(tcd::k_tc_direct<NP, 64, 2, TF, MAXG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       tcd::DCfg<NP, 64>::SMEM);
  cudaFuncSetAttribute(tcd::k_tc_direct<NP, 64, 4, TF, MAXG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       tcd::DCfg<NP, 64>::SMEM);
  cudaFuncSetAttribute(tcd::k_tc_direct<NP, 64, 6, TF, MAXG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       tcd::DCfg<NP, 64>::SMEM);
  cudaFuncSetAttribute(tcd::k_tc_direct<NP, 160, 2, TF, MAXG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       tcd::DCfg<NP, 160>::SMEM);
  cudaFuncSetAttribute(tcd::k_tc_direct<NP, 160, 4, TF, MAXG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       tcd::DCfg<NP, 160>::SMEM);
  cudaFuncSetAttribute(tcd::k_tc_direct<NP, 160, 6, TF, MAXG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       tcd::DCfg<NP, 160>::SMEM);
}
template <int NV, int NC>
void set_grouped_g2_attr() {
  cudaFuncSetAttribute(k_g2_32_t_grouped<NV, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}
void set_grouped_attrs_now() {
  set_grouped_attr<1, false>();
  set_grouped_attr<2, false>();
  set_grouped_attr<3, false>();
  set_grouped_attr<2, true>();
  set_grouped_direct_attr<1, false>();
  set_grouped_direct_attr<2, false>();
  set_grouped_direct_attr<3, false>();
  set_grouped_direct_attr<2, true>();
  set_grouped_g2_attr<2, 2>(); set_grouped_g2_attr<2, 4>(); set_grouped_g2_attr<2, 6>();
  set_grouped_g2_attr<4, 2>(); set_grouped_g2_attr<4, 4>(); set_grouped_g2_attr<4, 6>();
  set_grouped_g2_attr<6, 2>(); set_grouped_g2_attr<6, 4>(); set_grouped_g2_attr<6, 6>();
}

// A (system, q-slab) unit of a batch step.
struct BUnit {
  bse_ctx *c;
  float2 *H;
  int q0, nq;
};

bool window_blocked(const bse_ctx *c) {
  return (c->nv == 2 || c->nv == 4 || c->nv == 6) && (c->nc == 2 || c->nc == 4 || c->nc == 6);
}

// Register-blocked projections of units with one window and block size, MAXPG per launch.
template <int NV, int NC>
bse_status launch_proj_grouped_t(bse_ctx *c0, const std::vector<BUnit> &us, int bs) {
  for (size_t i0 = 0; i0 < us.size(); i0 += MAXPG) {
    const int n = (int)std::min<size_t>(MAXPG, us.size() - i0);
    ProjGroups G;
    long long b0 = 0;
    size_t sm = 0;
    for (int g = 0; g < n; g++) {
      const BUnit &u = us[i0 + g];
      bse_ctx *c = u.c;
      SplitWS *w = ws(c);
      ProjGroup &a = G.g[g];
      a.Y = y_tab(w);
      a.ck = ck_tab(c, w);
      a.nao_tot = c->nao_tot;
      a.naux = c->naux_tot;
      a.nao_max = c->nao_max;
      a.aux_atom = c->d_aux_atom;
      a.ao_start = c->d_ao_start;
      a.naoA = c->d_nao;
      a.n1 = c->mesh[0];
      a.n2 = c->mesh[1];
      a.n3 = c->mesh[2];
      a.q0 = u.q0;
      a.qlist = c->d_qplus;
      a.rows = w->rows;
      a.kmem = w->kmem;
      a.Ap = pieces(w, w->Ap);
      a.Mc = w->Mc32;
      a.mc_pad = w->fused ? w->naux_pad : 0;
      a.nq = u.nq;
      G.blk0[g] = b0;
      b0 += (long long)u.nq * c->nk;
      sm = std::max(sm, sizeof(float2) * 2 * c->nao_tot * (NV + NC));
    }
    for (int g = n; g <= MAXPG; g++) G.blk0[g] = b0;
    G.n = n;
    if (b0 > 0x7fffffffLL) return bse_fail(c0, BSE_EINVAL, "batch: projection grid too large");
    bse_prof_begin(c0, BSE_KP_PROJECT);
    k_proj32_t_grouped<NV, NC><<<(unsigned)b0, bs, sm, c0->stream>>>(G);
    bse_prof_end(c0, BSE_KP_PROJECT);
    bse_count_launch();
    const bse_status s = bse_check_launch(c0, "proj32 (grouped)");
    if (s != BSE_OK) return s;
  }
  return BSE_OK;
}

// Register-blocked second contractions of unfused units with one window, MAXPG per launch.
template <int NV, int NC>
bse_status launch_g2_grouped_t(bse_ctx *c0, const std::vector<BUnit> &us) {
  constexpr int threads = ((NV * NV + 1) / 2) * ((NC * NC + 1) / 2);
  const int bs = std::max(128, std::min(256, (threads + 31) / 32 * 32));
  for (size_t i0 = 0; i0 < us.size(); i0 += MAXPG) {
    const int n = (int)std::min<size_t>(MAXPG, us.size() - i0);
    G2Groups G;
    long long b0 = 0;
    size_t sm = 0;
    for (int g = 0; g < n; g++) {
      const BUnit &u = us[i0 + g];
      bse_ctx *c = u.c;
      SplitWS *w = ws(c);
      G2Group &a = G.g[g];
      a.T = w->T32;
      a.Mc = w->Mc32;
      a.eqp = e_tab(c, w);
      a.naux = c->naux_tot;
      a.n1 = c->mesh[0];
      a.n2 = c->mesh[1];
      a.n3 = c->mesh[2];
      a.q0 = u.q0;
      a.qlist = c->d_qplus;
      a.rows = w->rows;
      a.dim = c->dim;
      a.H = c->h64 ? nullptr : u.H;
      a.H64 = c->h64 ? reinterpret_cast<double2 *>(u.H) : nullptr;
      G.blk0[g] = b0;
      b0 += (long long)u.nq * c->nk;
      sm = std::max(sm, sizeof(float2) * (size_t)(NV * NV + NC * NC) * c->naux_tot);
    }
    for (int g = n; g <= MAXPG; g++) G.blk0[g] = b0;
    G.n = n;
    if (b0 > 0x7fffffffLL) return bse_fail(c0, BSE_EINVAL, "batch: second-contraction grid too large");
    bse_prof_begin(c0, BSE_KP_G2);
    k_g2_32_t_grouped<NV, NC><<<(unsigned)b0, bs, sm, c0->stream>>>(G);
    bse_prof_end(c0, BSE_KP_G2);
    bse_count_launch();
    const bse_status s = bse_check_launch(c0, "g2_32 (grouped)");
    if (s != BSE_OK) return s;
  }
  return BSE_OK;
}

// Fused direct term of fused units with one N tile and conduction window, MAXG per launch.
template <int NP, int BN, int NC, bool TF>
bse_status launch_direct_grouped_t(bse_ctx *c0, const std::vector<BUnit> &us) {
  using Cf = tcd::DCfg<NP, BN>;
  for (size_t i0 = 0; i0 < us.size(); i0 += MAXG) {
    const int n = (int)std::min<size_t>(MAXG, us.size() - i0);
    tcd::DGroups<MAXG> G;
    long long t0 = 0;
    for (int g = 0; g < n; g++) {
      const BUnit &u = us[i0 + g];
      SplitWS *w = ws(u.c);
      G.A[g] = w->tmA_g1;
      G.B[g] = w->tmB_d;
      G.M[g] = w->tmM_d;
      direct_args(u.c, w, u.q0, u.nq, u.H, G.a[g]);
      G.tile0[g] = t0;
      t0 += (long long)G.a[g].tiles_m * G.a[g].tiles_b;
    }
    for (int g = n; g <= MAXG; g++) G.tile0[g] = t0;
    G.n = n;
    if (t0 == 0) continue;
    const int ctas = (int)std::min<long long>(t0, c0->n_sm);
    bse_prof_begin(c0, BSE_KP_G1);
    tcd::k_tc_direct<NP, BN, NC, TF, MAXG><<<ctas, tcd::THREADS, Cf::SMEM, c0->stream>>>(G);
    bse_prof_end(c0, BSE_KP_G1);
    bse_count_launch();
    const bse_status s = bse_check_launch(c0, "tc_direct (grouped)");
    if (s != BSE_OK) return s;
  }
  return BSE_OK;
}

template <int NP, bool TF>
bse_status launch_direct_grouped_nc(bse_ctx *c0, int bn, int nc, const std::vector<BUnit> &us) {
#define BSE_DG(BN_, NC_) \
  if (bn == BN_ && nc == NC_) return launch_direct_grouped_t<NP, BN_, NC_, TF>(c0, us);
  BSE_DG(64, 2) BSE_DG(64, 4) BSE_DG(64, 6) BSE_DG(160, 2) BSE_DG(160, 4) BSE_DG(160, 6)
#undef BSE_DG
  return bse_fail(c0, BSE_EINVAL, "batch: no fused kernel for this tile");
}

bse_status launch_direct_grouped(bse_ctx *c0, const SplitWS *w0, int bn, int nc, const std::vector<BUnit> &us) {
  if (us.empty()) return BSE_OK;
  if (w0->tf32) return launch_direct_grouped_nc<2, true>(c0, bn, nc, us);
  if (w0->np == 3) return launch_direct_grouped_nc<3, false>(c0, bn, nc, us);
  if (w0->np == 2) return launch_direct_grouped_nc<2, false>(c0, bn, nc, us);
  return launch_direct_grouped_nc<1, false>(c0, bn, nc, us);
}

bse_status launch_proj_grouped(bse_ctx *c0, int nv, int nc, int bs, const std::vector<BUnit> &us) {
#define BSE_PG(NV_, NC_) \
  if (nv == NV_ && nc == NC_) return launch_proj_grouped_t<NV_, NC_>(c0, us, bs);
  BSE_PG(2, 2) BSE_PG(2, 4) BSE_PG(2, 6) BSE_PG(4, 2) BSE_PG(4, 4) BSE_PG(4, 6) BSE_PG(6, 2) BSE_PG(6, 4) BSE_PG(6, 6)
#undef BSE_PG
  return bse_fail(c0, BSE_EINVAL, "batch: no register-blocked projection for this window");
}

bse_status launch_g2_grouped(bse_ctx *c0, int nv, int nc, const std::vector<BUnit> &us) {
#define BSE_GG(NV_, NC_) \
  if (nv == NV_ && nc == NC_) return launch_g2_grouped_t<NV_, NC_>(c0, us);
  BSE_GG(2, 2) BSE_GG(2, 4) BSE_GG(2, 6) BSE_GG(4, 2) BSE_GG(4, 4) BSE_GG(4, 6) BSE_GG(6, 2) BSE_GG(6, 4) BSE_GG(6, 6)
#undef BSE_GG
  return bse_fail(c0, BSE_EINVAL, "batch: no register-blocked second contraction for this window");
}

}  // namespace

// The work-list schedule of a batch: the systems ctxs[order[0]], ctxs[order[1]], ...
// (smallest first).  Their (system, q-slab) units are dealt into steps: a step takes the next
// slab of each unfinished system in order, at most one per system (each system has one slab
// buffer), until its M_vv W(q) tiles fill two waves of the SMs; a system's exchange GEMM joins
// the step of its first slab.  Per step, every stage is one launch over the work list of its
// units (per kernel instantiation: window, N tile, block size): the exchange GEMMs, the
// projections, M_vv W(q) of unfused systems, then the second contractions of unfused systems
// and the fused direct term of fused ones.  Every launch goes to the first system's stream;
// stamp(i) is called once system i's work is enqueued.
bse_status split_batch_worklist(bse_ctx **ctxs, void **Hv, const int *order, int n,
                                const std::function<void(int)> &stamp) {
  bse_ctx *c0 = ctxs[order[0]];
  const SplitWS *w0 = ws(c0);
  for (int r = 0; r < n; r++) {
    const bse_ctx *c = ctxs[order[r]];
    const SplitWS *w = ws(ctxs[order[r]]);
    if (c->precision == BSE_FP64 || !w || w->np != w0->np || w->tf32 != w0->tf32)
      return bse_fail(c0, BSE_EINVAL, "batch work list: every system needs the same split precision");
    if (c->stream != c0->stream) return bse_fail(c0, BSE_EINVAL, "batch work list: streams differ");
  }
  bse_once_per_device(c0, BSE_ONCE_GROUPED, set_grouped_attrs_now);
  std::vector<int> next(n, 0), nslab(n);   // by position in order
  for (int r = 0; r < n; r++) {
    const bse_ctx *c = ctxs[order[r]];
    const int nqp = (int)c->qplus.size(), nq = ws(ctxs[order[r]])->nq;
    nslab[r] = (nqp + nq - 1) / nq;
  }
  const long long fill = 2LL * c0->n_sm;
  int left = 0;
  for (int r = 0; r < n; r++) left += nslab[r] > 0;
  struct Unit {
    int r, q0, nq;
  };
  while (left > 0) {
    std::vector<Unit> step;
    long long tiles = 0;
    for (int r = 0; r < n && tiles < fill && (int)step.size() < MAXG; r++) {
      if (next[r] >= nslab[r]) continue;
      const bse_ctx *c = ctxs[order[r]];
      const SplitWS *w = ws(ctxs[order[r]]);
      const int q0 = next[r] * w->nq, nq = std::min(w->nq, (int)c->qplus.size() - q0);
      step.push_back({r, q0, nq});
      const long long mt = w->fused ? (c->nk + w->pairs_d - 1) / w->pairs_d
                                    : (long long)((c->naux_tot + w->bn_g1 - 1) / w->bn_g1) *
                                          ((w->rows + tcg::BM - 1) / tcg::BM);
      tiles += mt * nq;
    }
    {  // exchange GEMMs of the systems starting here
      std::vector<GemmItem> ex;
      for (const Unit &u : step)
        if (u.q0 == 0) {
          const int i = order[u.r];
          GemmItem it;
          it.A = &ws(ctxs[i])->tmA_x;
          it.B = &ws(ctxs[i])->tmB_x;
          exchange_gemm(ctxs[i], ws(ctxs[i]), (float2 *)Hv[i], it.a, it.grid);
          ex.push_back(it);
        }
      const bse_status s = launch_grouped(c0, w0, TC_BN, ex, BSE_KP_EXCH);
      if (s != BSE_OK) return s;
    }
    {  // projections: register-blocked windows grouped by (Nv, Nc, block size), others one by one
      std::map<std::tuple<int, int, int>, std::vector<BUnit>> pg;
      for (const Unit &u : step) {
        const int i = order[u.r];
        bse_ctx *c = ctxs[i];
        SplitWS *w = ws(c);
        if (window_blocked(c)) {
          const int bs = w->proj_bs ? w->proj_bs : std::min(160, (c->naux_tot + 31) / 32 * 32);
          pg[std::make_tuple(c->nv, c->nc, bs)].push_back({c, (float2 *)Hv[i], u.q0, u.nq});
        } else {
          const bse_status s = slab_project(c, w, u.q0, u.nq, (float2 *)Hv[i]);
          if (s != BSE_OK) return s;
        }
      }
      for (const auto &kv : pg) {
        const bse_status s =
            launch_proj_grouped(c0, std::get<0>(kv.first), std::get<1>(kv.first), std::get<2>(kv.first), kv.second);
        if (s != BSE_OK) return s;
      }
    }
    for (int bn : TC_BN_CAND) {
      std::vector<GemmItem> g1;
      for (const Unit &u : step) {
        const int i = order[u.r];
        SplitWS *w = ws(ctxs[i]);
        if (w->fused || w->bn_g1 != bn) continue;
        GemmItem it;
        it.A = &w->tmA_g1;
        it.B = &w->tmB_g1;
        slab_g1(ctxs[i], w, u.q0, u.nq, it.a, it.grid);
        g1.push_back(it);
      }
      const bse_status s = launch_grouped(c0, w0, bn, g1, BSE_KP_G1);
      if (s != BSE_OK) return s;
    }
    {  // the fused direct term grouped by (N tile, Nc); the unfused second contraction grouped
       // by window where the pair's rows fit shared memory, else one by one
      std::map<std::pair<int, int>, std::vector<BUnit>> dg, gg;
      for (const Unit &u : step) {
        const int i = order[u.r];
        bse_ctx *c = ctxs[i];
        SplitWS *w = ws(c);
        const BUnit bu{c, (float2 *)Hv[i], u.q0, u.nq};
        if (w->fused) {
          dg[std::make_pair(w->bn_d, c->nc)].push_back(bu);
        } else if (window_blocked(c) &&
                   sizeof(float2) * (size_t)(c->nv * c->nv + c->nc * c->nc) * c->naux_tot <= 200 * 1024) {
          gg[std::make_pair(c->nv, c->nc)].push_back(bu);
        } else {
          const bse_status s = slab_g2(c, w, u.q0, u.nq, (float2 *)Hv[i]);
          if (s != BSE_OK) return s;
        }
      }
      for (const auto &kv : dg) {
        const bse_status s = launch_direct_grouped(c0, w0, kv.first.first, kv.first.second, kv.second);
        if (s != BSE_OK) return s;
      }
      for (const auto &kv : gg) {
        const bse_status s = launch_g2_grouped(c0, kv.first.first, kv.first.second, kv.second);
        if (s != BSE_OK) return s;
      }
    }
    for (const Unit &u : step)
      if (++next[u.r] == nslab[u.r]) {
        left--;
        stamp(order[u.r]);
      }
  }
  return BSE_OK;
}

// Coupling block B (full BSE) in the split precisions: the exchange part alpha/N_k P X^T as one
// tensor-core GEMM (operand B: pieces of X; B symmetric, so each element is stored at its
// transposed position for coalesced stores) writing every element, then per q-slab the
// conduction-valence projections, T1 = M1 W(q) on tensor cores and -T1 M2^T / N_k added by
// k_g2c_32 (with the transposed copy).
bse_status split_assemble_coupling(bse_ctx *c, void *Bv) {
  SplitWS *w = ws(c);
  float2 *B = (float2 *)Bv;
  const int na = c->naux_tot;
  if (c->nv > MAXB || c->nvc > 64) return bse_fail(c, BSE_EINVAL, "assemble_coupling: band window too wide");
  if (!w->ApB) {
    w->rowsB = c->nk * c->nc * c->nv;
    const size_t per_q = (size_t)w->pp * w->rowsB * w->kmem * w->pbytes + (size_t)c->nk * c->nvc * na * 8 +
                         (size_t)w->rowsB * na * 8;
    const size_t budget = (size_t)1536 << 20;
    w->nqB = (int)std::max<size_t>(1, std::min<size_t>((size_t)c->nk, budget / std::max<size_t>(per_q, 1)));
    w->nqB = std::min(w->nqB, 65535);
    if (c->mesh[2] > 1 && w->nqB >= c->mesh[2]) w->nqB = w->nqB / c->mesh[2] * c->mesh[2];
    const size_t apb = (size_t)w->nqB * w->pp * w->rowsB * w->kmem * w->pbytes,
                 xpb = (size_t)w->pp * c->dim * w->kmem * w->pbytes;
    if (!alloc((void **)&w->ApB, apb) || !alloc((void **)&w->XpB, xpb) ||
        !alloc((void **)&w->McB, (size_t)w->nqB * c->nk * c->nvc * na * 8) ||
        !alloc((void **)&w->TB, (size_t)w->nqB * w->rowsB * na * 8))
      return bse_fail(c, BSE_ENOMEM, "assemble_coupling: workspace allocation failed");
    if (cudaMemsetAsync(w->ApB, 0, apb, c->stream) != cudaSuccess ||
        cudaMemsetAsync(w->XpB, 0, xpb, c->stream) != cudaSuccess)
      return bse_fail(c, BSE_ECUDA, "assemble_coupling: workspace initialisation failed");
    if (!make_map(&w->tmA_B, w->ApB, na, w->rowsB, (long long)w->pp * w->nqB, w->kmem, tcg::BM, w->tf32) ||
        !make_map(&w->tmB_xB, w->XpB, na, c->dim, w->pp, w->kmem, TC_BN, w->tf32))
      return bse_fail(c, BSE_ECUDA, "assemble_coupling: tensor map encoding failed");
  }
  {
    const long long n = c->dim * na;
    k_pieces_f32<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(w->X32, c->dim, na, w->kmem,
                                                                      pieces(w, w->XpB));
    bse_count_launch();
    tcg::Args a{};
    a.rows = (int)c->dim;
    a.n_valid = (int)c->dim;
    a.k_chunks = w->kchunks;
    a.scale = (float)(c->alpha / c->nk);
    a.out = B;
    a.ld_row = 1;
    a.ld_col = c->dim;
    a.conj_out = 0;
    a.out_bstride = 0;
    a.b_batch_planes = 0;
    a.b_base = 0;
    a.qlist = nullptr;
    a.err = c->d_err;
    dim3 grid((unsigned)((c->dim + TC_BN - 1) / TC_BN), (unsigned)((c->dim + tcg::BM - 1) / tcg::BM), 1);
    bse_status s = launch_tc_np(c, w->np, TC_BN, w->tmA_x, w->tmB_xB, a, grid, BSE_KP_EXCH);
    if (s != BSE_OK) return s;
  }
  const int nchunk = (na + 127) / 128;
  const int nqp = (int)c->qplus.size();
  for (int q0 = 0; q0 < nqp; q0 += w->nqB) {
    const int nq = std::min(w->nqB, nqp - q0);
    {
      dim3 grid(nchunk * 2 * c->nc, nq, c->nk);
      size_t sm = sizeof(float2) * 2 * c->nao_tot * c->nb;
      bse_prof_begin(c, BSE_KP_PROJECT);
      if (!fast_cv_kernels(c, w, q0, nq, B, true))
        k_proj_cv32<<<grid, 128, sm, c->stream>>>(y_tab(w), ck_tab(c, w), c->nao_tot, c->nb, c->nv, c->nc, na,
                                                  c->nao_max, c->d_aux_atom, c->d_ao_start, c->d_nao, c->mesh[0],
                                                  c->mesh[1], c->mesh[2], q0, c->d_qplus, w->rowsB, w->kmem,
                                                  pieces(w, w->ApB), w->McB);
      bse_prof_end(c, BSE_KP_PROJECT);
      bse_count_launch();
      bse_status s = bse_check_launch(c, "proj_cv32");
      if (s != BSE_OK) return s;
    }
    {
      tcg::Args a{};
      a.rows = w->rowsB;
      a.n_valid = na;
      a.k_chunks = w->kchunks;
      a.scale = 1.0f;
      a.out = w->TB;
      a.ld_row = 1;
      a.ld_col = w->rowsB;
      a.out_bstride = (long long)w->rowsB * na;
      a.b_batch_planes = 1;
      a.b_base = q0;
      a.qlist = c->d_qplus;
      a.err = c->d_err;
      dim3 grid((unsigned)((na + w->bn_g1 - 1) / w->bn_g1), (unsigned)((w->rowsB + tcg::BM - 1) / tcg::BM), nq);
      bse_status s = launch_tc_np(c, w->np, w->bn_g1, w->tmA_B, w->tmB_g1, a, grid, BSE_KP_G1);
      if (s != BSE_OK) return s;
    }
    {
      dim3 grid(c->nk, nq);
      size_t sm = sizeof(float2) * 2 * c->nvc * G2CH;
      bse_prof_begin(c, BSE_KP_G2);
      if (!fast_cv_kernels(c, w, q0, nq, B, false))
        k_g2c_32<<<grid, 256, sm, c->stream>>>(w->TB, w->McB, c->nv, c->nc, na, c->mesh[0], c->mesh[1], c->mesh[2],
                                               q0, c->d_qplus, w->rowsB, c->dim, B);
      bse_prof_end(c, BSE_KP_G2);
      bse_count_launch();
      bse_status s = bse_check_launch(c, "g2c_32");
      if (s != BSE_OK) return s;
    }
  }
  return BSE_OK;
}

// W[p] = H x[p] for the split-precision context without H: exchange and diagonal, then the
// direct term slab by slab (projections and M_vv W(q) on tensor cores as in split_assemble).
bse_status split_matvec_free(bse_ctx *c, const double2 *x, long long xs, int n_pol, double2 *W) {
  SplitWS *w = ws(c);
  const int na = c->naux_tot;
  if (c->nv * c->nc > 64) return bse_fail(c, BSE_EINVAL, "matrix-free product: band window too wide");
  if (!w->mf_fwd) {
    w->mf_nch = (int)((c->dim + MF_RB - 1) / MF_RB);
    const size_t npart = (size_t)3 * w->nq * c->nk * c->nvc;
    if (!alloc((void **)&w->mf_fwd, npart * sizeof(double2)) || !alloc((void **)&w->mf_bwd, npart * sizeof(double2)) ||
        !alloc((void **)&w->mf_zp, (size_t)3 * w->mf_nch * na * sizeof(double2)) ||
        !alloc((void **)&w->mf_z2, (size_t)3 * na * sizeof(double2)))
      return bse_fail(c, BSE_ENOMEM, "matrix-free product: workspace allocation failed");
  }
  cudaStream_t st = c->stream;
  k_mf_xh<<<dim3(w->mf_nch, n_pol), 256, 0, st>>>(w->X32, c->dim, na, x, xs, w->mf_nch, w->mf_zp);
  k_mf_zv<<<n_pol, 256, sizeof(double2) * na, st>>>(w->mf_zp, w->mf_nch, na, w->V032, w->mf_z2);
  k_mf_xv<<<(unsigned)((c->dim + 7) / 8), 256, 0, st>>>(w->X32, c->dim, na, w->mf_z2, e_tab(c, w), c->nv, c->nc,
                                                        c->alpha / c->nk, x, xs, n_pol, W);
  bse_count_launch(3);
  bse_status s = bse_check_launch(c, "matrix-free exchange");
  if (s != BSE_OK) return s;
  const int nqp = (int)c->qplus.size();
  const int nchunk = (na + 127) / 128;
  // fused path (Nv = 2, 4): T stays in tensor memory and each block is applied from the
  // fused kernel's epilogue (fwd / bwd summed into by atomic adds, so zeroed per slab)
  const bool fused_mf = w->fused && (c->nv == 2 || c->nv == 4);
  const size_t mf_bytes = sizeof(double2) * (size_t)n_pol * w->nq * c->nk * c->nvc;
  for (int q0 = 0; fused_mf && q0 < nqp; q0 += w->nq) {
    const int nq = std::min(w->nq, nqp - q0);
    s = slab_project(c, w, q0, nq, nullptr);
    if (s != BSE_OK) return s;
    if (cudaMemsetAsync(w->mf_fwd, 0, mf_bytes, st) != cudaSuccess ||
        cudaMemsetAsync(w->mf_bwd, 0, mf_bytes, st) != cudaSuccess)
      return bse_fail(c, BSE_ECUDA, "matrix-free product: clearing the slab partials failed");
    tcd::DArgs a;
    direct_args(c, w, q0, nq, nullptr, a);
    a.x = x;
    a.xs = xs;
    a.n_pol = n_pol;
    a.nqs = w->nq;
    a.fwd = w->mf_fwd;
    a.bwd = w->mf_bwd;
    s = launch_direct_mf(c, w, a, -1);
    if (s != BSE_OK) return s;
    const long long n = (long long)n_pol * c->nk * c->nvc;
    k_mf_reduce<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(w->mf_fwd, w->mf_bwd, nq, w->nq, c->nk, c->nvc, n_pol, W);
    bse_count_launch();
    s = bse_check_launch(c, "matrix-free direct slab");
    if (s != BSE_OK) return s;
  }
  for (int q0 = 0; !fused_mf && q0 < nqp; q0 += w->nq) {
    const int nq = std::min(w->nq, nqp - q0);
    {
      dim3 grid(nchunk * (c->nv + c->nc), nq, c->nk);
      size_t sm = sizeof(float2) * 2 * c->nao_tot * c->nb;
      if (!fast_pair_kernels(c, w, q0, nq, nullptr, true))
        k_proj32<<<grid, 128, sm, st>>>(y_tab(w), ck_tab(c, w), c->nao_tot, c->nb, c->nv, c->nc, na, c->nao_max,
                                        c->d_aux_atom, c->d_ao_start, c->d_nao, c->mesh[0], c->mesh[1], c->mesh[2], q0,
                                        c->d_qplus, w->rows, w->kmem, pieces(w, w->Ap), w->Mc32);
      bse_count_launch();
    }
    {
      tcg::Args a{};
      a.rows = w->rows;
      a.n_valid = na;
      a.k_chunks = w->kchunks;
      a.scale = 1.0f;
      a.out = w->T32;
      a.ld_row = 1;
      a.ld_col = w->rows;
      a.out_bstride = (long long)w->rows * na;
      a.b_batch_planes = 1;
      a.b_base = q0;
      a.qlist = c->d_qplus;
      a.err = c->d_err;
      dim3 grid((unsigned)((na + w->bn_g1 - 1) / w->bn_g1), (unsigned)((w->rows + tcg::BM - 1) / tcg::BM), nq);
      s = launch_tc_np(c, w->np, w->bn_g1, w->tmA_g1, w->tmB_g1, a, grid, -1);
      if (s != BSE_OK) return s;
    }
    {
      const size_t sm = sizeof(float2) * ((size_t)(c->nv * c->nv + c->nc * c->nc) * G2CH + (size_t)c->nvc * c->nvc);
      if (!fast_g2mv(c, w, q0, nq, x, xs, n_pol))
        k_g2mv_32<<<dim3(c->nk, nq), 256, sm, st>>>(w->T32, w->Mc32, c->nv, c->nc, na, c->mesh[0], c->mesh[1],
                                                    c->mesh[2], q0, c->d_qplus, w->rows, x, xs, n_pol, w->nq, w->mf_fwd,
                                                    w->mf_bwd);
      const long long n = (long long)n_pol * c->nk * c->nvc;
      k_mf_reduce<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(w->mf_fwd, w->mf_bwd, nq, w->nq, c->nk, c->nvc, n_pol,
                                                               W);
      bse_count_launch(2);
      s = bse_check_launch(c, "matrix-free direct slab");
      if (s != BSE_OK) return s;
    }
  }
  return BSE_OK;
}

// ---- adjoint of the split-precision assembly --------------------------------------------
// dL/dW(q) = -(1/N_k) M_vv(q)^T U(q) with U[(k1,i,j)][nu] = sum_ab Gamma_(k2 j b),(k1 i a)
// M_cc(k1,q)^nu_ab (the same contraction as the FP64 adjoint, k_adjoint.cu), for every q one
// slab at a time: the projections from the FP32 pair table (M_vv written as plain FP32 planes,
// M_cc as the assembly writes it), U in FP32 and the product on CUDA cores with FP32 sums over
// the pairs, each dL/dW(q) stored in FP64 for the FP64 Fourier adjoint.  Its error (~1e-6 of
// the gradient) is the split forward's own.
namespace {

constexpr int APCH = 64;  // nu chunk of the Gamma contraction

__global__ void __launch_bounds__(256) k_adj_phi_mc32(const double2 *__restrict__ Gamma, const float2 *__restrict__ Mc,
                                                      int nv, int nc, int naux, int n1, int n2, int n3, int q0,
                                                      const int *__restrict__ qlist, long long dim,
                                                      float2 *__restrict__ U) {
  extern __shared__ float2 sa32[];
  const int nk = n1 * n2 * n3;
  const int k1 = blockIdx.x, qq = blockIdx.y, q = qlist[q0 + qq];
  const int k2 = kdiff(k1, q, n1, n2, n3);
  const int nvv = nv * nv, ncc = nc * nc, nvc = nv * nc;
  float2 *phi = sa32;                // [nvv][ncc]
  float2 *mcs = sa32 + nvv * ncc;    // [ncc][APCH]
  for (int e = threadIdx.x; e < nvv * ncc; e += blockDim.x) {
    const int ij = e / ncc, ab = e % ncc;
    const int i = ij / nv, j = ij % nv, a = ab / nc, b = ab % nc;
    const double2 g = Gamma[((long long)k2 * nvc + j * nc + b) * dim + (long long)k1 * nvc + i * nc + a];
    phi[e] = make_float2((float)g.x, (float)g.y);
  }
  const float2 *Mk = Mc + ((long long)qq * nk + k1) * ncc * naux;
  float2 *Uk = U + ((long long)qq * nk + k1) * nvv * naux;
  for (int n0 = 0; n0 < naux; n0 += APCH) {
    const int nn = min(APCH, naux - n0);
    __syncthreads();
    for (int e = threadIdx.x; e < ncc * APCH; e += blockDim.x) {
      const int ab = e / APCH, u = e % APCH;
      mcs[e] = u < nn ? Mk[(long long)ab * naux + n0 + u] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nvv * APCH; e += blockDim.x) {
      const int ij = e / APCH, u = e % APCH;
      if (u >= nn) continue;
      float xr = 0.f, xi = 0.f;
      for (int ab = 0; ab < ncc; ab++) {
        const float2 f = phi[ij * ncc + ab], m = mcs[ab * APCH + u];
        xr = fmaf(f.x, m.x, fmaf(-f.y, m.y, xr));
        xi = fmaf(f.x, m.y, fmaf(f.y, m.x, xi));
      }
      Uk[(long long)ij * naux + n0 + u] = make_float2(xr, xi);
    }
  }
}

// C[cidx[q0 + b]] = alpha A[b]^T B[b] for complex A [K x M] in two FP32 planes (row pitch lda,
// plane pitch `plane`, batch pitch 2 plane) and B [K x N] complex64 (batch pitch sB): FP32
// products and sums, stored as FP64.  64 x 64 output tiles, 4 x 4 per thread.
__global__ void __launch_bounds__(256) k_cgemm_tn32(int M, int N, int K, const float *__restrict__ A, long long plane,
                                                    int lda, const float2 *__restrict__ B, long long sB,
                                                    double2 *__restrict__ C, long long sC, const int *__restrict__ cidx,
                                                    int q0, double alpha) {
  __shared__ float2 As[16][64];
  __shared__ float2 Bs[16][64];
  const int bz = blockIdx.z;
  const float *Are = A + (long long)bz * 2 * plane, *Aim = Are + plane;
  B += (long long)bz * sB;
  C += (long long)cidx[q0 + bz] * sC;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int row0 = blockIdx.y * 64, col0 = blockIdx.x * 64;
  float2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; i++)
#pragma unroll
    for (int j = 0; j < 4; j++) acc[i][j] = make_float2(0.f, 0.f);
  for (int k0 = 0; k0 < K; k0 += 16) {
    for (int e = threadIdx.x; e < 1024; e += 256) {
      const int kk = e / 64, r = e % 64, gk = k0 + kk;
      const long long ia = (long long)gk * lda + row0 + r;
      As[kk][r] = (gk < K && row0 + r < M) ? make_float2(Are[ia], Aim[ia]) : make_float2(0.f, 0.f);
      Bs[kk][r] = (gk < K && col0 + r < N) ? B[(long long)gk * N + col0 + r] : make_float2(0.f, 0.f);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; kk++) {
      float2 a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; i++) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; j++) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) {
          acc[i][j].x = fmaf(a[i].x, b[j].x, fmaf(-a[i].y, b[j].y, acc[i][j].x));
          acc[i][j].y = fmaf(a[i].x, b[j].y, fmaf(a[i].y, b[j].x, acc[i][j].y));
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

// The projections of transfers qlist[q0 ..] into the given M_vv buffer (register-blocked
// windows, else the generic kernel), M_cc as the unfused assembly writes it.
template <int NV, int NC>
void launch_proj_list(bse_ctx *c, SplitWS *w, int q0, int nq, const int *qlist, PieceBuf Av) {
  const int na = c->naux_tot;
  const int bs = w->proj_bs ? w->proj_bs : std::min(160, (na + 31) / 32 * 32);
  const size_t sm = sizeof(float2) * 2 * c->nao_tot * (NV + NC);
  k_proj32_t<NV, NC><<<dim3(nq, c->nk), bs, sm, c->stream>>>(y_tab(w), ck_tab(c, w), c->nao_tot, na, c->nao_max,
                                                             c->d_aux_atom, c->d_ao_start, c->d_nao, c->mesh[0],
                                                             c->mesh[1], c->mesh[2], q0, qlist, w->rows, w->kmem, Av,
                                                             w->Mc32, 0);
}

void project_list(bse_ctx *c, SplitWS *w, int q0, int nq, const int *qlist, PieceBuf Av) {
#define BSE_PL(NV, NC)                                   \
  if (c->nv == NV && c->nc == NC) {                      \
    launch_proj_list<NV, NC>(c, w, q0, nq, qlist, Av);   \
    return;                                              \
  }
  BSE_PL(2, 2) BSE_PL(2, 4) BSE_PL(2, 6) BSE_PL(4, 2) BSE_PL(4, 4) BSE_PL(4, 6) BSE_PL(6, 2) BSE_PL(6, 4) BSE_PL(6, 6)
#undef BSE_PL
  const int na = c->naux_tot;
  dim3 grid(((na + 127) / 128) * (c->nv + c->nc), nq, c->nk);
  const size_t sm = sizeof(float2) * 2 * c->nao_tot * c->nb;
  k_proj32<<<grid, 128, sm, c->stream>>>(y_tab(w), ck_tab(c, w), c->nao_tot, c->nb, c->nv, c->nc, na, c->nao_max,
                                         c->d_aux_atom, c->d_ao_start, c->d_nao, c->mesh[0], c->mesh[1], c->mesh[2],
                                         q0, qlist, w->rows, w->kmem, Av, w->Mc32);
}

}  // namespace

bse_status split_adjoint_slabs(bse_ctx *c, const double2 *Gamma) {
  SplitWS *w = ws(c);
  const int na = c->naux_tot;
  if (!w->adjMv && !alloc((void **)&w->adjMv, sizeof(float) * 2 * (size_t)w->nq * w->rows * w->kmem))
    return bse_fail(c, BSE_ENOMEM, "adjoint: slab allocation failed");
  const size_t sm = sizeof(float2) * (c->nv * c->nv * c->nc * c->nc + c->nc * c->nc * APCH);
  if (sm > 200 * 1024) return bse_fail(c, BSE_EINVAL, "adjoint: band window too wide");
  if (sm > 48 * 1024) cudaFuncSetAttribute(k_adj_phi_mc32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  const long long plane = (long long)w->rows * w->kmem;
  for (int q0 = 0; q0 < c->nk; q0 += w->nq) {
    const int nq = std::min(w->nq, c->nk - q0);
    project_list(c, w, q0, nq, c->d_qall, PieceBuf{w->adjMv, 1, 2});
    k_adj_phi_mc32<<<dim3(c->nk, nq), 256, sm, c->stream>>>(Gamma, w->Mc32, c->nv, c->nc, na, c->mesh[0], c->mesh[1],
                                                          c->mesh[2], q0, c->d_qall, c->dim, w->T32);
    dim3 grid((na + 63) / 64, (na + 63) / 64, nq);
    k_cgemm_tn32<<<grid, 256, 0, c->stream>>>(na, na, w->rows, w->adjMv, plane, w->kmem, w->T32,
                                              (long long)w->rows * na, c->Aq, (long long)na * na, c->d_qall, q0,
                                              -1.0 / c->nk);
    bse_count_launch(3);
    const bse_status s = bse_check_launch(c, "adjoint slab (split)");
    if (s != BSE_OK) return s;
  }
  return BSE_OK;
}

bse_status split_matfree_hmax(bse_ctx *c, double *hmax) {
  SplitWS *w = ws(c);
  k_mf_hmax<<<1, 256, 0, c->stream>>>(e_tab(c, w), (long long)c->nk * c->nb, hmax);
  bse_count_launch();
  return bse_check_launch(c, "matrix-free scale");
}

// ---- autotuner ----------------------------------------------------------------------------
// Picks the N tile of the T = M_vv W(q) tensor-core GEMM by timing one q-slab launch per
// candidate (values do not change the timing, so no inputs are needed), keeps the fastest,
// and re-encodes the B-operand tensor map.  Results are cached per shape in the process.
namespace {
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int>, int> g_tune_cache;
std::map<std::tuple<int, int, int, int, int, int>, int> g_tune_proj;

// Threads per block of the register-blocked projection: one slab of projections timed for each
// candidate (a warp multiple up to the kernel's 160-thread bound and the ABF count); the
// fastest is kept for this context and cached per shape.  0 when the window has no
// register-blocked kernel.
int tune_projection(bse_ctx *c, SplitWS *w) {
  const int na = c->naux_tot;
  const int nq = std::min(w->nq, (int)c->qplus.size());
  const auto key = std::make_tuple(na, w->rows, nq, w->np + (w->tf32 ? 10 : 0), c->nv, c->nc);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_proj.find(key);
    if (it != g_tune_proj.end()) return it->second;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  int best_bs = 0;
  const int cap = std::min(160, (na + 31) / 32 * 32);
  for (int bs = 32; bs <= cap; bs += 32) {
    w->proj_bs = bs;
    if (!fast_pair_kernels(c, w, 0, nq, nullptr, true, w->fused ? w->naux_pad : 0)) break;  // warm-up
    float t = 0.f;
    for (int rep = 0; rep < 3; rep++) {
      cudaEventRecord(e0, c->stream);
      fast_pair_kernels(c, w, 0, nq, nullptr, true, w->fused ? w->naux_pad : 0);
      cudaEventRecord(e1, c->stream);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      t += ms;
    }
    bse_count_launch(4);
    if (t < best) {
      best = t;
      best_bs = bs;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  w->proj_bs = 0;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_proj[key] = best_bs;
  }
  return best_bs;
}
}  // namespace

bse_status split_autotune(bse_ctx *c, int *chosen, int *chosen_proj) {
  SplitWS *w = ws(c);
  const int na = c->naux_tot;
  {
    const bool prof = c->prof;
    c->prof = false;
    const int pbs = tune_projection(c, w);
    c->prof = prof;
    w->proj_bs = pbs;
    if (chosen_proj) *chosen_proj = pbs;
  }
  const auto key = std::make_tuple(na, w->rows, std::min(w->nq, (int)c->qplus.size()), w->np + (w->tf32 ? 10 : 0));
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      w->bn_g1 = it->second;
      if (!make_map(&w->tmB_g1, w->Wp, na, na, (long long)w->pp * c->nk, w->kmem, w->bn_g1, w->tf32))
        return bse_fail(c, BSE_ECUDA, "autotune: tensor map encoding failed");
      if (chosen) *chosen = w->bn_g1;
      return BSE_OK;
    }
  }
  const int nq = std::min(w->nq, (int)c->qplus.size());
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const bool prof = c->prof;
  c->prof = false;
  float best = 1e30f;
  int best_bn = TC_BN;
  for (int bn : TC_BN_CAND) {
    CUtensorMap tB;
    if (!make_map(&tB, w->Wp, na, na, (long long)w->pp * c->nk, w->kmem, bn, w->tf32)) continue;
    tcg::Args a{};
    a.rows = w->rows;
    a.n_valid = na;
    a.k_chunks = w->kchunks;
    a.scale = 1.0f;
    a.out = w->T32;
    a.ld_row = 1;
    a.ld_col = w->rows;
    a.out_bstride = (long long)w->rows * na;
    a.b_batch_planes = 1;
    a.b_base = 0;
    a.qlist = c->d_qplus;
    a.err = c->d_err;
    dim3 grid((unsigned)((na + bn - 1) / bn), (unsigned)((w->rows + tcg::BM - 1) / tcg::BM), nq);
    float t = 0.f;
    bool ok = launch_tc_np(c, w->np, bn, w->tmA_g1, tB, a, grid, -1) == BSE_OK;  // warm-up
    for (int rep = 0; rep < 3 && ok; rep++) {
      cudaEventRecord(e0, c->stream);
      ok = launch_tc_np(c, w->np, bn, w->tmA_g1, tB, a, grid, -1) == BSE_OK;
      cudaEventRecord(e1, c->stream);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      t += ms;
    }
    if (ok && t < best) {
      best = t;
      best_bn = bn;
    }
  }
  c->prof = prof;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  w->bn_g1 = best_bn;
  if (!make_map(&w->tmB_g1, w->Wp, na, na, (long long)w->pp * c->nk, w->kmem, w->bn_g1, w->tf32))
    return bse_fail(c, BSE_ECUDA, "autotune: tensor map encoding failed");
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = best_bn;
  }
  if (chosen) *chosen = best_bn;
  return bse_check_launch(c, "autotune");
}
