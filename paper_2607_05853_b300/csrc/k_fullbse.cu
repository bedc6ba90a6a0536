// Full BSE (§II.C): the spectrum with the Y term (Eq. full_BSE_epsilon2) and the lowest
// paired excitation energies, from the resonant block A and the coupling block B.
//
// H = [[A, B], [-B*, -A*]] = J M with J = diag(1, -1) and M = [[A, B], [B*, A*]], Hermitian
// positive definite for a stable excited state.  H is self-adjoint in the inner product
// <x, y>_M = x^H M y, so a Lanczos recursion in that inner product gives a real symmetric
// tridiagonal T whose Ritz values approximate the +-Omega pairs.
//
// Spectrum.  Start vector v = (u, conj u) with u = conj(d) the TDA dipole vector.  For the
// M-normalised eigenvectors Zh of H, |<Zh, v>_M|^2 = Omega_S |d X_S - conj(d) Y_S|^2 at both
// +Omega_S and -Omega_S, so
//   eps2(w) = pref <v, f_w(H) v>_M,   f_w(t) = L_eta(w - |t|) / (2 |t|),
// evaluated as the Gauss quadrature beta0^2 sum_i z_i0^2 f_w(theta_i) over the eigenpairs
// (theta_i, z_i) of T (exact once the Krylov space is invariant).  v is even under the
// antilinear swap C(x, y) = (conj y, conj x), which anticommutes with H: the Krylov basis
// alternates parity, every a_j vanishes, and for an even order m the Ritz values pair as
// +-theta with theta^2 the Rayleigh-Ritz values of H^2 on the even vectors, so |theta| never
// falls below the lowest Omega and f_w stays bounded.  Odd orders are cut to even.
//
// Lowest excitations.  The same recursion from a random C-even start; the smallest positive
// Ritz values of the even-order T (extremal for H^2) with residuals |b_m z_i,m|.
//
// Per step, with p_j = M q_j from the previous product: a_j = p_j^H J p_j,
// r = J p_j - a_j q_j - b_{j-1} q_{j-1} (= H q_j - ...), two passes of full
// reorthogonalisation in the M inner product (c_i = p_i^H r; r -= c_i q_i), then the one
// product s = M r (A and B each read once for all polarisations), b_j = sqrt(r^H s),
// q_{j+1} = r / b_j, p_{j+1} = s / b_j.  Forming s from the finished r keeps every p_j an
// explicit product: propagating s through the three-term recurrence instead lets the error
// of p_j grow by b_j / b_{j+1} every two steps (the b_j alternate in size), and M
// orthogonality is lost within tens of steps.  A negative r^H s (M not positive definite)
// stops the recursion of that polarisation and sets the device error word.
#include <algorithm>
#include <cmath>
#include <vector>

#include "bse_internal.cuh"

namespace {

template <class T> struct Cplx;
template <> struct Cplx<double2> { using R = double; };
template <> struct Cplx<float2> { using R = float; };

constexpr int FM_CC = 128;  // columns staged per pass

__device__ __forceinline__ float mfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double mfma(double a, double b, double c) { return fma(a, b, c); }

// S[p] = M V[p] for V[p] = (x, y) of length 2 dim:
//   upper = A x + B y,   lower = B* x + A* y = conj(B conj(x) + A conj(y)).
// Each warp owns RPW rows; lanes stride the columns; arithmetic in the element precision
// (FP32 for complex64 A, B), lane sums combined in FP64.
template <class T, int NP, int RPW>
__global__ void __launch_bounds__(256) k_mmv(const T *__restrict__ A, const T *__restrict__ B, long long dim,
                                             const double2 *__restrict__ V, long long vs,
                                             double2 *__restrict__ S, long long ss) {
  using R = typename Cplx<T>::R;
  __shared__ T xs[NP][FM_CC], ys[NP][FM_CC];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const long long r0 = ((long long)blockIdx.x * 8 + warp) * RPW;
  T ax[RPW][NP], ay[RPW][NP], by[RPW][NP], bx[RPW][NP];  // A x, A conj(y), B y, B conj(x)
#pragma unroll
  for (int r = 0; r < RPW; r++)
#pragma unroll
    for (int p = 0; p < NP; p++) {
      ax[r][p].x = ax[r][p].y = ay[r][p].x = ay[r][p].y = 0;
      by[r][p].x = by[r][p].y = bx[r][p].x = bx[r][p].y = 0;
    }
  for (long long c0 = 0; c0 < dim; c0 += FM_CC) {
    __syncthreads();
    for (int t = threadIdx.x; t < NP * FM_CC; t += blockDim.x) {
      const int p = t / FM_CC, cc = t % FM_CC;
      const long long c = c0 + cc;
      double2 x = make_double2(0, 0), y = make_double2(0, 0);
      if (c < dim) {
        x = V[p * vs + c];
        y = V[p * vs + dim + c];
      }
      xs[p][cc].x = (R)x.x;
      xs[p][cc].y = (R)x.y;
      ys[p][cc].x = (R)y.x;
      ys[p][cc].y = (R)y.y;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RPW; r++) {
      const long long row = r0 + r;
      if (row >= dim) continue;
      const T *ar = A + row * dim + c0, *br = B + row * dim + c0;
#pragma unroll
      for (int t = 0; t < FM_CC / 32; t++) {
        const int cc = lane + 32 * t;
        if (c0 + cc < dim) {
          const T a = ar[cc], b = br[cc];
#pragma unroll
          for (int p = 0; p < NP; p++) {
            const T x = xs[p][cc], y = ys[p][cc];
            ax[r][p].x = mfma(a.x, x.x, mfma(-a.y, x.y, ax[r][p].x));
            ax[r][p].y = mfma(a.x, x.y, mfma(a.y, x.x, ax[r][p].y));
            ay[r][p].x = mfma(a.x, y.x, mfma(a.y, y.y, ay[r][p].x));
            ay[r][p].y = mfma(a.y, y.x, mfma(-a.x, y.y, ay[r][p].y));
            by[r][p].x = mfma(b.x, y.x, mfma(-b.y, y.y, by[r][p].x));
            by[r][p].y = mfma(b.x, y.y, mfma(b.y, y.x, by[r][p].y));
            bx[r][p].x = mfma(b.x, x.x, mfma(b.y, x.y, bx[r][p].x));
            bx[r][p].y = mfma(b.y, x.x, mfma(-b.x, x.y, bx[r][p].y));
          }
        }
      }
    }
  }
#pragma unroll
  for (int r = 0; r < RPW; r++)
#pragma unroll
    for (int p = 0; p < NP; p++) {
      double v[8] = {(double)ax[r][p].x, (double)ax[r][p].y, (double)ay[r][p].x, (double)ay[r][p].y,
                     (double)by[r][p].x, (double)by[r][p].y, (double)bx[r][p].x, (double)bx[r][p].y};
#pragma unroll
      for (int k = 0; k < 8; k++)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
      const long long row = r0 + r;
      if (lane == 0 && row < dim) {
        S[p * ss + row] = make_double2(v[0] + v[4], v[1] + v[5]);
        S[p * ss + dim + row] = make_double2(v[6] + v[2], -(v[7] + v[3]));
      }
    }
}

constexpr int VB = 256;          // threads of the vector kernels
constexpr int VE = 8;            // elements per thread in the partial dots
constexpr int VCH = VB * VE;     // elements per partial

__device__ __forceinline__ double bsum(double v, double *red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < VB / 32; i++) s += red[i];
  __syncthreads();
  return s;  // every thread
}

// part[p][blk] = sum over the chunk of conj(X) Y, the lower half weighted by sgn.
__global__ void __launch_bounds__(VB) k_fl_dot_part(const double2 *__restrict__ X, long long xs,
                                                    const double2 *__restrict__ Y, long long ys, long long dim,
                                                    double sgn, const int *__restrict__ live, int j,
                                                    double2 *__restrict__ part, int nblk) {
  __shared__ double red[VB / 32];
  const int p = blockIdx.y;
  if (live && j >= live[p]) return;
  const long long n2 = 2 * dim, e0 = (long long)blockIdx.x * VCH;
  double sr = 0.0, si = 0.0;
  for (int k = 0; k < VE; k++) {
    const long long e = e0 + k * VB + threadIdx.x;
    if (e < n2) {
      const double2 x = X[p * xs + e], y = Y[p * ys + e];
      const double w = e >= dim ? sgn : 1.0;
      sr += w * (x.x * y.x + x.y * y.y);
      si += w * (x.x * y.y - x.y * y.x);
    }
  }
  sr = bsum(sr, red);
  si = bsum(si, red);
  if (threadIdx.x == 0) part[(long long)p * nblk + blockIdx.x] = make_double2(sr, si);
}

__device__ __forceinline__ double2 sum_parts(const double2 *part, int nblk, double *red) {
  double sr = 0.0, si = 0.0;
  for (int i = threadIdx.x; i < nblk; i += VB) {
    sr += part[i].x;
    si += part[i].y;
  }
  sr = bsum(sr, red);
  si = bsum(si, red);
  return make_double2(sr, si);
}

// Start: R = v = (u, conj u).  Random C-even start when u is null.
__device__ __forceinline__ unsigned long long mix64(unsigned long long x) {  // SplitMix64 finaliser
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}
__global__ void k_fl_start(const double2 *__restrict__ u, long long dim, unsigned long long seed,
                           double2 *__restrict__ R, long long vs) {
  const int p = blockIdx.y;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= dim) return;
  double2 x;
  if (u) {
    x = u[(long long)p * dim + e];
  } else {
    const unsigned long long r1 = mix64(seed ^ (2ull * (unsigned long long)e));
    const unsigned long long r2 = mix64(seed ^ (2ull * (unsigned long long)e + 1ull));
    x = make_double2((double)(r1 >> 11) * (1.0 / 9007199254740992.0) - 0.5,
                     (double)(r2 >> 11) * (1.0 / 9007199254740992.0) - 0.5);
  }
  R[p * vs + e] = x;
  R[p * vs + dim + e] = make_double2(x.x, -x.y);  // conj(x)
}

// beta0^2 = v^H M v (v = R, S = M v); q_0 = v / beta0, p_0 = S / beta0.
__global__ void __launch_bounds__(VB) k_fl_norm0(const double2 *__restrict__ R, const double2 *__restrict__ S,
                                                 long long vs, long long dim, const double2 *__restrict__ part,
                                                 int nblk, double2 *__restrict__ Q, double2 *__restrict__ P,
                                                 long long qs, double *__restrict__ beta0, int *__restrict__ meff,
                                                 int *err, float2 *__restrict__ Q32, float2 *__restrict__ P32) {
  __shared__ double red[VB / 32];
  const int p = blockIdx.y;
  const double b2 = sum_parts(part + (long long)p * nblk, nblk, red).x;
  if (!(b2 > 0.0)) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      beta0[p] = 0.0;
      meff[p] = 0;
      if (b2 < 0.0) atomicOr(err, BSE_DERR_INDEFINITE);
    }
    return;
  }
  const double b = sqrt(b2), inv = 1.0 / b;
  if (blockIdx.x == 0 && threadIdx.x == 0) beta0[p] = b;
  for (long long e = (long long)blockIdx.x * VB + threadIdx.x; e < 2 * dim; e += (long long)gridDim.x * VB) {
    const double2 v = R[p * vs + e], sv = S[p * vs + e];
    const double2 qv = make_double2(v.x * inv, v.y * inv), pv = make_double2(sv.x * inv, sv.y * inv);
    Q[p * qs + e] = qv;
    P[p * qs + e] = pv;
    if (Q32) {
      Q32[p * qs + e] = make_float2((float)qv.x, (float)qv.y);
      P32[p * qs + e] = make_float2((float)pv.x, (float)pv.y);
    }
  }
}

// a_j = p_j^H J p_j (partials in part); R = J p_j - a_j q_j - b_{j-1} q_{j-1}.
__global__ void __launch_bounds__(VB) k_fl_axpy(double2 *__restrict__ R, long long vs,
                                                long long dim, const double2 *__restrict__ Q,
                                                const double2 *__restrict__ P, long long qs, int j,
                                                double *__restrict__ a, const double *__restrict__ b, int ldab,
                                                const int *__restrict__ meff, const double2 *__restrict__ part,
                                                int nblk) {
  __shared__ double red[VB / 32];
  const int p = blockIdx.y;
  if (j >= meff[p]) return;
  const double aj = sum_parts(part + (long long)p * nblk, nblk, red).x;
  if (blockIdx.x == 0 && threadIdx.x == 0) a[p * ldab + j] = aj;
  const double bj = j > 0 ? b[p * ldab + j - 1] : 0.0;
  const long long n2 = 2 * dim;
  const double2 *qj = Q + p * qs + (long long)j * n2, *pj = P + p * qs + (long long)j * n2;
  const double2 *qm = j > 0 ? qj - n2 : qj;
  for (long long e = (long long)blockIdx.x * VB + threadIdx.x; e < n2; e += (long long)gridDim.x * VB) {
    const double sg = e >= dim ? -1.0 : 1.0;
    const double2 pv = pj[e], qv = qj[e], qmv = qm[e];
    R[p * vs + e] = make_double2(sg * pv.x - aj * qv.x - bj * qmv.x, sg * pv.y - aj * qv.y - bj * qmv.y);
  }
}

// coef[p][i] = p_i^H r, i <= j  (grid: x = i, y = p)
__global__ void __launch_bounds__(VB) k_fl_rdots(const double2 *__restrict__ R, long long vs, long long dim,
                                                 const double2 *__restrict__ P, long long qs, int j,
                                                 double2 *__restrict__ coef, int ldc, const int *__restrict__ meff) {
  __shared__ double red[VB / 32];
  const int i = blockIdx.x, p = blockIdx.y;
  if (j >= meff[p] || i > j) return;
  const long long n2 = 2 * dim;
  const double2 *pi = P + p * qs + (long long)i * n2, *r = R + p * vs;
  double sr = 0.0, si = 0.0;
  for (long long e = threadIdx.x; e < n2; e += VB) {
    const double2 x = pi[e], y = r[e];
    sr += x.x * y.x + x.y * y.y;
    si += x.x * y.y - x.y * y.x;
  }
  sr = bsum(sr, red);
  si = bsum(si, red);
  if (threadIdx.x == 0) coef[p * ldc + i] = make_double2(sr, si);
}

// r -= sum_i coef_i q_i
__global__ void __launch_bounds__(VB) k_fl_rupdate(double2 *__restrict__ R, long long vs, long long dim,
                                                   const double2 *__restrict__ Q, long long qs, int j,
                                                   const double2 *__restrict__ coef, int ldc,
                                                   const int *__restrict__ meff) {
  const int p = blockIdx.y;
  if (j >= meff[p]) return;
  const long long n2 = 2 * dim;
  const long long e = (long long)blockIdx.x * VB + threadIdx.x;
  if (e >= n2) return;
  double2 r = R[p * vs + e];
  for (int i = 0; i <= j; i++) {
    const double2 c = coef[p * ldc + i];
    const double2 q = Q[p * qs + (long long)i * n2 + e];
    r.x -= c.x * q.x - c.y * q.y;
    r.y -= c.x * q.y + c.y * q.x;
  }
  R[p * vs + e] = r;
}

// b_j^2 = r^H s; stop on breakdown (b_j <= 1e-12 b_0) or a negative value (M indefinite);
// else q_{j+1} = r / b_j, p_{j+1} = s / b_j.
__global__ void __launch_bounds__(VB) k_fl_scale(const double2 *__restrict__ R, const double2 *__restrict__ S,
                                                 long long vs, long long dim, double2 *__restrict__ Q,
                                                 double2 *__restrict__ P, long long qs, int j, int n_steps,
                                                 double *__restrict__ b, int ldab, int *__restrict__ meff,
                                                 const double2 *__restrict__ part, int nblk, int *err,
                                                 float2 *__restrict__ Q32, float2 *__restrict__ P32) {
  __shared__ double red[VB / 32];
  const int p = blockIdx.y;
  if (j >= meff[p]) return;
  const double b2 = sum_parts(part + (long long)p * nblk, nblk, red).x;
  const double bj = b2 > 0.0 ? sqrt(b2) : 0.0;
  if (blockIdx.x == 0 && threadIdx.x == 0) b[p * ldab + j] = bj;
  if (j == n_steps - 1) return;
  const double ref = j > 0 ? b[p * ldab] : bj;
  const double tol = 1e-12 * ref;
  if (!(bj > tol)) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      meff[p] = j + 1;
      if (b2 < -(tol * tol + 1e-300)) atomicOr(err, BSE_DERR_INDEFINITE);
    }
    return;
  }
  const double inv = 1.0 / bj;
  const long long n2 = 2 * dim;
  for (long long e = (long long)blockIdx.x * VB + threadIdx.x; e < n2; e += (long long)gridDim.x * VB) {
    const double2 r = R[p * vs + e], s = S[p * vs + e];
    const long long o = p * qs + (long long)(j + 1) * n2 + e;
    const double2 qv = make_double2(r.x * inv, r.y * inv), pv = make_double2(s.x * inv, s.y * inv);
    Q[o] = qv;
    P[o] = pv;
    if (Q32) {
      Q32[o] = make_float2((float)qv.x, (float)qv.y);
      P32[o] = make_float2((float)pv.x, (float)pv.y);
    }
  }
}

// Operands of the half-read products: Z[0][p] = x, Z[1][p] = conj(y), Z[2][p] = y,
// Z[3][p] = conj(x) for V[p] = (x, y), complex64.
__global__ void k_fl_pack(const double2 *__restrict__ V, long long vs, long long dim, int n_pol,
                          float2 *__restrict__ Z) {
  const int p = blockIdx.y;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= dim) return;
  const double2 x = V[p * vs + e], y = V[p * vs + dim + e];
  const long long zs = (long long)n_pol * dim, o = (long long)p * dim + e;
  Z[o] = make_float2((float)x.x, (float)x.y);
  Z[zs + o] = make_float2((float)y.x, -(float)y.y);
  Z[2 * zs + o] = make_float2((float)y.x, (float)y.y);
  Z[3 * zs + o] = make_float2((float)x.x, -(float)x.y);
}

// S[p] = (A x + B y, conj(B conj(x) + A conj(y))) from W[k][p] = product k of k_fl_pack's order.
__global__ void k_fl_combine(const double2 *__restrict__ W, long long dim, int n_pol, double2 *__restrict__ S,
                             long long ss) {
  const int p = blockIdx.y;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= dim) return;
  const long long ws = (long long)n_pol * dim, o = (long long)p * dim + e;
  const double2 ax = W[o], ay = W[ws + o], by = W[2 * ws + o], bx = W[3 * ws + o];
  S[p * ss + e] = make_double2(ax.x + by.x, ax.y + by.y);
  S[p * ss + dim + e] = make_double2(bx.x + ay.x, -(bx.y + ay.y));
}

// Eigenvalues of each tridiagonal (a_p, b_p; order mq[p]) with the first and last components
// of every eigenvector -- all the Gauss quadrature and the residual bounds need.  The implicit
// QL algorithm with Wilkinson-type shifts (Bowdler, Martin, Reinsch and Wilkinson, Numer. Math.
// 11 (1968) 293) run by one thread on shared-memory copies of the diagonal, off-diagonal and the
// two tracked rows of the eigenvector matrix (started at the identity), each rotation applied
// to them as it is formed.  Output: theta [p][mmax], z0 [p][mmax], zl [p][mmax].
constexpr int QL_SWEEPS = 60;
__global__ void k_tridiag_ql_ends(const double *__restrict__ a, const double *__restrict__ b, int ldab,
                                  const int *__restrict__ mq, int mmax, double *__restrict__ theta,
                                  double *__restrict__ z0o, double *__restrict__ zlo, int *err) {
  extern __shared__ double qs_[];
  const int p = blockIdx.x, m = mq[p];
  double *d = qs_, *e = d + m, *z0 = e + m, *zl = z0 + m;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    d[i] = a[p * ldab + i];
    e[i] = i < m - 1 ? b[p * ldab + i] : 0.0;
    z0[i] = i == 0 ? 1.0 : 0.0;
    zl[i] = i == m - 1 ? 1.0 : 0.0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int l = 0; l < m; l++) {
      for (int sweep = 0;; sweep++) {
        int mm = l;
        while (mm < m - 1) {
          const double scale = fabs(d[mm]) + fabs(d[mm + 1]);
          if (fabs(e[mm]) <= 1e-16 * scale || fabs(e[mm]) < 1e-300) break;
          mm++;
        }
        if (mm == l) break;
        if (sweep >= QL_SWEEPS) {
          atomicOr(err, BSE_DERR_BOUNDS);
          break;
        }
        double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
        double r = hypot(g, 1.0);
        g = d[mm] - d[l] + e[l] / (g + copysign(r, g));
        double sn = 1.0, cn = 1.0, pp = 0.0;
        bool split = false;
        for (int i = mm - 1; i >= l; i--) {
          const double f = sn * e[i], bb = cn * e[i];
          r = hypot(f, g);
          e[i + 1] = r;
          if (r == 0.0) {
            d[i + 1] -= pp;
            e[mm] = 0.0;
            split = true;
            break;
          }
          sn = f / r;
          cn = g / r;
          g = d[i + 1] - pp;
          r = (d[i] - g) * sn + 2.0 * cn * bb;
          pp = sn * r;
          d[i + 1] = g + pp;
          g = cn * r - bb;
          const double a0 = z0[i], a1 = z0[i + 1], c0 = zl[i], c1 = zl[i + 1];
          z0[i + 1] = sn * a0 + cn * a1;
          z0[i] = cn * a0 - sn * a1;
          zl[i + 1] = sn * c0 + cn * c1;
          zl[i] = cn * c0 - sn * c1;
        }
        if (!split) {
          d[l] -= pp;
          e[l] = g;
          e[mm] = 0.0;
        }
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < mmax; i += blockDim.x) {
    theta[(long long)p * mmax + i] = i < m ? d[i] : 0.0;
    z0o[(long long)p * mmax + i] = i < m ? z0[i] : 0.0;
    zlo[(long long)p * mmax + i] = i < m ? zl[i] : 0.0;
  }
}

__global__ void k_fl_even(const int *__restrict__ meff, int n_pol, int *__restrict__ meven) {
  const int p = threadIdx.x;
  if (p < n_pol) meven[p] = meff[p] & ~1;
}

// eps2[w] = pref sum_p beta0_p^2 sum_i z_i0^2 L(w - |theta_i|) / (2 |theta_i|)
__global__ void k_full_eps2(const double *__restrict__ dd, const double *__restrict__ Z0, const int *__restrict__ mq,
                            int mmax, const double *__restrict__ beta0, int n_pol, const double *__restrict__ omega,
                            int n_w, double eta, double pref, double *__restrict__ eps2) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= n_w) return;
  const double om = omega[w];
  double tot = 0.0;
  for (int p = 0; p < n_pol; p++) {
    const int m = mq[p];
    const double *d = dd + (long long)p * mmax, *Z = Z0 + (long long)p * mmax;
    double acc = 0.0;
    for (int i = 0; i < m; i++) {
      const double th = fabs(d[i]), z = Z[i];
      if (th > 0.0) {
        const double x = om - th;
        acc += z * z * (eta / M_PI) / (x * x + eta * eta) / (2.0 * th);
      }
    }
    tot += beta0[p] * beta0[p] * acc;
  }
  eps2[w] = pref * tot;
}

// The n_eig smallest positive Ritz values (ascending) and residuals |b_{m-1} z_i,m-1|.
__global__ void k_full_lowest(const double *__restrict__ dd, const double *__restrict__ ZL, const int *__restrict__ mq,
                              int mmax, const double *__restrict__ b, int n_eig, double *__restrict__ omega,
                              double *__restrict__ resid) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int m = mq[0];
  double last = 0.0;
  int last_i = -1;
  for (int e = 0; e < n_eig; e++) {
    int best = -1;
    for (int i = 0; i < m; i++) {
      const double t = dd[i];
      if (!(t > 0.0)) continue;
      if (t < last || (t == last && i <= last_i)) continue;
      if (best < 0 || t < dd[best] || (t == dd[best] && i < best)) best = i;
    }
    if (best < 0) {
      omega[e] = NAN;
      if (resid) resid[e] = NAN;
      continue;
    }
    omega[e] = dd[best];
    if (resid) resid[e] = fabs(b[m - 1] * ZL[best]);
    last = dd[best];
    last_i = best;
  }
}

struct FullScratch {
  HalfMV *hm = nullptr;    // half-read products (complex64 A, B of even order), else null
  float2 *Z = nullptr;     // [4][n_pol][dim] product operands
  float2 *Q32 = nullptr, *P32 = nullptr, *rpart = nullptr;  // complex64 A, B: FP32 shadows of the bases
  double2 *W = nullptr;    // [4][n_pol][dim] products
  double2 *Q = nullptr, *P = nullptr, *R = nullptr, *S = nullptr, *coef = nullptr, *part = nullptr;
  double *a = nullptr, *b = nullptr, *beta0 = nullptr, *dd = nullptr, *z0 = nullptr, *zl = nullptr;
  int *meff = nullptr, *meven = nullptr;
  int nblk = 0;
};

void full_release(bse_ctx *c, FullScratch &s) {
  void *ptrs[] = {s.Q, s.P, s.R, s.S, s.coef, s.part, s.a, s.b, s.beta0, s.dd, s.z0, s.zl, s.meff, s.meven,
                  s.Z, s.W, s.Q32, s.P32, s.rpart};
  for (void *p : ptrs)
    if (p) cudaFreeAsync(p, c->stream);
  halfmv_release(c, s.hm);
  s.hm = nullptr;
}

bse_status full_alloc(bse_ctx *c, FullScratch &s, int n_pol, int n_steps) {
  const long long n2 = 2 * c->dim;
  const size_t qn = (size_t)n_pol * (n_steps + 1) * n2;
  s.nblk = (int)((n2 + VCH - 1) / VCH);
  cudaStream_t st = c->stream;
  if (cudaMallocAsync((void **)&s.Q, sizeof(double2) * qn, st) != cudaSuccess ||
      cudaMallocAsync((void **)&s.P, sizeof(double2) * qn, st) != cudaSuccess ||
      cudaMallocAsync((void **)&s.R, sizeof(double2) * n_pol * n2, st) != cudaSuccess ||
      cudaMallocAsync((void **)&s.S, sizeof(double2) * n_pol * n2, st) != cudaSuccess ||
      cudaMallocAsync((void **)&s.coef, sizeof(double2) * n_pol * (n_steps + 1), st) != cudaSuccess ||
      cudaMallocAsync((void **)&s.part, sizeof(double2) * n_pol * s.nblk, st) != cudaSuccess ||
      cudaMallocAsync((void **)&s.a, sizeof(double) * n_pol * (n_steps + 1), st) != cudaSuccess ||
      cudaMallocAsync((void **)&s.b, sizeof(double) * n_pol * (n_steps + 1), st) != cudaSuccess ||
      cudaMallocAsync((void **)&s.beta0, sizeof(double) * n_pol, st) != cudaSuccess ||
      cudaMallocAsync((void **)&s.dd, sizeof(double) * n_pol * n_steps, st) != cudaSuccess ||
      cudaMallocAsync((void **)&s.z0, sizeof(double) * n_pol * n_steps, st) != cudaSuccess ||
      cudaMallocAsync((void **)&s.zl, sizeof(double) * n_pol * n_steps, st) != cudaSuccess ||
      cudaMallocAsync((void **)&s.meff, sizeof(int) * n_pol, st) != cudaSuccess ||
      cudaMallocAsync((void **)&s.meven, sizeof(int) * n_pol, st) != cudaSuccess) {
    cudaGetLastError();
    return bse_fail(c, BSE_ENOMEM, "full BSE: Krylov scratch allocation failed");
  }
  bse_status r = halfmv_alloc(c, &s.hm);
  if (r != BSE_OK) return r;
  if (c->precision != BSE_FP64 &&
      (cudaMallocAsync((void **)&s.Q32, sizeof(float2) * qn, st) != cudaSuccess ||
       cudaMallocAsync((void **)&s.P32, sizeof(float2) * qn, st) != cudaSuccess ||
       cudaMallocAsync((void **)&s.rpart, sizeof(float2) * (size_t)n_pol * (n_steps + 1) * reorth32_chunks(n2), st) !=
           cudaSuccess)) {
    cudaGetLastError();
    return bse_fail(c, BSE_ENOMEM, "full BSE: reorthogonalisation scratch allocation failed");
  }
  if (s.hm && (cudaMallocAsync((void **)&s.Z, sizeof(float2) * 4 * n_pol * c->dim, st) != cudaSuccess ||
               cudaMallocAsync((void **)&s.W, sizeof(double2) * 4 * n_pol * c->dim, st) != cudaSuccess)) {
    cudaGetLastError();
    return bse_fail(c, BSE_ENOMEM, "full BSE: product scratch allocation failed");
  }
  return BSE_OK;
}

template <class T, int NP>
void launch_mmv(bse_ctx *c, const void *A, const void *B, const double2 *V, long long vs, double2 *S) {
  constexpr int RPW = sizeof(T) == 16 ? 2 : 4;
  const unsigned blocks = (unsigned)((c->dim + 8 * RPW - 1) / (8 * RPW));
  k_mmv<T, NP, RPW><<<blocks, 256, 0, c->stream>>>((const T *)A, (const T *)B, c->dim, V, vs, S, 2 * c->dim);
}

// S [n_pol][2 dim] = M V, V[p] at V + p vs.  Complex64 A, B of even order: two half-read
// products through the TDA's tiled TMA kernel, A on (x, conj(y)) (Hermitian) and B on
// (y, conj(x)) (symmetric), 2 n_pol vectors each, so the upper-triangle tiles of A and of B
// are each read once per step; otherwise one full-read pass (k_mmv).
bse_status mmv(bse_ctx *c, FullScratch &s, int n_pol, const void *A, const void *B, const double2 *V, long long vs,
               double2 *S) {
  if (s.hm) {
    const long long dim = c->dim, zs = (long long)n_pol * dim;
    const dim3 g((unsigned)((dim + 255) / 256), n_pol);
    k_fl_pack<<<g, 256, 0, c->stream>>>(V, vs, dim, n_pol, s.Z);
    bse_count_launch();
    bse_status r = halfmv_run(c, s.hm, A, false, s.Z, 2 * n_pol, s.W);
    if (r == BSE_OK) r = halfmv_run(c, s.hm, B, true, s.Z + 2 * zs, 2 * n_pol, s.W + 2 * zs);
    if (r != BSE_OK) return r;
    k_fl_combine<<<g, 256, 0, c->stream>>>(s.W, dim, n_pol, S, 2 * dim);
    bse_count_launch();
    return BSE_OK;
  }
  const bool c64 = c->precision != BSE_FP64;
  bse_prof_begin(c, BSE_KP_MATVEC);
  if (c64) {
    if (n_pol == 1) launch_mmv<float2, 1>(c, A, B, V, vs, S);
    else if (n_pol == 2) launch_mmv<float2, 2>(c, A, B, V, vs, S);
    else launch_mmv<float2, 3>(c, A, B, V, vs, S);
  } else {
    if (n_pol == 1) launch_mmv<double2, 1>(c, A, B, V, vs, S);
    else if (n_pol == 2) launch_mmv<double2, 2>(c, A, B, V, vs, S);
    else launch_mmv<double2, 3>(c, A, B, V, vs, S);
  }
  bse_prof_end(c, BSE_KP_MATVEC);
  bse_count_launch();
  return BSE_OK;
}

// The recursion; leaves a, b, beta0, meff in s and the even orders in s.meven.
bse_status full_lanczos(bse_ctx *c, FullScratch &s, const void *A, const void *B, const double2 *u, uint64_t seed,
                        int n_pol, int n_steps) {
  const long long dim = c->dim, n2 = 2 * dim;
  const long long qs = (long long)(n_steps + 1) * n2, vs = n2;
  const int ldab = n_steps + 1;
  cudaStream_t st = c->stream;
  const unsigned gv = (unsigned)std::min<long long>((n2 + VB - 1) / VB, 4 * c->n_sm);
  const unsigned ge = (unsigned)((n2 + VB - 1) / VB);
  cudaMemsetAsync(s.a, 0, sizeof(double) * n_pol * ldab, st);
  cudaMemsetAsync(s.b, 0, sizeof(double) * n_pol * ldab, st);
  {
    std::vector<int> m0(n_pol, n_steps);
    cudaMemcpyAsync(s.meff, m0.data(), sizeof(int) * n_pol, cudaMemcpyHostToDevice, st);
    cudaStreamSynchronize(st);
  }
  k_fl_start<<<dim3((unsigned)((dim + 255) / 256), n_pol), 256, 0, st>>>(u, dim, seed, s.R, vs);
  bse_status r = mmv(c, s, n_pol, A, B, s.R, vs, s.S);  // S = M v
  if (r != BSE_OK) return r;
  k_fl_dot_part<<<dim3(s.nblk, n_pol), VB, 0, st>>>(s.R, vs, s.S, vs, dim, 1.0, nullptr, 0, s.part, s.nblk);
  k_fl_norm0<<<dim3(gv, n_pol), VB, 0, st>>>(s.R, s.S, vs, dim, s.part, s.nblk, s.Q, s.P, qs, s.beta0, s.meff,
                                              c->d_err, s.Q32, s.P32);
  bse_count_launch(3);
  r = bse_check_launch(c, "full BSE start");
  if (r != BSE_OK) return r;
  for (int j = 0; j < n_steps; j++) {
    const double2 *pj = s.P + (long long)j * n2;
    k_fl_dot_part<<<dim3(s.nblk, n_pol), VB, 0, st>>>(pj, qs, pj, qs, dim, -1.0, s.meff, j, s.part, s.nblk);
    k_fl_axpy<<<dim3(gv, n_pol), VB, 0, st>>>(s.R, vs, dim, s.Q, s.P, qs, j, s.a, s.b, ldab, s.meff, s.part,
                                              s.nblk);
    bse_prof_begin(c, BSE_KP_REORTH);
    for (int pass = 0; pass < 2; pass++) {
      if (s.Q32) {  // FP32 projections: c_i = p_i^H r from the P shadow, r -= c_i q_i from the Q shadow
        r = launch_reorth32_pass(c, s.R, n2, s.P32, s.Q32, qs, j, s.rpart, ldab, s.coef, s.meff, n_pol);
        if (r != BSE_OK) return r;
      } else {
        k_fl_rdots<<<dim3(j + 1, n_pol), VB, 0, st>>>(s.R, vs, dim, s.P, qs, j, s.coef, ldab, s.meff);
        k_fl_rupdate<<<dim3(ge, n_pol), VB, 0, st>>>(s.R, vs, dim, s.Q, qs, j, s.coef, ldab, s.meff);
        bse_count_launch(2);
      }
    }
    bse_prof_end(c, BSE_KP_REORTH);
    r = mmv(c, s, n_pol, A, B, s.R, vs, s.S);  // S = M r
    if (r != BSE_OK) return r;
    k_fl_dot_part<<<dim3(s.nblk, n_pol), VB, 0, st>>>(s.R, vs, s.S, vs, dim, 1.0, s.meff, j, s.part, s.nblk);
    k_fl_scale<<<dim3(gv, n_pol), VB, 0, st>>>(s.R, s.S, vs, dim, s.Q, s.P, qs, j, n_steps, s.b, ldab, s.meff,
                                               s.part, s.nblk, c->d_err, s.Q32, s.P32);
    bse_count_launch(4);
    r = bse_check_launch(c, "full BSE step");
    if (r != BSE_OK) return r;
  }
  k_fl_even<<<1, 32, 0, st>>>(s.meff, n_pol, s.meven);
  bse_count_launch();
  r = bse_check_launch(c, "full BSE order");
  if (r != BSE_OK) return r;
  const size_t sm = sizeof(double) * 4 * n_steps;
  if (sm > 200 * 1024) return bse_fail(c, BSE_EINVAL, "full BSE: recursion longer than the tridiagonal solver holds");
  if (sm > 48 * 1024)
    cudaFuncSetAttribute(k_tridiag_ql_ends, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_tridiag_ql_ends<<<n_pol, 32, sm, st>>>(s.a, s.b, ldab, s.meven, n_steps, s.dd, s.z0, s.zl, c->d_err);
  bse_count_launch();
  return bse_check_launch(c, "full BSE tridiagonal");
}

}  // namespace

bse_status run_spectrum_full(bse_ctx *c, const void *A, const void *B, const double2 *u, int n_pol, int n_steps,
                             const double *omega, int n_w, double eta, double pref, double *eps2) {
  FullScratch s;
  bse_status r = full_alloc(c, s, n_pol, n_steps);
  if (r == BSE_OK) r = full_lanczos(c, s, A, B, u, 0, n_pol, n_steps);
  if (r == BSE_OK) {
    k_full_eps2<<<(n_w + 127) / 128, 128, 0, c->stream>>>(s.dd, s.z0, s.meven, n_steps, s.beta0, n_pol, omega, n_w,
                                                          eta, pref, eps2);
    bse_count_launch();
    r = bse_check_launch(c, "full BSE spectrum");
  }
  full_release(c, s);
  return r;
}

bse_status run_lowest_full(bse_ctx *c, const void *A, const void *B, int n_eig, int n_steps, uint64_t seed,
                           double *omega_out, double *resid_out) {
  FullScratch s;
  bse_status r = full_alloc(c, s, 1, n_steps);
  if (r == BSE_OK) r = full_lanczos(c, s, A, B, nullptr, seed, 1, n_steps);
  if (r == BSE_OK) {
    k_full_lowest<<<1, 32, 0, c->stream>>>(s.dd, s.zl, s.meven, n_steps, s.b, n_eig, omega_out, resid_out);
    bse_count_launch();
    r = bse_check_launch(c, "full BSE lowest");
  }
  full_release(c, s);
  return r;
}
