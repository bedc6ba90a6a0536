// Internal declarations of libbse (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <functional>
#include <string>
#include <vector>

#include "../../include/bse.h"

// Device error word bits (read and cleared by bse_sync).
enum : int {
  BSE_DERR_BOUNDS = 1,      // an index check failed
  BSE_DERR_TIMEOUT = 2,     // a bounded mbarrier / flag wait gave up
  BSE_DERR_ZERO_DENOM = 4,  // E_c - E_v == 0 in a dipole denominator
  BSE_DERR_TMEM = 8,        // tensor-memory allocation returned an unusable address
  BSE_DERR_INDEFINITE = 16  // full BSE: [[A, B], [B*, A*]] is not positive definite
};

struct bse_ctx {
  // problem (copied from bse_params)
  int n_atoms = 0;
  std::vector<int> nao, naux, ao_start, aux_start;
  int nao_tot = 0, naux_tot = 0, nao_max = 0;
  int mesh[3] = {1, 1, 1};
  double koff[3] = {0, 0, 0};
  int nk = 0;
  int n_RC = 0, n_RW = 0;
  std::vector<int> R_C, R_W;
  std::vector<double> w_RW;
  int nv = 0, nc = 0, nb = 0, nvc = 0;
  double alpha = 2.0;
  int precision = BSE_FP64;
  bool h64 = true;         // H is stored complex128 (BSE_FP64, or a split precision with h_complex128)
  // exciton momentum Q (mesh steps): qQ is the flattened index of Q, qmQ of -Q, so the
  // conduction point of the pairs at k is kdiff(k, qmQ) and k - Q is kdiff(k, qQ)
  int Qm[3] = {0, 0, 0};
  int qQ = 0, qmQ = 0;
  bool vx_from_R = false;  // V0c holds sum_R w_R Vbar(R) e^{+iQ.R} (bse_set_momentum)
  int64_t dim = 0;
  cudaStream_t stream = nullptr;
  int device = 0;
  int n_sm = 148;
  int stage = 0;  // 0 setup, 1 interp_W done, 2 project_pairs done
  std::string err;

  // small device tables
  int *d_R_C = nullptr, *d_R_W = nullptr;
  double *d_w_RW = nullptr;
  int *d_aux_atom = nullptr;   // atom of each ABF
  int *d_ao_start = nullptr;   // first NAO of each atom
  int *d_nao = nullptr;        // NAOs of each atom
  int *d_aux_start = nullptr;  // first ABF of each atom
  int *d_naux = nullptr;       // ABFs of each atom
  int *d_err = nullptr;        // device error word

  // workspace
  double2 *Wq = nullptr;   // [nk][naux][naux]   W(q), row mu, column nu (FP64 path)
  double2 *V0c = nullptr;  // [naux][naux]       V(0) as complex
  double2 *Y = nullptr;    // [nk][nao_max][nb][naux]  Y^mu_{s n}(k), s local to atom(mu)
  double2 *ck = nullptr;   // [nk][nao][nb]      band coefficients
  double *eqp = nullptr;   // [nk][nb]
  double2 *X = nullptr;    // [nk][nv][nc][naux] C~^mu_{a k, i k}
  double2 *P = nullptr;    // [dim][naux]        X V0
  int slab = 1;            // q values per assembly slab
  // Half set of transfers: q and -q give conjugate-transposed blocks, so only one of each
  // pair is computed (self-conjugate q, every component 0 or N/2, are computed whole).
  std::vector<int> qplus;
  int *d_qplus = nullptr;
  int *d_qall = nullptr;   // 0 .. N_k-1 (every transfer, for the adjoint)
  double2 *Aq = nullptr;   // [nk][naux][naux] dL/dW(q) (adjoint workspace, allocated on first use)
  double2 *Mv = nullptr, *Mc = nullptr, *T = nullptr;  // [slab][nk][nv*nv | nc*nc][naux]
  // coupling block (full BSE, FP64 path; allocated on first use): [slab_cv][nk][nc*nv][naux]
  double2 *Bm1 = nullptr, *Bt1 = nullptr, *Bm2 = nullptr;
  int slab_cv = 0;

  // split-precision workspace (tensor-core path)
  void *tc = nullptr;

  // per-kernel event timing (bse_profile)
  bool prof = false;
  struct Pending { int id; cudaEvent_t a, b; };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;
  double prof_ms[BSE_KP_COUNT] = {0};
  long long prof_n[BSE_KP_COUNT] = {0};
};

// Bracket one launch with events when profiling is enabled.
void bse_prof_begin(bse_ctx *c, int id);
void bse_prof_end(bse_ctx *c, int id);

// ---- helpers shared by the .cu files --------------------------------------------------
void bse_count_launch(int n = 1);
// Per-device one-time set-up (kernel attributes such as the dynamic shared-memory limit are
// per device): the first call for (the context's device, key) in this process runs `fn`
// with that device current; every call returns only after it has run (thread-safe).
enum { BSE_ONCE_HMV_TDA = 0, BSE_ONCE_HMV_ALL = 1, BSE_ONCE_SPLIT = 2, BSE_ONCE_GROUPED = 3, BSE_ONCE_KEYS = 4 };
void bse_once_per_device(const bse_ctx *c, int key, void (*fn)());
bse_status bse_fail(bse_ctx *c, bse_status s, const std::string &msg);
bse_status bse_check_launch(bse_ctx *c, const char *what);

// fp64 path launchers (k_fp64.cu)
bse_status launch_interp_W_fp64(bse_ctx *c, const double *W_R, double2 *out, int q_first = 0, int n_q = -1);
bse_status launch_half_transform_fp64(bse_ctx *c, const double *C_R);
bse_status launch_exchange_factors_fp64(bse_ctx *c);
bse_status launch_zgemm_fp64(bse_ctx *c, int M, int N, int K, const double2 *A, int lda,
                             long long sA, const double2 *B, int ldb, long long sB, double2 *C,
                             int ldc, long long sC, int batch, int prof_id = -1,
                             const int *bidx = nullptr);
bse_status launch_project_slab_fp64(bse_ctx *c, int q0, int nq, const int *qlist);
bse_status launch_g2_write_fp64(bse_ctx *c, int q0, int nq, double2 *H);
bse_status launch_project_cv_slab_fp64(bse_ctx *c, int q0, int nq, const int *qlist, double2 *M1, double2 *M2);
bse_status launch_g2_coupling_fp64(bse_ctx *c, int q0, int nq, const double2 *T1, const double2 *M2, double2 *B);

// spectrum (k_haydock.cu)
bse_status run_dipole_vector(bse_ctx *c, const double *vel, const double *e_ks, double2 *u);
bse_status run_spectrum(bse_ctx *c, const void *H, const double2 *u, int n_pol, int n_steps,
                        const double *omega, int n_w, double eta, double pref, double *eps2, double *ab,
                        bool accumulate = false);
bse_status run_lowest(bse_ctx *c, const void *H, int n_eig, int n_steps, uint64_t seed,
                      double *omega_out, double *resid_out, double2 *vecs_out);
// adjoint (k_adjoint.cu)
bse_status run_adjoint(bse_ctx *c, const double2 *Gamma, double *dW_R, double *de_qp);
bse_status run_seed_lowrank(bse_ctx *c, const double2 *X, const double *g, int r, double2 *Gamma);
bse_status launch_zgemm_tn(bse_ctx *c, int M, int N, int K, const double2 *A, const double2 *B, double2 *C,
                           double alpha);
bse_status run_window_seed(bse_ctx *c, const void *H, const double2 *u, int n_pol, int n_steps, double w_lo,
                           double w_hi, double eta, double pref, double *I_out, double2 *Gamma);
// Half-read products W = Hm Z (np <= 3 vectors) of a complex64 Hermitian or complex symmetric
// matrix through the TDA's tiled TMA kernel (k_haydock.cu).  halfmv_alloc leaves *out null
// when the path does not apply (FP64 context or odd dim).
struct HalfMV;
bse_status halfmv_alloc(bse_ctx *c, HalfMV **out);
void halfmv_release(bse_ctx *c, HalfMV *h);
bse_status halfmv_run(bse_ctx *c, HalfMV *h, const void *Hm, bool sym, const float2 *Z, int np, double2 *W);
// FP32-projection reorthogonalisation pass (k_haydock.cu): coef_i = D32_i^H W,
// W -= sum_{i<=j} coef_i U32_i; rpart holds [n_pol][ldp][reorth32_chunks(n)] partials.
int reorth32_chunks(long long n);
bse_status launch_reorth32_pass(bse_ctx *c, double2 *W, long long n, const float2 *D32, const float2 *U32,
                                long long qs, int j, float2 *rpart, int ldp, double2 *coef, const int *meff,
                                int n_pol);
// full BSE (k_fullbse.cu); the tridiagonal solver keeps 4 x n_steps doubles in shared memory
constexpr int BSE_FULL_MAX_STEPS = 6400;
// full BSE (k_fullbse.cu)
bse_status run_spectrum_full(bse_ctx *c, const void *A, const void *B, const double2 *u, int n_pol, int n_steps,
                             const double *omega, int n_w, double eta, double pref, double *eps2);
bse_status run_lowest_full(bse_ctx *c, const void *A, const void *B, int n_eig, int n_steps, uint64_t seed,
                           double *omega_out, double *resid_out);
bse_status run_spectrum_static(bse_ctx *c, const void *H, const double2 *u, int n_pol, int n_steps,
                               const double *omega, int n_w, double eta, double pref, double *eps2,
                               double *ab);

// split-precision path (k_split.cu)
bse_status split_setup(bse_ctx *c);
bse_status split_interp_W(bse_ctx *c, const double *W_R, double2 *Wq_out);
bse_status split_assemble(bse_ctx *c, void *H);
// dL/dW(q) of every transfer into c->Aq from the split contexts' FP32 pair table (the
// adjoint's slab loop; the Fourier adjoint and the diagonal follow in k_adjoint.cu).
bse_status split_adjoint_slabs(bse_ctx *c, const double2 *Gamma);
// Batched assembly of the n split-precision systems ctxs[order[0..n-1]] (smallest first) as a
// work list of grouped launches on their (common) stream; stamp(i) runs when system i's last
// launch is enqueued.
bse_status split_batch_worklist(bse_ctx **ctxs, void **H, const int *order, int n,
                                const std::function<void(int)> &stamp);
bse_status split_assemble_coupling(bse_ctx *c, void *B);
// W[p] = H x[p] (x[p] at x + p xs, W [n_pol][dim]) without H (split precisions), and the
// early-stop scale of the matrix-free recursion
bse_status split_matvec_free(bse_ctx *c, const double2 *x, long long xs, int n_pol, double2 *W);
bse_status split_matfree_hmax(bse_ctx *c, double *hmax);
bse_status run_spectrum_matfree(bse_ctx *c, const double2 *u, int n_pol, int n_steps, const double *omega, int n_w,
                                double eta, double pref, double *eps2, double *ab);
bse_status split_project(bse_ctx *c, const double *C_R);
bse_status split_autotune(bse_ctx *c, int *chosen, int *chosen_proj);
void split_free(bse_ctx *c);

// mesh helpers
__host__ __device__ inline bool q_self_conjugate(int q, int n1, int n2, int n3) {
  int a1 = q / (n2 * n3), a2 = (q / n3) % n2, a3 = q % n3;
  return (n1 - a1) % n1 == a1 && (n2 - a2) % n2 == a2 && (n3 - a3) % n3 == a3;
}
__host__ __device__ inline int kdiff(int k1, int q, int n1, int n2, int n3) {
  // index of k2 = k1 - q on the mesh (integer parts; offsets cancel in differences)
  int a1 = k1 / (n2 * n3), a2 = (k1 / n3) % n2, a3 = k1 % n3;
  int b1 = q / (n2 * n3), b2 = (q / n3) % n2, b3 = q % n3;
  int c1 = a1 - b1; if (c1 < 0) c1 += n1;
  int c2 = a2 - b2; if (c2 < 0) c2 += n2;
  int c3 = a3 - b3; if (c3 < 0) c3 += n3;
  return (c1 * n2 + c2) * n3 + c3;
}

#ifdef __CUDACC__
// e^{-2 pi i q.R} with q = m/N (integers): exact argument reduction mod N_k.
__device__ __forceinline__ double2 phase_qR(int q, const int *R, int n1, int n2, int n3) {
  int m1 = q / (n2 * n3), m2 = (q / n3) % n2, m3 = q % n3;
  long long nk = (long long)n1 * n2 * n3;
  long long p = (long long)m1 * R[0] * n2 * n3 + (long long)m2 * R[1] * n1 * n3 +
                (long long)m3 * R[2] * n1 * n2;
  p %= nk;
  if (p < 0) p += nk;
  double s, c;
  sincospi(2.0 * (double)p / (double)nk, &s, &c);
  return make_double2(c, -s);
}

// e^{+2 pi i k.R} for k = (n + off)/N.
__device__ __forceinline__ double2 phase_kR(int k, const int *R, int n1, int n2, int n3,
                                            double o1, double o2, double o3) {
  int a1 = k / (n2 * n3), a2 = (k / n3) % n2, a3 = k % n3;
  long long i1 = ((long long)a1 * R[0]) % n1, i2 = ((long long)a2 * R[1]) % n2,
            i3 = ((long long)a3 * R[2]) % n3;
  double f = (double)i1 / n1 + (double)i2 / n2 + (double)i3 / n3 +
             (o1 * R[0]) / n1 + (o2 * R[1]) / n2 + (o3 * R[2]) / n3;
  f = f - floor(f);
  double s, c;
  sincospi(2.0 * f, &s, &c);
  return make_double2(c, s);
}
#endif
