/*
 * bse.h -- C ABI of the B300 (sm_103a) Tamm-Dancoff BSE hot path and its extensions
 * (full BSE, finite exciton momentum, matrix-free spectrum).
 *
 * The library builds the resonant block A of the BSE Hamiltonian on a dense k-mesh from
 * the unit-cell-indexed screened interaction W_mu,nu(R) and the localized-RI pair
 * coefficients C^mu_st(R), then computes the velocity-form absorption spectrum by a
 * Haydock (Lanczos) recursion.  The steps and where the paper defines them
 * (arXiv 2607.05853):
 *   bse_interp_W       W_mu,nu(q) = sum_R w_R W_mu,nu(R) exp(-i q.R), q = k1 - k2: the
 *                      R-sum of Eq. W_LRI (§III.A) on the dense mesh (§III.B).
 *   bse_project_pairs  C^mu_st(k) = sum_R C^mu_st(R) exp(i k.R) and the Kohn-Sham-basis
 *                      coefficients C~^mu_{j k2, i k1} (§III.A); the pair projections
 *                      themselves are formed inside bse_assemble, one q-slab at a time.
 *   bse_assemble       A_{ai k1, bj k2} = (E_a - E_i) delta + alpha (ak1*,ik1|V|jk2*,bk2)
 *                      - (jk2*,ik1|W|ak1*,bk2) (Eq. Hamiltonian, §II.C) with both kernels
 *                      in the LRI form of Eq. W_LRI (1/N_k, V at q = 0).
 *   bse_dipole_vector  u_alpha,(k,i,a) = conj(<ik|v_alpha|ak> / (E_ak - E_ik)) (Eq. abs_vel).
 *   bse_spectrum       eps2(w) = pref sum_alpha -(1/pi) Im <u|(w + i eta - A)^-1|u> -- Eq.
 *                      abs_vel with the delta broadened to a Lorentzian -- by a Lanczos
 *                      recursion with full reorthogonalisation and a continued fraction.
 *   bse_lowest         lowest Ritz values of A by Lanczos (the TDA eigenvalues, §II.C).
 *   bse_set_momentum   finite exciton momentum Q: pairs (v k, c k+Q) (the q != 0 extension, §V).
 *   bse_assemble_coupling, bse_spectrum_full, bse_lowest_full
 *                      full BSE: the coupling block B, eps2 with the Y amplitudes, the lowest
 *                      paired +-Omega (§II.C, Eq. full_BSE_epsilon2).
 *   bse_spectrum_matfree  the Haydock spectrum with H recomputed per Lanczos product.
 *
 * Conventions (all entry points):
 *  - Dense k-points are k = (n + k_offset)/N per axis, flattened (n1*N2 + n2)*N3 + n3.
 *    R vectors are integer lattice coordinates.  Phases are exp(2 pi i k.R).
 *  - NAOs s are numbered atom by atom (nao_per_atom), ABFs mu atom by atom (naux_per_atom).
 *  - Band window: columns 0..nv-1 are valence bands, column 0 the valence band maximum
 *    counting down; columns nv..nv+nc-1 conduction bands, nv the minimum counting up.
 *  - The row (and column) of the pair (k, v, c) in H is (k*nv + v)*nc + c;
 *    dim = N_k * nv * nc.  H is row-major and fully stored (both triangles).
 *  - complex128 arrays are interleaved (re, im) doubles; complex64 interleaved floats.
 *  - Every array argument is a DEVICE pointer on the context's device unless marked
 *    "host".  The caller owns every argument buffer; the context owns only its workspace
 *    and copies the host arrays of bse_params at setup.
 *  - Work is enqueued on the stream given to bse_setup and the call returns without
 *    waiting, except where stated.  Argument errors are reported before anything is
 *    enqueued.  A CUDA launch error returns BSE_ECUDA; bse_last_error() explains.
 *  - Calls must come in order: setup, interp_W, project_pairs, then assemble; spectrum,
 *    lowest and dipole_vector need only setup.  Out-of-order calls return BSE_ESTATE.
 *  - No kernel traps or asserts; kernels that wait on a barrier give up after a bounded
 *    number of polls, set a device error word, and bse_sync() then returns BSE_ETIMEOUT
 *    (or BSE_EDEVICE for a failed device-side check).
 */
#ifndef BSE_H
#define BSE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bse_ctx bse_ctx;

typedef enum {
  BSE_OK = 0,
  BSE_EINVAL = 1,    /* bad argument */
  BSE_ENOMEM = 2,    /* device allocation failed */
  BSE_ECUDA = 3,     /* a CUDA runtime call or launch failed */
  BSE_ETIMEOUT = 4,  /* a device-side bounded wait gave up */
  BSE_ESTATE = 5,    /* call out of order */
  BSE_EDEVICE = 6    /* a device-side check set the error word */
} bse_status;

/* Arithmetic of the kernel contractions in bse_assemble.
 *  BSE_FP64  : everything in FP64 on CUDA cores; H is complex128.
 *  BSE_BF16X3: contractions on tcgen05 tensor cores with each FP32 operand split into
 *              three bf16 pieces (6 piece products kept), FP32 accumulation; phases
 *              and the E_c - E_v diagonal in FP64; H is complex64, or complex128 with
 *              bse_params.h_complex128 (then the spectrum, lowest-exciton and window entries
 *              read it with the FP64 path's full-read products).
 *  BSE_BF16X2: as BF16X3 with two pieces (3 piece products).
 *  BSE_BF16X1: one bf16 piece (1 product) -- an accuracy ablation.
 *  BSE_TF32X2: as BF16X3 with two tf32 pieces per FP32 operand, x ~ tf32(x) + tf32(x - tf32(x))
 *              (about 22 significant bits), the 3 products of order <= 1 on tcgen05 kind::tf32
 *              MMAs (half the bf16 rate); H as for the bf16 splits. */
typedef enum { BSE_FP64 = 0, BSE_BF16X3 = 1, BSE_BF16X2 = 2, BSE_BF16X1 = 3, BSE_TF32X2 = 4 } bse_precision;

typedef struct {
  int32_t n_atoms;
  const int32_t *nao_per_atom;   /* host [n_atoms], NAOs per atom (Eq. 2 basis)       */
  const int32_t *naux_per_atom;  /* host [n_atoms], ABFs per atom (§III.A)            */
  int32_t dense[3];              /* dense k-mesh N1,N2,N3 (>= 1)                       */
  double k_offset[3];            /* mesh shift in units of the mesh spacing            */
  int32_t n_RC;                  /* R-set of C(R) (§III.A, truncated beyond 2 rcut)    */
  const int32_t *R_C;            /* host [n_RC][3]                                     */
  int32_t n_RW;                  /* Wigner-Seitz images of the coarse cell (§III.B)    */
  const int32_t *R_W;            /* host [n_RW][3]                                     */
  const double *w_RW;            /* host [n_RW] image weights (1/degeneracy)           */
  int32_t nv, nc;                /* band window, nv + nc <= total NAOs                 */
  double alpha;                  /* 2 singlet, 0 triplet (Eq. Hamiltonian)             */
  int32_t precision;             /* a bse_precision                                   */
  int32_t h_complex128;          /* split precisions: 1 stores H as complex128 (the    */
                                 /* E_c - E_v diagonal then exact in FP64), 0 complex64 */
  /* Optional consistency data of W's R-set (§III.B: W(R) is the Fourier transform of W on
   * the coarse mesh, folded into the Wigner-Seitz cell).  The arithmetic needs neither: phases
   * use integer R, and the coarse mesh enters only through R_W and w_RW.  When given they are
   * checked at setup (BSE_EINVAL on a mismatch):
   *  coarse  : the coarse (GW) mesh, or {0,0,0}: the weights w_RW of the images of each coarse
   *            Born-von Karman class (R mod coarse, per axis) sum to 1 (within 1e-9), every
   *            class included, and no image's weight is <= 0;
   *  lattice : host [3][3] float64 lattice vectors a_i as rows (any length unit), or NULL;
   *            with coarse, every image is a shortest member of its class under this metric
   *            (|sum_i R_i a_i| <= |sum_i (R_i + m_i coarse_i) a_i| (1 + 1e-9) + 1e-9 for all
   *            m in {-1,0,1}^3).
   * Atom positions and the occupied-band count do not enter the method's arithmetic (C(R) and
   * the band window's coefficients are inputs), so bse_params does not take them. */
  int32_t coarse[3];
  const double *lattice;
} bse_params;

/* The host-side checks of bse_setup alone (argument ranges, sizes and the optional coarse /
 * lattice consistency above); touches no device.  BSE_OK or BSE_EINVAL. */
bse_status bse_check_params(const bse_params *p);

/* Validate p (bse_check_params), copy its host arrays, allocate the workspace on the current
 * CUDA device and bind the context to `cuda_stream` (a cudaStream_t, NULL = default stream).
 * On success *out receives the context; on failure *out is NULL.  Synchronous. */
bse_status bse_setup(const bse_params *p, void *cuda_stream, bse_ctx **out);

/* Step (a): W(q) for every transfer q = k1 - k2 of the dense mesh (there are N_k).
 *  W_R : [n_RW][N_aux][N_aux] float64, real, the images listed in bse_params.R_W.
 *  V0  : [N_aux][N_aux] float64, V_mu,nu(q=0) = sum_R Vbar_mu,nu(R), real symmetric.
 *  Wq_out : optional [N_k][N_aux][N_aux] complex128 (row mu, column nu), or NULL.
 * Both inputs are read during this call's work only (the context keeps its own copy). */
bse_status bse_interp_W(bse_ctx *ctx, const double *W_R, const double *V0, void *Wq_out);

/* Optional output of step (a): the bare interaction at every dense transfer q,
 * V(q) = sum_R w_R Vbar(R) exp(-i q.R), with the R-set and weights of W (bse_params R_W,
 * w_RW); FP64 for every precision.  V(0) is what the exchange term uses (bse_interp_W's V0);
 * V(q != 0) is not needed by the Q = 0 Hamiltonian (§III.A).
 *  V_R    : [n_RW][N_aux][N_aux] float64, real.
 *  Vq_out : [N_k][N_aux][N_aux] complex128 (row mu, column nu). */
bse_status bse_interp_V(bse_ctx *ctx, const double *V_R, void *Vq_out);

/* Exciton momentum Q (the finite-momentum extension, §V: q != 0 blocks of the same
 * Hamiltonian).  The pair (k, v, c) then holds the valence band v at k and the conduction
 * band c at k + Q; the C~ coefficients (§III.A) are taken at those points, the direct kernel
 * keeps W at q = k1 - k2, the diagonal is E_c(k+Q) - E_v(k), and the exchange kernel of
 * Eq. W_LRI uses sum_R w_R Vbar(R) exp(+i Q.R) (= V(-Q) in bse_interp_V's convention; its
 * value at Q = 0 is V(0)) in place of V(0).
 *  Q   : host [3] int32, Q = Q_i / N_i per axis in dense-mesh steps (reduced mod N_i).
 *  V_R : [n_RW][N_aux][N_aux] float64 real Vbar(R) on the images of bse_params.R_W, or NULL.
 *        Required when Q != 0 and alpha != 0.  When given it replaces bse_interp_W's V0
 *        (which may then be NULL) until a later call with V_R = NULL.
 * Call after bse_setup and before bse_project_pairs; a call after bse_project_pairs
 * requires bse_project_pairs again (BSE_ESTATE from bse_assemble otherwise), and one with
 * V_R = NULL after one with V_R requires bse_interp_W again.  Every precision: the split
 * precisions take the complex V in FP32 into their X V pieces.  At Q != 0
 * bse_dipole_vector returns BSE_EINVAL: the optical
 * dipoles are vertical transitions; bse_spectrum and bse_lowest take H(Q) as any H. */
bse_status bse_set_momentum(bse_ctx *ctx, const int32_t *Q, const double *V_R);

/* Step (b), per-k part: C(k) and the half-transforms Y^mu_sn(k) = sum_t C^mu_st(k) c^k_tn
 * for s on the atom of mu (C real => the second LRI term is conj(Y), §III.A), the
 * exchange factors C~^mu_{a k, i k}, and a copy of the band energies.
 *  C_R  : [n_RC][N_ao][N_ao][N_aux] float64, C^mu_st(R); entries whose mu is not on the
 *         atom of s are ignored (the expansion has no such terms).
 *  c_k  : [N_k][N_ao][nv+nc] complex128 band coefficients (window columns).
 *  e_qp : [N_k][nv+nc] float64 quasiparticle energies (eV) for the diagonal. */
bse_status bse_project_pairs(bse_ctx *ctx, const double *C_R, const double *c_k,
                             const double *e_qp);

/* Steps (b)+(c): build H.  H : [dim][dim], complex128 for BSE_FP64 and for the split
 * precisions with bse_params.h_complex128, complex64 otherwise.  Every element is written. */
bse_status bse_assemble(bse_ctx *ctx, void *H);

/* Full BSE (§II.C): the coupling block
 *   B_{ai k1, bj k2} = alpha (a k1*, i k1|V|b k2*, j k2) - (b k2*, i k1|W|a k1*, j k2),
 * both kernels in the LRI form of Eq. W_LRI: (1/N_k) C~_{a k1, i k1} V(0) C~_{b k2, j k2} and
 * (1/N_k) C~_{b k2, i k1} W(k1 - k2) C~_{a k1, j k2}.  B is complex symmetric (B = B^T).
 *  B : [dim][dim], rows and columns ordered as H's; complex128 for BSE_FP64, complex64 for
 *      the split precisions (tensor-core contractions as in bse_assemble).  Every element is
 *      written.  Call after bse_project_pairs.  BSE_EINVAL at Q != 0 and for a split context
 *      with h_complex128 (the full-BSE entries take complex64 A and B).  Workspace for the
 *      conduction-valence projections is allocated on the first call. */
bse_status bse_assemble_coupling(bse_ctx *ctx, void *B);

/* Step (d) without H in memory: the same Haydock spectrum as bse_spectrum, with every Lanczos
 * product H x recomputed from the context's pair tables -- the exchange and diagonal as
 * small dense products, the direct term q-slab by q-slab (pair projections, M_vv W(q) on
 * tensor cores, each nvc x nvc block applied as soon as it is formed).  Memory stays at the
 * slab workspace instead of dim^2 elements; each step costs about one assembly.  For
 * Hamiltonians beyond HBM (dense meshes of §IV).  Split precisions only (BSE_EINVAL for
 * BSE_FP64); call after bse_project_pairs; arguments as bse_spectrum without H. */
bse_status bse_spectrum_matfree(bse_ctx *ctx, const double *u, int n_pol, int n_steps, const double *omega,
                                int n_w, double eta, double prefactor, double *eps2, double *ab);

/* Full-BSE spectrum (Eq. full_BSE_epsilon2, §II.C): for H = [[A, B], [-B*, -A*]] with
 * positive solutions Omega_S, amplitudes (X_S, Y_S) normalised X^dagger X - Y^dagger Y = 1,
 *   eps2(w) = prefactor sum_p sum_S |sum_r d_p,r X_rS - conj(d_p,r) Y_rS|^2 L_eta(w - Omega_S),
 * d_p = conj(u[p]) (u from bse_dipole_vector), L_eta the Lorentzian of half width eta.
 * Computed by a Lanczos recursion in the inner product of M = [[A, B], [B*, A*]] from the
 * start vector (u, conj u) and a Gauss quadrature of its tridiagonal (exact when n_steps
 * reaches an invariant subspace, e.g. n_steps = 2 dim); an odd recursion length is cut to
 * the even one below it.
 *  A, B : [dim][dim] from bse_assemble and bse_assemble_coupling (complex128 for BSE_FP64,
 *         complex64 otherwise), read only.
 *  u    : [n_pol][dim] complex128; n_pol 1..3; 2 <= n_steps <= min(2 dim, 6400); omega [n_w];
 *         eps2 [n_w].
 * M must be positive definite (a stable excited state): otherwise the recursion stops and
 * bse_sync returns BSE_EDEVICE.  Krylov workspace (2 x n_pol x (n_steps+1) x 2 dim complex128)
 * is allocated and freed on the stream per call. */
bse_status bse_spectrum_full(bse_ctx *ctx, const void *A, const void *B, const double *u, int n_pol,
                             int n_steps, const double *omega, int n_w, double eta, double prefactor,
                             double *eps2);

/* The n_eig lowest positive full-BSE excitation energies Omega_S (the paired eigenproblem of
 * §II.C) by the same recursion from a seeded random start, with Lanczos residual bounds.
 *  omega_out, resid_out : [n_eig] float64 (resid_out may be NULL);
 *  2 n_eig <= n_steps <= min(2 dim, 6400).
 * Unconverged or missing values are NaN. */
bse_status bse_lowest_full(bse_ctx *ctx, const void *A, const void *B, int n_eig, int n_steps,
                           uint64_t seed, double *omega_out, double *resid_out);

/* u_alpha,(k,i,a) = conj(vel[alpha][k][i][a] / (e_ks[k][nv+a] - e_ks[k][i])).
 *  vel : [3][N_k][nv][nc] complex128 <ik|v_alpha|ak>;  e_ks : [N_k][nv+nc] float64;
 *  u   : [3][dim] complex128 output.  A zero denominator gives BSE_EDEVICE at bse_sync. */
bse_status bse_dipole_vector(bse_ctx *ctx, const double *vel, const double *e_ks, double *u);

/* Step (d): Haydock spectrum.  For each of n_pol (1..3) start vectors u[p] (complex128
 * [n_pol][dim]) run n_steps (1..dim) Lanczos steps on H (type as in bse_assemble) in
 * FP64 with full reorthogonalisation (a second pass where the DGKS test asks for it),
 * stopping early when b_j < 1e-14 max|H|,
 * then eps2[w] = prefactor * sum_p -(1/pi) Im g_p(omega[w] + i eta), with
 * g = |u|^2/(z - a1 - b1^2/(z - a2 - ...)).  eps2 : [n_w] float64.  ab : optional
 * [n_pol][3][n_steps] float64 receiving a_j, b_j and (in [p][2][0]) |u|, or NULL.
 * Scratch: a Krylov basis of n_pol*(n_steps+1)*dim complex128, allocated per call. */
bse_status bse_spectrum(bse_ctx *ctx, const void *H, const double *u, int n_pol,
                        int n_steps, const double *omega, int n_w, double eta,
                        double prefactor, double *eps2, double *ab);

/* Weighted accumulation of spectra: eps2_acc[w] += weight * (the eps2 bse_spectrum would
 * write), with the same Lanczos recursion and arguments.  With one context per shifted
 * dense mesh this gives the k-offset average of §IV (k-point convergence): four offsets
 * (0,0,0), (1/3,0,0), (1/3,1/3,0), (2/3,1/3,0) of the mesh spacing, the symmetry-reduced
 * classes of a 3x3x3 offset grid, with weights 1/27, 8/27, 6/27, 12/27.
 *  eps2_acc : [n_w] float64, read and written (zero it before the first call). */
bse_status bse_spectrum_add(bse_ctx *ctx, const void *H, const double *u, int n_pol, int n_steps,
                            const double *omega, int n_w, double eta, double prefactor, double weight,
                            double *eps2_acc);

/* Allocation-free variant of bse_spectrum, for callers that cannot allocate device memory:
 * for example a host application that hands the library a slice of a device pool it owns
 * and forbids driver allocations inside its callbacks, or code already holding the GPU at
 * its memory limit, where the per-call Krylov allocation of bse_spectrum would fail.  The
 * paper has no counterpart; it is a deployment variant of step (d).
 * Arguments, results and errors are those of bse_spectrum.  The Krylov basis and every other
 * scratch buffer live in one file-scope device array of 64 MiB (67108864 bytes) that each
 * GPU loading the library keeps until the process exits; requests that need more (roughly
 * n_pol * (n_steps + 1) * dim * 24 bytes plus the matvec partials) return BSE_EINVAL with the
 * size in bse_last_error, before anything is enqueued.  The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress, with that device current); make that
 * first call before any stream capture.  No call allocates or frees memory, and none waits
 * for the device: the work is enqueued on the context's stream as bse_spectrum's is.  All calls
 * share the one array and it keeps the last call's contents (every value the recursion
 * reads is written by the same call first); calls that overlap on the GPU -- two streams or
 * two contexts on one device at once -- race on it, so serialise them. */
bse_status bse_spectrum_static(bse_ctx *ctx, const void *H, const double *u, int n_pol,
                               int n_steps, const double *omega, int n_w, double eta,
                               double prefactor, double *eps2, double *ab);

/* Lowest Ritz values of H after n_steps (<= dim) Lanczos steps with full
 * reorthogonalisation from a fixed pseudo-random start vector (seed `seed`); the TDA
 * eigenvalues Omega_S of §II.C for the converged pairs.
 *  omega_out : [n_eig] float64 ascending;  resid_out : optional [n_eig] float64
 *  receiving |b_m * s_m,i| (the Lanczos residual norm of each Ritz pair), or NULL;
 *  vecs_out : optional [n_eig][dim] complex128 receiving the unit Ritz vectors, or NULL. */
bse_status bse_lowest(bse_ctx *ctx, const void *H, int n_eig, int n_steps, uint64_t seed,
                      double *omega_out, double *resid_out, double *vecs_out);

/* Adjoint seed Gamma = sum_s g[s] x_s x_s^dagger (Hermitian, [dim][dim] complex128), so that
 * for L = sum_s g_s Omega_s the Hellmann-Feynman theorem gives dL = tr(Gamma dH).
 *  vecs : [r][dim] complex128 (e.g. Ritz vectors from bse_lowest);  g : [r] float64. */
bse_status bse_adjoint_seed(bse_ctx *ctx, const double *vecs, const double *g, int r, double *Gamma);

/* Adjoint seed of the windowed absorption integral (the spectrum of Eq. abs_vel, §II.C,
 * integrated over a frequency window; differentiated through Eq. Hamiltonian): with the Lorentzian of
 * Eq. abs_vel (half width eta) integrated over [w_lo, w_hi],
 *   I = prefactor * sum_p u_p^dagger f(H) u_p,
 *   f(x) = (1/pi) [atan((w_hi - x)/eta) - atan((w_lo - x)/eta)],
 * i.e. the integral of the bse_spectrum output over the window.  n_steps Lanczos steps per
 * start vector (FP64, full reorthogonalisation, as bse_spectrum) give the tridiagonal T_p;
 * its eigenpairs (implicit QL) give Ritz vectors y_i and weights v_i (first components), and
 *   Gamma = sum_p prefactor |u_p|^2 sum_{i,l} F_il v_i v_l y_i y_l^dagger,
 *   F_il = (f(theta_i) - f(theta_l)) / (theta_i - theta_l), F_ii = f'(theta_i)
 * (Daleckii-Krein in the Krylov subspace; exact when n_steps = dim), so that
 * dI = tr(Gamma dH) and bse_adjoint(Gamma) returns dI/dW(R) and dI/dE^QP.
 *  H : as bse_spectrum;  u : [n_pol][dim] complex128 (n_pol 1..3), e.g. from bse_dipole_vector;
 *  I_out : optional device float64 receiving I from the same Krylov data, or NULL;
 *  Gamma : [dim][dim] complex128 output, Hermitian, overwritten.
 * Scratch per call: the Krylov basis and 2 n_pol n_steps (n_steps + dim) doubles. */
bse_status bse_window_seed(bse_ctx *ctx, const void *H, const double *u, int n_pol, int n_steps,
                           double w_lo, double w_hi, double eta, double prefactor, double *I_out,
                           double *Gamma);

/* Gradient of a scalar L with dL = tr(Gamma dH) through the assembly (Eq. Hamiltonian with
 * the kernels of Eq. W_LRI), FP64 throughout; the pair projections are recomputed per q-slab.
 *  Gamma : [dim][dim] complex128 Hermitian seed.
 *  dW_R  : [n_RW][N_aux][N_aux] float64, dL/dW_mu,nu(R) = w_R Re sum_q e^{-iq.R} dL/dW(q)_mu,nu
 *          (a perturbation of the symmetric pair W_mu,nu(R), W_nu,mu(-R) moves L by the sum of
 *          the two entries);
 *  de_qp : [N_k][nv+nc] float64, dL/dE^QP of each window band at each k.
 * Needs interp_W and project_pairs first; the first call allocates the adjoint workspace
 * (N_k N_aux^2 complex128 plus one q-slab of projections). */
bse_status bse_adjoint(bse_ctx *ctx, const double *Gamma, double *dW_R, double *de_qp);

/* Batching of several crystals (one context each, every one past bse_project_pairs): their
 * assemblies run as one CUDA graph forked from and joined into `cuda_stream`, so the host
 * issues one launch.  The systems are ordered by estimated work, smallest first (so small
 * systems finish early instead of queueing behind large ones), and dealt in that order to two
 * concurrent chains.  Per chain, schedule
 *  BSE_BATCH_WORKLIST: the chain's (system, q-slab) units are packed into steps (the next slab
 *    of each unfinished system in order, at most one per system, until the step's M_vv W(q)
 *    tiles fill two waves of the SMs); each stage of a step (the exchange GEMMs of systems
 *    starting there, the pair projections, M_vv W(q), the second contraction or the fused
 *    direct term) runs as one launch over the work list of its (system, q, tile) units, per
 *    kernel instantiation (window, N tile, block size; the tensor-core ones persistent).
 *    Every system must use the same split precision (BSE_EINVAL otherwise).
 *  BSE_BATCH_CHAINS: each system's own assembly in turn.
 * The first call for a given list of (context, H) and schedule runs the assemblies once
 * eagerly, then captures and instantiates the graph; later calls with the same list replay it.
 *  H : [n] device pointers as in bse_assemble;  stamps_ns : optional host [n] receiving, for
 *  each system, the nanoseconds from the start of this replay to the end of its assembly
 *  (the call then waits for the stream), or NULL.  Contexts must not be freed while a graph
 *  that uses them is cached; bse_batch_release drops every cached graph. */
typedef enum { BSE_BATCH_WORKLIST = 0, BSE_BATCH_CHAINS = 1 } bse_batch_schedule;
bse_status bse_batch_assemble(bse_ctx **ctxs, void **H, int n, void *cuda_stream, int32_t schedule,
                              int64_t *stamps_ns);
void bse_batch_release(void);

/* Autotuner (call after bse_project_pairs): times one q-slab of the pair projections for each
 * thread-block size (warp multiples up to 160 threads and the ABF count) and the tensor-core
 * GEMM T = M_vv W(q) of the unfused direct term for each N tile (64, 96, 128, 160 columns),
 * keeps the fastest of each for this context and reports them in *chosen_tile and
 * *chosen_proj_threads (either pointer may be NULL; 0 for BSE_FP64, which has neither kernel,
 * and for a projection without a register-blocked kernel).  Results are cached per shape for
 * the life of the process.  Synchronous. */
bse_status bse_autotune(bse_ctx *ctx, int *chosen_tile, int *chosen_proj_threads);

/* Wait for the context's stream, then read and clear the device error word.
 *  timeout_ms >= 0: poll the stream for at most that many milliseconds (host clock); if its
 *                   work has not finished by then, return BSE_ETIMEOUT without touching the
 *                   error word -- the work keeps running and bse_sync may be called again;
 *  timeout_ms < 0 : wait without a limit.
 * After the work is done: BSE_ETIMEOUT if a bounded device-side wait gave up, BSE_EDEVICE if a
 * device-side check failed (see bse_last_error), BSE_ECUDA if the stream reported an error. */
bse_status bse_sync(bse_ctx *ctx, int32_t timeout_ms);

/* Failure-detection self tests (host-side and bounded; neither faults nor hangs the GPU):
 *  bse_selftest_delay enqueues on the context's stream a host function that sleeps `ms`
 *  (0..60000) milliseconds, so the stream stays busy for that long (a bse_sync with a shorter
 *  timeout returns BSE_ETIMEOUT);
 *  bse_selftest_wait launches one block that waits, through the same bounded mbarrier wait as
 *  the tensor-core and matvec pipelines, on a barrier nothing completes; after `cycles`
 *  (1..4e9) clock cycles it gives up and sets the error word, and the next bse_sync returns
 *  BSE_ETIMEOUT with the context still usable.  The paper has no counterpart. */
bse_status bse_selftest_delay(bse_ctx *ctx, int32_t ms);
bse_status bse_selftest_wait(bse_ctx *ctx, int64_t cycles);

/* Text of the last error on this context (never NULL; "" when none). */
const char *bse_last_error(const bse_ctx *ctx);

/* Size queries. */
int64_t bse_dim(const bse_ctx *ctx);
int32_t bse_naux(const bse_ctx *ctx);
int32_t bse_nao(const bse_ctx *ctx);

/* Number of kernels this library has launched in this process (all contexts). */
int64_t bse_launch_count(void);

/* Per-kernel CUDA-event timing on the context's stream (off by default).  While enabled,
 * each launch of the kernels below is bracketed by two events; bse_profile_read
 * synchronises the stream and returns the accumulated device time and launch count of
 * one kernel since profiling was (re-)enabled. */
typedef enum {
  BSE_KP_INTERP = 0,   /* W(q) interpolation                               */
  BSE_KP_HALF = 1,     /* C(k) and half-transform Y(k)                     */
  BSE_KP_PROJECT = 2,  /* pair projection M_vv, M_cc of one q-slab         */
  BSE_KP_G1 = 3,       /* T = M_vv W(q) contraction                        */
  BSE_KP_G2 = 4,       /* T M_cc^T + exchange + diagonal, H write          */
  BSE_KP_EXCH = 5,     /* exchange contraction (tensor-core path)          */
  BSE_KP_MATVEC = 6,   /* Lanczos H x                                      */
  BSE_KP_REORTH = 7,   /* Lanczos reorthogonalisation                      */
  BSE_KP_COUNT = 8
} bse_kernel_id;
bse_status bse_profile(bse_ctx *ctx, int enable);
bse_status bse_profile_read(bse_ctx *ctx, int kernel_id, double *total_ms, int64_t *launches);

/* Release the workspace and the context.  NULL-safe.  Synchronises the stream first. */
void bse_free(bse_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* BSE_H */
