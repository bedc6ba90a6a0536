// Host side of the C ABI declared in include/bse.h: validation, workspace, call order,
// and the q-slab loop of the FP64 assembly.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <set>
#include <string>
#include <thread>
#include <utility>

#include "bse_internal.cuh"
#include "tc_ptx.cuh"

static std::atomic<long long> g_launches{0};
void bse_count_launch(int n) { g_launches += n; }

static std::mutex g_once_mu;
static std::set<std::pair<int, int>> g_once_done;

void bse_once_per_device(const bse_ctx *c, int key, void (*fn)()) {
  std::lock_guard<std::mutex> lk(g_once_mu);
  if (!g_once_done.insert({c->device, key}).second) return;
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != c->device) cudaSetDevice(c->device);
  fn();
  if (cur != c->device && cur >= 0) cudaSetDevice(cur);
}

bse_status bse_fail(bse_ctx *c, bse_status s, const std::string &msg) {
  if (c) c->err = msg;
  return s;
}

bse_status bse_check_launch(bse_ctx *c, const char *what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return bse_fail(c, BSE_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return BSE_OK;
}

template <class T>
static bse_status dalloc(bse_ctx *c, T **p, size_t n) {
  *p = nullptr;
  if (n == 0) return BSE_OK;
  cudaError_t e = cudaMalloc((void **)p, n * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return bse_fail(c, BSE_ENOMEM, "cudaMalloc of " + std::to_string(n * sizeof(T)) + " bytes failed");
  }
  return BSE_OK;
}

template <class T>
static bse_status upload(bse_ctx *c, T **dst, const std::vector<T> &src) {
  bse_status s = dalloc(c, dst, src.size());
  if (s != BSE_OK) return s;
  if (src.empty()) return BSE_OK;
  if (cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
    return bse_fail(c, BSE_ECUDA, "upload of parameter tables failed");
  return BSE_OK;
}

static cudaEvent_t take_event(bse_ctx *c) {
  if (!c->pool.empty()) {
    cudaEvent_t e = c->pool.back();
    c->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

static int g_open_id = -1;
static cudaEvent_t g_open_ev = nullptr;

void bse_prof_begin(bse_ctx *c, int id) {
  if (!c->prof || id < 0 || id >= BSE_KP_COUNT) return;
  g_open_ev = take_event(c);
  g_open_id = id;
  cudaEventRecord(g_open_ev, c->stream);
}

void bse_prof_end(bse_ctx *c, int id) {
  if (!c->prof || g_open_id != id || !g_open_ev) return;
  cudaEvent_t e = take_event(c);
  cudaEventRecord(e, c->stream);
  c->pending.push_back({id, g_open_ev, e});
  g_open_ev = nullptr;
  g_open_id = -1;
}

static void prof_collect(bse_ctx *c) {
  for (auto &p : c->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      c->prof_ms[p.id] += ms;
      c->prof_n[p.id] += 1;
    }
    c->pool.push_back(p.a);
    c->pool.push_back(p.b);
  }
  c->pending.clear();
  cudaGetLastError();
}

static void release(bse_ctx *c) {
  if (!c) return;
  prof_collect(c);
  for (cudaEvent_t e : c->pool) cudaEventDestroy(e);
  c->pool.clear();
  void *ptrs[] = {c->d_qplus, c->d_qall, c->Aq, c->d_R_C, c->d_R_W, c->d_w_RW, c->d_aux_atom, c->d_ao_start, c->d_nao,
                  c->d_aux_start, c->d_naux, c->d_err, c->Wq, c->V0c, c->Y, c->ck,
                  c->eqp, c->X, c->P, c->Mv, c->Mc, c->T, c->Bm1, c->Bt1, c->Bm2};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  split_free(c);
}

// One mbarrier that expects an arrival nothing makes: the bounded wait of the library's
// tensor-core and matvec pipelines (tc::mbar_wait_bounded) runs out after `cycles` clock
// cycles, and the kernel records BSE_DERR_TIMEOUT in the error word as they do.
__global__ void k_selftest_wait(long long cycles, int *err) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    tc::fence_barrier_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && !tc::mbar_wait_bounded(&bar, 0, cycles)) atomicOr(err, BSE_DERR_TIMEOUT);
}

extern "C" {

int64_t bse_launch_count(void) { return g_launches.load(); }

const char *bse_last_error(const bse_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }
int64_t bse_dim(const bse_ctx *ctx) { return ctx ? ctx->dim : -1; }
int32_t bse_naux(const bse_ctx *ctx) { return ctx ? ctx->naux_tot : -1; }
int32_t bse_nao(const bse_ctx *ctx) { return ctx ? ctx->nao_tot : -1; }

// The optional coarse-mesh checks of W's R-set: per Born-von Karman class of the coarse mesh
// the image weights sum to one, and (with the lattice) each image is a shortest member of its
// class, i.e. the set is the Wigner-Seitz folding the interpolation of §III.B assumes.
static bool check_coarse(const bse_params *p) {
  const int *N = p->coarse;
  if (N[0] == 0 && N[1] == 0 && N[2] == 0) return true;
  for (int i = 0; i < 3; i++)
    if (N[i] < 1 || N[i] > 4096) return false;
  const long long ncls = (long long)N[0] * N[1] * N[2];
  if (ncls > (1 << 24)) return false;
  std::vector<double> wsum((size_t)ncls, 0.0);
  for (int r = 0; r < p->n_RW; r++) {
    const int *R = p->R_W + 3 * r;
    if (!(p->w_RW[r] > 0.0)) return false;
    long long idx = 0;
    for (int i = 0; i < 3; i++) idx = idx * N[i] + ((R[i] % N[i]) + N[i]) % N[i];
    wsum[(size_t)idx] += p->w_RW[r];
  }
  for (double w : wsum)
    if (std::fabs(w - 1.0) > 1e-9) return false;
  if (!p->lattice) return true;
  for (int i = 0; i < 9; i++)
    if (!std::isfinite(p->lattice[i])) return false;
  auto len = [&](double r0, double r1, double r2) {
    double s = 0.0;
    for (int j = 0; j < 3; j++) {
      const double x = r0 * p->lattice[j] + r1 * p->lattice[3 + j] + r2 * p->lattice[6 + j];
      s += x * x;
    }
    return std::sqrt(s);
  };
  for (int r = 0; r < p->n_RW; r++) {
    const int *R = p->R_W + 3 * r;
    const double l0 = len(R[0], R[1], R[2]);
    for (int m0 = -1; m0 <= 1; m0++)
      for (int m1 = -1; m1 <= 1; m1++)
        for (int m2 = -1; m2 <= 1; m2++) {
          const double l = len(R[0] + (double)m0 * N[0], R[1] + (double)m1 * N[1], R[2] + (double)m2 * N[2]);
          if (l0 > l * (1.0 + 1e-9) + 1e-9) return false;
        }
  }
  return true;
}

bse_status bse_check_params(const bse_params *p) {
  if (!p) return BSE_EINVAL;
  if (p->n_atoms < 1 || p->n_atoms > 4096 || !p->nao_per_atom || !p->naux_per_atom) return BSE_EINVAL;
  for (int i = 0; i < 3; i++) {
    if (p->dense[i] < 1 || p->dense[i] > 4096) return BSE_EINVAL;
    if (!std::isfinite(p->k_offset[i])) return BSE_EINVAL;
  }
  if (p->n_RC < 1 || !p->R_C || p->n_RW < 1 || !p->R_W || !p->w_RW) return BSE_EINVAL;
  if (p->nv < 1 || p->nc < 1 || p->nv > 8 || p->nc > 8) return BSE_EINVAL;
  if (p->precision < BSE_FP64 || p->precision > BSE_TF32X2) return BSE_EINVAL;
  if (!std::isfinite(p->alpha)) return BSE_EINVAL;
  long long nk = (long long)p->dense[0] * p->dense[1] * p->dense[2];
  if (nk > 65535) return BSE_EINVAL;
  int nao_tot = 0, naux_tot = 0;
  for (int a = 0; a < p->n_atoms; a++) {
    if (p->nao_per_atom[a] < 1 || p->naux_per_atom[a] < 1) return BSE_EINVAL;
    nao_tot += p->nao_per_atom[a];
    naux_tot += p->naux_per_atom[a];
  }
  if (p->nv + p->nc > nao_tot || naux_tot > 8192 || nao_tot > 4096) return BSE_EINVAL;
  for (int r = 0; r < p->n_RW; r++)
    if (!std::isfinite(p->w_RW[r])) return BSE_EINVAL;
  if (!check_coarse(p)) return BSE_EINVAL;
  return BSE_OK;
}

bse_status bse_setup(const bse_params *p, void *cuda_stream, bse_ctx **out) {
  if (!out) return BSE_EINVAL;
  *out = nullptr;
  const bse_status chk = bse_check_params(p);
  if (chk != BSE_OK) return chk;
  const long long nk = (long long)p->dense[0] * p->dense[1] * p->dense[2];
  int nao_tot = 0, naux_tot = 0, nao_max = 0;
  for (int a = 0; a < p->n_atoms; a++) {
    nao_tot += p->nao_per_atom[a];
    naux_tot += p->naux_per_atom[a];
    nao_max = std::max(nao_max, p->nao_per_atom[a]);
  }

  bse_ctx *c = new bse_ctx();
  c->n_atoms = p->n_atoms;
  c->nao.assign(p->nao_per_atom, p->nao_per_atom + p->n_atoms);
  c->naux.assign(p->naux_per_atom, p->naux_per_atom + p->n_atoms);
  int s0 = 0, m0 = 0;
  std::vector<int> aux_atom;
  for (int a = 0; a < p->n_atoms; a++) {
    c->ao_start.push_back(s0);
    c->aux_start.push_back(m0);
    for (int m = 0; m < c->naux[a]; m++) aux_atom.push_back(a);
    s0 += c->nao[a];
    m0 += c->naux[a];
  }
  c->nao_tot = nao_tot;
  c->naux_tot = naux_tot;
  c->nao_max = nao_max;
  for (int i = 0; i < 3; i++) {
    c->mesh[i] = p->dense[i];
    c->koff[i] = p->k_offset[i];
  }
  c->nk = (int)nk;
  c->n_RC = p->n_RC;
  c->n_RW = p->n_RW;
  c->R_C.assign(p->R_C, p->R_C + 3 * p->n_RC);
  c->R_W.assign(p->R_W, p->R_W + 3 * p->n_RW);
  c->w_RW.assign(p->w_RW, p->w_RW + p->n_RW);
  c->nv = p->nv;
  c->nc = p->nc;
  c->nb = p->nv + p->nc;
  c->nvc = p->nv * p->nc;
  c->alpha = p->alpha;
  c->precision = p->precision;
  c->h64 = p->precision == BSE_FP64 || p->h_complex128 != 0;
  c->dim = nk * c->nvc;
  c->stream = (cudaStream_t)cuda_stream;
  cudaGetDevice(&c->device);
  cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, c->device);

  // transfers q in a half set, ordered by lines along the last mesh axis
  {
    const int n1 = c->mesh[0], n2 = c->mesh[1], n3 = c->mesh[2];
    for (int q1 = 0; q1 < n1; q1++)
      for (int q2 = 0; q2 < n2; q2++) {
        const int m1 = (n1 - q1) % n1, m2 = (n2 - q2) % n2;
        if (q1 < m1 || (q1 == m1 && q2 < m2)) {
          for (int q3 = 0; q3 < n3; q3++) c->qplus.push_back((q1 * n2 + q2) * n3 + q3);
        } else if (q1 == m1 && q2 == m2) {
          for (int q3 = 0; q3 < n3; q3++)
            if (q3 <= (n3 - q3) % n3 || q3 == 0) c->qplus.push_back((q1 * n2 + q2) * n3 + q3);
        }
      }
  }
  bse_status s = BSE_OK;
#define TRY(x)              \
  do {                      \
    s = (x);                \
    if (s != BSE_OK) goto fail; \
  } while (0)
  {
    TRY(upload(c, &c->d_R_C, c->R_C));
    TRY(upload(c, &c->d_R_W, c->R_W));
    TRY(upload(c, &c->d_w_RW, c->w_RW));
    TRY(upload(c, &c->d_aux_atom, aux_atom));
    TRY(upload(c, &c->d_ao_start, c->ao_start));
    TRY(upload(c, &c->d_nao, c->nao));
    TRY(upload(c, &c->d_aux_start, c->aux_start));
    TRY(upload(c, &c->d_naux, c->naux));
    TRY(upload(c, &c->d_qplus, c->qplus));
    {
      std::vector<int> qall(c->nk);
      for (int q = 0; q < c->nk; q++) qall[q] = q;
      TRY(upload(c, &c->d_qall, qall));
    }
    TRY(dalloc(c, &c->d_err, 1));
    const size_t nn = (size_t)naux_tot * naux_tot;
    TRY(dalloc(c, &c->V0c, nn));
    TRY(dalloc(c, &c->Y, (size_t)nk * nao_max * c->nb * naux_tot));
    TRY(dalloc(c, &c->ck, (size_t)nk * nao_tot * c->nb));
    TRY(dalloc(c, &c->eqp, (size_t)nk * c->nb));
    TRY(dalloc(c, &c->X, (size_t)c->dim * naux_tot));
    TRY(dalloc(c, &c->P, (size_t)c->dim * naux_tot));
    if (cudaMemset(c->d_err, 0, sizeof(int)) != cudaSuccess ||
        cudaMemset(c->Y, 0, (size_t)nk * nao_max * c->nb * naux_tot * sizeof(double2)) != cudaSuccess) {
      s = bse_fail(c, BSE_ECUDA, "workspace initialisation failed");
      goto fail;
    }
    if (c->precision == BSE_FP64) {
      TRY(dalloc(c, &c->Wq, (size_t)nk * nn));
      const size_t per_q = (size_t)nk * (2 * c->nv * c->nv + c->nc * c->nc) * naux_tot * sizeof(double2);
      size_t budget = (size_t)768 << 20;
      c->slab = (int)std::max<size_t>(1, std::min<size_t>((size_t)c->nk, budget / std::max<size_t>(per_q, 1)));
      c->slab = std::min(c->slab, 65535);
      TRY(dalloc(c, &c->Mv, (size_t)c->slab * nk * c->nv * c->nv * naux_tot));
      TRY(dalloc(c, &c->T, (size_t)c->slab * nk * c->nv * c->nv * naux_tot));
      TRY(dalloc(c, &c->Mc, (size_t)c->slab * nk * c->nc * c->nc * naux_tot));
    } else {
      TRY(split_setup(c));
    }
  }
#undef TRY
  if (cudaDeviceSynchronize() != cudaSuccess) {
    s = bse_fail(c, BSE_ECUDA, "setup synchronisation failed");
    goto fail;
  }
  *out = c;
  return BSE_OK;
fail:
  release(c);
  delete c;
  return s;
}

namespace {
__global__ void k_real_to_complex(const double *src, double2 *dst, long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = make_double2(src[i], 0.0);
}
}  // namespace

bse_status bse_interp_W(bse_ctx *c, const double *W_R, const double *V0, void *Wq_out) {
  if (!c) return BSE_EINVAL;
  if (!W_R || (!V0 && !c->vx_from_R)) return bse_fail(c, BSE_EINVAL, "interp_W: null W_R or V0");
  const long long nn = (long long)c->naux_tot * c->naux_tot;
  bse_status s = BSE_OK;
  if (!c->vx_from_R) {  // bse_set_momentum's V_R, when given, fixes the exchange interaction
    k_real_to_complex<<<(unsigned)((nn + 255) / 256), 256, 0, c->stream>>>(V0, c->V0c, nn);
    bse_count_launch();
    s = bse_check_launch(c, "V0 copy");
    if (s != BSE_OK) return s;
  }
  if (c->precision == BSE_FP64) {
    s = launch_interp_W_fp64(c, W_R, c->Wq);
    if (s != BSE_OK) return s;
    if (Wq_out &&
        cudaMemcpyAsync(Wq_out, c->Wq, (size_t)c->nk * nn * sizeof(double2), cudaMemcpyDeviceToDevice,
                        c->stream) != cudaSuccess)
      return bse_fail(c, BSE_ECUDA, "interp_W: copy to Wq_out failed");
  } else {
    s = split_interp_W(c, W_R, (double2 *)Wq_out);
    if (s != BSE_OK) return s;
  }
  c->stage = std::max(c->stage, 1);
  return BSE_OK;
}

bse_status bse_interp_V(bse_ctx *c, const double *V_R, void *Vq_out) {
  if (!c) return BSE_EINVAL;
  if (!V_R || !Vq_out) return bse_fail(c, BSE_EINVAL, "interp_V: null V_R or Vq_out");
  return launch_interp_W_fp64(c, V_R, (double2 *)Vq_out);
}

bse_status bse_set_momentum(bse_ctx *c, const int32_t *Q, const double *V_R) {
  if (!c) return BSE_EINVAL;
  if (!Q) return bse_fail(c, BSE_EINVAL, "set_momentum: null Q");
  int m[3];
  bool finite = false;
  for (int i = 0; i < 3; i++) {
    m[i] = (int)(((long long)Q[i] % c->mesh[i] + c->mesh[i]) % c->mesh[i]);
    finite = finite || m[i] != 0;
  }
  if (finite && c->alpha != 0.0 && !V_R)
    return bse_fail(c, BSE_EINVAL, "set_momentum: the exchange at Q != 0 needs V_R");
  const int n1 = c->mesh[0], n2 = c->mesh[1], n3 = c->mesh[2];
  const bool had_vx = c->vx_from_R;
  for (int i = 0; i < 3; i++) c->Qm[i] = m[i];
  c->qQ = (m[0] * n2 + m[1]) * n3 + m[2];
  c->qmQ = (((n1 - m[0]) % n1) * n2 + (n2 - m[1]) % n2) * n3 + (n3 - m[2]) % n3;
  c->vx_from_R = V_R != nullptr;
  if (V_R) {
    // V at the transfer -Q: sum_R w_R Vbar(R) e^{+iQ.R}
    bse_status s = launch_interp_W_fp64(c, V_R, c->V0c, c->qmQ, 1);
    if (s != BSE_OK) return s;
  }
  // the exchange factors and P = X V depend on Q; a V(0) replaced by V_R must come back
  // through bse_interp_W before a Q = 0 assembly without V_R
  c->stage = std::min(c->stage, (had_vx && !V_R) ? 0 : 1);
  return BSE_OK;
}

bse_status bse_project_pairs(bse_ctx *c, const double *C_R, const double *c_k, const double *e_qp) {
  if (!c) return BSE_EINVAL;
  if (c->stage < 1) return bse_fail(c, BSE_ESTATE, "project_pairs before interp_W");
  if (!C_R || !c_k || !e_qp) return bse_fail(c, BSE_EINVAL, "project_pairs: null argument");
  if (cudaMemcpyAsync(c->ck, c_k, (size_t)c->nk * c->nao_tot * c->nb * sizeof(double2),
                      cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess ||
      cudaMemcpyAsync(c->eqp, e_qp, (size_t)c->nk * c->nb * sizeof(double), cudaMemcpyDeviceToDevice,
                      c->stream) != cudaSuccess)
    return bse_fail(c, BSE_ECUDA, "project_pairs: copy of c_k / e_qp failed");
  bse_status s;
  if (c->precision == BSE_FP64) {
    s = launch_half_transform_fp64(c, C_R);
    if (s != BSE_OK) return s;
    s = launch_exchange_factors_fp64(c);
    if (s != BSE_OK) return s;
    // P = X V(0): rows (k,i,a), K = N = N_aux
    s = launch_zgemm_fp64(c, (int)c->dim, c->naux_tot, c->naux_tot, c->X, c->naux_tot, 0, c->V0c,
                          c->naux_tot, 0, c->P, c->naux_tot, 0, 1);
    if (s != BSE_OK) return s;
  } else {
    s = split_project(c, C_R);
    if (s != BSE_OK) return s;
  }
  c->stage = 2;
  return BSE_OK;
}

bse_status bse_assemble(bse_ctx *c, void *H) {
  if (!c) return BSE_EINVAL;
  if (c->stage < 2) return bse_fail(c, BSE_ESTATE, "assemble before project_pairs");
  if (!H) return bse_fail(c, BSE_EINVAL, "assemble: null H");
  if (c->precision != BSE_FP64) return split_assemble(c, H);
  const int na = c->naux_tot;
  const long long rows = (long long)c->nk * c->nv * c->nv;
  const int nqp = (int)c->qplus.size();
  for (int q0 = 0; q0 < nqp; q0 += c->slab) {
    const int nq = std::min(c->slab, nqp - q0);
    bse_status s = launch_project_slab_fp64(c, q0, nq, c->d_qplus);
    if (s != BSE_OK) return s;
    s = launch_zgemm_fp64(c, (int)rows, na, na, c->Mv, na, rows * na, c->Wq, na, (long long)na * na, c->T, na,
                          rows * na, nq, BSE_KP_G1, c->d_qplus + q0);
    if (s != BSE_OK) return s;
    s = launch_g2_write_fp64(c, q0, nq, (double2 *)H);
    if (s != BSE_OK) return s;
  }
  return BSE_OK;
}

bse_status bse_assemble_coupling(bse_ctx *c, void *B) {
  if (!c) return BSE_EINVAL;
  if (c->stage < 2) return bse_fail(c, BSE_ESTATE, "assemble_coupling before project_pairs");
  if (!B) return bse_fail(c, BSE_EINVAL, "assemble_coupling: null B");
  if (c->qQ != 0) return bse_fail(c, BSE_EINVAL, "assemble_coupling: the full BSE is built at Q = 0");
  if (c->precision != BSE_FP64 && c->h64)
    return bse_fail(c, BSE_EINVAL, "assemble_coupling: the full BSE takes the complex64 split H (h_complex128 is for the TDA entries)");

  if (c->precision != BSE_FP64) return split_assemble_coupling(c, B);
  const int na = c->naux_tot;
  const long long rows = (long long)c->nk * c->nvc;
  if (!c->Bm1) {
    const size_t per_q = (size_t)3 * rows * na * sizeof(double2);
    const size_t budget = (size_t)768 << 20;
    c->slab_cv = (int)std::max<size_t>(1, std::min<size_t>((size_t)c->nk, budget / std::max<size_t>(per_q, 1)));
    c->slab_cv = std::min(c->slab_cv, 65535);
    const size_t n = (size_t)c->slab_cv * rows * na;
    bse_status s = dalloc(c, &c->Bm1, n);
    if (s == BSE_OK) s = dalloc(c, &c->Bt1, n);
    if (s == BSE_OK) s = dalloc(c, &c->Bm2, n);
    if (s != BSE_OK) return s;
  }
  const int nqp = (int)c->qplus.size();
  for (int q0 = 0; q0 < nqp; q0 += c->slab_cv) {
    const int nq = std::min(c->slab_cv, nqp - q0);
    bse_status s = launch_project_cv_slab_fp64(c, q0, nq, c->d_qplus, c->Bm1, c->Bm2);
    if (s != BSE_OK) return s;
    s = launch_zgemm_fp64(c, (int)rows, na, na, c->Bm1, na, rows * na, c->Wq, na, (long long)na * na, c->Bt1, na,
                          rows * na, nq, BSE_KP_G1, c->d_qplus + q0);
    if (s != BSE_OK) return s;
    s = launch_g2_coupling_fp64(c, q0, nq, c->Bt1, c->Bm2, (double2 *)B);
    if (s != BSE_OK) return s;
  }
  return BSE_OK;
}

bse_status bse_dipole_vector(bse_ctx *c, const double *vel, const double *e_ks, double *u) {
  if (!c) return BSE_EINVAL;
  if (!vel || !e_ks || !u) return bse_fail(c, BSE_EINVAL, "dipole_vector: null argument");
  if (c->qQ != 0) return bse_fail(c, BSE_EINVAL, "dipole_vector: optical transitions are vertical (Q = 0)");
  return run_dipole_vector(c, vel, e_ks, (double2 *)u);
}

bse_status bse_spectrum(bse_ctx *c, const void *H, const double *u, int n_pol, int n_steps,
                        const double *omega, int n_w, double eta, double prefactor, double *eps2,
                        double *ab) {
  if (!c) return BSE_EINVAL;
  if (!H || !u || !omega || !eps2) return bse_fail(c, BSE_EINVAL, "spectrum: null argument");
  if (n_pol < 1 || n_pol > 3 || n_steps < 1 || n_steps > c->dim || n_w < 1 || !(eta > 0.0) ||
      !std::isfinite(prefactor))
    return bse_fail(c, BSE_EINVAL, "spectrum: bad size or parameter");
  return run_spectrum(c, H, (const double2 *)u, n_pol, n_steps, omega, n_w, eta, prefactor, eps2, ab);
}

bse_status bse_spectrum_add(bse_ctx *c, const void *H, const double *u, int n_pol, int n_steps,
                            const double *omega, int n_w, double eta, double prefactor, double weight,
                            double *eps2_acc) {
  if (!c) return BSE_EINVAL;
  if (!H || !u || !omega || !eps2_acc) return bse_fail(c, BSE_EINVAL, "spectrum_add: null argument");
  if (n_pol < 1 || n_pol > 3 || n_steps < 1 || n_steps > c->dim || n_w < 1 || !(eta > 0.0) ||
      !std::isfinite(prefactor) || !std::isfinite(weight))
    return bse_fail(c, BSE_EINVAL, "spectrum_add: bad size or parameter");
  return run_spectrum(c, H, (const double2 *)u, n_pol, n_steps, omega, n_w, eta, prefactor * weight, eps2_acc,
                      nullptr, true);
}

bse_status bse_spectrum_static(bse_ctx *c, const void *H, const double *u, int n_pol, int n_steps,
                               const double *omega, int n_w, double eta, double prefactor, double *eps2,
                               double *ab) {
  if (!c) return BSE_EINVAL;
  if (!H || !u || !omega || !eps2) return bse_fail(c, BSE_EINVAL, "spectrum_static: null argument");
  if (n_pol < 1 || n_pol > 3 || n_steps < 1 || n_steps > c->dim || n_w < 1 || !(eta > 0.0) ||
      !std::isfinite(prefactor))
    return bse_fail(c, BSE_EINVAL, "spectrum_static: bad size or parameter");
  return run_spectrum_static(c, H, (const double2 *)u, n_pol, n_steps, omega, n_w, eta, prefactor, eps2, ab);
}

bse_status bse_spectrum_full(bse_ctx *c, const void *A, const void *B, const double *u, int n_pol, int n_steps,
                             const double *omega, int n_w, double eta, double prefactor, double *eps2) {
  if (!c) return BSE_EINVAL;
  if (!A || !B || !u || !omega || !eps2) return bse_fail(c, BSE_EINVAL, "spectrum_full: null argument");
  if (c->precision != BSE_FP64 && c->h64)
    return bse_fail(c, BSE_EINVAL, "spectrum_full: the full BSE takes the complex64 split H (h_complex128 is for the TDA entries)");

  if (n_pol < 1 || n_pol > 3 || n_steps < 2 || n_steps > 2 * c->dim || n_steps > BSE_FULL_MAX_STEPS || n_w < 1 ||
      !(eta > 0.0) || !std::isfinite(prefactor))
    return bse_fail(c, BSE_EINVAL, "spectrum_full: bad size or parameter");
  return run_spectrum_full(c, A, B, (const double2 *)u, n_pol, n_steps, omega, n_w, eta, prefactor, eps2);
}

bse_status bse_lowest_full(bse_ctx *c, const void *A, const void *B, int n_eig, int n_steps, uint64_t seed,
                           double *omega_out, double *resid_out) {
  if (!c) return BSE_EINVAL;
  if (!A || !B || !omega_out) return bse_fail(c, BSE_EINVAL, "lowest_full: null argument");
  if (c->precision != BSE_FP64 && c->h64)
    return bse_fail(c, BSE_EINVAL, "lowest_full: the full BSE takes the complex64 split H (h_complex128 is for the TDA entries)");

  if (n_steps < 2 || n_steps > 2 * c->dim || n_steps > BSE_FULL_MAX_STEPS || n_eig < 1 || 2 * n_eig > n_steps)
    return bse_fail(c, BSE_EINVAL, "lowest_full: bad size");
  return run_lowest_full(c, A, B, n_eig, n_steps, seed, omega_out, resid_out);
}

bse_status bse_spectrum_matfree(bse_ctx *c, const double *u, int n_pol, int n_steps, const double *omega, int n_w,
                                double eta, double prefactor, double *eps2, double *ab) {
  if (!c) return BSE_EINVAL;
  if (c->stage < 2) return bse_fail(c, BSE_ESTATE, "spectrum_matfree before project_pairs");
  if (!u || !omega || !eps2) return bse_fail(c, BSE_EINVAL, "spectrum_matfree: null argument");
  if (c->precision == BSE_FP64)
    return bse_fail(c, BSE_EINVAL, "spectrum_matfree: the matrix-free product runs in the split precisions");
  if (n_pol < 1 || n_pol > 3 || n_steps < 1 || n_steps > c->dim || n_w < 1 || !(eta > 0.0) ||
      !std::isfinite(prefactor))
    return bse_fail(c, BSE_EINVAL, "spectrum_matfree: bad size or parameter");
  return run_spectrum_matfree(c, (const double2 *)u, n_pol, n_steps, omega, n_w, eta, prefactor, eps2, ab);
}

bse_status bse_lowest(bse_ctx *c, const void *H, int n_eig, int n_steps, uint64_t seed,
                      double *omega_out, double *resid_out, double *vecs_out) {
  if (!c) return BSE_EINVAL;
  if (!H || !omega_out) return bse_fail(c, BSE_EINVAL, "lowest: null argument");
  if (n_steps < 1 || n_steps > c->dim || n_eig < 1 || n_eig > n_steps)
    return bse_fail(c, BSE_EINVAL, "lowest: bad size");
  return run_lowest(c, H, n_eig, n_steps, seed, omega_out, resid_out, (double2 *)vecs_out);
}

bse_status bse_window_seed(bse_ctx *c, const void *H, const double *u, int n_pol, int n_steps, double w_lo,
                           double w_hi, double eta, double prefactor, double *I_out, double *Gamma) {
  if (!c) return BSE_EINVAL;
  if (!H || !u || !Gamma) return bse_fail(c, BSE_EINVAL, "window_seed: null H, u or Gamma");
  if (n_pol < 1 || n_pol > 3) return bse_fail(c, BSE_EINVAL, "window_seed: n_pol must be 1..3");
  if (n_steps < 1 || n_steps > c->dim) return bse_fail(c, BSE_EINVAL, "window_seed: n_steps must be 1..dim");
  if (!(eta > 0.0) || !(w_hi > w_lo)) return bse_fail(c, BSE_EINVAL, "window_seed: need eta > 0 and w_hi > w_lo");
  return run_window_seed(c, H, (const double2 *)u, n_pol, n_steps, w_lo, w_hi, eta, prefactor, I_out,
                         (double2 *)Gamma);
}

bse_status bse_adjoint_seed(bse_ctx *c, const double *vecs, const double *g, int r, double *Gamma) {
  if (!c) return BSE_EINVAL;
  if (!vecs || !g || !Gamma || r < 1) return bse_fail(c, BSE_EINVAL, "adjoint_seed: bad argument");
  return run_seed_lowrank(c, (const double2 *)vecs, g, r, (double2 *)Gamma);
}

bse_status bse_adjoint(bse_ctx *c, const double *Gamma, double *dW_R, double *de_qp) {
  if (!c) return BSE_EINVAL;
  if (c->stage < 2) return bse_fail(c, BSE_ESTATE, "adjoint before project_pairs");
  if (!Gamma || !dW_R || !de_qp) return bse_fail(c, BSE_EINVAL, "adjoint: null argument");
  return run_adjoint(c, (const double2 *)Gamma, dW_R, de_qp);
}

bse_status bse_sync(bse_ctx *c, int32_t timeout_ms) {
  if (!c) return BSE_EINVAL;
  if (timeout_ms < 0) {
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return bse_fail(c, BSE_ECUDA, std::string("sync: ") + cudaGetErrorString(e));
  } else {
    // poll the stream until its work is done or the host-side deadline passes; the work is
    // left running on a timeout, so a later call can wait for it again
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
      const cudaError_t e = cudaStreamQuery(c->stream);
      if (e == cudaSuccess) break;
      if (e != cudaErrorNotReady) return bse_fail(c, BSE_ECUDA, std::string("sync: ") + cudaGetErrorString(e));
      const auto ms =
          std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0).count();
      if (ms >= timeout_ms)
        return bse_fail(c, BSE_ETIMEOUT,
                        "sync: the stream's work did not finish within " + std::to_string(timeout_ms) +
                            " ms (it keeps running; bse_sync may be called again)");
      std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
  }
  int w = 0;
  if (cudaMemcpy(&w, c->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemset(c->d_err, 0, sizeof(int)) != cudaSuccess)
    return bse_fail(c, BSE_ECUDA, "sync: error word unreadable");
  if (w & BSE_DERR_TIMEOUT) return bse_fail(c, BSE_ETIMEOUT, "a bounded device wait gave up");
  if (w & BSE_DERR_INDEFINITE)
    return bse_fail(c, BSE_EDEVICE, "full BSE: [[A, B], [B*, A*]] is not positive definite (unstable excitations)");
  if (w) return bse_fail(c, BSE_EDEVICE, "device check failed, code " + std::to_string(w));
  return BSE_OK;
}

static void CUDART_CB host_delay(void *ms) { std::this_thread::sleep_for(std::chrono::milliseconds((intptr_t)ms)); }

bse_status bse_selftest_delay(bse_ctx *c, int32_t ms) {
  if (!c) return BSE_EINVAL;
  if (ms < 0 || ms > 60000) return bse_fail(c, BSE_EINVAL, "selftest_delay: 0 <= ms <= 60000");
  if (cudaLaunchHostFunc(c->stream, host_delay, (void *)(intptr_t)ms) != cudaSuccess)
    return bse_fail(c, BSE_ECUDA, "selftest_delay: cudaLaunchHostFunc failed");
  return BSE_OK;
}

bse_status bse_selftest_wait(bse_ctx *c, int64_t cycles) {
  if (!c) return BSE_EINVAL;
  if (cycles < 1 || cycles > 4000000000LL) return bse_fail(c, BSE_EINVAL, "selftest_wait: 1 <= cycles <= 4e9");
  k_selftest_wait<<<1, 32, 0, c->stream>>>(cycles, c->d_err);
  bse_count_launch();
  return bse_check_launch(c, "selftest_wait");
}

bse_status bse_profile(bse_ctx *c, int enable) {
  if (!c) return BSE_EINVAL;
  cudaStreamSynchronize(c->stream);
  prof_collect(c);
  c->prof = enable != 0;
  for (int i = 0; i < BSE_KP_COUNT; i++) {
    c->prof_ms[i] = 0.0;
    c->prof_n[i] = 0;
  }
  return BSE_OK;
}

bse_status bse_profile_read(bse_ctx *c, int id, double *total_ms, int64_t *launches) {
  if (!c) return BSE_EINVAL;
  if (id < 0 || id >= BSE_KP_COUNT || !total_ms || !launches) return bse_fail(c, BSE_EINVAL, "profile_read: bad id");
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return bse_fail(c, BSE_ECUDA, "profile_read: sync failed");
  prof_collect(c);
  *total_ms = c->prof_ms[id];
  *launches = c->prof_n[id];
  return BSE_OK;
}

void bse_free(bse_ctx *c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  release(c);
  delete c;
}

}  // extern "C"
