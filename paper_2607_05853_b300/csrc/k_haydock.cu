// Spectrum step: velocity-form oscillator vector, Haydock/Lanczos recursion with full
// reorthogonalisation (FP64), continued fraction on the frequency grid (Eq. abs_vel with
// a Lorentzian of half-width eta), and lowest Ritz values (Sturm bisection + inverse
// iteration on the Lanczos tridiagonal).
//
// The matrix-vector product reads H once per Lanczos step for all polarisations.  For a
// complex128 H the products are FP64; for a complex64 H (split-precision assembly) the
// products are FP32 (H itself carries FP32 rounding), read through the upper-triangle tiles
// (k_hmv_tma) and summed across tiles with compensated FP32 sums (k_hmv_reduce); the
// recursion scalars, the basis, the norms and the three-term update are FP64, and the
// reorthogonalisation projects on an FP32 shadow of the basis (FP32 products, FP64 chunk
// sums) and subtracts from the FP64 vector.  The short kernels of a step are launched with
// programmatic stream serialization (launch_pdl).
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include <cudaTypedefs.h>

#include "bse_internal.cuh"
#include "tc_ptx.cuh"

namespace {


__global__ void k_dipole(const double2 *__restrict__ vel, const double *__restrict__ eks, int nk,
                         int nv, int nc, double2 *__restrict__ u, int *err) {
  const long long dim = (long long)nk * nv * nc;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int p = blockIdx.y;
  if (idx >= dim) return;
  const int k = (int)(idx / (nv * nc)), i = (int)((idx / nc) % nv), a = (int)(idx % nc);
  const int nb = nv + nc;
  double de = eks[(long long)k * nb + nv + a] - eks[(long long)k * nb + i];
  double2 v = vel[(long long)p * dim + idx];
  if (de == 0.0) {
    atomicOr(err, BSE_DERR_ZERO_DENOM);
    u[(long long)p * dim + idx] = make_double2(0.0, 0.0);
    return;
  }
  u[(long long)p * dim + idx] = make_double2(v.x / de, -v.y / de);
}

// ---- block reductions -------------------------------------------------------------------
template <int NT>
__device__ __forceinline__ double block_sum(double v, double *red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < NT / 32; i++) s += red[i];
  return s;  // valid in thread 0
}

// max |H| over all elements (for the early-stop threshold): per-block maxima, then one block.
template <class HT>
__global__ void k_absmax_part(const HT *__restrict__ H, long long n, double *part) {
  __shared__ double red[32];
  // squared magnitudes in FP32 (the stop threshold only needs max|H| approximately)
  float m2 = 0.f;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float x = (float)H[i].x, y = (float)H[i].y;
    m2 = fmaxf(m2, x * x + y * y);
  }
  double m = sqrt((double)m2);
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int i = 0; i < blockDim.x / 32; i++) r = fmax(r, red[i]);
    part[blockIdx.x] = r;
  }
}
__global__ void k_absmax_final(const double *part, int n, double *out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double r = 0.0;
    for (int i = 0; i < n; i++) r = fmax(r, part[i]);
    *out = r;
  }
}

// beta0[p] = |u_p|, Q[p][0] = u_p / beta0 (block per p).
__global__ void k_lanczos_init(const double2 *__restrict__ u, long long dim, double2 *Q, long long qs,
                               double *beta0, float2 *Q32) {
  __shared__ double red[32];
  __shared__ double sb;
  const int p = blockIdx.x;
  const double2 *up = u + (long long)p * dim;
  double s = 0.0;
  for (long long i = threadIdx.x; i < dim; i += blockDim.x) s += up[i].x * up[i].x + up[i].y * up[i].y;
  s = block_sum<1024>(s, red);
  if (threadIdx.x == 0) {
    sb = sqrt(s);
    beta0[p] = sb;
  }
  __syncthreads();
  const double inv = sb > 0.0 ? 1.0 / sb : 0.0;
  for (long long i = threadIdx.x; i < dim; i += blockDim.x) {
    const double2 v = make_double2(up[i].x * inv, up[i].y * inv);
    Q[p * qs + i] = v;
    if (Q32) Q32[p * qs + i] = make_float2((float)v.x, (float)v.y);
  }
}

constexpr int MV_WARPS = 8, MV_RPW = 4, MV_ROWS = MV_WARPS * MV_RPW, MV_CC = 256;

// W[p][r] = sum_c H[r][c] Q[p][j][c]  -- complex128 H, FP64 arithmetic.
template <int NP>
__global__ void __launch_bounds__(256) k_matvec_c128(const double2 *__restrict__ H, long long dim,
                                                     const double2 *__restrict__ Q, long long qs,
                                                     int j, double2 *__restrict__ W, const int *meff) {
  __shared__ double2 xs[NP][MV_CC];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const long long r0 = (long long)blockIdx.x * MV_ROWS + warp * MV_RPW;
  bool live = false;
  for (int p = 0; p < NP; p++) live |= (j < meff[p]);
  if (!live) return;
  double2 acc[MV_RPW][NP];
#pragma unroll
  for (int r = 0; r < MV_RPW; r++)
#pragma unroll
    for (int p = 0; p < NP; p++) acc[r][p] = make_double2(0, 0);
  for (long long c0 = 0; c0 < dim; c0 += MV_CC) {
    __syncthreads();
    for (int t = threadIdx.x; t < NP * MV_CC; t += blockDim.x) {
      int p = t / MV_CC, cc = t % MV_CC;
      long long c = c0 + cc;
      xs[p][cc] = c < dim ? Q[p * qs + (long long)j * dim + c] : make_double2(0, 0);
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < MV_RPW; r++) {
      const long long row = r0 + r;
      if (row >= dim) continue;
      const double2 *hr = H + row * dim + c0;
#pragma unroll
      for (int t = 0; t < MV_CC / 32; t++) {
        const int cc = lane + 32 * t;
        if (c0 + cc < dim) {
          const double2 h = hr[cc];
#pragma unroll
          for (int p = 0; p < NP; p++) {
            const double2 x = xs[p][cc];
            acc[r][p].x = fma(h.x, x.x, fma(-h.y, x.y, acc[r][p].x));
            acc[r][p].y = fma(h.x, x.y, fma(h.y, x.x, acc[r][p].y));
          }
        }
      }
    }
  }
#pragma unroll
  for (int r = 0; r < MV_RPW; r++)
#pragma unroll
    for (int p = 0; p < NP; p++) {
      double x = acc[r][p].x, y = acc[r][p].y;
      for (int o = 16; o > 0; o >>= 1) {
        x += __shfl_xor_sync(0xffffffffu, x, o);
        y += __shfl_xor_sync(0xffffffffu, y, o);
      }
      const long long row = r0 + r;
      if (lane == 0 && row < dim) W[(long long)p * dim + row] = make_double2(x, y);
    }
}

// Same for a complex64 H: FP32 products and per-lane sums, FP64 across lanes.
template <int NP>
__global__ void __launch_bounds__(256) k_matvec_c64(const float2 *__restrict__ H, long long dim,
                                                    const double2 *__restrict__ Q, long long qs, int j,
                                                    double2 *__restrict__ W, const int *meff) {
  __shared__ float2 xs[NP][MV_CC];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const long long r0 = (long long)blockIdx.x * MV_ROWS + warp * MV_RPW;
  bool live = false;
  for (int p = 0; p < NP; p++) live |= (j < meff[p]);
  if (!live) return;
  float2 acc[MV_RPW][NP];
#pragma unroll
  for (int r = 0; r < MV_RPW; r++)
#pragma unroll
    for (int p = 0; p < NP; p++) acc[r][p] = make_float2(0.f, 0.f);
  for (long long c0 = 0; c0 < dim; c0 += MV_CC) {
    __syncthreads();
    for (int t = threadIdx.x; t < NP * MV_CC; t += blockDim.x) {
      int p = t / MV_CC, cc = t % MV_CC;
      long long c = c0 + cc;
      double2 v = c < dim ? Q[p * qs + (long long)j * dim + c] : make_double2(0, 0);
      xs[p][cc] = make_float2((float)v.x, (float)v.y);
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < MV_RPW; r++) {
      const long long row = r0 + r;
      if (row >= dim) continue;
      const float2 *hr = H + row * dim + c0;
#pragma unroll
      for (int t = 0; t < MV_CC / 32; t++) {
        const int cc = lane + 32 * t;
        if (c0 + cc < dim) {
          const float2 h = __ldcs(hr + cc);
#pragma unroll
          for (int p = 0; p < NP; p++) {
            const float2 x = xs[p][cc];
            acc[r][p].x = fmaf(h.x, x.x, fmaf(-h.y, x.y, acc[r][p].x));
            acc[r][p].y = fmaf(h.x, x.y, fmaf(h.y, x.x, acc[r][p].y));
          }
        }
      }
    }
  }
#pragma unroll
  for (int r = 0; r < MV_RPW; r++)
#pragma unroll
    for (int p = 0; p < NP; p++) {
      double x = acc[r][p].x, y = acc[r][p].y;
      for (int o = 16; o > 0; o >>= 1) {
        x += __shfl_xor_sync(0xffffffffu, x, o);
        y += __shfl_xor_sync(0xffffffffu, y, o);
      }
      const long long row = r0 + r;
      if (lane == 0 && row < dim) W[(long long)p * dim + row] = make_double2(x, y);
    }
}


// ---- Hermitian half-read matvec (complex64 H) ---------------------------------------------
// H = H^dagger, so only tiles (bi <= bj) of HT x HT are read.  An off-diagonal tile
// gives y[bi] += H_t x[bj] and y[bj] += H_t^dagger x[bi]; a diagonal tile gives
// y[bi] += H_t x[bi].  Each contribution lands in its own slot part[target][source], and
// k_hmv_reduce sums the slots in a fixed order (deterministic, no atomics).
// 128 x 128 tiles, 4 warps of 32 rows; a lane owns columns {2f, 2f+1}, f = lane + 32 t.
constexpr int HT = 128;

// Sum over the 32 lanes of 32 values per lane with 31 shuffles; lane L returns the total of
// value index L.
__device__ __forceinline__ float warp_transpose_sum32(float (&v)[32], int lane) {
#pragma unroll
  for (int half = 16; half >= 1; half >>= 1) {
    const bool up = (lane & half) != 0;
#pragma unroll
    for (int i = 0; i < half; i++) {
      const float send = up ? v[i] : v[i + half];
      const float keep = up ? v[i + half] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, half);
    }
  }
  return v[0];
}

template <int NP>
__global__ void __launch_bounds__(128, 4) k_hmatvec_c64(const float2 *__restrict__ H, long long dim, int nb,
                                                        const float2 *__restrict__ Q32, long long qs, int j,
                                                        float2 *__restrict__ part, const int *meff) {
  static_assert(NP * 2 * 4 <= 32, "4 rows x NP polarisations x (re, im) per reduction group");
  const int bi = blockIdx.y, bj = blockIdx.x;
  if (bi > bj) return;
  bool live = false;
  for (int p = 0; p < NP; p++) live |= (j < meff[p]);
  if (!live) return;
  __shared__ float2 xr[NP][HT], xc[NP][HT];
  __shared__ float2 vs[4][HT][NP];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const long long r0 = (long long)bi * HT, c0 = (long long)bj * HT;
  for (int t = threadIdx.x; t < NP * HT; t += blockDim.x) {
    const int p = t / HT, l = t % HT;
    const float2 z = make_float2(0.f, 0.f);
    xr[p][l] = r0 + l < dim ? Q32[p * qs + (long long)j * dim + r0 + l] : z;
    xc[p][l] = c0 + l < dim ? Q32[p * qs + (long long)j * dim + c0 + l] : z;
  }
  __syncthreads();
  const bool diag = bi == bj;
  float2 v[4][NP];  // column partials for columns 2(lane + 32t) + {0,1}, t < 2
#pragma unroll
  for (int q = 0; q < 4; q++)
#pragma unroll
    for (int p = 0; p < NP; p++) v[q][p] = make_float2(0.f, 0.f);
  for (int g = 0; g < 8; g++) {  // 8 groups of 4 rows = the warp's 32 rows
    float4 h[4][2];
#pragma unroll
    for (int rr = 0; rr < 4; rr++) {
      const long long row = r0 + warp * 32 + g * 4 + rr;
#pragma unroll
      for (int t = 0; t < 2; t++) {
        const long long col = c0 + 2 * (lane + 32 * t);
        if (row < dim && col < dim)
          h[rr][t] = __ldcs(reinterpret_cast<const float4 *>(H + row * dim + col));
        else
          h[rr][t] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    float u[32];
#pragma unroll
    for (int i = 0; i < 32; i++) u[i] = 0.f;
#pragma unroll
    for (int rr = 0; rr < 4; rr++) {
      const int lr = warp * 32 + g * 4 + rr;
#pragma unroll
      for (int t = 0; t < 2; t++) {
        const int lc = 2 * (lane + 32 * t);
        const float4 hh = h[rr][t];
#pragma unroll
        for (int p = 0; p < NP; p++) {
          const float2 x0 = xc[p][lc], x1 = xc[p][lc + 1];
          u[(rr * NP + p) * 2 + 0] += hh.x * x0.x - hh.y * x0.y + hh.z * x1.x - hh.w * x1.y;
          u[(rr * NP + p) * 2 + 1] += hh.x * x0.y + hh.y * x0.x + hh.z * x1.y + hh.w * x1.x;
          if (!diag) {
            const float2 xrow = xr[p][lr];
            v[2 * t][p].x += hh.x * xrow.x + hh.y * xrow.y;
            v[2 * t][p].y += hh.x * xrow.y - hh.y * xrow.x;
            v[2 * t + 1][p].x += hh.z * xrow.x + hh.w * xrow.y;
            v[2 * t + 1][p].y += hh.z * xrow.y - hh.w * xrow.x;
          }
        }
      }
    }
    const float tot = warp_transpose_sum32(u, lane);
    if (lane < 4 * NP * 2) {
      const int rr = lane / (2 * NP), p = (lane / 2) % NP, ri = lane % 2;
      const int lr = warp * 32 + g * 4 + rr;
      float *dst = reinterpret_cast<float *>(part + (((long long)bi * nb + bj) * HT + lr) * NP + p);
      dst[ri] = tot;
    }
  }
  if (diag) return;
#pragma unroll
  for (int t = 0; t < 2; t++)
#pragma unroll
    for (int p = 0; p < NP; p++) {
      vs[warp][2 * (lane + 32 * t)][p] = v[2 * t][p];
      vs[warp][2 * (lane + 32 * t) + 1][p] = v[2 * t + 1][p];
    }
  __syncthreads();
  for (int e = threadIdx.x; e < HT * NP; e += blockDim.x) {
    const int l = e / NP, p = e % NP;
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int w = 0; w < 4; w++) {
      acc.x += vs[w][l][p].x;
      acc.y += vs[w][l][p].y;
    }
    part[(((long long)bj * nb + bi) * HT + l) * NP + p] = acc;
  }
}



// Launch with programmatic stream serialization: the kernel may be scheduled while its
// predecessor in the stream drains (hiding the launch latency of the Lanczos step's short
// kernels); every kernel launched this way opens with tc::griddep_wait().  Launch errors
// surface through cudaGetLastError as for <<<>>>.
template <typename... KArgs, typename... Args>
void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Packed FP32 pairs (Blackwell fma.rn.f32x2): one instruction performs two FP32 FMAs.
__device__ __forceinline__ unsigned long long pk2(float a, float b) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ float2 up2(unsigned long long v) {
  float a, b;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
  return make_float2(a, b);
}
__device__ __forceinline__ void ffma2(unsigned long long &acc, unsigned long long a, unsigned long long b) {
  asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc) : "l"(a), "l"(b));
}

// ---- TMA-fed Hermitian matvec (complex64 H), persistent ------------------------------------
// Same tiles and partial slots as k_hmatvec_c64.  Each CTA (four warps, no dedicated
// producer warp) walks its tiles in 16-row chunks through a shared-memory ring
// filled by TMA: the last of the four warps to copy its rows of a stage into registers refills
// it, so the other stages' chunks are in flight while one is computed (CTAs per SM and stages
// in HmvSmem).  A stage is 16 rows x 128 complex64 = 16 KB;
// rows/columns past dim arrive zero-filled.
constexpr int MV_CHUNK = 16, MV_STAGE_BYTES = MV_CHUNK * HT * 8;
constexpr long long MV_WAIT = 4000000000LL;

// Three CTAs per SM for up to three vectors; more vectors (the full-BSE product's four or six)
// need more registers: two CTAs.  (Four CTAs of 128 registers with two-stage rings measured
// the same 0.63 ms per 27648-dim product as three: not latency-bound by warp count.)
template <int NP>
struct HmvSmem {
  static constexpr int STAGES = 3;
  static constexpr int CTAS = NP <= 3 ? 3 : 2;
  static constexpr int RSTR = 8 * NP + 4;                 // floats per lane in the U-sum scratch
  static constexpr int XB = NP * HT * 24;                 // x vectors: (yr,-yr,yi,yi) + (xr,xi)
  static constexpr int USTR = (HT * NP * 8 > 32 * RSTR * 4) ? HT * NP * 8 : 32 * RSTR * 4;
  static constexpr int BYTES = 128 + STAGES * MV_STAGE_BYTES + XB + 4 * USTR;
};

// SYM = true: H is complex symmetric (H^T = H) instead of Hermitian; the mirrored tile then
// contributes H_t^T y, which only changes how the row vector y is parked for the column sums.
// More than three vectors (the full-BSE product's six) need more registers: two CTAs per SM.
template <int NP, bool SYM = false>
__global__ void __launch_bounds__(128, HmvSmem<NP>::CTAS) k_hmv_tma(const __grid_constant__ CUtensorMap tmH, long long dim,
                                                         int nb, const int2 *__restrict__ tiles, int ntiles,
                                                         const float2 *__restrict__ Q32, long long qs, int j,
                                                         float2 *__restrict__ part, const int *meff, int *err) {
  using S = HmvSmem<NP>;
  constexpr int MV_STAGES = S::STAGES;
  extern __shared__ __align__(128) uint8_t smv[];
  uint64_t *full = reinterpret_cast<uint64_t *>(smv);
  uint64_t *empty = full + MV_STAGES;
  int *taken = reinterpret_cast<int *>(empty + MV_STAGES);  // [MV_STAGES] warps done with a stage
  int *issued = taken + MV_STAGES;                           // chunks copied so far
  uint8_t *ring = smv + 128;
  float4 *yb = reinterpret_cast<float4 *>(ring + MV_STAGES * MV_STAGE_BYTES);  // [NP][HT] (yr,-yr,yi,yi)
  float2 *xc = reinterpret_cast<float2 *>(yb + NP * HT);                       // [NP][HT] (xr,xi)
  uint8_t *uni = reinterpret_cast<uint8_t *>(xc + NP * HT);  // per warp: U-sum scratch, then V partials
  tc::griddep_wait();
  tc::griddep_launch();
  bool live = false;
  for (int p = 0; p < NP; p++) live |= (j < meff[p]);
  if (!live) return;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (threadIdx.x == 0) {
    for (int st = 0; st < MV_STAGES; st++) {
      tc::mbar_init(&full[st], 1);
      tc::mbar_init(&empty[st], 4);
      taken[st] = 0;
    }
    *issued = 0;
    tc::fence_barrier_init();
  }
  __syncthreads();
  // ---- copies: chunk n of this CTA's sequence goes to stage n % MV_STAGES.  The first
  // MV_STAGES are issued here; afterwards the last warp to take a stage refills it ----
  constexpr int CPT = HT / MV_CHUNK;
  const int n_chunks = (ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x * CPT;
  auto issue = [&](int n, int2 tl) {
    const int st = n % MV_STAGES;
    tc::mbar_arrive_expect_tx(&full[st], MV_STAGE_BYTES);
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            tc::smem_u32(ring + st * MV_STAGE_BYTES)),
        "l"(reinterpret_cast<uint64_t>(&tmH)), "r"(2 * tl.y * HT), "r"(tl.x * HT + (n % CPT) * MV_CHUNK),
        "r"(tc::smem_u32(&full[st]))
        : "memory");
    atomicAdd(issued, 1);
  };
  if (threadIdx.x == 0) {
    tc::prefetch_tmap(&tmH);
    const int2 tl0 = tiles[blockIdx.x];
    for (int k = 0; k < MV_STAGES && k < n_chunks; k++) issue(k, tl0);
  }
  int it = 0;
  bool aborted = false;  // warp-uniform; after a timeout the warp runs on without waiting so that
                         // every named barrier below is still reached by all four warps
  // x vectors of the next tile are fetched into registers during the current one
  constexpr int XPT = (NP * HT + 127) / 128;
  float2 pre_r[XPT], pre_c[XPT];
  int2 tl_next = make_int2(0, 0);
#define HMV_FETCH(T)                                                                              \
  do {                                                                                            \
    tl_next = tiles[(T)];                                                                         \
    const long long r0 = (long long)tl_next.x * HT, c0 = (long long)tl_next.y * HT;              \
    _Pragma("unroll") for (int k = 0; k < XPT; k++) {                                             \
      const int e = threadIdx.x + 128 * k;                                                        \
      const int p = e / HT, l = e % HT;                                                           \
      const float2 z = make_float2(0.f, 0.f);                                                     \
      pre_r[k] = (e < NP * HT && r0 + l < dim) ? Q32[p * qs + (long long)j * dim + r0 + l] : z;   \
      pre_c[k] = (e < NP * HT && c0 + l < dim) ? Q32[p * qs + (long long)j * dim + c0 + l] : z;   \
    }                                                                                             \
  } while (0)
#define HMV_PARK()                                                                                \
  do {                                                                                            \
    _Pragma("unroll") for (int k = 0; k < XPT; k++) {                                             \
      const int e = threadIdx.x + 128 * k;                                                        \
      if (e < NP * HT) {                                                                          \
        yb[e] = SYM ? make_float4(pre_r[k].x, pre_r[k].x, -pre_r[k].y, pre_r[k].y)                \
                    : make_float4(pre_r[k].x, -pre_r[k].x, pre_r[k].y, pre_r[k].y);               \
        xc[e] = pre_c[k];                                                                         \
      }                                                                                           \
    }                                                                                             \
  } while (0)
  if (blockIdx.x < ntiles) {
    HMV_FETCH(blockIdx.x);
    HMV_PARK();
  }
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int bi = tl_next.x, bj = tl_next.y;
    const bool diag = bi == bj;
    asm volatile("bar.sync 1, 128;" ::: "memory");  // this tile's x vectors are parked
    const bool has_next = t + (int)gridDim.x < ntiles;
    if (has_next) HMV_FETCH(t + gridDim.x);
    // a lane owns columns 2f, 2f+1 (f = lane, lane + 32): x as (xr, xr) and (-xi, xi) pairs
    unsigned long long XA[4][NP], XB[4][NP], V[4][NP];
#pragma unroll
    for (int q = 0; q < 4; q++)
#pragma unroll
      for (int p = 0; p < NP; p++) {
        const float2 xv = xc[p * HT + 2 * (lane + 32 * (q / 2)) + (q % 2)];
        XA[q][p] = pk2(xv.x, xv.x);
        XB[q][p] = pk2(-xv.y, xv.y);
        V[q][p] = 0ull;
      }
    for (int c = 0; c < CPT; c++, it++) {
      const int st = it % MV_STAGES;
      bool ok = aborted ? false : tc::mbar_wait_bounded(&full[st], (it / MV_STAGES) & 1, MV_WAIT);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok && !aborted) {
        if (lane == 0) atomicOr(err, 2);
        aborted = true;
      }
      const float4 *rows = reinterpret_cast<const float4 *>(ring + st * MV_STAGE_BYTES);
      float4 h[4][2];
#pragma unroll
      for (int rr = 0; rr < 4; rr++)
#pragma unroll
        for (int tt = 0; tt < 2; tt++) h[rr][tt] = rows[(warp * 4 + rr) * (HT / 2) + lane + 32 * tt];
      __syncwarp();
      if (lane == 0 && !aborted) {
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(&empty[st])) : "memory");
        if (atomicAdd(&taken[st], 1) == 3) {
          // the last of the four warps to take chunk it out of stage st refills it with chunk
          // it + MV_STAGES (this tile's or the next one's), so no warp waits for the others
          atomicExch(&taken[st], 0);
          const int n = it + MV_STAGES;
          if (n < n_chunks) {
            if (tc::mbar_wait_bounded(&empty[st], (it / MV_STAGES) & 1, MV_WAIT))
              issue(n, n / CPT == it / CPT ? make_int2(bi, bj) : tl_next);
            else
              atomicOr(err, 2);
          }
        }
      }
      __syncwarp();
      // with hp = (hr, hi) as loaded and hs = (hi, hr):
      //   h x       = hp (xr, xr) + hs (-xi, xi)
      //   conj(h) y = hp (yr, -yr) + hs (yi, yi)      (Hermitian: the mirrored tile is H_t^dagger)
      //   h y       = hp (yr, yr) + hs (-yi, yi)      (SYM: the mirrored tile is H_t^T)
      unsigned long long U[4][NP];
#pragma unroll
      for (int rr = 0; rr < 4; rr++)
#pragma unroll
        for (int p = 0; p < NP; p++) U[rr][p] = 0ull;
#pragma unroll
      for (int rr = 0; rr < 4; rr++) {
        const int lr = c * MV_CHUNK + warp * 4 + rr;
        unsigned long long YA[NP], YB[NP];
        if (!diag) {
#pragma unroll
          for (int p = 0; p < NP; p++) {
            const float4 y = yb[p * HT + lr];
            YA[p] = pk2(y.x, y.y);
            YB[p] = pk2(y.z, y.w);
          }
        }
#pragma unroll
        for (int tt = 0; tt < 2; tt++) {
          const float4 hh = h[rr][tt];
#pragma unroll
          for (int e2 = 0; e2 < 2; e2++) {
            const float hre = e2 ? hh.z : hh.x, him = e2 ? hh.w : hh.y;
            const unsigned long long hp = pk2(hre, him), hs = pk2(him, hre);
            const int q = 2 * tt + e2;
#pragma unroll
            for (int p = 0; p < NP; p++) {
              ffma2(U[rr][p], hp, XA[q][p]);
              ffma2(U[rr][p], hs, XB[q][p]);
              if (!diag) {
                ffma2(V[q][p], hp, YA[p]);
                ffma2(V[q][p], hs, YB[p]);
              }
            }
          }
        }
      }
      // row sums of U over the 32 lanes through shared memory: each lane parks its 4*NP pairs,
      // lane L < 8*NP sums pair L % (4*NP) over 16 of the lanes, and the two halves are added
      {
        float *red = reinterpret_cast<float *>(uni + warp * S::USTR);
        float4 *mine = reinterpret_cast<float4 *>(red + lane * S::RSTR);
#pragma unroll
        for (int k = 0; k < 2 * NP; k++) {
          const int i0 = 2 * k, i1 = 2 * k + 1;
          const float2 a = up2(U[i0 / NP][i0 % NP]), b = up2(U[i1 / NP][i1 % NP]);
          mine[k] = make_float4(a.x, a.y, b.x, b.y);
        }
        __syncwarp();
        if constexpr (8 * NP <= 32) {
          const int i = lane % (4 * NP), g = lane / (4 * NP);
          unsigned long long s0 = 0ull, s1 = 0ull;
          const unsigned long long one = pk2(1.f, 1.f);
          if (lane < 8 * NP) {
            const float *src = red + 16 * g * S::RSTR + 2 * i;
#pragma unroll
            for (int k = 0; k < 16; k += 2) {
              const float2 v0 = *reinterpret_cast<const float2 *>(src + k * S::RSTR);
              const float2 v1 = *reinterpret_cast<const float2 *>(src + (k + 1) * S::RSTR);
              ffma2(s0, pk2(v0.x, v0.y), one);
              ffma2(s1, pk2(v1.x, v1.y), one);
            }
          }
          ffma2(s0, s1, one);
          float2 tot = up2(s0);
          tot.x += __shfl_down_sync(0xffffffffu, tot.x, 4 * NP);
          tot.y += __shfl_down_sync(0xffffffffu, tot.y, 4 * NP);
          if (lane < 4 * NP) {
            const int rr = i / NP, p = i % NP;
            const int lr = c * MV_CHUNK + warp * 4 + rr;
            part[(((long long)bi * nb + bj) * HT + lr) * NP + p] = tot;
          }
        } else {
          // more pairs (4 NP) than half-warps can cover: lane i < 4 NP sums pair i over all
          // 32 lanes in two interleaved chains
          for (int i = lane; i < 4 * NP; i += 32) {
            const float *src = red + 2 * i;
            unsigned long long s0 = 0ull, s1 = 0ull;
            const unsigned long long one = pk2(1.f, 1.f);
#pragma unroll
            for (int k = 0; k < 32; k += 2) {
              const float2 v0 = *reinterpret_cast<const float2 *>(src + k * S::RSTR);
              const float2 v1 = *reinterpret_cast<const float2 *>(src + (k + 1) * S::RSTR);
              ffma2(s0, pk2(v0.x, v0.y), one);
              ffma2(s1, pk2(v1.x, v1.y), one);
            }
            ffma2(s0, s1, one);
            const int rr = i / NP, p = i % NP;
            const int lr = c * MV_CHUNK + warp * 4 + rr;
            part[(((long long)bi * nb + bj) * HT + lr) * NP + p] = up2(s0);
          }
        }
        __syncwarp();
      }
    }
    if (!diag) {
      // column sums H_t^dagger y: the four warps' partials meet in shared memory
      float2 (*vs)[NP] = reinterpret_cast<float2 (*)[NP]>(uni + warp * S::USTR);
#pragma unroll
      for (int q = 0; q < 4; q++)
#pragma unroll
        for (int p = 0; p < NP; p++) vs[2 * (lane + 32 * (q / 2)) + (q % 2)][p] = up2(V[q][p]);
    }
    // every warp is past its last read of the x buffers (and, off the diagonal, has parked V)
    asm volatile("bar.sync 1, 128;" ::: "memory");
    if (!diag) {
      for (int e = threadIdx.x; e < HT * NP; e += 128) {
        const int l = e / NP, p = e % NP;
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int w = 0; w < 4; w++) {
          const float2 v = reinterpret_cast<const float2 (*)[NP]>(uni + w * S::USTR)[l][p];
          acc.x += v.x;
          acc.y += v.y;
        }
        part[(((long long)bj * nb + bi) * HT + l) * NP + p] = acc;
      }
    }
    if (has_next) HMV_PARK();  // visible after the next tile's opening barrier
  }
  // chunks copied but never consumed (only after a timeout) must land before the CTA exits
  asm volatile("bar.sync 1, 128;" ::: "memory");
  if (threadIdx.x == 0) {
    const int n_issued = *issued;
    for (int k = it; k < n_issued; k++)
      if (!tc::mbar_wait_bounded(&full[k % MV_STAGES], (k / MV_STAGES) & 1, MV_WAIT)) atomicOr(err, 2);
  }
}
#undef HMV_FETCH
#undef HMV_PARK

template <int NP>
constexpr int hmv_tma_smem() {
  return HmvSmem<NP>::BYTES;
}

// W[p][row] = sum_s part[t][s][row_local][p] for the rows of block t, and the block's share
// of alpha_j = Re(Q_j^H W) per polarisation (apart[p][t]).  Two threads per output stream
// the two halves of the block's slot slab; each keeps a compensated (Kahan) FP32 sum, so the
// result carries FP64-like accuracy without FP64 adds (B300's FP64 rate is ~1/60 of FP32),
// and the two halves meet in FP64 in a fixed order.
// HALVES = 1 (more than four vectors): one thread per output streams the whole slab.
template <int NP, int HALVES = 2>
__global__ void __launch_bounds__(HALVES * HT * NP, 1) k_hmv_reduce(const float2 *__restrict__ part, long long dim,
                                                                int nb, double2 *__restrict__ W,
                                                                const double2 *__restrict__ Q, long long qs, int j,
                                                                const int *__restrict__ meff, double *__restrict__ apart) {
  tc::griddep_wait();
  tc::griddep_launch();
  __shared__ double2 hs[HT * NP];
  __shared__ double av[HT * NP];
  const int t = blockIdx.x;
  const int o = threadIdx.x % (HT * NP), h = threadIdx.x / (HT * NP);
  const int l = o / NP, p = o % NP;
  const long long row = (long long)t * HT + l;
  const bool on = row < dim && j < meff[p];
  const int s0 = h ? nb / 2 : 0, s1 = (h || HALVES == 1) ? nb : nb / 2;
  // Kahan: sum + (-comp) is the running total; each add is y = v - comp; t = sum + y;
  // comp = (t - sum) - y; sum = t
  float sx = 0.f, cx = 0.f, sy = 0.f, cy = 0.f;
  if (on) {
    const float2 *src = part + ((long long)t * nb * HT + l) * NP + p;
    const long long step = (long long)HT * NP;
    int s = s0;
    for (; s + 8 <= s1; s += 8) {
      float2 v[8];
#pragma unroll
      for (int u = 0; u < 8; u++) v[u] = src[(s + u) * step];
#pragma unroll
      for (int u = 0; u < 8; u++) {
        const float yx = v[u].x - cx, tx = sx + yx;
        cx = (tx - sx) - yx;
        sx = tx;
        const float yy = v[u].y - cy, ty = sy + yy;
        cy = (ty - sy) - yy;
        sy = ty;
      }
    }
    for (; s < s1; s++) {
      const float2 v = src[s * step];
      const float yx = v.x - cx, tx = sx + yx;
      cx = (tx - sx) - yx;
      sx = tx;
      const float yy = v.y - cy, ty = sy + yy;
      cy = (ty - sy) - yy;
      sy = ty;
    }
  }
  double tx = (double)sx - (double)cx, ty = (double)sy - (double)cy;
  if (h) hs[o] = make_double2(tx, ty);
  __syncthreads();
  if (!h) {
    double ar = 0.0;
    if (on) {
      if (HALVES == 2) {
        tx += hs[o].x;
        ty += hs[o].y;
      }
      W[(long long)p * dim + row] = make_double2(tx, ty);
      const double2 q = Q[p * qs + (long long)j * dim + row];
      ar = q.x * tx + q.y * ty;
    }
    av[o] = ar;
  }
  __syncthreads();
  if (threadIdx.x < NP) {
    double sa = 0.0;
    for (int ll = 0; ll < HT; ll++) sa += av[ll * NP + threadIdx.x];
    apart[threadIdx.x * nb + t] = sa;
  }
}

// Block sum returned to every thread (tree order fixed by NT).
template <int NT>
__device__ __forceinline__ double block_sum_all(double v, double *red, double *out) {
  v = block_sum<NT>(v, red);
  if (threadIdx.x == 0) *out = v;
  __syncthreads();
  return *out;
}

// apart[p][t] = sum of Re(conj(Q_j) W) over rows of block t (matvec paths that write W directly)
__global__ void k_alpha_part(const double2 *__restrict__ W, long long dim, const double2 *__restrict__ Q,
                             long long qs, int j, const int *__restrict__ meff, int nb, double *__restrict__ apart) {
  __shared__ double red[32];
  const int t = blockIdx.x, p = blockIdx.y;
  const long long row = (long long)t * HT + threadIdx.x;
  double ar = 0.0;
  if (row < dim && j < meff[p]) {
    const double2 w = W[(long long)p * dim + row], q = Q[p * qs + (long long)j * dim + row];
    ar = q.x * w.x + q.y * w.y;
  }
  ar = block_sum<HT>(ar, red);
  if (threadIdx.x == 0) apart[p * nb + t] = ar;
}

// Per 128-row block sums of v (one value per thread, blockDim = 256, rows in thread order):
// out[2 blockIdx.x + h] for the block's two halves h (those below nb).
__device__ __forceinline__ void half_block_sums(double v, double *red, double *out, int nb) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = v;
  __syncthreads();
  if (threadIdx.x < 2 && 2 * (int)blockIdx.x + (int)threadIdx.x < nb) {
    const double *r = red + 4 * threadIdx.x;
    out[2 * blockIdx.x + threadIdx.x] = ((r[0] + r[1]) + r[2]) + r[3];
  }
}

// alpha_j = sum_t apart[p][t] (same order in every block); W -= alpha_j Q_j + b_{j-1} Q_{j-1};
// with n0part, also the per-row-block sums of |W|^2 of the result (n0part[p][t]).
__global__ void __launch_bounds__(256) k_axpy(double2 *__restrict__ W, long long dim, const double2 *__restrict__ Q,
                                              long long qs, int j, double *__restrict__ a, const double *__restrict__ b,
                                              int ldab, const int *__restrict__ meff, int nb,
                                              const double *__restrict__ apart, double *__restrict__ n0part) {
  tc::griddep_wait();
  tc::griddep_launch();
  __shared__ double red[32];
  __shared__ double sa;
  const int p = blockIdx.y;
  if (j >= meff[p]) return;
  double s = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) s += apart[p * nb + i];
  const double aj = block_sum_all<256>(s, red, &sa);
  if (blockIdx.x == 0 && threadIdx.x == 0) a[p * ldab + j] = aj;
  const double bj = j > 0 ? b[p * ldab + j - 1] : 0.0;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double nv = 0.0;
  if (e < dim) {
    const double2 *qj = Q + p * qs + (long long)j * dim;
    const double2 *qm = j > 0 ? qj - dim : qj;
    double2 v = W[(long long)p * dim + e];
    const double2 x = qj[e], y = qm[e];
    v.x -= aj * x.x + bj * y.x;
    v.y -= aj * x.y + bj * y.y;
    W[(long long)p * dim + e] = v;
    nv = v.x * v.x + v.y * v.y;
  }
  if (n0part) half_block_sums(nv, red, n0part + (long long)p * nb, nb);
}

// npart[p][t] = sum over the rows of block t of |W|^2
__global__ void k_norm_part(const double2 *__restrict__ W, long long dim, int j, const int *__restrict__ meff, int nb,
                            double *__restrict__ npart) {
  tc::griddep_wait();
  tc::griddep_launch();
  __shared__ double red[32];
  const int t = blockIdx.x, p = blockIdx.y;
  const long long row = (long long)t * HT + threadIdx.x;
  double v = 0.0;
  if (row < dim && j < meff[p]) {
    const double2 w = W[(long long)p * dim + row];
    v = w.x * w.x + w.y * w.y;
  }
  v = block_sum<HT>(v, red);
  if (threadIdx.x == 0) npart[p * nb + t] = v;
}

// b[p][j] = |W| from the partials (same order in every block); Q[p][j+1] = W / b (and its FP32
// shadow); early stop when b < 1e-14 max|H|.
__global__ void __launch_bounds__(256) k_scale(const double2 *__restrict__ W, long long dim, double2 *__restrict__ Q,
                                               long long qs, int j, double *__restrict__ b, int ldab, int *meff,
                                               const double *__restrict__ hmax, int n_steps, float2 *__restrict__ Q32,
                                               int nb, const double *__restrict__ npart) {
  tc::griddep_wait();
  tc::griddep_launch();
  __shared__ double red[32];
  __shared__ double sb;
  const int p = blockIdx.y;
  if (j >= meff[p]) return;
  double s = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) s += npart[p * nb + i];
  const double bj = sqrt(block_sum_all<256>(s, red, &sb));
  if (blockIdx.x == 0 && threadIdx.x == 0) b[p * ldab + j] = bj;
  if (j == n_steps - 1) return;
  if (bj < 1e-14 * hmax[0]) {
    if (blockIdx.x == 0 && threadIdx.x == 0) meff[p] = j + 1;
    return;
  }
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= dim) return;
  const double inv = 1.0 / bj;
  const double2 w = W[(long long)p * dim + e];
  const double2 v = make_double2(w.x * inv, w.y * inv);
  Q[p * qs + (long long)(j + 1) * dim + e] = v;
  if (Q32) Q32[p * qs + (long long)(j + 1) * dim + e] = make_float2((float)v.x, (float)v.y);
}

// coef[p][i] = Q_i^H W, i <= j   (grid: x = i, y = p)
__global__ void k_reorth_dots(const double2 *W, long long dim, const double2 *Q, long long qs, int j,
                              double2 *coef, int ldc, const int *meff) {
  __shared__ double red[32];
  const int i = blockIdx.x, p = blockIdx.y;
  if (j >= meff[p] || i > j) return;
  const double2 *w = W + (long long)p * dim;
  const double2 *qi = Q + p * qs + (long long)i * dim;
  double sr = 0.0, si = 0.0;
  for (long long e = threadIdx.x; e < dim; e += blockDim.x) {
    const double2 q = qi[e], v = w[e];
    sr += q.x * v.x + q.y * v.y;
    si += q.x * v.y - q.y * v.x;
  }
  sr = block_sum<256>(sr, red);
  __syncthreads();
  si = block_sum<256>(si, red);
  if (threadIdx.x == 0) coef[p * ldc + i] = make_double2(sr, si);
}

// W -= sum_{i<=j} coef_i Q_i   (grid: x over elements, y = p)
__global__ void k_reorth_update(double2 *W, long long dim, const double2 *Q, long long qs, int j,
                                const double2 *coef, int ldc, const int *meff) {
  const int p = blockIdx.y;
  if (j >= meff[p]) return;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= dim) return;
  const double2 *qp = Q + p * qs + e;
  const double2 *cp = coef + p * ldc;
  double2 v = W[(long long)p * dim + e];
  for (int i = 0; i <= j; i++) {
    const double2 c = cp[i], q = qp[(long long)i * dim];
    v.x -= c.x * q.x - c.y * q.y;
    v.y -= c.x * q.y + c.y * q.x;
  }
  W[(long long)p * dim + e] = v;
}

// FP32 projections for a complex64 H: coef[p][i] = Q32_i^H W (FP32 products and per-thread
// sums, FP64 block reduction); the correction sum_i coef_i Q32_i is formed in FP32 and
// subtracted from the FP64 vector.  W is already nearly orthogonal to the basis, so the
// FP32 relative error lands on a small correction.


// Chunked projections for the complex64 path: block (chunk, p, row group) stages 256
// elements of W once (FP32) and its warps stream 4 basis rows at a time over the chunk,
// issuing all 16 float4 loads of a pass before the first use; the per-row sums over the
// 32 lanes are one butterfly transpose.  Writes the chunk partial of Q32_i^H W to
// partial[p][i][chunk]; k_reorth_coef sums the chunk partials in FP64.  Needs an even dim (float4 = 2 elements).
constexpr int RCH = 256, RROWS = 64, RPW = 4;

template <int N>
__device__ __forceinline__ float warp_transpose_sum(float (&v)[N], int lane) {
  int bit = 16;
#pragma unroll
  for (int half = N / 2; half >= 1; half >>= 1, bit >>= 1) {
    const bool up = (lane & bit) != 0;
#pragma unroll
    for (int i = 0; i < half; i++) {
      const float send = up ? v[i] : v[i + half];
      const float keep = up ? v[i + half] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, bit);
    }
  }
  for (; bit >= 1; bit >>= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], bit);
  return v[0];  // lane L holds the total of value L / (32 / N)
}

__global__ void __launch_bounds__(256, 2) k_reorth_dots_chunk(const double2 *__restrict__ W, long long dim,
                                                              const float2 *__restrict__ Q32, long long qs, int j,
                                                              float2 *__restrict__ partial, int nchunk, int ldp,
                                                              const int *__restrict__ meff) {
  tc::griddep_wait();
  tc::griddep_launch();
  __shared__ float4 ws[RCH / 2];
  const int chunk = blockIdx.x, p = blockIdx.y;
  if (j >= meff[p]) return;
  const int ib = blockIdx.z * RROWS;
  if (ib > j) return;
  const int ie = min(j, ib + RROWS - 1);
  const long long e0 = (long long)chunk * RCH;
  for (int t = threadIdx.x; t < RCH / 2; t += blockDim.x) {
    const long long e = e0 + 2 * t;
    float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
    if (e < dim) {
      const double2 a = W[(long long)p * dim + e], b = W[(long long)p * dim + e + 1];
      w = make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
    }
    ws[t] = w;
  }
  __syncthreads();
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const float4 *qp = reinterpret_cast<const float4 *>(Q32 + p * qs + e0);
  const long long rs = dim / 2;
  for (int i0 = ib + RPW * warp; i0 <= ie; i0 += RPW * 8) {
    float4 q[RPW][RCH / 64];
#pragma unroll
    for (int r = 0; r < RPW; r++) {
      const int row = min(i0 + r, ie);  // rows past ie repeat row ie; their sums are dropped
#pragma unroll
      for (int t = 0; t < RCH / 64; t++) {
        const int f = lane + 32 * t;
        q[r][t] = (e0 + 2 * f < dim) ? __ldg(qp + (long long)row * rs + f) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    float v[2 * RPW];
#pragma unroll
    for (int r = 0; r < 2 * RPW; r++) v[r] = 0.f;
#pragma unroll
    for (int t = 0; t < RCH / 64; t++) {
      const float4 w = ws[lane + 32 * t];
#pragma unroll
      for (int r = 0; r < RPW; r++) {
        const float4 a = q[r][t];  // conj(q) w for two elements
        v[2 * r] = fmaf(a.x, w.x, fmaf(a.y, w.y, fmaf(a.z, w.z, fmaf(a.w, w.w, v[2 * r]))));
        v[2 * r + 1] = fmaf(a.x, w.y, fmaf(-a.y, w.x, fmaf(a.z, w.w, fmaf(-a.w, w.z, v[2 * r + 1]))));
      }
    }
    const float tot = warp_transpose_sum<2 * RPW>(v, lane);
    constexpr int G = 32 / (2 * RPW);
    if (lane % G == 0) {
      const int idx = lane / G, r = idx / 2;
      if (i0 + r <= ie)
        reinterpret_cast<float *>(partial + ((long long)p * ldp + i0 + r) * nchunk + chunk)[idx % 2] = tot;
    }
  }
}

// coef[p][i] = sum over chunks of partial[p][i][chunk] (FP64): one warp per (i, p)
__global__ void __launch_bounds__(256) k_reorth_coef(const float2 *__restrict__ partial, int nchunk, int ldp, int j,
                                                     double2 *__restrict__ coef, int ldc, const int *__restrict__ meff) {
  tc::griddep_wait();
  tc::griddep_launch();
  const int i = blockIdx.x * 8 + threadIdx.x / 32, lane = threadIdx.x % 32, p = blockIdx.y;
  if (j >= meff[p] || i > j) return;
  const float2 *src = partial + ((long long)p * ldp + i) * nchunk;
  double sr = 0.0, si = 0.0;
  for (int c = lane; c < nchunk; c += 32) {
    const float2 v = src[c];
    sr += v.x;
    si += v.y;
  }
  for (int o = 16; o > 0; o >>= 1) {
    sr += __shfl_xor_sync(0xffffffffu, sr, o);
    si += __shfl_xor_sync(0xffffffffu, si, o);
  }
  if (lane == 0) coef[p * ldc + i] = make_double2(sr, si);
}

// W -= sum_i coef_i Q32_i for two elements per thread (float4 loads, 16 basis rows in flight
// per thread); FP32 products and sums, subtracted from the FP64 vector.  Needs an even dim.
// With npart, also the per-row-block sums of |W|^2 of the result (npart[p][t], four 128-row
// blocks per 256-thread block).
constexpr int RUN = 16;
__global__ void __launch_bounds__(256, 2) k_reorth_update32(double2 *__restrict__ W, long long dim,
                                                            const float2 *__restrict__ Q32, long long qs, int j,
                                                            const double2 *__restrict__ coef, int ldc,
                                                            const int *__restrict__ meff, int nb,
                                                            double *__restrict__ npart) {
  tc::griddep_wait();
  tc::griddep_launch();
  __shared__ float2 cs[1024];
  const int p = blockIdx.y;
  if (j >= meff[p]) return;
  const long long e = 2 * ((long long)blockIdx.x * blockDim.x + threadIdx.x);
  const bool in = e < dim;
  const float4 *qp = reinterpret_cast<const float4 *>(Q32 + p * qs + e);
  const long long rs = dim / 2;
  float a0r = 0.f, a0i = 0.f, a1r = 0.f, a1i = 0.f;
  // basis rows are taken from j down to 0: the dots pass that precedes this one read them
  // upwards, so its most recent rows (the ones still in L2) come first here
  for (int i0 = (j / 1024) * 1024; i0 >= 0; i0 -= 1024) {
    const int n = min(1024, j + 1 - i0);
    __syncthreads();
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
      const double2 c = coef[p * ldc + i0 + t];
      cs[t] = make_float2((float)c.x, (float)c.y);
    }
    __syncthreads();
    if (in) {
      int i = n;
      for (; i >= RUN; i -= RUN) {
        float4 q[RUN];
#pragma unroll
        for (int u = 0; u < RUN; u++) q[u] = __ldg(qp + (long long)(i0 + i - 1 - u) * rs);
#pragma unroll
        for (int u = 0; u < RUN; u++) {
          const float2 c = cs[i - 1 - u];
          a0r = fmaf(c.x, q[u].x, fmaf(-c.y, q[u].y, a0r));
          a0i = fmaf(c.x, q[u].y, fmaf(c.y, q[u].x, a0i));
          a1r = fmaf(c.x, q[u].z, fmaf(-c.y, q[u].w, a1r));
          a1i = fmaf(c.x, q[u].w, fmaf(c.y, q[u].z, a1i));
        }
      }
      while (i > 0) {
        i--;
        const float2 c = cs[i];
        const float4 q = __ldg(qp + (long long)(i0 + i) * rs);
        a0r = fmaf(c.x, q.x, fmaf(-c.y, q.y, a0r));
        a0i = fmaf(c.x, q.y, fmaf(c.y, q.x, a0i));
        a1r = fmaf(c.x, q.z, fmaf(-c.y, q.w, a1r));
        a1i = fmaf(c.x, q.w, fmaf(c.y, q.z, a1i));
      }
    }
  }
  double nv = 0.0;
  if (in) {
    double2 *wp = W + (long long)p * dim + e;
    double2 v0 = wp[0], v1 = wp[1];
    v0.x -= (double)a0r;
    v0.y -= (double)a0i;
    v1.x -= (double)a1r;
    v1.y -= (double)a1i;
    wp[0] = v0;
    wp[1] = v1;
    nv = (v0.x * v0.x + v0.y * v0.y) + (v1.x * v1.x + v1.y * v1.y);
  }
  if (npart) {
    __shared__ double red[8];
    for (int o = 16; o > 0; o >>= 1) nv += __shfl_xor_sync(0xffffffffu, nv, o);
    if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = nv;
    __syncthreads();
    const int t = 4 * blockIdx.x + threadIdx.x;  // 128-row block of warps 2 threadIdx.x, +1
    if (threadIdx.x < 4 && t < nb) npart[(long long)p * nb + t] = red[2 * threadIdx.x] + red[2 * threadIdx.x + 1];
  }
}


// eps2[w] = pref * sum_p -(1/pi) Im( beta0^2 / (z - a1 - b1^2/(z - a2 - ...)) )
__global__ void k_contfrac(const double *a, const double *b, int ldab, const double *beta0, const int *meff,
                           int n_pol, const double *omega, int n_w, double eta, double pref, double *eps2,
                           int accumulate) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= n_w) return;
  const double zr = omega[w], zi = eta;
  double tot = 0.0;
  for (int p = 0; p < n_pol; p++) {
    const int m = meff[p];
    const double *ap = a + p * ldab, *bp = b + p * ldab;
    double fr = zr - ap[m - 1], fi = zi;
    for (int jj = m - 2; jj >= 0; jj--) {
      const double d = fr * fr + fi * fi, bb = bp[jj] * bp[jj];
      // f = z - a_jj - bb / f
      const double qr = bb * fr / d, qi = -bb * fi / d;
      fr = zr - ap[jj] - qr;
      fi = zi - qi;
    }
    const double d = fr * fr + fi * fi, b0 = beta0[p] * beta0[p];
    const double gi = -b0 * fi / d;  // Im(b0 / f)
    tot += -gi / M_PI;
  }
  eps2[w] = accumulate ? eps2[w] + pref * tot : pref * tot;
}

__global__ void k_pack_ab(const double *a, const double *b, const double *beta0, int ldab, int n_pol,
                          int n_steps, double *ab) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x, p = blockIdx.y;
  if (j >= n_steps || p >= n_pol) return;
  ab[((long long)p * 3 + 0) * n_steps + j] = a[p * ldab + j];
  ab[((long long)p * 3 + 1) * n_steps + j] = b[p * ldab + j];
  ab[((long long)p * 3 + 2) * n_steps + j] = j == 0 ? beta0[p] : 0.0;
}

__global__ void k_fill_meff(int *meff, int n_pol, int n_steps, double *a, double *b, int ldab) {
  const int p = blockIdx.x;
  for (int j = threadIdx.x; j < ldab; j += blockDim.x) {
    a[p * ldab + j] = 0.0;
    b[p * ldab + j] = 0.0;
  }
  if (threadIdx.x == 0 && p < n_pol) meff[p] = n_steps;
}

// SplitMix64 (Steele, Lea, Flood 2014) -> uniform doubles -> a complex start vector.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}
__global__ void k_random_start(double2 *u, long long dim, unsigned long long seed) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= dim) return;
  const unsigned long long r1 = splitmix64(seed ^ (2ull * (unsigned long long)i));
  const unsigned long long r2 = splitmix64(seed ^ (2ull * (unsigned long long)i + 1ull));
  u[i] = make_double2((double)(r1 >> 11) * (1.0 / 9007199254740992.0) - 0.5,
                      (double)(r2 >> 11) * (1.0 / 9007199254740992.0) - 0.5);
}

// Lowest Ritz values of the m x m tridiagonal (a, b) by Sturm-sequence bisection, and the
// Lanczos residual |b_m s_m| from an inverse-iteration eigenvector (one thread each).
__device__ int sturm_count(const double *a, const double *b, int m, double x) {
  int cnt = 0;
  double d = 1.0;
  for (int i = 0; i < m; i++) {
    const double bb = i > 0 ? b[i - 1] * b[i - 1] : 0.0;
    d = (a[i] - x) - (i > 0 ? bb / d : 0.0);
    if (d == 0.0) d = -1e-300;
    if (d < 0.0) cnt++;
  }
  return cnt;
}
__global__ void k_ritz(const double *a, const double *b, const int *meff, int n_eig, double *omega,
                       double *resid, double *work) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_eig) return;
  const int m = meff[0];
  if (e >= m) {
    omega[e] = NAN;
    if (resid) resid[e] = NAN;
    return;
  }
  double lo = 1e300, hi = -1e300;
  for (int i = 0; i < m; i++) {
    const double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i < m - 1 ? fabs(b[i]) : 0.0);
    lo = fmin(lo, a[i] - r);
    hi = fmax(hi, a[i] + r);
  }
  for (int it = 0; it < 200; it++) {
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (sturm_count(a, b, m, mid) >= e + 1) hi = mid; else lo = mid;
  }
  const double th = hi;
  omega[e] = th;
  if (!resid) return;
  // inverse iteration (T - th I) v = rhs, Thomas algorithm, two sweeps
  double *v = work + (long long)e * 3 * m, *cp = v + m, *dp = cp + m;
  const double scale = fmax(fabs(lo), fabs(hi)) + 1.0;
  const double shift = th + 1e-13 * scale;
  for (int i = 0; i < m; i++) v[i] = 1.0;
  for (int sweep = 0; sweep < 3; sweep++) {
    double piv = a[0] - shift;
    if (piv == 0.0) piv = 1e-300;
    cp[0] = m > 1 ? b[0] / piv : 0.0;
    dp[0] = v[0] / piv;
    for (int i = 1; i < m; i++) {
      piv = (a[i] - shift) - b[i - 1] * cp[i - 1];
      if (piv == 0.0) piv = 1e-300;
      cp[i] = i < m - 1 ? b[i] / piv : 0.0;
      dp[i] = (v[i] - b[i - 1] * dp[i - 1]) / piv;
    }
    v[m - 1] = dp[m - 1];
    for (int i = m - 2; i >= 0; i--) v[i] = dp[i] - cp[i] * v[i + 1];
    double nrm = 0.0;
    for (int i = 0; i < m; i++) nrm += v[i] * v[i];
    nrm = sqrt(nrm);
    for (int i = 0; i < m; i++) v[i] /= nrm;
  }
  resid[e] = fabs(b[m - 1] * v[m - 1]);
}

bool encode_rows_f32(CUtensorMap *m, const void *base, unsigned long long inner, unsigned long long rows,
                     unsigned box_inner, unsigned box_rows) {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return false;
    fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  cuuint64_t dims[2] = {inner, rows};
  cuuint64_t strides[1] = {inner * 4};
  cuuint32_t box[2] = {box_inner, box_rows};
  cuuint32_t es[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Second reorthogonalisation pass only where it is needed (Daniel, Gragg, Kaufman and Stewart
// 1976): when the first pass left more than half of the squared norm, |W'|^2 > |W|^2 / 2, W' is
// orthogonal to the basis to working accuracy and a second pass would change nothing, so
// meff2[p] = 0 makes the pass-two kernels skip polarisation p; otherwise meff2[p] = meff[p].
__global__ void k_dgks(const double *__restrict__ n0part, const double *__restrict__ n1part, int nb,
                       const int *__restrict__ meff, int *__restrict__ meff2) {
  tc::griddep_wait();
  tc::griddep_launch();
  __shared__ double r0[32], r1[32];
  const int p = blockIdx.x;
  double a0 = 0.0, a1 = 0.0;
  for (int i = threadIdx.x; i < nb; i += 32) {
    a0 += n0part[p * nb + i];
    a1 += n1part[p * nb + i];
  }
  r0[threadIdx.x] = a0;
  r1[threadIdx.x] = a1;
  __syncwarp();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0;
    for (int i = 0; i < 32; i++) {
      s0 += r0[i];
      s1 += r1[i];
    }
    meff2[p] = (s1 > 0.5 * s0) ? 0 : meff[p];
  }
}

// Upper-triangle tile list of the half-read matvec, (bi, bj) for bj >= bi in row order, written
// on the device (no host copy, no stream synchronisation): thread bi writes its row, which
// starts at bi nbt - bi (bi - 1) / 2.
__global__ void k_fill_tiles(int nbt, int2 *__restrict__ tiles) {
  const int bi = blockIdx.x * blockDim.x + threadIdx.x;
  if (bi >= nbt) return;
  const long long off = (long long)bi * nbt - (long long)bi * (bi - 1) / 2;
  for (int bj = bi; bj < nbt; bj++) tiles[off + bj - bi] = make_int2(bi, bj);
}

void fill_tiles(bse_ctx *c, int nbt, int2 *tiles) {
  k_fill_tiles<<<(nbt + 127) / 128, 128, 0, c->stream>>>(nbt, tiles);
  bse_count_launch();
}

struct LanczosScratch {
  double2 *Q = nullptr, *W = nullptr, *coef = nullptr;
  float2 *Q32 = nullptr;  // FP32 shadow of Q (complex64 H only): reorthogonalisation projections
  float2 *hpart = nullptr; // Hermitian matvec partials [nb][nb][HT][n_pol]
  int nbt = 0;
  int2 *tiles = nullptr;    // upper-triangle tile list for the TMA matvec
  float2 *rpart = nullptr;  // chunk partials of the reorthogonalisation projections
  int nrch = 0;
  int ntiles = 0;
  CUtensorMap tmH;
  bool tma = false;
  double *a = nullptr, *b = nullptr, *beta0 = nullptr, *hmax = nullptr, *part = nullptr;
  double *apart = nullptr, *npart = nullptr;  // per-row-block partials of alpha_j and |W|^2
  double *n0part = nullptr;  // |W|^2 partials before the first reorthogonalisation pass
  int *meff = nullptr;
  int *meff2 = nullptr;      // meff for the second pass, 0 where the DGKS test skips it
};

bse_status lanczos_alloc(bse_ctx *c, LanczosScratch &s, int n_pol, int n_steps, bool matfree = false) {
  const long long dim = c->dim;
  // FP32 shadow basis and half-read products for a complex64 H (and the matrix-free product)
  const bool c64 = matfree || !c->h64;
  const size_t qbytes = sizeof(double2) * (size_t)n_pol * (n_steps + 1) * dim;
  cudaStream_t st = c->stream;
  if (cudaMallocAsync((void **)&s.Q, qbytes, st) != cudaSuccess ||
      cudaMallocAsync((void **)&s.W, sizeof(double2) * n_pol * dim, st) != cudaSuccess ||
      cudaMallocAsync((void **)&s.coef, sizeof(double2) * n_pol * (n_steps + 1), st) != cudaSuccess ||
      cudaMallocAsync((void **)&s.a, sizeof(double) * n_pol * (n_steps + 1), st) != cudaSuccess ||
      cudaMallocAsync((void **)&s.b, sizeof(double) * n_pol * (n_steps + 1), st) != cudaSuccess ||
      cudaMallocAsync((void **)&s.beta0, sizeof(double) * n_pol, st) != cudaSuccess ||
      cudaMallocAsync((void **)&s.hmax, sizeof(double), st) != cudaSuccess ||
      cudaMallocAsync((void **)&s.part, sizeof(double) * 1024, st) != cudaSuccess ||
      cudaMallocAsync((void **)&s.meff, sizeof(int) * n_pol, st) != cudaSuccess ||
      cudaMallocAsync((void **)&s.apart, sizeof(double) * 3 * n_pol * ((dim + HT - 1) / HT), st) != cudaSuccess ||
      cudaMallocAsync((void **)&s.meff2, sizeof(int) * n_pol, st) != cudaSuccess ||
      (c64 &&
       cudaMallocAsync((void **)&s.Q32, qbytes / 2, st) != cudaSuccess)) {
    cudaGetLastError();
    return bse_fail(c, BSE_ENOMEM, "spectrum: Krylov scratch allocation failed");
  }
  s.nbt = (int)((dim + HT - 1) / HT);
  s.npart = s.apart + (size_t)n_pol * s.nbt;
  s.n0part = s.npart + (size_t)n_pol * s.nbt;
  s.nrch = (int)((dim + RCH - 1) / RCH);
  if (c64 &&
      cudaMallocAsync((void **)&s.rpart, sizeof(float2) * (size_t)n_pol * s.nrch * (n_steps + 1), st) != cudaSuccess) {
    cudaGetLastError();
    return bse_fail(c, BSE_ENOMEM, "spectrum: reorthogonalisation scratch allocation failed");
  }
  if (c64 && dim % 2 == 0 && !matfree) {
    if (cudaMallocAsync((void **)&s.hpart, sizeof(float2) * (size_t)s.nbt * s.nbt * HT * n_pol, st) != cudaSuccess) {
      cudaGetLastError();
      return bse_fail(c, BSE_ENOMEM, "spectrum: Krylov scratch allocation failed");
    }
    s.ntiles = s.nbt * (s.nbt + 1) / 2;
    if (cudaMallocAsync((void **)&s.tiles, sizeof(int2) * s.ntiles, st) != cudaSuccess) {
      cudaGetLastError();
      return bse_fail(c, BSE_ENOMEM, "spectrum: tile list allocation failed");
    }
    fill_tiles(c, s.nbt, s.tiles);
  }
  return BSE_OK;
}

void lanczos_release(bse_ctx *c, LanczosScratch &s) {
  void *ptrs[] = {s.Q, s.W, s.coef, s.a, s.b, s.beta0, s.hmax, s.part, s.meff, s.meff2, s.apart, s.Q32, s.hpart,
                  s.tiles, s.rpart};
  for (void *p : ptrs)
    if (p) cudaFreeAsync(p, c->stream);
}

// Runs the recursion; a, b, beta0, meff are left in s.  H == nullptr: the matrix-free product
// (split precisions; H x recomputed from the pair tables each step).
bse_status lanczos_run(bse_ctx *c, LanczosScratch &s, const void *H, const double2 *u, int n_pol,
                       int n_steps) {
  const bool matfree = H == nullptr;
  const long long dim = c->dim;
  const long long qs = (long long)(n_steps + 1) * dim;
  const int ldab = n_steps + 1;
  cudaStream_t st = c->stream;
  const bool c64 = matfree || !c->h64;  // complex64 H (or the matrix-free product)
  if (c64 && s.hpart && s.tiles) {
    s.tma = encode_rows_f32(&s.tmH, H, 2ull * dim, (unsigned long long)dim, 2 * HT, MV_CHUNK);
    if (s.tma)
      bse_once_per_device(c, BSE_ONCE_HMV_TDA, [] {
        cudaFuncSetAttribute(k_hmv_tma<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, hmv_tma_smem<1>());
        cudaFuncSetAttribute(k_hmv_tma<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, hmv_tma_smem<2>());
        cudaFuncSetAttribute(k_hmv_tma<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, hmv_tma_smem<3>());
      });
  }
  // max |H| (matrix-free: twice the largest band energy)
  if (matfree) {
    bse_status rr = split_matfree_hmax(c, s.hmax);
    if (rr != BSE_OK) return rr;
  } else {
    if (c64)
      k_absmax_part<float2><<<1024, 256, 0, st>>>((const float2 *)H, dim * dim, s.part);
    else
      k_absmax_part<double2><<<1024, 256, 0, st>>>((const double2 *)H, dim * dim, s.part);
    k_absmax_final<<<1, 32, 0, st>>>(s.part, 1024, s.hmax);
  }
  k_fill_meff<<<n_pol, 256, 0, st>>>(s.meff, n_pol, n_steps, s.a, s.b, ldab);
  k_lanczos_init<<<n_pol, 1024, 0, st>>>(u, dim, s.Q, qs, s.beta0, s.Q32);
  bse_count_launch(4);
  bse_status r = bse_check_launch(c, "lanczos init");
  if (r != BSE_OK) return r;
  const unsigned mv_blocks = (unsigned)((dim + MV_ROWS - 1) / MV_ROWS);
  const unsigned el_blocks = (unsigned)((dim + 255) / 256);
  const unsigned el2_blocks = (unsigned)((dim / 2 + 255) / 256);
  for (int j = 0; j < n_steps; j++) {
    bse_prof_begin(c, BSE_KP_MATVEC);
    if (matfree) {
      r = split_matvec_free(c, s.Q + (long long)j * dim, qs, n_pol, s.W);
      if (r != BSE_OK) return r;
    } else if (c64 && s.tma) {
      const int grid = std::min(s.ntiles, HmvSmem<3>::CTAS * c->n_sm);
      if (n_pol == 1) {
        launch_pdl(k_hmv_tma<1>, dim3(grid), dim3(128), hmv_tma_smem<1>(), st, s.tmH, dim, s.nbt, s.tiles,
                   s.ntiles, (const float2 *)s.Q32, qs, j, s.hpart, (const int *)s.meff, c->d_err);
        bse_prof_end(c, BSE_KP_MATVEC);
        launch_pdl(k_hmv_reduce<1>, dim3(s.nbt), dim3(2 * HT * 1), 0, st, (const float2 *)s.hpart, dim, s.nbt,
                   s.W, (const double2 *)s.Q, qs, j, (const int *)s.meff, s.apart);
      } else if (n_pol == 2) {
        launch_pdl(k_hmv_tma<2>, dim3(grid), dim3(128), hmv_tma_smem<2>(), st, s.tmH, dim, s.nbt, s.tiles,
                   s.ntiles, (const float2 *)s.Q32, qs, j, s.hpart, (const int *)s.meff, c->d_err);
        bse_prof_end(c, BSE_KP_MATVEC);
        launch_pdl(k_hmv_reduce<2>, dim3(s.nbt), dim3(2 * HT * 2), 0, st, (const float2 *)s.hpart, dim, s.nbt,
                   s.W, (const double2 *)s.Q, qs, j, (const int *)s.meff, s.apart);
      } else {
        launch_pdl(k_hmv_tma<3>, dim3(grid), dim3(128), hmv_tma_smem<3>(), st, s.tmH, dim, s.nbt, s.tiles,
                   s.ntiles, (const float2 *)s.Q32, qs, j, s.hpart, (const int *)s.meff, c->d_err);
        bse_prof_end(c, BSE_KP_MATVEC);
        launch_pdl(k_hmv_reduce<3>, dim3(s.nbt), dim3(2 * HT * 3), 0, st, (const float2 *)s.hpart, dim, s.nbt,
                   s.W, (const double2 *)s.Q, qs, j, (const int *)s.meff, s.apart);
      }
      bse_count_launch(2);
    } else if (c64 && s.hpart) {
      dim3 g(s.nbt, s.nbt);
      if (n_pol == 1) {
        k_hmatvec_c64<1><<<g, 128, 0, st>>>((const float2 *)H, dim, s.nbt, s.Q32, qs, j, s.hpart, s.meff);
        bse_prof_end(c, BSE_KP_MATVEC);
        k_hmv_reduce<1><<<s.nbt, 2 * HT * 1, 0, st>>>(s.hpart, dim, s.nbt, s.W, s.Q, qs, j, s.meff, s.apart);
      } else if (n_pol == 2) {
        k_hmatvec_c64<2><<<g, 128, 0, st>>>((const float2 *)H, dim, s.nbt, s.Q32, qs, j, s.hpart, s.meff);
        bse_prof_end(c, BSE_KP_MATVEC);
        k_hmv_reduce<2><<<s.nbt, 2 * HT * 2, 0, st>>>(s.hpart, dim, s.nbt, s.W, s.Q, qs, j, s.meff, s.apart);
      } else {
        k_hmatvec_c64<3><<<g, 128, 0, st>>>((const float2 *)H, dim, s.nbt, s.Q32, qs, j, s.hpart, s.meff);
        bse_prof_end(c, BSE_KP_MATVEC);
        k_hmv_reduce<3><<<s.nbt, 2 * HT * 3, 0, st>>>(s.hpart, dim, s.nbt, s.W, s.Q, qs, j, s.meff, s.apart);
      }
      bse_count_launch(2);
    } else if (c64) {
      if (n_pol == 1) k_matvec_c64<1><<<mv_blocks, 256, 0, st>>>((const float2 *)H, dim, s.Q, qs, j, s.W, s.meff);
      else if (n_pol == 2) k_matvec_c64<2><<<mv_blocks, 256, 0, st>>>((const float2 *)H, dim, s.Q, qs, j, s.W, s.meff);
      else k_matvec_c64<3><<<mv_blocks, 256, 0, st>>>((const float2 *)H, dim, s.Q, qs, j, s.W, s.meff);
    } else {
      if (n_pol == 1) k_matvec_c128<1><<<mv_blocks, 256, 0, st>>>((const double2 *)H, dim, s.Q, qs, j, s.W, s.meff);
      else if (n_pol == 2) k_matvec_c128<2><<<mv_blocks, 256, 0, st>>>((const double2 *)H, dim, s.Q, qs, j, s.W, s.meff);
      else k_matvec_c128<3><<<mv_blocks, 256, 0, st>>>((const double2 *)H, dim, s.Q, qs, j, s.W, s.meff);
    }
    if (!s.hpart && !matfree) bse_count_launch();
    bse_prof_end(c, BSE_KP_MATVEC);
    if (!s.hpart) {  // the full-read matvecs write W directly: alpha_j partials in a separate pass
      k_alpha_part<<<dim3(s.nbt, n_pol), HT, 0, st>>>(s.W, dim, s.Q, qs, j, s.meff, s.nbt, s.apart);
      bse_count_launch();
    }
    const bool proj32 = c64 && dim % 2 == 0;
    // |W|^2 per row block before the reorthogonalisation (the DGKS test's reference)
    launch_pdl(k_axpy, dim3(el_blocks, n_pol), dim3(256), 0, st, s.W, dim, (const double2 *)s.Q, qs, j, s.a,
               (const double *)s.b, ldab, (const int *)s.meff, s.nbt, (const double *)s.apart,
               proj32 ? s.n0part : (double *)nullptr);
    bse_prof_begin(c, BSE_KP_REORTH);
    for (int pass = 0; pass < 2; pass++) {
      if (proj32) {
        // the second pass runs where the DGKS test asks for it (meff2); the first pass left the
        // norms of its result in npart, and the second overwrites them where it runs, so npart
        // holds the final norms either way
        if (pass == 1) {
          launch_pdl(k_dgks, dim3(n_pol), dim3(32), 0, st, (const double *)s.n0part, (const double *)s.npart, s.nbt,
                     (const int *)s.meff, s.meff2);
          bse_count_launch();
        }
        const int *mp = pass ? s.meff2 : s.meff;
        launch_pdl(k_reorth_dots_chunk, dim3(s.nrch, n_pol, (j + RROWS) / RROWS), dim3(256), 0, st,
                   (const double2 *)s.W, dim, (const float2 *)s.Q32, qs, j, s.rpart, s.nrch, ldab, mp);
        launch_pdl(k_reorth_coef, dim3((j + 1 + 7) / 8, n_pol), dim3(256), 0, st, (const float2 *)s.rpart, s.nrch,
                   ldab, j, s.coef, ldab, mp);
        launch_pdl(k_reorth_update32, dim3(el2_blocks, n_pol), dim3(256), 0, st, s.W, dim, (const float2 *)s.Q32, qs,
                   j, (const double2 *)s.coef, ldab, mp, s.nbt, s.npart);
      } else {  // complex128 H, or an odd dim: FP64 projections on the FP64 basis
        k_reorth_dots<<<dim3(j + 1, n_pol), 256, 0, st>>>(s.W, dim, s.Q, qs, j, s.coef, ldab, s.meff);
        k_reorth_update<<<dim3(el_blocks, n_pol), 256, 0, st>>>(s.W, dim, s.Q, qs, j, s.coef, ldab, s.meff);
      }
    }
    bse_prof_end(c, BSE_KP_REORTH);
    if (!proj32)
      launch_pdl(k_norm_part, dim3(s.nbt, n_pol), dim3(HT), 0, st, (const double2 *)s.W, dim, j, (const int *)s.meff,
                 s.nbt, s.npart);
    launch_pdl(k_scale, dim3(el_blocks, n_pol), dim3(256), 0, st, (const double2 *)s.W, dim, s.Q, qs, j, s.b, ldab,
               s.meff, (const double *)s.hmax, n_steps, s.Q32, s.nbt, (const double *)s.npart);
    bse_count_launch(proj32 ? 8 : 7);  // axpy, two reorthogonalisation passes (+ the DGKS test), (norm,) scale
    r = bse_check_launch(c, "lanczos step");
    if (r != BSE_OK) return r;
  }
  return BSE_OK;
}

}  // namespace

bse_status run_dipole_vector(bse_ctx *c, const double *vel, const double *e_ks, double2 *u) {
  dim3 grid((unsigned)((c->dim + 255) / 256), 3);
  k_dipole<<<grid, 256, 0, c->stream>>>((const double2 *)vel, e_ks, c->nk, c->nv, c->nc, u, c->d_err);
  bse_count_launch();
  return bse_check_launch(c, "dipole_vector");
}

bse_status run_spectrum(bse_ctx *c, const void *H, const double2 *u, int n_pol, int n_steps,
                        const double *omega, int n_w, double eta, double pref, double *eps2, double *ab,
                        bool accumulate) {
  LanczosScratch s;
  bse_status r = lanczos_alloc(c, s, n_pol, n_steps);
  if (r == BSE_OK) r = lanczos_run(c, s, H, u, n_pol, n_steps);
  if (r == BSE_OK) {
    k_contfrac<<<(n_w + 127) / 128, 128, 0, c->stream>>>(s.a, s.b, n_steps + 1, s.beta0, s.meff, n_pol, omega,
                                                         n_w, eta, pref, eps2, accumulate ? 1 : 0);
    bse_count_launch();
    if (ab) {
      k_pack_ab<<<dim3((n_steps + 127) / 128, n_pol), 128, 0, c->stream>>>(s.a, s.b, s.beta0, n_steps + 1,
                                                                          n_pol, n_steps, ab);
      bse_count_launch();
    }
    r = bse_check_launch(c, "continued fraction");
  }
  lanczos_release(c, s);
  return r;
}

bse_status run_spectrum_matfree(bse_ctx *c, const double2 *u, int n_pol, int n_steps, const double *omega, int n_w,
                                double eta, double pref, double *eps2, double *ab) {
  LanczosScratch s;
  bse_status r = lanczos_alloc(c, s, n_pol, n_steps, true);
  if (r == BSE_OK) r = lanczos_run(c, s, nullptr, u, n_pol, n_steps);
  if (r == BSE_OK) {
    k_contfrac<<<(n_w + 127) / 128, 128, 0, c->stream>>>(s.a, s.b, n_steps + 1, s.beta0, s.meff, n_pol, omega,
                                                         n_w, eta, pref, eps2, 0);
    bse_count_launch();
    if (ab) {
      k_pack_ab<<<dim3((n_steps + 127) / 128, n_pol), 128, 0, c->stream>>>(s.a, s.b, s.beta0, n_steps + 1,
                                                                          n_pol, n_steps, ab);
      bse_count_launch();
    }
    r = bse_check_launch(c, "matrix-free continued fraction");
  }
  lanczos_release(c, s);
  return r;
}

// y[e][x] = sum_l v_e[l] Q[l][x]: Ritz vectors from the tridiagonal eigenvectors v_e (stored
// in work[e*3m .. e*3m+m)) and the Krylov basis of the first start vector.
__global__ void k_ritz_vectors(const double *work, const int *meff, int n_eig, const double2 *Q, long long dim,
                               double2 *Y) {
  const long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= dim) return;
  const int m = meff[0];
  for (int e = 0; e < n_eig; e++) {
    double2 acc = make_double2(0.0, 0.0);
    if (e < m) {
      const double *v = work + (long long)e * 3 * m;
      for (int l = 0; l < m; l++) {
        const double2 q = Q[(long long)l * dim + x];
        acc.x += v[l] * q.x;
        acc.y += v[l] * q.y;
      }
    }
    Y[(long long)e * dim + x] = acc;
  }
}

bse_status run_lowest(bse_ctx *c, const void *H, int n_eig, int n_steps, uint64_t seed, double *omega_out,
                      double *resid_out, double2 *vecs_out) {
  LanczosScratch s;
  double2 *u = nullptr;
  double *work = nullptr;
  bse_status r = lanczos_alloc(c, s, 1, n_steps);
  if (r == BSE_OK && (cudaMallocAsync((void **)&u, sizeof(double2) * c->dim, c->stream) != cudaSuccess ||
                      cudaMallocAsync((void **)&work, sizeof(double) * 3 * n_eig * n_steps, c->stream) != cudaSuccess)) {
    cudaGetLastError();
    r = bse_fail(c, BSE_ENOMEM, "lowest: scratch allocation failed");
  }
  if (r == BSE_OK) {
    k_random_start<<<(unsigned)((c->dim + 255) / 256), 256, 0, c->stream>>>(u, c->dim, seed);
    bse_count_launch();
    r = lanczos_run(c, s, H, u, 1, n_steps);
  }
  if (r == BSE_OK) {
    // the residual pass also leaves the tridiagonal eigenvectors in work, which the Ritz
    // vectors need; use a scratch residual array when the caller passed none
    double *res = resid_out;
    if (!res && vecs_out && cudaMallocAsync((void **)&res, sizeof(double) * n_eig, c->stream) != cudaSuccess) {
      cudaGetLastError();
      r = bse_fail(c, BSE_ENOMEM, "lowest: scratch allocation failed");
    }
    if (r == BSE_OK) {
      k_ritz<<<(n_eig + 31) / 32, 32, 0, c->stream>>>(s.a, s.b, s.meff, n_eig, omega_out, res, work);
      bse_count_launch();
      if (vecs_out) {
        k_ritz_vectors<<<(unsigned)((c->dim + 255) / 256), 256, 0, c->stream>>>(work, s.meff, n_eig, s.Q, c->dim,
                                                                                vecs_out);
        bse_count_launch();
      }
      r = bse_check_launch(c, "ritz");
    }
    if (res && res != resid_out) cudaFreeAsync(res, c->stream);
  }
  if (u) cudaFreeAsync(u, c->stream);
  if (work) cudaFreeAsync(work, c->stream);
  lanczos_release(c, s);
  return r;
}

namespace {

// ---- adjoint seed of the windowed absorption integral (bse_window_seed) --------------------
// I = pref sum_p u_p^dagger f(H) u_p with f(x) = (1/pi)[atan((w_hi - x)/eta) - atan((w_lo - x)/eta)],
// the Lorentzian of Eq. abs_vel integrated over [w_lo, w_hi].  From the Lanczos tridiagonal
// T = Z diag(theta) Z^T of each start vector: the Ritz vectors Y = Z^T Q (rows), v = first
// components of Z's columns, and (Daleckii-Krein in the Krylov subspace)
//   Gamma = sum_p Y_p^T M_p conj(Y_p),  M_p = pref |u_p|^2 (F o v v^T),
//   F_il = (f(theta_i) - f(theta_l)) / (theta_i - theta_l),  F_ii = f'(theta_i),
// so that dI = tr(Gamma dH); I = sum_p pref |u_p|^2 sum_i v_i^2 f(theta_i).

__device__ __forceinline__ double window_f(double x, double lo, double hi, double eta) {
  return (atan((hi - x) / eta) - atan((lo - x) / eta)) * (1.0 / M_PI);
}
__device__ __forceinline__ double window_df(double x, double lo, double hi, double eta) {
  const double ya = lo - x, yb = hi - x;
  return (eta / (ya * ya + eta * eta) - eta / (yb * yb + eta * eta)) * (1.0 / M_PI);
}

// Eigen-decomposition of each tridiagonal T_p (diagonal a, off-diagonal b, order m = meff[p])
// by the implicit QL algorithm with Wilkinson-type shifts (Bowdler, Martin, Reinsch and
// Wilkinson, Numer. Math. 11 (1968) 293).  Thread 0 runs the shifted sweeps on (d, e) and
// records each sweep's Givens rotations; then every thread applies them, in order, to its
// columns of Zt (Zt[i][k] = component k of eigenvector i), so the updates are coalesced.
// On exit d holds the eigenvalues (unsorted) and Zt the eigenvectors.  A block that fails to
// converge sets the error word.
constexpr int QL_MAX_SWEEPS = 60;
// With in_smem, d, e and the sweep's rotations live in shared memory (4 mmax doubles,
// dynamic): thread 0's sweeps are a serial chain of dependent updates, which global memory
// stretches to its latency per step; d is copied to dd at the end.  Without, they live in
// dd, ee and rot (orders beyond the shared-memory budget).
__global__ void __launch_bounds__(256) k_tridiag_ql(const double *__restrict__ a, const double *__restrict__ b,
                                                    int ldab, const int *__restrict__ meff, int mmax,
                                                    double *__restrict__ dd, double *__restrict__ ee,
                                                    double *__restrict__ Zt, double2 *__restrict__ rot, int *err,
                                                    int in_smem) {
  __shared__ int s_mm, s_first, s_last;
  extern __shared__ double ql_sm[];
  const int p = blockIdx.x;
  const int m = meff[p];
  double *d = in_smem ? ql_sm : dd + (long long)p * mmax, *e = in_smem ? d + mmax : ee + (long long)p * mmax;
  double *Z = Zt + (long long)p * mmax * mmax;
  double2 *cs = in_smem ? reinterpret_cast<double2 *>(ql_sm + 2 * mmax) : rot + (long long)p * mmax;
  for (int i = threadIdx.x; i < mmax; i += blockDim.x) {
    d[i] = i < m ? a[p * ldab + i] : 0.0;
    e[i] = i < m - 1 ? b[p * ldab + i] : 0.0;
  }
  for (long long t = threadIdx.x; t < (long long)mmax * mmax; t += blockDim.x)
    Z[t] = (t / mmax == t % mmax && t / mmax < m) ? 1.0 : 0.0;
  __syncthreads();
  for (int l = 0; l < m; l++) {
    for (int sweep = 0;; sweep++) {
      if (threadIdx.x == 0) {
        int mm = l;
        while (mm < m - 1) {
          const double scale = fabs(d[mm]) + fabs(d[mm + 1]);
          if (fabs(e[mm]) <= 1e-16 * scale || fabs(e[mm]) < 1e-300) break;
          mm++;
        }
        s_mm = mm;
        s_first = mm - 1;
        s_last = mm;  // rotations i = s_first down to s_last are valid (none when s_last > s_first)
        if (mm != l && sweep < QL_MAX_SWEEPS) {
          // shift from the leading 2x2 block at l
          double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
          double r = hypot(g, 1.0);
          g = d[mm] - d[l] + e[l] / (g + copysign(r, g));
          double sn = 1.0, cn = 1.0, pp = 0.0;
          bool split = false;
          int i = mm - 1;
          for (; i >= l; i--) {
            const double f = sn * e[i], bb = cn * e[i];
            r = hypot(f, g);
            e[i + 1] = r;
            if (r == 0.0) {  // underflow: the block splits here
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
            cs[i] = make_double2(cn, sn);
          }
          s_last = split ? i + 1 : l;
          if (!split) {
            d[l] -= pp;
            e[l] = g;
            e[mm] = 0.0;
          }
        } else if (mm != l) {
          atomicOr(err, BSE_DERR_BOUNDS);
          s_mm = l;  // give up on this eigenvalue
        }
      }
      __syncthreads();
      if (s_mm == l) break;
      const int first = s_first, last = s_last;
      for (int k = threadIdx.x; k < m; k += blockDim.x) {
        for (int i = first; i >= last; i--) {
          const double2 r = cs[i];
          const double zi = Z[(long long)i * mmax + k], zn = Z[(long long)(i + 1) * mmax + k];
          Z[(long long)(i + 1) * mmax + k] = r.y * zi + r.x * zn;
          Z[(long long)i * mmax + k] = r.x * zi - r.y * zn;
        }
      }
      __syncthreads();
    }
  }
  if (in_smem)
    for (int i = threadIdx.x; i < mmax; i += blockDim.x) dd[(long long)p * mmax + i] = d[i];
}

// Launch k_tridiag_ql with its working arrays in shared memory when they fit.
void tridiag_ql(bse_ctx *c, const double *a, const double *b, int ldab, const int *meff, int mmax, int n_pol,
                double *dd, double *ee, double *Zt, double2 *rot) {
  const size_t sm = sizeof(double) * 4 * (size_t)mmax;
  const int in_smem = sm <= 200 * 1024;
  if (in_smem && sm > 48 * 1024)
    cudaFuncSetAttribute(k_tridiag_ql, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_tridiag_ql<<<n_pol, 256, in_smem ? sm : 0, c->stream>>>(a, b, ldab, meff, mmax, dd, ee, Zt, rot, c->d_err,
                                                            in_smem);
}

// M_p[i][l] = pref |u_p|^2 F_il v_i v_l with v_i = Zt[i][0]; Ipart[p] = pref |u_p|^2 sum_i v_i^2 f(theta_i).
__global__ void k_window_M(const double *__restrict__ dd, const double *__restrict__ Zt, const int *__restrict__ meff,
                           int mmax, const double *__restrict__ beta0, double lo, double hi, double eta, double pref,
                           double *__restrict__ M, double *__restrict__ Ipart) {
  const int p = blockIdx.y;
  const int m = meff[p];
  const double *d = dd + (long long)p * mmax, *Z = Zt + (long long)p * mmax * mmax;
  const double sc = pref * beta0[p] * beta0[p];
  const long long nm = (long long)mmax * mmax;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < nm; t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t / mmax), l = (int)(t % mmax);
    double v = 0.0;
    if (i < m && l < m) {
      const double ti = d[i], tl = d[l];
      const double gap = ti - tl, tol = 1e-9 * (fabs(ti) + fabs(tl) + eta);
      const double F = fabs(gap) > tol ? (window_f(ti, lo, hi, eta) - window_f(tl, lo, hi, eta)) / gap
                                       : window_df(0.5 * (ti + tl), lo, hi, eta);
      v = sc * F * Z[(long long)i * mmax] * Z[(long long)l * mmax];
    }
    M[(long long)p * nm + t] = v;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    double acc = 0.0;
    for (int i = 0; i < m; i++) {
      const double vi = Z[(long long)i * mmax];
      acc += vi * vi * window_f(d[i], lo, hi, eta);
    }
    Ipart[p] = sc * acc;
  }
}

__global__ void k_sum_small(const double *__restrict__ x, int n, double *__restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < n; i++) s += x[i];
    *out = s;
  }
}

// C[p][i][x] = sum_l A[p][i][l] * (conj ? conj(B[p][l][x]) : B[p][l][x]) for l < meff[p]; A real
// [mmax][mmax], B complex [mmax rows, stride ldb][dim]; rows i >= meff[p] are written as zero.
__global__ void __launch_bounds__(256) k_real_cgemm(const double *__restrict__ A, const double2 *__restrict__ B,
                                                    long long ldb_p, int conj, const int *__restrict__ meff,
                                                    int mmax, long long dim, double2 *__restrict__ C) {
  __shared__ double As[16][64];
  __shared__ double2 Bs[16][64];
  const int p = blockIdx.z, m = meff[p];
  A += (long long)p * mmax * mmax;
  B += p * ldb_p;
  C += (long long)p * mmax * dim;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int row0 = blockIdx.y * 64;
  const long long col0 = (long long)blockIdx.x * 64;
  double2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; i++)
#pragma unroll
    for (int j = 0; j < 4; j++) acc[i][j] = make_double2(0, 0);
  for (int k0 = 0; k0 < m; k0 += 16) {
    for (int e = threadIdx.x; e < 1024; e += 256) {
      const int r = e / 16, kk = e % 16, gr = row0 + r, gk = k0 + kk;
      As[kk][r] = (gr < m && gk < m) ? A[(long long)gr * mmax + gk] : 0.0;
      const int kb = e / 64, cc = e % 64, gkb = k0 + kb;
      const long long gc = col0 + cc;
      double2 v = make_double2(0, 0);
      if (gkb < m && gc < dim) {
        v = B[(long long)gkb * dim + gc];
        if (conj) v.y = -v.y;
      }
      Bs[kb][cc] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; kk++) {
      double a[4];
      double2 bv[4];
#pragma unroll
      for (int i = 0; i < 4; i++) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; j++) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) {
          acc[i][j].x = fma(a[i], bv[j].x, acc[i][j].x);
          acc[i][j].y = fma(a[i], bv[j].y, acc[i][j].y);
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; i++)
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const int r = row0 + ty + 16 * i;
      const long long cc = col0 + tx + 16 * j;
      if (r < mmax && cc < dim) C[(long long)r * dim + cc] = r < m ? acc[i][j] : make_double2(0, 0);
    }
}

}  // namespace

// ---- half-read products for other callers (full BSE) -------------------------------------
struct HalfMV {
  int nbt = 0, ntiles = 0;
  int2 *tiles = nullptr;
  float2 *part = nullptr;   // [nbt][nbt][HT][6]
  int *ones = nullptr;      // [6] recursion lengths for the kernels' liveness test (all live)
  double *apart = nullptr;  // [6][nbt] (unused alpha partials of the reduction)
  double2 *Qdummy = nullptr;
};

bse_status halfmv_alloc(bse_ctx *c, HalfMV **out) {
  *out = nullptr;
  if (c->precision == BSE_FP64 || c->dim % 2) return BSE_OK;  // complex64 H of even order only
  HalfMV *h = new HalfMV();
  const long long dim = c->dim;
  h->nbt = (int)((dim + HT - 1) / HT);
  std::vector<int2> tl;
  for (int bi = 0; bi < h->nbt; bi++)
    for (int bj = bi; bj < h->nbt; bj++) tl.push_back(make_int2(bi, bj));
  h->ntiles = (int)tl.size();
  const int ones[6] = {1, 1, 1, 1, 1, 1};
  cudaStream_t st = c->stream;
  if (cudaMallocAsync((void **)&h->part, sizeof(float2) * (size_t)h->nbt * h->nbt * HT * 6, st) != cudaSuccess ||
      cudaMallocAsync((void **)&h->tiles, sizeof(int2) * tl.size(), st) != cudaSuccess ||
      cudaMallocAsync((void **)&h->ones, sizeof(int) * 6, st) != cudaSuccess ||
      cudaMallocAsync((void **)&h->apart, sizeof(double) * 6 * h->nbt, st) != cudaSuccess ||
      cudaMallocAsync((void **)&h->Qdummy, sizeof(double2) * 6 * dim, st) != cudaSuccess ||
      cudaMemcpyAsync(h->tiles, tl.data(), sizeof(int2) * tl.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(h->ones, ones, sizeof(ones), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemsetAsync(h->Qdummy, 0, sizeof(double2) * 6 * dim, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    halfmv_release(c, h);
    return bse_fail(c, BSE_ENOMEM, "half-read product scratch allocation failed");
  }
  bse_once_per_device(c, BSE_ONCE_HMV_ALL, [] {
    cudaFuncSetAttribute(k_hmv_tma<1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, hmv_tma_smem<1>());
    cudaFuncSetAttribute(k_hmv_tma<2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, hmv_tma_smem<2>());
    cudaFuncSetAttribute(k_hmv_tma<3, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, hmv_tma_smem<3>());
    cudaFuncSetAttribute(k_hmv_tma<1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, hmv_tma_smem<1>());
    cudaFuncSetAttribute(k_hmv_tma<2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, hmv_tma_smem<2>());
    cudaFuncSetAttribute(k_hmv_tma<3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, hmv_tma_smem<3>());
    cudaFuncSetAttribute(k_hmv_tma<4, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, hmv_tma_smem<4>());
    cudaFuncSetAttribute(k_hmv_tma<4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, hmv_tma_smem<4>());
    cudaFuncSetAttribute(k_hmv_tma<6, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, hmv_tma_smem<6>());
    cudaFuncSetAttribute(k_hmv_tma<6, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, hmv_tma_smem<6>());
  });
  *out = h;
  return BSE_OK;
}

void halfmv_release(bse_ctx *c, HalfMV *h) {
  if (!h) return;
  void *ptrs[] = {h->part, h->tiles, h->ones, h->apart, h->Qdummy};
  for (void *p : ptrs)
    if (p) cudaFreeAsync(p, c->stream);
  delete h;
}

// W[p] = Hm Z[p] (np in 1, 2, 3, 4, 6) for a complex64 Hm, Hermitian (sym = false) or
// complex symmetric (sym = true), reading only its upper-triangle 128 x 128 tiles once for
// all np vectors.  Z [np][dim] complex64, W [np][dim] complex128.
bse_status halfmv_run(bse_ctx *c, HalfMV *h, const void *Hm, bool sym, const float2 *Z, int np, double2 *W) {
  const long long dim = c->dim;
  CUtensorMap tm;
  if (!encode_rows_f32(&tm, Hm, 2ull * dim, (unsigned long long)dim, 2 * HT, MV_CHUNK))
    return bse_fail(c, BSE_ECUDA, "half-read product: tensor map encoding failed");
  cudaStream_t st = c->stream;
  const int grid = std::min(h->ntiles, (np <= 3 ? HmvSmem<3>::CTAS : HmvSmem<6>::CTAS) * c->n_sm);  // resident CTAs per SM
  bse_prof_begin(c, BSE_KP_MATVEC);
#define HALF_LAUNCH(NPV, SYMV)                                                                                 \
  k_hmv_tma<NPV, SYMV><<<grid, 128, hmv_tma_smem<NPV>(), st>>>(tm, dim, h->nbt, h->tiles, h->ntiles, Z, dim, 0, \
                                                             h->part, h->ones, c->d_err)
  if (np != 1 && np != 2 && np != 3 && np != 4 && np != 6)
    return bse_fail(c, BSE_EINVAL, "half-read product: unsupported vector count");
  if (np == 1) { if (sym) HALF_LAUNCH(1, true); else HALF_LAUNCH(1, false); }
  else if (np == 2) { if (sym) HALF_LAUNCH(2, true); else HALF_LAUNCH(2, false); }
  else if (np == 3) { if (sym) HALF_LAUNCH(3, true); else HALF_LAUNCH(3, false); }
  else if (np == 4) { if (sym) HALF_LAUNCH(4, true); else HALF_LAUNCH(4, false); }
  else { if (sym) HALF_LAUNCH(6, true); else HALF_LAUNCH(6, false); }
#undef HALF_LAUNCH
  bse_prof_end(c, BSE_KP_MATVEC);
#define HALF_REDUCE(NPV, HV) \
  k_hmv_reduce<NPV, HV><<<h->nbt, HV * HT * NPV, 0, st>>>(h->part, dim, h->nbt, W, h->Qdummy, dim, 0, h->ones, h->apart)
  if (np == 1) HALF_REDUCE(1, 2);
  else if (np == 2) HALF_REDUCE(2, 2);
  else if (np == 3) HALF_REDUCE(3, 2);
  else if (np == 4) HALF_REDUCE(4, 2);
  else HALF_REDUCE(6, 1);
#undef HALF_REDUCE
  bse_count_launch(2);
  return bse_check_launch(c, "half-read product");
}

int reorth32_chunks(long long n) { return (int)((n + RCH - 1) / RCH); }

// One reorthogonalisation pass with FP32 projections (the complex64 path's chunked kernels):
// coef_i = D32_i^H W, W -= sum_{i<=j} coef_i U32_i, per polarisation; vectors of even length n.
bse_status launch_reorth32_pass(bse_ctx *c, double2 *W, long long n, const float2 *D32, const float2 *U32,
                                long long qs, int j, float2 *rpart, int ldp, double2 *coef, const int *meff,
                                int n_pol) {
  if (n % 2) return bse_fail(c, BSE_EINVAL, "reorthogonalisation: odd vector length");
  const int nrch = reorth32_chunks(n);
  cudaStream_t st = c->stream;
  k_reorth_dots_chunk<<<dim3(nrch, n_pol, (j + RROWS) / RROWS), 256, 0, st>>>(W, n, D32, qs, j, rpart, nrch, ldp,
                                                                             meff);
  k_reorth_coef<<<dim3((j + 1 + 7) / 8, n_pol), 256, 0, st>>>(rpart, nrch, ldp, j, coef, ldp, meff);
  k_reorth_update32<<<dim3((unsigned)((n / 2 + 255) / 256), n_pol), 256, 0, st>>>(W, n, U32, qs, j, coef, ldp, meff, 0,
                                                                                  nullptr);
  bse_count_launch(3);
  return BSE_OK;
}

bse_status run_window_seed(bse_ctx *c, const void *H, const double2 *u, int n_pol, int n_steps, double w_lo,
                           double w_hi, double eta, double pref, double *I_out, double2 *Gamma) {
  LanczosScratch s;
  bse_status r = lanczos_alloc(c, s, n_pol, n_steps);
  const int mmax = n_steps;
  const long long dim = c->dim;
  double *dd = nullptr, *ee = nullptr, *Zt = nullptr, *M = nullptr, *Ip = nullptr;
  double2 *rot = nullptr, *Y = nullptr, *Z = nullptr;
  const size_t nm = (size_t)n_pol * mmax * mmax;
  const size_t ny = (size_t)n_pol * mmax * dim;
  if (r == BSE_OK && (cudaMallocAsync((void **)&dd, sizeof(double) * n_pol * mmax, c->stream) != cudaSuccess ||
                      cudaMallocAsync((void **)&ee, sizeof(double) * n_pol * mmax, c->stream) != cudaSuccess ||
                      cudaMallocAsync((void **)&rot, sizeof(double2) * n_pol * mmax, c->stream) != cudaSuccess ||
                      cudaMallocAsync((void **)&Zt, sizeof(double) * nm, c->stream) != cudaSuccess ||
                      cudaMallocAsync((void **)&M, sizeof(double) * nm, c->stream) != cudaSuccess ||
                      cudaMallocAsync((void **)&Ip, sizeof(double) * n_pol, c->stream) != cudaSuccess ||
                      cudaMallocAsync((void **)&Y, sizeof(double2) * ny, c->stream) != cudaSuccess ||
                      cudaMallocAsync((void **)&Z, sizeof(double2) * ny, c->stream) != cudaSuccess)) {
    cudaGetLastError();
    r = bse_fail(c, BSE_ENOMEM, "window_seed: scratch allocation failed");
  }
  if (r == BSE_OK) r = lanczos_run(c, s, H, u, n_pol, n_steps);
  if (r == BSE_OK) {
    tridiag_ql(c, s.a, s.b, n_steps + 1, s.meff, mmax, n_pol, dd, ee, Zt, rot);
    k_window_M<<<dim3(64, n_pol), 256, 0, c->stream>>>(dd, Zt, s.meff, mmax, s.beta0, w_lo, w_hi, eta, pref, M, Ip);
    // Ritz vectors Y_p = Zt_p Q_p, then Z_p = M_p conj(Y_p)
    dim3 g((unsigned)((dim + 63) / 64), (unsigned)((mmax + 63) / 64), n_pol);
    const long long qs = (long long)(n_steps + 1) * dim;
    k_real_cgemm<<<g, 256, 0, c->stream>>>(Zt, s.Q, qs, 0, s.meff, mmax, dim, Y);
    k_real_cgemm<<<g, 256, 0, c->stream>>>(M, Y, (long long)mmax * dim, 1, s.meff, mmax, dim, Z);
    bse_count_launch(4);
    if (I_out) {
      k_sum_small<<<1, 32, 0, c->stream>>>(Ip, n_pol, I_out);
      bse_count_launch();
    }
    r = bse_check_launch(c, "window seed");
  }
  // Gamma = sum_p Y_p^T Z_p: one transposed GEMM over the stacked (p, i) rows
  if (r == BSE_OK) r = launch_zgemm_tn(c, (int)dim, (int)dim, n_pol * mmax, Y, Z, Gamma, 1.0);
  void *ptrs[] = {dd, ee, rot, Zt, M, Ip, Y, Z};
  for (void *ptr : ptrs)
    if (ptr) cudaFreeAsync(ptr, c->stream);
  lanczos_release(c, s);
  return r;
}

// ---- allocation-free variant of the spectrum (bse_spectrum_static) -------------------------
// Its Lanczos scratch lives in one file-scope device array instead of per-call allocations.
// Every GPU that loads the library holds this array until the process exits.
constexpr size_t BSE_STATIC_SCRATCH_BYTES = (size_t)64 << 20;
static __device__ __align__(256) unsigned char g_spectrum_scratch[BSE_STATIC_SCRATCH_BYTES];

namespace {
std::mutex g_static_mu;
void *g_static_addr[64] = {nullptr};

// Device address of g_spectrum_scratch on the context's device, looked up once per device
// with that device current.  In host code the array's name is only a host-side stand-in.
bse_status static_scratch_base(bse_ctx *c, unsigned char **out) {
  std::lock_guard<std::mutex> lk(g_static_mu);
  const int dev = c->device;
  if (dev < 0 || dev >= 64) return bse_fail(c, BSE_EINVAL, "spectrum_static: device index out of range");
  if (!g_static_addr[dev]) {
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) return bse_fail(c, BSE_ECUDA, "spectrum_static: cudaGetDevice failed");
    if (cur != dev && cudaSetDevice(dev) != cudaSuccess)
      return bse_fail(c, BSE_ECUDA, "spectrum_static: cannot make the context's device current");
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_spectrum_scratch);
    if (cur != dev) cudaSetDevice(cur);
    if (e != cudaSuccess || !p)
      return bse_fail(c, BSE_ECUDA, std::string("spectrum_static: cudaGetSymbolAddress failed: ") +
                                        cudaGetErrorString(e));
    g_static_addr[dev] = p;
  }
  *out = static_cast<unsigned char *>(g_static_addr[dev]);
  return BSE_OK;
}

// Lay the Lanczos scratch out in [base, base + bytes) (256-byte aligned pieces) and return the
// bytes it needs; with base == nullptr only the size is computed.
size_t carve_scratch(bse_ctx *c, LanczosScratch &s, int n_pol, int n_steps, unsigned char *base) {
  const long long dim = c->dim;
  const bool c64 = !c->h64;
  size_t off = 0;
  auto take = [&](size_t bytes) -> unsigned char * {
    off = (off + 255) & ~(size_t)255;
    unsigned char *p = base ? base + off : nullptr;
    off += bytes;
    return p;
  };
  const size_t qn = (size_t)n_pol * (n_steps + 1) * dim;
  s.Q = (double2 *)take(sizeof(double2) * qn);
  s.W = (double2 *)take(sizeof(double2) * n_pol * dim);
  s.coef = (double2 *)take(sizeof(double2) * n_pol * (n_steps + 1));
  s.a = (double *)take(sizeof(double) * n_pol * (n_steps + 1));
  s.b = (double *)take(sizeof(double) * n_pol * (n_steps + 1));
  s.beta0 = (double *)take(sizeof(double) * n_pol);
  s.hmax = (double *)take(sizeof(double));
  s.part = (double *)take(sizeof(double) * 1024);
  s.meff = (int *)take(sizeof(int) * n_pol);
  s.meff2 = (int *)take(sizeof(int) * n_pol);
  s.nbt = (int)((dim + HT - 1) / HT);
  s.apart = (double *)take(sizeof(double) * 3 * n_pol * s.nbt);
  s.npart = s.apart ? s.apart + (size_t)n_pol * s.nbt : nullptr;
  s.n0part = s.apart ? s.apart + (size_t)2 * n_pol * s.nbt : nullptr;
  s.nrch = (int)((dim + RCH - 1) / RCH);
  s.Q32 = c64 ? (float2 *)take(sizeof(float2) * qn) : nullptr;
  s.rpart = c64 ? (float2 *)take(sizeof(float2) * (size_t)n_pol * s.nrch * (n_steps + 1)) : nullptr;
  s.ntiles = s.nbt * (s.nbt + 1) / 2;
  if (c64 && dim % 2 == 0) {
    s.hpart = (float2 *)take(sizeof(float2) * (size_t)s.nbt * s.nbt * HT * n_pol);
    s.tiles = (int2 *)take(sizeof(int2) * (size_t)s.ntiles);
  } else {
    s.hpart = nullptr;
    s.tiles = nullptr;
  }
  return off;
}
}  // namespace

bse_status run_spectrum_static(bse_ctx *c, const void *H, const double2 *u, int n_pol, int n_steps,
                               const double *omega, int n_w, double eta, double pref, double *eps2, double *ab) {
  LanczosScratch sz;
  const size_t need = carve_scratch(c, sz, n_pol, n_steps, nullptr);
  if (need > BSE_STATIC_SCRATCH_BYTES)
    return bse_fail(c, BSE_EINVAL,
                    "spectrum_static: needs " + std::to_string(need) + " bytes of scratch, the static array holds " +
                        std::to_string(BSE_STATIC_SCRATCH_BYTES) + " (reduce n_steps, n_pol or dim)");
  unsigned char *base = nullptr;
  bse_status r = static_scratch_base(c, &base);
  if (r != BSE_OK) return r;
  LanczosScratch s;
  carve_scratch(c, s, n_pol, n_steps, base);
  if (s.tiles) fill_tiles(c, s.nbt, s.tiles);
  r = lanczos_run(c, s, H, u, n_pol, n_steps);
  if (r != BSE_OK) return r;
  k_contfrac<<<(n_w + 127) / 128, 128, 0, c->stream>>>(s.a, s.b, n_steps + 1, s.beta0, s.meff, n_pol, omega, n_w, eta,
                                                       pref, eps2, 0);
  bse_count_launch();
  if (ab) {
    k_pack_ab<<<dim3((n_steps + 127) / 128, n_pol), 128, 0, c->stream>>>(s.a, s.b, s.beta0, n_steps + 1, n_pol,
                                                                        n_steps, ab);
    bse_count_launch();
  }
  return bse_check_launch(c, "spectrum_static");
}
