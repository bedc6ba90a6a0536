// Split-precision complex GEMM on tcgen05 tensor cores (sm_103a).
//
//   out[b][m][n] = scale * sum_{pa+pb <= NP-1} sum_k A_pa[b][m][k] * B_pb[b][n][k]   (complex)
//
// A and B are complex matrices stored K-major as planar bf16 "pieces": a real value x is
// x ~ p0 + p1 + p2 with p0 = bf16(x), p1 = bf16(x - p0), p2 = bf16(x - p0 - p1), and only
// piece products whose orders sum to at most NP-1 are kept (NP = 3: 6 products, NP = 2: 3,
// NP = 1: 1), accumulated in FP32 in tensor memory.  A complex product uses four real
// MMAs: Re += Ar Br^T - Ai Bi^T (the minus through the A-negate bit of the instruction
// descriptor), Im += Ar Bi^T + Ai Br^T.
//
// With TF = true the pieces are tf32 values in FP32 words instead (x ~ p0 + p1, p0 = tf32(x),
// p1 = tf32(x - p0), NP = 2: 3 products of kind::tf32 MMAs); everything else is the same.
//
// Operands arrive by TMA as 3-D tensors {K, rows, plane-piece(-batch)} with 64-byte
// swizzled rows (32 bf16 or 16 tf32 of K per stage); rows and K beyond the tensor are
// zero-filled.
// Persistent CTAs (one per SM) walk the 128 x BN output tiles of a work list (one GEMM, or
// several independent ones of a batch, Groups below): warp 0 issues TMA, warp 1
// allocates tensor memory and issues the MMAs from one thread, warps 2-5 drain the
// accumulators of one tile while the next tile's operands stream in.  Every barrier wait
// is bounded; a timeout sets the device error word and the CTA winds down.
#pragma once

#include "tc_ptx.cuh"

namespace tcg {

constexpr int BM = 128;
constexpr int BK = 32;                // bf16 elements of K per stage (64-byte rows)
constexpr int BK_TF32 = 16;           // tf32 elements of K per stage (the same 64-byte rows)
template <bool TF>
__host__ __device__ constexpr int bk_elems() { return TF ? BK_TF32 : BK; }
constexpr int ROWB = BK * 2;          // bytes per smem row
constexpr int A_TILE = BM * ROWB;     // 8 KB
constexpr int SMEM_BUDGET = 221184;   // stage bytes per CTA
constexpr long long WAIT_LIMIT = 4000000000LL;  // clock cycles (~2 s) before a wait gives up

template <int NP, int BN>
struct Cfg {
  static constexpr int PP = 2 * NP;                   // planes x pieces
  static constexpr int B_TILE = BN * ROWB;
  static constexpr int STAGE = PP * (A_TILE + B_TILE);
  static constexpr int S = SMEM_BUDGET / STAGE < 8 ? SMEM_BUDGET / STAGE : 8;
  static constexpr int TMEM_COLS = 2 * BN <= 32 ? 32 : 2 * BN <= 64 ? 64 : 2 * BN <= 128 ? 128 : 2 * BN <= 256 ? 256 : 512;
  static constexpr int SMEM = S * STAGE + 1024 + 256;  // + alignment slack + barriers
  static_assert(S >= 2, "at least two pipeline stages");
  static_assert(BN % 16 == 0 && BN >= 16 && BN <= 256, "M=128 MMA needs N % 16 == 0, N <= 256");
};

struct Args {
  int rows;              // valid rows of A per batch (tensor extent)
  int n_valid;           // valid columns of the output (rows of B per batch)
  int k_chunks;          // ceil(K / BK)
  float scale;
  float2 *out;           // interleaved complex; element (row, col) of batch b at
  long long ld_row;      //   out[b * out_bstride + row * ld_row + col * ld_col]
  long long ld_col;      //   (ld_row = 1 makes the epilogue's stores coalesced: a lane owns a row)
  long long out_bstride;
  int conj_out;          // store the conjugate of each element
  int out64;             // out holds complex128 elements (same strides, in elements)
  int b_batch_planes;    // 0: B has no batch dimension (z = pp), else z = qlist[b_base + b]*PP + pp
  int b_base;
  const int *qlist;
  int *err;
  int tiles_n, tiles_m, tiles_b;  // output tiles along N, M and the batch (set by the launcher)
};

// The work list of one launch: NG independent GEMMs (operand tensor maps and output
// arguments each), their output tiles numbered consecutively, group g owning tiles
// tile0[g] .. tile0[g + 1] - 1 (n of them in use).  A single GEMM is the list with NG = 1; the
// batched assembly of several systems puts each system's GEMM of one step in a group.
template <int NG>
struct Groups {
  CUtensorMap A[NG], B[NG];
  Args a[NG];
  long long tile0[NG + 1];
  int n;
};

template <int NP, int BN, bool TF = false, int NG = 1>
__global__ void __launch_bounds__(192, 1) k_tc_zgemm(const __grid_constant__ Groups<NG> G) {
  using C = Cfg<NP, BN>;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t *full = (uint64_t *)(smem + C::S * C::STAGE);
  uint64_t *empty = full + C::S;
  uint64_t *tfull = empty + C::S;   // accumulators of a tile are complete (MMA -> epilogue)
  uint64_t *tempty = tfull + 1;     // accumulators drained (epilogue -> MMA)
  uint32_t *tmem_slot = (uint32_t *)(tempty + 1);
  volatile int *abort_flag = (volatile int *)(tmem_slot + 1);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const long long total = G.tile0[G.n];
  // group of work-list tile t; a CTA's tiles only grow, so its group index only advances
  // (a single GEMM, NG = 1, indexes its arguments with a constant)
  auto group_of = [&](long long t, int &g) {
    if constexpr (NG > 1)
      while (g + 1 < G.n && t >= G.tile0[g + 1]) g++;
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::S; s++) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    tc::mbar_init(tfull, 1);
    tc::mbar_init(tempty, 128);
    *abort_flag = 0;
    tc::fence_barrier_init();
  }
  if (warp == 0 && lane == 0)
    for (int g = 0; g < G.n; g++) {
      tc::prefetch_tmap(&G.A[g]);
      tc::prefetch_tmap(&G.B[g]);
    }
  if (warp == 1) {
    tc::tmem_alloc(tmem_slot, C::TMEM_COLS);
    tc::tmem_relinquish();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t tm_re = tmem, tm_im = tmem + BN;

  // Persistent: this CTA takes tiles blockIdx.x, blockIdx.x + gridDim.x, ...; tile t is
  // (n, m, b) with n fastest, so CTAs running together share the B operand of one batch.
  // The producer runs ahead through the stage ring across tile boundaries, and the epilogue
  // of tile t drains the accumulators while the producer already loads tile t + gridDim.x.
  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer ----------------
    int it = 0, g = 0;
    bool ok = true;
    for (long long t = blockIdx.x; t < total && ok; t += gridDim.x) {
      group_of(t, g);
      const Args args = G.a[NG == 1 ? 0 : g];  // a register copy: the stores below cannot alias it
      const int lt = (int)(t - G.tile0[NG == 1 ? 0 : g]);
      const int n0 = (lt % args.tiles_n) * BN, m0 = ((lt / args.tiles_n) % args.tiles_m) * BM;
      const int b = lt / (args.tiles_n * args.tiles_m);
      const int zb = args.b_batch_planes ? args.qlist[args.b_base + b] * C::PP : 0;
      for (int kc = 0; kc < args.k_chunks; kc++, it++) {
        const int s = it % C::S;
        if (it >= C::S && !tc::mbar_wait_bounded(&empty[s], ((it / C::S) & 1) ^ 1, WAIT_LIMIT)) {
          atomicOr(args.err, 2);
          *abort_flag = 1;
          ok = false;
          break;
        }
        if (*abort_flag) {
          ok = false;
          break;
        }
        uint8_t *st = smem + s * C::STAGE;
        tc::mbar_arrive_expect_tx(&full[s], C::STAGE);
        for (int pp = 0; pp < C::PP; pp++) {
          tc::tma_load_3d(st + pp * A_TILE, &G.A[NG == 1 ? 0 : g], &full[s], kc * bk_elems<TF>(), m0, b * C::PP + pp);
          tc::tma_load_3d(st + C::PP * A_TILE + pp * C::B_TILE, &G.B[NG == 1 ? 0 : g], &full[s], kc * bk_elems<TF>(), n0,
                          zb + pp);
        }
      }
    }
    // every copy this CTA started lands before the CTA can exit
    for (int k = it - C::S < 0 ? 0 : it - C::S; k < it; k++)
      if (!tc::mbar_wait_bounded(&full[k % C::S], (k / C::S) & 1, WAIT_LIMIT)) atomicOr(G.a[NG == 1 ? 0 : g].err, 2);
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer ----------------
    constexpr uint32_t IPOS = tc::idesc<TF>(BM, BN, false);
    constexpr uint32_t INEG = tc::idesc<TF>(BM, BN, true);
    int it = 0, tcount = 0, g = 0;
    bool ok = true;
    for (long long t = blockIdx.x; t < total && ok; t += gridDim.x, tcount++) {
      group_of(t, g);
      const Args args = G.a[NG == 1 ? 0 : g];  // a register copy: the stores below cannot alias it
      if (*abort_flag) break;
      if (tcount > 0 && !tc::mbar_wait_bounded(tempty, (tcount - 1) & 1, 4 * WAIT_LIMIT)) {
        atomicOr(args.err, 2);
        *abort_flag = 1;
        break;
      }
      tc::tc_fence_after();
      uint32_t acc_r = 0, acc_i = 0;
      for (int kc = 0; kc < args.k_chunks; kc++, it++) {
        const int s = it % C::S;
        if (!tc::mbar_wait_bounded(&full[s], (it / C::S) & 1, WAIT_LIMIT)) {
          atomicOr(args.err, 2);
          *abort_flag = 1;
          ok = false;
          break;
        }
        if (*abort_flag) {
          ok = false;
          break;
        }
        tc::tc_fence_after();
        const uint32_t sa = tc::smem_u32(smem + s * C::STAGE);
        const uint32_t sb = sa + C::PP * A_TILE;
        // two MMAs per 64-byte row: K = 16 bf16 or 8 tf32 each (32 bytes)
#pragma unroll
        for (int k16 = 0; k16 < ROWB / 32; k16++) {
#pragma unroll
          for (int pa = 0; pa < NP; pa++) {
#pragma unroll
            for (int pb = 0; pb < NP; pb++) {
              if (pa + pb > NP - 1) continue;
              const uint64_t ar = tc::smem_desc(sa + (2 * pa) * A_TILE + k16 * 32, 16, 8 * ROWB, tc::SWZ_64B);
              const uint64_t ai = tc::smem_desc(sa + (2 * pa + 1) * A_TILE + k16 * 32, 16, 8 * ROWB, tc::SWZ_64B);
              const uint64_t br = tc::smem_desc(sb + (2 * pb) * C::B_TILE + k16 * 32, 16, 8 * ROWB, tc::SWZ_64B);
              const uint64_t bi = tc::smem_desc(sb + (2 * pb + 1) * C::B_TILE + k16 * 32, 16, 8 * ROWB, tc::SWZ_64B);
              tc::mma<TF>(tm_re, ar, br, IPOS, acc_r);
              acc_r = 1;
              tc::mma<TF>(tm_re, ai, bi, INEG, 1);
              tc::mma<TF>(tm_im, ar, bi, IPOS, acc_i);
              acc_i = 1;
              tc::mma<TF>(tm_im, ai, br, IPOS, 1);
            }
          }
        }
        tc::mma_commit(&empty[s]);
      }
      tc::mma_commit(tfull);  // also after an abort, so the epilogue is released
    }
  } else if (warp >= 2) {
    // ---------------- epilogue: TMEM -> registers -> global ----------------
    const int quarter = warp % 4;
    const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
    int tcount = 0, g = 0;
    for (long long t = blockIdx.x; t < total; t += gridDim.x, tcount++) {
      group_of(t, g);
      const Args args = G.a[NG == 1 ? 0 : g];  // a register copy: the stores below cannot alias it
      const bool ok = !*abort_flag && tc::mbar_wait_bounded(tfull, tcount & 1, 4 * WAIT_LIMIT);
      if (!ok) {
        atomicOr(args.err, 2);
        *abort_flag = 1;
        break;
      }
      tc::tc_fence_after();
      const int lt = (int)(t - G.tile0[NG == 1 ? 0 : g]);
      const int n0 = (lt % args.tiles_n) * BN, m0 = ((lt / args.tiles_n) % args.tiles_m) * BM;
      const int b = lt / (args.tiles_n * args.tiles_m);
      const int row = m0 + quarter * 32 + lane;
      const long long orow = (long long)b * args.out_bstride + (long long)row * args.ld_row;
      const bool row_ok = row < args.rows;
      const float sim = args.conj_out ? -args.scale : args.scale;
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 16) {
        uint32_t rr[16], ri[16];
        tc::tmem_ld16(tm_re + lane_off + c0, rr);
        tc::tmem_ld16(tm_im + lane_off + c0, ri);
        tc::tmem_ld_wait();
        if (row_ok) {
#pragma unroll
          for (int j = 0; j < 16; j++) {
            const int col = n0 + c0 + j;
            if (col < args.n_valid) {
              const float re = args.scale * __uint_as_float(rr[j]), im = sim * __uint_as_float(ri[j]);
              if (args.out64)
                reinterpret_cast<double2 *>(args.out)[orow + col * args.ld_col] = make_double2(re, im);
              else
                args.out[orow + col * args.ld_col] = make_float2(re, im);
            }
          }
        }
      }
      tc::tc_fence_before();
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(tempty)) : "memory");
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, C::TMEM_COLS);
  }
}

}  // namespace tcg
