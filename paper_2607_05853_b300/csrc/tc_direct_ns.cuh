// Direct term of the Hamiltonian, the same two contractions as k_tc_direct (Eq. W_LRI's
// direct kernel: T = M_vv W(q) on tcgen05, D = T M_cc^T per pair, H += -D / N_k and its
// mirror), with the accumulators split by T's columns so that the FP32 epilogue runs under
// the MMAs.
//
// T's N_aux (<= 160) columns are taken in two halves nu = 0..79 and 80..159, each with its own
// tensor-memory buffer (real and imaginary parts, 2 x 80 columns).  The MMA warp computes half
// 0 of a tile, then half 1, then half 0 of the next tile; the epilogue contracts half 0 of a
// tile while the MMAs of its half 1 run, and half 1 (then the H update) while the MMAs of the
// next tile's half 0 run.  The cost is that the tile's M_vv K chunks are streamed twice (once
// per half, the second time from L2).
//
// Two rings in shared memory, each with its own producer thread, so that neither waits on the
// other's consumer: operand K chunks of one half-tile (A rows and 80 rows of B per piece plane)
// for the MMA warp, and M_cc slices of 16 columns (one TMA box {16, Nc^2, P}) for the
// epilogue warps.  Warp roles: 0 operand producer, 1 tensor-memory allocation and MMA issue,
// 2-9 epilogue (as in k_tc_direct: warp w reads lanes 32 (w % 4) .. + 31, the two warps of a
// lane quarter split the pair's Nc^2 columns of D), 10 M_cc producer.  Every barrier wait is
// bounded; a timeout sets the device error word and the CTA winds down.
#pragma once

#include "tc_direct.cuh"

namespace tcd {

constexpr int NS_HALF = 80;                 // T columns per half
constexpr int NS_MC_COLS = 16;              // M_cc columns per ring item
constexpr int NS_MC_STAGE = 16384;          // bytes per M_cc stage (pairs Nc^2 <= 128)
constexpr int NS_MC_STAGES = 4;
constexpr int NS_THREADS = 32 * (3 + EPI_WARPS);
constexpr int NS_MAX_SMEM = 232448;         // opt-in shared memory per block on sm_103

template <int NP>
struct NsCfg {
  static constexpr int PP = 2 * NP;
  static constexpr int B_HALF = NS_HALF * ROWB;                  // 5 KB per piece plane
  static constexpr int OSTAGE = PP * (A_TILE + B_HALF);
  static constexpr int RING_BUDGET = NS_MAX_SMEM - 1024 - 256 - NS_MC_STAGES * NS_MC_STAGE;
  static constexpr int SO = RING_BUDGET / OSTAGE < 6 ? RING_BUDGET / OSTAGE : 6;
  static constexpr int SMEM = SO * OSTAGE + NS_MC_STAGES * NS_MC_STAGE + 1024 + 256;
  static_assert(SO >= 2, "at least two operand stages");
  static_assert(SMEM <= NS_MAX_SMEM, "shared memory");
  static_assert(B_HALF % 1024 == 0 && OSTAGE % 1024 == 0, "swizzle atoms stay 1024-byte aligned");
};

// Operand ring items per tile: 2 x k_chunks (half 0's chunks, then half 1's).  M_cc ring items
// per tile: the 16-column slices of each half below naux_pad, half 0's first.
__device__ __forceinline__ int ns_mitems(int naux_pad, int h) {
  const int lo = h * NS_HALF, hi = min(lo + NS_HALF, naux_pad);
  return hi > lo ? (hi - lo + NS_MC_COLS - 1) / NS_MC_COLS : 0;
}

// G.B[0]: W(q) pieces with a box of NS_HALF rows; G.M[0]: M_cc with a box {16, Nc^2, pairs}.
template <int NP, int NC, bool TF = false>
__global__ void __launch_bounds__(NS_THREADS, 1) k_tc_direct_ns(const __grid_constant__ DGroups<1> G) {
  using C = NsCfg<NP>;
  constexpr int NCC = NC * NC, HALF = NCC / 2;

  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t *mring = smem + C::SO * C::OSTAGE;
  uint64_t *ofull = (uint64_t *)(mring + NS_MC_STAGES * NS_MC_STAGE);
  uint64_t *oempty = ofull + C::SO;
  uint64_t *mfull = oempty + C::SO;
  uint64_t *mempty = mfull + NS_MC_STAGES;
  uint64_t *tfull = mempty + NS_MC_STAGES;   // [2] a half's accumulators are complete
  uint64_t *tempty = tfull + 2;              // [2] a half's accumulators are drained
  uint32_t *tmem_slot = (uint32_t *)(tempty + 2);
  volatile int *abort_flag = (volatile int *)(tmem_slot + 1);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const DArgs &ga = G.a[0];
  const long long total = G.tile0[1];

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::SO; s++) {
      tc::mbar_init(&ofull[s], 1);
      tc::mbar_init(&oempty[s], 1);
    }
    for (int s = 0; s < NS_MC_STAGES; s++) {
      tc::mbar_init(&mfull[s], 1);
      tc::mbar_init(&mempty[s], EPI_WARPS);
    }
    for (int h = 0; h < 2; h++) {
      tc::mbar_init(&tfull[h], 1);
      tc::mbar_init(&tempty[h], 32 * EPI_WARPS);
    }
    *abort_flag = 0;
    tc::fence_barrier_init();
  }
  if (warp == 0 && lane == 0) {
    tc::prefetch_tmap(&G.A[0]);
    tc::prefetch_tmap(&G.B[0]);
  }
  if (warp == 10 && lane == 0) tc::prefetch_tmap(&G.M[0]);
  if (warp == 1) {
    tc::tmem_alloc(tmem_slot, 512);
    tc::tmem_relinquish();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;   // half h: real part at column 160 h, imaginary at 160 h + 80

  if (warp == 0 && lane == 0) {
    // ---------------- operand producer: per tile, half 0's K chunks then half 1's ----------------
    const DArgs args = ga;
    const int rpp = args.nv * args.nv;
    int it = 0;
    bool ok = true;
    for (long long t = blockIdx.x; t < total && ok; t += gridDim.x) {
      const int m = (int)(t % args.tiles_m), b = (int)(t / args.tiles_m);
      const int m0 = m * args.pairs * rpp;
      const int q = args.qlist[args.b_base + b];
      for (int h = 0; h < 2 && ok; h++)
        for (int kc = 0; kc < args.k_chunks; kc++, it++) {
          const int s = it % C::SO;
          if (it >= C::SO && !tc::mbar_wait_bounded(&oempty[s], ((it / C::SO) & 1) ^ 1, WAIT_LIMIT)) {
            atomicOr(args.err, 2);
            *abort_flag = 1;
            ok = false;
            break;
          }
          if (*abort_flag) {
            ok = false;
            break;
          }
          uint8_t *st = smem + s * C::OSTAGE;
          tc::mbar_arrive_expect_tx(&ofull[s], C::OSTAGE);
          for (int pp = 0; pp < C::PP; pp++) {
            tc::tma_load_3d(st + pp * A_TILE, &G.A[0], &ofull[s], kc * tcg::bk_elems<TF>(), m0, b * C::PP + pp);
            tc::tma_load_3d(st + C::PP * A_TILE + pp * C::B_HALF, &G.B[0], &ofull[s], kc * tcg::bk_elems<TF>(),
                            h * NS_HALF, q * C::PP + pp);
          }
        }
    }
    // every copy this CTA started lands before the CTA can exit
    for (int k = it - C::SO < 0 ? 0 : it - C::SO; k < it; k++)
      if (!tc::mbar_wait_bounded(&ofull[k % C::SO], (k / C::SO) & 1, WAIT_LIMIT)) atomicOr(args.err, 2);
  } else if (warp == 10 && lane == 0) {
    // ---------------- M_cc producer: per tile, half 0's 16-column slices then half 1's ----------------
    const DArgs args = ga;
    const int rpp = args.nv * args.nv;
    const uint32_t bytes = (uint32_t)args.pairs * NCC * NS_MC_COLS * 8;
    int it = 0;
    bool ok = true;
    for (long long t = blockIdx.x; t < total && ok; t += gridDim.x) {
      const int m = (int)(t % args.tiles_m), b = (int)(t / args.tiles_m);
      const int k1_0 = m * args.pairs;
      for (int h = 0; h < 2 && ok; h++) {
        const int nm = ns_mitems(args.naux_pad, h);
        for (int mi = 0; mi < nm; mi++, it++) {
          const int s = it % NS_MC_STAGES;
          if (it >= NS_MC_STAGES &&
              !tc::mbar_wait_bounded(&mempty[s], ((it / NS_MC_STAGES) & 1) ^ 1, WAIT_LIMIT)) {
            atomicOr(args.err, 2);
            *abort_flag = 1;
            ok = false;
            break;
          }
          if (*abort_flag) {
            ok = false;
            break;
          }
          tc::mbar_arrive_expect_tx(&mfull[s], bytes);
          tc::tma_load_3d(mring + s * NS_MC_STAGE, &G.M[0], &mfull[s], h * NS_HALF + mi * NS_MC_COLS, 0,
                          b * (args.rows / rpp) + k1_0);
        }
      }
    }
    for (int k = it - NS_MC_STAGES < 0 ? 0 : it - NS_MC_STAGES; k < it; k++)
      if (!tc::mbar_wait_bounded(&mfull[k % NS_MC_STAGES], (k / NS_MC_STAGES) & 1, WAIT_LIMIT))
        atomicOr(args.err, 2);
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer: half h of each tile into buffer h ----------------
    const DArgs args = ga;
    constexpr uint32_t IPOS = tc::idesc<TF>(BM, NS_HALF, false);
    constexpr uint32_t INEG = tc::idesc<TF>(BM, NS_HALF, true);
    int it = 0, tcount = 0;
    bool ok = true;
    for (long long t = blockIdx.x; t < total && ok; t += gridDim.x, tcount++) {
      for (int h = 0; h < 2 && ok; h++) {
        if (*abort_flag) {
          ok = false;
          break;
        }
        if (tcount > 0 && !tc::mbar_wait_bounded(&tempty[h], (tcount - 1) & 1, 4 * WAIT_LIMIT)) {
          atomicOr(args.err, 2);
          *abort_flag = 1;
          ok = false;
          break;
        }
        tc::tc_fence_after();
        const uint32_t tm_re = tmem + h * (2 * NS_HALF), tm_im = tm_re + NS_HALF;
        uint32_t acc_r = 0, acc_i = 0;
        for (int kc = 0; kc < args.k_chunks; kc++, it++) {
          const int s = it % C::SO;
          if (!tc::mbar_wait_bounded(&ofull[s], (it / C::SO) & 1, WAIT_LIMIT)) {
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
          const uint32_t sa = tc::smem_u32(smem + s * C::OSTAGE);
          const uint32_t sb = sa + C::PP * A_TILE;
#pragma unroll
          for (int k16 = 0; k16 < ROWB / 32; k16++) {  // two MMAs (32 bytes of K each) per row
#pragma unroll
            for (int pa = 0; pa < NP; pa++) {
#pragma unroll
              for (int pb = 0; pb < NP; pb++) {
                if (pa + pb > NP - 1) continue;
                const uint64_t ar = tc::smem_desc(sa + (2 * pa) * A_TILE + k16 * 32, 16, 8 * ROWB, tc::SWZ_64B);
                const uint64_t ai = tc::smem_desc(sa + (2 * pa + 1) * A_TILE + k16 * 32, 16, 8 * ROWB, tc::SWZ_64B);
                const uint64_t br = tc::smem_desc(sb + (2 * pb) * C::B_HALF + k16 * 32, 16, 8 * ROWB, tc::SWZ_64B);
                const uint64_t bi = tc::smem_desc(sb + (2 * pb + 1) * C::B_HALF + k16 * 32, 16, 8 * ROWB, tc::SWZ_64B);
                tc::mma<TF>(tm_re, ar, br, IPOS, acc_r);
                acc_r = 1;
                tc::mma<TF>(tm_re, ai, bi, INEG, 1);
                tc::mma<TF>(tm_im, ar, bi, IPOS, acc_i);
                acc_i = 1;
                tc::mma<TF>(tm_im, ai, br, IPOS, 1);
              }
            }
          }
          tc::mma_commit(&oempty[s]);
        }
        tc::mma_commit(&tfull[h]);  // also after an abort, so the epilogue is released
      }
    }
  } else if (warp >= 2 && warp < 2 + EPI_WARPS) {
    // ---------------- epilogue: D = T M_cc^T, half by half, from tensor memory ----------------
    const DArgs args = ga;  // a register copy: the H stores below cannot alias it
    const int quarter = warp % 4, half = (warp - 2) / 4;   // lane quarter; which half of D's columns
    const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
    const int rpp = args.nv * args.nv;
    int tcount = 0, it = 0;
    // Control flow is the same in every epilogue thread whatever the waits return; after an
    // abort the waits are skipped and nothing is computed or stored.
    for (long long t = blockIdx.x; t < total; t += gridDim.x, tcount++) {
      const int m = (int)(t % args.tiles_m), b = (int)(t / args.tiles_m);
      const int m0 = m * args.pairs * rpp;
      const int lrow = quarter * 32 + lane;                 // row of the tile (tensor-memory lane)
      const int row = m0 + lrow;                            // (k1, i, j) within this q
      const bool row_ok = lrow < args.pairs * rpp && row < args.rows;
      const int pr = lrow / rpp;                            // pair of the tile
      // D[e], e = half HALF + e', as re / im accumulators: acc1 = sum (mr, mi) tr, acc2 = sum (mr, mi) ti
      unsigned long long acc1[HALF], acc2[HALF];
#pragma unroll
      for (int e = 0; e < HALF; e++) acc1[e] = acc2[e] = 0ull;
      bool ok = !*abort_flag;
      for (int h = 0; h < 2; h++) {
        const bool got = ok && !*abort_flag && tc::mbar_wait_bounded(&tfull[h], tcount & 1, 4 * WAIT_LIMIT);
        if (ok && !got) {
          atomicOr(args.err, 2);
          *abort_flag = 1;
        }
        ok = got;
        tc::tc_fence_after();
        const uint32_t tm_re = tmem + lane_off + h * (2 * NS_HALF), tm_im = tm_re + NS_HALF;
        const int nm = ns_mitems(args.naux_pad, h);
        // slice mi of this half: T columns 16 mi .. 16 mi + 15 of the buffer times the staged
        // M_cc columns nu0 .. nu0 + 15 (nu0 = 80 h + 16 mi) of the pair's (a, b) rows; columns
        // in pairs (nu, nu + 1), those at or past N_aux skipped
        auto slice = [&](const uint32_t (&rr)[16], const uint32_t (&ri)[16], int mi) {
          const int s = it % NS_MC_STAGES;
          const bool g2 = ok && !*abort_flag && tc::mbar_wait_bounded(&mfull[s], (it / NS_MC_STAGES) & 1, WAIT_LIMIT);
          if (ok && !g2) {
            atomicOr(args.err, 2);
            *abort_flag = 1;
          }
          ok = g2;
          const int cmax = min(NS_MC_COLS, args.naux - (h * NS_HALF + mi * NS_MC_COLS));
          const float2 *mcs = reinterpret_cast<const float2 *>(mring + s * NS_MC_STAGE) +
                              ((size_t)pr * NCC + half * HALF) * NS_MC_COLS;
          if (ok && row_ok) {
#pragma unroll
            for (int u = 0; u < NS_MC_COLS; u += 2) {
              if (u >= cmax) break;
              const float tr0 = __uint_as_float(rr[u]), ti0 = __uint_as_float(ri[u]);
              const float tr1 = __uint_as_float(rr[u + 1]), ti1 = __uint_as_float(ri[u + 1]);
              const unsigned long long TR0 = tc::pk2(tr0, tr0), TI0 = tc::pk2(ti0, ti0);
              const unsigned long long TR1 = tc::pk2(tr1, tr1), TI1 = tc::pk2(ti1, ti1);
              const bool tail = u + 1 >= cmax;
#pragma unroll
              for (int e = 0; e < HALF; e++) {
                const float4 mm = *reinterpret_cast<const float4 *>(mcs + (size_t)e * NS_MC_COLS + u);
                const unsigned long long m0v = tc::pk2(mm.x, mm.y),
                                         m1v = tc::pk2(tail ? 0.f : mm.z, tail ? 0.f : mm.w);
                tc::ffma2(acc1[e], m0v, TR0);
                tc::ffma2(acc2[e], m0v, TI0);
                tc::ffma2(acc1[e], m1v, TR1);
                tc::ffma2(acc2[e], m1v, TI1);
              }
            }
          }
          // this warp is done with the slice: its lane 0 releases it (EPI_WARPS arrivals free the stage)
          __syncwarp();
          if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(&mempty[s])) : "memory");
          it++;
        };
        // tensor-memory loads one slice ahead of the FMAs that use them (the wait covers every
        // load the thread issued before it)
        uint32_t ra[16], ia[16], rb[16], ib[16];
        if (nm > 0) {
          tc::tmem_ld16(tm_re, ra);
          tc::tmem_ld16(tm_im, ia);
        }
        for (int mi = 0; mi < nm; mi += 2) {
          tc::tmem_ld_wait();
          if (mi + 1 < nm) {
            tc::tmem_ld16(tm_re + (mi + 1) * NS_MC_COLS, rb);
            tc::tmem_ld16(tm_im + (mi + 1) * NS_MC_COLS, ib);
          }
          slice(ra, ia, mi);
          if (mi + 1 < nm) {
            tc::tmem_ld_wait();
            if (mi + 2 < nm) {
              tc::tmem_ld16(tm_re + (mi + 2) * NS_MC_COLS, ra);
              tc::tmem_ld16(tm_im + (mi + 2) * NS_MC_COLS, ia);
            }
            slice(rb, ib, mi + 1);
          }
        }
        // this half's accumulators are drained: its next MMAs may start
        tc::tc_fence_before();
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(&tempty[h])) : "memory");
      }
      if (!ok || !row_ok) continue;
      d_apply_h<NC>(args, acc1, acc2, row, b, half);
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, 512);
  }
}

}  // namespace tcd
