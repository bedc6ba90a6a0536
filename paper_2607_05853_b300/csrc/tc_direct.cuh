// Direct term of the Hamiltonian in one persistent tensor-core kernel (sm_103a):
//
//   T = M_vv W(q)                      (tcgen05, bf16 or tf32 pieces, FP32 accumulation in tensor memory)
//   D = T M_cc^T   per pair (k1, k2 = k1 - q),   H block (k1, k2) += -D / N_k   (and its mirror)
//
// the two contractions of Eq. W_LRI's direct kernel, with T never leaving the SM.  One tile
// holds the rows (k1, i, j) of P whole pairs (P = floor(128 / Nv^2)) and every column nu of T
// (BN >= N_aux), so the epilogue finishes D for those pairs from tensor memory alone.
//
// The shared-memory ring carries one sequence of items per tile: the tile's K chunks of the
// GEMM operands (consumed by the MMA warp), then the tile's M_cc rows in slices of NUI columns,
// one TMA box {NUI, Nc^2, P} each (consumed by the epilogue warps).  Each item takes stage it % S; the producer waits for the
// stage to be released (by the MMA's commit or by one epilogue thread) before refilling it.
// The epilogue releases the accumulators as soon as its last M_cc slice is done and then
// adds D to H (read-modify-write: the exchange GEMM wrote every element first), so the next
// tile's operand loads and MMAs overlap the H traffic.
//
// Warp roles: 0 TMA / bulk-copy producer, 1 tensor-memory allocation and MMA issue, 2-9
// epilogue: warp w reads tensor-memory lanes 32 (w % 4) .. + 31 (one T row per thread), and the
// two warps of a lane quarter split the pair's Nc^2 columns of D, so each SM sub-partition has
// two epilogue warps to hide the latencies of its FP32 contraction.
// Every barrier wait is bounded; a timeout sets the device error word and the CTA winds down.
#pragma once

#include "tc_gemm.cuh"

namespace tcd {

using tcg::A_TILE;
using tcg::BM;
using tcg::ROWB;
using tcg::WAIT_LIMIT;

constexpr int EPI_WARPS = 8;
constexpr int THREADS = 32 * (2 + EPI_WARPS);

// Epilogue warps' named barrier (warps 2-9 only).
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 2, %0;" ::"n"(32 * EPI_WARPS) : "memory"); }

template <int NP, int BN>
struct DCfg {
  static constexpr int PP = 2 * NP;
  static constexpr int B_TILE = BN * ROWB;
  static constexpr int STAGE = PP * (A_TILE + B_TILE);
  static constexpr int S = tcg::SMEM_BUDGET / STAGE < 8 ? tcg::SMEM_BUDGET / STAGE : 8;
  static constexpr int TMEM_COLS = 2 * BN <= 32 ? 32 : 2 * BN <= 64 ? 64 : 2 * BN <= 128 ? 128 : 2 * BN <= 256 ? 256 : 512;
  static constexpr int SMEM = S * STAGE + 1024 + 256;
  static_assert(S >= 2, "at least two pipeline stages");
  static_assert(BN % 16 == 0 && BN >= 16 && BN <= 256, "M=128 MMA needs N % 16 == 0, N <= 256");
};

struct DArgs {
  int nv;                 // valence bands of the window (rows per pair = nv^2)
  int pairs;              // pairs per tile; a tile covers rows m0 .. m0 + pairs nv^2 - 1
  int rows;               // rows of M_vv per q (N_k nv^2)
  int tiles_m, tiles_b;   // tiles per q, q values in this launch
  int k_chunks;           // ceil(N_aux / K per stage): 32 bf16 or 16 tf32 (TF)
  int naux, naux_pad;     // columns of T; M_cc row length in the slab buffer (multiple of 16)
  int nui;                // M_cc columns per ring item (multiple of 16)
  int n_mitems;           // ceil(naux_pad / nui)
  const float2 *Mc;       // M_cc, [q][k1][a b][nu (naux_pad)] complex64 (read through tmM)
  const int *qlist;       // transfer of batch b: qlist[b_base + b]
  int b_base;
  int n1, n2, n3;
  const double *eqp;      // [N_k][nv + nc] quasiparticle energies (diagonal, q = 0 only)
  long long dim;
  float2 *H;              // complex64 H, or
  double2 *H64;           // complex128 H (then H is null)
  int *err;
  // matrix-free form (MF): the block is applied to x instead of added to H
  const double2 *x;       // [n_pol][..] complex128, polarisation p at x + p xs
  long long xs;
  int n_pol, nqs;         // vectors; q stride of fwd / bwd
  double2 *fwd, *bwd;     // [n_pol][nqs][N_k][nv nc], summed into (zeroed before the launch)
};

__device__ __forceinline__ int d_kdiff(int k1, int q, int n1, int n2, int n3) {
  const int a1 = k1 / (n2 * n3), a2 = (k1 / n3) % n2, a3 = k1 % n3;
  const int b1 = q / (n2 * n3), b2 = (q / n3) % n2, b3 = q % n3;
  int c1 = a1 - b1; if (c1 < 0) c1 += n1;
  int c2 = a2 - b2; if (c2 < 0) c2 += n2;
  int c3 = a3 - b3; if (c3 < 0) c3 += n3;
  return (c1 * n2 + c2) * n3 + c3;
}

__device__ __forceinline__ bool d_self_conj(int q, int n1, int n2, int n3) {
  const int a1 = q / (n2 * n3), a2 = (q / n3) % n2, a3 = q % n3;
  return (n1 - a1) % n1 == a1 && (n2 - a2) % n2 == a2 && (n3 - a3) % n3 == a3;
}

// H block (k1, k2) += -D / N_k and its mirror (k2, k1) += conj(-D / N_k) for the D columns
// (a, b) = half Nc^2 / 2 + e of one row (k1, i, j) of a q's tile, D[e] = acc1[e] (mr, mi) tr
// sums and acc2[e] (mr, mi) ti sums; the q = 0 diagonal sums in FP64 with E_c - E_v.  For a
// complex128 H the D contribution is added in FP64.
template <int NC>
__device__ __forceinline__ void d_apply_h(const DArgs &args, const unsigned long long (&acc1)[NC * NC / 2],
                                          const unsigned long long (&acc2)[NC * NC / 2], int row, int b, int half) {
  constexpr int HALF = NC * NC / 2;
  const double inv = 1.0 / ((double)args.n1 * args.n2 * args.n3);
  const float invf = (float)inv;
  const int nb = args.nv + NC, rpp = args.nv * args.nv;
  const int q = args.qlist[args.b_base + b];
  const int k1 = row / rpp, ij = row % rpp, i = ij / args.nv, j = ij % args.nv;
  const int k2 = d_kdiff(k1, q, args.n1, args.n2, args.n3);
  const bool mirror = !d_self_conj(q, args.n1, args.n2, args.n3);
  const int nvc = args.nv * NC;
#pragma unroll
  for (int e = 0; e < HALF; e++) {
    const int ab = half * HALF + e, a = ab / NC, bb = ab % NC;
    const float2 x1 = tc::up2(acc1[e]), x2 = tc::up2(acc2[e]);
    const float dr = x1.x - x2.y, di = x1.y + x2.x;
    const int ia = i * NC + a, jb = j * NC + bb;
    const long long ih = ((long long)k1 * nvc + ia) * args.dim + (long long)k2 * nvc + jb;
    const long long im = ((long long)k2 * nvc + jb) * args.dim + (long long)k1 * nvc + ia;
    if (args.H64) {
      double2 hv = args.H64[ih];
      hv.x -= inv * (double)dr;
      hv.y -= inv * (double)di;
      if (q == 0 && ia == jb) hv.x += args.eqp[(long long)k1 * nb + args.nv + a] - args.eqp[(long long)k1 * nb + i];
      args.H64[ih] = hv;
      if (mirror) {
        double2 mv = args.H64[im];
        mv.x -= inv * (double)dr;
        mv.y += inv * (double)di;
        args.H64[im] = mv;
      }
      continue;
    }
    float2 *hp = args.H + ih;
    const float2 hx = *hp;
    float2 hv = make_float2(fmaf(-invf, dr, hx.x), fmaf(-invf, di, hx.y));
    if (q == 0 && ia == jb)
      hv.x = (float)((double)hx.x - inv * (double)dr + args.eqp[(long long)k1 * nb + args.nv + a] -
                     args.eqp[(long long)k1 * nb + i]);
    *hp = hv;
    if (mirror) {
      float2 *hm = args.H + im;
      const float2 mx = *hm;
      *hm = make_float2(fmaf(-invf, dr, mx.x), fmaf(invf, di, mx.y));
    }
  }
}

// The work list of one launch: NG systems' q-slabs (operand, W and M_cc tensor maps and
// arguments each), their tiles numbered consecutively, group g owning tiles tile0[g] ..
// tile0[g + 1] - 1 (n groups in use); a single slab is the list with NG = 1.
template <int NG>
struct DGroups {
  CUtensorMap A[NG], B[NG], M[NG];
  DArgs a[NG];
  long long tile0[NG + 1];
  int n;
};

// MF: the matrix-free product's form.  Each pair block D is applied as soon as it is formed,
// fwd[p][qq][k1] += D x_p[k2] and, for a mirrored transfer, bwd[p][qq][k2] += D^dagger x_p[k1],
// with no H; for Nv = 2 or 4, whose pairs are rpp consecutive lanes of one warp, so that the
// sums over j and over i are warp shuffles (the two column halves and the q-slab's pairs meet
// in FP64 atomic adds).
template <int NP, int BN, int NC, bool TF = false, int NG = 1, bool MF = false>
__global__ void __launch_bounds__(THREADS, 1) k_tc_direct(const __grid_constant__ DGroups<NG> G) {
  using C = DCfg<NP, BN>;
  constexpr int NCC = NC * NC, HALF = NCC / 2;  // D columns (a, b) per epilogue warp

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
  // group of work-list tile t (a CTA's tiles only grow; a single slab indexes with a constant)
  auto group_of = [&](long long t, int &g) {
    if constexpr (NG > 1)
      while (g + 1 < G.n && t >= G.tile0[g + 1]) g++;
  };
#define GI (NG == 1 ? 0 : g)

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::S; s++) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    tc::mbar_init(tfull, 1);
    tc::mbar_init(tempty, 32 * EPI_WARPS);
    *abort_flag = 0;
    tc::fence_barrier_init();
  }
  if (warp == 0 && lane == 0)
    for (int g = 0; g < G.n; g++) {
      tc::prefetch_tmap(&G.A[g]);
      tc::prefetch_tmap(&G.B[g]);
      tc::prefetch_tmap(&G.M[g]);
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

  if (warp == 0 && lane == 0) {
    // ---------------- producer: operand K chunks, then the tile's M_cc slices ----------------
    int it = 0, g = 0;
    bool ok = true;
    for (long long t = blockIdx.x; t < total && ok; t += gridDim.x) {
      group_of(t, g);
      const DArgs args = G.a[GI];  // a register copy: the stores below cannot alias it
      const int items = args.k_chunks + args.n_mitems;  // ring items per tile
      const int rpp = args.nv * args.nv;                // rows per pair
      const int lt = (int)(t - G.tile0[GI]);
      const int m = lt % args.tiles_m, b = lt / args.tiles_m;
      const int m0 = m * args.pairs * rpp;
      const int q = args.qlist[args.b_base + b];
      const int k1_0 = m0 / rpp;
      for (int item = 0; item < items; item++, it++) {
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
        if (item < args.k_chunks) {
          const int kc = item;
          tc::mbar_arrive_expect_tx(&full[s], C::STAGE);
          for (int pp = 0; pp < C::PP; pp++) {
            tc::tma_load_3d(st + pp * A_TILE, &G.A[GI], &full[s], kc * tcg::bk_elems<TF>(), m0, b * C::PP + pp);
            tc::tma_load_3d(st + C::PP * A_TILE + pp * C::B_TILE, &G.B[GI], &full[s], kc * tcg::bk_elems<TF>(), 0,
                            q * C::PP + pp);
          }
        } else {
          // columns nu0 .. nu0 + nui - 1 of M_cc for the tile's pairs, one TMA box
          // {nui, Nc^2, pairs}: smem [pair][ab][nu] (columns or pairs past the tensor zero-filled)
          const int nu0 = (item - args.k_chunks) * args.nui;
          tc::mbar_arrive_expect_tx(&full[s], (uint32_t)args.pairs * NCC * args.nui * 8);
          tc::tma_load_3d(st, &G.M[GI], &full[s], nu0, 0, b * (args.rows / rpp) + k1_0);
        }
      }
    }
    // every copy this CTA started lands before the CTA can exit
    for (int k = it - C::S < 0 ? 0 : it - C::S; k < it; k++)
      if (!tc::mbar_wait_bounded(&full[k % C::S], (k / C::S) & 1, WAIT_LIMIT)) atomicOr(G.a[GI].err, 2);
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer ----------------
    constexpr uint32_t IPOS = tc::idesc<TF>(BM, BN, false);
    constexpr uint32_t INEG = tc::idesc<TF>(BM, BN, true);
    int it = 0, tcount = 0, g = 0;
    bool ok = true;
    for (long long t = blockIdx.x; t < total && ok; t += gridDim.x, tcount++) {
      group_of(t, g);
      const DArgs args = G.a[GI];
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
#pragma unroll
        for (int k16 = 0; k16 < ROWB / 32; k16++) {  // two MMAs (32 bytes of K each) per row
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
      it += args.n_mitems;    // the tile's M_cc items belong to the epilogue
    }
  } else if (warp >= 2) {
    // ---------------- epilogue: D = T M_cc^T from tensor memory and the staged M_cc ----------
    const int quarter = warp % 4, half = (warp - 2) / 4;   // lane quarter; which half of D's columns
    const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
    int tcount = 0, it = 0, g = 0;
    // Control flow is the same in every epilogue thread whatever the waits return (each tile's
    // items each end in the warps' named barrier); after an abort the waits are skipped.
    for (long long t = blockIdx.x; t < total; t += gridDim.x, tcount++) {
      group_of(t, g);
      const DArgs args = G.a[GI];  // a register copy: the H stores below cannot alias it
      const float invf = (float)(1.0 / ((double)args.n1 * args.n2 * args.n3));
      const int rpp = args.nv * args.nv;
      it += args.k_chunks;
      bool ok = !*abort_flag && tc::mbar_wait_bounded(tfull, tcount & 1, 4 * WAIT_LIMIT);
      if (!ok) {
        atomicOr(args.err, 2);
        *abort_flag = 1;
      }
      tc::tc_fence_after();
      const int lt = (int)(t - G.tile0[GI]);
      const int m = lt % args.tiles_m, b = lt / args.tiles_m;
      const int m0 = m * args.pairs * rpp;
      const int lrow = quarter * 32 + lane;                 // row of the tile (tensor-memory lane)
      const int row = m0 + lrow;                            // (k1, i, j) within this q
      const bool row_ok = lrow < args.pairs * rpp && row < args.rows;
      const int pr = lrow / rpp;                            // pair of the tile
      // D[e], e = half HALF + e', as re / im accumulators: acc1 = sum (mr, mi) tr, acc2 = sum (mr, mi) ti
      unsigned long long acc1[HALF], acc2[HALF];
#pragma unroll
      for (int e = 0; e < HALF; e++) acc1[e] = acc2[e] = 0ull;
      for (int mi = 0; mi < args.n_mitems; mi++, it++) {
        const int s = it % C::S;
        const bool got = ok && !*abort_flag && tc::mbar_wait_bounded(&full[s], (it / C::S) & 1, WAIT_LIMIT);
        if (ok && !got) {
          atomicOr(args.err, 2);
          *abort_flag = 1;
        }
        ok = got;
        const int nu0 = mi * args.nui;
        const int nn = min(args.nui, args.naux - nu0);     // padded columns carry T = 0
        // this warp's (a, b) rows of the pair: [ab][nu], nui columns each
        const float2 *mcs = reinterpret_cast<const float2 *>(smem + s * C::STAGE) +
                            ((size_t)pr * NCC + half * HALF) * args.nui;
        // T columns c0 .. c0 + 15 of this slice times the pair's M_cc rows: columns in pairs
        // (nu, nu + 1); T is zero past N_aux, and the M_cc column paired with the last one of an
        // odd N_aux is ignored
        auto fma_group = [&](const uint32_t (&rr)[16], const uint32_t (&ri)[16], int c0) {
          const int cmax = min(16, nn - c0);
#pragma unroll
          for (int u = 0; u < 16; u += 2) {
            if (u >= cmax) break;
            const float tr0 = __uint_as_float(rr[u]), ti0 = __uint_as_float(ri[u]);
            const float tr1 = __uint_as_float(rr[u + 1]), ti1 = __uint_as_float(ri[u + 1]);
            const unsigned long long TR0 = tc::pk2(tr0, tr0), TI0 = tc::pk2(ti0, ti0);
            const unsigned long long TR1 = tc::pk2(tr1, tr1), TI1 = tc::pk2(ti1, ti1);
#pragma unroll
            for (int e = 0; e < HALF; e++) {
              const float4 mm = *reinterpret_cast<const float4 *>(mcs + (size_t)e * args.nui + c0 + u);
              const bool tail = u + 1 >= cmax;
              const unsigned long long m0v = tc::pk2(mm.x, mm.y),
                                       m1v = tc::pk2(tail ? 0.f : mm.z, tail ? 0.f : mm.w);
              tc::ffma2(acc1[e], m0v, TR0);
              tc::ffma2(acc2[e], m0v, TI0);
              tc::ffma2(acc1[e], m1v, TR1);
              tc::ffma2(acc2[e], m1v, TI1);
            }
          }
        };
        if constexpr (NC <= 4 && NG == 1) {
          // tensor-memory loads one 16-column group ahead of the FMAs that use them (the wait
          // covers every load the thread issued before it); Nc = 6 and the batched work list
          // keep one group in flight (their accumulators and group arguments leave no
          // registers for a second)
          uint32_t ra[16], ia[16], rb[16], ib[16];
          tc::tmem_ld16(tm_re + lane_off + nu0, ra);
          tc::tmem_ld16(tm_im + lane_off + nu0, ia);
          for (int c0 = 0; c0 < nn; c0 += 32) {
            tc::tmem_ld_wait();
            const bool next1 = c0 + 16 < nn, next2 = c0 + 32 < nn;
            if (next1) {
              tc::tmem_ld16(tm_re + lane_off + nu0 + c0 + 16, rb);
              tc::tmem_ld16(tm_im + lane_off + nu0 + c0 + 16, ib);
            }
            if (ok && row_ok) fma_group(ra, ia, c0);
            tc::tmem_ld_wait();
            if (next2) {
              tc::tmem_ld16(tm_re + lane_off + nu0 + c0 + 32, ra);
              tc::tmem_ld16(tm_im + lane_off + nu0 + c0 + 32, ia);
            }
            if (next1 && ok && row_ok) fma_group(rb, ib, c0 + 16);
          }
        } else {
          for (int c0 = 0; c0 < nn; c0 += 16) {
            uint32_t rr[16], ri[16];
            tc::tmem_ld16(tm_re + lane_off + nu0 + c0, rr);
            tc::tmem_ld16(tm_im + lane_off + nu0 + c0, ri);
            tc::tmem_ld_wait();
            if (ok && row_ok) fma_group(rr, ri, c0);
          }
        }
        // the epilogue warps are done with this slice: one thread releases the stage
        epi_sync();
        if (threadIdx.x == 64) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(&empty[s])) : "memory");
      }
      // accumulators drained: the next tile's MMAs may start while H is updated
      tc::tc_fence_before();
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(tempty)) : "memory");
      if constexpr (MF) {
        // every lane takes part in the shuffles; dead rows contribute zero and add nothing
        const bool live = ok && row_ok;
        const int rowc = live ? row : 0;
        const int q = args.qlist[args.b_base + b];
        const int k1 = rowc / rpp, ij = rowc % rpp, i = ij / args.nv, j = ij % args.nv;
        const int k2 = d_kdiff(k1, q, args.n1, args.n2, args.n3);
        const bool mirror = !d_self_conj(q, args.n1, args.n2, args.n3);
        const int nvc = args.nv * NC, nk = args.n1 * args.n2 * args.n3;
        float2 dv[HALF];
#pragma unroll
        for (int e = 0; e < HALF; e++) {
          const float2 x1 = tc::up2(acc1[e]), x2 = tc::up2(acc2[e]);
          dv[e] = live ? make_float2(-invf * (x1.x - x2.y), -invf * (x1.y + x2.x)) : make_float2(0.f, 0.f);
        }
        for (int p = 0; p < args.n_pol; p++) {
          const double2 *xk2 = args.x + p * args.xs + (long long)k2 * nvc + j * NC;  // x[k2][(j, b)]
          const double2 *xk1 = args.x + p * args.xs + (long long)k1 * nvc + i * NC;  // x[k1][(i, a)]
          double2 *fw = args.fwd + (((long long)p * args.nqs + b) * nk + k1) * nvc + i * NC + half * (NC / 2);
          double2 *bw = args.bwd + (((long long)p * args.nqs + b) * nk + k2) * nvc + j * NC;
#pragma unroll
          for (int aa = 0; aa < NC / 2; aa++) {  // row (i, a = half NC/2 + aa) of D times x[k2]
            double fr = 0.0, fi = 0.0;
#pragma unroll
            for (int bb = 0; bb < NC; bb++) {
              const float2 d = dv[aa * NC + bb];
              const double2 xv = xk2[bb];
              fr += (double)d.x * xv.x - (double)d.y * xv.y;
              fi += (double)d.x * xv.y + (double)d.y * xv.x;
            }
            for (int o = 1; o < args.nv; o <<= 1) {  // sum over j
              fr += __shfl_xor_sync(0xffffffffu, fr, o);
              fi += __shfl_xor_sync(0xffffffffu, fi, o);
            }
            if (live && j == 0) {
              atomicAdd(&fw[aa].x, fr);
              atomicAdd(&fw[aa].y, fi);
            }
          }
#pragma unroll
          for (int bb = 0; bb < NC; bb++) {  // column (j, b) of D, conjugated, times x[k1]
            double gr = 0.0, gi = 0.0;
#pragma unroll
            for (int aa = 0; aa < NC / 2; aa++) {
              const float2 d = dv[aa * NC + bb];
              const double2 xv = xk1[half * (NC / 2) + aa];
              gr += (double)d.x * xv.x + (double)d.y * xv.y;
              gi += (double)d.x * xv.y - (double)d.y * xv.x;
            }
            for (int o = args.nv; o < rpp; o <<= 1) {  // sum over i
              gr += __shfl_xor_sync(0xffffffffu, gr, o);
              gi += __shfl_xor_sync(0xffffffffu, gi, o);
            }
            if (live && mirror && i == 0) {
              atomicAdd(&bw[bb].x, gr);
              atomicAdd(&bw[bb].y, gi);
            }
          }
        }
        continue;
      }
      if (!ok || !row_ok) continue;
      d_apply_h<NC>(args, acc1, acc2, row, b, half);
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, C::TMEM_COLS);
  }
#undef GI
}

}  // namespace tcd
