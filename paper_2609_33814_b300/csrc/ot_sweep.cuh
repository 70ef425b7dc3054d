// Sweep kernels of Dual (O-)BDRS (Algorithm 1, log domain) with the certificate of
// Proposition 3 / Algorithm 2 fused into the column sweep, for sm_103a.
//
// Notation.  A sweep has a "thread side" P (the points whose LSE is computed, R per thread) and a
// "tile side" Q (the points reduced over, streamed through shared memory by TMA bulk copies).
// Row sweep: P = sources x_i, Q = targets y_j.  Column sweep: P = targets, Q = sources.
// With C_pq = kappa ||u_p - w_q||^2 and the tile-side log scaling lv_q (log beta-tilde for the
// row sweep, log alpha-hat for the column sweep), the exponent of Algorithm 1 in base 2 is
//
//     (lv_q - C_pq/eps) log2(e) = z_pq - kappa ||u_p||^2 log2(e) / eps,
//     z_pq = h_q + <A_p, w_q>,   h_q = (lv_q - kappa ||w_q||^2 / eps) log2(e),
//                                A_p = (2 kappa log2(e) / eps) u_p,
//
// so one entry costs d fused multiply-adds for z, one subtraction of the running shift, one exp2
// and one addition: the cost matrix is recomputed in registers and never stored.
//
// Every (point block, split) work item writes a partial (shift, sum[, cost sum]) per point; the
// last CTA to finish a point block merges the splits in a fixed order (deterministic) and runs
// the FP64 epilogue of Algorithm 1 for those points; on the column side the last point block of
// an instance also advances k and, on certificate iterations, finishes the certificate sums.
#pragma once
#include <cfloat>
#include <cmath>
#include <cstdint>
#include <type_traits>

#include "ot_device.cuh"
#include "ot_exp2_poly.cuh"
#include "ot_kernels.cuh"

namespace ot {

constexpr double kLog2e = 1.4426950408889634074;
constexpr double kLn2 = 0.69314718055994530942;
constexpr float kTau = 32.0f;            // lazy-rescale threshold (base-2 units above the shift)
// A validated hint E (see Inst::hint) starts a micro-split's running shift at floor(E) - kHintMargin
// (never below its first chunk's maximum), so the terms near the row's maximum stay below 2^(8 +
// the hint's error) and a tile sum only overflows 2^64 if the hint is ~48 too low.  Terms more
// than 126 below the shift flush to zero: at most m 2^(E - L - 134) of the total 2^L, which the
// epilogue keeps below 2^-38 by rejecting a sweep whose hint exceeded L by more than kHintGuard.
constexpr float kHintMargin = 8.0f;
constexpr float kHintTol = 16.0f;
constexpr float kHintGuard = 72.0f;
constexpr float kPadH = -1.0e30f;        // h of padding points: contributes exp2(-1e30) = 0
// Coordinate runs of 2-D packs (see tile_runs_kernel): a tile's free pack component (kNComp - 1)
// holds, in its first entry, 1 + k when coordinate k is constant within every aligned group of
// kRunCols points of the tile, else 0.
constexpr int kRunCols = 16;
// The fast sweeps' chunk loop is unrolled twice (the exp2 and sums of one chunk overlap the next
// chunk's exponents) and the first chunk of a micro-split, which sets the running shifts, runs
// outside it.  Measured on B300 against no unrolling and no peeling: +1.5 % (256^2, 512^2 grids),
// +10 % (2^18 RGB points).
#ifndef OT_CHUNK_UNROLL
#define OT_CHUNK_UNROLL 2
#endif
#ifndef OT_PEEL_FRESH
#define OT_PEEL_FRESH 1
#endif
constexpr int kChunkUnroll = OT_CHUNK_UNROLL;
constexpr bool kPeelFresh = OT_PEEL_FRESH != 0;

// ---------------------------------------------------------------------------------------------
// Small helpers
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ void kahan_add(float& s, float& c, float x) {
  const float y = __fsub_rn(x, c);
  const float t = __fadd_rn(s, y);
  c = __fsub_rn(__fsub_rn(t, s), y);
  s = t;
}


// The exponent z_pq - shift (base 2) in float-float: h = hh + hl, A = Ah + Al, the products
// Ah_k w_k and the partial sums taken exactly by error-free transforms, then rounded once.  Its
// error is the FP32 rounding of the (small) result, not of the 1/eps-sized terms it is made of.
template <int D>
__device__ __forceinline__ float comp_exponent(float hh, float hl, const float (&w)[D], const float (&Ah)[D],
                                               const float (&Al)[D], float shift) {
  float sb, e0;
  two_sum(hh, -shift, sb, e0);
  float lo = __fadd_rn(e0, hl);
#pragma unroll
  for (int k = 0; k < D; ++k) {
    float pp, pe, s2, e2;
    two_prod(Ah[k], w[k], pp, pe);
    two_sum(sb, pp, s2, e2);
    sb = s2;
    lo = __fadd_rn(lo, __fadd_rn(e2, pe));
    lo = __fmaf_rn(Al[k], w[k], lo);
  }
  return __fadd_rn(sb, lo);
}

constexpr float kNoRefine = 3.0e38f;  // refinement threshold of an item that is not refined

__device__ __forceinline__ size_t pack_idx(int p, int comp) {
  return ((size_t)(p / kTQ) * kNComp + comp) * kTQ + (p % kTQ);
}

__device__ __forceinline__ void store_h(float* pack, int p, int d, double h) {
  const float hi = __double2float_rn(h);
  const float lo = __double2float_rn(h - (double)hi);
  pack[pack_idx(p, d)] = hi;
  pack[pack_idx(p, d + 1)] = lo;
}

// Offset of the pack of `side` (0 rows, 1 columns) that iteration k reads (Inst::goff).  The slot may
// have been written earlier in the same launch, so it is read through L2.
__device__ __forceinline__ double pack_offset(const Inst* I, int side, long long k) {
  return I->goff != nullptr ? __ldcg(&I->goff[4 * side + (int)(k & 3)]) : 0.0;
}

// 2^e for an integer-valued e <= 0, exact; 0 below the normal range.
__device__ __forceinline__ double pow2i(double e) {
  if (!(e > -1022.0)) return 0.0;
  return __longlong_as_double((long long)(1023 + (int)e) << 52);
}

__device__ __forceinline__ double eps_of(const Inst* I, long long k) {
  return I->eta / (I->lambda * (double)k + 1.0);
}

// Inverse temperature of iteration k's row sweep: 1 / eta_k with the current kernel, 1 / eta_{k-1}
// = k / eta with the old one (lambda = 1; 0 at k = 0, where K^(0) = 1).
__device__ __forceinline__ double row_inv_eps(const Inst* I, long long k) {
  return alg_old_kernel(I->alg) ? (double)k / I->eta : 1.0 / eps_of(I, k);
}

// Deterministic CTA-wide sum (fixed tree order); all threads must call it.
__device__ __forceinline__ double block_sum(double v, double* red) {
  const int tid = threadIdx.x;
  red[tid] = v;
  __syncthreads();
#pragma unroll
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if (tid < s) red[tid] += red[tid + s];
    __syncthreads();
  }
  const double r = red[0];
  __syncthreads();
  return r;
}

// Split partial per point: (shift, sum) in the fast sweeps, (shift, sum, cost-weighted sum, 0) in the
// compensated ones, PartF64 in the FP64 ones.
template <int MODE>
struct PartT { typedef float2 type; };
template <>
struct PartT<kSweepComp> { typedef float4 type; };
template <>
struct PartT<kSweepF64> { typedef PartF64 type; };
// Row stride (points) of the partials of one micro-split: a multiple of 4 in the fast sweeps, so
// that a pair of adjacent points' (shift, sum) partials is one aligned 16-byte load.
template <int MODE>
__host__ __device__ constexpr size_t part_stride(int np) {
  return is_fast_mode(MODE) ? (size_t)((np + 3) & ~3) : (size_t)np;
}
__device__ __forceinline__ float part_z(const float2&) { return 0.0f; }
__device__ __forceinline__ float part_z(const float4& v) { return v.z; }

// Partials written by other CTAs are read through L2 (the L1 of this SM is not coherent).
__device__ __forceinline__ float2 load_part(const float2* p) { return __ldcg(p); }
__device__ __forceinline__ float4 load_part(const float4* p) { return __ldcg(p); }
__device__ __forceinline__ PartF64 load_part(const PartF64* p) {
  const double2* q = reinterpret_cast<const double2*>(p);
  const double2 a = __ldcg(q), b = __ldcg(q + 1);
  return PartF64{a.x, a.y, b.x, b.y};
}

// ---------------------------------------------------------------------------------------------
// Per-thread accumulator state for R thread-side points.
// ---------------------------------------------------------------------------------------------
template <int R, int MODE, bool FAST = is_fast_mode(MODE)>
struct Acc;

template <int R, int MODE>
struct Acc<R, MODE, true> {
  float mref[R], s[R], kc[R], n[R], nc[R];
  u64 acc[R], M2[R];
};
template <int R>
struct Acc<R, kSweepComp, false> {
  float mref[R], s[R], kc[R], n[R], nc[R];
};
template <int R>
struct Acc<R, kSweepF64, false> {
  double mref[R], s[R], n[R];
};

// ---------------------------------------------------------------------------------------------
// The sweep kernel.
//   MODE   kSweepFast: FP32 exponent, f32x2 FMAs, MUFU exp2 (the hot path)
//          kSweepFastPoly / kSweepFastSplit: the same with exp2 by the FMA-pipe polynomial for
//          all pairs / a quarter of the pairs
//          kSweepComp: exponent in float-float (error-free transforms), MUFU exp2, Kahan sums
//          kSweepF64 : exponent, exp2 and sums in FP64
//   CERT   column sweep also accumulates N_q = sum_p ||u-w||^2 E_pq (Algorithm 2)
//   UPDATE false: standalone certificate of the current state, no state update
// ---------------------------------------------------------------------------------------------
// Fast sweeps keep five CTAs resident per SM (<= 102 registers) when R x D <= 4 and three
// (<= 170) when R x D <= 12; the rarely run epilogue may spill rather than the hot loop lose warps.
template <int D, int R, int MODE>
constexpr int sweep_min_blocks() {
  return !is_fast_mode(MODE) ? 1 : (R * D <= 4 ? 5 : (R * D <= 12 ? 3 : 1));
}

// One launch runs `iters` iterations of every instance in the table: ticket t is work item
// t % nitems of the launch's iteration t / nitems, and the host lists each iteration's row items
// before its column items, each group longest first.  Tickets are handed out in order from
// sched[0]; an update item waits until its instance has finished the previous phase (the column
// sweep of the previous iteration for a row item, the row sweep of the same iteration for a column
// item).  A CTA only waits while it holds no unfinished item, and every ticket it waits on is
// smaller than its own and held by a running CTA, so the launch needs no co-residency.  sched[1]
// counts CTAs that have finished and the last one resets sched[0..2]; sched[2] is set when a CTA
// gives up, so that waiting CTAs stop too.
template <int D, int R, int MODE, bool CERT, bool UPDATE, int CHF>
__global__ void __launch_bounds__(kThreads, sweep_min_blocks<D, R, MODE>()) sweep_kernel(const Inst* __restrict__ insts,
                                                         const Item* __restrict__ items, int nitems, int iters,
                                                         unsigned* __restrict__ sched) {
  static_assert(!(CERT && is_fast_mode(MODE)), "certificate sweeps use the compensated or FP64 mode");
  constexpr bool FAST = is_fast_mode(MODE);
  // micro-split plan of the instance this kernel runs on (Inst::nms): the fast plan for the fast
  // modes, the certificate plan for the compensated and FP64 sweeps (certificate iterations, and
  // the compensated iterations before them; an instance whose every iteration runs compensated or
  // in FP64 has the same plan in both slots)
  constexpr int PL = FAST ? 0 : 1;
  static_assert(UPDATE || CERT, "a non-updating sweep is the standalone certificate");
  typedef typename PartT<MODE>::type Part;
  constexpr uint32_t kPackTileBytes = kNComp * kTQ * 4;  // one pack tile, all components
  constexpr int kStageFloats = kStageTiles * kNComp * kTQ;
  constexpr int CH = FAST ? CHF : 8;  // columns per chunk (one max + rescale test)
  static_assert(CH % 4 == 0 && kTQ % CH == 0, "chunk must divide the tile");

  extern __shared__ __align__(128) float smem[];
  __shared__ __align__(8) uint64_t bars[kStages];
  __shared__ double red[kThreads];
  __shared__ int s_flag;
  __shared__ int s_abort;
  __shared__ long long s_kit[2];  // per item (double-buffered by item parity): iteration k
  __shared__ int s_tk[2];         // and ticket
  __shared__ float s_rthr[2];     // and refinement threshold (fast sweeps; kNoRefine: none)
  __shared__ int s_ring[8];  // tickets in the order the producer took them (<= kStages + 1 ahead)
  __shared__ double s_ep[9];  // epilogue scalars of the current item (formed by thread 0)
  __shared__ int s_use_hint;
  __shared__ long long s_ring_k[8];  // per ring slot: the iteration its item's dependency check saw

  const int tid = threadIdx.x;
  if (tid == 0) {
#pragma unroll
    for (int s = 0; s < kStages; ++s) mbar_init(&bars[s], 1);
    fence_mbar_init();
  }
  __syncthreads();

  const int total = nitems * iters;
  // has the instance finished the phase that ticket (item it, launch iteration j) depends on?
  // (k0 does not change while the instance still has items in this launch)
  // Once met, the item's iteration is k0 + j: the instance's k cannot pass it before the item is done.
  auto dep_met = [&](const Item& it, int j, long long& need) -> bool {
    if constexpr (!UPDATE) return true;  // the standalone certificate reads a finished state
    const Inst* Ip = insts + it.inst;
    need = __ldcg(Ip->k0) + j;
    return it.side == 0 ? ld_acquire(Ip->k) >= need : ld_acquire(Ip->rows) >= need + 1;
  };

  // The TMA pipeline runs across work items: thread 0 keeps up to kStages stages in flight, taking
  // the CTA's next ticket before the current item ends.  It stops at an item whose dependency is
  // not met yet (re-checking whenever it is called) and never waits itself.  The ticket reaches the
  // other threads through s_ring: it is written before any stage of its item is issued and before a
  // CTA barrier that every consumer of the item passes.
  // producer state: used by thread 0 only, kept in shared memory to spare every thread's registers
  struct Producer {
    const float* qpack;
    Item item;
    uint32_t gprod, pseq, seq;  // stages issued, tickets taken, sequence number of the current one
    int t, j, us, nst, qt0, ntl;
    bool ok;                    // the current item may be issued (dependency met)
  };
  __shared__ Producer ps;
  uint32_t gcons = 0;  // stages consumed by this CTA (stage slot and mbarrier parity)
  auto pr_next = [&]() {
    ps.t = (int)atomicAdd(&sched[0], 1u);
    ps.seq = ps.pseq++;
    s_ring[ps.seq & 7u] = ps.t;
    ps.ok = false;
    if (ps.t >= total) return;
    const Item it = items[ps.t % nitems];
    ps.item = it;
    ps.j = ps.t / nitems;
    const Inst* Ip = insts + it.inst;
    const int qtl = it.side == 0 ? Ip->tiles_y : Ip->tiles_x;
    const int mstp = Ip->ms_tiles[PL][it.side];
    ps.qt0 = it.ms0 * mstp;
    ps.ntl = min(qtl, (it.ms0 + it.nms) * mstp) - ps.qt0;
    ps.nst = (ps.ntl + kStageTiles - 1) / kStageTiles;
    ps.qpack = it.side == 0 ? Ip->ypack : Ip->xpack;
    ps.us = 0;
  };
  auto pr_ready = [&]() -> bool {
    if (ps.t >= total) return false;
    if (!ps.ok) {
      long long need = 0;
      if (!dep_met(ps.item, ps.j, need)) return false;
      fence_proxy_async_global();
      s_ring_k[ps.seq & 7u] = need;
      ps.ok = true;
    }
    return true;
  };
  // issue stages until kStages are in flight beyond the `consumed` ones, or the producer stops
  auto refill = [&](uint32_t consumed) {
    while (ps.gprod - consumed < (uint32_t)kStages && pr_ready()) {
      const int stg = ps.gprod % kStages;
      const int tiles = min(kStageTiles, ps.ntl - ps.us * kStageTiles);
      mbar_expect_tx(&bars[stg], tiles * kPackTileBytes);
      bulk_g2s(smem + stg * kStageFloats, ps.qpack + (size_t)(ps.qt0 + ps.us * kStageTiles) * kNComp * kTQ,
               tiles * kPackTileBytes, &bars[stg]);
      ++ps.gprod;
      if (++ps.us == ps.nst) pr_next();
    }
  };
  if (tid == 0) {
    ps.gprod = 0;
    ps.pseq = 0;
    pr_next();
    refill(0);
  }
  __syncthreads();

  bool aborted = false;
  for (uint32_t cseq = 0;; ++cseq) {
    // If the producer stopped at this very item, wait here for its dependency (the CTA holds no
    // unfinished item now), then start its stages.  Thread 0 also publishes the item's iteration.
    if (tid == 0) {
      s_abort = 0;
      const int t = s_ring[cseq & 7u];
      if (ps.seq == cseq && t < total && !ps.ok) {
        const Inst* Ip = insts + ps.item.inst;
        uint32_t polls = 0;
        long long need = 0;
        while (!dep_met(ps.item, ps.j, need)) {
          if (polls++ >= Ip->wait_limit || *(volatile unsigned*)&sched[2] != 0u) {
            atomicOr(Ip->err, kErrTimeout);
            atomicExch(&sched[2], 1u);
            s_abort = 1;
            break;
          }
          __nanosleep(256);
        }
        if (!s_abort) {
          fence_proxy_async_global();
          s_ring_k[ps.seq & 7u] = need;
          ps.ok = true;
          refill(gcons);
        }
      }
      s_tk[cseq & 1u] = t;
      if (t < total && !s_abort) {
        const Item& it = items[t % nitems];
        const Inst* Ip = insts + it.inst;
        // an updating item's iteration was seen by its dependency check; the standalone certificate
        // certifies the last completed iteration
        const long long kk = UPDATE ? s_ring_k[cseq & 7u] : ld_acquire(Ip->k) - 1;
        s_kit[cseq & 1u] = kk;
        // Refinement of the dominant terms (fast FP32 sweeps): the FP32 exponent's parts grow as
        // 1/eps, so its rounding reaches e_fast = (d + 2) 2^-24 Zeps / eps (base 2; Inst::rzeps bounds
        // the parts' magnitude times eps).  Once e_fast exceeds refine_on, chunks whose sum reaches
        // the threshold (in units of the running shift, which the shift hints put about 2^-8 below
        // the point's total) are re-evaluated in float-float: the unrefined rest then carries at most
        // about refine_tol (natural log units) of error when some 16 chunks sit at the threshold.
        float rthr = kNoRefine;
        if constexpr (MODE == kSweepFast) {
          if (Ip->rzeps != nullptr && Ip->refine_on > 0.0) {
            const double inv = it.side == 0 ? row_inv_eps(Ip, kk) : 1.0 / eps_of(Ip, kk);
            const double ef = (D + 2) * 0x1p-24 * __ldcg(Ip->rzeps) * inv;
            if (ef > Ip->refine_on) rthr = (float)fmax(16.0 * Ip->refine_tol / ef, 0x1p-100);
          }
        }
        s_rthr[cseq & 1u] = rthr;
      }
    }
    __syncthreads();
    if (s_abort) {
      aborted = true;
      break;
    }
    if (s_tk[cseq & 1u] >= total) break;
    {  // ---- the item's sweep (its locals end here; the epilogue re-derives what it needs) ----
    const Item item = items[s_tk[cseq & 1u] % nitems];
    const int side = item.side;
    const bool accn = CERT && side == 1;  // accumulate N_q (Algorithm 2) on the column sweep
    const Inst* __restrict__ I = insts + item.inst;
    const int np = side == 0 ? I->n : I->m;
    const int qtiles = side == 0 ? I->tiles_y : I->tiles_x;
    const int mst = I->ms_tiles[PL][side];    // tiles per micro-split
    const float* __restrict__ ppack = side == 0 ? I->xpack : I->ypack;
    const int qt0 = item.ms0 * mst;
    const int qt1 = min(qtiles, (item.ms0 + item.nms) * mst);
    const int ntl = qt1 - qt0;
    const long long kiter = s_kit[cseq & 1u];
    const double sig = 2.0 * I->kappa * kLog2e * (side == 0 ? row_inv_eps(I, kiter) : 1.0 / eps_of(I, kiter));

    // ---- thread-side points ----
    float u[R][D];
    float Ah[R][D], Al[R][D];
    double Ad[R][D];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int p = item.pblk * (kThreads * R) + r * kThreads + tid;
      const bool valid = p < np;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        u[r][k] = valid ? ppack[pack_idx(p, k)] : 0.0f;
        const double A = sig * (double)u[r][k];
        Ad[r][k] = A;
        Ah[r][k] = __double2float_rn(A);
        Al[r][k] = __double2float_rn(A - (double)Ah[r][k]);
      }
    }
    Acc<R, MODE> st;
    auto reset = [&]() {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        st.mref[r] = 0;
        st.s[r] = 0;
        if constexpr (MODE != kSweepF64) {
          st.kc[r] = 0.0f;
          st.n[r] = 0.0f;
          st.nc[r] = 0.0f;
        } else {
          st.n[r] = 0.0;
        }
        if constexpr (FAST) {
          st.acc[r] = 0ull;
          st.M2[r] = 0ull;
        }
      }
    };
    reset();
    Part* part = reinterpret_cast<Part*>(I->part);
    // one split partial per micro-split: (shift, sum[, cost-weighted sum]) per point
    auto write_partial = [&](int ms) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int p = item.pblk * (kThreads * R) + r * kThreads + tid;
        if (p < np) {
          Part pr;
          pr.x = st.mref[r];
          pr.y = st.s[r];
          if constexpr (!FAST) {
            pr.z = st.n[r];
            pr.w = 0;
          }
          part[(size_t)ms * part_stride<MODE>(np) + p] = pr;
        }
      }
    };
    u64 A2[R][D];
    if constexpr (FAST) {
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int k = 0; k < D; ++k) A2[r][k] = pk2(Ah[r][k], Ah[r][k]);
    }


    // running-shift floor of each point from its validated hint (fast sweeps, k >= 1)
    float hs[R];
    bool use_hint = false;
    if constexpr (FAST) {
      // the hints are loaded with the miss counter (one round trip), and used if it is zero
      const bool have = kiter >= 1 && I->hint_bad != nullptr && I->hint[side] != nullptr;
      float hv[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int p = item.pblk * (kThreads * R) + r * kThreads + tid;
        hv[r] = (have && p < np) ? __ldcg(&I->hint[side][p]) : 0.0f;
      }
      use_hint = have && __ldcg(&I->hint_bad[2 * side + ((kiter - 1) & 1)]) == 0;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int p = item.pblk * (kThreads * R) + r * kThreads + tid;
        hs[r] = (use_hint && p < np) ? floorf(hv[r]) - kHintMargin : -INFINITY;
      }
    }

    const int nst = (ntl + kStageTiles - 1) / kStageTiles;  // pipeline stages of this item

    bool fresh = true;
    int tiles_done = 0, ms_cur = item.ms0, ms_end = min(ntl, mst);  // micro-split bookkeeping
    for (int us = 0; us < nst; ++us) {
      const uint32_t g = gcons + us;
      const int stg = g % kStages;
      const uint32_t par = (g / kStages) & 1u;
      const bool ok = mbar_wait_bounded(&bars[stg], par, I->wait_limit);
      const int stage_tiles = min(kStageTiles, ntl - us * kStageTiles);
      for (int tt = 0; tt < stage_tiles; ++tt) {
      const float* __restrict__ S = smem + stg * kStageFloats + tt * (kNComp * kTQ);

      if constexpr (FAST) {
        // The tile body is instantiated per coordinate-run variant KC (2-D packs only, Inst::runs
        // below): -1 general; 0 or 1 when coordinate KC is the same for every point of each aligned
        // group of kRunCols tile points (a row-major pixel grid's row coordinate), so that chunk's
        // exponents share the term A_p,KC w_KC - shift_p and cost one f32x2 FMA and one add per pair.
        auto fast_tile = [&](auto kc_tag) {
        constexpr int KC = decltype(kc_tag)::value;
        static_assert(KC < 0 || (D == 2 && kRunCols % CH == 0), "coordinate runs: 2-D packs, chunks within a run");
        // Per chunk of CH columns: exponents (f32x2 FMAs), chunk maximum and lazy rescale, then
        // exp2 on the SFU with a pairwise sum.
        u64 va[R][CH / 2];
        auto exponents = [&](u64 (&v)[R][CH / 2], int c0) {
          if constexpr (KC >= 0) {
            constexpr int KV = 1 - KC;
            const float wc = S[KC * kTQ + c0];  // the chunk's shared coordinate
            u64 T2[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
              float ac, ac1;
              up2(A2[r][KC], ac, ac1);
              const float t = __fmaf_rn(ac, wc, -st.mref[r]);
              T2[r] = pk2(t, t);
            }
#pragma unroll
            for (int gq = 0; gq < CH / 4; ++gq) {
              const int c = c0 + 4 * gq;
              const float4 hq = *reinterpret_cast<const float4*>(S + D * kTQ + c);
              const float4 wq = *reinterpret_cast<const float4*>(S + KV * kTQ + c);
              const u64 h01 = pk2(hq.x, hq.y), h23 = pk2(hq.z, hq.w);
              const u64 w01 = pk2(wq.x, wq.y), w23 = pk2(wq.z, wq.w);
#pragma unroll
              for (int r = 0; r < R; ++r) {
                v[r][2 * gq] = add2(fma2(A2[r][KV], w01, h01), T2[r]);
                v[r][2 * gq + 1] = add2(fma2(A2[r][KV], w23, h23), T2[r]);
              }
            }
          } else {
#pragma unroll
          for (int gq = 0; gq < CH / 4; ++gq) {
            const int c = c0 + 4 * gq;
            const float4 hq = *reinterpret_cast<const float4*>(S + D * kTQ + c);
            const u64 h01 = pk2(hq.x, hq.y), h23 = pk2(hq.z, hq.w);
            u64 w01[D], w23[D];
#pragma unroll
            for (int k = 0; k < D; ++k) {
              const float4 wq = *reinterpret_cast<const float4*>(S + k * kTQ + c);
              w01[k] = pk2(wq.x, wq.y);
              w23[k] = pk2(wq.z, wq.w);
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
              u64 a0 = fma2(A2[r][0], w01[0], h01);
              u64 a1 = fma2(A2[r][0], w23[0], h23);
#pragma unroll
              for (int k = 1; k < D; ++k) {
                a0 = fma2(A2[r][k], w01[k], a0);
                a1 = fma2(A2[r][k], w23[k], a1);
              }
              v[r][2 * gq] = sub2(a0, st.M2[r]);
              v[r][2 * gq + 1] = sub2(a1, st.M2[r]);
            }
          }
          }
        };
        // chunk maximum (max3 tree), one warp vote, rare lazy rescale of shift and sums
        auto rescale = [&](u64 (&v)[R][CH / 2]) {
          float cm[R];
          float amax = -INFINITY;
#pragma unroll
          for (int r = 0; r < R; ++r) {
            float t[CH];
#pragma unroll
            for (int j = 0; j < CH / 2; ++j) up2(v[r][j], t[2 * j], t[2 * j + 1]);
#pragma unroll
            for (int w = 1; w < CH; w *= 3)
#pragma unroll
              for (int j = 0; j < CH; j += 3 * w) {
                if (j + 2 * w < CH) t[j] = max3f(t[j], t[j + w], t[j + 2 * w]);
                else if (j + w < CH) t[j] = fmaxf(t[j], t[j + w]);
              }
            cm[r] = t[0];
            amax = fmaxf(amax, t[0]);
          }
          if (__any_sync(0xffffffffu, fresh || amax > kTau)) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
              if (fresh || cm[r] > kTau) {
                const float sh = fresh ? fmaxf(floorf(cm[r]), hs[r]) : floorf(cm[r]);
                if (!fresh) {
                  const float f = exp2_neg_int(sh);
                  st.acc[r] = mul2(st.acc[r], pk2(f, f));
                  st.s[r] *= f;
                  st.kc[r] *= f;
                }
                st.mref[r] += sh;
                st.M2[r] = pk2(st.mref[r], st.mref[r]);
                const u64 s2 = pk2(sh, sh);
#pragma unroll
                for (int j = 0; j < CH / 2; ++j) v[r][j] = sub2(v[r][j], s2);
              }
            }
          }
          fresh = false;
        };
        // exp2 and a pairwise (tree) sum of the chunk per point
        auto chunk_sums = [&](u64 (&v)[R][CH / 2], u64 (&cs)[R]) {
#pragma unroll
          for (int r = 0; r < R; ++r) {
            u64 e[CH / 2];
#pragma unroll
            for (int j = 0; j < CH / 2; ++j) {
              // exp2 on the SFU, or by the FMA-pipe polynomial (all pairs, or the first quarter)
              if (MODE == kSweepFastPoly || (MODE == kSweepFastSplit && j < CH / 8)) {
                e[j] = exp2_poly2(v[r][j]);
              } else {
                float lo, hi;
                up2(v[r][j], lo, hi);
                e[j] = pk2(ex2_mufu(lo), ex2_mufu(hi));
              }
            }
#pragma unroll
            for (int w = 1; w < CH / 2; w *= 2)
#pragma unroll
              for (int j = 0; j + w < CH / 2; j += 2 * w) e[j] = add2(e[j], e[j + w]);
            cs[r] = e[0];
          }
        };
        // The running shift only has to stay within ~64 (base 2) of the largest value seen, so the
        // tile is first run with no maximum at all (exponent FMAs, exp2, pairwise sums); only the
        // first chunk of a work item takes the exact maximum to set the shift.  If the tile's sum
        // then exceeds 2^64 (or overflowed), the tile, still in shared memory, is recomputed chunk
        // by chunk with the exact maximum and an exact power-of-two rescale of the running sums.
        int c0s = 0;
        if (kPeelFresh && fresh) {  // the first chunk of a micro-split sets the running shifts
          exponents(va, 0);
          rescale(va);
          u64 cs[R];
          chunk_sums(va, cs);
#pragma unroll
          for (int r = 0; r < R; ++r) st.acc[r] = add2(st.acc[r], cs[r]);
          c0s = CH;
        }
#pragma unroll kChunkUnroll
        for (int c0 = c0s; c0 < kTQ; c0 += CH) {
          exponents(va, c0);
          if (!kPeelFresh && fresh) rescale(va);
          u64 cs[R];
          chunk_sums(va, cs);
#pragma unroll
          for (int r = 0; r < R; ++r) st.acc[r] = add2(st.acc[r], cs[r]);
        }
        bool big = false;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          float lo, hi;
          up2(st.acc[r], lo, hi);
          const float t = lo + hi;
          big |= !(t <= 0x1p64f) && (t == t);  // above 2^64 or +inf (a NaN is left to propagate)
        }
        if (__any_sync(0xffffffffu, big)) {
          if (I->recomp != nullptr && (tid & 31) == 0) atomicAdd(I->recomp, 1ull);
#pragma unroll
          for (int r = 0; r < R; ++r) st.acc[r] = 0ull;
#pragma unroll 1
          for (int c0 = 0; c0 < kTQ; c0 += CH) {
            exponents(va, c0);
            rescale(va);
            u64 cs[R];
            chunk_sums(va, cs);
#pragma unroll
            for (int r = 0; r < R; ++r) st.acc[r] = add2(st.acc[r], cs[r]);
          }
        }
        // refinement: a tile whose sum reaches rthr (for some point of the warp) is run again chunk by
        // chunk; a chunk whose fast sum reaches rthr is replaced by its float-float evaluation
        if constexpr (MODE == kSweepFast) {
          const float rthr = s_rthr[cseq & 1u];
          if (rthr < kNoRefine) {
            bool sigt = false;
#pragma unroll
            for (int r = 0; r < R; ++r) {
              float lo, hi;
              up2(st.acc[r], lo, hi);
              sigt |= lo + hi > rthr;
            }
            if (__any_sync(0xffffffffu, sigt)) {
              // A_p in float-float, formed again here (not kept live through the fast loop)
              float rAh[R][D], rAl[R][D];
              {
                const long long kk = s_kit[cseq & 1u];
                const double sg =
                    2.0 * I->kappa * kLog2e * (side == 0 ? row_inv_eps(I, kk) : 1.0 / eps_of(I, kk));
#pragma unroll
                for (int r = 0; r < R; ++r) {
                  const int p = item.pblk * (kThreads * R) + r * kThreads + tid;
#pragma unroll
                  for (int k = 0; k < D; ++k) {
                    const double A = sg * (double)(p < np ? ppack[pack_idx(p, k)] : 0.0f);
                    rAh[r][k] = __double2float_rn(A);
                    rAl[r][k] = __double2float_rn(A - (double)rAh[r][k]);
                  }
                }
              }
#pragma unroll
              for (int r = 0; r < R; ++r) st.acc[r] = 0ull;
#pragma unroll 1
              for (int c0 = 0; c0 < kTQ; c0 += CH) {
                exponents(va, c0);
                u64 cs[R];
                chunk_sums(va, cs);
                bool need[R];
                bool any = false;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                  float lo, hi;
                  up2(cs[r], lo, hi);
                  need[r] = lo + hi > rthr;
                  any |= need[r];
                }
                if (__any_sync(0xffffffffu, any)) {
                  float csr[R];
#pragma unroll
                  for (int r = 0; r < R; ++r) csr[r] = 0.0f;
#pragma unroll 1
                  for (int cc = 0; cc < CH; ++cc) {
                    const int c = c0 + cc;
                    float w[D];
#pragma unroll
                    for (int k = 0; k < D; ++k) w[k] = S[k * kTQ + c];
                    const float hh = S[D * kTQ + c], hl = S[(D + 1) * kTQ + c];
#pragma unroll
                    for (int r = 0; r < R; ++r)
                      csr[r] += ex2_mufu(comp_exponent<D>(hh, hl, w, rAh[r], rAl[r], st.mref[r]));
                  }
#pragma unroll
                  for (int r = 0; r < R; ++r)
                    if (need[r]) cs[r] = pk2(csr[r], 0.0f);
                }
#pragma unroll
                for (int r = 0; r < R; ++r) st.acc[r] = add2(st.acc[r], cs[r]);
              }
              if ((tid & 31) == 0 && I->refined != nullptr) atomicAdd(I->refined, 1ull);
            }
          }
        }
        // fold the tile's pair sums into the compensated running sum
#pragma unroll
        for (int r = 0; r < R; ++r) {
          float lo, hi;
          up2(st.acc[r], lo, hi);
          st.acc[r] = 0ull;
          kahan_add(st.s[r], st.kc[r], lo + hi);
        }
        };  // fast_tile
        if constexpr (D == 2) {
          const float runs = S[(kNComp - 1) * kTQ];
          if (runs == 2.0f) fast_tile(std::integral_constant<int, 1>{});
          else if (runs == 1.0f) fast_tile(std::integral_constant<int, 0>{});
          else fast_tile(std::integral_constant<int, -1>{});
        } else {
          fast_tile(std::integral_constant<int, -1>{});
        }
      } else {
        // compensated (float-float) or FP64 exponent
        typedef typename std::conditional<MODE == kSweepF64, double, float>::type V;
        // The compensated exponent is exact only until it is rounded to FP32 relative to the
        // shift, so its shift follows the maximum closely (threshold 1: the dominant terms stay
        // within 2 of it) and a chunk whose shift moves is evaluated again against the new shift;
        // subtracting the new shift from values rounded against the old one would keep their
        // rounding, up to |old shift - value| * 2^-24.  FP64 loses nothing by subtracting.
        constexpr V tau = MODE == kSweepF64 ? (V)kTau : (V)1;
#pragma unroll 1
        for (int c0 = 0; c0 < kTQ; c0 += CH) {
          V v[R][CH];
          auto eval = [&]() {
#pragma unroll
          for (int cc = 0; cc < CH; ++cc) {
            const int c = c0 + cc;
            float w[D];
#pragma unroll
            for (int k = 0; k < D; ++k) w[k] = S[k * kTQ + c];
            const float hh = S[D * kTQ + c], hl = S[(D + 1) * kTQ + c];
#pragma unroll
            for (int r = 0; r < R; ++r) {
              if constexpr (MODE == kSweepF64) {
                double z = (double)hh + (double)hl;
#pragma unroll
                for (int k = 0; k < D; ++k) z = fma(Ad[r][k], (double)w[k], z);
                v[r][cc] = z - st.mref[r];
              } else {
                float sb, e0;
                two_sum(hh, -st.mref[r], sb, e0);
                float lo = __fadd_rn(e0, hl);
#pragma unroll
                for (int k = 0; k < D; ++k) {
                  float pp, pe, s2, e2;
                  two_prod(Ah[r][k], w[k], pp, pe);
                  two_sum(sb, pp, s2, e2);
                  sb = s2;
                  lo = __fadd_rn(lo, __fadd_rn(e2, pe));
                  lo = __fmaf_rn(Al[r][k], w[k], lo);
                }
                v[r][cc] = __fadd_rn(sb, lo);
              }
            }
          }
          };
          eval();
          V cm[R];
          bool need = fresh;
#pragma unroll
          for (int r = 0; r < R; ++r) {
            V mx = v[r][0];
#pragma unroll
            for (int cc = 1; cc < CH; ++cc) mx = mx > v[r][cc] ? mx : v[r][cc];
            cm[r] = mx;
            need |= mx > tau;
          }
          if (__any_sync(0xffffffffu, need)) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
              if (fresh || cm[r] > tau) {
                const V sh = floor(cm[r]);
                if (!fresh) {
                  if constexpr (MODE == kSweepF64) {
                    st.s[r] = ldexp(st.s[r], -(int)fmin(sh, 4000.0));
                    st.n[r] = ldexp(st.n[r], -(int)fmin(sh, 4000.0));
                  } else {
                    const float f = exp2_neg_int(sh);
                    st.s[r] *= f;
                    st.kc[r] *= f;
                    st.n[r] *= f;
                    st.nc[r] *= f;
                  }
                }
                st.mref[r] += sh;
                if constexpr (MODE == kSweepF64) {
#pragma unroll
                  for (int cc = 0; cc < CH; ++cc) v[r][cc] -= sh;
                }
              }
            }
            if constexpr (MODE != kSweepF64) eval();
          }
          fresh = false;
          V cs[R], cn[R];
#pragma unroll
          for (int r = 0; r < R; ++r) cs[r] = cn[r] = 0;
#pragma unroll
          for (int cc = 0; cc < CH; ++cc) {
            const int c = c0 + cc;
            float w[D];
            if (accn) {
#pragma unroll
              for (int k = 0; k < D; ++k) w[k] = S[k * kTQ + c];
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
              V E;
              if constexpr (MODE == kSweepF64) E = exp2(v[r][cc]);
              else E = ex2_mufu(v[r][cc]);
              cs[r] += E;
              if (accn) {
                V d2 = 0;
#pragma unroll
                for (int k = 0; k < D; ++k) {
                  const V df = (V)u[r][k] - (V)w[k];
                  d2 = df * df + d2;
                }
                cn[r] = d2 * E + cn[r];
              }
            }
          }
#pragma unroll
          for (int r = 0; r < R; ++r) {
            if constexpr (MODE == kSweepF64) {
              st.s[r] += cs[r];
              st.n[r] += cn[r];
            } else {
              kahan_add(st.s[r], st.kc[r], cs[r]);
              if (accn) kahan_add(st.n[r], st.nc[r], cn[r]);
            }
          }
        }
      }

        // end of a micro-split: publish its partial and start the next one afresh
        if (++tiles_done == ms_end) {
          write_partial(ms_cur++);
          reset();
          fresh = true;
          ms_end = min(ntl, ms_end + mst);
        }
      }  // tiles of the stage

      const int all_ok = __syncthreads_and(ok ? 1 : 0);
      if (!all_ok) {
        if (tid == 0) {
          atomicOr(I->err, kErrTimeout);
          atomicExch(&sched[2], 1u);  // stop CTAs that wait for a phase this CTA will not finish
          // let every copy still in flight (the stage that timed out included) land before the
          // CTA's shared memory is released; waits on a completed phase return at once
          for (uint32_t gj = g; gj < ps.gprod; ++gj)
            mbar_wait_bounded(&bars[gj % kStages], (gj / kStages) & 1u, kWaitLimit);
        }
        aborted = true;
        break;
      }
      if (tid == 0) refill(g + 1);  // refill the slot just consumed (possibly with later items' tiles)
    }
    if (aborted) break;
    gcons += nst;
    }

    // ---- last CTA of this point block runs the epilogue ----
    const int tk = s_tk[cseq & 1u];
    const int jit = tk / nitems;  // iteration of this launch the item belongs to
    const Item item = items[tk % nitems];
    const int side = item.side;
    const Inst* __restrict__ I = insts + item.inst;
    const int np = side == 0 ? I->n : I->m;
    const int splits = I->nms[PL][side];  // partials per point (all micro-splits)
    const int pblks = (np + kThreads * R - 1) / (kThreads * R);
    // point blocks this instance updates on this side: all of them, or the slice of a sharded state
    // (Inst::slice: point ranges aligned to 512 points, so to every R)
    const int own_blks = (min(I->slice[side][1], np) + kThreads * R - 1) / (kThreads * R) -
                         I->slice[side][0] / (kThreads * R);
    const long long kiter = s_kit[cseq & 1u];
    const bool accn = CERT && side == 1;
    const Part* part = reinterpret_cast<const Part*>(I->part);
    __threadfence();
    __syncthreads();
    if (tid == 0) {
      const bool last =
          atomicAdd(&I->cnt[item.pblk], (unsigned)item.nms) + (unsigned)item.nms == (unsigned)splits;
      s_flag = last;
      if (last) {
        __threadfence();
        // The epilogue's scalars, formed once for the CTA (FP64 divisions are slow on this GPU):
        // eps_k, 1 / eps_k, 1 / lambda, the next row sweep's inverse temperature (for the column
        // pack) and this one's, the hint ratio (hints predict this side's next log-sum-exp: this
        // one scaled by the ratio of the temperatures), the offsets of the pack this sweep read
        // (the other side's) for this and the next iteration and of the pack this epilogue writes.
        const double e = eps_of(I, kiter);
        const double ir = row_inv_eps(I, kiter);
        s_ep[0] = e;
        s_ep[1] = 1.0 / e;
        s_ep[2] = 1.0 / I->lambda;
        s_ep[3] = row_inv_eps(I, kiter + 1);
        s_ep[4] = ir;
        s_ep[5] = side == 0 ? row_inv_eps(I, kiter + 1) / ir : e / eps_of(I, kiter + 1);
        s_ep[6] = pack_offset(I, 1 - side, kiter);
        s_ep[7] = pack_offset(I, 1 - side, kiter + 1);
        s_ep[8] = side == 0 ? pack_offset(I, 0, kiter) : pack_offset(I, 1, kiter + 1);
        s_use_hint = FAST && kiter >= 1 && I->hint_bad != nullptr &&
                     __ldcg(&I->hint_bad[2 * side + ((kiter - 1) & 1)]) == 0;
      }
    }
    __syncthreads();
    if (!s_flag) continue;
    __threadfence();

    double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0;
    bool bad = false;
    bool hmiss = false;  // a stored hint missed this sweep's log-sum-exp by more than kHintTol
    float* const hint = UPDATE ? I->hint[side] : nullptr;
    // Points of this thread in the epilogue: R adjacent ones in the fast sweeps (their (shift, sum)
    // partials come in pairs, one 16-byte load per pair and split), else the sweep's own layout.
    auto ep_point = [&](int r) -> int {
      return FAST ? item.pblk * (kThreads * R) + R * tid + r : item.pblk * (kThreads * R) + r * kThreads + tid;
    };
    // The point block's merge waits on L2 for its split partials, and it is on the critical path of
    // the instance's phase: every round loads a batch of splits of all the thread's points before
    // merging them (16 registers of loads in flight).  Each point's splits are still merged one by one
    // in index order (a fixed order keeps the result deterministic).
    // FP32 partials are merged in FP32: exact power-of-two rescaling and Kahan sums (B300's FP64
    // pipe is slow, and an instance can have tens of split partials per point).
    float mxf[R], Sf[R], Sc[R], Nf[R], Nc[R];
    // per-point state the epilogue reads, loaded before the merge so that its latency overlaps it
    double st_a[R], st_b[R], st_c[R], st_d[R];
    float st_h[R];
    if constexpr (MODE != kSweepF64) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        mxf[r] = -INFINITY;
        Sf[r] = Sc[r] = Nf[r] = Nc[r] = 0.0f;
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int p = ep_point(r);
      st_a[r] = st_b[r] = st_c[r] = st_d[r] = 0.0;
      st_h[r] = 0.0f;
      if (p < np) {
        if (hint != nullptr) st_h[r] = __ldcg(&hint[p]);
        if (side == 0) {
          st_a[r] = I->xn2[p];
          st_b[r] = I->log_a[p];
          st_c[r] = __ldcg(&I->log_alpha[p]);
        } else {
          st_a[r] = I->yn2[p];
          st_b[r] = I->log_b[p];
          st_c[r] = UPDATE ? __ldcg(&I->log_beta_tilde_next[p]) : __ldcg(&I->log_beta_tilde[p]);
          if (UPDATE) st_d[r] = __ldcg(&I->log_beta[p]);
        }
      }
    }
    // one partial (m, s, n) into the running merge of point r: splits must come in index order
    auto merge_one = [&](int r, bool first, float ms, float sv, float nv) {
      if (first) {
        mxf[r] = ms;
        Sf[r] = sv;
        Nf[r] = nv;
      } else if (ms > mxf[r]) {
        const float f = exp2_neg_int(ms - mxf[r]);
        Sf[r] *= f;
        Sc[r] *= f;
        Nf[r] *= f;
        Nc[r] *= f;
        mxf[r] = ms;
        kahan_add(Sf[r], Sc[r], sv);
        if (accn) kahan_add(Nf[r], Nc[r], nv);
      } else {
        const float f = exp2_neg_int(mxf[r] - ms);
        kahan_add(Sf[r], Sc[r], sv * f);
        if (accn) kahan_add(Nf[r], Nc[r], nv * f);
      }
    };
    if constexpr (FAST) {
      // (shift, sum) partials of the thread's R adjacent points: R / 2 16-byte loads per split
      // (one 8-byte load when R = 1); the row stride keeps every pair aligned
      constexpr int kW = R >= 2 ? R / 2 : 1;          // loads per split
      constexpr int kB = R >= 2 ? 4 / kW : 8;         // splits per round (a larger batch spills into the sweep)
      const size_t pst = part_stride<MODE>(np);
      const int p0 = ep_point(0);
      const float* pf = reinterpret_cast<const float*>(I->part);
      for (int s0 = 0; s0 < splits; s0 += kB) {
        float4 q[kB][kW];
#pragma unroll
        for (int u = 0; u < kB; ++u)
#pragma unroll
          for (int w = 0; w < kW; ++w) {
            if (p0 < np && s0 + u < splits) {
              const float* a = pf + 2 * ((size_t)(s0 + u) * pst + p0 + 2 * w);
              if constexpr (R >= 2) {
                q[u][w] = __ldcg(reinterpret_cast<const float4*>(a));
              } else {
                const float2 v = __ldcg(reinterpret_cast<const float2*>(a));
                q[u][w] = make_float4(v.x, v.y, 0.0f, 0.0f);
              }
            }
          }
#pragma unroll
        for (int u = 0; u < kB; ++u) {
          if (s0 + u >= splits) break;
#pragma unroll
          for (int r = 0; r < R; ++r) {
            if (p0 + r >= np) continue;
            const float4 v = q[u][r / 2];
            const float ms = (r & 1) ? v.z : v.x;
            const float sv = (r & 1) ? v.w : v.y;
            merge_one(r, s0 + u == 0, ms, sv, 0.0f);
          }
        }
      }
    } else if constexpr (MODE != kSweepF64) {
      constexpr int kMergeBatch = R >= 2 ? 4 : 8;
      for (int s0 = 0; s0 < splits; s0 += kMergeBatch) {
        Part pr[R][kMergeBatch];
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int p = ep_point(r);
#pragma unroll
          for (int u = 0; u < kMergeBatch; ++u)
            if (p < np && s0 + u < splits) pr[r][u] = load_part(&part[(size_t)(s0 + u) * np + p]);
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int p = ep_point(r);
          if (p >= np) continue;
#pragma unroll
          for (int u = 0; u < kMergeBatch; ++u) {
            if (s0 + u >= splits) break;
            merge_one(r, s0 + u == 0, pr[r][u].x, pr[r][u].y, part_z(pr[r][u]));
          }
        }
      }
    }
    // the epilogue's scalars (read after the merge, which needs the registers)
    const double eps = s_ep[0];
    const double inv_eps = s_ep[1];
    const bool use_hint = s_use_hint != 0;
    const double lam = I->lambda;
    const double inv_lam = s_ep[2];
    const double inv_eps1 = s_ep[3];
    const double inv_row = s_ep[4];
    const double hint_ratio = s_ep[5];
    const double off_q = s_ep[6];
    const double off_q1 = s_ep[7];
    const double off_w = s_ep[8];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int p = ep_point(r);
      if (p >= np) continue;
      // merge the splits in index order: a fixed order keeps the result deterministic
      double mx, S, N;
      if constexpr (MODE == kSweepF64) {
        mx = -INFINITY;
        S = 0.0;
        N = 0.0;
        for (int s0 = 0; s0 < splits; s0 += 8) {
          Part pr[8];
#pragma unroll
          for (int u = 0; u < 8; ++u)
            if (s0 + u < splits) pr[u] = load_part(&part[(size_t)(s0 + u) * np + p]);
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            if (s0 + u >= splits) break;
            const double ms = (double)pr[u].x;  // integer-valued shifts: rescaling is exact
            if (ms > mx) {
              const double f = pow2i(mx - ms);
              S = S * f + (double)pr[u].y;
              N = N * f + (double)pr[u].z;
              mx = ms;
            } else {
              const double f = pow2i(ms - mx);
              S += (double)pr[u].y * f;
              N += (double)pr[u].z * f;
            }
          }
        }
      } else {
        mx = (double)mxf[r];
        S = (double)Sf[r] - (double)Sc[r];
        N = (double)Nf[r] - (double)Nc[r];
      }
      double lse2;
      if constexpr (FAST) {
        lse2 = mx + (double)__log2f((float)S);  // FP32 log2 is below the FP32 sweep's own rounding
      } else {
        lse2 = mx + log2(S);
      }
      if (hint != nullptr) {
        const float e = st_h[r];
        const float l = (float)lse2;
        hmiss |= kiter == 0 || !(fabsf(e - l) <= kHintTol);
        bad |= use_hint && e - l > kHintGuard;  // flushed terms could matter: reject the sweep
        hint[p] = (float)((lse2 + off_q) * hint_ratio - off_q1);
      }
      lse2 += off_q;  // the sweep ran on h - G
      // state written by other CTAs of this launch (earlier phases) is read through L2
      if (side == 0) {
        const double xn2 = st_a[r], la_old = st_c[r];
        const double lse = lse2 * kLn2 - xn2 * inv_row;
        double lah = st_b[r] - lse;
        if (I->alg == kAlgDAS && kiter >= 2) lah += la_old / (double)kiter;  // theta_k = 1/k
        bad |= !isfinite(lah);
        I->log_alpha_hat[p] = lah;
        I->log_alpha[p] = (1.0 - lam) * la_old + lam * lah;
        store_h(I->xpack, p, I->d, (lah - xn2 * inv_eps) * kLog2e - off_w);
        if constexpr (CERT) {
          const double f = eps * lah;
          I->f_cur[p] = f;
          acc0 += I->a[p] * f;
        }
      } else {
        const double yn2 = st_a[r];
        const double lse = lse2 * kLn2 - yn2 * inv_eps;  // d_j of Algorithm 2
        double lbh;
        double t;
        if constexpr (UPDATE) {
          lbh = st_b[r] - lse;
          bad |= !isfinite(lbh);
          t = st_c[r];
          I->log_beta_tilde[p] = t;
          const double bold = st_d[r];
          const double bnew = (1.0 - lam) * bold + lam * lbh;
          I->log_beta_prev[p] = bold;
          I->log_beta[p] = bnew;
          I->log_beta_hat[p] = lbh;
          const double tn = alg_momentum(I->alg) ? bnew + (bnew - bold) * inv_lam : bnew;
          I->log_beta_tilde_next[p] = tn;
          store_h(I->ypack, p, I->d, (tn - yn2 * inv_eps1) * kLog2e - off_w);
        } else {
          lbh = __ldcg(&I->log_beta_hat[p]);
          t = st_c[r];
        }
        if constexpr (CERT) {
          const double sj = exp(t + lse);
          const double mu = I->kappa * N / S;
          const double gj = eps * (lbh - st_b[r]);
          I->g_cur[p] = gj;
          acc0 += I->b[p] * gj;
          acc1 += sj * mu;
          acc2 += fabs(sj - I->b[p]);
        }
      }
    }
    if (bad) atomicOr(I->err, kErrNonFinite);
    if (hint != nullptr && __syncthreads_or(hmiss ? 1 : 0) && tid == 0)
      atomicAdd(&I->hint_bad[2 * side + (kiter & 1)], 1);
    if constexpr (CERT) {
      const double s0 = block_sum(acc0, red);
      if (side == 0) {
        if (tid == 0) I->blk[item.pblk] = s0;
      } else {
        const double s1 = block_sum(acc1, red);
        const double s2 = block_sum(acc2, red);
        if (tid == 0) {
          double* bb = I->blk + I->pblk_x + 3 * item.pblk;
          bb[0] = s0;
          bb[1] = s1;
          bb[2] = s2;
        }
      }
    }
    if (tid == 0) I->cnt[item.pblk] = 0u;

    // ---- last point block of the instance's phase ----
    fence_proxy_async_global();  // the packed h just written is read by bulk copies of a later phase
    __threadfence();
    __syncthreads();
    if (tid == 0) s_flag = (atomicAdd(I->done, 1u) == (unsigned)(own_blks - 1));
    __syncthreads();
    if (!s_flag) continue;
    __threadfence();
    if (side == 0) {
      // row sweep complete: release the instance's column sweep of this iteration
      if constexpr (UPDATE) {
        if (tid == 0) {
          *I->done = 0u;
          __threadfence();
          st_release(I->rows, kiter + 1);
        }
      }
      continue;
    }
    // column sweep complete: finish the certificate, advance k (releasing the next iteration)
    if constexpr (CERT) {
      double rf;
      if constexpr (UPDATE) {
        double v = 0.0;
        for (int b = tid; b < I->pblk_x; b += kThreads) v += __ldcg(&I->blk[b]);
        rf = block_sum(v, red);
      } else {
        // standalone certificate: <r, f> with f = eps log alpha-hat from the state
        double v = 0.0;
        for (int i = tid; i < I->n; i += kThreads) {
          const double f = eps * __ldcg(&I->log_alpha_hat[i]);
          I->f_cur[i] = f;
          v += I->a[i] * f;
        }
        rf = block_sum(v, red);
      }
      double v0 = 0.0, v1 = 0.0, v2 = 0.0;
      for (int b = tid; b < pblks; b += kThreads) {
        const double* bb = I->blk + I->pblk_x + 3 * b;
        v0 += __ldcg(&bb[0]);
        v1 += __ldcg(&bb[1]);
        v2 += __ldcg(&bb[2]);
      }
      const double cg = block_sum(v0, red);
      const double smu = block_sum(v1, red);
      const double dab = block_sum(v2, red);
      if (tid == 0) {
        const double delta = 0.5 * dab;
        double* cr = I->cert;
        cr[kCertIter] = (double)kiter;
        cr[kCertEps] = eps;
        cr[kCertU] = smu + I->omega * delta;
        cr[kCertL] = rf + cg;
        cr[kCertDelta] = delta;
        cr[kCertCostZ] = smu;
        cr[kCertRF] = rf;
        cr[kCertCG] = cg;
      }
    }
    if (tid == 0) {
      *I->done = 0u;
      if constexpr (UPDATE) {
        // the hint-miss counters iteration kiter + 1 fills (last read by iteration kiter)
        if (I->hint_bad != nullptr) {
          I->hint_bad[(kiter + 1) & 1] = 0;
          I->hint_bad[2 + ((kiter + 1) & 1)] = 0;
        }
        // pack offsets of iteration kiter + 2 (their slots last served iteration kiter - 2): the
        // current values of the first point, which the drift moves by a few steps until then
        if (I->goff != nullptr) {
          I->goff[(kiter + 2) & 3] = kLog2e * __ldcg(&I->log_alpha_hat[0]);
          I->goff[4 + ((kiter + 2) & 3)] = kLog2e * __ldcg(&I->log_beta_tilde_next[0]);
        }
        if (jit == iters - 1) *I->k0 = kiter + 1;  // the next launch starts here
        __threadfence();
        st_release(I->k, kiter + 1);
      }
    }
  }
  // the last CTA out resets the scheduler (every CTA has taken its final ticket by now)
  if (tid == 0) {
    __threadfence();
    if (atomicAdd(&sched[1], 1u) == gridDim.x - 1) {
      sched[0] = 0u;
      sched[2] = 0u;
      __threadfence();
      sched[1] = 0u;
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Launch table: one entry per instantiated (D, R, MODE, CERT, UPDATE, chunk).
// ---------------------------------------------------------------------------------------------
typedef void (*SweepFn)(const Inst*, const Item*, int, int, unsigned*);

template <int D, int R, int MODE, bool CERT, bool UPDATE, int CHF>
static SweepFn sweep_ptr() {
  return &sweep_kernel<D, R, MODE, CERT, UPDATE, CHF>;
}

// variant index: 0 fast iterations, 1 certificate iterations, 2 standalone certificate
template <int D, int R, int MODE, int CHF>
static SweepFn sweep_variant(int v) {
  switch (v) {
    case 0: return sweep_ptr<D, R, MODE, false, true, CHF>();
    case 1:
      if constexpr (!is_fast_mode(MODE)) return sweep_ptr<D, R, MODE, true, true, CHF>();
      return nullptr;
    case 2:
      if constexpr (!is_fast_mode(MODE)) return sweep_ptr<D, R, MODE, true, false, CHF>();
      return nullptr;
  }
  return nullptr;
}

// Tile plans of the fast sweep: points per thread R in {1, 2, 4, 8} and chunk width CH in {8, 16}
// (R = 8 only with CH = 8).  The compensated and FP64 sweeps use CH = 8 and R in {1, 2, 4}.
template <int D>
static SweepFn sweep_m(int mode, int R, int ch, int v) {
  if (mode == kSweepFast) {
    if (R == 1) return ch == 8 ? sweep_variant<D, 1, kSweepFast, 8>(v) : sweep_variant<D, 1, kSweepFast, 16>(v);
    if (R == 2) return ch == 8 ? sweep_variant<D, 2, kSweepFast, 8>(v) : sweep_variant<D, 2, kSweepFast, 16>(v);
    if (R == 4) return ch == 8 ? sweep_variant<D, 4, kSweepFast, 8>(v) : sweep_variant<D, 4, kSweepFast, 16>(v);
    if (R == 8 && ch == 8) return sweep_variant<D, 8, kSweepFast, 8>(v);
    return nullptr;
  }
  if (mode == kSweepFastPoly || mode == kSweepFastSplit) {
    // the polynomial arms exist for the canonical fast plans only
    if (R == 2 && ch == 16)
      return mode == kSweepFastPoly ? sweep_variant<D, 2, kSweepFastPoly, 16>(v)
                                    : sweep_variant<D, 2, kSweepFastSplit, 16>(v);
    if (R == 4 && ch == 16)
      return mode == kSweepFastPoly ? sweep_variant<D, 4, kSweepFastPoly, 16>(v)
                                    : sweep_variant<D, 4, kSweepFastSplit, 16>(v);
    return nullptr;
  }
  if (mode == kSweepComp) {
    if (R == 1) return sweep_variant<D, 1, kSweepComp, 8>(v);
    if (R == 2) return sweep_variant<D, 2, kSweepComp, 8>(v);
    if (R == 4) return sweep_variant<D, 4, kSweepComp, 8>(v);
    return nullptr;
  }
  if (mode == kSweepF64) {
    if (R == 1) return sweep_variant<D, 1, kSweepF64, 8>(v);
    if (R == 2) return sweep_variant<D, 2, kSweepF64, 8>(v);
    return nullptr;
  }
  return nullptr;
}

}  // namespace ot
