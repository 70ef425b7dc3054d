// Shared definitions between the sweep kernels and the host runtime.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace ot {

constexpr int kThreads = 128;  // threads per CTA in every sweep kernel
constexpr int kTQ = 128;       // points per shared-memory tile (per pipeline stage)
constexpr int kStages = 4;     // TMA pipeline depth
constexpr int kStageTiles = 4; // pack tiles per pipeline stage (one bulk copy, one CTA barrier)
constexpr int kNComp = 5;      // pack components per point: up to 3 coords, h (hi), h (lo)
constexpr uint32_t kWaitLimit = 1u << 26;  // mbarrier polls before a sweep gives up (~seconds)

// Error bits written to Inst::err by device code.
enum : int { kErrTimeout = 1, kErrNonFinite = 2 };

// Precision of one sweep launch.  The three fast modes differ only in how exp2 is evaluated:
// MUFU, an FMA-pipe polynomial, or a fixed split between the two.
enum : int { kSweepFast = 0, kSweepComp = 1, kSweepF64 = 2, kSweepFastPoly = 3, kSweepFastSplit = 4 };
// Row-update methods (App. B; App. G "Momentum and Kernel Ablation"; lambda = 1 for all but BDRS):
// the row sweep's kernel is the current K^(k+1) or the old K^(k), and its column scaling is the
// momentum extrapolation or v^{k-1}; DAS also multiplies r by (u^{k-1})^theta_k.
enum : int { kAlgBDRS = 0, kAlgAS = 1, kAlgASMomentum = 2, kAlgASCurrent = 3, kAlgDAS = 4 };
__host__ __device__ constexpr bool alg_old_kernel(int a) { return a == kAlgAS || a == kAlgASMomentum || a == kAlgDAS; }
__host__ __device__ constexpr bool alg_momentum(int a) { return a == kAlgBDRS || a == kAlgASMomentum; }

__host__ __device__ constexpr bool is_fast_mode(int mode) {
  return mode == kSweepFast || mode == kSweepFastPoly || mode == kSweepFastSplit;
}

// Certificate record layout (doubles) written by the last CTA of a certificate iteration.
enum : int {
  kCertIter = 0, kCertEps, kCertU, kCertL, kCertDelta, kCertCostZ, kCertRF, kCertCG, kCertLen = 8
};

// One OT instance as the kernels see it.  All device pointers are owned by the runtime.
//
// Packs are tile-blocked structure-of-arrays: point p lives in tile p / kTQ at offset p % kTQ,
// and tile t holds kNComp rows of kTQ floats: coords 0..d-1, then h (hi), then h (lo).
// The coordinates are the caller's float32 points; h is the per-point offset of the
// exponent in base 2 (see the sweep kernels), rewritten by every epilogue.
struct Inst {
  int n, m, d;
  int tiles_x, tiles_y;          // ceil(n / kTQ), ceil(m / kTQ)
  int pblk_x;                    // point blocks of the certificate row sweep (layout of blk)
  // Micro-splits of the reduced side, per plan (0: fast iterations, 1: certificate iterations)
  // and sweep (0 row, 1 column): the reduced side's tiles are cut into nms runs of ms_tiles tiles
  // (the last may be shorter), one split partial each.  They are fixed per instance, so its
  // results do not depend on how a launch groups micro-splits into work items.
  int nms[2][2];
  int ms_tiles[2][2];
  // Points whose updates this instance runs, per side (0 rows, 1 columns): [slice[s][0],
  // slice[s][1]), the whole side unless the state is one slice of a row-sharded solve; the phase of
  // a side completes when the point blocks of the slice are done.
  int slice[2][2];
  uint32_t wait_limit;           // mbarrier polls before a sweep gives up waiting for a tile
  int alg;                       // row-update method (kAlg*): Dual (O-)BDRS or an ablation method
  double kappa, eta, lambda, omega;
  float* xpack;                  // [tiles_x][kNComp][kTQ]
  float* ypack;                  // [tiles_y][kNComp][kTQ]
  const double* a;               // source weights r (normalised)
  const double* b;               // target weights c (normalised)
  const double* log_a;           // log r
  const double* log_b;           // log c
  const double* xn2;             // kappa * ||x_i||^2
  const double* yn2;             // kappa * ||y_j||^2
  double* log_alpha;             // alpha^{k-1} -> alpha^k
  double* log_alpha_hat;         // alpha-hat^k
  double* log_beta;              // beta^{k-1} -> beta^k
  double* log_beta_prev;         // beta^{k-2} -> beta^{k-1}
  double* log_beta_hat;          // beta-hat^k
  double* log_beta_tilde;        // beta-tilde^{k-1} used by the last completed iteration
  double* log_beta_tilde_next;   // beta-tilde^{k} for the next iteration (packed into ypack)
  double* f_cur;                 // certificate potentials of the latest certificate iteration
  double* g_cur;
  void* part;                    // split partials per point and split: float2 (shift, sum) in the fast sweeps
                                 // (rows of part_stride points), float4 in the compensated ones, PartF64 in FP64
  unsigned* cnt;                 // per point-block arrival counters (sized for R = 1)
  unsigned* done;                // per-instance epilogue counter
  double* blk;                   // certificate partial sums: pblk_x row blocks, then 3 per column block
  // Shift hints of the fast sweeps: per point, the base-2 log-sum-exp that point's next sweep is
  // expected to reach (this sweep's value scaled by eps_k / eps_{k+1}), less the offset of the pack
  // that sweep will read (goff below), so in the units of its running shift; and per side and iteration
  // parity the count of points whose stored hint missed the exact value by more than
  // kHintTol (hint_bad[2 * side + parity]).  A sweep starts its running shifts from the hints only
  // when the previous iteration of the same side had no miss.  Null: no hints.
  float* hint[2];                // row side (n floats), column side (m floats)
  int* hint_bad;                 // 4 counters
  // Base-2 offsets G of the packed h components: a pack stores h - G and its consumer adds G back
  // to the log-sum-exp in FP64, which is exact (LSE_q(h_q - G + z_q) = LSE_q(h_q + z_q) - G).  The
  // log-scalings drift in gauge (alpha c, beta / c) by a constant step per iteration, so h can grow
  // far beyond the 1/eps scale of the exponents; the offset keeps the FP32 rounding of the pack at
  // that scale.  [side][k mod 4], side 0 the row pack, 1 the column pack, for the packs iteration k
  // reads; null: no offsets.
  double* goff;
  long long* k;                  // completed iterations (released by the last column epilogue)
  long long* rows;               // completed row sweeps (released by the last row epilogue)
  long long* k0;                 // k at the start of the current launch (set by the previous one)
  double* cert;                  // certificate record (kCertLen doubles)
  int* err;                      // error bits
  unsigned long long* recomp;    // warp-tiles of the fast sweeps recomputed with the exact maximum
                                 // (a tile sum above 2^64); null: not counted
  const float* origin;           // translation the packs' coordinates carry (3 floats), or null
  // Refinement of the fast sweeps' dominant terms (see the sweep kernel): rzeps bounds eps times the
  // magnitude of the FP32 exponent's parts (base 2; written at set-up), refine_on the FP32 rounding
  // (base 2) above which it applies, refine_tol the error (natural log units) the unrefined terms
  // may carry; refined counts warp-tiles evaluated again.  rzeps null or refine_on <= 0: off.
  const double* rzeps;
  double refine_on, refine_tol;
  unsigned long long* refined;
};

// Split partial of the FP64 sweep: (shift, sum, cost-weighted sum, unused).
struct alignas(32) PartF64 {
  double x, y, z, w;
};

// A unit of sweep work: instance, side (0 row sweep, 1 column sweep), point block (kThreads * R
// points of the launched kernel), and a run of consecutive micro-splits of the reduced side: first
// one and count.
struct Item {
  int inst, side, pblk, ms0, nms;
};

}  // namespace ot
