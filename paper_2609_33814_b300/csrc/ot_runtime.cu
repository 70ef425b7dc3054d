// Host runtime of the solver: validation, device buffers, launch plans, CUDA graphs of iteration
// chunks, certificate read-back with best-so-far bounds and the stop rule (Algorithm 1 with the
// certificate of Proposition 3 every cert_every iterations; best bounds as in App. G.3).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <dlfcn.h>

#include "../../include/ot.h"
#include "ot_kernels.cuh"
#include "ot_runtime.h"

namespace ot {

size_t sweep_smem_bytes();
size_t plan_scratch_bytes(int64_t n, int64_t m);
size_t round_scratch_bytes(int64_t n, int64_t m);
cudaError_t plan_rounding(const Inst& h, int which, double eps, const double* f_best, const double* g_best,
                          void* scratch, double* sums, cudaStream_t st);
cudaError_t plan_diagnostics(const Inst& h, int which, double eps, const double* f_best, const double* g_best,
                             void* scratch, float* y_hat, double* row, double* col, double* err, cudaStream_t st);
cudaError_t launch_sweep(SweepFn fn, const Inst* insts, const Item* items, int nitems, int iters, int grid,
                         unsigned* sched, cudaStream_t stream);
cudaError_t launch_pack_coords(const float* pts, int npts, int d, int tiles, double kappa, float* pack,
                               double* n2, cudaStream_t s, const float* origin);
cudaError_t launch_centre(const float* x, int n, const float* y, int m, int d, int* scratch, float* origin,
                          double kappa, double omega, double* rzeps, int sms, cudaStream_t s);
cudaError_t launch_normalise(const double* w, int npts, double floor_mass, double* wn, double* logw,
                             double* scratch, int* err, cudaStream_t s);
cudaError_t launch_repack_cols(const Inst* I, int m, cudaStream_t s);
cudaError_t launch_pair_cost_range(const float* x, int n, const float* y, int m, int d, unsigned* mx,
                                   unsigned* mn, int sms, cudaStream_t s);

// ---------------------------------------------------------------------------------------------
// Context
// ---------------------------------------------------------------------------------------------
void Context::set_error(const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  last_error = buf;
}

int Context::resident_ctas(SweepFn fn) {
  auto it = occ.find((const void*)fn);
  if (it != occ.end()) return it->second;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)fn, kThreads, sweep_smem_bytes()) !=
          cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  const int r = per_sm * sms;
  occ[(const void*)fn] = r;
  return r;
}

// ---------------------------------------------------------------------------------------------
// Launch plans: points per thread R, chunk width and the split counts of both sweeps.
// ---------------------------------------------------------------------------------------------
constexpr int kMaxSplits = 64;      // split cap: bounds the partial buffer and the epilogue merge
constexpr int kMinSplitTiles = 4;   // a micro-split covers at least 4 tiles (512 points)
static int env_int(const char* name, int dflt) {
  const char* v = getenv(name);
  return v && *v ? atoi(v) : dflt;
}

// The plan that fixes an instance's numerics: points per thread R and chunk width CH depend only on
// (d, precision mode), the split counts only on the instance's own sizes.  An instance therefore
// produces bitwise the same results alone or inside any batch; only the launch grid (which does
// not affect results) depends on the device's occupancy.
//
// The plan per (d, mode) comes from a table that the autotuner (autotune.py beside this library)
// fills by timing every instantiated (R, CH) on the device and writes to tile_plans.txt; the table
// is loaded when the first context is created (OT_TILE_PLANS names another file, empty: none) and
// can be set with ot_set_tile_plan.  Entries left unset use the built-in plans below, which are the
// autotuner's choices on B300.  A table changes results bitwise (another summation order), never
// their accuracy.
namespace {
std::mutex g_plan_mu;
int g_plan[4][5][2] = {};  // [d][mode] -> {R, CH}; R = 0: built-in
}  // namespace

// Built-in plans: the autotuner's choices on B300 (tile_plans.txt in the package holds its
// measurements), indexed [d - 1][mode] with modes fast, compensated, FP64, fast+poly, fast+split.
static void builtin_tile(int d, int mode, int* R, int* ch) {
  static const int kPlan[3][5][2] = {
      {{2, 16}, {2, 8}, {2, 8}, {2, 16}, {2, 16}},  // d = 1
      {{4, 16}, {1, 8}, {1, 8}, {4, 16}, {2, 16}},  // d = 2
      {{4, 8}, {1, 8}, {2, 8}, {2, 16}, {4, 16}},   // d = 3
  };
  const int di = (d >= 1 && d <= 3) ? d - 1 : 1;
  const int mi = (mode >= 0 && mode <= 4) ? mode : 0;
  *R = kPlan[di][mi][0];
  *ch = kPlan[di][mi][1];
}

void canonical_tile(int d, int mode, int* R, int* ch) {
  builtin_tile(d, mode, R, ch);
  if (d < 1 || d > 3 || mode < 0 || mode > 4) return;
  std::lock_guard<std::mutex> lk(g_plan_mu);
  if (g_plan[d][mode][0] > 0) {
    *R = g_plan[d][mode][0];
    *ch = g_plan[d][mode][1];
  }
}

// Sets the table entry of (d, mode); R = 0 restores the built-in plan.  False if that kernel is not
// instantiated.
static bool set_tile(int d, int mode, int R, int ch) {
  if (d < 1 || d > 3 || mode < 0 || mode > 4) return false;
  if (R != 0 && !get_sweep(d, mode, R, ch, 0)) return false;
  if (R != 0 && (mode == kSweepComp || mode == kSweepF64) && ch != 8) return false;  // built with CH = 8 only
  std::lock_guard<std::mutex> lk(g_plan_mu);
  g_plan[d][mode][0] = R;
  g_plan[d][mode][1] = R ? ch : 0;
  return true;
}

int sweep_mode_of(int precision);

// Lines "d precision R CH" (ot_precision values; '#' starts a comment); invalid lines are skipped.
static void load_tile_plans() {
  std::string path;
  if (const char* e = getenv("OT_TILE_PLANS")) {
    path = e;
  } else {
    Dl_info info;
    if (dladdr((void*)&load_tile_plans, &info) && info.dli_fname) {
      path = info.dli_fname;
      const size_t slash = path.rfind('/');
      path = (slash == std::string::npos ? std::string(".") : path.substr(0, slash)) + "/tile_plans.txt";
    }
  }
  if (path.empty()) return;
  FILE* f = fopen(path.c_str(), "r");
  if (!f) return;
  char line[256];
  while (fgets(line, sizeof(line), f)) {
    if (char* h = strchr(line, '#')) *h = 0;
    int d, prec, R, ch;
    if (sscanf(line, "%d %d %d %d", &d, &prec, &R, &ch) == 4 && prec >= 0 && prec <= 4)
      set_tile(d, sweep_mode_of(prec), R, ch);
  }
  fclose(f);
}

// Micro-splits of one sweep of an instance: enough runs of the reduced side that any launch can
// cut the instance into balanced work items (about 65536 point-block runs), each run at least 4
// tiles and an even number of tiles, at most 64 runs (a run may end inside a pipeline stage: the
// sweep closes runs tile by tile).
// The layout depends only on the instance's sizes and the plan's R, so the instance's partials,
// and hence its results, are the same in every launch that contains it.
void micro_splits(int64_t np, int64_t nq, int R, int* nms, int* mst) {
  const int pblks = (int)((np + kThreads * R - 1) / (kThreads * R));
  const int qtiles = (int)((nq + kTQ - 1) / kTQ);
  int n = std::max(1, std::min({(65536 + pblks - 1) / pblks, kMaxSplits, qtiles / kMinSplitTiles}));
  int t = (qtiles + n - 1) / n;
  if (n > 1 && (t & 1)) ++t;
  n = (qtiles + t - 1) / t;
  *nms = n;
  *mst = n > 1 ? t : qtiles;
}

// Micro-splits per work item for an instance that runs alone: the largest grouping whose items
// (all about the same size) fill close to a whole number of waves of the resident CTAs.
int solo_group(int pblks, int nms, int resident) {
  int best = nms, last_per = -1;
  double best_eff = -1.0, best_waves = 0.0;
  for (int g = nms; g >= 1; --g) {
    const int per = (nms + g - 1) / g;  // items per point block
    if (per == last_per) continue;       // a larger grouping already gave this item count
    last_per = per;
    const double waves = (double)pblks * per / resident;
    const double eff = waves / std::ceil(waves);
    if (eff >= 0.95 && waves >= 2.0) return g;
    if (eff > best_eff + 0.01 || (eff > best_eff - 0.01 && waves > best_waves)) {
      best_eff = std::max(eff, best_eff);
      best_waves = waves;
      best = g;
    }
  }
  return best;
}

void plan_launch(Context& ctx, const Instance& in, int mode, LaunchPlan& pl) {
  int R, ch;
  canonical_tile(in.d, mode, &R, &ch);
  // tuning overrides for experiments (they change the numerics): OT_FORCE_R, OT_FORCE_CH
  if (mode == kSweepFast) {
    R = env_int("OT_FORCE_R", R);
    ch = env_int("OT_FORCE_CH", ch);
  }
  if (!get_sweep(in.d, mode, R, ch, 0)) canonical_tile(in.d, mode, &R, &ch);
  pl.mode = mode;
  pl.R = R;
  pl.ch = ch;
  const int rpb = kThreads * R;
  pl.pblk_row = (int)((in.n + rpb - 1) / rpb);
  pl.pblk_col = (int)((in.m + rpb - 1) / rpb);
  SweepFn fn = get_sweep(in.d, mode, R, ch, 0);
  const int resident = ctx.resident_ctas(fn);
  micro_splits(in.n, in.m, R, &pl.nms_row, &pl.mst_row);
  micro_splits(in.m, in.n, R, &pl.nms_col, &pl.mst_col);
  pl.group_row = solo_group(pl.pblk_row, pl.nms_row, resident);
  pl.group_col = solo_group(pl.pblk_col, pl.nms_col, resident);
  pl.n_row = pl.pblk_row * ((pl.nms_row + pl.group_row - 1) / pl.group_row);
  pl.n_col = pl.pblk_col * ((pl.nms_col + pl.group_col - 1) / pl.group_col);
  pl.resident = resident;
}

// Work items of one sweep of one instance: every point block times runs of `group` consecutive
// micro-splits (the last run may be shorter).
void build_items(std::vector<Item>& out, int inst, int side, int pblks, int nms, int group) {
  for (int m0 = 0; m0 < nms; m0 += group)
    for (int b = 0; b < pblks; ++b) out.push_back(Item{inst, side, b, m0, std::min(group, nms - m0)});
}

// ---------------------------------------------------------------------------------------------
// Instance: device buffers and set-up
// ---------------------------------------------------------------------------------------------
struct Carve {
  size_t off = 0;
  template <class T>
  size_t take(size_t count) {
    const size_t o = (off + 255) & ~(size_t)255;
    off = o + count * sizeof(T);
    return o;
  }
};

#define OT_CUDA(call)                                                                 \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) {                                                          \
      ctx.set_error("%s failed: %s", #call, cudaGetErrorString(e_));                 \
      return OT_ECUDA;                                                                \
    }                                                                                 \
  } while (0)

int sweep_mode_of(int precision) {
  if (precision == OT_FP64) return kSweepF64;
  if (precision == OT_FP32_COMP) return kSweepComp;
  if (precision == OT_EXP_POLY) return kSweepFastPoly;
  if (precision == OT_EXP_SPLIT) return kSweepFastSplit;
  return kSweepFast;
}

// Refinement of the fast sweeps' dominant terms (OT_EXP_MUFU; see ot_params): on when the FP32
// exponent's rounding bound (base 2) exceeds refine_on > 0, with refine_tol the error the unrefined
// terms may carry (0: the default).  refine_on <= 0: off (*on = 0).
constexpr double kRefineTolDefault = 1e-5;
void refine_policy(const ot_params* q, double* on, double* tol) {
  *on = 0.0;
  *tol = q->refine_tol > 0.0 ? q->refine_tol : kRefineTolDefault;
  if (q->precision != OT_EXP_MUFU || !(q->refine_on > 0.0)) return;
  *on = q->refine_on;
}

ot_status validate(Context& ctx, const ot_problem* p, const ot_params* q) {
  if (!p || !q) {
    ctx.set_error("null problem or params");
    return OT_EINVAL;
  }
  if (p->n < 1 || p->m < 1 || p->n >= (1ll << 31) - kTQ || p->m >= (1ll << 31) - kTQ) {
    ctx.set_error("sizes must satisfy 1 <= n, m < 2^31 (got n=%lld m=%lld)", (long long)p->n, (long long)p->m);
    return OT_EINVAL;
  }
  if (p->d < 1 || p->d > 3) {
    ctx.set_error("d must be 1, 2 or 3 (got %d)", p->d);
    return OT_EINVAL;
  }
  if (!p->x || !p->y || !p->a || !p->b) {
    ctx.set_error("null x, y, a or b");
    return OT_EINVAL;
  }
  if (!(p->cost_scale >= 0.0) || !std::isfinite(p->cost_scale) || !(p->omega >= 0.0) || !std::isfinite(p->omega) ||
      !(p->zero_mass_floor >= 0.0)) {
    ctx.set_error("cost_scale, omega and zero_mass_floor must be finite and >= 0");
    return OT_EINVAL;
  }
  if (!std::isfinite(q->refine_on) || !(q->refine_tol >= 0.0) || !std::isfinite(q->refine_tol)) {
    ctx.set_error("refine_on and refine_tol must be finite (refine_tol >= 0)");
    return OT_EINVAL;
  }
  if (!(q->eps0 > 0.0) || !std::isfinite(q->eps0)) {
    ctx.set_error("eps0 must be finite and > 0");
    return OT_EINVAL;
  }
  if (!(q->lambda >= 1.0 && q->lambda < 2.0)) {
    ctx.set_error("lambda must lie in [1, 2) (got %g)", q->lambda);
    return OT_EINVAL;
  }
  if (q->algorithm < OT_ALG_BDRS || q->algorithm > OT_ALG_DAS) {
    ctx.set_error("unknown algorithm %d", q->algorithm);
    return OT_EINVAL;
  }
  if (q->algorithm != OT_ALG_BDRS && q->lambda != 1.0) {
    ctx.set_error("the annealed-Sinkhorn ablation methods run on the lambda = 1 schedule");
    return OT_EINVAL;
  }
  if (alg_old_kernel(q->algorithm) && q->cert_every != 0) {
    ctx.set_error("certificates need a current-kernel row update: set cert_every = 0 for this algorithm");
    return OT_EINVAL;
  }
  if (q->max_iters < 0 || q->cert_every < 0) {
    ctx.set_error("max_iters and cert_every must be >= 0");
    return OT_EINVAL;
  }
  if (q->precision != OT_EXP_MUFU && q->precision != OT_FP64 && q->precision != OT_FP32_COMP &&
      q->precision != OT_EXP_POLY && q->precision != OT_EXP_SPLIT) {
    ctx.set_error("unknown precision %d", q->precision);
    return OT_EINVAL;
  }
  return OT_OK;
}

// Validate, plan and lay out the device buffers of an instance (no allocation): in.bytes is the
// device memory the instance will hold.
ot_status instance_prepare(Context& ctx, Instance& in, const ot_problem* p, const ot_params* q, cudaStream_t stream) {
  ot_status vs = validate(ctx, p, q);
  if (vs != OT_OK) return vs;
  in.n = p->n;
  in.m = p->m;
  in.d = p->d;
  in.params = *q;
  in.stream = stream;
  in.sweep_mode = sweep_mode_of(q->precision);
  in.cert_mode = q->precision == OT_FP64 ? kSweepF64 : kSweepComp;
  refine_policy(q, &in.refine_on, &in.refine_tol);
  plan_launch(ctx, in, in.sweep_mode, in.fast);
  plan_launch(ctx, in, in.cert_mode, in.cert);
  Inst& h = in.h;
  h.tiles_x = (int)((in.n + kTQ - 1) / kTQ);
  h.tiles_y = (int)((in.m + kTQ - 1) / kTQ);
  h.pblk_x = in.cert.pblk_row;
  h.wait_limit = ctx.wait_limit;
  {
    const LaunchPlan* pls[2] = {&in.fast, &in.cert};
    for (int q = 0; q < 2; ++q) {
      h.nms[q][0] = pls[q]->nms_row;
      h.nms[q][1] = pls[q]->nms_col;
      h.ms_tiles[q][0] = pls[q]->mst_row;
      h.ms_tiles[q][1] = pls[q]->mst_col;
    }
  }
  h.n = (int)in.n;
  h.m = (int)in.m;
  h.d = in.d;
  h.eta = q->eps0;
  h.lambda = q->lambda;
  h.alg = q->algorithm;
  h.slice[0][0] = 0;
  h.slice[0][1] = (int)in.n;
  h.slice[1][0] = 0;
  h.slice[1][1] = (int)in.m;

  const size_t n = in.n, m = in.m;
  size_t nsp = 0;
  for (const LaunchPlan* pl : {&in.fast, &in.cert})
    nsp = std::max(nsp, std::max((size_t)pl->nms_row * n, (size_t)pl->nms_col * m));
  const size_t maxblk = (std::max(n, m) + kThreads - 1) / kThreads;
  Layout& L = in.layout;
  Carve cv;
  L.xpack = cv.take<float>((size_t)h.tiles_x * kNComp * kTQ);
  L.ypack = cv.take<float>((size_t)h.tiles_y * kNComp * kTQ);
  L.xraw = cv.take<float>(n * in.d);
  L.yraw = cv.take<float>(m * in.d);
  L.a = cv.take<double>(n);
  L.b = cv.take<double>(m);
  L.ain = cv.take<double>(n);
  L.bin = cv.take<double>(m);
  L.la = cv.take<double>(n);
  L.lb = cv.take<double>(m);
  L.xn2 = cv.take<double>(n);
  L.yn2 = cv.take<double>(m);
  L.state0 = cv.take<double>(2 * n + 5 * m);  // alpha, alpha_hat, beta, beta_prev, beta_hat, tilde, tilde_next
  L.fg = cv.take<double>(2 * (n + m));         // f_cur, g_cur, f_best, g_best
  L.hint = cv.take<float>(n + m);              // shift hints, row side then column side
  L.part = cv.take<PartF64>(nsp);
  L.cnt = cv.take<unsigned>(maxblk + 4);  // point-block counters, epilogue counter, 3 scheduler counters
  L.maxblk = maxblk;
  L.blk = cv.take<double>((n + kThreads - 1) / kThreads + 3 * ((m + kThreads - 1) / kThreads));
  L.ctrl = cv.take<double>(40);  // see instance_setup for the slots
  L.range = cv.take<unsigned>(2);
  L.inst = cv.take<Inst>(1);
  const size_t n_items = (size_t)in.fast.n_row + in.fast.n_col + in.cert.n_row + in.cert.n_col;
  L.items = cv.take<Item>(n_items);
  in.bytes = cv.off;
  return OT_OK;
}

// Allocate, upload and initialise a prepared instance (Algorithm 1 initialisation).
ot_status instance_setup(Context& ctx, Instance& in, const ot_problem* p) {
  Inst& h = in.h;
  const size_t n = in.n, m = in.m;
  const Layout& L = in.layout;
  const size_t maxblk = L.maxblk;
  const size_t o_xpack = L.xpack, o_ypack = L.ypack, o_xraw = L.xraw, o_yraw = L.yraw, o_a = L.a, o_b = L.b,
               o_ain = L.ain, o_bin = L.bin, o_la = L.la, o_lb = L.lb, o_xn2 = L.xn2, o_yn2 = L.yn2,
               o_state0 = L.state0, o_fg = L.fg, o_part = L.part, o_cnt = L.cnt, o_blk = L.blk, o_ctrl = L.ctrl,
               o_range = L.range, o_inst = L.inst, o_items = L.items;
  (void)o_blk;
  cudaError_t ae = in.async_alloc ? cudaMallocAsync(&in.mem, in.bytes, in.stream) : cudaMalloc(&in.mem, in.bytes);
  if (ae != cudaSuccess) {
    cudaGetLastError();
    in.mem = nullptr;
    ctx.set_error("device allocation of %zu bytes failed", in.bytes);
    return OT_ENOMEM;
  }
  char* base = (char*)in.mem;
  h.xpack = (float*)(base + o_xpack);
  h.ypack = (float*)(base + o_ypack);
  in.xraw = (float*)(base + o_xraw);
  in.yraw = (float*)(base + o_yraw);
  h.a = (double*)(base + o_a);
  h.b = (double*)(base + o_b);
  double* ain = (double*)(base + o_ain);
  double* bin = (double*)(base + o_bin);
  h.log_a = (double*)(base + o_la);
  h.log_b = (double*)(base + o_lb);
  h.xn2 = (double*)(base + o_xn2);
  h.yn2 = (double*)(base + o_yn2);
  double* s0 = (double*)(base + o_state0);
  h.log_alpha = s0;
  h.log_alpha_hat = s0 + n;
  h.log_beta = s0 + 2 * n;
  h.log_beta_prev = s0 + 2 * n + m;
  h.log_beta_hat = s0 + 2 * n + 2 * m;
  h.log_beta_tilde = s0 + 2 * n + 3 * m;
  h.log_beta_tilde_next = s0 + 2 * n + 4 * m;
  double* fg = (double*)(base + o_fg);
  h.f_cur = fg;
  h.g_cur = fg + n;
  h.hint[0] = (float*)(base + L.hint);
  h.hint[1] = h.hint[0] + n;
  in.f_best = fg + n + m;
  in.g_best = fg + 2 * n + m;
  h.part = base + o_part;
  h.cnt = (unsigned*)(base + o_cnt);
  h.done = h.cnt + maxblk;
  in.sched = h.cnt + maxblk + 1;
  h.blk = (double*)(base + o_blk);
  double* ctrl = (double*)(base + o_ctrl);
  h.cert = ctrl;
  h.k = (long long*)(ctrl + 8);
  h.err = (int*)(ctrl + 9);
  h.hint_bad = (int*)(ctrl + 14);  // ctrl[14..15]: four hint-miss counters (zeroed: see the k >= 1 rule)
  h.rows = (long long*)(ctrl + 16);
  h.k0 = (long long*)(ctrl + 17);
  h.recomp = (unsigned long long*)(ctrl + 18);  // ctrl[18]: tile recomputes of the fast sweeps
  h.goff = ctrl + 24;  // ctrl[24..31]: pack offsets, seeded by the column repack
  in.ctrl = ctrl;
  unsigned* range = (unsigned*)(base + o_range);
  in.d_inst = (Inst*)(base + o_inst);
  Item* items_base = (Item*)(base + o_items);
  in.fast.d_row = items_base;
  in.fast.d_col = in.fast.d_row + in.fast.n_row;
  in.cert.d_row = in.fast.d_col + in.fast.n_col;
  in.cert.d_col = in.cert.d_row + in.cert.n_row;

  cudaStream_t s = in.stream;
  OT_CUDA(cudaMemsetAsync(in.mem, 0, in.bytes, s));
  const cudaMemcpyKind k_in = p->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  OT_CUDA(cudaMemcpyAsync(in.xraw, p->x, n * in.d * sizeof(float), k_in, s));
  OT_CUDA(cudaMemcpyAsync(in.yraw, p->y, m * in.d * sizeof(float), k_in, s));
  OT_CUDA(cudaMemcpyAsync(ain, p->a, n * sizeof(double), k_in, s));
  OT_CUDA(cudaMemcpyAsync(bin, p->b, m * sizeof(double), k_in, s));

  // cost scale and oscillation bound (App. G: kappa = 1 / max pair cost; omega >= osc(C))
  double kappa = p->cost_scale, omega = p->omega;
  if (kappa == 0.0 || omega == 0.0) {
    const unsigned init[2] = {0u, 0x7f7fffffu};
    OT_CUDA(cudaMemcpyAsync(range, init, sizeof(init), cudaMemcpyHostToDevice, s));
    OT_CUDA(launch_pair_cost_range(in.xraw, (int)n, in.yraw, (int)m, in.d, range, range + 1, ctx.sms, s));
    ctx.launches += 1;
    unsigned hr[2];
    OT_CUDA(cudaMemcpyAsync(hr, range, sizeof(hr), cudaMemcpyDeviceToHost, s));
    OT_CUDA(cudaStreamSynchronize(s));
    float fmx, fmn;
    memcpy(&fmx, &hr[0], 4);
    memcpy(&fmn, &hr[1], 4);
    if (kappa == 0.0) {
      if (!(fmx > 0.0f)) {
        ctx.set_error("all pair costs are zero: cost_scale must be given");
        return OT_EINVAL;
      }
      kappa = 1.0 / (double)fmx;
    }
    if (omega == 0.0) omega = kappa * ((double)fmx - (double)fmn);
    if (!(omega > 0.0)) omega = kappa * (double)fmx;
  }
  h.kappa = kappa;
  h.omega = omega;
  in.kappa = kappa;
  in.omega = omega;

  // ctrl[32..35]: scratch of the exact centring; ctrl[36..37]: its translation (3 floats, zeros when
  // it would not be exact), which the packs subtract and the barycentric projection adds back;
  // ctrl[38]: the exponent bound of the fast sweeps' refinement; ctrl[39]: refined warp-tiles
  float* origin = (float*)(ctrl + 36);
  h.origin = origin;
  h.rzeps = ctrl + 38;
  h.refined = (unsigned long long*)(ctrl + 39);
  h.refine_on = in.refine_on;
  h.refine_tol = in.refine_tol;
  OT_CUDA(launch_centre(in.xraw, (int)n, in.yraw, (int)m, in.d, (int*)(ctrl + 32), origin, kappa, omega, ctrl + 38,
                        ctx.sms, s));
  OT_CUDA(launch_pack_coords(in.xraw, (int)n, in.d, h.tiles_x, kappa, h.xpack, (double*)h.xn2, s, h.origin));
  OT_CUDA(launch_pack_coords(in.yraw, (int)m, in.d, h.tiles_y, kappa, h.ypack, (double*)h.yn2, s, h.origin));
  // ctrl[10..13]: scratch of the two normalisations (total, arrival counter), zeroed above
  OT_CUDA(launch_normalise(ain, (int)n, p->zero_mass_floor, (double*)h.a, (double*)h.log_a, ctrl + 10, h.err, s));
  OT_CUDA(launch_normalise(bin, (int)m, p->zero_mass_floor, (double*)h.b, (double*)h.log_b, ctrl + 12, h.err, s));
  ctx.launches += 9;

  std::vector<Item> items;
  for (const LaunchPlan* pl : {&in.fast, &in.cert}) {
    build_items(items, 0, 0, pl->pblk_row, pl->nms_row, pl->group_row);
    build_items(items, 0, 1, pl->pblk_col, pl->nms_col, pl->group_col);
  }
  OT_CUDA(cudaMemcpyAsync(items_base, items.data(), items.size() * sizeof(Item), cudaMemcpyHostToDevice, s));
  OT_CUDA(cudaMemcpyAsync(in.d_inst, &h, sizeof(Inst), cudaMemcpyHostToDevice, s));
  OT_CUDA(launch_repack_cols(in.d_inst, (int)m, s));
  ctx.launches += 1;
  if (in.h_ctrl_external) {
    in.h_ctrl = in.h_ctrl_external;
  } else if (cudaMallocHost(&in.h_ctrl, 16 * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    in.h_ctrl = nullptr;
    ctx.set_error("cudaMallocHost failed");
    return OT_ENOMEM;
  }
  OT_CUDA(cudaMemcpyAsync(in.h_ctrl, in.ctrl, 16 * sizeof(double), cudaMemcpyDeviceToHost, s));
  OT_CUDA(cudaStreamSynchronize(s));
  const int err = ((int*)in.h_ctrl)[18];
  if (err & kErrNonFinite) {
    ctx.set_error("weights must be finite and > 0 (or set zero_mass_floor)");
    return OT_EINVAL;
  }
  in.k = 0;
  return OT_OK;
}

ot_status instance_init(Context& ctx, Instance& in, const ot_problem* p, const ot_params* q, cudaStream_t stream) {
  ot_status st = instance_prepare(ctx, in, p, q, stream);
  if (st != OT_OK) return st;
  return instance_setup(ctx, in, p);
}

void instance_free(Instance& in) {
  for (auto& kv : in.graphs) cudaGraphExecDestroy(kv.second);
  in.graphs.clear();
  for (auto& kv : in.graph_events)
    for (cudaEvent_t e : kv.second) cudaEventDestroy(e);
  in.graph_events.clear();
  if (in.mem) {
    if (in.async_alloc)
      cudaFreeAsync(in.mem, in.stream);
    else
      cudaFree(in.mem);
  }
  if (in.h_ctrl && !in.h_ctrl_external) cudaFreeHost(in.h_ctrl);
  in.mem = nullptr;
  in.h_ctrl = nullptr;
}

// ---------------------------------------------------------------------------------------------
// Iterations
// ---------------------------------------------------------------------------------------------
// `iters` iterations of one plan as one launch (row and column sweeps of every iteration).
// (More than 2^30 tickets are split over several launches: the kernel counts tickets in int.)
static cudaError_t launch_iterations(Instance& in, bool cert, int64_t iters) {
  const LaunchPlan& pl = cert ? in.cert : in.fast;
  SweepFn fn = get_sweep(in.d, pl.mode, pl.R, pl.ch, cert ? 1 : 0);
  const int nitems = pl.n_row + pl.n_col;
  const int64_t per_launch = std::max<int64_t>(1, ((int64_t)1 << 30) / nitems);
  for (int64_t done = 0; done < iters;) {
    const int64_t j = std::min(iters - done, per_launch);
    // one iteration's items bound the useful CTAs: more would only wait for the next phase
    const int grid = std::min(nitems, pl.resident);
    const cudaError_t e = launch_sweep(fn, in.d_inst, pl.d_row, nitems, (int)j, grid, in.sched, in.stream);
    if (e != cudaSuccess) return e;
    done += j;
  }
  return cudaSuccess;
}

// A chunk: its fast iterations as one launch, then the certificate iteration (if any) as another;
// in profiling mode an event before, between and after them (ev[0..2]).
static cudaError_t issue_launches(Instance& in, int64_t count, bool cert_last, cudaEvent_t* ev) {
  const int64_t nfast = count - (cert_last ? 1 : 0);
  cudaError_t e;
  if (ev && (e = cudaEventRecordWithFlags(ev[0], in.stream, cudaEventRecordExternal)) != cudaSuccess) return e;
  if (nfast > 0 && (e = launch_iterations(in, false, nfast)) != cudaSuccess) return e;
  if (ev && (e = cudaEventRecordWithFlags(ev[1], in.stream, cudaEventRecordExternal)) != cudaSuccess) return e;
  if (cert_last && (e = launch_iterations(in, true, 1)) != cudaSuccess) return e;
  if (ev && (e = cudaEventRecordWithFlags(ev[2], in.stream, cudaEventRecordExternal)) != cudaSuccess) return e;
  return cudaSuccess;
}

// `count` iterations, the last one a certificate iteration if cert_last: at most two launches,
// replayed from a CUDA graph.  In profiling mode the graph also records events around them and the
// chunk is waited for, so that the launch durations can be read.
static ot_status issue_chunk(Context& ctx, Instance& in, int64_t count, bool cert_last) {
  if (count <= 0) return OT_OK;
  const bool prof = ctx.profile;
  const std::pair<int64_t, int> key(count, (cert_last ? 1 : 0) | (prof ? 2 : 0));
  auto it = in.graphs.find(key);
  std::vector<cudaEvent_t>* evs = nullptr;
  if (prof) {
    evs = &in.graph_events[key];
    if (evs->empty()) {
      evs->resize(3);
      for (auto& e : *evs) OT_CUDA(cudaEventCreate(&e));
    }
  }
  if (it == in.graphs.end() && in.use_graphs) {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    if (cudaStreamBeginCapture(in.stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      const cudaError_t e = issue_launches(in, count, cert_last, prof ? evs->data() : nullptr);
      const cudaError_t e2 = cudaStreamEndCapture(in.stream, &g);
      if (e == cudaSuccess && e2 == cudaSuccess && cudaGraphInstantiate(&ge, g, 0) == cudaSuccess) {
        it = in.graphs.emplace(key, ge).first;
      }
      if (g) cudaGraphDestroy(g);
    }
    cudaGetLastError();
  }
  if (it != in.graphs.end()) {
    OT_CUDA(cudaGraphLaunch(it->second, in.stream));
  } else {
    OT_CUDA(issue_launches(in, count, cert_last, prof ? evs->data() : nullptr));
  }
  const int64_t nfast = count - (cert_last ? 1 : 0);
  in.k += count;
  ctx.launches += (nfast > 0 ? 1 : 0) + (cert_last ? 1 : 0);
  if (prof) {
    OT_CUDA(cudaStreamSynchronize(in.stream));
    const double entries = 2.0 * (double)in.n * (double)in.m;  // row and column sweep
    float ms[2] = {0, 0};
    OT_CUDA(cudaEventElapsedTime(&ms[0], (*evs)[0], (*evs)[1]));
    OT_CUDA(cudaEventElapsedTime(&ms[1], (*evs)[1], (*evs)[2]));
    const int64_t its[2] = {nfast, cert_last ? 1 : 0};
    for (int kind = 0; kind < 2; ++kind) {
      if (its[kind] <= 0) continue;
      KernelStats& ks = ctx.stats[kind];
      ks.launches += 1;
      ks.entries += entries * (double)its[kind];
      ks.ms += ms[kind];
    }
  }
  return OT_OK;
}

// Read the control block (certificate record, k, error bits) after the stream drains.
ot_status read_ctrl(Context& ctx, Instance& in) {
  OT_CUDA(cudaMemcpyAsync(in.h_ctrl, in.ctrl, 16 * sizeof(double), cudaMemcpyDeviceToHost, in.stream));
  OT_CUDA(cudaStreamSynchronize(in.stream));
  const int err = ((int*)in.h_ctrl)[18];
  in.device_errors |= err;
  if (err & kErrTimeout) {
    ctx.set_error("a device wait exceeded its bound");
    return OT_ETIMEDOUT;
  }
  if (err & kErrNonFinite) {
    ctx.set_error("non-finite potential at iteration %lld", (long long)in.k);
    return OT_ENUMERIC;
  }
  return OT_OK;
}

// Fold the certificate just read into the best-so-far bounds (App. G.3) and the retained iterate.
ot_status absorb_cert(Context& ctx, Instance& in) {
  const double* c = in.h_ctrl;
  in.U = c[kCertU];
  in.L = c[kCertL];
  in.eps_last = c[kCertEps];
  in.n_certs += 1;
  in.last_cert_k = in.k;
  in.U_best = std::min(in.U_best, in.U);
  in.L_best = std::max(in.L_best, in.L);
  const double rel = (in.U - in.L) / std::fabs(in.U);
  if (in.best_iter < 0 || rel < in.best_rel) {
    in.best_rel = rel;
    in.best_iter = in.k - 1;
    OT_CUDA(cudaMemcpyAsync(in.f_best, in.h.f_cur, in.n * sizeof(double), cudaMemcpyDeviceToDevice, in.stream));
    OT_CUDA(cudaMemcpyAsync(in.g_best, in.h.g_cur, in.m * sizeof(double), cudaMemcpyDeviceToDevice, in.stream));
  }
  return OT_OK;
}

void fill_result(const Instance& in, ot_result* r) {
  if (!r) return;
  r->iters = in.k;
  r->best_iter = in.best_iter;
  r->n_certs = in.n_certs;
  r->U = in.U;
  r->L = in.L;
  r->U_best = in.U_best;
  r->L_best = in.L_best;
  r->gap_abs = in.U_best - in.L_best;
  r->gap_rel = (in.U_best - in.L_best) / std::fabs(in.U_best);
  r->eps_final = in.k > 0 ? in.h.eta / (in.h.lambda * (double)(in.k - 1) + 1.0) : in.h.eta;
  r->elapsed_s = in.elapsed_s;
  r->kappa = in.kappa;
  r->omega = in.omega;
  r->stop = in.stop;
  r->device_errors = in.device_errors;
  r->latency_s = 0;
  r->queue_s = 0;
}

// Run n iterations; certificate iterations where (k+1) % cert_every == 0, plus the final iteration
// when final_cert.  Stops early when `stop_rule` and the tolerance is met or time runs out.
ot_status run_iterations(Context& ctx, Instance& in, int64_t n_iters, bool stop_rule, bool final_cert) {
  const auto t0 = std::chrono::steady_clock::now();
  const int ce = in.params.cert_every;
  const int64_t k_end = in.k + n_iters;
  in.stop = OT_STOP_NONE;
  while (in.k < k_end) {
    int64_t chunk = k_end - in.k;
    if (ce > 0) chunk = std::min<int64_t>(chunk, ce - (in.k % ce));
    const bool cert = ce > 0 && ((in.k + chunk) % ce == 0 || (final_cert && in.k + chunk == k_end));
    ot_status st = issue_chunk(ctx, in, chunk, cert);
    if (st != OT_OK) return st;
    if (cert || in.k == k_end) {
      st = read_ctrl(ctx, in);
      if (st != OT_OK) return st;
      if (cert) {
        st = absorb_cert(ctx, in);
        if (st != OT_OK) return st;
      }
    }
    const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    in.elapsed_s = in.elapsed_base + el;
    if (stop_rule && cert) {
      const double gap = in.U_best - in.L_best;
      const double ta = in.params.tol_abs, tr = in.params.tol_rel;
      if ((ta > 0 && gap <= ta) || (tr > 0 && gap <= tr * std::fabs(in.U_best))) {
        in.stop = OT_STOP_TOL;
        break;
      }
    }
    if (stop_rule && in.params.time_budget_s > 0 && el >= in.params.time_budget_s) {
      in.stop = OT_STOP_TIME;
      break;
    }
  }
  if (in.stop == OT_STOP_NONE && stop_rule) in.stop = OT_STOP_MAX_ITERS;
  in.elapsed_base = in.elapsed_s;
  return OT_OK;
}

ot_status standalone_certificate(Context& ctx, Instance& in) {
  const LaunchPlan& pl = in.cert;
  SweepFn fc = get_sweep(in.d, pl.mode, pl.R, pl.ch, 2);
  OT_CUDA(launch_sweep(fc, in.d_inst, pl.d_col, pl.n_col, 1, std::min(pl.n_col, pl.resident), in.sched, in.stream));
  ctx.launches += 1;
  return read_ctrl(ctx, in);
}

}  // namespace ot

// =============================================================================================
// C ABI
// =============================================================================================
using namespace ot;

struct ot_context {
  Context c;
};
struct ot_state {
  ot_context* ctx;
  Instance in;
};

extern "C" {

void ot_params_default(ot_params* p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->eps0 = 1.0;
  p->lambda = 1.0;
  p->max_iters = 1000;
  p->cert_every = 100;
  p->precision = OT_EXP_MUFU;
}

const char* ot_status_str(ot_status s) {
  switch (s) {
    case OT_OK: return "OT_OK";
    case OT_EINVAL: return "OT_EINVAL: invalid argument";
    case OT_ENOMEM: return "OT_ENOMEM: allocation failed";
    case OT_ECUDA: return "OT_ECUDA: CUDA error";
    case OT_ENUMERIC: return "OT_ENUMERIC: non-finite value";
    case OT_ETIMEDOUT: return "OT_ETIMEDOUT: device wait bound exceeded";
    case OT_EBUSY: return "OT_EBUSY: not finished";
    case OT_ECANCELLED: return "OT_ECANCELLED: cancelled";
    case OT_ENOTFOUND: return "OT_ENOTFOUND: unknown request";
  }
  return "unknown status";
}

const char* ot_last_error(const ot_context* ctx) { return ctx ? ctx->c.last_error.c_str() : "null context"; }

ot_status ot_context_create(int device, ot_context** out) {
  if (!out) return OT_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return OT_EINVAL;
  }
  if (cudaSetDevice(device) != cudaSuccess) return OT_ECUDA;
  static std::once_flag plans_once;
  std::call_once(plans_once, load_tile_plans);
  ot_context* c = new (std::nothrow) ot_context();
  if (!c) return OT_ENOMEM;
  c->c.device = device;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->c.stream, cudaStreamNonBlocking) != cudaSuccess) {
    delete c;
    return OT_ECUDA;
  }
  c->c.sms = prop.multiProcessorCount;
  c->c.cc_major = prop.major;
  c->c.cc_minor = prop.minor;
  *out = c;
  return OT_OK;
}

void ot_context_destroy(ot_context* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->c.device);
  if (ctx->c.stream) cudaStreamDestroy(ctx->c.stream);
  delete ctx;
}

static cudaStream_t pick_stream(ot_context* ctx, const ot_params* p) {
  return (p && p->stream) ? (cudaStream_t)(uintptr_t)p->stream : ctx->c.stream;
}

ot_status ot_state_create(ot_context* ctx, const ot_problem* prob, const ot_params* params, ot_state** out) {
  if (!ctx || !out) return OT_EINVAL;
  *out = nullptr;
  cudaSetDevice(ctx->c.device);
  ot_state* s = new (std::nothrow) ot_state();
  if (!s) return OT_ENOMEM;
  s->ctx = ctx;
  ot_status st = instance_init(ctx->c, s->in, prob, params, pick_stream(ctx, params));
  if (st != OT_OK) {
    instance_free(s->in);
    delete s;
    return st;
  }
  *out = s;
  return OT_OK;
}

void ot_state_destroy(ot_state* st) {
  if (!st) return;
  cudaSetDevice(st->ctx->c.device);
  cudaStreamSynchronize(st->in.stream);
  instance_free(st->in);
  delete st;
}

ot_status ot_step(ot_state* st, int64_t n_iters, ot_result* res) {
  if (!st || n_iters < 0 || st->in.shard_world > 0) return OT_EINVAL;
  cudaSetDevice(st->ctx->c.device);
  ot_status s = run_iterations(st->ctx->c, st->in, n_iters, false, false);
  if (s == OT_OK && st->in.k > 0) s = read_ctrl(st->ctx->c, st->in);
  fill_result(st->in, res);
  return s;
}

ot_status ot_certificate(ot_state* st, ot_result* res) {
  if (!st || st->in.shard_world > 0) return OT_EINVAL;
  Instance& in = st->in;
  if (in.k < 1) {
    st->ctx->c.set_error("no completed iteration to certify");
    return OT_EINVAL;
  }
  if (alg_old_kernel(in.h.alg)) {
    st->ctx->c.set_error("no certificate for an old-kernel row update (Prop. 3's intermediate plan needs the current one)");
    return OT_EINVAL;
  }
  cudaSetDevice(st->ctx->c.device);
  if (in.last_cert_k != in.k) {
    ot_status s = standalone_certificate(st->ctx->c, in);
    if (s != OT_OK) return s;
  } else {
    ot_status s = read_ctrl(st->ctx->c, in);
    if (s != OT_OK) return s;
  }
  fill_result(in, res);
  if (res) {
    res->U = in.h_ctrl[kCertU];
    res->L = in.h_ctrl[kCertL];
    res->eps_final = in.h_ctrl[kCertEps];
  }
  return OT_OK;
}

static double* vec_ptr(Instance& in, int which, size_t* len) {
  Inst& h = in.h;
  switch (which) {
    case OT_LOG_ALPHA: *len = in.n; return h.log_alpha;
    case OT_LOG_ALPHA_HAT: *len = in.n; return h.log_alpha_hat;
    case OT_LOG_BETA: *len = in.m; return h.log_beta;
    case OT_LOG_BETA_PREV: *len = in.m; return h.log_beta_prev;
    case OT_LOG_BETA_HAT: *len = in.m; return h.log_beta_hat;
    case OT_LOG_BETA_TILDE: *len = in.m; return h.log_beta_tilde;
    case OT_F_CERT: *len = in.n; return h.f_cur;
    case OT_G_CERT: *len = in.m; return h.g_cur;
    case OT_F_BEST: *len = in.n; return in.f_best;
    case OT_G_BEST: *len = in.m; return in.g_best;
  }
  return nullptr;
}

ot_status ot_state_get(ot_state* st, int which, double* out, int64_t* k) {
  if (!st) return OT_EINVAL;
  Context& ctx = st->ctx->c;
  cudaSetDevice(ctx.device);
  size_t len = 0;
  double* p = vec_ptr(st->in, which, &len);
  if (!p) return OT_EINVAL;
  if (out) {
    OT_CUDA(cudaMemcpyAsync(out, p, len * sizeof(double), cudaMemcpyDeviceToHost, st->in.stream));
    OT_CUDA(cudaStreamSynchronize(st->in.stream));
  }
  if (k) *k = st->in.k;
  return OT_OK;
}

ot_status ot_state_set(ot_state* st, int which, const double* in_vec, int64_t k) {
  if (!st || !in_vec || k < 0) return OT_EINVAL;
  if (which != OT_LOG_ALPHA && which != OT_LOG_BETA && which != OT_LOG_BETA_PREV) return OT_EINVAL;
  Context& ctx = st->ctx->c;
  Instance& in = st->in;
  cudaSetDevice(ctx.device);
  size_t len = 0;
  double* p = vec_ptr(in, which, &len);
  OT_CUDA(cudaMemcpyAsync(p, in_vec, len * sizeof(double), cudaMemcpyHostToDevice, in.stream));
  // k, the completed row sweeps and the next launch's starting k all become k
  const long long kk[2] = {k, k};
  OT_CUDA(cudaMemcpyAsync(in.h.k, &kk[0], sizeof(long long), cudaMemcpyHostToDevice, in.stream));
  OT_CUDA(cudaMemcpyAsync(in.h.rows, kk, 2 * sizeof(long long), cudaMemcpyHostToDevice, in.stream));
  // the stored shift hints belong to the replaced state: mark both sides as missed, so the next
  // iteration runs without them and re-validates its own
  static const int kMissed[4] = {1, 1, 1, 1};
  OT_CUDA(cudaMemcpyAsync(in.h.hint_bad, kMissed, sizeof(kMissed), cudaMemcpyHostToDevice, in.stream));
  OT_CUDA(launch_repack_cols(in.d_inst, (int)in.m, in.stream));
  ctx.launches += 1;
  OT_CUDA(cudaStreamSynchronize(in.stream));
  in.k = k;
  in.last_cert_k = -1;
  return OT_OK;
}

ot_status ot_profile_enable(ot_context* ctx, int on) {
  if (!ctx) return OT_EINVAL;
  ctx->c.profile = on != 0;
  return OT_OK;
}

ot_status ot_profile_reset(ot_context* ctx) {
  if (!ctx) return OT_EINVAL;
  for (auto& s : ctx->c.stats) s = KernelStats();
  ctx->c.launches = 0;
  return OT_OK;
}

ot_status ot_debug_set_wait_limit(ot_context* ctx, uint32_t polls) {
  if (!ctx) return OT_EINVAL;
  ctx->c.wait_limit = polls;
  return OT_OK;
}

ot_status ot_launch_count(ot_context* ctx, int64_t* launches) {
  if (!ctx || !launches) return OT_EINVAL;
  *launches = ctx->c.launches;
  return OT_OK;
}

ot_status ot_state_counters(ot_state* st, int64_t* out, int32_t nout) {
  if (!st || !out || nout < 9) return OT_EINVAL;
  Context& ctx = st->ctx->c;
  Instance& in = st->in;
  cudaSetDevice(ctx.device);
  double c[40];
  OT_CUDA(cudaMemcpyAsync(c, in.ctrl, sizeof(c), cudaMemcpyDeviceToHost, in.stream));
  OT_CUDA(cudaStreamSynchronize(in.stream));
  int hb[4];
  memcpy(hb, &c[14], sizeof(hb));
  unsigned long long rc;
  memcpy(&rc, &c[18], sizeof(rc));
  for (int i = 0; i < 4; ++i) out[i] = hb[i];
  out[4] = (int64_t)rc;
  out[5] = in.fast.nms_row;
  out[6] = in.fast.nms_col;
  out[7] = in.cert.nms_row;
  out[8] = in.cert.nms_col;
  if (nout >= 10) {
    unsigned long long rf;
    memcpy(&rf, &c[39], sizeof(rf));
    out[9] = (int64_t)rf;
  }
  return OT_OK;
}

ot_status ot_profile_read(ot_context* ctx, int kind, int64_t* launches, double* entries, double* ms) {
  if (!ctx || kind < 0 || kind > 1) return OT_EINVAL;
  const KernelStats& s = ctx->c.stats[kind];
  if (launches) *launches = s.launches;
  if (entries) *entries = s.entries;
  if (ms) *ms = s.ms;
  return OT_OK;
}

// Temperature of a state's plan (see ot_plan_kind); false with the error set if there is none.
static bool plan_eps(Context& ctx, const Instance& in, int32_t plan, double* eps) {
  if (plan == OT_PLAN_BEST) {
    if (in.best_iter < 0) {
      ctx.set_error("no certificate has been computed yet");
      return false;
    }
    *eps = in.h.eta / (in.h.lambda * (double)in.best_iter + 1.0);
  } else {
    if (in.k < 1) {
      ctx.set_error("the state has no completed iteration");
      return false;
    }
    *eps = in.h.eta / (in.h.lambda * (double)(in.k - 1) + 1.0);
  }
  return true;
}

ot_status ot_plan_round(ot_state* st, int32_t plan, double* cost_rounded, double* cost_unrounded) {
  if (!st || plan < OT_PLAN_BEST || plan > OT_PLAN_INTERMEDIATE) return OT_EINVAL;
  Context& ctx = st->ctx->c;
  Instance& in = st->in;
  cudaSetDevice(ctx.device);
  double eps;
  if (!plan_eps(ctx, in, plan, &eps)) return OT_EINVAL;
  const size_t o_sums = (round_scratch_bytes(in.n, in.m) + 255) & ~(size_t)255;
  const size_t bytes = o_sums + 16 * sizeof(double);
  char* mem = nullptr;
  if (cudaMalloc(&mem, bytes) != cudaSuccess) {
    cudaGetLastError();
    ctx.set_error("device allocation of %zu bytes failed", bytes);
    return OT_ENOMEM;
  }
  double h[16];
  cudaError_t e = plan_rounding(in.h, plan, eps, in.f_best, in.g_best, mem, (double*)(mem + o_sums), in.stream);
  ctx.launches += 10;
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, mem + o_sums, sizeof(h), cudaMemcpyDeviceToHost, in.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(in.stream);
  cudaFree(mem);
  if (e != cudaSuccess) {
    ctx.set_error("plan rounding failed: %s", cudaGetErrorString(e));
    return OT_ECUDA;
  }
  // rank-one correction err_r err_c^T / |err_r|_1 (separable cost; see plan_rounding)
  const double kappa = in.h.kappa;
  double corr = 0.0;
  if (h[5] > 0.0) {
    double cross = 0.0;
    for (int k = 0; k < in.d; ++k) cross += h[2 + k] * h[10 + k];
    corr = kappa * (h[0] * h[9] + h[1] * h[8] - 2.0 * cross) / h[5];
  }
  if (cost_rounded) *cost_rounded = h[6] + corr;
  if (cost_unrounded) *cost_unrounded = h[7];
  return OT_OK;
}

ot_status ot_plan_project(ot_state* st, int32_t plan, float* y_hat, double* row_sums, double* col_sums,
                          ot_marginal_errors* err) {
  if (!st || plan < OT_PLAN_BEST || plan > OT_PLAN_INTERMEDIATE) return OT_EINVAL;
  Context& ctx = st->ctx->c;
  Instance& in = st->in;
  cudaSetDevice(ctx.device);
  double eps;
  if (!plan_eps(ctx, in, plan, &eps)) return OT_EINVAL;
  const int64_t n = in.n, m = in.m;
  // one temporary allocation: working memory, then the device outputs
  const size_t o_y = (plan_scratch_bytes(n, m) + 255) & ~(size_t)255;
  const size_t o_row = (o_y + sizeof(float) * n * in.d + 255) & ~(size_t)255;
  const size_t o_col = (o_row + sizeof(double) * n + 255) & ~(size_t)255;
  const size_t o_err = (o_col + sizeof(double) * m + 255) & ~(size_t)255;
  const size_t bytes = o_err + 6 * sizeof(double);
  char* mem = nullptr;
  if (cudaMalloc(&mem, bytes) != cudaSuccess) {
    cudaGetLastError();
    ctx.set_error("device allocation of %zu bytes failed", bytes);
    return OT_ENOMEM;
  }
  ot_status status = OT_OK;
  double herr[6] = {0, 0, 0, 0, 0, 0};
  cudaError_t e = plan_diagnostics(in.h, plan, eps, in.f_best, in.g_best, mem, (float*)(mem + o_y),
                                   (double*)(mem + o_row), (double*)(mem + o_col), (double*)(mem + o_err), in.stream);
  ctx.launches += 7;
  if (e == cudaSuccess && y_hat)
    e = cudaMemcpyAsync(y_hat, mem + o_y, sizeof(float) * n * in.d, cudaMemcpyDeviceToHost, in.stream);
  if (e == cudaSuccess && row_sums)
    e = cudaMemcpyAsync(row_sums, mem + o_row, sizeof(double) * n, cudaMemcpyDeviceToHost, in.stream);
  if (e == cudaSuccess && col_sums)
    e = cudaMemcpyAsync(col_sums, mem + o_col, sizeof(double) * m, cudaMemcpyDeviceToHost, in.stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(herr, mem + o_err, sizeof(herr), cudaMemcpyDeviceToHost, in.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(in.stream);
  if (e != cudaSuccess) {
    ctx.set_error("plan diagnostics failed: %s", cudaGetErrorString(e));
    status = OT_ECUDA;
  }
  cudaFree(mem);
  if (status == OT_OK && err) {
    err->row_l1 = herr[0];
    err->row_max_abs = herr[1];
    err->row_max_rel = herr[2];
    err->col_l1 = herr[3];
    err->col_max_abs = herr[4];
    err->col_max_rel = herr[5];
    err->eps = eps;
  }
  return status;
}

ot_status ot_set_tile_plan(int32_t d, int32_t precision, int32_t R, int32_t ch) {
  if (precision < OT_EXP_MUFU || precision > OT_FP32_COMP) return OT_EINVAL;
  return set_tile(d, sweep_mode_of(precision), R, ch) ? OT_OK : OT_EINVAL;
}

ot_status ot_get_tile_plan(int32_t d, int32_t precision, int32_t* R, int32_t* ch) {
  if (d < 1 || d > 3 || precision < OT_EXP_MUFU || precision > OT_FP32_COMP || !R || !ch) return OT_EINVAL;
  int r, c;
  canonical_tile(d, sweep_mode_of(precision), &r, &c);
  *R = r;
  *ch = c;
  return OT_OK;
}

ot_status ot_state_cost(ot_state* st, double* kappa, double* omega) {
  if (!st) return OT_EINVAL;
  if (kappa) *kappa = st->in.kappa;
  if (omega) *omega = st->in.omega;
  return OT_OK;
}

ot_status ot_solve(ot_context* ctx, const ot_problem* prob, const ot_params* params, double* f_out, double* g_out,
                   ot_result* res) {
  if (!ctx) return OT_EINVAL;
  ot_state* st = nullptr;
  ot_status s = ot_state_create(ctx, prob, params, &st);
  if (s != OT_OK) return s;
  Context& c = ctx->c;
  Instance& in = st->in;
  s = run_iterations(c, in, params->max_iters, true, true);
  if (s == OT_OK) {
    const cudaMemcpyKind kd = prob->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    const bool have = in.best_iter >= 0;
    if (f_out && have &&
        cudaMemcpyAsync(f_out, in.f_best, in.n * sizeof(double), kd, in.stream) != cudaSuccess)
      s = OT_ECUDA;
    if (g_out && have &&
        cudaMemcpyAsync(g_out, in.g_best, in.m * sizeof(double), kd, in.stream) != cudaSuccess)
      s = OT_ECUDA;
    if (cudaStreamSynchronize(in.stream) != cudaSuccess) s = OT_ECUDA;
  }
  fill_result(in, res);
  ot_state_destroy(st);
  return s;
}

// ---------------------------------------------------------------------------------------------
// Row-sharded execution (one slice of the points per process; the host exchanges packed operands)
// ---------------------------------------------------------------------------------------------
namespace {
constexpr int kShardUnit = 4 * kTQ;  // slice granularity in points: a multiple of every point block

// Points [p0, p1) of `side` owned by `rank` of `world`: contiguous runs of whole 512-point units,
// split as evenly as the units allow.
void shard_range(int64_t np, int rank, int world, int64_t* p0, int64_t* p1) {
  const int64_t units = (np + kShardUnit - 1) / kShardUnit;
  *p0 = std::min<int64_t>(np, kShardUnit * (units * rank / world));
  *p1 = std::min<int64_t>(np, kShardUnit * (units * (rank + 1) / world));
}
}  // namespace

ot_status ot_shard_range(int64_t np, int32_t rank, int32_t world, int64_t* p0, int64_t* p1) {
  if (np < 1 || world < 1 || rank < 0 || rank >= world || !p0 || !p1) return OT_EINVAL;
  shard_range(np, rank, world, p0, p1);
  return OT_OK;
}

ot_status ot_shard_create(ot_context* ctx, const ot_problem* prob, const ot_params* params, int32_t rank,
                          int32_t world, ot_state** out) {
  if (!ctx || !out || !prob || world < 1 || rank < 0 || rank >= world) return OT_EINVAL;
  *out = nullptr;
  const int64_t ux = (prob->n + kShardUnit - 1) / kShardUnit, uy = (prob->m + kShardUnit - 1) / kShardUnit;
  if (prob->n < 1 || prob->m < 1 || ux < world || uy < world) {
    ctx->c.set_error("each of the %d ranks needs at least %d points of each side", world, kShardUnit);
    return OT_EINVAL;
  }
  ot_state* st = nullptr;
  ot_status s = ot_state_create(ctx, prob, params, &st);
  if (s != OT_OK) return s;
  Context& c = ctx->c;
  Instance& in = st->in;
  in.shard_rank = rank;
  in.shard_world = world;
  int64_t r[2][2];
  shard_range(in.n, rank, world, &r[0][0], &r[0][1]);
  shard_range(in.m, rank, world, &r[1][0], &r[1][1]);
  for (int side = 0; side < 2; ++side) {
    in.h.slice[side][0] = (int)r[side][0];
    in.h.slice[side][1] = (int)r[side][1];
  }
  // the slice's work items: the instance's items of its own point blocks, per plan and side
  std::vector<Item> items;
  int off[2][2];
  const LaunchPlan* pls[2] = {&in.fast, &in.cert};
  for (int q = 0; q < 2; ++q) {
    const LaunchPlan& pl = *pls[q];
    for (int side = 0; side < 2; ++side) {
      std::vector<Item> all;
      build_items(all, 0, side, side == 0 ? pl.pblk_row : pl.pblk_col, side == 0 ? pl.nms_row : pl.nms_col,
                  side == 0 ? pl.group_row : pl.group_col);
      const int rpb = kThreads * pl.R;
      const int b0 = (int)(r[side][0] / rpb), b1 = (int)((r[side][1] + rpb - 1) / rpb);
      off[q][side] = (int)items.size();
      for (const Item& it : all)
        if (it.pblk >= b0 && it.pblk < b1) items.push_back(it);
      in.shard_nitems[q][side] = (int)items.size() - off[q][side];
    }
  }
  Item* base = in.fast.d_row;  // the instance's item buffer (its items are not used by a slice)
  for (int q = 0; q < 2; ++q)
    for (int side = 0; side < 2; ++side) in.shard_items[q][side] = base + off[q][side];
  cudaError_t e = cudaMemcpyAsync(base, items.data(), items.size() * sizeof(Item), cudaMemcpyHostToDevice, in.stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(in.d_inst, &in.h, sizeof(Inst), cudaMemcpyHostToDevice, in.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(in.stream);
  if (e != cudaSuccess) {
    c.set_error("shard set-up failed: %s", cudaGetErrorString(e));
    ot_state_destroy(st);
    return OT_ECUDA;
  }
  *out = st;
  return OT_OK;
}

ot_status ot_shard_slice(ot_state* st, int32_t side, int64_t* p0, int64_t* p1) {
  if (!st || side < 0 || side > 1 || st->in.shard_world < 1) return OT_EINVAL;
  if (p0) *p0 = st->in.h.slice[side][0];
  if (p1) *p1 = st->in.h.slice[side][1];
  return OT_OK;
}

ot_status ot_shard_half_sweep(ot_state* st, int32_t side, int32_t cert) {
  if (!st || side < 0 || side > 1 || st->in.shard_world < 1) return OT_EINVAL;
  Context& ctx = st->ctx->c;
  Instance& in = st->in;
  cudaSetDevice(ctx.device);
  const int q = cert ? 1 : 0;
  const LaunchPlan& pl = cert ? in.cert : in.fast;
  SweepFn fn = get_sweep(in.d, pl.mode, pl.R, pl.ch, cert ? 1 : 0);
  const int nitems = in.shard_nitems[q][side];
  OT_CUDA(launch_sweep(fn, in.d_inst, in.shard_items[q][side], nitems, 1, std::min(nitems, pl.resident), in.sched,
                       in.stream));
  ctx.launches += 1;
  if (side == 1) {
    in.k += 1;
    if (cert) in.last_cert_k = in.k;
  }
  return read_ctrl(ctx, in);
}

// A pack slice travels as its tiles (kNComp x kTQ floats each) followed by the eight pack offsets,
// which every rank takes from rank 0 (they come from the first point, which rank 0 owns).
ot_status ot_shard_pack_bytes(ot_state* st, int32_t side, int32_t rank, size_t* bytes) {
  if (!st || !bytes || side < 0 || side > 1 || st->in.shard_world < 1 || rank < 0 || rank >= st->in.shard_world)
    return OT_EINVAL;
  int64_t p0, p1;
  shard_range(side == 0 ? st->in.n : st->in.m, rank, st->in.shard_world, &p0, &p1);
  const int64_t tiles = (p1 + kTQ - 1) / kTQ - p0 / kTQ;
  *bytes = (size_t)tiles * kNComp * kTQ * sizeof(float) + 8 * sizeof(double);
  return OT_OK;
}

static ot_status shard_pack_copy(ot_state* st, int32_t side, int32_t rank, void* host, bool to_host) {
  Context& ctx = st->ctx->c;
  Instance& in = st->in;
  cudaSetDevice(ctx.device);
  int64_t p0, p1;
  shard_range(side == 0 ? in.n : in.m, rank, in.shard_world, &p0, &p1);
  const int64_t t0 = p0 / kTQ, t1 = (p1 + kTQ - 1) / kTQ;
  const size_t tile_bytes = (size_t)kNComp * kTQ * sizeof(float);
  float* pack = side == 0 ? in.h.xpack : in.h.ypack;
  char* dev = (char*)(pack + (size_t)t0 * kNComp * kTQ);
  char* h = (char*)host;
  const size_t nb = (size_t)(t1 - t0) * tile_bytes;
  double* goff = in.ctrl + 24;
  if (to_host) {
    OT_CUDA(cudaMemcpyAsync(h, dev, nb, cudaMemcpyDeviceToHost, in.stream));
    OT_CUDA(cudaMemcpyAsync(h + nb, goff, 8 * sizeof(double), cudaMemcpyDeviceToHost, in.stream));
  } else {
    OT_CUDA(cudaMemcpyAsync(dev, h, nb, cudaMemcpyHostToDevice, in.stream));
    if (rank == 0) OT_CUDA(cudaMemcpyAsync(goff, h + nb, 8 * sizeof(double), cudaMemcpyHostToDevice, in.stream));
  }
  OT_CUDA(cudaStreamSynchronize(in.stream));
  return OT_OK;
}

ot_status ot_shard_pack_get(ot_state* st, int32_t side, void* host_buf) {
  if (!st || !host_buf || side < 0 || side > 1 || st->in.shard_world < 1) return OT_EINVAL;
  return shard_pack_copy(st, side, st->in.shard_rank, host_buf, true);
}

ot_status ot_shard_pack_put(ot_state* st, int32_t side, int32_t rank, const void* host_buf) {
  if (!st || !host_buf || side < 0 || side > 1 || st->in.shard_world < 1 || rank < 0 ||
      rank >= st->in.shard_world || rank == st->in.shard_rank)
    return OT_EINVAL;
  return shard_pack_copy(st, side, rank, const_cast<void*>(host_buf), false);
}

ot_status ot_shard_cert_partials(ot_state* st, double* out) {
  if (!st || !out || st->in.shard_world < 1) return OT_EINVAL;
  if (st->in.last_cert_k != st->in.k) {
    st->ctx->c.set_error("the last column half-sweep was not a certificate sweep");
    return OT_EINVAL;
  }
  const double* c = st->in.h_ctrl;  // read back by the half-sweep
  out[0] = c[kCertRF];
  out[1] = c[kCertCG];
  out[2] = c[kCertCostZ];
  out[3] = c[kCertDelta];
  out[4] = c[kCertEps];
  return OT_OK;
}

}  // extern "C"
