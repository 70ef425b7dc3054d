// Internal host-side types of the solver runtime (not part of the C ABI).
#pragma once
#include <cmath>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "../../include/ot.h"
#include "ot_kernels.cuh"

namespace ot {

typedef void (*SweepFn)(const Inst*, const Item*, int, int, unsigned*);
SweepFn get_sweep(int d, int mode, int R, int ch, int variant);

// Accumulated timing of one kind of sweep launch (profiling mode).
struct KernelStats {
  int64_t launches = 0;
  double entries = 0;  // algorithmic implicit entries (n * m per sweep)
  double ms = 0;       // summed CUDA-event durations on the launching stream
};

struct Context {
  int device = 0;
  bool profile = false;
  KernelStats stats[2];  // fast iterations, certificate iterations
  int64_t launches = 0;  // every kernel this context has launched (graph nodes included)
  uint32_t wait_limit = kWaitLimit;  // tile-wait bound given to the states created from now on
  int sms = 148;
  int cc_major = 0, cc_minor = 0;
  cudaStream_t stream = nullptr;
  std::string last_error;
  std::map<const void*, int> occ;  // resident CTAs per sweep kernel
  void set_error(const char* fmt, ...);
  int resident_ctas(SweepFn fn);
};

// Launch plan of one kind of sweep (fast iterations, or certificate iterations): points per
// thread, chunk width, split counts, work items and grid of both sweeps.
struct LaunchPlan {
  int mode = 0;
  int R = 1, ch = 16;
  int pblk_row = 0, pblk_col = 0;
  int nms_row = 1, nms_col = 1;      // micro-splits of the reduced side (fixed per instance)
  int mst_row = 1, mst_col = 1;      // tiles per micro-split
  int group_row = 1, group_col = 1;  // micro-splits per work item when the instance runs alone
  Item* d_row = nullptr;              // the instance's items: row sweep, then (d_col) column sweep
  Item* d_col = nullptr;
  int n_row = 0, n_col = 0;
  int resident = 0;                    // CTAs of the plan's kernel resident on the device
};

// Byte offsets of an instance's buffers inside its single device allocation.
struct Layout {
  size_t xpack, ypack, xraw, yraw, a, b, ain, bin, la, lb, xn2, yn2, state0, fg, hint, part, cnt, blk, ctrl, range,
      inst, items;
  size_t maxblk;
};

// One resident instance: descriptor, device buffers, launch plans and host-side bookkeeping.
struct Instance {
  Inst h{};                      // host mirror of the device descriptor
  Inst* d_inst = nullptr;        // device descriptor (inside mem)
  LaunchPlan fast, cert;
  void* mem = nullptr;
  size_t bytes = 0;
  float* xraw = nullptr;
  float* yraw = nullptr;
  double* f_best = nullptr;
  double* g_best = nullptr;
  double* ctrl = nullptr;        // device control block: cert record, k, error bits
  unsigned* sched = nullptr;     // work-item ticket counters of this instance's sweeps (inside mem)
  double* h_ctrl = nullptr;      // pinned host copy
  cudaStream_t stream = nullptr;
  ot_params params{};
  int64_t n = 0, m = 0;
  int d = 0;
  int sweep_mode = 0, cert_mode = 1;
  double refine_on = 0.0, refine_tol = 1e-5;  // refinement of the fast sweeps' dominant terms
  bool use_graphs = true;
  // used by the batched server: stream-ordered allocation and a shared pinned read-back slot
  bool async_alloc = false;
  double* h_ctrl_external = nullptr;
  Layout layout{};
  double kappa = 0, omega = 0;
  // iteration bookkeeping
  int64_t k = 0;
  int64_t last_cert_k = -1;
  int64_t n_certs = 0;
  int64_t best_iter = -1;
  double U = NAN, L = NAN, U_best = INFINITY, L_best = -INFINITY, best_rel = INFINITY, eps_last = NAN;
  double elapsed_s = 0, elapsed_base = 0;
  int stop = OT_STOP_NONE;
  int device_errors = 0;
  // Row-sharded execution (ot_shard_*): this process's rank of `shard_world`, and the work items of
  // its slice per plan (0 fast, 1 certificate) and side, written over the instance's item buffer.
  int shard_rank = -1, shard_world = 0;
  Item* shard_items[2][2] = {};
  int shard_nitems[2][2] = {};
  std::map<std::pair<int64_t, int>, cudaGraphExec_t> graphs;
  std::map<std::pair<int64_t, int>, std::vector<cudaEvent_t>> graph_events;  // profiling mode
};

ot_status validate(Context& ctx, const ot_problem* p, const ot_params* q);
void plan_launch(Context& ctx, const Instance& in, int mode, LaunchPlan& pl);
void canonical_tile(int d, int mode, int* R, int* ch);
int sweep_mode_of(int precision);
void build_items(std::vector<Item>& out, int inst, int side, int pblks, int nms, int group);
ot_status instance_init(Context& ctx, Instance& in, const ot_problem* p, const ot_params* q, cudaStream_t stream);
ot_status instance_prepare(Context& ctx, Instance& in, const ot_problem* p, const ot_params* q, cudaStream_t stream);
ot_status instance_setup(Context& ctx, Instance& in, const ot_problem* p);
ot_status read_ctrl(Context& ctx, Instance& in);
ot_status absorb_cert(Context& ctx, Instance& in);
void fill_result(const Instance& in, ot_result* r);
// One launch of `iters` iterations over the instance table (nitems work items per iteration);
// grid = CTAs (at most the resident count), sched = the stream's two-plus-one scheduler counters.
cudaError_t launch_sweep(SweepFn fn, const Inst* insts, const Item* items, int nitems, int iters, int grid,
                         unsigned* sched, cudaStream_t stream);
void instance_free(Instance& in);
ot_status run_iterations(Context& ctx, Instance& in, int64_t n_iters, bool stop_rule, bool final_cert);
ot_status standalone_certificate(Context& ctx, Instance& in);

}  // namespace ot
