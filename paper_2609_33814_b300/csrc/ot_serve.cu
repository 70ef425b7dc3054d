// Continuous-batching server for OT solves on one GPU.
//
// Requests are queued on submission (their arrays copied).  A scheduler thread admits queued
// requests, in arrival order, into free slots while the HBM budget allows, and runs the active
// solves in lanes (same d, precision and certificate period): every chunk of cert_every
// iterations is issued as batched launches whose work items cover all active instances of the
// lane (uneven sizes), the last iteration of the chunk being a certificate iteration for all of
// them.  Admission and retirement happen at chunk boundaries, so certificate iterations stay
// aligned across the lane.  After each chunk every instance's certificate is read back and its
// own stop rule (relative or absolute certified gap, max_iters, time budget, cancellation) decides
// whether it retires; retired slots are freed and refilled at the next boundary.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/ot.h"
#include "ot_kernels.cuh"
#include "ot_runtime.h"

namespace ot {

static double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

enum ReqState { kPending = 0, kActive, kDone, kCancelled, kFailed };

struct Request {
  uint64_t id = 0;
  ot_problem prob{};
  ot_params params{};
  std::vector<float> hx, hy;
  std::vector<double> ha, hb;
  int state = kPending;
  bool cancel = false;
  ot_status status = OT_OK;
  ot_result res{};
  std::vector<double> f, g;
  double t_submit = 0, t_admit = 0, t_done = 0;
  Instance* inst = nullptr;
  size_t bytes = 0;
  int lane = -1;
  int ctrl_slot = -1;
  void* dstage = nullptr;  // device copy of device-resident inputs until the instance is set up
  std::string error;
};

struct Lane {
  int d = 2, mode = kSweepFast, cert_mode = kSweepComp, ce = 100;
  int R_fast = 2, ch_fast = 16, R_cert = 2;
  std::vector<Request*> active;
  bool dirty = true;
  Inst* d_table = nullptr;
  Inst* h_table = nullptr;
  size_t table_cap = 0;
  Item* d_items = nullptr;
  Item* h_items = nullptr;
  size_t items_cap = 0;
  int off[2] = {0, 0}, cnt[2] = {0, 0}, resident[2] = {0, 0};  // items per iteration of each kind
  unsigned* d_sched = nullptr;         // scheduler counters of the lane's launches
  double entries_per_sweep = 0;        // sum of n * m over the active instances
  std::vector<cudaEvent_t> evs;        // profiling: before, between and after the chunk's launches
  bool timed = false;                  // the last chunk recorded events
};

struct Server {
  Context ctx;
  bool own_stream = false;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> pending;
  std::unordered_map<uint64_t, Request*> reqs;
  static const int kMaxLanes = 16;
  Lane lanes[kMaxLanes];
  int nlanes = 0;  // lanes are created under mu and never removed
  std::thread th;
  bool stop = false;
  size_t budget = 0, used = 0;
  int max_slots = 0, active = 0;
  uint64_t next_id = 1;
  double* h_ctrl_pool = nullptr;
  std::vector<int> free_ctrl;
  // statistics since the last reset
  std::vector<double> latencies;
  int64_t submitted = 0, completed = 0, cancelled = 0, failed = 0, chunks = 0;
  double entries = 0, t_stats = 0;
  std::string fatal;
  // profiling: per fast launch (entries, milliseconds, instances in the lane), in launch order
  std::vector<double> launch_log;
  bool profile = false;

  void loop();
  int lane_for(const Request* r);  // called with mu held
  bool admit(Request* r);
  void run_chunk(Lane& L);
  void retire(Lane& L, std::vector<Request*>& done_now);
  void finish(Request* r, ot_status st);
};

static const int kMaxLaunch = 2;  // fast iterations, certificate iteration

// A lane runs instances of one (d, mode, cert_every) and one tile plan (the plans are taken from the
// prepared instance, so a plan table changed between submissions opens a new lane).
int Server::lane_for(const Request* r) {
  const int mode = sweep_mode_of(r->params.precision);
  const LaunchPlan& pf = r->inst->fast;
  const LaunchPlan& pc = r->inst->cert;
  const int cert_mode = mode == kSweepF64 ? kSweepF64 : kSweepComp;
  for (int i = 0; i < nlanes; ++i) {
    const Lane& L = lanes[i];
    if (L.d == r->prob.d && L.mode == mode && L.ce == r->params.cert_every && L.R_fast == pf.R &&
        L.ch_fast == pf.ch && L.R_cert == pc.R)
      return i;
  }
  if (nlanes == kMaxLanes) return -1;
  Lane& L = lanes[nlanes];
  L.d = r->prob.d;
  L.mode = mode;
  L.cert_mode = cert_mode;
  L.ce = r->params.cert_every;
  L.R_fast = pf.R;
  L.ch_fast = pf.ch;
  L.R_cert = pc.R;
  return nlanes++;
}

// Allocate and initialise the request's instance on the server stream (called with mu unlocked).
bool Server::admit(Request* r) {
  Instance* in = r->inst;
  ot_status st = instance_setup(ctx, *in, &r->prob);
  if (r->dstage) {
    cudaFreeAsync(r->dstage, ctx.stream);
    r->dstage = nullptr;
  }
  if (st != OT_OK) {
    r->error = ctx.last_error;
    finish(r, st);
    return false;
  }
  r->hx.clear();
  r->hx.shrink_to_fit();
  r->hy.clear();
  r->hy.shrink_to_fit();
  return true;
}

void Server::finish(Request* r, ot_status st) {
  // caller holds no lock; takes it to publish the outcome
  if (r->inst) {
    instance_free(*r->inst);  // the pinned read-back slot belongs to the server pool
    delete r->inst;
    r->inst = nullptr;
  }
  std::lock_guard<std::mutex> lk(mu);
  if (r->ctrl_slot >= 0) {
    free_ctrl.push_back(r->ctrl_slot);
    r->ctrl_slot = -1;
  }
  if (r->state == kActive) {
    active -= 1;
    used -= r->bytes;
  }
  r->t_done = now_s();
  r->status = st;
  r->res.latency_s = r->t_done - r->t_submit;
  r->res.queue_s = (r->t_admit > 0 ? r->t_admit : r->t_done) - r->t_submit;
  if (st == OT_OK) {
    r->state = kDone;
    completed += 1;
    latencies.push_back(r->t_done - r->t_submit);
    entries += 2.0 * (double)r->prob.n * (double)r->prob.m * (double)r->res.iters;
  } else if (st == OT_ECANCELLED) {
    r->state = kCancelled;
    cancelled += 1;
  } else {
    r->state = kFailed;
    failed += 1;
  }
  cv_done.notify_all();
}

void Server::run_chunk(Lane& L) {
  cudaStream_t s = ctx.stream;
  const size_t na = L.active.size();
  if (L.dirty) {
    // instance table and work items of the four launch kinds for the current composition
    if (!L.d_sched) {
      cudaMalloc(&L.d_sched, 4 * sizeof(unsigned));
      cudaMemsetAsync(L.d_sched, 0, 4 * sizeof(unsigned), s);
    }
    if (L.table_cap < na) {
      if (L.d_table) cudaFree(L.d_table);
      if (L.h_table) cudaFreeHost(L.h_table);
      L.table_cap = std::max<size_t>(na, 2 * L.table_cap);
      cudaMalloc(&L.d_table, L.table_cap * sizeof(Inst));
      cudaMallocHost(&L.h_table, L.table_cap * sizeof(Inst));
    }
    for (size_t i = 0; i < na; ++i) L.h_table[i] = L.active[i]->inst->h;
    std::vector<Item> items;
    for (int kind = 0; kind < kMaxLaunch; ++kind) {
      const bool cert = kind == 1;
      SweepFn fn = get_sweep(L.d, cert ? L.cert_mode : L.mode, cert ? L.R_cert : L.R_fast, cert ? 8 : L.ch_fast,
                             cert ? 1 : 0);
      const int resident = ctx.resident_ctas(fn);
      L.resident[kind] = resident;
      L.off[kind] = (int)items.size();
      for (int side = 0; side < 2; ++side) {
        const bool row = side == 0;
        // Each instance's micro-split layout is fixed (its numerics do not depend on the batch);
        // the launch groups micro-splits into items of about equal size for this composition:
        // roughly four waves of resident CTAs per sweep.
        double tiles_total = 0;
        for (size_t i = 0; i < na; ++i) {
          const Instance& in = *L.active[i]->inst;
          const LaunchPlan& pl = cert ? in.cert : in.fast;
          const int64_t nq = row ? in.m : in.n;
          tiles_total += (double)(row ? pl.pblk_row : pl.pblk_col) * (double)((nq + kTQ - 1) / kTQ);
        }
        const double target = std::max(1.0, tiles_total / (4.0 * resident));
        const size_t first = items.size();
        for (size_t i = 0; i < na; ++i) {
          const Instance& in = *L.active[i]->inst;
          const LaunchPlan& pl = cert ? in.cert : in.fast;
          const int nms = row ? pl.nms_row : pl.nms_col;
          const int mst = row ? pl.mst_row : pl.mst_col;
          const int group = std::max(1, std::min(nms, (int)std::lround(target / mst)));
          build_items(items, (int)i, side, row ? pl.pblk_row : pl.pblk_col, nms, group);
        }
        // longest items first within the sweep (the kernel hands them out in order)
        auto work_of = [&](const Item& it) {
          const Instance& in = *L.active[it.inst]->inst;
          const LaunchPlan& pl = cert ? in.cert : in.fast;
          const int64_t nq = row ? in.m : in.n;
          const int qtiles = (int)((nq + kTQ - 1) / kTQ);
          const int mst = row ? pl.mst_row : pl.mst_col;
          return std::min(qtiles, (it.ms0 + it.nms) * mst) - it.ms0 * mst;
        };
        std::stable_sort(items.begin() + first, items.end(),
                         [&](const Item& a, const Item& b) { return work_of(a) > work_of(b); });
      }
      L.cnt[kind] = (int)items.size() - L.off[kind];
    }
    if (L.items_cap < items.size()) {
      if (L.d_items) cudaFree(L.d_items);
      if (L.h_items) cudaFreeHost(L.h_items);
      L.items_cap = std::max(items.size(), 2 * L.items_cap);
      cudaMalloc(&L.d_items, L.items_cap * sizeof(Item));
      cudaMallocHost(&L.h_items, L.items_cap * sizeof(Item));
    }
    memcpy(L.h_items, items.data(), items.size() * sizeof(Item));
    L.entries_per_sweep = 0;
    for (size_t i = 0; i < na; ++i) L.entries_per_sweep += (double)L.active[i]->inst->n * (double)L.active[i]->inst->m;
    cudaMemcpyAsync(L.d_table, L.h_table, na * sizeof(Inst), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(L.d_items, L.h_items, items.size() * sizeof(Item), cudaMemcpyHostToDevice, s);
    L.dirty = false;
  }
  // the chunk: ce - 1 fast iterations as one launch, then the certificate iteration
  SweepFn fns[2] = {get_sweep(L.d, L.mode, L.R_fast, L.ch_fast, 0), get_sweep(L.d, L.cert_mode, L.R_cert, 8, 1)};
  const int iters[2] = {L.ce - 1, 1};
  L.timed = profile;
  if (profile && L.evs.size() != 3) {
    for (cudaEvent_t e : L.evs) cudaEventDestroy(e);
    L.evs.assign(3, nullptr);
    for (auto& e : L.evs) cudaEventCreate(&e);
  }
  if (profile) cudaEventRecord(L.evs[0], s);
  for (int kind = 0; kind < kMaxLaunch; ++kind) {
    if (iters[kind] > 0) {
      const int grid = std::min(L.cnt[kind], L.resident[kind]);  // one iteration's items bound the CTAs
      launch_sweep(fns[kind], L.d_table, L.d_items + L.off[kind], L.cnt[kind], iters[kind], grid, L.d_sched, s);
      ctx.launches += 1;
    }
    if (profile) cudaEventRecord(L.evs[kind + 1], s);
  }
  for (Request* r : L.active) {
    r->inst->k += L.ce;
    cudaMemcpyAsync(r->inst->h_ctrl, r->inst->ctrl, 16 * sizeof(double), cudaMemcpyDeviceToHost, s);
  }
  chunks += 1;
}

void Server::retire(Lane& L, std::vector<Request*>& done_now) {
  const double t = now_s();
  std::vector<Request*> keep;
  for (Request* r : L.active) {
    Instance& in = *r->inst;
    const int err = ((const int*)in.h_ctrl)[18];
    ot_status st = OT_OK;
    bool stop = false;
    if (err & kErrTimeout) {
      st = OT_ETIMEDOUT;
      stop = true;
    } else if (err & kErrNonFinite) {
      st = OT_ENUMERIC;
      stop = true;
    } else {
      absorb_cert(ctx, in);
      const double gap = in.U_best - in.L_best;
      const ot_params& q = r->params;
      if ((q.tol_abs > 0 && gap <= q.tol_abs) || (q.tol_rel > 0 && gap <= q.tol_rel * std::fabs(in.U_best))) {
        in.stop = OT_STOP_TOL;
        stop = true;
      } else if (in.k >= q.max_iters) {
        in.stop = OT_STOP_MAX_ITERS;
        stop = true;
      } else if (q.time_budget_s > 0 && t - r->t_admit >= q.time_budget_s) {
        in.stop = OT_STOP_TIME;
        stop = true;
      }
      if (r->cancel) {
        st = OT_ECANCELLED;
        stop = true;
      }
    }
    if (!stop) {
      keep.push_back(r);
      continue;
    }
    in.elapsed_s = t - r->t_admit;
    fill_result(in, &r->res);
    if (st == OT_OK && in.best_iter >= 0) {
      r->f.resize(in.n);
      r->g.resize(in.m);
      cudaMemcpyAsync(r->f.data(), in.f_best, in.n * sizeof(double), cudaMemcpyDeviceToHost, ctx.stream);
      cudaMemcpyAsync(r->g.data(), in.g_best, in.m * sizeof(double), cudaMemcpyDeviceToHost, ctx.stream);
    }
    r->status = st;
    done_now.push_back(r);
  }
  if (keep.size() != L.active.size()) {
    L.active.swap(keep);
    L.dirty = true;
  }
}

void Server::loop() {
  cudaSetDevice(ctx.device);
  while (true) {
    std::vector<Request*> to_admit;
    {
      std::unique_lock<std::mutex> lk(mu);
      bool any_active = false;
      for (int i = 0; i < nlanes; ++i) any_active |= !lanes[i].active.empty();
      while (!stop && pending.empty() && !any_active) cv_work.wait(lk);
      if (stop) break;
      // FIFO admission by free slots and HBM budget
      while (!pending.empty() && active < max_slots) {
        Request* r = pending.front();
        if (r->cancel) {
          pending.pop_front();
          r->state = kCancelled;
          r->status = OT_ECANCELLED;
          r->t_done = now_s();
          cancelled += 1;
          cv_done.notify_all();
          continue;
        }
        if (used + r->bytes > budget && active > 0) break;
        pending.pop_front();
        used += r->bytes;
        active += 1;
        r->state = kActive;
        r->t_admit = now_s();
        r->ctrl_slot = free_ctrl.back();
        free_ctrl.pop_back();
        r->inst->h_ctrl_external = h_ctrl_pool + 16 * r->ctrl_slot;
        to_admit.push_back(r);
      }
    }
    int nl;
    {
      std::lock_guard<std::mutex> lk(mu);
      nl = nlanes;
    }
    for (Request* r : to_admit) {
      if (admit(r)) {
        Lane& L = lanes[r->lane];
        // every instance of a lane has the same (d, precision) and hence the same tile plans
        L.R_fast = r->inst->fast.R;
        L.ch_fast = r->inst->fast.ch;
        L.R_cert = r->inst->cert.R;
        L.active.push_back(r);
        L.dirty = true;
      }
    }
    bool ran = false;
    for (int i = 0; i < nl; ++i) {
      Lane& L = lanes[i];
      if (L.active.empty()) continue;
      run_chunk(L);
      ran = true;
    }
    if (!ran) continue;
    if (cudaStreamSynchronize(ctx.stream) != cudaSuccess) {
      fatal = cudaGetErrorString(cudaGetLastError());
      std::vector<Request*> all;
      for (int i = 0; i < nl; ++i) {
        Lane& L = lanes[i];
        for (Request* r : L.active) all.push_back(r);
        L.active.clear();
        L.dirty = true;
      }
      for (Request* r : all) {
        r->error = fatal;
        finish(r, OT_ECUDA);
      }
      continue;
    }
    for (int i = 0; i < nl; ++i) {
      Lane& L = lanes[i];
      if (!L.timed || L.active.empty()) continue;
      L.timed = false;
      const int iters[2] = {L.ce - 1, 1};
      for (int kind = 0; kind < kMaxLaunch; ++kind) {
        if (iters[kind] <= 0) continue;
        float ms = 0;
        cudaEventElapsedTime(&ms, L.evs[kind], L.evs[kind + 1]);
        KernelStats& ks = ctx.stats[kind];
        ks.launches += 1;
        ks.entries += 2.0 * L.entries_per_sweep * iters[kind];  // row and column sweeps
        ks.ms += ms;
        if (kind == 0) {
          std::lock_guard<std::mutex> lk(mu);
          launch_log.push_back(2.0 * L.entries_per_sweep * iters[kind]);
          launch_log.push_back(ms);
          launch_log.push_back((double)L.active.size());
        }
      }
    }
    std::vector<Request*> done_now;
    for (int i = 0; i < nl; ++i) retire(lanes[i], done_now);
    if (!done_now.empty()) {
      cudaStreamSynchronize(ctx.stream);  // result copies
      for (Request* r : done_now) finish(r, r->status);
    }
  }
}

}  // namespace ot

using namespace ot;

struct ot_server {
  Server s;
};

extern "C" {

ot_status ot_serve_create(ot_context* ctx, size_t hbm_budget_bytes, int32_t max_slots, uint64_t stream,
                          ot_server** out) {
  if (!ctx || !out || max_slots < 1 || hbm_budget_bytes == 0) return OT_EINVAL;
  *out = nullptr;
  ot_server* sv = new (std::nothrow) ot_server();
  if (!sv) return OT_ENOMEM;
  Server& S = sv->s;
  (void)ctx;
  int device = 0;
  cudaGetDevice(&device);
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
    delete sv;
    return OT_ECUDA;
  }
  S.ctx.device = device;
  S.ctx.sms = prop.multiProcessorCount;
  S.ctx.cc_major = prop.major;
  S.ctx.cc_minor = prop.minor;
  if (stream) {
    S.ctx.stream = (cudaStream_t)(uintptr_t)stream;
  } else {
    cudaStreamCreateWithFlags(&S.ctx.stream, cudaStreamNonBlocking);
    S.own_stream = true;
  }
  S.budget = hbm_budget_bytes;
  S.max_slots = max_slots;
  if (cudaMallocHost(&S.h_ctrl_pool, (size_t)max_slots * 16 * sizeof(double)) != cudaSuccess) {
    delete sv;
    return OT_ENOMEM;
  }
  for (int i = max_slots - 1; i >= 0; --i) S.free_ctrl.push_back(i);
  S.t_stats = now_s();
  S.th = std::thread([&S] { S.loop(); });
  *out = sv;
  return OT_OK;
}

void ot_serve_destroy(ot_server* sv) {
  if (!sv) return;
  Server& S = sv->s;
  {
    std::lock_guard<std::mutex> lk(S.mu);
    S.stop = true;
  }
  S.cv_work.notify_all();
  if (S.th.joinable()) S.th.join();
  cudaSetDevice(S.ctx.device);
  cudaStreamSynchronize(S.ctx.stream);
  for (int i = 0; i < S.nlanes; ++i) {
    Lane& L = S.lanes[i];
    for (Request* r : L.active) {
      if (r->inst) {
        instance_free(*r->inst);
        delete r->inst;
        r->inst = nullptr;
      }
    }
    if (L.d_table) cudaFree(L.d_table);
    if (L.h_table) cudaFreeHost(L.h_table);
    if (L.d_sched) cudaFree(L.d_sched);
    if (L.d_items) cudaFree(L.d_items);
    if (L.h_items) cudaFreeHost(L.h_items);
    for (cudaEvent_t e : L.evs) cudaEventDestroy(e);
  }
  for (auto& kv : S.reqs) {
    if (kv.second->inst) {
      instance_free(*kv.second->inst);
      delete kv.second->inst;
    }
    if (kv.second->dstage) cudaFree(kv.second->dstage);
    delete kv.second;
  }
  cudaStreamSynchronize(S.ctx.stream);
  if (S.h_ctrl_pool) cudaFreeHost(S.h_ctrl_pool);
  if (S.own_stream) cudaStreamDestroy(S.ctx.stream);
  delete sv;
}

ot_status ot_serve_submit(ot_server* sv, const ot_problem* prob, const ot_params* params, uint64_t* req_id) {
  if (!sv || !prob || !params || !req_id) return OT_EINVAL;
  Server& S = sv->s;
  if (params->cert_every < 1 || params->algorithm != OT_ALG_BDRS) return OT_EINVAL;
  Request* r = new (std::nothrow) Request();
  if (!r) return OT_ENOMEM;
  r->params = *params;
  r->prob = *prob;
  const size_t n = prob->n > 0 ? (size_t)prob->n : 0, m = prob->m > 0 ? (size_t)prob->m : 0;
  const int d = prob->d;
  if (n == 0 || m == 0 || d < 1 || d > 3 || !prob->x || !prob->y || !prob->a || !prob->b) {
    delete r;
    return OT_EINVAL;
  }
  // copy the inputs: host arrays into host vectors, device arrays into a device staging buffer
  if (prob->on_device) {
    const size_t bx = n * d * sizeof(float), by = m * d * sizeof(float);
    const size_t ox = 0, oy = (bx + 255) & ~(size_t)255, oa = oy + ((by + 255) & ~(size_t)255),
                 ob = oa + ((n * sizeof(double) + 255) & ~(size_t)255), tot = ob + m * sizeof(double);
    cudaStream_t cs = cudaStreamPerThread;
    if (cudaMallocAsync(&r->dstage, tot, cs) != cudaSuccess) {
      cudaGetLastError();
      delete r;
      return OT_ENOMEM;
    }
    char* b = (char*)r->dstage;
    cudaMemcpyAsync(b + ox, prob->x, bx, cudaMemcpyDeviceToDevice, cs);
    cudaMemcpyAsync(b + oy, prob->y, by, cudaMemcpyDeviceToDevice, cs);
    cudaMemcpyAsync(b + oa, prob->a, n * sizeof(double), cudaMemcpyDeviceToDevice, cs);
    cudaMemcpyAsync(b + ob, prob->b, m * sizeof(double), cudaMemcpyDeviceToDevice, cs);
    if (cudaStreamSynchronize(cs) != cudaSuccess) {
      cudaFree(r->dstage);
      delete r;
      return OT_ECUDA;
    }
    r->prob.x = (const float*)(b + ox);
    r->prob.y = (const float*)(b + oy);
    r->prob.a = (const double*)(b + oa);
    r->prob.b = (const double*)(b + ob);
  } else {
    r->hx.assign(prob->x, prob->x + n * d);
    r->hy.assign(prob->y, prob->y + m * d);
    r->ha.assign(prob->a, prob->a + n);
    r->hb.assign(prob->b, prob->b + m);
    r->prob.x = r->hx.data();
    r->prob.y = r->hy.data();
    r->prob.a = r->ha.data();
    r->prob.b = r->hb.data();
  }
  std::lock_guard<std::mutex> lk(S.mu);
  // plan and size the instance now, so that admission can check the budget
  r->inst = new Instance();
  r->inst->async_alloc = true;
  r->inst->use_graphs = false;
  ot_status st = instance_prepare(S.ctx, *r->inst, &r->prob, &r->params, S.ctx.stream);
  if (st == OT_OK) {
    r->lane = S.lane_for(r);  // a lane of the instance's own tile plans
    if (r->lane < 0) st = OT_EINVAL;
  }
  r->bytes = r->inst->bytes;
  if (st == OT_OK && r->bytes > S.budget) st = OT_ENOMEM;
  if (st != OT_OK) {
    if (r->dstage) cudaFree(r->dstage);
    delete r->inst;
    delete r;
    return st;
  }
  r->id = S.next_id++;
  r->t_submit = now_s();
  S.reqs[r->id] = r;
  S.pending.push_back(r);
  S.submitted += 1;
  *req_id = r->id;
  S.cv_work.notify_all();
  return OT_OK;
}

static ot_status collect(Server& S, Request* r, double* f_out, double* g_out, ot_result* res) {
  // called with S.mu held, r finished
  const ot_status st = r->status;
  if (res) *res = r->res;
  if (st == OT_OK) {
    if (f_out && !r->f.empty()) memcpy(f_out, r->f.data(), r->f.size() * sizeof(double));
    if (g_out && !r->g.empty()) memcpy(g_out, r->g.data(), r->g.size() * sizeof(double));
  }
  S.reqs.erase(r->id);
  delete r;
  return st;
}

ot_status ot_serve_poll(ot_server* sv, uint64_t req_id, double* f_out, double* g_out, ot_result* res) {
  if (!sv) return OT_EINVAL;
  Server& S = sv->s;
  std::lock_guard<std::mutex> lk(S.mu);
  auto it = S.reqs.find(req_id);
  if (it == S.reqs.end()) return OT_ENOTFOUND;
  Request* r = it->second;
  if (r->state == kPending || r->state == kActive) return OT_EBUSY;
  return collect(S, r, f_out, g_out, res);
}

ot_status ot_serve_wait(ot_server* sv, uint64_t req_id, double timeout_s, double* f_out, double* g_out,
                        ot_result* res) {
  if (!sv) return OT_EINVAL;
  Server& S = sv->s;
  std::unique_lock<std::mutex> lk(S.mu);
  auto it = S.reqs.find(req_id);
  if (it == S.reqs.end()) return OT_ENOTFOUND;
  Request* r = it->second;
  auto pred = [r] { return r->state != kPending && r->state != kActive; };
  if (timeout_s < 0) {
    S.cv_done.wait(lk, pred);
  } else if (!S.cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), pred)) {
    return OT_EBUSY;
  }
  return collect(S, r, f_out, g_out, res);
}

ot_status ot_serve_cancel(ot_server* sv, uint64_t req_id) {
  if (!sv) return OT_EINVAL;
  Server& S = sv->s;
  std::lock_guard<std::mutex> lk(S.mu);
  auto it = S.reqs.find(req_id);
  if (it == S.reqs.end()) return OT_ENOTFOUND;
  it->second->cancel = true;
  S.cv_work.notify_all();
  return OT_OK;
}

ot_status ot_serve_stats(ot_server* sv, ot_serve_statistics* out) {
  if (!sv || !out) return OT_EINVAL;
  Server& S = sv->s;
  std::lock_guard<std::mutex> lk(S.mu);
  memset(out, 0, sizeof(*out));
  out->submitted = S.submitted;
  out->completed = S.completed;
  out->cancelled = S.cancelled;
  out->failed = S.failed;
  out->active = S.active;
  out->pending = (int64_t)S.pending.size();
  out->chunks = S.chunks;
  out->launches = S.ctx.launches;
  out->hbm_used_bytes = (double)S.used;
  const double el = now_s() - S.t_stats;
  out->elapsed_s = el;
  if (!S.latencies.empty()) {
    std::vector<double> v = S.latencies;
    std::sort(v.begin(), v.end());
    auto pct = [&v](double p) {
      const double x = p * (double)(v.size() - 1);
      const size_t i = (size_t)x;
      const double fr = x - (double)i;
      return i + 1 < v.size() ? v[i] * (1 - fr) + v[i + 1] * fr : v[i];
    };
    out->p50_latency_s = pct(0.50);
    out->p99_latency_s = pct(0.99);
    double sum = 0;
    for (double x : v) sum += x;
    out->mean_latency_s = sum / (double)v.size();
  }
  out->solves_per_s = el > 0 ? (double)S.completed / el : 0;
  out->entries_per_s = el > 0 ? S.entries / el : 0;
  out->entries = S.entries;
  return OT_OK;
}

ot_status ot_serve_profile_enable(ot_server* sv, int on) {
  if (!sv) return OT_EINVAL;
  std::lock_guard<std::mutex> lk(sv->s.mu);
  sv->s.profile = on != 0;
  return OT_OK;
}

ot_status ot_serve_profile_read(ot_server* sv, int kind, int64_t* launches, double* entries, double* ms) {
  if (!sv || kind < 0 || kind > 1) return OT_EINVAL;
  std::lock_guard<std::mutex> lk(sv->s.mu);
  const KernelStats& k = sv->s.ctx.stats[kind];
  if (launches) *launches = k.launches;
  if (entries) *entries = k.entries;
  if (ms) *ms = k.ms;
  return OT_OK;
}

ot_status ot_serve_profile_launches(ot_server* sv, double* out, int64_t max_launches, int64_t* count) {
  if (!sv || !count) return OT_EINVAL;
  Server& S = sv->s;
  std::lock_guard<std::mutex> lk(S.mu);
  const int64_t n = (int64_t)S.launch_log.size() / 3;
  *count = n;
  if (out)
    for (int64_t i = 0; i < std::min(n, max_launches) * 3; ++i) out[i] = S.launch_log[i];
  return OT_OK;
}

ot_status ot_serve_reset_stats(ot_server* sv) {
  if (!sv) return OT_EINVAL;
  Server& S = sv->s;
  std::lock_guard<std::mutex> lk(S.mu);
  S.latencies.clear();
  S.launch_log.clear();
  for (auto& k : S.ctx.stats) k = KernelStats();
  S.ctx.launches = 0;
  S.completed = S.cancelled = S.failed = S.chunks = 0;
  S.submitted = 0;
  S.entries = 0;
  S.t_stats = now_s();
  return OT_OK;
}

}  // extern "C"
