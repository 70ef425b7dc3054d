// An allocation-free variant of the row sweep, for callers that must not allocate device memory
// (for example code running inside a memory-capped plugin or a runtime that owns every device
// allocation and forbids cudaMalloc from libraries).  Everything the sweep needs beyond the
// caller's inputs and output lives in one fixed-size scratch array in this file's device memory.
#include <cmath>
#include <cstdint>
#include <mutex>

#include "../../include/ot.h"
#include "ot_kernels.cuh"
#include "ot_runtime.h"

namespace ot {

cudaError_t launch_pack_coords(const float* pts, int npts, int d, int tiles, double kappa, float* pack,
                               double* n2, cudaStream_t s, const float* origin);
cudaError_t launch_repack_cols(const Inst* I, int m, cudaStream_t s);
size_t sweep_smem_bytes();

namespace {

constexpr int64_t kMaxPts = OT_NOALLOC_MAX_POINTS;
constexpr int kMaxTiles = (int)((kMaxPts + kTQ - 1) / kTQ);
constexpr int kMaxBlocks = (int)((kMaxPts + kThreads - 1) / kThreads);  // R = 1 point blocks
constexpr int kMaxSplits = 8;

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Scratch layout (byte offsets); everything except the caller's arrays.
constexpr size_t kOffXPack = 0;
constexpr size_t kOffYPack = kOffXPack + align256((size_t)kMaxTiles * kNComp * kTQ * sizeof(float));
constexpr size_t kOffXN2 = kOffYPack + align256((size_t)kMaxTiles * kNComp * kTQ * sizeof(float));
constexpr size_t kOffYN2 = kOffXN2 + align256(kMaxPts * sizeof(double));
constexpr size_t kOffAlpha = kOffYN2 + align256(kMaxPts * sizeof(double));
constexpr size_t kOffTilde = kOffAlpha + align256(kMaxPts * sizeof(double));
constexpr size_t kOffPart = kOffTilde + align256(kMaxPts * sizeof(double));
constexpr size_t kOffCnt = kOffPart + align256((size_t)kMaxSplits * kMaxPts * sizeof(float4));
constexpr size_t kOffCtrl = kOffCnt + align256((kMaxBlocks + 6) * sizeof(unsigned));
constexpr size_t kOffInst = kOffCtrl + align256(24 * sizeof(double));
constexpr size_t kOffItems = kOffInst + align256(sizeof(Inst));
constexpr size_t kScratchBytes = kOffItems + align256((size_t)kMaxBlocks * kMaxSplits * sizeof(Item));

}  // namespace

// The scratch array.  Host code must not use its name as a device address (in host code it names a
// host-side stand-in): the address comes from cudaGetSymbolAddress in device_setup below, with the
// device current.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Writes the instance descriptor (passed by value) and the work items into the scratch.
__global__ void noalloc_setup_kernel(Inst inst, Inst* dst, Item* items, int pblks, int splits) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) *dst = inst;
  if (i < pblks * splits) items[i] = Item{0, 0, i % pblks, i / pblks, 1};
}

// Per-device set-up: the scratch address (looked up with the device current) and the launch
// shape of the sweep kernel.  The address is looked up again on every call made outside stream
// capture, so a context that was torn down and created again (whose module, and hence the array,
// may have moved) never sees a stale address; the SM count and occupancy are fixed per device.
struct DeviceSetup {
  void* base = nullptr;
  int resident[4] = {0, 0, 0, 0};  // per d: CTAs of the sweep kernel resident on the device (0: not yet)
};
static std::mutex g_mu;
static DeviceSetup g_dev[256];

static cudaError_t device_setup(int dev, int d, cudaStream_t s, SweepFn fn, void** base, int* resident) {
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(s, &cap);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_mu);
  DeviceSetup& D = g_dev[dev];
  if (cap == cudaStreamCaptureStatusNone || D.base == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    if (p == nullptr) return cudaErrorInvalidSymbol;
    D.base = p;
  }
  if (D.resident[d] == 0) {
    int sms = 0, per_sm = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)fn, kThreads, sweep_smem_bytes());
    if (e != cudaSuccess) return e;
    D.resident[d] = (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
  }
  *base = D.base;
  *resident = D.resident[d];
  return cudaSuccess;
}

}  // namespace ot

using namespace ot;

extern "C" ot_status ot_row_update_noalloc(int64_t n, int64_t m, int32_t d, const float* x, const float* y,
                                           const double* log_r, const double* log_bt, double kappa, double eps,
                                           double* log_alpha_hat, uint64_t stream) {
  if (n < 1 || m < 1 || n > kMaxPts || m > kMaxPts) return OT_EINVAL;  // beyond the scratch capacity
  if (d < 1 || d > 3 || !x || !y || !log_r || !log_bt || !log_alpha_hat) return OT_EINVAL;
  if (!(kappa > 0.0) || !(eps > 0.0) || !std::isfinite(kappa) || !std::isfinite(eps)) return OT_EINVAL;
  // Every CUDA call below is checked where it is made, and kernels are launched with
  // cudaLaunchKernel, which returns the launch's own status: an error that the caller left
  // pending is neither reported here nor cleared.
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return OT_ECUDA;
  cudaStream_t s = (cudaStream_t)(uintptr_t)stream;
  SweepFn fn = get_sweep(d, kSweepFast, 1, 16, 0);
  if (fn == nullptr) return OT_EINVAL;
  char* base = nullptr;
  int resident = 0;
  {
    void* b = nullptr;
    if (device_setup(dev, d, s, fn, &b, &resident) != cudaSuccess) return OT_ECUDA;
    base = (char*)b;
  }
  const int tiles_x = (int)((n + kTQ - 1) / kTQ), tiles_y = (int)((m + kTQ - 1) / kTQ);
  const int pblks = (int)((n + kThreads - 1) / kThreads);  // R = 1
  int splits = (4 * resident + pblks - 1) / pblks;
  splits = splits < 1 ? 1 : (splits > kMaxSplits ? kMaxSplits : splits);
  if (splits > tiles_y) splits = tiles_y;
  int tps = (tiles_y + splits - 1) / splits;
  if (splits > 1 && (tps & 1)) ++tps;  // runs of an even number of tiles, as the instance plans use
  splits = (tiles_y + tps - 1) / tps;

  Inst h{};
  h.n = (int)n;
  h.m = (int)m;
  h.d = d;
  h.tiles_x = tiles_x;
  h.tiles_y = tiles_y;
  h.pblk_x = pblks;
  h.slice[0][0] = 0;  // every row is updated (the column side is not swept)
  h.slice[0][1] = (int)n;
  h.slice[1][0] = 0;
  h.slice[1][1] = (int)m;
  h.nms[0][0] = splits;  // fast row sweep: one micro-split per split
  h.ms_tiles[0][0] = tps;
  h.wait_limit = kWaitLimit;
  h.hint[0] = h.hint[1] = nullptr;  // a single sweep at k = 0: no shift hints
  h.hint_bad = nullptr;
  h.kappa = kappa;
  h.eta = eps;       // k = 0 and lambda = 1 give the sweep temperature eta / (lambda k + 1) = eps
  h.lambda = 1.0;
  h.omega = 1.0;
  h.xpack = (float*)(base + kOffXPack);
  h.ypack = (float*)(base + kOffYPack);
  h.log_a = log_r;
  h.log_b = nullptr;
  h.xn2 = (const double*)(base + kOffXN2);
  h.yn2 = (const double*)(base + kOffYN2);
  h.log_alpha = (double*)(base + kOffAlpha);
  h.log_alpha_hat = log_alpha_hat;
  h.log_beta = const_cast<double*>(log_bt);        // read only: beta^{k-1} = beta^{k-2} = beta-tilde
  h.log_beta_prev = const_cast<double*>(log_bt);
  h.log_beta_tilde_next = (double*)(base + kOffTilde);
  h.part = base + kOffPart;
  h.cnt = (unsigned*)(base + kOffCnt);
  h.done = h.cnt + kMaxBlocks;
  double* ctrl = (double*)(base + kOffCtrl);
  h.cert = ctrl;
  h.k = (long long*)(ctrl + 8);
  h.err = (int*)(ctrl + 9);
  h.rows = (long long*)(ctrl + 16);  // k = k0 = 0: the row items wait for nothing
  h.k0 = (long long*)(ctrl + 17);
  Inst* d_inst = (Inst*)(base + kOffInst);
  Item* d_items = (Item*)(base + kOffItems);

  // every call shares the scratch: clear the counters, k, the error bits and the relaxation input
  if (cudaMemsetAsync(h.cnt, 0, (kMaxBlocks + 6) * sizeof(unsigned), s) != cudaSuccess ||
      cudaMemsetAsync(ctrl, 0, 24 * sizeof(double), s) != cudaSuccess ||
      cudaMemsetAsync(h.log_alpha, 0, n * sizeof(double), s) != cudaSuccess)
    return OT_ECUDA;
  int nitems = pblks * splits;
  {
    int pb = pblks, sp = splits;
    void* args[] = {(void*)&h, (void*)&d_inst, (void*)&d_items, (void*)&pb, (void*)&sp};
    if (cudaLaunchKernel((const void*)noalloc_setup_kernel, dim3((nitems + 255) / 256), dim3(256), args, 0, s) !=
        cudaSuccess)
      return OT_ECUDA;
  }
  if (launch_pack_coords(x, (int)n, d, tiles_x, kappa, h.xpack, (double*)h.xn2, s, nullptr) != cudaSuccess ||
      launch_pack_coords(y, (int)m, d, tiles_y, kappa, h.ypack, (double*)h.yn2, s, nullptr) != cudaSuccess ||
      launch_repack_cols(d_inst, (int)m, s) != cudaSuccess)
    return OT_ECUDA;
  const int grid = nitems < resident ? nitems : resident;
  unsigned* sched = h.cnt + kMaxBlocks + 2;  // scheduler counters (3)
  if (launch_sweep(fn, d_inst, d_items, nitems, 1, grid, sched, s) != cudaSuccess) return OT_ECUDA;
  int err = 0;
  if (cudaMemcpyAsync(&err, h.err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return OT_ECUDA;
  if (err & kErrTimeout) return OT_ETIMEDOUT;
  if (err & kErrNonFinite) return OT_ENUMERIC;
  return OT_OK;
}
