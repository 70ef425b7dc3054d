// Pipe-throughput microbenchmarks used to derive the roofline of the sweep (it is bound by the
// SFU (MUFU.EX2) and FP32 pipes and by instruction issue, not by HBM or tensor cores).
// Each probe runs one CTA of 512 threads per SM; every thread runs kChains independent dependency
// chains so that latency is hidden, and thread 0 of each CTA times the loop with clock64().
#include <cstdint>
#include <cstdio>
#include <vector>

#include "../../include/ot.h"
#include "ot_device.cuh"

namespace ot {

constexpr int kProbeThreads = 512;
constexpr int kChains = 8;

struct ProbeOut {
  unsigned long long cycles;
  float sink;
  float pad;
};

template <int KIND>
__global__ void __launch_bounds__(kProbeThreads) pipe_probe(int iters, ProbeOut* out, float seed) {
  float x[kChains];
  u64 xp[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) {
    x[c] = seed * (0.01f * (threadIdx.x + c)) * 1e-3f;
    xp[c] = pk2(x[c], x[c] + 0.5f);
  }
  const float a = 0.999f, b = 1e-4f;
  const u64 a2 = pk2(a, a), b2 = pk2(b, b);
  __syncthreads();
  const unsigned long long t0 = clock64();
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
      if constexpr (KIND == 0) x[c] = ex2_mufu(-x[c]);                       // MUFU.EX2
      if constexpr (KIND == 1) x[c] = fmaf(x[c], a, b);                     // FFMA
      if constexpr (KIND == 2) xp[c] = fma2(xp[c], a2, b2);                 // FFMA2 (2 lane ops)
      if constexpr (KIND == 3) x[c] = max3f(-x[c], -1.0f, -2.0f);            // FMNMX3
      if constexpr (KIND == 4) {                                            // 1 ex2 : 2 FFMA2 : 1 FADD2
        xp[c] = fma2(xp[c], a2, b2);
        xp[c] = fma2(xp[c], a2, b2);
        float lo, hi;
        up2(xp[c], lo, hi);
        x[c] = ex2_mufu(-lo) + x[c];
      }
      if constexpr (KIND == 5) x[c] = x[c] + b;                             // FADD
    }
  }
  __syncthreads();
  const unsigned long long t1 = clock64();
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) {
    float lo, hi;
    up2(xp[c], lo, hi);
    s += x[c] + lo + hi;
  }
  if (s == 12345.678f) out[blockIdx.x].pad = s;  // keep the chains alive
  if (threadIdx.x == 0) {
    out[blockIdx.x].cycles = t1 - t0;
    out[blockIdx.x].sink = s;
  }
}

}  // namespace ot

using namespace ot;

extern "C" ot_status ot_probe_pipes(int device, int iters, double* out, int nout) {
  // out[6*k + 0..]: per probe k: lane-ops per clock per SM, SM MHz during the probe
  if (!out || nout < 12 || iters < 1) return OT_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return OT_ECUDA;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return OT_ECUDA;
  const int sms = prop.multiProcessorCount;
  ProbeOut* d_out = nullptr;
  if (cudaMalloc(&d_out, sms * sizeof(ProbeOut)) != cudaSuccess) return OT_ENOMEM;
  typedef void (*Fn)(int, ProbeOut*, float);
  Fn fns[6] = {pipe_probe<0>, pipe_probe<1>, pipe_probe<2>, pipe_probe<3>, pipe_probe<4>, pipe_probe<5>};
  // lane operations per thread per (iteration, chain) for each probe
  const double ops[6] = {1.0, 1.0, 2.0, 1.0, 1.0 /* counted as ex2 per chain */, 1.0};
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  std::vector<ProbeOut> h(sms);
  ot_status st = OT_OK;
  const int nprobe = nout / 2 < 6 ? nout / 2 : 6;
  for (int k = 0; k < nprobe; ++k) {
    fns[k]<<<sms, kProbeThreads>>>(iters / 8 + 1, d_out, 1.0f);  // warm-up
    cudaEventRecord(e0);
    fns[k]<<<sms, kProbeThreads>>>(iters, d_out, 1.0f);
    cudaEventRecord(e1);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      st = OT_ECUDA;
      break;
    }
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaMemcpy(h.data(), d_out, sms * sizeof(ProbeOut), cudaMemcpyDeviceToHost);
    double cyc = 0;
    for (int i = 0; i < sms; ++i) cyc += (double)h[i].cycles;
    cyc /= sms;
    const double lane_ops = (double)kProbeThreads * iters * kChains * ops[k];
    out[2 * k + 0] = lane_ops / cyc;            // per SM per clock
    out[2 * k + 1] = cyc / (ms * 1e-3) / 1e6;   // MHz
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(d_out);
  return st;
}

namespace ot {
// exp2 of each input by the method the fast sweeps use: MUFU ex2.approx.ftz (method 0) or the
// FMA-pipe polynomial (method 1), two lanes at a time as in the sweep.
__global__ void exp2_probe_kernel(const float* __restrict__ x, float* __restrict__ y, int64_t n, int method) {
  const int64_t i = 2 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
  if (i >= n) return;
  const float a = x[i], b = i + 1 < n ? x[i + 1] : 0.0f;
  float ra, rb;
  if (method == 0) {
    ra = ex2_mufu(a);
    rb = ex2_mufu(b);
  } else {
    up2(exp2_poly2(pk2(a, b)), ra, rb);
  }
  y[i] = ra;
  if (i + 1 < n) y[i + 1] = rb;
}
}  // namespace ot

extern "C" ot_status ot_probe_exp2(int device, int method, const float* x, float* out, int64_t n) {
  using namespace ot;
  if (!x || !out || n < 1 || (method != 0 && method != 1)) return OT_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return OT_ECUDA;
  float *dx = nullptr, *dy = nullptr;
  if (cudaMalloc(&dx, n * sizeof(float)) != cudaSuccess) return OT_ENOMEM;
  if (cudaMalloc(&dy, n * sizeof(float)) != cudaSuccess) {
    cudaFree(dx);
    return OT_ENOMEM;
  }
  ot_status st = OT_OK;
  const int64_t pairs = (n + 1) / 2;
  if (cudaMemcpy(dx, x, n * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) st = OT_ECUDA;
  if (st == OT_OK) {
    exp2_probe_kernel<<<(unsigned)((pairs + 255) / 256), 256>>>(dx, dy, n, method);
    if (cudaGetLastError() != cudaSuccess || cudaMemcpy(out, dy, n * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
      st = OT_ECUDA;
  }
  cudaFree(dx);
  cudaFree(dy);
  return st;
}
