// Set-up kernels, launch helpers and the sweep dispatch table of the solver.
#include <cfloat>
#include <climits>
#include <cmath>
#include <cstdint>

#include "ot_sweep.cuh"

namespace ot {

SweepFn get_sweep_d1(int mode, int R, int ch, int v);
SweepFn get_sweep_d2(int mode, int R, int ch, int v);
SweepFn get_sweep_d3(int mode, int R, int ch, int v);

// ---------------------------------------------------------------------------------------------
// Set-up kernels
// ---------------------------------------------------------------------------------------------

// Coordinates into the tile-blocked pack (padding: coords 0, h = kPadH), kappa ||.||^2 in FP64.
// origin (3 floats, or null) is subtracted from every coordinate first; the caller only passes one
// for which every subtraction is exact, so the cost kappa ||x - y||^2 is unchanged.
__global__ void pack_coords_kernel(const float* __restrict__ pts, int npts, int d, int tiles, double kappa,
                                   float* __restrict__ pack, double* __restrict__ n2, const float* origin) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= tiles * kTQ) return;
  double s = 0.0;
  for (int k = 0; k < d; ++k) {
    float v = p < npts ? pts[(size_t)p * d + k] : 0.0f;
    if (origin != nullptr && p < npts) v = __fsub_rn(v, origin[k]);
    pack[pack_idx(p, k)] = v;
    s += (double)v * (double)v;
  }
  for (int k = d; k < kNComp; ++k) pack[pack_idx(p, k)] = (k == d && p >= npts) ? kPadH : 0.0f;
  if (p < npts) n2[p] = kappa * s;
}

// Coordinate runs of a 2-D pack (read by the fast sweeps, kRunCols): for each tile, 1 + k in the
// first entry of its free component (kNComp - 1) when coordinate k takes one value over every
// aligned group of kRunCols points of the tile, else 0 (coordinate 1 preferred).  Padding points are
// left out: their h = kPadH makes each of their terms vanish whatever coordinate is used.  One
// block of kTQ threads per tile; runs after pack_coords_kernel (and its centring) on the same stream.
__global__ void tile_runs_kernel(float* __restrict__ pack, int npts) {
  const int t = blockIdx.x, c = threadIdx.x;
  const int p = t * kTQ + c;
  const int head = t * kTQ + (c & ~(kRunCols - 1));  // a valid point whenever p is
  bool same0 = true, same1 = true;
  if (p < npts) {
    same0 = pack[pack_idx(p, 0)] == pack[pack_idx(head, 0)];
    same1 = pack[pack_idx(p, 1)] == pack[pack_idx(head, 1)];
  }
  const int all0 = __syncthreads_and(same0 ? 1 : 0);
  const int all1 = __syncthreads_and(same1 ? 1 : 0);
  if (c == 0) pack[pack_idx(t * kTQ, kNComp - 1)] = all1 ? 2.0f : (all0 ? 1.0f : 0.0f);
}

// Exact centring of the two clouds (translation leaves the squared-Euclidean cost unchanged).  The
// FP32 exponent of the fast sweeps rounds at the scale of kappa ||w||^2 / eps and of <A_p, w_q>, so
// coordinates near the origin make it more accurate; the translation is only applied when it is
// exact for every coordinate (integer pixel grids always are), so the cost does not change at all.
// c[0..5]: per dimension the ordered-int encoded minimum and maximum over both clouds; c[6]: set
// when some coordinate's difference from the midpoint is not exact in FP32; origin[0..2]: the
// translation (zeros when none applies).
__device__ __forceinline__ int ordered_int(float f) {
  const int i = __float_as_int(f);
  return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float from_ordered_int(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }

__global__ void centre_range_kernel(const float* __restrict__ x, int n, const float* __restrict__ y, int m, int d,
                                    int* c) {
  int mn[3] = {INT_MAX, INT_MAX, INT_MAX}, mx[3] = {INT_MIN, INT_MIN, INT_MIN};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n + m; i += gridDim.x * blockDim.x) {
    const float* p = i < n ? x + (size_t)i * d : y + (size_t)(i - n) * d;
    for (int k = 0; k < d; ++k) {
      const int v = ordered_int(p[k]);
      mn[k] = min(mn[k], v);
      mx[k] = max(mx[k], v);
    }
  }
  for (int k = 0; k < d; ++k) {
    atomicMin(&c[2 * k], mn[k]);
    atomicMax(&c[2 * k + 1], mx[k]);
  }
}

__device__ __forceinline__ float centre_of(const int* c, int k) {
  const double lo = (double)from_ordered_int(c[2 * k]), hi = (double)from_ordered_int(c[2 * k + 1]);
  return __double2float_rn(0.5 * (lo + hi));
}

__global__ void centre_check_kernel(const float* __restrict__ x, int n, const float* __restrict__ y, int m, int d,
                                    int* c) {
  bool bad = false;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n + m; i += gridDim.x * blockDim.x) {
    const float* p = i < n ? x + (size_t)i * d : y + (size_t)(i - n) * d;
    for (int k = 0; k < d; ++k) {
      const float o = centre_of(c, k);
      const float v = p[k];
      bad |= (double)__fsub_rn(v, o) != (double)v - (double)o;  // not exact in FP32
    }
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&c[6], 1);
}

// Also writes rzeps: a bound on eps times the magnitude of the fast sweeps' FP32 exponent parts
// (base 2), log2 e (3 kappa sum_k M_k^2 + 2 omega) with M_k the largest |coordinate k| after the
// translation: kappa ||w||^2 and <A_p, w_q> eps / log2 e are at most kappa sum M_k^2 and
// 2 kappa sum M_k^2, and the offset-relative log scalings times eps at most about 2 omega.
__global__ void centre_origin_kernel(const int* c, int d, float* origin, double kappa, double omega,
                                     double* rzeps) {
  double m2 = 0.0;
  for (int k = 0; k < 3; ++k) {
    const float o = (k < d && c[6] == 0) ? centre_of(c, k) : 0.0f;
    origin[k] = o;
    if (k < d) {
      const double lo = (double)from_ordered_int(c[2 * k]) - o, hi = (double)from_ordered_int(c[2 * k + 1]) - o;
      const double M = fmax(fabs(lo), fabs(hi));
      m2 += M * M;
    }
  }
  *rzeps = 1.4426950408889634 * (3.0 * kappa * m2 + 2.0 * omega);
}

// Weight normalisation w / sum(w) with an optional floor for zero masses, and log w, in two
// launches.  The sum is deterministic: block b adds the fixed range [b * kNormChunk, (b + 1) *
// kNormChunk) in a fixed order and stores its partial in logw[b] (overwritten by the second
// launch); the last block to finish adds the partials in block order and stores the total in
// scratch[0].  scratch[1] is the arrival counter (reset by that block).  Sets err bit
// kErrNonFinite on a non-positive or non-finite weight.
constexpr int kNormPer = 16;                    // elements per thread in the sum pass
constexpr int kNormChunk = kThreads * kNormPer;  // elements per block in the sum pass

__device__ __forceinline__ double floored(double v, double floor_mass) {
  return (floor_mass > 0.0 && v < floor_mass && v >= 0.0) ? floor_mass : v;
}

__global__ void weight_sum_kernel(const double* __restrict__ w, int npts, double floor_mass,
                                  double* __restrict__ logw, double* scratch, int* err) {
  __shared__ double red[kThreads];
  __shared__ bool last;
  const int tid = threadIdx.x;
  const int i0 = blockIdx.x * kNormChunk;
  double s = 0.0;
  bool bad = false;
#pragma unroll 4
  for (int k = 0; k < kNormPer; ++k) {
    const int i = i0 + k * kThreads + tid;
    if (i < npts) {
      const double v = floored(w[i], floor_mass);
      bad |= !(v > 0.0) || !isfinite(v);
      s += v;
    }
  }
  if (bad) atomicOr(err, kErrNonFinite);
  const double part = block_sum(s, red);
  if (tid == 0) {
    logw[blockIdx.x] = part;
    __threadfence();
    unsigned* cnt = (unsigned*)(scratch + 1);
    last = atomicAdd(cnt, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double t = 0.0;
  for (int b = tid; b < (int)gridDim.x; b += kThreads) t += __ldcg(logw + b);
  const double tot = block_sum(t, red);
  if (tid == 0) {
    scratch[0] = tot;
    *(unsigned*)(scratch + 1) = 0u;
  }
}

__global__ void weight_log_kernel(const double* __restrict__ w, int npts, double floor_mass,
                                  const double* __restrict__ scratch, double* __restrict__ wn,
                                  double* __restrict__ logw) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npts) return;
  const double q = floored(w[i], floor_mass) / scratch[0];
  wn[i] = q;
  logw[i] = log(q);
}

// Column pack for iteration k from log beta^{k-1}, log beta^{k-2}:
// beta-tilde^{k-1} = beta^{k-1} + (beta^{k-1} - beta^{k-2}) / lambda (Algorithm 1 momentum).
// It also seeds the pack offsets (Inst::goff) of iterations k and k + 1 from the first point's
// beta-tilde and alpha; each iteration's finalisation sets those of two iterations ahead.
__global__ void repack_cols_kernel(const Inst* __restrict__ I) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= I->m) return;
  const long long k = *I->k;
  const double inv_eps = row_inv_eps(I, k);
  auto tilde = [&](int q) {
    const double b1 = I->log_beta[q], b2 = I->log_beta_prev[q];
    return alg_momentum(I->alg) ? b1 + (b1 - b2) / I->lambda : b1;
  };
  const double tn = tilde(j);
  double gy = 0.0;
  if (I->goff != nullptr) {
    gy = kLog2e * tilde(0);  // every thread derives the same value from the same inputs
    if (j == 0) {
      const double gx = kLog2e * I->log_alpha[0];
      for (int t = 0; t < 2; ++t) {
        I->goff[(k + t) & 3] = gx;
        I->goff[4 + ((k + t) & 3)] = gy;
      }
    }
  }
  I->log_beta_tilde_next[j] = tn;
  store_h(I->ypack, j, I->d, (tn - I->yn2[j] * inv_eps) * kLog2e - gy);
}

// max and min of ||x_i - y_j||^2 over all pairs (FP32, one launch, any grid size).
__global__ void pair_cost_range_kernel(const float* __restrict__ x, int n, const float* __restrict__ y, int m,
                                       int d, unsigned* __restrict__ out_max, unsigned* __restrict__ out_min) {
  __shared__ float ys[3][256];
  float mx = 0.0f, mn = FLT_MAX;
  for (int i0 = blockIdx.x * blockDim.x; i0 < n; i0 += gridDim.x * blockDim.x) {
    const int i = i0 + threadIdx.x;
    float xi[3] = {0, 0, 0};
    if (i < n)
      for (int k = 0; k < d; ++k) xi[k] = x[(size_t)i * d + k];
    for (int j0 = 0; j0 < m; j0 += 256) {
      __syncthreads();
      for (int t = threadIdx.x; t < 256; t += blockDim.x) {
        const int j = j0 + t;
        for (int k = 0; k < 3; ++k) ys[k][t] = (j < m && k < d) ? y[(size_t)j * d + k] : 0.0f;
      }
      __syncthreads();
      if (i < n) {
        const int jn = min(256, m - j0);
        for (int t = 0; t < jn; ++t) {
          float s = 0.0f;
          for (int k = 0; k < 3; ++k) {
            const float df = xi[k] - ys[k][t];
            s = fmaf(df, df, s);
          }
          mx = fmaxf(mx, s);
          mn = fminf(mn, s);
        }
      }
    }
  }
  // non-negative floats order like their bit patterns
  for (int o = 16; o > 0; o >>= 1) {
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(out_max, __float_as_uint(mx));
    atomicMin(out_min, __float_as_uint(mn));
  }
}

// Sweep kernel for dimension d, precision mode, points per thread R, chunk width ch and variant
// (0 row, 1 column, 2 column + certificate, 3 standalone certificate, 4 row + certificate).
SweepFn get_sweep(int d, int mode, int R, int ch, int variant) {
  switch (d) {
    case 1: return get_sweep_d1(mode, R, ch, variant);
    case 2: return get_sweep_d2(mode, R, ch, variant);
    case 3: return get_sweep_d3(mode, R, ch, variant);
  }
  return nullptr;
}
size_t sweep_smem_bytes() { return (size_t)kStages * kStageTiles * kNComp * kTQ * sizeof(float); }

cudaError_t launch_sweep(SweepFn fn, const Inst* insts, const Item* items, int nitems, int iters, int grid,
                         unsigned* sched, cudaStream_t stream) {
  if (nitems <= 0 || iters <= 0 || grid <= 0) return cudaSuccess;
  void* args[] = {(void*)&insts, (void*)&items, (void*)&nitems, (void*)&iters, (void*)&sched};
  return cudaLaunchKernel((const void*)fn, dim3(grid), dim3(kThreads), args, sweep_smem_bytes(), stream);
}

// The launch helpers go through cudaLaunchKernel, which returns the status of that launch: they
// neither read nor clear an error that an earlier call of the caller left pending.
cudaError_t launch_pack_coords(const float* pts, int npts, int d, int tiles, double kappa, float* pack,
                               double* n2, cudaStream_t s, const float* origin) {
  const int tot = tiles * kTQ;
  void* args[] = {(void*)&pts, (void*)&npts, (void*)&d, (void*)&tiles, (void*)&kappa, (void*)&pack, (void*)&n2,
                  (void*)&origin};
  cudaError_t e = cudaLaunchKernel((const void*)pack_coords_kernel, dim3((tot + 255) / 256), dim3(256), args, 0, s);
  if (e != cudaSuccess || d != 2 || tiles <= 0) return e;
  static_assert(kNComp - 1 >= 2 + 2, "a 2-D pack has a free component for the run flags");
  void* a2[] = {(void*)&pack, (void*)&npts};
  return cudaLaunchKernel((const void*)tile_runs_kernel, dim3(tiles), dim3(kTQ), a2, 0, s);
}

// The centring translation of the two clouds into origin (3 floats): zeros unless it is exact;
// and the fast sweeps' exponent bound rzeps (centre_origin_kernel).  scratch: 7 ints, initialised here.
cudaError_t launch_centre(const float* x, int n, const float* y, int m, int d, int* scratch, float* origin,
                          double kappa, double omega, double* rzeps, int sms, cudaStream_t s) {
  const int init[7] = {INT_MAX, INT_MIN, INT_MAX, INT_MIN, INT_MAX, INT_MIN, 0};
  cudaError_t e = cudaMemcpyAsync(scratch, init, sizeof(init), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  const int blocks = min((n + m + 255) / 256, sms * 4);
  void* a1[] = {(void*)&x, (void*)&n, (void*)&y, (void*)&m, (void*)&d, (void*)&scratch};
  if ((e = cudaLaunchKernel((const void*)centre_range_kernel, dim3(blocks), dim3(256), a1, 0, s)) != cudaSuccess)
    return e;
  if ((e = cudaLaunchKernel((const void*)centre_check_kernel, dim3(blocks), dim3(256), a1, 0, s)) != cudaSuccess)
    return e;
  const int* c = scratch;
  void* a2[] = {(void*)&c, (void*)&d, (void*)&origin, (void*)&kappa, (void*)&omega, (void*)&rzeps};
  return cudaLaunchKernel((const void*)centre_origin_kernel, dim3(1), dim3(1), a2, 0, s);
}

cudaError_t launch_normalise(const double* w, int npts, double floor_mass, double* wn, double* logw,
                             double* scratch, int* err, cudaStream_t s) {
  void* a1[] = {(void*)&w, (void*)&npts, (void*)&floor_mass, (void*)&logw, (void*)&scratch, (void*)&err};
  cudaError_t e = cudaLaunchKernel((const void*)weight_sum_kernel, dim3((npts + kNormChunk - 1) / kNormChunk),
                                   dim3(kThreads), a1, 0, s);
  if (e != cudaSuccess) return e;
  const double* sc = scratch;
  void* a2[] = {(void*)&w, (void*)&npts, (void*)&floor_mass, (void*)&sc, (void*)&wn, (void*)&logw};
  return cudaLaunchKernel((const void*)weight_log_kernel, dim3((npts + 255) / 256), dim3(256), a2, 0, s);
}

cudaError_t launch_repack_cols(const Inst* I, int m, cudaStream_t s) {
  void* args[] = {(void*)&I};
  return cudaLaunchKernel((const void*)repack_cols_kernel, dim3((m + 255) / 256), dim3(256), args, 0, s);
}

cudaError_t launch_pair_cost_range(const float* x, int n, const float* y, int m, int d, unsigned* mx,
                                   unsigned* mn, int sms, cudaStream_t s) {
  const int blocks = min((n + 255) / 256, sms * 8);
  void* args[] = {(void*)&x, (void*)&n, (void*)&y, (void*)&m, (void*)&d, (void*)&mx, (void*)&mn};
  return cudaLaunchKernel((const void*)pair_cost_range_kernel, dim3(blocks), dim3(256), args, 0, s);
}

}  // namespace ot
