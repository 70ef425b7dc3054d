// Output of the colour-transfer application (App. G, "Implicit implementation and output"): the
// barycentric projection of an implicit plan X = diag(u) K diag(v), K = exp(-C / eps),
//     y-hat_i = sum_j X_ij y_j / sum_j X_ij,
// and the marginal errors of Tables 3 and 4 (row sums of X against r, column sums against c).
// X is never formed: one sweep over the rows gives each row's sum and weighted target sum, one
// sweep over the columns gives each column's sum.  These run once per solve, so they favour a
// simple, accurate form over speed: the exponent is formed in float-float (error-free transforms)
// as in the certificate sweeps, the running shift follows the maximum exactly in powers of two,
// sums are Kahan-compensated FP32, and each CTA reduces its points over the whole other side in
// index order (deterministic).
#include <cmath>
#include <cstdint>

#include "ot_device.cuh"
#include "ot_kernels.cuh"

namespace ot {

namespace {

constexpr int kPlanR = 2;                      // points per thread
constexpr int kPlanCh = 8;                     // columns per chunk (one maximum and rescale test)
constexpr int kPlanChunkPts = 2048;            // points per block of the error reduction
constexpr double kL2e = 1.4426950408889634074;
// The exponent is exact in float-float until it is rounded to FP32 relative to the shift, so the
// shift follows the maximum closely (rescale when a chunk exceeds it by more than 1: the dominant
// terms stay within 2 of it, where that rounding costs < 2^-23 in log2), and a chunk whose shift
// moves is evaluated again against the new shift.
constexpr float kPlanTau = 1.0f;

__device__ __forceinline__ size_t pk_idx(int p, int comp) {
  return ((size_t)(p / kTQ) * kNComp + comp) * kTQ + (p % kTQ);
}

__device__ __forceinline__ void kadd(float& s, float& c, float x) {
  const float y = x - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

// One side of a plan sweep.
struct PlanSide {
  int np;                 // points of this side (the sums are per point)
  int qtiles;             // tiles of the other side
  int d;
  const float* ppack;     // this side's pack (coordinates used)
  const double* plog;     // this side's log scaling (log u or log v)
  const double* pn2;      // kappa ||p||^2
  const float* qpack;     // other side: coordinates and h = (log scaling - kappa ||q||^2 / eps) log2 e
  double kappa, inv_eps;
  double* log2_sum;       // out: log2 of the point's sum of plan entries
  float* proj;            // out (row side only): np x d barycentric projection, or null
  double* log2_cost;      // out (cost passes): log2 of sum_q ||p - q||^2 X_pq, or null
  const float* origin;    // translation of the packs' coordinates, added back to proj (or null)
};

// Exponent in base 2 (as in the sweep kernels): log2 X_pq = rc_p + h_q + <A_p, q>, with
// A_p = (2 kappa log2 e / eps) p and rc_p = (log scaling_p - kappa ||p||^2 / eps) log2 e.
template <int D, bool PROJ, bool COST>
__global__ void __launch_bounds__(kThreads) plan_sweep_kernel(PlanSide s) {
  __shared__ float tile[kNComp * kTQ];
  const int tid = threadIdx.x;
  const int p0 = blockIdx.x * (kThreads * kPlanR);
  float Ah[kPlanR][D], Al[kPlanR][D], pu[kPlanR][D];
  double rc[kPlanR];
  const double sig = 2.0 * s.kappa * kL2e * s.inv_eps;
#pragma unroll
  for (int r = 0; r < kPlanR; ++r) {
    const int p = p0 + r * kThreads + tid;
    const bool ok = p < s.np;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const float u = ok ? s.ppack[pk_idx(p, k)] : 0.0f;
      pu[r][k] = u;
      const double A = sig * (double)u;
      Ah[r][k] = __double2float_rn(A);
      Al[r][k] = __double2float_rn(A - (double)Ah[r][k]);
    }
    rc[r] = ok ? (s.plog[p] - s.pn2[p] * s.inv_eps) * kL2e : 0.0;
  }
  float mref[kPlanR], S[kPlanR], Sc[kPlanR], Y[kPlanR][D], Yc[kPlanR][D], N[kPlanR], Nc[kPlanR];
#pragma unroll
  for (int r = 0; r < kPlanR; ++r) {
    mref[r] = 0.0f;
    S[r] = Sc[r] = 0.0f;
    N[r] = Nc[r] = 0.0f;
#pragma unroll
    for (int k = 0; k < D; ++k) Y[r][k] = Yc[r][k] = 0.0f;
  }
  bool fresh = true;
  for (int t = 0; t < s.qtiles; ++t) {
    __syncthreads();
    for (int i = tid; i < kNComp * kTQ; i += kThreads) tile[i] = s.qpack[(size_t)t * kNComp * kTQ + i];
    __syncthreads();
    for (int c0 = 0; c0 < kTQ; c0 += kPlanCh) {
      float v[kPlanR][kPlanCh];
      auto eval = [&]() {
#pragma unroll
      for (int cc = 0; cc < kPlanCh; ++cc) {
        const int c = c0 + cc;
        float w[D];
#pragma unroll
        for (int k = 0; k < D; ++k) w[k] = tile[k * kTQ + c];
        const float hh = tile[D * kTQ + c], hl = tile[(D + 1) * kTQ + c];
#pragma unroll
        for (int r = 0; r < kPlanR; ++r) {
          // z - shift in float-float: (hh - shift) + hl + sum_k (Ah_k + Al_k) w_k, rounded once
          float sb, e0;
          two_sum(hh, -mref[r], sb, e0);
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
      };
      eval();
      bool moved = false;
#pragma unroll
      for (int r = 0; r < kPlanR; ++r) {
        float cm = v[r][0];
#pragma unroll
        for (int cc = 1; cc < kPlanCh; ++cc) cm = fmaxf(cm, v[r][cc]);
        if (fresh || cm > kPlanTau) {
          const float sh = floorf(cm);
          if (!fresh) {  // exact power-of-two rescale of the running sums
            const float f = exp2_neg_int(sh);
            S[r] *= f;
            Sc[r] *= f;
            N[r] *= f;
            Nc[r] *= f;
#pragma unroll
            for (int k = 0; k < D; ++k) {
              Y[r][k] *= f;
              Yc[r][k] *= f;
            }
          }
          mref[r] += sh;
          moved = true;
        }
      }
      if (moved) eval();  // against the new shifts
      fresh = false;
#pragma unroll
      for (int r = 0; r < kPlanR; ++r) {
        float cs = 0.0f, cn = 0.0f, cy[D];
#pragma unroll
        for (int k = 0; k < D; ++k) cy[k] = 0.0f;
#pragma unroll
        for (int cc = 0; cc < kPlanCh; ++cc) {
          const float E = ex2_mufu(v[r][cc]);
          cs += E;
          if constexpr (COST) {
            float d2 = 0.0f;
#pragma unroll
            for (int k = 0; k < D; ++k) {
              const float df = pu[r][k] - tile[k * kTQ + c0 + cc];
              d2 = __fmaf_rn(df, df, d2);
            }
            cn = __fmaf_rn(d2, E, cn);
          }
          if constexpr (PROJ) {
#pragma unroll
            for (int k = 0; k < D; ++k) cy[k] = __fmaf_rn(E, tile[k * kTQ + c0 + cc], cy[k]);
          }
        }
        kadd(S[r], Sc[r], cs);
        if constexpr (COST) kadd(N[r], Nc[r], cn);
        if constexpr (PROJ) {
#pragma unroll
          for (int k = 0; k < D; ++k) kadd(Y[r][k], Yc[r][k], cy[k]);
        }
      }
    }
  }
#pragma unroll
  for (int r = 0; r < kPlanR; ++r) {
    const int p = p0 + r * kThreads + tid;
    if (p >= s.np) continue;
    const double sum = (double)S[r] - (double)Sc[r];
    s.log2_sum[p] = rc[r] + (double)mref[r] + log2(sum);
    if constexpr (COST) s.log2_cost[p] = rc[r] + (double)mref[r] + log2((double)N[r] - (double)Nc[r]);
    if constexpr (PROJ) {
#pragma unroll
      for (int k = 0; k < D; ++k)
        s.proj[(size_t)p * D + k] =
            (float)(((double)Y[r][k] - (double)Yc[r][k]) / sum + (s.origin != nullptr ? (double)s.origin[k] : 0.0));
    }
  }
}

// The plan's log scalings from the state: which = 0 best certificate (u = exp(f / eps),
// v = c exp(g / eps)), 1 latest iterate (alpha-hat, beta-hat), 2 intermediate plan (alpha-hat,
// beta-tilde).
__global__ void plan_logs_kernel(int which, int n, int m, double inv_eps, const double* f, const double* g,
                                 const double* log_b, const double* lah, const double* lbh, const double* lbt,
                                 double* lu, double* lv) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) lu[i] = which == 0 ? f[i] * inv_eps : lah[i];
  if (i < m) lv[i] = which == 0 ? log_b[i] + g[i] * inv_eps : (which == 1 ? lbh[i] : lbt[i]);
}

// A pack with the coordinates of `src` and h = (lv - n2 / eps) log2 e (hi/lo pair); padding points
// get h = -1e30 so that they contribute nothing.
__global__ void plan_pack_kernel(const float* src, int np, int tiles, int d, const double* lv, const double* n2,
                                 double inv_eps, float* dst) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= tiles * kTQ) return;
  for (int k = 0; k < d; ++k) dst[pk_idx(p, k)] = src[pk_idx(p, k)];
  float hi = -1.0e30f, lo = 0.0f;
  if (p < np) {
    const double h = (lv[p] - n2[p] * inv_eps) * kL2e;
    hi = __double2float_rn(h);
    lo = __double2float_rn(h - (double)hi);
  }
  dst[pk_idx(p, d)] = hi;
  dst[pk_idx(p, d + 1)] = lo;
  for (int k = d + 2; k < kNComp; ++k) dst[pk_idx(p, k)] = 0.0f;
}

// sums = 2^log2_sum and their errors against the prescribed masses w: out = {l1, max abs, max rel}.
// Deterministic: block b adds the fixed range [b * kPlanChunkPts, ...) in index order, and the last
// block adds the block partials in block order (maxima do not depend on the order).
__global__ void marginal_error_kernel(const double* log2_sum, const double* w, int np, double* sums, double* part,
                                      unsigned* counter, double* out) {
  __shared__ double red[3][kThreads];
  __shared__ bool last;
  const int tid = threadIdx.x;
  double l1 = 0.0, mabs = 0.0, mrel = 0.0;
  const int i0 = blockIdx.x * kPlanChunkPts;
  for (int k = 0; k < kPlanChunkPts / kThreads; ++k) {
    const int i = i0 + k * kThreads + tid;
    if (i < np) {
      const double sv = exp2(log2_sum[i]);
      sums[i] = sv;
      const double e = fabs(sv - w[i]);
      l1 += e;
      mabs = fmax(mabs, e);
      mrel = fmax(mrel, e / w[i]);
    }
  }
  red[0][tid] = l1;
  red[1][tid] = mabs;
  red[2][tid] = mrel;
  __syncthreads();
  for (int st = kThreads / 2; st > 0; st >>= 1) {
    if (tid < st) {
      red[0][tid] += red[0][tid + st];
      red[1][tid] = fmax(red[1][tid], red[1][tid + st]);
      red[2][tid] = fmax(red[2][tid], red[2][tid + st]);
    }
    __syncthreads();
  }
  if (tid == 0) {
    part[3 * blockIdx.x] = red[0][0];
    part[3 * blockIdx.x + 1] = red[1][0];
    part[3 * blockIdx.x + 2] = red[2][0];
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last || tid != 0) return;
  __threadfence();
  double a = 0.0, b = 0.0, c = 0.0;
  for (unsigned k = 0; k < gridDim.x; ++k) {
    a += __ldcg(&part[3 * k]);
    b = fmax(b, __ldcg(&part[3 * k + 1]));
    c = fmax(c, __ldcg(&part[3 * k + 2]));
  }
  out[0] = a;
  out[1] = b;
  out[2] = c;
  *counter = 0u;
}

template <bool PROJ, bool COST = false>
cudaError_t launch_plan_sweep(const PlanSide& s, cudaStream_t st) {
  const int blocks = (s.np + kThreads * kPlanR - 1) / (kThreads * kPlanR);
  switch (s.d) {
    case 1: plan_sweep_kernel<1, PROJ, COST><<<blocks, kThreads, 0, st>>>(s); break;
    case 2: plan_sweep_kernel<2, PROJ, COST><<<blocks, kThreads, 0, st>>>(s); break;
    case 3: plan_sweep_kernel<3, PROJ, COST><<<blocks, kThreads, 0, st>>>(s); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// lu_out = lu + min(log w - ln 2 * log2_sum, 0): the scalings of diag(min(w / sums, 1)) X.
__global__ void plan_scale_kernel(int np, const double* lu, const double* log2_sum, const double* log_w,
                                  double* lu_out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < np) lu_out[i] = lu[i] + fmin(log_w[i] - log2_sum[i] * 0.69314718055994530942, 0.0);
}

constexpr int kRoundThreads = 1024;

// One side's sums for the rounding (one block, fixed order: deterministic).  With e = w - sums of
// the rounded-down plan (sums = 2^(log2_sum + (lu_new - lu_old) log2 e) when lu_old is given), writes
// out = {sum e ||p||^2, sum e, sum e p_0..p_2, sum |e|, kappa sum 2^log2_cost (if given),
//        kappa sum 2^log2_cost0 (if given)}.
__global__ void __launch_bounds__(kRoundThreads) round_sums_kernel(int np, int d, const double* w,
                                                                   const double* log2_sum, const double* lu_new,
                                                                   const double* lu_old, const float* pack,
                                                                   const double* n2, double kappa,
                                                                   const double* log2_cost,
                                                                   const double* log2_cost0, double* out) {
  __shared__ double red[kRoundThreads];
  double acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int i = threadIdx.x; i < np; i += kRoundThreads) {
    double l2 = log2_sum[i];
    if (lu_old) l2 += (lu_new[i] - lu_old[i]) * kL2e;
    const double e = w[i] - exp2(l2);
    acc[0] += e * n2[i] / kappa;
    acc[1] += e;
    for (int k = 0; k < d; ++k) acc[2 + k] += e * (double)pack[pk_idx(i, k)];
    acc[5] += fabs(e);
    if (log2_cost) acc[6] += kappa * exp2(log2_cost[i]);
    if (log2_cost0) acc[7] += kappa * exp2(log2_cost0[i]);
  }
  for (int q = 0; q < 8; ++q) {
    red[threadIdx.x] = acc[q];
    __syncthreads();
    for (int st = kRoundThreads / 2; st > 0; st >>= 1) {
      if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[q] = red[0];
    __syncthreads();
  }
}

}  // namespace

// Bytes of working memory plan_diagnostics needs for an n x m instance.
size_t plan_scratch_bytes(int64_t n, int64_t m) {
  const int64_t tx = (n + kTQ - 1) / kTQ, ty = (m + kTQ - 1) / kTQ;
  const int64_t bx = (n + kPlanChunkPts - 1) / kPlanChunkPts, by = (m + kPlanChunkPts - 1) / kPlanChunkPts;
  return 256 * 10 + sizeof(double) * (size_t)(2 * n + 2 * m + 3 * (bx + by)) +
         sizeof(float) * (size_t)((tx + ty) * kNComp * kTQ) + 2 * sizeof(unsigned);
}

// Diagnostics of the plan `which` (see plan_logs_kernel) at temperature eps on the instance's device
// data; scratch holds plan_scratch_bytes(n, m) bytes.  Outputs (device): y_hat [n x d] floats,
// row [n] and col [m] doubles, err[6] = row {l1, max abs, max rel}, then the same for the columns.
cudaError_t plan_diagnostics(const Inst& h, int which, double eps, const double* f_best, const double* g_best,
                             void* scratch, float* y_hat, double* row, double* col, double* err, cudaStream_t st) {
  const int n = h.n, m = h.m, d = h.d;
  const int tx = h.tiles_x, ty = h.tiles_y;
  const int bx = (n + kPlanChunkPts - 1) / kPlanChunkPts, by = (m + kPlanChunkPts - 1) / kPlanChunkPts;
  char* base = (char*)scratch;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    off = (off + 255) & ~(size_t)255;
    void* p = base + off;
    off += bytes;
    return p;
  };
  double* lu = (double*)take(sizeof(double) * n);
  double* lv = (double*)take(sizeof(double) * m);
  double* l2r = (double*)take(sizeof(double) * n);
  double* l2c = (double*)take(sizeof(double) * m);
  float* xp = (float*)take(sizeof(float) * (size_t)tx * kNComp * kTQ);
  float* yp = (float*)take(sizeof(float) * (size_t)ty * kNComp * kTQ);
  double* part = (double*)take(sizeof(double) * 3 * (bx + by));
  unsigned* counter = (unsigned*)take(2 * sizeof(unsigned));
  const double inv_eps = 1.0 / eps;
  cudaError_t e;
  if ((e = cudaMemsetAsync(counter, 0, 2 * sizeof(unsigned), st)) != cudaSuccess) return e;
  const int nm = n > m ? n : m;
  plan_logs_kernel<<<(nm + 255) / 256, 256, 0, st>>>(which, n, m, inv_eps, f_best, g_best, h.log_b,
                                                     h.log_alpha_hat, h.log_beta_hat, h.log_beta_tilde, lu, lv);
  // rows reduce over columns (the column pack carries log v); columns reduce over rows (log u)
  plan_pack_kernel<<<(ty * kTQ + 255) / 256, 256, 0, st>>>(h.ypack, m, ty, d, lv, h.yn2, inv_eps, yp);
  plan_pack_kernel<<<(tx * kTQ + 255) / 256, 256, 0, st>>>(h.xpack, n, tx, d, lu, h.xn2, inv_eps, xp);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  PlanSide rs{n, ty, d, h.xpack, lu, h.xn2, yp, h.kappa, inv_eps, l2r, y_hat, nullptr, h.origin};
  PlanSide cs{m, tx, d, h.ypack, lv, h.yn2, xp, h.kappa, inv_eps, l2c, nullptr, nullptr};
  if ((e = launch_plan_sweep<true>(rs, st)) != cudaSuccess) return e;
  if ((e = launch_plan_sweep<false>(cs, st)) != cudaSuccess) return e;
  marginal_error_kernel<<<bx, kThreads, 0, st>>>(l2r, h.a, n, row, part, counter, err);
  marginal_error_kernel<<<by, kThreads, 0, st>>>(l2c, h.b, m, col, part + 3 * bx, counter + 1, err + 3);
  return cudaGetLastError();
}

// Bytes of working memory plan_rounding needs for an n x m instance.
size_t round_scratch_bytes(int64_t n, int64_t m) {
  const int64_t tx = (n + kTQ - 1) / kTQ, ty = (m + kTQ - 1) / kTQ;
  return 256 * 14 + sizeof(double) * (size_t)(6 * n + 4 * m + 32) + sizeof(float) * (size_t)((tx + ty) * kNComp * kTQ);
}

// Rounding of the plan `which` at temperature eps onto Pi(r, c) without forming it: scale the rows
// of X down to at most r (one row pass), the columns of the result down to at most c (one column
// pass), then add err_r err_c^T / |err_r|_1, whose cost separates for the squared-Euclidean cost:
//   err_r^T C err_c = kappa [(sum err_r |x|^2)(sum err_c) + (sum err_r)(sum err_c |y|^2)
//                            - 2 <sum err_r x, sum err_c y>].
// A third (row) pass gives the scaled plan's row sums and cost.  sums (device, 16 doubles): [0..7]
// the row-side sums of round_sums_kernel (with the rounded and the unrounded plan's costs), [8..15]
// the column side's.
cudaError_t plan_rounding(const Inst& h, int which, double eps, const double* f_best, const double* g_best,
                          void* scratch, double* sums, cudaStream_t st) {
  const int n = h.n, m = h.m, d = h.d;
  const int tx = h.tiles_x, ty = h.tiles_y;
  char* base = (char*)scratch;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    off = (off + 255) & ~(size_t)255;
    void* p = base + off;
    off += bytes;
    return p;
  };
  double* lu = (double*)take(sizeof(double) * n);
  double* lu1 = (double*)take(sizeof(double) * n);
  double* l2r = (double*)take(sizeof(double) * n);
  double* l2cost0 = (double*)take(sizeof(double) * n);
  double* l2r2 = (double*)take(sizeof(double) * n);
  double* l2cost = (double*)take(sizeof(double) * n);
  double* lv = (double*)take(sizeof(double) * m);
  double* lv1 = (double*)take(sizeof(double) * m);
  double* l2c = (double*)take(sizeof(double) * m);
  double* unused = (double*)take(sizeof(double) * m);
  (void)unused;
  float* xp = (float*)take(sizeof(float) * (size_t)tx * kNComp * kTQ);
  float* yp = (float*)take(sizeof(float) * (size_t)ty * kNComp * kTQ);
  const double inv_eps = 1.0 / eps;
  const int nm = n > m ? n : m;
  cudaError_t e;
  plan_logs_kernel<<<(nm + 255) / 256, 256, 0, st>>>(which, n, m, inv_eps, f_best, g_best, h.log_b,
                                                     h.log_alpha_hat, h.log_beta_hat, h.log_beta_tilde, lu, lv);
  // pass 1 (rows of X): row sums and cost; scale the rows down to at most r
  plan_pack_kernel<<<(ty * kTQ + 255) / 256, 256, 0, st>>>(h.ypack, m, ty, d, lv, h.yn2, inv_eps, yp);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  PlanSide r1{n, ty, d, h.xpack, lu, h.xn2, yp, h.kappa, inv_eps, l2r, nullptr, l2cost0};
  if ((e = launch_plan_sweep<false, true>(r1, st)) != cudaSuccess) return e;
  plan_scale_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, lu, l2r, h.log_a, lu1);
  // pass 2 (columns of the row-scaled plan): scale the columns down to at most c
  plan_pack_kernel<<<(tx * kTQ + 255) / 256, 256, 0, st>>>(h.xpack, n, tx, d, lu1, h.xn2, inv_eps, xp);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  PlanSide c2{m, tx, d, h.ypack, lv, h.yn2, xp, h.kappa, inv_eps, l2c, nullptr, nullptr};
  if ((e = launch_plan_sweep<false>(c2, st)) != cudaSuccess) return e;
  plan_scale_kernel<<<(m + 255) / 256, 256, 0, st>>>(m, lv, l2c, h.log_b, lv1);
  // pass 3 (rows of the scaled plan): row sums (for err_r) and cost
  plan_pack_kernel<<<(ty * kTQ + 255) / 256, 256, 0, st>>>(h.ypack, m, ty, d, lv1, h.yn2, inv_eps, yp);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  PlanSide r3{n, ty, d, h.xpack, lu1, h.xn2, yp, h.kappa, inv_eps, l2r2, nullptr, l2cost};
  if ((e = launch_plan_sweep<false, true>(r3, st)) != cudaSuccess) return e;
  // err_r = r - rows of the scaled plan; err_c = c - columns: the column sums of pass 2 times the
  // column factors (lv1 - lv)
  round_sums_kernel<<<1, kRoundThreads, 0, st>>>(n, d, h.a, l2r2, nullptr, nullptr, h.xpack, h.xn2, h.kappa,
                                                 l2cost, l2cost0, sums);
  round_sums_kernel<<<1, kRoundThreads, 0, st>>>(m, d, h.b, l2c, lv1, lv, h.ypack, h.yn2, h.kappa, nullptr,
                                                 nullptr, sums + 8);
  return cudaGetLastError();
}

}  // namespace ot
