// Fused pass over the observations: utilities, row softmax, log-likelihood and
// gradient (Sec. 2.1 eqs. "unormalized utility", "probability", "base
// probability"; Sec. 3.1 eq. "log-lik function"; Sec. 3.3 eq. "loglik gradient").
//
// Utilities are formed over all K alternatives from the raw data,
//     u_ik = X_i.beta_k + Y_ik.gamma_k + Z_ik.alpha   (beta_0 = gamma_0 = 0),
// which differs from the paper's normalized V_ik = u_ik - u_i0 by a per-row
// constant; the softmax, l and every derivative are unchanged by it, and
// Z_ik - Z_i0 never has to be formed.
//
// Work layout: a persistent grid walks tiles of `rows` consecutive
// observations.  Each tile's X, Y and Z rows (contiguous in memory) are staged
// in shared memory with 16-byte loads; one warp per observation computes the
// utilities with lanes over alternatives, and warp shuffles give the max and
// the sum of the softmax.  The residuals r_ik = I(y_i = k) - P_ik of the tile
// stay in shared memory and every thread then adds its own gradient
// accumulators
//     beta_k[j]  += sum_rows r_ik X_ij,   gamma_k[j] += sum_rows r_ik Y_ikj,
//     alpha_k[j] += sum_rows r_ik Z_ikj   (summed over k at the end).
// In float32 the per-tile sums are folded into Kahan-compensated running sums;
// each CTA writes float64 partials that a second kernel adds in fixed order.
#include <algorithm>
#include <cfloat>

#include "mnl_internal.cuh"

namespace mnl {
namespace {

constexpr int kMaxClassSlots = 8;  // K <= 256 alternatives (lanes x slots)

template <typename T>
struct Acc;  // running sum with compensation in float32, plain in float64

template <>
struct Acc<float> {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float v) {
    const float y = v - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

template <>
struct Acc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double v) { s += v; }
  __device__ __forceinline__ double value() const { return s; }
};

__device__ __forceinline__ float fexp(float x) { return expf(x); }
__device__ __forceinline__ double fexp(double x) { return exp(x); }
__device__ __forceinline__ float flog(float x) { return logf(x); }
__device__ __forceinline__ double flog(double x) { return log(x); }

template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Copy `count` floats from global (src) to shared (dst); 16-byte moves when
// both sides are 16-byte aligned.
__device__ __forceinline__ void stage(float *dst, const float *src, int64_t count) {
  const int tid = threadIdx.x, nt = blockDim.x;
  if (((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15) == 0) {
    const int64_t n4 = count >> 2;
    const float4 *s4 = reinterpret_cast<const float4 *>(src);
    float4 *d4 = reinterpret_cast<float4 *>(dst);
    for (int64_t e = tid; e < n4; e += nt) d4[e] = __ldcs(s4 + e);
    for (int64_t e = (n4 << 2) + tid; e < count; e += nt) dst[e] = __ldcs(src + e);
  } else {
    for (int64_t e = tid; e < count; e += nt) dst[e] = __ldcs(src + e);
  }
}

struct PassDims {
  int64_t N;
  int K, p, d, f;
  int64_t nb, ng, mc, nout;
  int rows;  // rows per tile
  int64_t ntiles;
};

// Shared memory (bytes, 16-aligned pieces):
//   coef  T   [(p + d) * K + f]   Bt[j][k] = beta_k[j], Gt[j][k] = gamma_k[j], alpha
//   tile  f32 [rows * (p + K d + K f)]   Xs | Ys | Zs
//   res   T   [rows * K]          residuals (FULL only)
//   red   f64 [32 * 4]            per-warp log-likelihood partials
// One CTA processes tiles tile0, tile0 + tstride, ... < tile1 of one problem
// and writes its partial row `out` = [l, sum |l_i|, g (FULL only)].
template <typename T, bool FULL, int NPT>
__device__ __forceinline__ void pass_segment(const PassDims &D, const PassIO &io, int64_t tile0, int64_t tile1,
                                             int64_t tstride, double *out) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int K = D.K, p = D.p, d = D.d, f = D.f, R = D.rows;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;

  size_t off = 0;
  T *coef = reinterpret_cast<T *>(smem);
  off += (((size_t)(p + d) * K + f) * sizeof(T) + 15) & ~(size_t)15;
  float *Xs = reinterpret_cast<float *>(smem + off);
  float *Ys = Xs + (size_t)R * p;
  float *Zs = Ys + (size_t)R * K * d;
  off += (((size_t)R * (p + (size_t)K * d + (size_t)K * f)) * sizeof(float) + 15) & ~(size_t)15;
  T *res = reinterpret_cast<T *>(smem + off);
  if (FULL) off += (((size_t)R * K) * sizeof(T) + 15) & ~(size_t)15;
  double *red = reinterpret_cast<double *>(smem + off);

  T *Bt = coef, *Gt = coef + (size_t)p * K, *al = coef + (size_t)(p + d) * K;

  // Coefficients theta (+ t * delta) in the transposed per-alternative layout.
  const double t = io.delta ? *io.tscale : 0.0;
  for (int64_t e = tid; e < (int64_t)(p + d) * K + f; e += blockDim.x) {
    double v = 0.0;
    if (e < (int64_t)p * K) {
      const int j = (int)(e / K), k = (int)(e % K);
      if (k > 0) {
        const int64_t a = (int64_t)(k - 1) * p + j;
        v = io.theta[a] + (io.delta ? t * io.delta[a] : 0.0);
      }
    } else if (e < (int64_t)(p + d) * K) {
      const int64_t e2 = e - (int64_t)p * K;
      const int j = (int)(e2 / K), k = (int)(e2 % K);
      if (k > 0) {
        const int64_t a = D.nb + (int64_t)(k - 1) * d + j;
        v = io.theta[a] + (io.delta ? t * io.delta[a] : 0.0);
      }
    } else {
      const int64_t a = D.mc + (e - (int64_t)(p + d) * K);
      v = io.theta[a] + (io.delta ? t * io.delta[a] : 0.0);
    }
    coef[e] = (T)v;
  }

  Acc<T> lsum, labs;  // lane 0 of each warp
  Acc<T> acc[FULL ? NPT : 1];

  for (int64_t tile = tile0; tile < tile1; tile += tstride) {
    const int64_t row0 = tile * R;
    const int nrows = (int)min((int64_t)R, D.N - row0);
    __syncthreads();  // previous tile fully consumed (and coefficients written)
    stage(Xs, io.X + row0 * p, (int64_t)nrows * p);
    if (d) stage(Ys, io.Y + row0 * K * d, (int64_t)nrows * K * d);
    if (f) stage(Zs, io.Z + row0 * K * f, (int64_t)nrows * K * f);
    __syncthreads();

    // ---- utilities, softmax, log-likelihood: one warp per observation ----
    for (int r = warp; r < nrows; r += nwarps) {
      const int64_t i = row0 + r;
      const float *x = Xs + (size_t)r * p;
      const int yi = __ldg(io.choice + i);
      const T wi = io.w ? (T)__ldg(io.w + i) : (T)1;  // case weight (Sec. 2.3 "weights")
      T u[kMaxClassSlots];
      T umax = -(T)FLT_MAX, uy = 0;
#pragma unroll
      for (int c = 0; c < kMaxClassSlots; ++c) {
        const int k = lane + 32 * c;
        u[c] = -(T)FLT_MAX;
        if (k < K) {
          T v = 0;
          for (int j = 0; j < p; ++j) v = fma((T)x[j], Bt[(size_t)j * K + k], v);
          const float *y = Ys + ((size_t)r * K + k) * d;
          for (int j = 0; j < d; ++j) v = fma((T)y[j], Gt[(size_t)j * K + k], v);
          const float *z = Zs + ((size_t)r * K + k) * f;
          for (int j = 0; j < f; ++j) v = fma((T)z[j], al[j], v);
          u[c] = v;
          umax = fmax(umax, v);
          if (k == yi) uy = v;
        }
      }
      if (FULL && io.Pin) {  // Hessian-vector product: r_ik = w_i P_ik (u_ik - ubar_i)
        const T *Pr = reinterpret_cast<const T *>(io.Pin) + i * K;
        T pk[kMaxClassSlots], ub = 0;
#pragma unroll
        for (int c = 0; c < kMaxClassSlots; ++c) {
          const int k = lane + 32 * c;
          pk[c] = k < K ? Pr[k] : (T)0;
          if (k < K) ub = fma(pk[c], u[c], ub);
        }
        ub = warp_sum(ub);
#pragma unroll
        for (int c = 0; c < kMaxClassSlots; ++c) {
          const int k = lane + 32 * c;
          if (k < K) res[(size_t)r * K + k] = wi * pk[c] * (u[c] - ub);
        }
        continue;
      }
      umax = warp_max(umax);
      T s = 0;
#pragma unroll
      for (int c = 0; c < kMaxClassSlots; ++c) {
        const int k = lane + 32 * c;
        if (k < K) { u[c] = fexp(u[c] - umax); s += u[c]; }
      }
      s = warp_sum(s);
      uy = warp_sum(uy);  // one lane holds the chosen alternative's utility
      const T inv = (T)1 / s;
      const T lse = umax + flog(s);
      if (lane == 0) {
        const T li = uy - lse;
        lsum.add(wi * li);
        labs.add(wi * fabs(li));
      }
      if (FULL) {
        T *pr = reinterpret_cast<T *>(io.P) + i * K;
#pragma unroll
        for (int c = 0; c < kMaxClassSlots; ++c) {
          const int k = lane + 32 * c;
          if (k < K) {
            const T P = u[c] * inv;
            u[c] = P;
            pr[k] = P;
            res[(size_t)r * K + k] = wi * ((k == yi ? (T)1 : (T)0) - P);
          }
        }
        for (int j = 0; j < f; ++j) {
          T zb = 0;
#pragma unroll
          for (int c = 0; c < kMaxClassSlots; ++c) {
            const int k = lane + 32 * c;
            if (k < K) zb = fma(u[c], (T)Zs[((size_t)r * K + k) * f + j], zb);
          }
          zb = warp_sum(zb);
          if (lane == 0) reinterpret_cast<T *>(io.zbar)[i * f + j] = zb;
        }
      }
    }

    if (FULL) {
      __syncthreads();
      // ---- gradient accumulators owned by this thread ----
#pragma unroll
      for (int sl = 0; sl < NPT; ++sl) {
        const int64_t o = tid + (int64_t)sl * blockDim.x;
        if (o < D.nout) {
          int k;
          const float *src;
          int64_t stride;
          if (o < D.nb) { k = (int)(o / p) + 1; src = Xs + (o % p); stride = p; }
          else if (o < D.mc) {
            const int64_t e = o - D.nb;
            k = (int)(e / d) + 1;
            src = Ys + (size_t)k * d + (e % d);
            stride = (int64_t)K * d;
          } else {
            const int64_t e = o - D.mc;
            k = (int)(e / f);
            src = Zs + (size_t)k * f + (e % f);
            stride = (int64_t)K * f;
          }
          T part = 0;
          for (int r = 0; r < nrows; ++r) part = fma(res[(size_t)r * K + k], (T)src[r * stride], part);
          acc[sl].add(part);
        }
      }
    }
  }

  // ---- CTA partials (float64) ----
  if (lane == 0) {
    red[warp * 2 + 0] = lsum.value();
    red[warp * 2 + 1] = labs.value();
  }
  __syncthreads();
  // Partials row: [l, sum |l_i|, g (theta order: class coefficients, then alpha)].
  if (tid == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < nwarps; ++w) { a += red[w * 2]; b += red[w * 2 + 1]; }
    out[0] = a;
    out[1] = b;
  }
  if (FULL) {
    // alpha: this CTA's K partial sums per generic column, added over k in fixed order
    double *az = reinterpret_cast<double *>(Xs);  // the tile area is free now (>= K f doubles)
    __syncthreads();
#pragma unroll
    for (int sl = 0; sl < NPT; ++sl) {
      const int64_t o = tid + (int64_t)sl * blockDim.x;
      if (o < D.mc) out[2 + o] = acc[sl].value();
      else if (o < D.nout) az[o - D.mc] = acc[sl].value();
    }
    __syncthreads();
    for (int j = tid; j < f; j += blockDim.x) {
      double sa = 0.0;
      for (int k = 0; k < K; ++k) sa += az[k * f + j];
      out[2 + D.mc + j] = sa;
    }
  }
  __syncthreads();  // the shared memory is reused by the caller's next segment
}

template <typename T, bool FULL, int NPT>
__global__ void __launch_bounds__(512) pass_kernel(PassDims D, PassIO io) {
  double *out = io.partials + (int64_t)blockIdx.x * (FULL ? 2 + D.mc + D.f : 2);
  pass_segment<T, FULL, NPT>(D, io, blockIdx.x, D.ntiles, gridDim.x, out);
}

// Grouped pass over many problems: CTA c walks its segments
// segs[seg_start[c] .. seg_start[c+1]), skipping problems with active == 0.
template <typename T, bool FULL, int NPT>
__global__ void __launch_bounds__(512) grouped_pass_kernel(const GroupProblem *__restrict__ probs,
                                                           const PassSeg *__restrict__ segs,
                                                           const int *__restrict__ seg_start,
                                                           const int *__restrict__ active, int rows,
                                                           double *__restrict__ partials) {
  for (int si = seg_start[blockIdx.x]; si < seg_start[blockIdx.x + 1]; ++si) {
    const PassSeg sg = segs[si];
    const GroupProblem &gp = probs[sg.problem];
    if (active[sg.problem] == 0) continue;
    PassDims D;
    D.N = gp.N; D.K = gp.K; D.p = gp.p; D.d = gp.d; D.f = gp.f;
    D.nb = (int64_t)(gp.K - 1) * gp.p; D.ng = (int64_t)(gp.K - 1) * gp.d; D.mc = D.nb + D.ng;
    D.nout = D.mc + (int64_t)gp.K * gp.f;
    D.rows = rows;
    D.ntiles = (gp.N + rows - 1) / rows;
    PassIO io{};
    io.X = gp.X; io.Y = gp.Y; io.Z = gp.Z; io.choice = gp.choice;
    io.theta = gp.theta;
    io.delta = FULL ? nullptr : gp.delta;
    io.tscale = gp.scal + kGsT;
    io.P = gp.P; io.zbar = gp.zbar;
    io.partials = nullptr;
    pass_segment<T, FULL, NPT>(D, io, sg.tile0, sg.tile1, 1, partials + (FULL ? sg.slot_full : sg.slot_ll));
  }
}

// Per-problem fixed-order reduction of the grouped pass partials:
// l -> scal[base], sum |l_i| -> scal[base+1]; FULL: g -> grad, max|g| -> scal[kGsGinf].
template <bool FULL>
__global__ void __launch_bounds__(128) grouped_reduce_kernel(const GroupProblem *__restrict__ probs,
                                                             const int *__restrict__ slot_start,
                                                             const PassSeg *__restrict__ segs,
                                                             const int *__restrict__ slot_segs,
                                                             const int *__restrict__ active,
                                                             const double *__restrict__ partials, int base) {
  const int b = blockIdx.x;
  if (active[b] == 0) return;
  const GroupProblem &gp = probs[b];
  const int64_t n = (int64_t)(gp.K - 1) * (gp.p + gp.d) + gp.f;
  const int64_t len = FULL ? 2 + n : 2;
  const int s0 = slot_start[b], s1 = slot_start[b + 1];
  __shared__ double red[4];
  double gmax = 0.0;
  for (int64_t o = threadIdx.x; o < len; o += blockDim.x) {
    double acc = 0.0;
    for (int s = s0; s < s1; ++s) {
      const PassSeg &sg = segs[slot_segs[s]];
      acc += partials[(FULL ? sg.slot_full : sg.slot_ll) + o];
    }
    if (o < 2) gp.scal[base + o] = acc;
    else {
      gp.grad[o - 2] = acc;
      gmax = fmax(gmax, isfinite(acc) ? fabs(acc) : INFINITY);
    }
  }
  if (FULL) {
    for (int off = 16; off > 0; off >>= 1) gmax = fmax(gmax, __shfl_xor_sync(0xffffffffu, gmax, off));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = gmax;
    __syncthreads();
    if (threadIdx.x == 0) {
      double m = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
      gp.scal[kGsGinf] = m;
    }
  }
}

// Fixed-order float64 reduction of the CTA partials (rows of `stride` values,
// `grid` rows): a CTA takes 32 consecutive columns; warp w adds rows w, w + 8,
// ... with lanes over the columns (coalesced), two accumulators per lane, and
// the 8 warp sums are added in warp order.  Column 0, 1 -> scal[0], scal[1];
// column 2 + o -> grad[o].
__global__ void __launch_bounds__(256) pass_reduce_kernel(int64_t ncols, int64_t stride, int grid,
                                                          const double *__restrict__ part, double *__restrict__ scal,
                                                          double *__restrict__ grad) {
  __shared__ double red[8][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t col = (int64_t)blockIdx.x * 32 + lane;
  double s0 = 0.0, s1 = 0.0;
  if (col < ncols) {
    int g = warp;
    for (; g + 8 < grid; g += 16) {
      s0 += part[(int64_t)g * stride + col];
      s1 += part[(int64_t)(g + 8) * stride + col];
    }
    if (g < grid) s0 += part[(int64_t)g * stride + col];
  }
  red[warp][lane] = s0 + s1;
  __syncthreads();
  if (warp == 0 && col < ncols) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w][lane];
    if (col < 2) scal[col] = t;
    else grad[col - 2] = t;
  }
}

__global__ void validate_kernel(int64_t N, int K, int p, int d, int f, const float *X, const float *Y, const float *Z,
                                const int32_t *choice, int *status) {
  int bad = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (int64_t i = t0; i < N; i += stride) {
    const int c = choice[i];
    if (c < 0 || c >= K) bad |= 1;
  }
  for (int64_t e = t0; e < N * p; e += stride) if (!isfinite(X[e])) bad |= 2;
  if (Y) for (int64_t e = t0; e < N * K * d; e += stride) if (!isfinite(Y[e])) bad |= 2;
  if (Z) for (int64_t e = t0; e < N * K * f; e += stride) if (!isfinite(Z[e])) bad |= 2;
  if (bad) atomicOr(status, bad);
}

PassDims dims_of(const Shape &s, int rows) {
  PassDims D;
  D.N = s.N; D.K = s.K; D.p = s.p; D.d = s.d; D.f = s.f;
  D.nb = s.nb; D.ng = s.ng; D.mc = s.mc; D.nout = s.nout;
  D.rows = rows;
  D.ntiles = (s.N + rows - 1) / rows;
  return D;
}

size_t pass_smem(const Shape &s, int rows, size_t tsz, bool full) {
  size_t b = (((size_t)(s.p + s.d) * s.K + s.f) * tsz + 15) & ~(size_t)15;
  b += (((size_t)rows * (s.p + (size_t)s.K * s.d + (size_t)s.K * s.f)) * 4 + 15) & ~(size_t)15;
  if (full) b += (((size_t)rows * s.K) * tsz + 15) & ~(size_t)15;
  b += 32 * 4 * sizeof(double);
  return b;
}

template <typename T, bool FULL, int NPT>
cudaError_t launch_t(const PassDims &D, const PassPlan &pl, const PassIO &io, cudaStream_t st) {
  auto kern = pass_kernel<T, FULL, NPT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem);
  if (e != cudaSuccess) return e;
  kern<<<pl.grid, pl.block, pl.smem, st>>>(D, io);
  return cudaGetLastError();
}

template <typename T, bool FULL>
cudaError_t launch_npt(const PassDims &D, const PassPlan &pl, const PassIO &io, cudaStream_t st) {
  if (!FULL) return launch_t<T, false, 1>(D, pl, io, st);
  switch (pl.npt) {
    case 1: return launch_t<T, FULL, 1>(D, pl, io, st);
    case 2: return launch_t<T, FULL, 2>(D, pl, io, st);
    case 4: return launch_t<T, FULL, 4>(D, pl, io, st);
    case 8: return launch_t<T, FULL, 8>(D, pl, io, st);
    case 16: return launch_t<T, FULL, 16>(D, pl, io, st);
    case 24: return launch_t<T, FULL, 24>(D, pl, io, st);
    case 32: return launch_t<T, FULL, 32>(D, pl, io, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

PassPlan plan_pass(const Shape &s, bool fp64, bool full, int num_sms, bool allow_tiled) {
  PassPlan pl{};
  pl.ok = false;
  pl.tiled = false;
  if (!fp64 && allow_tiled && plan_pass_tiled(s, full, num_sms, pl)) return pl;
  if (s.K > 32 * kMaxClassSlots) return pl;
  const size_t tsz = fp64 ? 8 : 4;
  // threads: enough for the gradient accumulators at <= 32 per thread
  pl.block = 256;
  int need = (int)((s.nout + pl.block - 1) / pl.block);
  if (full && need > 16) { pl.block = 512; need = (int)((s.nout + pl.block - 1) / pl.block); }
  if (full) {
    static const int opts[] = {1, 2, 4, 8, 16, 24, 32};
    pl.npt = 0;
    for (int o : opts) if (o >= need) { pl.npt = o; break; }
    if (!pl.npt) return pl;
  } else {
    pl.npt = 1;
  }
  // rows per tile: the largest multiple of 4 (<= 32) whose tile fits ~100 KB (two CTAs per SM)
  const size_t budget = 100 * 1024, hard = 220 * 1024;
  int rows = 32;
  while (rows > 4 && pass_smem(s, rows, tsz, full) > budget) rows -= 4;
  if (pass_smem(s, rows, tsz, full) > hard) return pl;
  pl.rows = rows;
  pl.smem = pass_smem(s, rows, tsz, full);
  const int per_sm = (pl.smem <= budget && pl.block == 256) ? 2 : 1;
  const int64_t ntiles = (s.N + rows - 1) / rows;
  pl.grid = (int)std::min<int64_t>(ntiles, (int64_t)num_sms * per_sm);
  if (pl.grid < 1) pl.grid = 1;
  pl.ok = true;
  return pl;
}

cudaError_t launch_pass(const Shape &s, const PassPlan &pl, bool fp64, bool full, const PassIO &io, cudaStream_t st) {
  if (pl.tiled) return launch_pass_tiled(s, pl, full, io, st);
  const PassDims D = dims_of(s, pl.rows);
  if (fp64) return full ? launch_npt<double, true>(D, pl, io, st) : launch_npt<double, false>(D, pl, io, st);
  return full ? launch_npt<float, true>(D, pl, io, st) : launch_npt<float, false>(D, pl, io, st);
}

cudaError_t launch_pass_reduce(const Shape &s, int grid, bool full, const double *partials, double *scal,
                               double *grad, cudaStream_t st) {
  const int64_t stride = full ? 2 + s.n : 2;
  const int blocks = (int)((stride + 31) / 32);
  pass_reduce_kernel<<<blocks, 256, 0, st>>>(stride, stride, grid, partials, scal, grad);
  return cudaGetLastError();
}

template <typename T, bool FULL, int NPT>
cudaError_t launch_grouped_t(const GroupedPassPlan &pl, const GroupProblem *probs, const PassSeg *segs,
                             const int *seg_start, const int *active, double *partials, cudaStream_t st) {
  auto kern = grouped_pass_kernel<T, FULL, NPT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem);
  if (e != cudaSuccess) return e;
  kern<<<pl.grid, pl.block, pl.smem, st>>>(probs, segs, seg_start, active, pl.rows, partials);
  return cudaGetLastError();
}

template <typename T, bool FULL>
cudaError_t launch_grouped_npt(const GroupedPassPlan &pl, const GroupProblem *probs, const PassSeg *segs,
                               const int *seg_start, const int *active, double *partials, cudaStream_t st) {
  if (!FULL) return launch_grouped_t<T, false, 1>(pl, probs, segs, seg_start, active, partials, st);
  switch (pl.npt) {
    case 1: return launch_grouped_t<T, FULL, 1>(pl, probs, segs, seg_start, active, partials, st);
    case 2: return launch_grouped_t<T, FULL, 2>(pl, probs, segs, seg_start, active, partials, st);
    case 4: return launch_grouped_t<T, FULL, 4>(pl, probs, segs, seg_start, active, partials, st);
    case 8: return launch_grouped_t<T, FULL, 8>(pl, probs, segs, seg_start, active, partials, st);
    case 16: return launch_grouped_t<T, FULL, 16>(pl, probs, segs, seg_start, active, partials, st);
    case 24: return launch_grouped_t<T, FULL, 24>(pl, probs, segs, seg_start, active, partials, st);
    case 32: return launch_grouped_t<T, FULL, 32>(pl, probs, segs, seg_start, active, partials, st);
    default: return cudaErrorInvalidValue;
  }
}

__global__ void validate_weights_kernel(int64_t N, const float *__restrict__ w, int *status) {
  int bad = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const float v = w[i];
    if (!isfinite(v)) bad |= 2;
    else if (v < 0.f) bad |= 1;
  }
  if (bad) atomicOr(status, bad);
}

__global__ void augment_z_kernel(int64_t N, int K, int d, int f, const float *__restrict__ Y,
                                 const float *__restrict__ Z, float *__restrict__ Za) {
  const int fa = f + d;
  const int64_t total = N * K * fa;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ik = e / fa;
    const int j = (int)(e - ik * fa);
    const int64_t i = ik / K;
    const int k = (int)(ik - i * K);
    Za[e] = j < f ? Z[ik * f + j] : (k == 0 ? Y[i * K * d + (j - f)] : 0.f);
  }
}

__global__ void perm_kernel(int64_t n, const int64_t *__restrict__ perm, const double *__restrict__ in,
                            double *__restrict__ out, int to_user) {
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
    if (to_user) out[u] = in[perm[u]];
    else out[perm[u]] = in[u];
  }
}

__global__ void export_hessian_perm_kernel(int64_t n, const double *__restrict__ F, const int64_t *__restrict__ perm,
                                           double *__restrict__ H) {
  const int64_t v = blockIdx.y + (int64_t)gridDim.y * blockIdx.z;
  if (v >= n) return;
  const int64_t pv = perm[v];
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x)
    H[v * n + u] = -F[pv * n + perm[u]];
}

cudaError_t launch_augment_z(int64_t N, int K, int d, int f, const float *Y, const float *Z, float *Zaug,
                             cudaStream_t st) {
  const int64_t total = N * K * (f + d);
  const int64_t blocks = std::min<int64_t>((total + 255) / 256, 8192);
  augment_z_kernel<<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, st>>>(N, K, d, f, Y, Z, Zaug);
  return cudaGetLastError();
}

cudaError_t launch_perm_to_internal(int64_t n, const int64_t *perm, const double *user, double *internal,
                                    cudaStream_t st) {
  perm_kernel<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 1024)), 256, 0, st>>>(
      n, perm, user, internal, 0);
  return cudaGetLastError();
}

cudaError_t launch_perm_to_user(int64_t n, const int64_t *perm, const double *internal, double *user,
                                cudaStream_t st) {
  perm_kernel<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 1024)), 256, 0, st>>>(
      n, perm, internal, user, 1);
  return cudaGetLastError();
}

cudaError_t launch_export_hessian_perm(int64_t n, const double *F, const int64_t *perm, double *H, cudaStream_t st) {
  const dim3 grid((unsigned)std::min<int64_t>((n + 255) / 256, 64), (unsigned)std::min<int64_t>(n, 65535),
                  (unsigned)((n + 65534) / 65535));
  export_hessian_perm_kernel<<<grid, 256, 0, st>>>(n, F, perm, H);
  return cudaGetLastError();
}

cudaError_t launch_validate_weights(int64_t N, const float *w, int *status, cudaStream_t st) {
  validate_weights_kernel<<<1024, 256, 0, st>>>(N, w, status);
  return cudaGetLastError();
}

cudaError_t launch_validate(const Shape &s, const float *X, const float *Y, const float *Z, const int32_t *choice,
                            int *status, cudaStream_t st) {
  validate_kernel<<<1024, 256, 0, st>>>(s.N, s.K, s.p, s.d, s.f, X, s.d ? Y : nullptr, s.f ? Z : nullptr, choice,
                                        status);
  return cudaGetLastError();
}

}  // namespace mnl

namespace mnl {

GroupedPassPlan plan_grouped_pass(const std::vector<Shape> &shapes, bool fp64, int rows, int num_sms) {
  GroupedPassPlan pl{};
  pl.ok = false;
  int64_t max_nout = 0;
  size_t smem = 0;
  const size_t tsz = fp64 ? 8 : 4;
  for (const Shape &s : shapes) {
    if (s.K > 32 * kMaxClassSlots) return pl;
    max_nout = std::max<int64_t>(max_nout, s.nout);
    smem = std::max(smem, pass_smem(s, rows, tsz, true));
  }
  pl.block = 256;
  int need = (int)((max_nout + pl.block - 1) / pl.block);
  if (need > 16) { pl.block = 512; need = (int)((max_nout + pl.block - 1) / pl.block); }
  static const int opts[] = {1, 2, 4, 8, 16, 24, 32};
  pl.npt = 0;
  for (int o : opts) if (o >= need) { pl.npt = o; break; }
  if (!pl.npt || smem > 220 * 1024) return pl;
  pl.rows = rows;
  pl.smem = smem;
  // as many CTAs per SM as shared memory and threads allow (latency hiding for the staged tiles)
  const int per_sm = std::max(1, std::min<int>(2048 / pl.block, (int)((227 * 1024) / (smem + 1024))));
  pl.grid = num_sms * per_sm;
  pl.ok = true;
  return pl;
}

cudaError_t launch_grouped_pass(const GroupedPassPlan &pl, bool fp64, bool full, const GroupProblem *probs,
                                const PassSeg *segs, const int *seg_start, const int *active, double *partials,
                                cudaStream_t st) {
  if (fp64)
    return full ? launch_grouped_npt<double, true>(pl, probs, segs, seg_start, active, partials, st)
                : launch_grouped_npt<double, false>(pl, probs, segs, seg_start, active, partials, st);
  return full ? launch_grouped_npt<float, true>(pl, probs, segs, seg_start, active, partials, st)
              : launch_grouped_npt<float, false>(pl, probs, segs, seg_start, active, partials, st);
}

cudaError_t launch_grouped_reduce(int nprob, bool full, const GroupProblem *probs, const int *slot_start,
                                  const PassSeg *segs, const int *slot_segs, const int *active,
                                  const double *partials, int base, cudaStream_t st) {
  if (full)
    grouped_reduce_kernel<true><<<nprob, 128, 0, st>>>(probs, slot_start, segs, slot_segs, active, partials, base);
  else
    grouped_reduce_kernel<false><<<nprob, 128, 0, st>>>(probs, slot_start, segs, slot_segs, active, partials, base);
  return cudaGetLastError();
}

}  // namespace mnl
