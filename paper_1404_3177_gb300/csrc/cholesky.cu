// Newton solve pieces outside the cooperative factorisation (solve_coop.cu):
//
// FP64 triangular solves with a factor from launch_cholesky: forward and back
// substitution by blocks of kNb unknowns, each block one small kernel (one
// warp, the diagonal block in shared memory) and one update kernel spread over
// many CTAs.
//
// Batched solves: one CTA factors and solves one problem (n up to a few
// thousand) for the grouped Newton phases.
//
// Small float64 vector kernels of the Newton update.
#include "mnl_internal.cuh"

namespace mnl {
namespace {

constexpr int kNb = 64;

// ---------------------------------------------------------------------------
// FP64 solve by blocks of kNb unknowns.
// ---------------------------------------------------------------------------

// One warp: x[b0..b0+w) = L_bb^{-1} x (forward) or L_bb^{-T} x (backward), in place.
template <bool FWD>
__global__ void __launch_bounds__(32) solve_diag_kernel(const double *__restrict__ L, const double *__restrict__ dinv,
                                                        int64_t n, int64_t b0, double *__restrict__ x,
                                                        const int *__restrict__ status) {
  __shared__ double Ld[kNb][kNb + 1];
  __shared__ double di[kNb];
  if (*status & 4) return;
  const int lane = threadIdx.x;
  const int w = (int)min((int64_t)kNb, n - b0);
  for (int e = lane; e < kNb * kNb; e += 32) {
    const int r = e % kNb, c = e / kNb;
    Ld[r][c] = (r < w && c < w && r >= c) ? L[(b0 + c) * n + b0 + r] : 0.0;
  }
  for (int c = lane; c < kNb; c += 32) di[c] = c < w ? dinv[b0 + c] : 0.0;
  __syncwarp();
  double v0 = lane < w ? x[b0 + lane] : 0.0, v1 = lane + 32 < w ? x[b0 + lane + 32] : 0.0;
  if (FWD) {
    for (int c = 0; c < w; ++c) {
      const double src = c < 32 ? v0 : v1;
      double xc = __shfl_sync(0xffffffffu, src, c & 31) * di[c];
      if (lane == (c & 31)) { if (c < 32) v0 = xc; else v1 = xc; }
      if (lane > c) v0 = fma(-Ld[lane][c], xc, v0);
      if (lane + 32 > c) v1 = fma(-Ld[lane + 32][c], xc, v1);
    }
  } else {
    for (int c = w - 1; c >= 0; --c) {
      const double src = c < 32 ? v0 : v1;
      double xc = __shfl_sync(0xffffffffu, src, c & 31) * di[c];
      if (lane == (c & 31)) { if (c < 32) v0 = xc; else v1 = xc; }
      if (lane < c) v0 = fma(-Ld[c][lane], xc, v0);
      if (lane + 32 < c) v1 = fma(-Ld[c][lane + 32], xc, v1);
    }
  }
  if (lane < w) x[b0 + lane] = v0;
  if (lane + 32 < w) x[b0 + lane + 32] = v1;
}

// Forward update: rows r >= b0 + kNb: x_r -= sum_c L[r][b0 + c] x_{b0+c} (thread per row).
__global__ void __launch_bounds__(64) solve_update_fwd_kernel(const double *__restrict__ L, int64_t n, int64_t b0,
                                                              double *__restrict__ x, const int *__restrict__ status) {
  __shared__ double xb[kNb];
  if (*status & 4) return;
  if (threadIdx.x < kNb) xb[threadIdx.x] = x[b0 + threadIdx.x];
  __syncthreads();
  const int64_t r = b0 + kNb + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  double s0 = 0.0, s1 = 0.0;
#pragma unroll 8
  for (int c = 0; c < kNb; c += 2) {
    s0 = fma(L[(b0 + c) * n + r], xb[c], s0);
    s1 = fma(L[(b0 + c + 1) * n + r], xb[c + 1], s1);
  }
  x[r] -= s0 + s1;
}

// Backward update: rows r < b0: x_r -= sum_c L[b0 + c][r] x_{b0+c} (warp per row, contiguous reads).
__global__ void __launch_bounds__(256) solve_update_bwd_kernel(const double *__restrict__ L, int64_t n, int64_t b0,
                                                               double *__restrict__ x, const int *__restrict__ status) {
  __shared__ double xb[kNb];
  if (*status & 4) return;
  const int w = (int)min((int64_t)kNb, n - b0);
  if (threadIdx.x < kNb) xb[threadIdx.x] = threadIdx.x < w ? x[b0 + threadIdx.x] : 0.0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= b0) return;
  double t = 0.0;
  if (lane < w) t = L[r * n + b0 + lane] * xb[lane];
  if (lane + 32 < w) t = fma(L[r * n + b0 + lane + 32], xb[lane + 32], t);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if (lane == 0) x[r] -= t;
}

__global__ void copy_or_zero_kernel(int64_t n, const double *b, double *x, const int *status, int bad_mask) {
  const bool bad = (*status & bad_mask) != 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = bad ? 0.0 : b[i];
}

__device__ __forceinline__ void atomic_max_nonneg(double *addr, double v) {
  // non-negative doubles order like their bit patterns
  atomicMax(reinterpret_cast<unsigned long long *>(addr), (unsigned long long)__double_as_longlong(v));
}

// theta += t * delta; scal_out[0] = max|t delta|, scal_out[1] = max|theta| (after).
__global__ void axpy_theta_kernel(int64_t n, double *theta, const double *delta, const double *tscale,
                                  double *scal_out) {
  const double t = *tscale;
  double m1 = 0.0, m2 = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double st = t * delta[i];
    const double th = theta[i] + st;
    theta[i] = th;
    m1 = fmax(m1, fabs(st));
    m2 = fmax(m2, fabs(th));
  }
  for (int o = 16; o > 0; o >>= 1) {
    m1 = fmax(m1, __shfl_xor_sync(0xffffffffu, m1, o));
    m2 = fmax(m2, __shfl_xor_sync(0xffffffffu, m2, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomic_max_nonneg(scal_out, m1);
    atomic_max_nonneg(scal_out + 1, m2);
  }
}

// The full Newton step theta += delta, applied when it is acceptable as the
// first trial of the step halving (Sec. 3.1): l(theta + delta) >= l0 - u8 * labs
// (u8 * labs: the noise level of the float sums), the factorisation and solve
// succeeded (status bits 4, 8, 16 clear) and no wait timed out.  Sets status
// bit 32 when applied; scal_out as axpy_theta_kernel.
__global__ void try_full_step_kernel(int64_t n, double *theta, const double *delta, const double *l0,
                                     const double *labs, const double *lt, int *status, const int *err, double u8,
                                     double *scal_out) {
  const double a = *l0, b = *lt;
  const bool ok = (*status & (4 | 8 | 16)) == 0 && *err == 0 && isfinite(a) && isfinite(b) && b >= a - u8 * *labs;
  if (!ok) return;
  double m1 = 0.0, m2 = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double st = delta[i];
    const double th = theta[i] + st;
    theta[i] = th;
    m1 = fmax(m1, fabs(st));
    m2 = fmax(m2, fabs(th));
  }
  for (int o = 16; o > 0; o >>= 1) {
    m1 = fmax(m1, __shfl_xor_sync(0xffffffffu, m1, o));
    m2 = fmax(m2, __shfl_xor_sync(0xffffffffu, m2, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomic_max_nonneg(scal_out, m1);
    atomic_max_nonneg(scal_out + 1, m2);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(status, 32);
}

__global__ void vec_absmax_kernel(int64_t n, const double *v, double *out) {
  double m = 0.0;
  bool nonfinite = false;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double a = fabs(v[i]);
    if (!isfinite(a)) nonfinite = true;
    else m = fmax(m, a);
  }
  if (nonfinite) m = __longlong_as_double(0x7ff0000000000000LL);  // +inf flags a non-finite entry
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomic_max_nonneg(out, m);
}

// ---------------------------------------------------------------------------
// Batched solves: one CTA factors and solves one problem (n up to a few
// thousand).  Right-looking Cholesky by panels of W columns: the panel rows
// are staged in shared memory, warp 0 factors the W x W diagonal block, every
// thread solves one panel row against it, and the trailing lower triangle
// takes the rank-W update in 4 x 4 register blocks.  L^T is written to the
// upper triangle so both triangular solves read contiguous columns.
// ---------------------------------------------------------------------------

constexpr int kCtaThreads = 256;

template <typename T, int W>
__device__ bool cta_cholesky(T *__restrict__ A, int64_t n, T *__restrict__ Ps, T *__restrict__ dinv) {
  constexpr int PS = W + 1;  // panel row stride: rows of the panel fall in different banks
  __shared__ int bad;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) bad = 0;
  for (int64_t j0 = 0; j0 < n; j0 += W) {
    const int nb = (int)min((int64_t)W, n - j0);
    const int64_t m = n - j0;  // panel rows
    __syncthreads();
    for (int64_t e = tid; e < m * nb; e += blockDim.x) {
      const int k = (int)(e / m);
      const int64_t rr = e % m;
      Ps[rr * PS + k] = A[(j0 + k) * n + j0 + rr];
    }
    __syncthreads();
    if (warp == 0) {  // diagonal block, lane = row
      for (int c = 0; c < nb; ++c) {
        T lcc = (T)1;
        if (lane == c) {
          const T piv = Ps[c * PS + c];
          if (!(piv > (T)0) || !isfinite(piv)) bad = 1;
          else lcc = sqrt(piv);
          Ps[c * PS + c] = lcc;
          dinv[c] = (T)1 / lcc;
        }
        __syncwarp();
        const T ri = dinv[c];
        if (lane > c && lane < nb) Ps[lane * PS + c] *= ri;
        __syncwarp();
        if (lane > c && lane < nb) {
          const T lrc = Ps[lane * PS + c];
          for (int cc = c + 1; cc <= lane; ++cc) Ps[lane * PS + cc] -= lrc * Ps[cc * PS + c];
        }
        __syncwarp();
      }
    }
    __syncthreads();
    for (int64_t rr = nb + tid; rr < m; rr += blockDim.x) {  // rows below: solve against the block
      T x[W];
#pragma unroll
      for (int c = 0; c < W; ++c) x[c] = c < nb ? Ps[rr * PS + c] : (T)0;
#pragma unroll
      for (int c = 0; c < W; ++c) {
        if (c < nb) {
          T v = x[c];
#pragma unroll
          for (int t = 0; t < c; ++t) v -= x[t] * Ps[c * PS + t];
          x[c] = v * dinv[c];
        }
      }
#pragma unroll
      for (int c = 0; c < W; ++c)
        if (c < nb) Ps[rr * PS + c] = x[c];
    }
    __syncthreads();
    // panel back to A: L (lower) and L^T (upper)
    for (int64_t e = tid; e < m * nb; e += blockDim.x) {
      const int k = (int)(e / m);
      const int64_t rr = e % m;
      if (rr >= k) {
        const T v = Ps[rr * PS + k];
        A[(j0 + k) * n + j0 + rr] = v;
        A[(j0 + rr) * n + j0 + k] = v;
      }
    }
    // trailing update in 4 x 4 blocks: A[r][c] -= sum_k L[r][k] L[c][k], c <= r
    const int64_t mt = m - nb;
    const int64_t nb4 = (mt + 3) / 4;
    const int64_t nblk = nb4 * (nb4 + 1) / 2;
    for (int64_t t = tid; t < nblk; t += blockDim.x) {
      int64_t bi = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
      while ((bi + 1) * (bi + 2) / 2 <= t) ++bi;
      while (bi * (bi + 1) / 2 > t) --bi;
      const int64_t bj = t - bi * (bi + 1) / 2;
      T acc[4][4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = (T)0;
      const int64_t r0 = nb + bi * 4, c0 = nb + bj * 4;
      for (int k = 0; k < nb; ++k) {
        T a[4], b[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          a[u] = r0 + u < m ? Ps[(r0 + u) * PS + k] : (T)0;
          b[u] = c0 + u < m ? Ps[(c0 + u) * PS + k] : (T)0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[u][v] += a[u] * b[v];
      }
      // the 16 old values are loaded before any store (no load waits on a possibly aliasing store)
      T old[4][4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const int64_t r = r0 + u, c = c0 + v;
          old[u][v] = (r < m && c < m && r >= c) ? A[(j0 + c) * n + j0 + r] : (T)0;
        }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const int64_t r = r0 + u, c = c0 + v;
          if (r < m && c < m && r >= c) A[(j0 + c) * n + j0 + r] = old[u][v] - acc[u][v];
        }
    }
    __syncthreads();
    if (bad) return false;
  }
  __syncthreads();
  return bad == 0;
}

// x <- (L L^T)^{-1} x for a factor with L^T in the upper triangle; x in shared
// memory.  Blocks of 32 unknowns: warp 0 solves the diagonal block (lane = row,
// the block's pivots broadcast by shuffles), then every thread updates the
// unknowns below (forward) or above (backward) from the block's 32 columns,
// which are contiguous in the stored factor (L below the diagonal for the
// forward sweep, L^T above it for the backward one).
template <typename T, typename V>
__device__ void cta_chol_solve(const T *__restrict__ A, int64_t n, V *__restrict__ x) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t nblk = (n + 31) / 32;
  for (int64_t bb = 0; bb < nblk; ++bb) {  // forward: L y = x
    const int64_t b0 = bb * 32;
    const int w = (int)(n - b0 < 32 ? n - b0 : 32);
    __syncthreads();
    if (warp == 0) {
      V v = lane < w ? x[b0 + lane] : (V)0;
      for (int c = 0; c < w; ++c) {
        const V xc = __shfl_sync(0xffffffffu, v, c) / (V)A[(b0 + c) * n + b0 + c];
        if (lane == c) v = xc;
        else if (lane > c && lane < w) v -= (V)A[(b0 + c) * n + b0 + lane] * xc;
      }
      if (lane < w) x[b0 + lane] = v;
    }
    __syncthreads();
    for (int64_t r = b0 + w + tid; r < n; r += blockDim.x) {
      V s0 = (V)0, s1 = (V)0;
      int c = 0;
      for (; c + 1 < w; c += 2) {
        s0 += (V)A[(b0 + c) * n + r] * x[b0 + c];
        s1 += (V)A[(b0 + c + 1) * n + r] * x[b0 + c + 1];
      }
      if (c < w) s0 += (V)A[(b0 + c) * n + r] * x[b0 + c];
      x[r] -= s0 + s1;
    }
  }
  for (int64_t bb = nblk - 1; bb >= 0; --bb) {  // backward: L^T z = y
    const int64_t b0 = bb * 32;
    const int w = (int)(n - b0 < 32 ? n - b0 : 32);
    __syncthreads();
    if (warp == 0) {
      V v = lane < w ? x[b0 + lane] : (V)0;
      for (int c = w - 1; c >= 0; --c) {
        const V xc = __shfl_sync(0xffffffffu, v, c) / (V)A[(b0 + c) * n + b0 + c];
        if (lane == c) v = xc;
        else if (lane < c) v -= (V)A[(b0 + c) * n + b0 + lane] * xc;  // (L^T)(b0+lane, b0+c), above the diagonal
      }
      if (lane < w) x[b0 + lane] = v;
    }
    __syncthreads();
    for (int64_t r = tid; r < b0; r += blockDim.x) {
      V s0 = (V)0, s1 = (V)0;
      int c = 0;
      for (; c + 1 < w; c += 2) {
        s0 += (V)A[(b0 + c) * n + r] * x[b0 + c];
        s1 += (V)A[(b0 + c + 1) * n + r] * x[b0 + c + 1];
      }
      if (c < w) s0 += (V)A[(b0 + c) * n + r] * x[b0 + c];
      x[r] -= s0 + s1;
    }
  }
  __syncthreads();
}

__device__ double cta_max_abs(const double *v, int64_t n, double *red) {
  double m = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, fabs(v[i]));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  double r = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = fmax(r, red[w]);
  __syncthreads();
  return r;
}

// One CTA per active problem: delta = F^{-1} g.  MIXED: float32 factor +
// float64 refinement (stops as in the single-problem mixed solve), falling back
// to a float64 factor in the same CTA; else float64 factor.  Sets
// status[b] = MNL_ERR_NOT_PD when -H is not positive definite.
template <bool MIXED>
__global__ void __launch_bounds__(kCtaThreads) grouped_chol_solve_kernel(const GroupProblem *__restrict__ probs,
                                                                         const int *__restrict__ plist,
                                                                         const int *__restrict__ active, int iters,
                                                                         int *__restrict__ status, int64_t max_n) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[32];
  __shared__ float dinv32[32];
  __shared__ double dinv64[16];
  const int b = plist[blockIdx.x];
  if (active[b] == 0) return;
  const GroupProblem &g = probs[b];
  const int64_t n = g.n;
  if (n > max_n) return;  // solved by the multi-CTA path
  double *xs = reinterpret_cast<double *>(smem);  // [n] solution work vector
  double *ds = xs + n;                            // [n] correction
  unsigned char *panel = smem + (((size_t)2 * n * sizeof(double) + 15) & ~(size_t)15);
  bool done = false;
  if (MIXED) {
    for (int64_t e = threadIdx.x; e < n * n; e += blockDim.x) g.F32[e] = (float)g.F[e];
    __syncthreads();
    if (cta_cholesky<float, 32>(g.F32, n, reinterpret_cast<float *>(panel), dinv32)) {
      for (int64_t i = threadIdx.x; i < n; i += blockDim.x) xs[i] = g.grad[i];
      cta_chol_solve<float, double>(g.F32, n, xs);
      for (int64_t i = threadIdx.x; i < n; i += blockDim.x) g.delta[i] = xs[i];
      double prev = cta_max_abs(xs, n, red);
      int steps = 0;
      bool ok = false;
      for (int it = 0; it < iters; ++it) {
        __syncthreads();
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {  // r = g - F delta (float64)
          double sacc = 0.0;
          for (int64_t j = 0; j < n; ++j) sacc = fma(g.F[j * n + i], g.delta[j], sacc);
          ds[i] = g.grad[i] - sacc;
        }
        cta_chol_solve<float, double>(g.F32, n, ds);
        const double dn = cta_max_abs(ds, n, red);
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) xs[i] = g.delta[i] + ds[i];
        const double xn = cta_max_abs(xs, n, red);
        ++steps;
        const bool improving = dn < 0.5 * prev;
        if (improving || dn <= 1e-12 * xn)
          for (int64_t i = threadIdx.x; i < n; i += blockDim.x) g.delta[i] = xs[i];
        __syncthreads();
        if (dn <= 1e-12 * xn) { ok = true; break; }
        if (!improving) { ok = dn <= 1e-8 * xn; break; }
        prev = dn;
      }
      if (threadIdx.x == 0) g.scal[kGsRefine] = steps;
      done = ok;
    }
    __syncthreads();
  }
  if (!done) {  // float64 factor (and the fallback of the mixed solve)
    if (!cta_cholesky<double, 16>(g.F, n, reinterpret_cast<double *>(panel), dinv64)) {
      if (threadIdx.x == 0) status[b] = MNL_ERR_NOT_PD;
      return;
    }
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) xs[i] = g.grad[i];
    cta_chol_solve<double, double>(g.F, n, xs);
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) g.delta[i] = xs[i];
  }
}

}  // namespace

cudaError_t launch_cholesky_solve(int64_t n, const double *L, const double *dinv, const double *b, double *x,
                                  const int *status, cudaStream_t st, int *launches) {
  copy_or_zero_kernel<<<64, 256, 0, st>>>(n, b, x, status, 4);
  int cnt = 1;
  const int64_t nblk = (n + kNb - 1) / kNb;
  for (int64_t bb = 0; bb < nblk; ++bb) {
    const int64_t b0 = bb * kNb;
    solve_diag_kernel<true><<<1, 32, 0, st>>>(L, dinv, n, b0, x, status);
    ++cnt;
    if (b0 + kNb < n) {
      solve_update_fwd_kernel<<<(unsigned)((n - b0 - kNb + 63) / 64), 64, 0, st>>>(L, n, b0, x, status);
      ++cnt;
    }
  }
  for (int64_t bb = nblk - 1; bb >= 0; --bb) {
    const int64_t b0 = bb * kNb;
    solve_diag_kernel<false><<<1, 32, 0, st>>>(L, dinv, n, b0, x, status);
    ++cnt;
    if (b0 > 0) {
      solve_update_bwd_kernel<<<(unsigned)((b0 + 7) / 8), 256, 0, st>>>(L, n, b0, x, status);
      ++cnt;
    }
  }
  if (launches) *launches = cnt;
  return cudaGetLastError();
}

cudaError_t launch_axpy_theta(int64_t n, double *theta, const double *delta, const double *tscale, double *scal_out,
                              cudaStream_t st) {
  const int blocks = (int)std::min<int64_t>(64, (n + 255) / 256);
  axpy_theta_kernel<<<blocks < 1 ? 1 : blocks, 256, 0, st>>>(n, theta, delta, tscale, scal_out);
  return cudaGetLastError();
}

cudaError_t launch_try_full_step(int64_t n, double *theta, const double *delta, const double *l0, const double *labs,
                                 const double *lt, int *status, const int *err, double u8, double *scal_out,
                                 cudaStream_t st) {
  const int blocks = (int)std::min<int64_t>(64, (n + 255) / 256);
  try_full_step_kernel<<<blocks < 1 ? 1 : blocks, 256, 0, st>>>(n, theta, delta, l0, labs, lt, status, err, u8,
                                                                 scal_out);
  return cudaGetLastError();
}

namespace {
// out[0] = a . b in a fixed order (one CTA: strided partial sums, then a tree over the threads).
__global__ void __launch_bounds__(1024) dot_kernel(int64_t n, const double *__restrict__ a,
                                                   const double *__restrict__ b, double *__restrict__ out) {
  __shared__ double red[1024];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s = fma(a[i], b[i], s);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = red[0];
}

// y = a x + b y
__global__ void axpby_kernel(int64_t n, double a, const double *__restrict__ x, double b, double *__restrict__ y) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = b == 0.0 ? a * x[i] : fma(a, x[i], b * y[i]);  // b = 0: y's old value is not read
}
}  // namespace

cudaError_t launch_dot(int64_t n, const double *a, const double *b, double *out, cudaStream_t st) {
  dot_kernel<<<1, 1024, 0, st>>>(n, a, b, out);
  return cudaGetLastError();
}

cudaError_t launch_axpby(int64_t n, double a, const double *x, double b, double *y, cudaStream_t st) {
  const int blocks = (int)std::min<int64_t>(256, (n + 255) / 256);
  axpby_kernel<<<blocks < 1 ? 1 : blocks, 256, 0, st>>>(n, a, x, b, y);
  return cudaGetLastError();
}

cudaError_t launch_vec_absmax(int64_t n, const double *v, double *out, cudaStream_t st) {
  const int blocks = (int)std::min<int64_t>(64, (n + 255) / 256);
  vec_absmax_kernel<<<blocks < 1 ? 1 : blocks, 256, 0, st>>>(n, v, out);
  return cudaGetLastError();
}

}  // namespace mnl

namespace mnl {

size_t grouped_chol_smem(int64_t nmax) {
  const size_t vec = (((size_t)2 * nmax * sizeof(double) + 15) & ~(size_t)15);
  const size_t p32 = (size_t)nmax * 33 * sizeof(float), p64 = (size_t)nmax * 17 * sizeof(double);
  return vec + std::max(p32, p64);
}

cudaError_t launch_grouped_chol_solve(bool mixed, const GroupProblem *probs, const int *plist, int nprob,
                                      const int *active, int iters, int *status, size_t smem, int64_t max_n,
                                      cudaStream_t st) {
  if (nprob <= 0) return cudaSuccess;
  cudaError_t e;
  if (mixed) {
    if ((e = cudaFuncSetAttribute(grouped_chol_solve_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem)))
      return e;
    grouped_chol_solve_kernel<true><<<nprob, kCtaThreads, smem, st>>>(probs, plist, active, iters, status, max_n);
  } else {
    if ((e = cudaFuncSetAttribute(grouped_chol_solve_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem)))
      return e;
    grouped_chol_solve_kernel<false><<<nprob, kCtaThreads, smem, st>>>(probs, plist, active, iters, status, max_n);
  }
  return cudaGetLastError();
}

}  // namespace mnl
