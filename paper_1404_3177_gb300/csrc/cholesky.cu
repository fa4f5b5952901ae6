// FP64 Newton solve (eq. "NR update"): F = -H = L L^T by a blocked
// right-looking Cholesky factorisation, then L L^T delta = g by forward and
// back substitution.  F is column-major with leading dimension n; only the
// lower triangle is read or written.
//
// Per panel of kNb columns: (1) one CTA factors the diagonal block in shared
// memory and checks every pivot (> 0 and finite), (2) one thread per row below
// solves its row of L21 against L11, (3) 64 x 64 tiles of the trailing lower
// triangle take the rank-kNb update F22 -= L21 L21^T.
#include "mnl_internal.cuh"

namespace mnl {
namespace {

constexpr int kNb = 64;

__global__ void __launch_bounds__(256) potrf_diag_kernel(double *F, int64_t n, int64_t j0, int *status) {
  __shared__ double A[kNb][kNb + 1];
  __shared__ int bad;
  const int nb = (int)min((int64_t)kNb, n - j0);
  const int tid = threadIdx.x;
  if (tid == 0) bad = (*status & 4) ? 1 : 0;
  for (int e = tid; e < nb * nb; e += blockDim.x) {
    const int c = e / nb, r = e % nb;
    A[r][c] = r >= c ? F[(j0 + c) * n + j0 + r] : 0.0;
  }
  __syncthreads();
  for (int c = 0; c < nb; ++c) {
    if (tid == 0) {
      const double piv = A[c][c];
      if (!(piv > 0.0) || !isfinite(piv)) { bad = 1; A[c][c] = 1.0; }
      else A[c][c] = sqrt(piv);
    }
    __syncthreads();
    const double lcc = A[c][c];
    for (int r = c + 1 + tid; r < nb; r += blockDim.x) A[r][c] /= lcc;
    __syncthreads();
    // trailing update of the block: A[r][cc] -= A[r][c] A[cc][c], c < cc <= r
    const int m = nb - c - 1;
    for (int e = tid; e < m * m; e += blockDim.x) {
      const int rr = c + 1 + e / m, cc = c + 1 + e % m;
      if (rr >= cc) A[rr][cc] -= A[rr][c] * A[cc][c];
    }
    __syncthreads();
  }
  for (int e = tid; e < nb * nb; e += blockDim.x) {
    const int c = e / nb, r = e % nb;
    if (r >= c) F[(j0 + c) * n + j0 + r] = A[r][c];
  }
  if (tid == 0 && bad) atomicOr(status, 4);
}

// Rows r >= j0 + nb: L21[r][:] = A21[r][:] L11^{-T}  (forward substitution per row).
__global__ void __launch_bounds__(128) trsm_panel_kernel(double *F, int64_t n, int64_t j0) {
  __shared__ double L[kNb][kNb + 1];
  const int nb = kNb;  // only launched for full panels
  const int tid = threadIdx.x;
  for (int e = tid; e < nb * nb; e += blockDim.x) {
    const int c = e / nb, r = e % nb;
    L[r][c] = r >= c ? F[(j0 + c) * n + j0 + r] : 0.0;
  }
  __syncthreads();
  const int64_t r = j0 + nb + (int64_t)blockIdx.x * blockDim.x + tid;
  if (r >= n) return;
  double x[kNb];
#pragma unroll
  for (int c = 0; c < kNb; ++c) x[c] = F[(j0 + c) * n + r];
#pragma unroll
  for (int c = 0; c < kNb; ++c) {
    double v = x[c];
#pragma unroll
    for (int t = 0; t < c; ++t) v = fma(-x[t], L[c][t], v);
    x[c] = v / L[c][c];
  }
#pragma unroll
  for (int c = 0; c < kNb; ++c) F[(j0 + c) * n + r] = x[c];
}

// Trailing update, tile (bi, bj), bi >= bj, of the rows/columns >= j1 = j0 + kNb.
__global__ void __launch_bounds__(256) syrk_update_kernel(double *F, int64_t n, int64_t j0) {
  __shared__ double Ar[kNb][65];
  __shared__ double Ac[kNb][65];
  const int64_t j1 = j0 + kNb;
  const int64_t t = blockIdx.x;
  int64_t bi = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while ((bi + 1) * (bi + 2) / 2 <= t) ++bi;
  while (bi * (bi + 1) / 2 > t) --bi;
  const int64_t bj = t - bi * (bi + 1) / 2;
  const int64_t r0 = j1 + bi * 64, c0 = j1 + bj * 64;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  for (int e = tid; e < 64 * kNb; e += blockDim.x) {
    const int kk = e / 64, rr = e % 64;
    Ar[kk][rr] = (r0 + rr < n) ? F[(j0 + kk) * n + r0 + rr] : 0.0;
    Ac[kk][rr] = (c0 + rr < n) ? F[(j0 + kk) * n + c0 + rr] : 0.0;
  }
  __syncthreads();
  double acc[4][4] = {};
#pragma unroll 8
  for (int kk = 0; kk < kNb; ++kk) {
    double a[4], b[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) a[v] = Ar[kk][ty + 16 * v];
#pragma unroll
    for (int u = 0; u < 4; ++u) b[u] = Ac[kk][tx + 16 * u];
#pragma unroll
    for (int v = 0; v < 4; ++v)
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[v][u] = fma(a[v], b[u], acc[v][u]);
  }
#pragma unroll
  for (int v = 0; v < 4; ++v)
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t r = r0 + ty + 16 * v, c = c0 + tx + 16 * u;
      if (r < n && c < n && r >= c) F[c * n + r] -= acc[v][u];
    }
}

// Forward and back substitution in one CTA, 32 unknowns per step.
__global__ void __launch_bounds__(1024) cholesky_solve_kernel(int64_t n, const double *__restrict__ L,
                                                              const double *__restrict__ b, double *__restrict__ x,
                                                              const int *__restrict__ status) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (*status & 4) {
    for (int64_t i = tid; i < n; i += blockDim.x) x[i] = 0.0;
    return;
  }
  for (int64_t i = tid; i < n; i += blockDim.x) x[i] = b[i];
  __syncthreads();
  // L y = b
  for (int64_t b0 = 0; b0 < n; b0 += 32) {
    const int w = (int)min((int64_t)32, n - b0);
    if (warp == 0) {
      double v = lane < w ? x[b0 + lane] : 0.0;
      for (int c = 0; c < w; ++c) {
        if (lane == c) v /= L[(b0 + c) * n + b0 + c];
        const double xc = __shfl_sync(0xffffffffu, v, c);
        if (lane > c && lane < w) v = fma(-L[(b0 + c) * n + b0 + lane], xc, v);
      }
      if (lane < w) x[b0 + lane] = v;
    }
    __syncthreads();
    for (int64_t r = b0 + w + tid; r < n; r += blockDim.x) {
      double s = 0.0;
      for (int c = 0; c < w; ++c) s = fma(L[(b0 + c) * n + r], x[b0 + c], s);
      x[r] -= s;
    }
    __syncthreads();
  }
  // L^T x = y
  const int64_t nblk = (n + 31) / 32;
  for (int64_t bb = nblk - 1; bb >= 0; --bb) {
    const int64_t b0 = bb * 32;
    const int w = (int)min((int64_t)32, n - b0);
    if (warp == 0) {
      double v = lane < w ? x[b0 + lane] : 0.0;
      for (int c = w - 1; c >= 0; --c) {
        if (lane == c) v /= L[(b0 + c) * n + b0 + c];
        const double xc = __shfl_sync(0xffffffffu, v, c);
        // row c of L^T, column lane < c: L[c][lane] = L[(b0+lane)*n + b0+c]
        if (lane < c) v = fma(-L[(b0 + lane) * n + b0 + c], xc, v);
      }
      if (lane < w) x[b0 + lane] = v;
    }
    __syncthreads();
    for (int64_t r = tid; r < b0; r += blockDim.x) {
      double s = 0.0;
      for (int c = 0; c < w; ++c) s = fma(L[r * n + b0 + c], x[b0 + c], s);
      x[r] -= s;
    }
    __syncthreads();
  }
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

}  // namespace

cudaError_t launch_cholesky(int64_t n, double *F, int *status, cudaStream_t st) {
  for (int64_t j0 = 0; j0 < n; j0 += kNb) {
    potrf_diag_kernel<<<1, 256, 0, st>>>(F, n, j0, status);
    const int64_t j1 = j0 + kNb;
    if (j1 >= n) break;
    const int64_t rows = n - j1;
    trsm_panel_kernel<<<(unsigned)((rows + 127) / 128), 128, 0, st>>>(F, n, j0);
    const int64_t T = (rows + 63) / 64;
    syrk_update_kernel<<<(unsigned)(T * (T + 1) / 2), 256, 0, st>>>(F, n, j0);
  }
  return cudaGetLastError();
}

cudaError_t launch_cholesky_solve(int64_t n, const double *L, const double *b, double *x, const int *status,
                                  cudaStream_t st) {
  cholesky_solve_kernel<<<1, 1024, 0, st>>>(n, L, b, x, status);
  return cudaGetLastError();
}

cudaError_t launch_axpy_theta(int64_t n, double *theta, const double *delta, const double *tscale, double *scal_out,
                              cudaStream_t st) {
  const int blocks = (int)std::min<int64_t>(64, (n + 255) / 256);
  axpy_theta_kernel<<<blocks < 1 ? 1 : blocks, 256, 0, st>>>(n, theta, delta, tscale, scal_out);
  return cudaGetLastError();
}

cudaError_t launch_vec_absmax(int64_t n, const double *v, double *out, cudaStream_t st) {
  const int blocks = (int)std::min<int64_t>(64, (n + 255) / 256);
  vec_absmax_kernel<<<blocks < 1 ? 1 : blocks, 256, 0, st>>>(n, v, out);
  return cudaGetLastError();
}

}  // namespace mnl
