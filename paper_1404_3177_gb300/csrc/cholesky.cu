// Newton solve (eq. "NR update"):  F delta = g  with F = -H symmetric positive
// definite, stored column-major with leading dimension n (both triangles are
// filled by the assembly; factorisations use and overwrite the lower one).
//
// Blocked right-looking Cholesky F = L L^T, per panel of kNb columns:
//   (1) one CTA factors the diagonal block in shared memory, checks every
//       pivot (> 0 and finite) and records 1/L_jj,
//   (2) thin CTAs (32 rows each, so the work spreads over many SMs) solve the
//       rows below against L11 by forward substitution with those reciprocals,
//   (3) 64 x 64 tiles of the trailing lower triangle take the rank-kNb update.
// The kernels are templated on the arithmetic type: float64 for the FP64
// path; float32 for the mixed path below.
//
// FP64 solve: forward and back substitution by blocks of kNb unknowns, each
// block one small kernel (one warp, the diagonal block in shared memory) and
// one update kernel spread over many CTAs.
//
// Mixed solve (TF32/BF16 modes): on this GPU float64 arithmetic runs at about
// 1/67 of float32, so F is factored in float32 and the solution is refined in
// float64 (iterative refinement): delta_0 = (L32 L32^T)^{-1} g, then repeatedly
// r = g - F delta in float64 and delta += (L32 L32^T)^{-1} r.  The refinement
// stops when the correction is below 1e-12 of delta, or when it stagnates at
// a level below 1e-8 (the attainable accuracy for the conditioning of F);
// otherwise (or if the float32 factorisation fails) the caller falls back to
// the float64 Cholesky.
#include "mnl_internal.cuh"

namespace mnl {
namespace {

constexpr int kNb = 64;

template <typename T>
__device__ __forceinline__ bool good_pivot(T v) {
  return v > (T)0 && isfinite(v);
}

template <typename T>
__global__ void __launch_bounds__(256) potrf_diag_kernel(T *F, int64_t n, int64_t j0, T *dinv, int *status,
                                                         int bad_bit) {
  __shared__ T A[kNb][kNb + 1];
  __shared__ T rinv;
  __shared__ int bad;
  const int nb = (int)min((int64_t)kNb, n - j0);
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  if (tid == 0) bad = 0;
  for (int e = tid; e < nb * nb; e += blockDim.x) {
    const int c = e / nb, r = e % nb;
    A[r][c] = r >= c ? F[(j0 + c) * n + j0 + r] : (T)0;
  }
  __syncthreads();
  for (int c = 0; c < nb; ++c) {
    if (tid == 0) {
      const T piv = A[c][c];
      T l = (T)1;
      if (!good_pivot(piv)) bad = 1;
      else l = sqrt(piv);
      A[c][c] = l;
      rinv = (T)1 / l;
    }
    __syncthreads();
    const T ri = rinv;
    for (int r = c + 1 + tid; r < nb; r += blockDim.x) A[r][c] *= ri;
    __syncthreads();
    for (int rr = c + 1 + ty; rr < nb; rr += 16) {
      const T arc = A[rr][c];
      for (int cc = c + 1 + tx; cc <= rr; cc += 16) A[rr][cc] = fma(-arc, A[cc][c], A[rr][cc]);
    }
    __syncthreads();
  }
  for (int e = tid; e < nb * nb; e += blockDim.x) {
    const int c = e / nb, r = e % nb;
    if (r >= c) F[(j0 + c) * n + j0 + r] = A[r][c];
  }
  for (int c = tid; c < nb; c += blockDim.x) dinv[j0 + c] = (T)1 / A[c][c];
  if (tid == 0 && bad) atomicOr(status, bad_bit);
}

// Rows r >= j0 + kNb: L21[r][:] = A21[r][:] L11^{-T}, one thread per row.
template <typename T>
__global__ void __launch_bounds__(32) trsm_panel_kernel(T *F, int64_t n, int64_t j0, const T *dinv) {
  __shared__ T L[kNb][kNb + 1];
  __shared__ T ri[kNb];
  const int tid = threadIdx.x;
  for (int e = tid; e < kNb * kNb; e += blockDim.x) {
    const int c = e / kNb, r = e % kNb;
    L[r][c] = r >= c ? F[(j0 + c) * n + j0 + r] : (T)0;
  }
  for (int c = tid; c < kNb; c += blockDim.x) ri[c] = dinv[j0 + c];
  __syncthreads();
  const int64_t r = j0 + kNb + (int64_t)blockIdx.x * blockDim.x + tid;
  if (r >= n) return;
  T x[kNb];
#pragma unroll
  for (int c = 0; c < kNb; ++c) x[c] = F[(j0 + c) * n + r];
#pragma unroll
  for (int c = 0; c < kNb; ++c) {
    T v = x[c];
#pragma unroll
    for (int t = 0; t < c; ++t) v = fma(-x[t], L[c][t], v);
    x[c] = v * ri[c];
  }
#pragma unroll
  for (int c = 0; c < kNb; ++c) F[(j0 + c) * n + r] = x[c];
}

// Trailing update, tile (bi, bj), bi >= bj, of the rows/columns >= j1 = j0 + kNb.
template <typename T>
__global__ void __launch_bounds__(256) syrk_update_kernel(T *F, int64_t n, int64_t j0) {
  __shared__ T Ar[kNb][65];
  __shared__ T Ac[kNb][65];
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
    Ar[kk][rr] = (r0 + rr < n) ? F[(j0 + kk) * n + r0 + rr] : (T)0;
    Ac[kk][rr] = (c0 + rr < n) ? F[(j0 + kk) * n + c0 + rr] : (T)0;
  }
  __syncthreads();
  T acc[4][4];
#pragma unroll
  for (int v = 0; v < 4; ++v)
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[v][u] = (T)0;
#pragma unroll 8
  for (int kk = 0; kk < kNb; ++kk) {
    T a[4], b[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) a[v] = Ar[kk][tx + 16 * v];
#pragma unroll
    for (int u = 0; u < 4; ++u) b[u] = Ac[kk][ty + 16 * u];
#pragma unroll
    for (int v = 0; v < 4; ++v)
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[v][u] = fma(a[v], b[u], acc[v][u]);
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int64_t r = r0 + tx + 16 * v, c = c0 + ty + 16 * u;
      if (r < n && c < n && r >= c) F[c * n + r] -= acc[v][u];
    }
}

template <typename T>
cudaError_t cholesky_t(int64_t n, T *F, T *dinv, int *status, int bad_bit, cudaStream_t st) {
  for (int64_t j0 = 0; j0 < n; j0 += kNb) {
    potrf_diag_kernel<T><<<1, 256, 0, st>>>(F, n, j0, dinv, status, bad_bit);
    const int64_t j1 = j0 + kNb;
    if (j1 >= n) break;
    const int64_t rows = n - j1;
    trsm_panel_kernel<T><<<(unsigned)((rows + 31) / 32), 32, 0, st>>>(F, n, j0, dinv);
    const int64_t nt = (rows + 63) / 64;
    syrk_update_kernel<T><<<(unsigned)(nt * (nt + 1) / 2), 256, 0, st>>>(F, n, j0);
  }
  return cudaGetLastError();
}

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

// ---------------------------------------------------------------------------
// Mixed solve pieces.
// ---------------------------------------------------------------------------

// Copy the strictly lower triangle of L into the upper triangle as L^T
// (32 x 32 tiles through shared memory; reads and writes are coalesced).
__global__ void lower_to_upper_kernel(int64_t n, float *__restrict__ A) {
  __shared__ float t[32][33];
  const int64_t bi = blockIdx.y, bj = blockIdx.x;  // source tile rows bi*32.., columns bj*32.. (bi >= bj)
  if (bj > bi) return;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int k = ty; k < 32; k += blockDim.y) {
    const int64_t r = bi * 32 + tx, c = bj * 32 + k;  // t[tx][k] = L(r, c)
    t[tx][k] = (r < n && c < n && r > c) ? A[c * n + r] : 0.f;
  }
  __syncthreads();
  for (int k = ty; k < 32; k += blockDim.y) {
    const int64_t row = bj * 32 + tx, col = bi * 32 + k;  // U(row, col) = L(col, row) = t[k][tx]
    if (row < n && col < n && col > row) A[col * n + row] = t[k][tx];
  }
}

__global__ void to_f32_lower_kernel(int64_t n, const double *__restrict__ F, float *__restrict__ F32) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t c = blockIdx.y + (int64_t)gridDim.y * blockIdx.z;
  if (r >= n || c >= n || r < c) return;
  F32[c * n + r] = (float)F[c * n + r];
}

// Single-CTA float32 solve L L^T d = rhs (rhs float64), then the refinement
// bookkeeping: delta += d (or delta = d when `first`), convergence flags.
// ref[0] = max|d| of the previous correction, ref[1] = 1 when converged.
__global__ void __launch_bounds__(1024) solve_f32_kernel(int64_t n, const float *__restrict__ L,
                                                         const float *__restrict__ dinv,
                                                         const double *__restrict__ rhs, float *__restrict__ work,
                                                         double *__restrict__ delta, double *__restrict__ ref,
                                                         int *__restrict__ status, int first) {
  __shared__ float Ld[32][33];
  __shared__ float di[32];
  __shared__ float xb[32];
  __shared__ float red_d[32], red_x[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  if (*status & 8) return;
  if (!first && ref[1] != 0.0) return;
  float *x = work;
  for (int64_t i = tid; i < n; i += blockDim.x) x[i] = (float)rhs[i];
  const int64_t nblk = (n + 31) / 32;
  for (int64_t bb = 0; bb < nblk; ++bb) {
    const int64_t b0 = bb * 32;
    const int w = (int)min((int64_t)32, n - b0);
    __syncthreads();
    for (int e = tid; e < 32 * 32; e += blockDim.x) {
      const int r = e & 31, c = e >> 5;
      Ld[r][c] = (r < w && c < w && r >= c) ? L[(b0 + c) * n + b0 + r] : 0.f;
    }
    if (tid < 32) di[tid] = tid < w ? dinv[b0 + tid] : 0.f;
    __syncthreads();
    if (warp == 0) {
      float v = lane < w ? x[b0 + lane] : 0.f;
      for (int c = 0; c < w; ++c) {
        const float xc = __shfl_sync(0xffffffffu, v, c) * di[c];
        if (lane == c) v = xc;
        if (lane > c) v = fmaf(-Ld[lane][c], xc, v);
      }
      if (lane < w) { x[b0 + lane] = v; xb[lane] = v; }
    }
    __syncthreads();
    for (int64_t r = b0 + w + tid; r < n; r += blockDim.x) {
      float s = 0.f;
#pragma unroll 8
      for (int c = 0; c < w; ++c) s = fmaf(L[(b0 + c) * n + r], xb[c], s);
      x[r] -= s;
    }
  }
  for (int64_t bb = nblk - 1; bb >= 0; --bb) {
    const int64_t b0 = bb * 32;
    const int w = (int)min((int64_t)32, n - b0);
    __syncthreads();
    for (int e = tid; e < 32 * 32; e += blockDim.x) {
      const int r = e & 31, c = e >> 5;
      Ld[r][c] = (r < w && c < w && r >= c) ? L[(b0 + c) * n + b0 + r] : 0.f;
    }
    if (tid < 32) di[tid] = tid < w ? dinv[b0 + tid] : 0.f;
    __syncthreads();
    if (warp == 0) {
      float v = lane < w ? x[b0 + lane] : 0.f;
      for (int c = w - 1; c >= 0; --c) {
        const float xc = __shfl_sync(0xffffffffu, v, c) * di[c];
        if (lane == c) v = xc;
        if (lane < c) v = fmaf(-Ld[c][lane], xc, v);
      }
      if (lane < w) { x[b0 + lane] = v; xb[lane] = v; }
    }
    __syncthreads();
    // rows r < b0: x_r -= sum_c L(b0+c, r) x_c, read from the transposed copy U(r, b0+c) = L(b0+c, r)
    // kept in the upper triangle (column b0+c, row r), so consecutive threads read consecutive rows.
    for (int64_t r = tid; r < b0; r += blockDim.x) {
      float s = 0.f;
#pragma unroll 8
      for (int c = 0; c < w; ++c) s = fmaf(L[(b0 + c) * n + r], xb[c], s);
      x[r] -= s;
    }
  }
  __syncthreads();
  // delta update and convergence bookkeeping (fixed-order max reductions)
  float md = 0.f, mx = 0.f;
  for (int64_t i = tid; i < n; i += blockDim.x) {
    const double di = (double)x[i];
    const double nv = first ? di : delta[i] + di;
    md = fmaxf(md, fabsf(x[i]));
    mx = fmaxf(mx, (float)fabs(nv));
  }
  for (int o = 16; o > 0; o >>= 1) {
    md = fmaxf(md, __shfl_xor_sync(0xffffffffu, md, o));
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  if (lane == 0) { red_d[warp] = md; red_x[warp] = mx; }
  __syncthreads();
  if (tid == 0) {
    float a = 0.f, b = 0.f;
    for (int w2 = 0; w2 < nwarp; ++w2) { a = fmaxf(a, red_d[w2]); b = fmaxf(b, red_x[w2]); }
    red_d[0] = a;
    red_x[0] = b;
  }
  __syncthreads();
  const double dn = red_d[0], xn = red_x[0];
  if (first) {
    for (int64_t i = tid; i < n; i += blockDim.x) delta[i] = (double)x[i];
    if (tid == 0) { ref[0] = dn; ref[1] = 0.0; ref[2] = 0.0; }
    return;
  }
  const double prev = ref[0];
  const bool improving = dn < 0.5 * prev;
  if (improving || dn <= 1e-12 * xn)
    for (int64_t i = tid; i < n; i += blockDim.x) delta[i] += (double)x[i];
  if (tid == 0) {
    ref[2] += 1.0;  // refinement steps taken
    if (dn <= 1e-12 * xn) ref[1] = 1.0;
    else if (!improving) {
      if (dn <= 1e-8 * xn) ref[1] = 1.0;  // stagnated at the attainable accuracy
      else { ref[1] = 2.0; atomicOr(status, 16); }
    }
    ref[0] = dn;
  }
}

// r = g - F delta in float64 (F full symmetric, column-major): grid (row blocks x column chunks),
// partial sums per column chunk then a fixed-order reduction.
constexpr int kGemvChunks = 8;
__global__ void __launch_bounds__(128) resid_partial_kernel(int64_t n, const double *__restrict__ F,
                                                            const double *__restrict__ delta,
                                                            double *__restrict__ part, const double *__restrict__ ref) {
  if (ref[1] != 0.0) return;
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const int64_t c0 = n * blockIdx.y / gridDim.y, c1 = n * (blockIdx.y + 1) / gridDim.y;
  double s0 = 0.0, s1 = 0.0;
  int64_t c = c0;
  for (; c + 1 < c1; c += 2) {
    s0 = fma(F[c * n + r], delta[c], s0);
    s1 = fma(F[(c + 1) * n + r], delta[c + 1], s1);
  }
  if (c < c1) s0 = fma(F[c * n + r], delta[c], s0);
  part[blockIdx.y * n + r] = s0 + s1;
}

__global__ void resid_reduce_kernel(int64_t n, const double *__restrict__ g, const double *__restrict__ part,
                                    double *__restrict__ r, const double *__restrict__ ref) {
  if (ref[1] != 0.0) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < kGemvChunks; ++k) s += part[k * n + i];
    r[i] = g[i] - s;
  }
}

__global__ void refine_check_kernel(const double *ref, int *status) {
  if (ref[1] != 1.0) atomicOr(status, 16);
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
      Ps[rr * W + k] = A[(j0 + k) * n + j0 + rr];
    }
    __syncthreads();
    if (warp == 0) {  // diagonal block, lane = row
      for (int c = 0; c < nb; ++c) {
        T lcc = (T)1;
        if (lane == c) {
          const T piv = Ps[c * W + c];
          if (!(piv > (T)0) || !isfinite(piv)) bad = 1;
          else lcc = sqrt(piv);
          Ps[c * W + c] = lcc;
          dinv[c] = (T)1 / lcc;
        }
        __syncwarp();
        const T ri = dinv[c];
        if (lane > c && lane < nb) Ps[lane * W + c] *= ri;
        __syncwarp();
        if (lane > c && lane < nb) {
          const T lrc = Ps[lane * W + c];
          for (int cc = c + 1; cc <= lane; ++cc) Ps[lane * W + cc] -= lrc * Ps[cc * W + c];
        }
        __syncwarp();
      }
    }
    __syncthreads();
    for (int64_t rr = nb + tid; rr < m; rr += blockDim.x) {  // rows below: solve against the block
      T x[W];
#pragma unroll
      for (int c = 0; c < W; ++c) x[c] = c < nb ? Ps[rr * W + c] : (T)0;
#pragma unroll
      for (int c = 0; c < W; ++c) {
        if (c < nb) {
          T v = x[c];
#pragma unroll
          for (int t = 0; t < c; ++t) v -= x[t] * Ps[c * W + t];
          x[c] = v * dinv[c];
        }
      }
#pragma unroll
      for (int c = 0; c < W; ++c)
        if (c < nb) Ps[rr * W + c] = x[c];
    }
    __syncthreads();
    // panel back to A: L (lower) and L^T (upper)
    for (int64_t e = tid; e < m * nb; e += blockDim.x) {
      const int k = (int)(e / m);
      const int64_t rr = e % m;
      if (rr >= k) {
        const T v = Ps[rr * W + k];
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
          a[u] = r0 + u < m ? Ps[(r0 + u) * W + k] : (T)0;
          b[u] = c0 + u < m ? Ps[(c0 + u) * W + k] : (T)0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[u][v] += a[u] * b[v];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const int64_t r = r0 + u, c = c0 + v;
          if (r < m && c < m && r >= c) A[(j0 + c) * n + j0 + r] -= acc[u][v];
        }
    }
    __syncthreads();
    if (bad) return false;
  }
  __syncthreads();
  return bad == 0;
}

// x <- (L L^T)^{-1} x for a factor with L^T in the upper triangle; x in shared memory.
template <typename T, typename V>
__device__ void cta_chol_solve(const T *__restrict__ A, int64_t n, V *__restrict__ x) {
  const int tid = threadIdx.x;
  for (int64_t j = 0; j < n; ++j) {  // forward, one column at a time (n is small)
    __syncthreads();
    const V xj = x[j] / (V)A[j * n + j];
    __syncthreads();
    if (tid == 0) x[j] = xj;
    for (int64_t r = j + 1 + tid; r < n; r += blockDim.x) x[r] -= (V)A[j * n + r] * xj;
  }
  for (int64_t j = n - 1; j >= 0; --j) {  // backward with U = L^T: column j of U lies above the diagonal
    __syncthreads();
    const V xj = x[j] / (V)A[j * n + j];
    __syncthreads();
    if (tid == 0) x[j] = xj;
    for (int64_t r = tid; r < j; r += blockDim.x) x[r] -= (V)A[j * n + r] * xj;
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
                                                                         const int *__restrict__ active, int iters,
                                                                         int *__restrict__ status, int64_t max_n) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[32];
  __shared__ float dinv32[32];
  __shared__ double dinv64[16];
  const int b = blockIdx.x;
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

int cholesky_launches(int64_t n) { return (int)(3 * ((n + kNb - 1) / kNb) - 2); }

cudaError_t launch_cholesky(int64_t n, double *F, double *dinv, int *status, cudaStream_t st) {
  return cholesky_t<double>(n, F, dinv, status, 4, st);
}

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

cudaError_t launch_mixed_solve(int64_t n, const double *F, float *F32, float *dinv32, const double *g, double *delta,
                               double *rwork, float *fwork, double *ref, int *status, int iters, cudaStream_t st,
                               int *launches) {
  dim3 grid((unsigned)((n + 255) / 256), (unsigned)std::min<int64_t>(n, 65535),
            (unsigned)((n + 65534) / 65535));
  to_f32_lower_kernel<<<grid, 256, 0, st>>>(n, F, F32);
  cudaError_t e = cholesky_t<float>(n, F32, dinv32, status, 8, st);
  if (e != cudaSuccess) return e;
  const unsigned nt = (unsigned)((n + 31) / 32);
  lower_to_upper_kernel<<<dim3(nt, nt), dim3(32, 8), 0, st>>>(n, F32);
  int cnt = 2 + cholesky_launches(n);
  solve_f32_kernel<<<1, 1024, 0, st>>>(n, F32, dinv32, g, fwork, delta, ref, status, 1);
  ++cnt;
  double *part = rwork + n;
  for (int it = 0; it < iters; ++it) {
    resid_partial_kernel<<<dim3((unsigned)((n + 127) / 128), kGemvChunks), 128, 0, st>>>(n, F, delta, part, ref);
    resid_reduce_kernel<<<(unsigned)std::min<int64_t>(256, (n + 255) / 256), 256, 0, st>>>(n, g, part, rwork, ref);
    solve_f32_kernel<<<1, 1024, 0, st>>>(n, F32, dinv32, rwork, fwork, delta, ref, status, 0);
    cnt += 3;
  }
  refine_check_kernel<<<1, 1, 0, st>>>(ref, status);
  ++cnt;
  if (launches) *launches = cnt;
  return cudaGetLastError();
}

size_t mixed_solve_rwork_doubles(int64_t n) { return (size_t)n * (1 + kGemvChunks); }

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

namespace mnl {

size_t grouped_chol_smem(int64_t nmax) {
  const size_t vec = (((size_t)2 * nmax * sizeof(double) + 15) & ~(size_t)15);
  const size_t p32 = (size_t)nmax * 32 * sizeof(float), p64 = (size_t)nmax * 16 * sizeof(double);
  return vec + std::max(p32, p64);
}

cudaError_t launch_grouped_chol_solve(bool mixed, const GroupProblem *probs, int nprob, const int *active,
                                      int iters, int *status, size_t smem, int64_t max_n, cudaStream_t st) {
  cudaError_t e;
  if (mixed) {
    if ((e = cudaFuncSetAttribute(grouped_chol_solve_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem)))
      return e;
    grouped_chol_solve_kernel<true><<<nprob, kCtaThreads, smem, st>>>(probs, active, iters, status, max_n);
  } else {
    if ((e = cudaFuncSetAttribute(grouped_chol_solve_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem)))
      return e;
    grouped_chol_solve_kernel<false><<<nprob, kCtaThreads, smem, st>>>(probs, active, iters, status, max_n);
  }
  return cudaGetLastError();
}

}  // namespace mnl
