// Newton solve F delta = g (eq. "NR update"; F = -H symmetric positive
// definite, column-major, both triangles filled by the assembly).
//
// Factorisation: one cooperative (co-resident) grid walks the panels of
// kCb = 64 columns of a blocked right-looking Cholesky F = L L^T.  Per panel k:
//   A (CTA 0)  factor the diagonal block: two 32 x 32 Cholesky steps held in
//              the registers of one warp with the 32 x 32 block between them,
//              and the inverse of the 64 x 64 factor block (Inv_kk) by the same
//              2 x 2 block recursion;
//   B (all)    L_ik = A_ik Inv_kk^T for the row blocks below (a product instead
//              of a substitution); with the inverse, B_kj = Inv_kk B_kj (j < k)
//              and B_kk = Inv_kk;
//   C (all)    trailing update A_ij -= L_ik L_jk^T (k < j <= i); with the
//              inverse, B_ij -= L_ik B_kj (i > k, j <= k).  CTA 0 updates the
//              next diagonal block first and factors it (step A of panel k+1)
//              while the other CTAs take the remaining tiles.
// B = L^{-1} is the block forward substitution L B = I carried along with the
// factorisation (n^3/3 more flops, no extra barrier).  Every tile operation is
// a 64 x 64 x 64 product staged in shared memory, 4 x 4 outputs per thread.
// The steps are separated by grid-wide barriers whose waits are bounded on
// %globaltimer; a wait that runs out raises an abort flag that every CTA sees,
// all CTAs return, and *err is set.
//
// Mixed solve (TF32/BF16 modes): on this GPU float64 arithmetic runs at about
// 1/67 of float32, so F is factored (and L inverted) in float32 and the
// solution is refined in float64: delta_0 = L^{-T} L^{-1} g, then repeatedly
// r = g - F delta (float64) and delta += L^{-T} L^{-1} r.  With the explicit
// inverse each solve is two matrix-vector products spread over the whole GPU.
// The refinement stops when the correction is below 1e-12 of delta, or when it
// stagnates at a level below 1e-8 (the attainable accuracy for the
// conditioning of F); otherwise (or if the float32 factor fails) the caller
// falls back to the float64 factorisation, which is the same kernel without
// the inverse.
#include "mnl_internal.cuh"

namespace mnl {

constexpr int kMaxCoopGrid = 1024;
struct GridBarrier {
  unsigned count, gen;
  int abort, pad;
  int smid[kMaxCoopGrid];  // SM of each CTA
};

namespace {

constexpr int kCb = 64;           // panel width and tile edge
constexpr int kCs = 68;           // shared row stride of the product operands
constexpr int kDs = 65;           // shared row stride of the diagonal-block work
constexpr int kCoopThreads = 256;
constexpr uint64_t kWaitNs = 4000000000ull;  // bound of one barrier wait

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier with a bounded wait.  Returns false in every thread of the
// CTA when this CTA or another one gave up; the caller then returns.
__device__ bool grid_sync(GridBarrier *b, unsigned nblocks, int *err) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned *vgen = &b->gen;
    volatile int *vab = &b->abort;
    int good = *vab == 0;
    if (good) {
      const unsigned g = *vgen;
      __threadfence();
      if (atomicAdd(&b->count, 1u) == nblocks - 1) {
        atomicExch(&b->count, 0u);
        __threadfence();
        atomicAdd(&b->gen, 1u);
      } else {
        const uint64_t t0 = gtimer();
        while (*vgen == g) {
          if (*vab) { good = 0; break; }
          if (gtimer() - t0 > kWaitNs) {
            atomicExch(&b->abort, 1);
            atomicOr(err, 2);
            good = 0;
            break;
          }
          __nanosleep(64);
        }
      }
      __threadfence();
    }
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

template <typename T>
struct Ld4;
template <>
struct Ld4<float> {
  __device__ static void load(const float *p, float v[4]) {
    const float4 a = *reinterpret_cast<const float4 *>(p);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  }
};
template <>
struct Ld4<double> {
  __device__ static void load(const double *p, double v[4]) {
    const double2 a = reinterpret_cast<const double2 *>(p)[0], b = reinterpret_cast<const double2 *>(p)[1];
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  }
};

// S[m][r] = element (r, m) of a 64 x 64 operand, zero outside r < rmax, m < mmax.
//   TR = false: (r, m) at base[m * ld + r]  (a column-major block)
//   TR = true : (r, m) at base[r * ld + m]  (the transpose of one)
// Loads are issued kBatch at a time before the shared stores (latency).
constexpr int kPer = kCb * kCb / kCoopThreads;  // elements per thread
template <typename T, bool TR, int kBatch>
__device__ __forceinline__ void stage64(T *S, const T *__restrict__ base, int64_t ld, int rmax, int mmax) {
#pragma unroll
  for (int u0 = 0; u0 < kPer; u0 += kBatch) {
    T v[kBatch];
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const int e = threadIdx.x + (u0 + u) * kCoopThreads;
      const int hi = e >> 6, lo = e & 63;
      const int r = TR ? hi : lo, m = TR ? lo : hi;
      v[u] = (r < rmax && m < mmax) ? base[TR ? (int64_t)r * ld + m : (int64_t)m * ld + r] : (T)0;
    }
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const int e = threadIdx.x + (u0 + u) * kCoopThreads;
      const int hi = e >> 6, lo = e & 63;
      const int r = TR ? hi : lo, m = TR ? lo : hi;
      S[m * kCs + r] = v[u];
    }
  }
}

// acc[u][v] = sum_m As[m][4 tx + u] Bs[m][4 ty + v]
template <typename T>
__device__ __forceinline__ void prod64(const T *As, const T *Bs, T acc[4][4]) {
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = (T)0;
#pragma unroll 4
  for (int m = 0; m < kCb; ++m) {
    T a[4], b[4];
    Ld4<T>::load(As + m * kCs + tx * 4, a);
    Ld4<T>::load(Bs + m * kCs + ty * 4, b);
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
  }
}

// Block (r, c) at base[c * ld + r], r < rmax, c < cmax: = acc (SUB false) or -= acc.
// The 16 old values are loaded before any store, so the loads are not held
// back by possible aliasing with the stores.
template <typename T, bool SUB>
__device__ __forceinline__ void put64(T *base, int64_t ld, int rmax, int cmax, const T acc[4][4]) {
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T old[4][4];
#pragma unroll
  for (int v = 0; v < 4; ++v)
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int r = tx * 4 + u, c = ty * 4 + v;
      old[v][u] = (SUB && r < rmax && c < cmax) ? base[(int64_t)c * ld + r] : (T)0;
    }
#pragma unroll
  for (int v = 0; v < 4; ++v)
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int r = tx * 4 + u, c = ty * 4 + v;
      if (r < rmax && c < cmax) base[(int64_t)c * ld + r] = SUB ? old[v][u] - acc[u][v] : acc[u][v];
    }
}

// One product tile: C (+)= opA opB^T over 64 inner indices.
template <typename T, bool TRB, bool SUB>
__device__ __forceinline__ void tile_op(T *sm, const T *Abase, int64_t lda, int rmax, const T *Bbase, int64_t ldb,
                                        int cmax, int mmax, T *Cbase, int64_t ldc) {
  T *As = sm, *Bs = sm + kCb * kCs;
  __syncthreads();  // the previous tile's readers are done with As, Bs
  constexpr int kBatch = sizeof(T) == 4 ? 8 : 4;
  stage64<T, false, kBatch>(As, Abase, lda, rmax, mmax);
  stage64<T, TRB, kBatch>(Bs, Bbase, ldb, cmax, mmax);
  __syncthreads();
  T acc[4][4];
  prod64<T>(As, Bs, acc);
  put64<T, SUB>(Cbase, ldc, rmax, cmax, acc);
}

// Pivot step: 1/sqrt(d) and sqrt(d).  float32 (the factor that the float64
// refinement corrects) uses the hardware reciprocal square root; float64 keeps
// correctly rounded operations.
__device__ __forceinline__ void pivot(float d, float &lc, float &ri) {
  ri = rsqrtf(d);
  lc = d * ri;
}
__device__ __forceinline__ void pivot(double d, double &lc, double &ri) {
  lc = sqrt(d);
  ri = 1.0 / lc;
}

// Cholesky of a 32 x 32 block by one warp: lane r holds row r of the lower
// triangle in a[0..31].  Column c of the factor is published in row c of Lt
// (Lt[c][r] = L_rc, zero above the diagonal) so that every row's updates are
// independent loads and FMAs; rinv[c] = 1 / L_cc.  The next pivot depends only
// on row c+1 (a_{c+1,c+1} - L_{c+1,c}^2), so it is taken from that lane before
// the column's other updates, which keeps them off the critical path.  Entries
// of a[] above the diagonal are left unspecified (finite) and are never used.
// Returns false when a pivot is not positive or not finite (the factor then
// continues with 1 there).
constexpr int kLts = 36;  // row stride of Lt (16-byte aligned rows)
template <typename T>
__device__ __forceinline__ bool warp_chol32(T a[32], T *Lt, T *rinv) {
  const int lane = threadIdx.x & 31;
  bool ok = true;
  T dg = __shfl_sync(0xffffffffu, a[0], 0);
#pragma unroll
  for (int c = 0; c < 32; ++c) {
    const bool good = dg > (T)0 && isfinite(dg);
    ok = ok && good;
    T lc = (T)1, ri = (T)1;
    if (good) pivot(dg, lc, ri);
    const T v = lane == c ? lc : a[c] * ri;
    a[c] = v;
    if (c + 1 < 32) dg = __shfl_sync(0xffffffffu, fma(-v, v, a[c + 1]), c + 1);
    Lt[c * kLts + lane] = lane >= c ? v : (T)0;
    if (lane == 0) rinv[c] = ri;
    __syncwarp();
    const T ac = lane > c ? v : (T)0;
#pragma unroll
    for (int j = c + 1; j < 32; ++j) a[j] = fma(-ac, Lt[c * kLts + j], a[j]);
  }
  __syncwarp();
  return ok;
}

// Column `lane` of the inverse of the 32 x 32 lower-triangular factor (given
// as Lt and its reciprocal diagonal rinv) into X (row-major, stride kDs), by a
// column sweep: x = e_lane; for each m, x_m *= rinv_m, then x_i -= L_im x_m.
template <typename T>
__device__ __forceinline__ void warp_trinv32(const T *Lt, const T *rinv, T *X) {
  const int lane = threadIdx.x & 31;
  T x[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) x[i] = i == lane ? (T)1 : (T)0;
#pragma unroll
  for (int m = 0; m < 32; ++m) {
    x[m] *= rinv[m];
#pragma unroll
    for (int g = (m + 1) / 4; g < 8; ++g) {
      T l4[4];
      Ld4<T>::load(Lt + m * kLts + 4 * g, l4);
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (4 * g + u > m) x[4 * g + u] = fma(-l4[u], x[m], x[4 * g + u]);
    }
  }
#pragma unroll
  for (int i = 0; i < 32; ++i) X[i * kDs + lane] = x[i];
}

// 32 x 32 products over 32 inner indices on shared blocks, all 256 threads:
// thread (r0 = tid / 32, c = lane) makes rows r0, r0 + 8, r0 + 16, r0 + 24 of
// column c.  out(r, c) = sum_m A(r, m) B(c, m) with A(r, m) = Ab[r * kDs + m]
// and B(c, m) = Bb[c * sb + m * sm] (sb, sm select B or B^T).
template <typename T>
__device__ __forceinline__ void prod32(const T *Ab, const T *Bb, int sb, int sm, T out[4]) {
  const int c = threadIdx.x & 31, r0 = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < 4; ++q) out[q] = (T)0;
#pragma unroll 8
  for (int m = 0; m < 32; ++m) {
    const T b = Bb[c * sb + m * sm];
#pragma unroll
    for (int q = 0; q < 4; ++q) out[q] = fma(Ab[(r0 + 8 * q) * kDs + m], b, out[q]);
  }
}

template <typename T>
struct CoopArgs {
  T *A;     // n x n column-major; lower triangle: F in, L out
  T *Li;    // n x n: L^{-1} in the lower triangle (inverse only), zero on entry
  T *Dinv;  // [np][64 * 64]: inverses of the diagonal blocks, column-major
  T *dinv;  // [n]: 1 / L_jj
  int64_t n;
  GridBarrier *bar;
  int *status;
  int bad_bit;
  int *err;
};

// Step A for panel k (one CTA): factor the (already updated) diagonal block and
// invert the factor block, by the 2 x 2 block recursion
//   L11 = chol(D11), L21 = D21 Inv11^T, L22 = chol(D22 - L21 L21^T),
//   Inv21 = -Inv22 (L21 Inv11).
// Rows/columns past n are padded with the identity.  Kept out of line: the
// per-lane register rows of the warp steps then stay in registers.
template <typename T>
__device__ __noinline__ void factor_diag(const CoopArgs<T> &a, int k, T *sm) {
  T *D = sm, *Iv = sm + 64 * kDs, *Tm = sm + 128 * kDs;  // [64][kDs], [64][kDs], [32][kDs]
  T *rinv = sm + 160 * kDs, *Lt = rinv + 64;              // [64], [32][kLts]
  const int64_t n = a.n, j0 = (int64_t)k * kCb;
  const int nb = (int)(n - j0 < kCb ? n - j0 : kCb);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  __syncthreads();
#pragma unroll
  for (int u0 = 0; u0 < kPer; u0 += 8) {
    T v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = tid + (u0 + u) * kCoopThreads, c = e >> 6, r = e & 63;
      v[u] = (r < nb && c < nb) ? (r >= c ? a.A[(j0 + c) * n + j0 + r] : (T)0) : (r == c ? (T)1 : (T)0);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = tid + (u0 + u) * kCoopThreads, c = e >> 6, r = e & 63;
      D[r * kDs + c] = v[u];
      Iv[r * kDs + c] = (T)0;
    }
  }
  __syncthreads();
  if (warp == 0) {  // L11 and its inverse
    T x[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) x[c] = D[lane * kDs + c];
    const bool ok = warp_chol32<T>(x, Lt, rinv);
#pragma unroll
    for (int c = 0; c < 32; ++c) D[lane * kDs + c] = x[c];
    if (!ok && lane == 0) atomicOr(a.status, a.bad_bit);
    __syncwarp();
    warp_trinv32<T>(Lt, rinv, Iv);
  }
  __syncthreads();
  const int c = lane, r0 = warp;
  T v[4];
  prod32<T>(D + 32 * kDs, Iv, kDs, 1, v);  // L21 = D21 Inv11^T (Inv11 is zero above the diagonal)
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 4; ++q) D[(32 + r0 + 8 * q) * kDs + c] = v[q];
  __syncthreads();
  prod32<T>(D + 32 * kDs, D + 32 * kDs, kDs, 1, v);  // L21 L21^T
#pragma unroll
  for (int q = 0; q < 4; ++q)  // D22 -= L21 L21^T (lower; columns >= 32 only)
    if (r0 + 8 * q >= c) D[(32 + r0 + 8 * q) * kDs + 32 + c] -= v[q];
  __syncthreads();
  if (warp == 0) {  // L22 and its inverse
    T x[32];
#pragma unroll
    for (int cc = 0; cc < 32; ++cc) x[cc] = lane >= cc ? D[(32 + lane) * kDs + 32 + cc] : (T)0;
    const bool ok = warp_chol32<T>(x, Lt, rinv + 32);
#pragma unroll
    for (int cc = 0; cc < 32; ++cc) D[(32 + lane) * kDs + 32 + cc] = x[cc];
    if (!ok && lane == 0) atomicOr(a.status, a.bad_bit);
    __syncwarp();
    warp_trinv32<T>(Lt, rinv + 32, Iv + 32 * kDs + 32);
  }
  __syncthreads();
  prod32<T>(D + 32 * kDs, Iv, 1, kDs, v);  // Tm = L21 Inv11 (B(c, m) = Inv11[m][c])
#pragma unroll
  for (int q = 0; q < 4; ++q) Tm[(r0 + 8 * q) * kDs + c] = v[q];
  __syncthreads();
  prod32<T>(Iv + 32 * kDs + 32, Tm, 1, kDs, v);  // Inv22 Tm
#pragma unroll
  for (int q = 0; q < 4; ++q) Iv[(32 + r0 + 8 * q) * kDs + c] = -v[q];
  __syncthreads();
  T *Dk = a.Dinv + (int64_t)k * kCb * kCb;
  for (int e = tid; e < 64 * 64; e += kCoopThreads) {
    const int cc = e >> 6, r = e & 63;
    if (r < nb && cc < nb && r >= cc) a.A[(j0 + cc) * n + j0 + r] = D[r * kDs + cc];
    Dk[cc * kCb + r] = r >= cc ? Iv[r * kDs + cc] : (T)0;
  }
  for (int cc = tid; cc < nb; cc += kCoopThreads) a.dinv[j0 + cc] = (T)1 / D[cc * kDs + cc];
}

// Tile (i, j), i >= j, of the lower triangle of the tile grid from its index t.
__device__ __forceinline__ void tri_tile(int t, int &bi, int &bj) {
  int i = (int)((sqrtf(8.f * (float)t + 1.f) - 1.f) * 0.5f);
  while ((i + 1) * (i + 2) / 2 <= t) ++i;
  while (i * (i + 1) / 2 > t) --i;
  bi = i;
  bj = t - i * (i + 1) / 2;
}

template <typename T, bool INV>
__global__ void __launch_bounds__(kCoopThreads, sizeof(T) == 4 ? 2 : 1) coop_cholesky_kernel(CoopArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *sm = reinterpret_cast<T *>(smem_raw);
  const int64_t n = a.n;
  const int np = (int)((n + kCb - 1) / kCb);
  const int G = (int)gridDim.x, b = (int)blockIdx.x;
  // The CTAs that share CTA 0's SM take no trailing-update tiles, so that the
  // diagonal factorisation (CTA 0, one warp at a time) has the SM to itself;
  // the other CTAs are the workers, numbered densely.
  __shared__ int s_quiet, s_widx, s_nw;
  if (threadIdx.x == 0) {
    unsigned sid;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(sid));
    a.bar->smid[b] = (int)sid;
  }
  if (b == 0) factor_diag<T>(a, 0, sm);
  if (!grid_sync(a.bar, G, a.err)) return;
  if (threadIdx.x == 0) {
    const volatile int *ids = a.bar->smid;
    const int s0 = ids[0];
    int before = 0, total = 0;
    for (int i = 1; i < G; ++i)
      if (ids[i] != s0) {
        ++total;
        if (i < b) ++before;
      }
    s_quiet = b != 0 && ids[b] == s0;
    s_widx = before;
    s_nw = total;
  }
  __syncthreads();
  for (int k = 0; k < np; ++k) {
    const int64_t j0 = (int64_t)k * kCb;
    const int nbk = (int)(n - j0 < kCb ? n - j0 : kCb);
    const T *Dk = a.Dinv + (int64_t)k * kCb * kCb;
    const int m = np - 1 - k;  // row blocks below the panel
    // ---- B: panel rows and (inverse) row block k of L^{-1} ----
    const int nB = m + (INV ? k + 1 : 0);
    for (int t = b; t < nB; t += G) {
      if (t < m) {
        const int64_t r0 = (int64_t)(k + 1 + t) * kCb;
        const int rmax = (int)(n - r0 < kCb ? n - r0 : kCb);
        tile_op<T, false, false>(sm, a.A + j0 * n + r0, n, rmax, Dk, kCb, nbk, nbk, a.A + j0 * n + r0, n);
      } else if (t < m + k) {
        const int64_t c0 = (int64_t)(t - m) * kCb;
        T *Bkj = a.Li + c0 * n + j0;
        // B_kj = Inv_kk B_kj: A operand (r, q) = Inv[r][q]; B operand (c, q) = B_kj[q][c]
        tile_op<T, true, false>(sm, Dk, kCb, nbk, Bkj, n, kCb, nbk, Bkj, n);
      } else {
        for (int e = threadIdx.x; e < kCb * kCb; e += kCoopThreads) {
          const int c = e >> 6, r = e & 63;
          if (r < nbk && c < nbk && r >= c) a.Li[(j0 + c) * n + j0 + r] = Dk[c * kCb + r];
        }
      }
    }
    if (k == np - 1) break;
    if (!grid_sync(a.bar, G, a.err)) return;
    // ---- C: trailing update (and the inverse's rows below) ----
    const int U = m * (m + 1) / 2;
    const int nC = U + (INV ? m * (k + 1) : 0);
    auto item = [&](int t) {
      if (t < U) {
        int bi, bj;
        tri_tile(t, bi, bj);
        const int64_t r0 = (int64_t)(k + 1 + bi) * kCb, c0 = (int64_t)(k + 1 + bj) * kCb;
        const int rmax = (int)(n - r0 < kCb ? n - r0 : kCb), cmax = (int)(n - c0 < kCb ? n - c0 : kCb);
        tile_op<T, false, true>(sm, a.A + j0 * n + r0, n, rmax, a.A + j0 * n + c0, n, cmax, kCb, a.A + c0 * n + r0,
                                n);
      } else {
        const int e = t - U;
        const int64_t r0 = (int64_t)(k + 1 + e / (k + 1)) * kCb, c0 = (int64_t)(e % (k + 1)) * kCb;
        const int rmax = (int)(n - r0 < kCb ? n - r0 : kCb);
        // B_ij -= L_ik B_kj: B operand (c, q) = B_kj[q][c]
        tile_op<T, true, true>(sm, a.A + j0 * n + r0, n, rmax, a.Li + c0 * n + j0, n, kCb, kCb, a.Li + c0 * n + r0,
                               n);
      }
    };
    if (b == 0) {  // the next diagonal block first, then its factorisation
      item(0);
      factor_diag<T>(a, k + 1, sm);
    }
    if (s_nw == 0) {  // no other SM: CTA 0 takes every tile
      if (b == 0)
        for (int t = 1; t < nC; ++t) item(t);
    } else if (b != 0 && !s_quiet) {
      for (int t = 1 + s_widx; t < nC; t += s_nw) item(t);
    }
    if (!grid_sync(a.bar, G, a.err)) return;
  }
}

// Copy the strictly lower triangle into the upper one (M^T), 32 x 32 tiles.
template <typename T>
__global__ void mirror_lower_kernel(int64_t n, T *__restrict__ M) {
  __shared__ T t[32][33];
  const int64_t bi = blockIdx.y, bj = blockIdx.x;
  if (bj > bi) return;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int k = ty; k < 32; k += blockDim.y) {
    const int64_t r = bi * 32 + tx, c = bj * 32 + k;
    t[tx][k] = (r < n && c < n && r > c) ? M[c * n + r] : (T)0;
  }
  __syncthreads();
  for (int k = ty; k < 32; k += blockDim.y) {
    const int64_t row = bj * 32 + tx, col = bi * 32 + k;
    if (row < n && col < n && col > row) M[col * n + row] = t[k][tx];
  }
}

__global__ void f64_to_f32_lower_kernel(int64_t n, const double *__restrict__ F, float *__restrict__ F32) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t c = blockIdx.y + (int64_t)gridDim.y * blockIdx.z;
  if (r >= n || c >= n || r < c) return;
  F32[c * n + r] = (float)F[c * n + r];
}

// y[o] = (g ? g[o] : 0) -/+ sum_{i in range} M[o n + i] x[i], warp per output o:
// column o of M is contiguous.  RANGE 0: rows 0..o, 1: rows o..n-1, 2: all.
// Skipped once the refinement has converged (ref[1] != 0).
template <typename TM, typename TX, typename TY, int RANGE>
__global__ void __launch_bounds__(256) gemv_col_kernel(int64_t n, const TM *__restrict__ M, const TX *__restrict__ x,
                                                       TY *__restrict__ y, const double *__restrict__ g,
                                                       const double *__restrict__ ref) {
  if (ref && ref[1] != 0.0) return;
  const int lane = threadIdx.x & 31;
  const int64_t o = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (o >= n) return;
  const int64_t i0 = RANGE == 1 ? o : 0, i1 = RANGE == 0 ? o + 1 : n;
  const TM *col = M + o * n;
  TM s[4] = {(TM)0, (TM)0, (TM)0, (TM)0};
  int64_t i = i0 + lane;
  for (; i + 96 < i1; i += 128) {
#pragma unroll
    for (int u = 0; u < 4; ++u) s[u] = fma(col[i + 32 * u], (TM)x[i + 32 * u], s[u]);
  }
  for (; i < i1; i += 32) s[0] = fma(col[i], (TM)x[i], s[0]);
  TM t = (s[0] + s[1]) + (s[2] + s[3]);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
  if (lane == 0) y[o] = g ? (TY)(g[o] - (double)t) : (TY)t;
}

// Refinement bookkeeping (one CTA): delta += z (delta = z when `first`), with
// ref[0] = max|z| of the previous correction, ref[1] = 1 once converged (2 when
// the refinement failed, status |= 16), ref[2] = refinement steps taken.
__global__ void __launch_bounds__(1024) refine_update_kernel(int64_t n, const float *__restrict__ z,
                                                             double *__restrict__ delta, double *__restrict__ ref,
                                                             int *__restrict__ status, int first) {
  __shared__ float red_d[32], red_x[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  if (*status & 8) return;
  if (!first && ref[1] != 0.0) return;
  float md = 0.f, mx = 0.f;
  for (int64_t i = tid; i < n; i += blockDim.x) {
    const double nv = first ? (double)z[i] : delta[i] + (double)z[i];
    md = fmaxf(md, fabsf(z[i]));
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
    for (int64_t i = tid; i < n; i += blockDim.x) delta[i] = (double)z[i];
    if (tid == 0) { ref[0] = dn; ref[1] = 0.0; ref[2] = 0.0; }
    return;
  }
  const double prev = ref[0];
  const bool improving = dn < 0.5 * prev;
  if (improving || dn <= 1e-12 * xn)
    for (int64_t i = tid; i < n; i += blockDim.x) delta[i] += (double)z[i];
  if (tid == 0) {
    ref[2] += 1.0;
    if (dn <= 1e-12 * xn) ref[1] = 1.0;
    else if (!improving) {
      if (dn <= 1e-8 * xn) ref[1] = 1.0;  // stagnated at the attainable accuracy
      else { ref[1] = 2.0; atomicOr(status, 16); }
    }
    ref[0] = dn;
  }
}

__global__ void refine_check_kernel(const double *ref, int *status) {
  if (ref[1] != 1.0) atomicOr(status, 16);
}

__global__ void status_and_kernel(int *status, int mask) { atomicAnd(status, mask); }

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

int64_t panels(int64_t n) { return (n + kCb - 1) / kCb; }

template <typename T, bool INV>
cudaError_t launch_coop(int64_t n, T *A, T *Li, T *Dinv, T *dinv, GridBarrier *bar, int *status, int bad_bit,
                        int *err, cudaStream_t st) {
  auto kern = coop_cholesky_kernel<T, INV>;
  const size_t smem = (size_t)std::max(160 * kDs + 64 + 32 * kLts, 2 * kCb * kCs) * sizeof(T);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, nsm = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kCoopThreads, smem)) != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int grid = std::min(nsm * std::min(per_sm, 2), kMaxCoopGrid);
  if ((e = cudaMemsetAsync(bar, 0, sizeof(GridBarrier), st)) != cudaSuccess) return e;
  CoopArgs<T> a;
  a.A = A; a.Li = Li; a.Dinv = Dinv; a.dinv = dinv; a.n = n; a.bar = bar;
  a.status = status; a.bad_bit = bad_bit; a.err = err;
  void *args[] = {&a};
  return cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(kern), dim3(grid), dim3(kCoopThreads), args, smem,
                                     st);
}

// Mixed-solve workspace pieces (byte offsets, 256-aligned).
struct MixedLayout {
  size_t li, dblk, dinv, y, z, r, ref, bar, total;
};
MixedLayout mixed_layout(int64_t n) {
  MixedLayout L;
  size_t o = 0;
  L.li = o; o += round256((size_t)n * n * 4);
  L.dblk = o; o += round256((size_t)panels(n) * kCb * kCb * 4);
  L.dinv = o; o += round256((size_t)n * 4);
  L.y = o; o += round256((size_t)n * 4);
  L.z = o; o += round256((size_t)n * 4);
  L.r = o; o += round256((size_t)n * 8);
  L.ref = o; o += round256(4 * 8);
  L.bar = o; o += round256(sizeof(GridBarrier));
  L.total = o;
  return L;
}

}  // namespace

size_t chol_work_bytes(int64_t n) {
  return round256((size_t)panels(n) * kCb * kCb * 8) + round256(sizeof(GridBarrier));
}

int cholesky_launches(int64_t) { return 1; }

cudaError_t launch_cholesky(int64_t n, double *F, double *dinv, void *work, int *status, int *err, cudaStream_t st) {
  unsigned char *w = static_cast<unsigned char *>(work);
  double *Dinv = reinterpret_cast<double *>(w);
  GridBarrier *bar = reinterpret_cast<GridBarrier *>(w + round256((size_t)panels(n) * kCb * kCb * 8));
  return launch_coop<double, false>(n, F, nullptr, Dinv, dinv, bar, status, 4, err, st);
}

size_t mixed_solve_bytes(int64_t n) { return mixed_layout(n).total; }

double *mixed_solve_ref(void *work, int64_t n) {
  return reinterpret_cast<double *>(static_cast<unsigned char *>(work) + mixed_layout(n).ref);
}

cudaError_t launch_mixed_solve(int64_t n, const double *F, float *F32, const double *g, double *delta, void *work,
                               int *status, int *err, int iters, cudaStream_t st, int *launches) {
  const MixedLayout L = mixed_layout(n);
  unsigned char *w = static_cast<unsigned char *>(work);
  float *Li = reinterpret_cast<float *>(w + L.li), *Dblk = reinterpret_cast<float *>(w + L.dblk);
  float *dinv = reinterpret_cast<float *>(w + L.dinv), *y = reinterpret_cast<float *>(w + L.y);
  float *z = reinterpret_cast<float *>(w + L.z);
  double *r = reinterpret_cast<double *>(w + L.r), *ref = reinterpret_cast<double *>(w + L.ref);
  GridBarrier *bar = reinterpret_cast<GridBarrier *>(w + L.bar);
  cudaError_t e;
  dim3 grid((unsigned)((n + 255) / 256), (unsigned)std::min<int64_t>(n, 65535), (unsigned)((n + 65534) / 65535));
  f64_to_f32_lower_kernel<<<grid, 256, 0, st>>>(n, F, F32);
  if ((e = cudaMemsetAsync(Li, 0, (size_t)n * n * 4, st)) != cudaSuccess) return e;
  if ((e = launch_coop<float, true>(n, F32, Li, Dblk, dinv, bar, status, 8, err, st)) != cudaSuccess) return e;
  const unsigned nt = (unsigned)((n + 31) / 32);
  mirror_lower_kernel<float><<<dim3(nt, nt), dim3(32, 8), 0, st>>>(n, Li);
  const unsigned gb = (unsigned)((n + 7) / 8);
  // delta_0 = L^{-T} (L^{-1} g)
  gemv_col_kernel<float, double, float, 0><<<gb, 256, 0, st>>>(n, Li, g, y, nullptr, nullptr);
  gemv_col_kernel<float, float, float, 1><<<gb, 256, 0, st>>>(n, Li, y, z, nullptr, nullptr);
  refine_update_kernel<<<1, 1024, 0, st>>>(n, z, delta, ref, status, 1);
  int cnt = 7;
  for (int it = 0; it < iters; ++it) {
    gemv_col_kernel<double, double, double, 2><<<gb, 256, 0, st>>>(n, F, delta, r, g, ref);  // r = g - F delta
    gemv_col_kernel<float, double, float, 0><<<gb, 256, 0, st>>>(n, Li, r, y, nullptr, ref);
    gemv_col_kernel<float, float, float, 1><<<gb, 256, 0, st>>>(n, Li, y, z, nullptr, ref);
    refine_update_kernel<<<1, 1024, 0, st>>>(n, z, delta, ref, status, 0);
    cnt += 4;
  }
  refine_check_kernel<<<1, 1, 0, st>>>(ref, status);
  ++cnt;
  if (launches) *launches = cnt;
  return cudaGetLastError();
}

cudaError_t launch_status_and(int *status, int mask, cudaStream_t st) {
  status_and_kernel<<<1, 1, 0, st>>>(status, mask);
  return cudaGetLastError();
}

cudaError_t launch_mixed_refine(int64_t n, const double *F, const double *g, double *delta, void *work, int *status,
                                int iters, cudaStream_t st, int *launches) {
  const MixedLayout L = mixed_layout(n);
  unsigned char *w = static_cast<unsigned char *>(work);
  float *Li = reinterpret_cast<float *>(w + L.li), *y = reinterpret_cast<float *>(w + L.y);
  float *z = reinterpret_cast<float *>(w + L.z);
  double *r = reinterpret_cast<double *>(w + L.r), *ref = reinterpret_cast<double *>(w + L.ref);
  const unsigned gb = (unsigned)((n + 7) / 8);
  int cnt = 0;
  for (int it = 0; it < iters; ++it) {
    gemv_col_kernel<double, double, double, 2><<<gb, 256, 0, st>>>(n, F, delta, r, g, ref);
    gemv_col_kernel<float, double, float, 0><<<gb, 256, 0, st>>>(n, Li, r, y, nullptr, ref);
    gemv_col_kernel<float, float, float, 1><<<gb, 256, 0, st>>>(n, Li, y, z, nullptr, ref);
    refine_update_kernel<<<1, 1024, 0, st>>>(n, z, delta, ref, status, 0);
    cnt += 4;
  }
  refine_check_kernel<<<1, 1, 0, st>>>(ref, status);
  if (launches) *launches = cnt + 1;
  return cudaGetLastError();
}

}  // namespace mnl
