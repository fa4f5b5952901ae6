// Newton solve F delta = g (eq. "NR update"; F = -H symmetric positive
// definite, column-major, both triangles filled by the assembly).
//
// Factorisation: one cooperative (co-resident) grid walks the panels of
// kCb = 64 columns of a blocked right-looking Cholesky F = L L^T.  Per panel k:
//   A (CTA 0)  factor the diagonal block and invert the factor block
//              (Inv_kk): two 32 x 32 steps, each a fused column-by-column
//              Cholesky and inverse in the registers of one warp, joined by
//              the 2 x 2 block recursion whose products use all warps;
//   B (all)    L_ik = A_ik Inv_kk^T for the row blocks below (a product instead
//              of a substitution); with the inverse, B_kj = Inv_kk B_kj (j < k)
//              and B_kk = Inv_kk;
//   C (all)    trailing update A_ij -= L_ik L_jk^T (k < j <= i); with the
//              inverse, B_ij -= L_ik B_kj (i > k, j <= k).  CTA 0 applies the
//              update of the next diagonal block inside step A of panel k+1,
//              which it runs while the other CTAs take the remaining tiles.
// B = L^{-1} is the block forward substitution L B = I carried along with the
// factorisation (n^3/3 more flops, no extra barrier).  Every tile operation is
// a 64 x 64 x 64 product staged in shared memory, 4 x 4 outputs per thread;
// each CTA copies the operands of its next tile (cp.async, two buffers) while
// it multiplies the current one.
// B and C are separated by a grid-wide barrier that CTA 0 (and the CTAs on its
// SM) only arrive at, so step A of the next panel starts as soon as CTA 0's
// own panel rows are done; C and the next B by one that every CTA waits at.
// The waits are bounded on %globaltimer; a wait that runs out raises an abort
// flag that every CTA sees, all CTAs return, and *err is set.
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
#include <algorithm>
#include <cstdlib>

#include "mnl_internal.cuh"

namespace mnl {

constexpr int kMaxCoopGrid = 1024;
struct GridBarrier {
  unsigned count[2], gen[2];  // two barriers, used alternately within a panel
  int abort, pad;
  int smid[kMaxCoopGrid];  // SM of each CTA
};

namespace {

constexpr int kCb = 64;           // panel width and tile edge
constexpr int kCs = 68;           // shared row stride of the product operands
constexpr int kDs = 68;           // shared stride of the diagonal-block work arrays (16-byte rows)
constexpr int kLts = 36;          // row stride of the published factor columns
constexpr int kCoopThreads = 256;
constexpr uint64_t kWaitNs = 4000000000ull;  // bound of one barrier wait

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier `w` with a bounded wait.  With wait = false the CTA only
// arrives (its writes are released to the waiting CTAs) and goes on.  Returns
// false in every thread of the CTA when this CTA or another one gave up; the
// caller then returns.
__device__ bool grid_sync(GridBarrier *b, int w, unsigned nblocks, int *err, uint64_t bound_ns, bool wait = true) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned *vgen = &b->gen[w];
    volatile int *vab = &b->abort;
    int good = *vab == 0;
    if (good) {
      const unsigned g = *vgen;
      __threadfence();
      if (atomicAdd(&b->count[w], 1u) == nblocks - 1) {
        atomicExch(&b->count[w], 0u);
        __threadfence();
        atomicAdd(&b->gen[w], 1u);
      } else if (wait) {
        const uint64_t t0 = gtimer();
        while (*vgen == g) {
          if (*vab) { good = 0; break; }
          if (gtimer() - t0 > bound_ns) {
            atomicExch(&b->abort, 1);
            atomicOr(err, kWaitCoop);
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
  __device__ static void store(float *p, const float v[4]) {
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
  }
};
template <>
struct Ld4<double> {
  __device__ static void load(const double *p, double v[4]) {
    const double2 a = reinterpret_cast<const double2 *>(p)[0], b = reinterpret_cast<const double2 *>(p)[1];
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  }
  __device__ static void store(double *p, const double v[4]) {
    reinterpret_cast<double2 *>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2 *>(p)[1] = make_double2(v[2], v[3]);
  }
};

// Element (r, m) of a 64 x 64 operand, zero outside r < rmax, m < mmax, for
// the kPer elements e = tid + u * kCoopThreads of this thread:
//   TR = false: (r, m) at base[m * ld + r]  (a column-major block)
//   TR = true : (r, m) at base[r * ld + m]  (the transpose of one)
// All loads of a tile are issued before any of them is used.
constexpr int kPer = kCb * kCb / kCoopThreads;  // elements per thread
template <typename T, bool TR>
__device__ __forceinline__ void load64(T v[kPer], const T *__restrict__ base, int64_t ld, int rmax, int mmax) {
#pragma unroll
  for (int u = 0; u < kPer; ++u) {
    const int e = threadIdx.x + u * kCoopThreads;
    const int hi = e >> 6, lo = e & 63;
    const int r = TR ? hi : lo, m = TR ? lo : hi;
    v[u] = (r < rmax && m < mmax) ? base[TR ? (int64_t)r * ld + m : (int64_t)m * ld + r] : (T)0;
  }
}
// S[m][r] = element (r, m) from load64.
template <typename T, bool TR>
__device__ __forceinline__ void store64(T *S, const T v[kPer]) {
#pragma unroll
  for (int u = 0; u < kPer; ++u) {
    const int e = threadIdx.x + u * kCoopThreads;
    const int hi = e >> 6, lo = e & 63;
    const int r = TR ? hi : lo, m = TR ? lo : hi;
    S[m * kCs + r] = v[u];
  }
}

// acc[u][v] = sum_m As[m][4 tx + u] Bs[m][4 ty + v], tx = tid % 16, ty = tid / 16.
// The operands of step m + 1 are loaded while step m is multiplied.
template <typename T>
__device__ __forceinline__ void prod64(const T *As, const T *Bs, T acc[4][4]) {
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const T *pa = As + tx * 4, *pb = Bs + ty * 4;
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = (T)0;
  T a[2][4], b[2][4];
  Ld4<T>::load(pa, a[0]);
  Ld4<T>::load(pb, b[0]);
#pragma unroll 2
  for (int m = 0; m < kCb; m += 2) {
    Ld4<T>::load(pa + (m + 1) * kCs, a[1]);
    Ld4<T>::load(pb + (m + 1) * kCs, b[1]);
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[0][u], b[0][v], acc[u][v]);
    if (m + 2 < kCb) {
      Ld4<T>::load(pa + (m + 2) * kCs, a[0]);
      Ld4<T>::load(pb + (m + 2) * kCs, b[0]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[1][u], b[1][v], acc[u][v]);
  }
}

// Asynchronous element copies global -> shared (zero fill when !valid).
template <typename T>
__device__ __forceinline__ void cp_elem(T *dst, const T *src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  if (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 4 : 0) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 8 : 0) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// S[m][r] = element (r, m) of a 64 x 64 operand (zero outside r < rmax,
// m < mmax) by asynchronous copies: tr = false: (r, m) at base[m * ld + r];
// tr = true: (r, m) at base[r * ld + m].
template <typename T>
__device__ __forceinline__ void cp64(T *S, const T *base, int64_t ld, bool tr, int rmax, int mmax) {
#pragma unroll
  for (int u = 0; u < kPer; ++u) {
    const int e = threadIdx.x + u * kCoopThreads;
    const int hi = e >> 6, lo = e & 63;
    const int r = tr ? hi : lo, m = tr ? lo : hi;
    const bool ok = r < rmax && m < mmax;
    cp_elem(S + m * kCs + r, ok ? base + (tr ? (int64_t)r * ld + m : (int64_t)m * ld + r) : base, ok);
  }
}

// One product tile: C (+)= opA opB^T over the inner indices m < mmax, with
// opA(r, m) = A[m * lda + r] (r < rmax), opB(c, m) = B[m * ldb + c] or
// B[c * ldb + m] (c < cmax); block (r, c) of C at C[c * ldc + r].
template <typename T>
struct Tile {
  const T *A, *B;
  T *C;
  int64_t lda, ldb, ldc;
  int rmax, cmax, mmax;
  bool sub;
};

// The product tiles t = t0, t0 + step, ... < tend given by desc(t), all with
// the same form of opB (TRB: B[c * ldb + m]).  The
// operands of the next tile are copied into the other shared buffer while the
// current one is multiplied, and the old values of C are loaded while the
// copies complete.
template <typename T, bool TRB, typename F>
__device__ __forceinline__ void tile_loop(T *sm, int t0, int step, int tend, F desc) {
  if (t0 >= tend) return;
  T *const buf0 = sm, *const buf1 = sm + 2 * kCb * kCs;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  __syncthreads();  // earlier users of the buffers are done
  {
    const Tile<T> d = desc(t0);
    cp64<T>(buf0, d.A, d.lda, false, d.rmax, d.mmax);
    cp64<T>(buf0 + kCb * kCs, d.B, d.ldb, TRB, d.cmax, d.mmax);
  }
  cp_commit();
  int i = 0;
  for (int t = t0; t < tend; t += step, ++i) {
    T *cur = (i & 1) ? buf1 : buf0;
    if (t + step < tend) {
      const Tile<T> e = desc(t + step);
      T *nxt = (i & 1) ? buf0 : buf1;
      cp64<T>(nxt, e.A, e.lda, false, e.rmax, e.mmax);
      cp64<T>(nxt + kCb * kCs, e.B, e.ldb, TRB, e.cmax, e.mmax);
    }
    cp_commit();
    const Tile<T> d = desc(t);
    // float32: the old values of C are loaded while the copies complete;
    // float64 (registers are short there): after the product.
    constexpr bool kEarly = sizeof(T) == 4;
    T old[4][4];
    auto load_old = [&]() {
#pragma unroll
      for (int v = 0; v < 4; ++v)
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int r = tx * 4 + u, c = ty * 4 + v;
          old[u][v] = (d.sub && r < d.rmax && c < d.cmax) ? d.C[(int64_t)c * d.ldc + r] : (T)0;
        }
    };
    if (kEarly) load_old();
    cp_wait<1>();
    __syncthreads();
    T acc[4][4];
    prod64<T>(cur, cur + kCb * kCs, acc);
    if (!kEarly) load_old();
#pragma unroll
    for (int v = 0; v < 4; ++v)
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int r = tx * 4 + u, c = ty * 4 + v;
        if (r < d.rmax && c < d.cmax) d.C[(int64_t)c * d.ldc + r] = d.sub ? old[u][v] - acc[u][v] : acc[u][v];
      }
    __syncthreads();  // `cur` is refilled by the next iteration's copies
  }
  cp_wait<0>();
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

// Cholesky factor and inverse of a 32 x 32 block by one warp, one column per
// step (right-looking).  Element (r, c) of the block is Bc[c * kDs + r]; lane
// r keeps the not yet eliminated part of row r in a[] and the pending part of
// column r of the inverse in x[], both shifted down by one place per step, so
// that every step has the same code (the loop is unrolled by kCholUnroll, which
// keeps the code small) and the published column is read with aligned vector
// loads.  Step c:
//   pivot d = a_cc (taken from lane c during the previous step), L_cc = sqrt d;
//   L_rc = a_rc / L_cc, published as Lt[c][r - c - 1] (shifted column);
//   a_rj -= L_rc L_jc (j > c); inverse column sweep x_c /= L_cc, x_j -= L_jc x_c.
// Column c of the factor replaces column c of the block (Bc[c * kDs + r],
// zero above the diagonal); element (c, r) of the inverse goes to
// Xb[r * kDs + c] (zero for c < r); rinv[c] = 1 / L_cc.  Lt rows must be
// finite beyond their written part (they are zeroed once).  Returns false when
// a pivot is not positive or not finite (the factor then continues with 1).
constexpr int kCholUnroll = 8;
template <typename T, int DS = kDs>
__device__ __forceinline__ bool warp_chol_inv32(T *Bc, T *Xb, T *Lt, T *rinv) {
  constexpr int kUnroll = sizeof(T) == 4 ? kCholUnroll : 1;  // float64: registers are short
  const int lane = threadIdx.x & 31;
  T a[32], x[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    a[j] = j <= lane ? Bc[j * DS + lane] : (T)0;
    x[j] = j == lane ? (T)1 : (T)0;
  }
  bool ok = true;
  T dg = __shfl_sync(0xffffffffu, a[0], 0);
#pragma unroll kUnroll
  for (int c = 0; c < 32; ++c) {
    const bool good = dg > (T)0 && isfinite(dg);
    ok = ok && good;
    T lc = (T)1, ri = (T)1;
    if (good) pivot(dg, lc, ri);
    const T v = lane == c ? lc : a[0] * ri;  // L_lane,c for lane >= c
    dg = __shfl_sync(0xffffffffu, fma(-v, v, a[1]), (c + 1) & 31);
    if (lane > c) Lt[c * kLts + lane - c - 1] = v;
    Bc[c * DS + lane] = lane >= c ? v : (T)0;
    const T xc = x[0] * ri;
    Xb[lane * DS + c] = xc;
    if (lane == 0) rinv[c] = ri;
    __syncwarp();
    const T ac = lane > c ? v : (T)0;
#pragma unroll
    for (int g = 0; g < 8; ++g) {
      T l4[4];
      Ld4<T>::load(Lt + c * kLts + 4 * g, l4);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int j = 4 * g + u;
        if (j < 31) {
          a[j] = fma(-ac, l4[u], a[j + 1]);
          x[j] = fma(-xc, l4[u], x[j + 1]);
        }
      }
    }
    a[31] = (T)0;
    x[31] = (T)0;
  }
  __syncwarp();
  return ok;
}

// out[u] = sum_{m < 32} A(r0 + u, m) B(c, m) for u < 4, with A(r, m) =
// Ab[m * lda + r] (rows contiguous, 16-byte aligned) and B(c, m) =
// Bb[c * sbc + m * sbm]; BV: B(c, m .. m+3) contiguous and aligned.
template <typename T, bool BV>
__device__ __forceinline__ void prod4x1(const T *Ab, int lda, int r0, const T *Bb, int sbc, int sbm, int c,
                                        T out[4]) {
#pragma unroll
  for (int u = 0; u < 4; ++u) out[u] = (T)0;
#pragma unroll 2
  for (int m0 = 0; m0 < 32; m0 += 4) {
    T b[4];
    if (BV) {
      Ld4<T>::load(Bb + c * sbc + m0, b);
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) b[q] = Bb[c * sbc + (m0 + q) * sbm];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      T a4[4];
      Ld4<T>::load(Ab + (m0 + q) * lda + r0, a4);
#pragma unroll
      for (int u = 0; u < 4; ++u) out[u] = fma(a4[u], b[q], out[u]);
    }
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
  uint64_t wait_ns;  // bound of one grid-barrier wait
};

// Shared-memory plan of the diagonal step (elements): Dc [64][kDs] the block
// (column-major: Dc[c * kDs + r]), Xc [64][kDs] its inverse (column-major),
// Tm [32][kDs], Lt [32][kLts], rinv [64].  The update operand is staged over
// Xc and Tm before they are used.
constexpr int kDiagSmem = 64 * kDs + 64 * kDs + 32 * kDs + 32 * kLts + 64;
// The warp that runs the 32 x 32 steps; warp 0 of CTA 0 also carries the grid
// barrier's atomics and was measured to run these steps several times slower.
constexpr int kDiagWarp = 7;

// Step A for panel k (one CTA).  With `upd`, the diagonal block first takes
// the update of panel k - 1, D = A_kk - L_k,k-1 L_k,k-1^T (the product is
// formed here, so the updated block never goes through global memory).  Then
// the block is factored and its factor inverted by the 2 x 2 block recursion
//   L11 = chol(D11), L21 = D21 Inv11^T, L22 = chol(D22 - L21 L21^T),
//   Inv21 = -Inv22 (L21 Inv11),
// the two 32 x 32 steps by one warp each while the other warps form the
// products that do not wait for them.  Rows/columns past n are padded with the
// identity.  Kept out of line: the per-lane register rows of the warp steps
// then stay in registers.
template <typename T>
__device__ __noinline__ void factor_diag(const CoopArgs<T> &a, int k, bool upd) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *sm = reinterpret_cast<T *>(smem_raw);
  T *Dc = sm, *Xc = sm + 64 * kDs, *Tm = Xc + 64 * kDs, *Lt = Tm + 32 * kDs, *rinv = Lt + 32 * kLts;
  const int64_t n = a.n, j0 = (int64_t)k * kCb;
  const int nb = (int)(n - j0 < kCb ? n - j0 : kCb);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  T *Ag = a.A + j0 * n + j0;  // the diagonal block in global memory
  __syncthreads();
  if (upd) {
    T *S = Xc;  // staging of L_k,k-1: S[m][r] = A(j0 + r, j0 - 64 + m)
    const int tx = tid & 15, ty = tid >> 4;
    T v[kPer], old[4][4];
    load64<T, false>(v, a.A + (j0 - kCb) * n + j0, n, nb, kCb);
#pragma unroll
    for (int vv = 0; vv < 4; ++vv)
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int r = tx * 4 + u, c = ty * 4 + vv;
        old[u][vv] = (r < nb && c < nb && r >= c) ? Ag[(int64_t)c * n + r] : (T)0;
      }
    store64<T, false>(S, v);
    for (int e = tid; e < 32 * kLts; e += kCoopThreads) Lt[e] = (T)0;
    __syncthreads();
    T acc[4][4];
    prod64<T>(S, S, acc);
#pragma unroll
    for (int vv = 0; vv < 4; ++vv) {
      T d[4];
      const int c = ty * 4 + vv;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int r = tx * 4 + u;
        d[u] = (r < nb && c < nb) ? (r >= c ? old[u][vv] - acc[u][vv] : (T)0) : (r == c ? (T)1 : (T)0);
      }
      Ld4<T>::store(Dc + c * kDs + tx * 4, d);
    }
  } else {
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int e = tid + u * kCoopThreads, c = e >> 6, r = e & 63;
      Dc[c * kDs + r] = (r < nb && c < nb) ? (r >= c ? Ag[(int64_t)c * n + r] : (T)0) : (r == c ? (T)1 : (T)0);
    }
    for (int e = tid; e < 32 * kLts; e += kCoopThreads) Lt[e] = (T)0;
  }
  __syncthreads();
  if (warp == kDiagWarp) {  // L11 and Inv11
    const bool ok = warp_chol_inv32<T>(Dc, Xc, Lt, rinv);
    if (!ok && lane == 0) atomicOr(a.status, a.bad_bit);
  }
  __syncthreads();
  const int r0 = 4 * warp;  // rows r0 .. r0 + 3 of the 32 x 32 products, column `lane`
  T o[4];
  // L21 = D21 Inv11^T: D21(r, m) = Dc[m * kDs + 32 + r], Inv11(c, m) = Xc[m * kDs + c]
  prod4x1<T, false>(Dc + 32, kDs, r0, Xc, 1, kDs, lane, o);
  __syncthreads();
  Ld4<T>::store(Dc + lane * kDs + 32 + r0, o);  // L21 over D21
  __syncthreads();
  // D22 -= L21 L21^T (column `lane` of D22, rows r0 .. r0 + 3)
  prod4x1<T, false>(Dc + 32, kDs, r0, Dc + 32, 1, kDs, lane, o);
  {
    T d[4];
    T *p = Dc + (32 + lane) * kDs + 32 + r0;
    Ld4<T>::load(p, d);
#pragma unroll
    for (int u = 0; u < 4; ++u) d[u] -= o[u];
    Ld4<T>::store(p, d);
  }
  __syncthreads();
  if (warp == kDiagWarp) {  // L22 and Inv22
    const bool ok = warp_chol_inv32<T>(Dc + 32 * kDs + 32, Xc + 32 * kDs + 32, Lt, rinv + 32);
    if (!ok && lane == 0) atomicOr(a.status, a.bad_bit);
  } else {
    // meanwhile Tm = L21 Inv11 (row-major Tm[r][c]); Inv11(m, c) = Xc[c * kDs + m]
    for (int g = warp; g < 8; g += 7) {
      prod4x1<T, true>(Dc + 32, kDs, 4 * g, Xc, kDs, 1, lane, o);
#pragma unroll
      for (int u = 0; u < 4; ++u) Tm[(4 * g + u) * kDs + lane] = o[u];
    }
  }
  __syncthreads();
  // Inv21 = -Inv22 Tm: Inv22(r, m) = Xc[(32 + m) * kDs + 32 + r], Tm(m, c) = Tm[m * kDs + c]
  prod4x1<T, false>(Xc + 32 * kDs + 32, kDs, r0, Tm, 1, kDs, lane, o);
#pragma unroll
  for (int u = 0; u < 4; ++u) o[u] = -o[u];
  Ld4<T>::store(Xc + lane * kDs + 32 + r0, o);
  __syncthreads();
  // L (lower triangle) and Inv_kk to global memory; with the inverse of the
  // whole factor, its diagonal block B_kk = Inv_kk as well.
  T *Dk = a.Dinv + (int64_t)k * kCb * kCb;
  T *Lik = a.Li ? a.Li + j0 * n + j0 : nullptr;
#pragma unroll
  for (int u = 0; u < kPer; ++u) {
    const int e = tid + u * kCoopThreads, cc = e >> 6, r = e & 63;
    const T iv = r >= cc ? Xc[cc * kDs + r] : (T)0;
    Dk[cc * kCb + r] = iv;
    if (r >= cc && r < nb) {
      Ag[(int64_t)cc * n + r] = Dc[cc * kDs + r];
      if (Lik) Lik[(int64_t)cc * n + r] = iv;
    }
  }
  for (int cc = tid; cc < nb; cc += kCoopThreads) a.dinv[j0 + cc] = rinv[cc];
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
  // diagonal factorisation (CTA 0) has the SM to itself; the other CTAs are
  // the workers, numbered densely.
  __shared__ int s_quiet, s_widx, s_nw;
  if (threadIdx.x == 0) {
    unsigned sid;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(sid));
    a.bar->smid[b] = (int)sid;
  }
  if (b == 0) factor_diag<T>(a, 0, false);
  if (!grid_sync(a.bar, 1, G, a.err, a.wait_ns)) return;
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
  const bool worker = s_nw > 0 && b != 0 && !s_quiet;
  // CTAs without trailing-update tiles only arrive at the barrier between the
  // panel step and the update (their panel rows are then released) and go on.
  const bool arrive_only = s_nw > 0 && !worker;
  auto rows = [&](int64_t r0) { return (int)(n - r0 < kCb ? n - r0 : kCb); };
  for (int k = 0; k < np; ++k) {
    const int64_t j0 = (int64_t)k * kCb;
    const int nbk = rows(j0);
    const T *Dk = a.Dinv + (int64_t)k * kCb * kCb;
    const int m = np - 1 - k;  // row blocks below the panel
    // ---- B: panel rows L_ik = A_ik Inv_kk^T and (inverse) B_kj = Inv_kk B_kj ----
    const int nB = m + (INV ? k : 0);
    auto bdesc = [&](int t) {
      Tile<T> d;
      if (t < m) {
        const int64_t r0 = (int64_t)(k + 1 + t) * kCb;
        d.A = a.A + j0 * n + r0; d.lda = n; d.rmax = rows(r0);
        d.B = Dk; d.ldb = kCb; d.cmax = nbk; d.mmax = nbk;
        d.C = a.A + j0 * n + r0; d.ldc = n; d.sub = false;
      } else {
        T *Bkj = a.Li + (int64_t)(t - m) * kCb * n + j0;  // opB(c, q) = B_kj(q, c)
        d.A = Dk; d.lda = kCb; d.rmax = nbk;
        d.B = Bkj; d.ldb = n; d.cmax = kCb; d.mmax = nbk;
        d.C = Bkj; d.ldc = n; d.sub = false;
      }
      return d;
    };
    // CTA 0 takes the first panel row block (the one the next diagonal step
    // needs), the workers the rest.
    // Panel rows (t < m, plain opB) and inverse rows (t >= m, transposed opB)
    // run as two loops.
    auto bsplit = [&](int t0, int step) {
      const int t1 = t0 < m ? t0 + (m - 1 - t0) / step * step + step : t0;  // first t >= m of the sequence
      tile_loop<T, false>(sm, t0, step, m < nB ? m : nB, bdesc);
      tile_loop<T, true>(sm, t1, step, nB, bdesc);
    };
    if (s_nw == 0) {
      if (b == 0) bsplit(0, 1);
    } else if (b == 0) {
      if (nB > 0) bsplit(0, nB);  // the first tile only
    } else if (worker) {
      bsplit(1 + s_widx, s_nw);
    }
    if (k == np - 1) break;
    if (!grid_sync(a.bar, 0, G, a.err, a.wait_ns, !arrive_only)) return;
    // ---- C: trailing update (and the inverse's rows below) ----
    const int U = m * (m + 1) / 2;
    const int nC = U + (INV ? m * (k + 1) : 0);
    auto cdesc = [&](int t) {
      Tile<T> d;
      if (t < U) {
        int bi, bj;
        tri_tile(t, bi, bj);
        const int64_t r0 = (int64_t)(k + 1 + bi) * kCb, c0 = (int64_t)(k + 1 + bj) * kCb;
        d.A = a.A + j0 * n + r0; d.lda = n; d.rmax = rows(r0);
        d.B = a.A + j0 * n + c0; d.ldb = n; d.cmax = rows(c0); d.mmax = kCb;
        d.C = a.A + c0 * n + r0; d.ldc = n; d.sub = true;
      } else {
        const int e = t - U;
        const int64_t r0 = (int64_t)(k + 1 + e / (k + 1)) * kCb, c0 = (int64_t)(e % (k + 1)) * kCb;
        // B_ij -= L_ik B_kj: opB(c, q) = B_kj(q, c)
        d.A = a.A + j0 * n + r0; d.lda = n; d.rmax = rows(r0);
        d.B = a.Li + c0 * n + j0; d.ldb = n; d.cmax = kCb; d.mmax = kCb;
        d.C = a.Li + c0 * n + r0; d.ldc = n; d.sub = true;
      }
      return d;
    };
    // Tile 0 is the next diagonal block: CTA 0 applies its update inside the
    // factorisation of that block (step A of panel k + 1); the workers take
    // the remaining tiles meanwhile.
    auto csplit = [&](int t0, int step) {
      const int t1 = t0 < U ? t0 + (U - 1 - t0) / step * step + step : t0;  // first t >= U of the sequence
      tile_loop<T, false>(sm, t0, step, U, cdesc);
      tile_loop<T, true>(sm, t1, step, nC, cdesc);
    };
    if (b == 0) factor_diag<T>(a, k + 1, true);
    if (s_nw == 0) {
      if (b == 0) csplit(1, 1);
    } else if (worker) {
      csplit(1 + s_widx, s_nw);
    }
    if (!grid_sync(a.bar, 1, G, a.err, a.wait_ns)) return;
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
  for (; i + 480 < i1; i += 512) {  // 16 loads of M and x in flight per lane (L2 latency)
    TM m[16];
    TX xv[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      m[u] = col[i + 32 * u];
      xv[u] = x[i + 32 * u];
    }
#pragma unroll
    for (int u = 0; u < 16; ++u) s[u & 3] = fma(m[u], (TM)xv[u], s[u & 3]);
  }
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

// ---------------------------------------------------------------------------
// Tensor-core factorisation for large n (launch_mixed_solve_tc).  Panels of
// kDp = 128 columns; per panel k (columns j0 = 128 k ...):
//   diagonal step (one CTA): factor and invert the diagonal block;
//   panel step (many CTAs):  the panel rows L(i, j0 + kk) for i >= j0 + 128,
//     stored only as the TF32 hi/lo operands Ph/Pl of the trailing update, and
//     the row block of the inverse B = L^{-1}: B_kj <- Inv_kk B_kj (j < k),
//     with its hi/lo copies Rh/Rl;
//   trailing update (tcgen05, syrk_tc.cu): F_ij -= L_ik L_jk^T (j > k) and
//     B_ij -= L_ik B_kj (i > k, j <= k).
// B is the block forward substitution L B = I carried along with the
// factorisation, as in the cooperative kernel above.
// Look-ahead: panel k's update is two launches, first the tiles that panel
// k + 1's diagonal and panel steps read (tile column k + 1 of the factor, tile
// row k + 1 of the inverse), then the rest on all but a few SMs, while a
// second stream runs panel k + 1's diagonal and panel steps beside it.  The
// panel buffers (Ph, Pl, Rh, Rl) come in two sets, by panel parity.
// ---------------------------------------------------------------------------
constexpr int kDp = kCholPanel;  // panel width = diagonal block edge
constexpr int kCholReserve = 8;  // SMs kept free for the look-ahead's diagonal and panel steps
constexpr int kDd = kDp + 4;     // shared stride of the diagonal step's arrays
constexpr size_t kDiag128Smem = (size_t)(2 * kDp * kDd + 32 * kLts + kDp) * sizeof(float);
constexpr int kPr = 64;          // panel step: rows (or inverse columns) per item
constexpr int kPs = kPr + 4;     // shared stride of the operand chunk
constexpr size_t kPanelSmem = (size_t)(kDp * kDd + kDp * kPs) * sizeof(float);

// x = hi + lo with hi, lo rounded to TF32 (lo carries the bits hi drops).
__device__ __forceinline__ void tf32_split(float x, float &hi, float &lo) {
  uint32_t h, l;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
  hi = __uint_as_float(h);
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(x - hi));
  lo = __uint_as_float(l);
}

// Diagonal step of panel k: D = F(j0.., j0..) (already updated by the earlier
// panels; identity past n) is factored D = L L^T and L inverted in four
// 32-column steps.  Step b (j = 32 b): one warp factors and inverts the 32 x 32
// diagonal block (warp_chol_inv32); then the rows below, L_ib = D_ib Inv_bb^T,
// and the inverse's row block X_b,: = Inv_bb W_b,: (W: the accumulated
// right-hand side, zero at first); then the trailing part of the block,
// D_ij -= L_ib L_jb^T, and W_i,: -= L_ib X_b,: for the rows below.
// Writes InvT[m][r] = Inv(r, m), the diagonal block of L^{-1} into Li, and its
// hi/lo rows Rh/Rl[j0 + c][r] = Inv(r, c).  status |= bad_bit on a pivot that
// is not positive.
__global__ void __launch_bounds__(256, 1) chol_diag128_kernel(const float *__restrict__ F32, int64_t ld, int64_t n,
                                                              int k, float *__restrict__ Li, float *__restrict__ InvT,
                                                              float *__restrict__ Rh, float *__restrict__ Rl,
                                                              int *status, int bad_bit) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float *D = reinterpret_cast<float *>(smem_raw);  // D[c * kDd + r] = element (r, c)
  float *X = D + kDp * kDd;                        // the inverse, same layout
  float *Lt = X + kDp * kDd;                       // [32][kLts], warp-step scratch
  float *rinv = Lt + 32 * kLts;                    // [128]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t j0 = (int64_t)k * kDp;
  const int nb = (int)(n - j0 < kDp ? n - j0 : kDp);
  // Loads in batches of 16 per thread, unconditional (an element outside the
  // block's lower triangle reads the diagonal's first element instead and is
  // replaced afterwards), so that they are all in flight at once.
  for (int u0 = 0; u0 < kDp * kDp / 256; u0 += 16) {
    float v[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int e = tid + 256 * (u0 + u), c = e >> 7, r = e & 127;
      const bool in = r < nb && c < nb && r >= c;
      v[u] = F32[in ? (j0 + c) * ld + j0 + r : j0 * ld + j0];
    }
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int e = tid + 256 * (u0 + u), c = e >> 7, r = e & 127;
      D[c * kDd + r] = (r < nb && c < nb) ? (r >= c ? v[u] : 0.f) : (r == c ? 1.f : 0.f);
      X[c * kDd + r] = 0.f;
    }
  }
  for (int e = tid; e < 32 * kLts; e += 256) Lt[e] = 0.f;
  __syncthreads();
  for (int b = 0; b < 4; ++b) {
    const int j = 32 * b, nr = kDp - j - 32;  // rows below the step
    if (warp == kDiagWarp) {
      const bool ok = warp_chol_inv32<float, kDd>(D + j * kDd + j, X + j * kDd + j, Lt, rinv + j);
      if (!ok && lane == 0) atomicOr(status, bad_bit);
    }
    __syncthreads();
    // Rows below: strips of 4 rows (r) with column j + lane.  Inverse row
    // block: strips of 4 rows j + r' with columns c' < j (lanes, groups of 32).
    const int nsa = nr / 4, nsb = j / 32 * 8;
    float oa[3][4], ob[3][4];
    int na = 0, nbk = 0;
    for (int t = warp; t < nsa; t += 8, ++na) {
      const int r = j + 32 + 4 * t;
      float o[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 8
      for (int m = 0; m < 32; ++m) {
        const float iv = X[(j + m) * kDd + j + lane];  // Inv_bb(lane, m)
        const float4 d4 = *reinterpret_cast<const float4 *>(D + (j + m) * kDd + r);
        o[0] = fmaf(d4.x, iv, o[0]); o[1] = fmaf(d4.y, iv, o[1]);
        o[2] = fmaf(d4.z, iv, o[2]); o[3] = fmaf(d4.w, iv, o[3]);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) oa[na][u] = o[u];
    }
    for (int t = warp; t < nsb; t += 8, ++nbk) {
      const int rp = 4 * (t & 7), cp = 32 * (t >> 3) + lane;
      float o[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 8
      for (int m = 0; m < 32; ++m) {
        const float w = X[cp * kDd + j + m];  // W(j + m, cp)
        const float4 i4 = *reinterpret_cast<const float4 *>(X + (j + m) * kDd + j + rp);  // Inv_bb(rp.., m)
        o[0] = fmaf(i4.x, w, o[0]); o[1] = fmaf(i4.y, w, o[1]);
        o[2] = fmaf(i4.z, w, o[2]); o[3] = fmaf(i4.w, w, o[3]);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) ob[nbk][u] = o[u];
    }
    __syncthreads();
    na = 0;
    for (int t = warp; t < nsa; t += 8, ++na) {
      const int r = j + 32 + 4 * t;
#pragma unroll
      for (int u = 0; u < 4; ++u) D[(j + lane) * kDd + r + u] = oa[na][u];
    }
    nbk = 0;
    for (int t = warp; t < nsb; t += 8, ++nbk) {
      const int rp = 4 * (t & 7), cp = 32 * (t >> 3) + lane;
#pragma unroll
      for (int u = 0; u < 4; ++u) X[cp * kDd + j + rp + u] = ob[nbk][u];
    }
    __syncthreads();
    if (nr > 0) {
      // Trailing part: 32 x 32 blocks (RB >= CB) of the nr x nr lower part, in strips of 8 rows;
      // inverse: strips of 8 rows below with 32-column groups of the first j + 32 columns.
      const int nrb = nr / 32;
      const int nc = nrb * (nrb + 1) / 2 * 4, nd = (nr / 8) * (j / 32 + 1);
      for (int t = warp; t < nc + nd; t += 8) {
        float o[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (t < nc) {
          const int pr = t >> 2, strip = t & 3;
          int RB = 0;
          while ((RB + 1) * (RB + 2) / 2 <= pr) ++RB;
          const int CB = pr - RB * (RB + 1) / 2;
          const int r = j + 32 + 32 * RB + 8 * strip, c = j + 32 + 32 * CB + lane;
#pragma unroll 8
          for (int m = 0; m < 32; ++m) {
            const float lc = D[(j + m) * kDd + c];
            const float4 a = *reinterpret_cast<const float4 *>(D + (j + m) * kDd + r);
            const float4 b4 = *reinterpret_cast<const float4 *>(D + (j + m) * kDd + r + 4);
            o[0] = fmaf(a.x, lc, o[0]); o[1] = fmaf(a.y, lc, o[1]); o[2] = fmaf(a.z, lc, o[2]);
            o[3] = fmaf(a.w, lc, o[3]); o[4] = fmaf(b4.x, lc, o[4]); o[5] = fmaf(b4.y, lc, o[5]);
            o[6] = fmaf(b4.z, lc, o[6]); o[7] = fmaf(b4.w, lc, o[7]);
          }
#pragma unroll
          for (int u = 0; u < 8; ++u)
            if (c <= r + u) D[c * kDd + r + u] -= o[u];
        } else {
          const int e = t - nc, strip = e % (nr / 8), cg = e / (nr / 8);
          const int r = j + 32 + 8 * strip, c = 32 * cg + lane;
#pragma unroll 8
          for (int m = 0; m < 32; ++m) {
            const float xv = X[c * kDd + j + m];
            const float4 a = *reinterpret_cast<const float4 *>(D + (j + m) * kDd + r);
            const float4 b4 = *reinterpret_cast<const float4 *>(D + (j + m) * kDd + r + 4);
            o[0] = fmaf(a.x, xv, o[0]); o[1] = fmaf(a.y, xv, o[1]); o[2] = fmaf(a.z, xv, o[2]);
            o[3] = fmaf(a.w, xv, o[3]); o[4] = fmaf(b4.x, xv, o[4]); o[5] = fmaf(b4.y, xv, o[5]);
            o[6] = fmaf(b4.z, xv, o[6]); o[7] = fmaf(b4.w, xv, o[7]);
          }
#pragma unroll
          for (int u = 0; u < 8; ++u) X[c * kDd + r + u] -= o[u];
        }
      }
      __syncthreads();
    }
  }
  float *Ik = InvT + (int64_t)k * kDp * kDp;
  for (int e = tid; e < kDp * kDp; e += 256) {
    const int c = e >> 7, r = e & 127;
    const float v = X[c * kDd + r];  // zero above the diagonal
    Ik[e] = v;                       // InvT[c][r] = Inv(r, c)
    if (r >= c && r < nb && c < nb) Li[(j0 + c) * ld + j0 + r] = v;
    float hi, lo;
    tf32_split(v, hi, lo);
    Rh[(j0 + c) * kDp + r] = hi;
    Rl[(j0 + c) * kDp + r] = lo;
  }
}

// Panel step of panel k, items of 64 rows ((a), i >= j0 + 128, up to n_pad)
// or 64 columns ((b), c < j0), each a 64 x 128 product with the inverse of
// the diagonal block (lower triangular: Inv(kk, m) = 0 for m > kk):
//   (a) L(i, j0 + kk) = sum_m F(i, j0 + m) Inv(kk, m) -> Ph/Pl[i][kk] (zero rows past n);
//   (b) B(j0 + kk, c) <- sum_m Inv(kk, m) B(j0 + m, c) in Li, and Rh/Rl[c][kk].
__global__ void __launch_bounds__(256, 2) chol_panel_kernel(const float *__restrict__ F32, int64_t ld, int64_t n,
                                                            int64_t n_pad, int k, float *__restrict__ Li,
                                                            const float *__restrict__ InvT, float *__restrict__ Ph,
                                                            float *__restrict__ Pl, float *__restrict__ Rh,
                                                            float *__restrict__ Rl) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float *Is = reinterpret_cast<float *>(smem_raw);  // Is[m * kDd + kk] = Inv(kk, m)
  float *Os = Is + kDp * kDd;                        // Os[m * kPs + x]: operand chunk
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t j0 = (int64_t)k * kDp, r_begin = j0 + kDp;
  const int na = (int)((n_pad - r_begin) / kPr), nbi = (int)(j0 / kPr);
  const float *Ik = InvT + (int64_t)k * kDp * kDp;
#pragma unroll 16
  for (int u = 0; u < kDp * kDp / 256; ++u) {
    const int e = tid + 256 * u;
    Is[(e >> 7) * kDd + (e & 127)] = Ik[e];
  }
  const int mend = 8 * ty + 8;  // Inv(kk, m) = 0 for m > kk >= 8 ty + 7
  for (int item = blockIdx.x; item < na + nbi; item += gridDim.x) {
    const bool rows = item < na;
    const int64_t x0 = rows ? r_begin + (int64_t)item * kPr : (int64_t)(item - na) * kPr;
    __syncthreads();  // Is is loaded; the previous item is done with Os
    // batches of 16 unconditional loads per thread (out-of-range elements read
    // element (j0, 0) of the operand and are replaced by zero)
    const float *src = rows ? F32 : Li;
    for (int u0 = 0; u0 < kDp * kPr / 256; u0 += 16) {
      float v[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int e = tid + 256 * (u0 + u);
        const int m = rows ? e >> 6 : e & 127, x = rows ? e & 63 : e >> 7;
        const bool in = rows ? (x0 + x < n && j0 + m < n) : j0 + m < n;
        v[u] = src[in ? (rows ? (j0 + m) * ld + x0 + x : (x0 + x) * ld + j0 + m) : j0];
      }
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int e = tid + 256 * (u0 + u);
        const int m = rows ? e >> 6 : e & 127, x = rows ? e & 63 : e >> 7;
        const bool in = rows ? (x0 + x < n && j0 + m < n) : j0 + m < n;
        Os[m * kPs + x] = in ? v[u] : 0.f;
      }
    }
    __syncthreads();
    float acc[4][8];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 8; ++v) acc[u][v] = 0.f;
#pragma unroll 4
    for (int m = 0; m < mend; ++m) {
      const float4 a = *reinterpret_cast<const float4 *>(Os + m * kPs + 4 * tx);
      const float4 b0 = *reinterpret_cast<const float4 *>(Is + m * kDd + 8 * ty);
      const float4 b1 = *reinterpret_cast<const float4 *>(Is + m * kDd + 8 * ty + 4);
      const float av[4] = {a.x, a.y, a.z, a.w};
      const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 8; ++v) acc[u][v] = fmaf(av[u], bv[v], acc[u][v]);
    }
    if (rows) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        float h[8], l[8];
#pragma unroll
        for (int v = 0; v < 8; ++v) tf32_split(acc[u][v], h[v], l[v]);
        const int64_t o = (x0 + 4 * tx + u) * kDp + 8 * ty;
        *reinterpret_cast<float4 *>(Ph + o) = make_float4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<float4 *>(Ph + o + 4) = make_float4(h[4], h[5], h[6], h[7]);
        *reinterpret_cast<float4 *>(Pl + o) = make_float4(l[0], l[1], l[2], l[3]);
        *reinterpret_cast<float4 *>(Pl + o + 4) = make_float4(l[4], l[5], l[6], l[7]);
      }
    } else {
      // through shared memory (Os reused as Res[x * kDd + kk]) so that the column writes are coalesced
      __syncthreads();
      float *Res = Os;
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 8; ++v) Res[(4 * tx + u) * kDd + 8 * ty + v] = acc[u][v];
      __syncthreads();
      for (int e = tid; e < kPr * kDp; e += 256) {
        const int x = e >> 7, kk = e & 127;
        const float v = Res[x * kDd + kk];
        if (j0 + kk < n) Li[(x0 + x) * ld + j0 + kk] = v;
        float hi, lo;
        tf32_split(v, hi, lo);
        Rh[(x0 + x) * kDp + kk] = hi;
        Rl[(x0 + x) * kDp + kk] = lo;
      }
    }
  }
}

// Refinement from the explicit inverse Li (lower triangle; mirrored here):
// delta_0 = L^{-T} L^{-1} g, then `iters` steps of r = g - F delta (float64),
// delta += L^{-T} L^{-1} r.  Returns the number of launches.
int refine_with_inverse(int64_t n, const double *F, float *Li, const double *g, double *delta, float *y, float *z,
                        double *r, double *ref, int *status, int iters, cudaStream_t st) {
  const unsigned nt = (unsigned)((n + 31) / 32);
  mirror_lower_kernel<float><<<dim3(nt, nt), dim3(32, 8), 0, st>>>(n, Li);
  const unsigned gb = (unsigned)((n + 7) / 8);
  gemv_col_kernel<float, double, float, 0><<<gb, 256, 0, st>>>(n, Li, g, y, nullptr, nullptr);
  gemv_col_kernel<float, float, float, 1><<<gb, 256, 0, st>>>(n, Li, y, z, nullptr, nullptr);
  refine_update_kernel<<<1, 1024, 0, st>>>(n, z, delta, ref, status, 1);
  int cnt = 4;
  for (int it = 0; it < iters; ++it) {
    gemv_col_kernel<double, double, double, 2><<<gb, 256, 0, st>>>(n, F, delta, r, g, ref);  // r = g - F delta
    gemv_col_kernel<float, double, float, 0><<<gb, 256, 0, st>>>(n, Li, r, y, nullptr, ref);
    gemv_col_kernel<float, float, float, 1><<<gb, 256, 0, st>>>(n, Li, y, z, nullptr, ref);
    refine_update_kernel<<<1, 1024, 0, st>>>(n, z, delta, ref, status, 0);
    cnt += 4;
  }
  refine_check_kernel<<<1, 1, 0, st>>>(ref, status);
  return cnt + 1;
}

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

int64_t panels(int64_t n) { return (n + kCb - 1) / kCb; }

template <typename T, bool INV>
cudaError_t launch_coop(int64_t n, T *A, T *Li, T *Dinv, T *dinv, GridBarrier *bar, int *status, int bad_bit,
                        int *err, cudaStream_t st, uint64_t wait_ns) {
  auto kern = coop_cholesky_kernel<T, INV>;
  const size_t smem = (size_t)std::max(kDiagSmem, 4 * kCb * kCs) * sizeof(T);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, nsm = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kCoopThreads, smem)) != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int grid = std::min(nsm * std::min(per_sm, 2), kMaxCoopGrid);
  if ((e = cudaMemsetAsync(bar, 0, sizeof(GridBarrier), st)) != cudaSuccess) return e;
  CoopArgs<T> a{};
  a.A = A; a.Li = Li; a.Dinv = Dinv; a.dinv = dinv; a.n = n; a.bar = bar;
  a.status = status; a.bad_bit = bad_bit; a.err = err;
  a.wait_ns = wait_ns ? wait_ns : kWaitNs;
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

// Standard errors: se_j = sqrt((F^{-1})_jj) = the norm of column j of L^{-1}
// (F^{-1} = L^{-T} L^{-1}), one warp per column (contiguous, rows j .. n-1).
__global__ void __launch_bounds__(256) column_norms_kernel(int64_t n, const double *__restrict__ B,
                                                           const int *__restrict__ status, double *__restrict__ se) {
  const int lane = threadIdx.x & 31;
  const int64_t j = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (j >= n) return;
  double s = 0.0;
  for (int64_t i = j + lane; i < n; i += 32) {
    const double b = B[j * n + i];
    s = fma(b, b, s);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) se[j] = (*status & 4) ? nan("") : sqrt(s);
}

}  // namespace

size_t chol_work_bytes(int64_t n) {
  return round256((size_t)panels(n) * kCb * kCb * 8) + round256(sizeof(GridBarrier));
}

int cholesky_launches(int64_t) { return 1; }

cudaError_t launch_cholesky(int64_t n, double *F, double *dinv, void *work, int *status, int *err, cudaStream_t st,
                            uint64_t wait_ns) {
  unsigned char *w = static_cast<unsigned char *>(work);
  double *Dinv = reinterpret_cast<double *>(w);
  GridBarrier *bar = reinterpret_cast<GridBarrier *>(w + round256((size_t)panels(n) * kCb * kCb * 8));
  return launch_coop<double, false>(n, F, nullptr, Dinv, dinv, bar, status, 4, err, st, wait_ns);
}

cudaError_t launch_std_errors(int64_t n, double *F, double *Binv, double *dinv, void *work, int *status, int *err,
                              double *se, cudaStream_t st, uint64_t wait_ns) {
  unsigned char *w = static_cast<unsigned char *>(work);
  double *Dinv = reinterpret_cast<double *>(w);
  GridBarrier *bar = reinterpret_cast<GridBarrier *>(w + round256((size_t)panels(n) * kCb * kCb * 8));
  cudaError_t e = cudaMemsetAsync(Binv, 0, (size_t)n * n * 8, st);
  if (e != cudaSuccess) return e;
  if ((e = launch_coop<double, true>(n, F, Binv, Dinv, dinv, bar, status, 4, err, st, wait_ns)) != cudaSuccess)
    return e;
  column_norms_kernel<<<(unsigned)((n + 7) / 8), 256, 0, st>>>(n, Binv, status, se);
  return cudaGetLastError();
}

cudaError_t launch_f64_to_f32_lower(int64_t n, const double *F, float *F32, cudaStream_t st) {
  dim3 grid((unsigned)((n + 255) / 256), (unsigned)std::min<int64_t>(n, 65535), (unsigned)((n + 65534) / 65535));
  f64_to_f32_lower_kernel<<<grid, 256, 0, st>>>(n, F, F32);
  return cudaGetLastError();
}

size_t mixed_solve_bytes(int64_t n) { return mixed_layout(n).total; }

double *mixed_solve_ref(void *work, int64_t n) {
  return reinterpret_cast<double *>(static_cast<unsigned char *>(work) + mixed_layout(n).ref);
}

cudaError_t launch_mixed_solve(int64_t n, const double *F, float *F32, const double *g, double *delta, void *work,
                               int *status, int *err, int iters, cudaStream_t st, int *launches, bool f32_ready,
                               uint64_t wait_ns) {
  const MixedLayout L = mixed_layout(n);
  unsigned char *w = static_cast<unsigned char *>(work);
  float *Li = reinterpret_cast<float *>(w + L.li), *Dblk = reinterpret_cast<float *>(w + L.dblk);
  float *dinv = reinterpret_cast<float *>(w + L.dinv), *y = reinterpret_cast<float *>(w + L.y);
  float *z = reinterpret_cast<float *>(w + L.z);
  double *r = reinterpret_cast<double *>(w + L.r), *ref = reinterpret_cast<double *>(w + L.ref);
  GridBarrier *bar = reinterpret_cast<GridBarrier *>(w + L.bar);
  cudaError_t e;
  dim3 grid((unsigned)((n + 255) / 256), (unsigned)std::min<int64_t>(n, 65535), (unsigned)((n + 65534) / 65535));
  if (!f32_ready) f64_to_f32_lower_kernel<<<grid, 256, 0, st>>>(n, F, F32);
  if ((e = cudaMemsetAsync(Li, 0, (size_t)n * n * 4, st)) != cudaSuccess) return e;
  if ((e = launch_coop<float, true>(n, F32, Li, Dblk, dinv, bar, status, 8, err, st, wait_ns)) != cudaSuccess)
    return e;
  const int cnt = (f32_ready ? 1 : 2) + refine_with_inverse(n, F, Li, g, delta, y, z, r, ref, status, iters, st);
  if (launches) *launches = cnt;
  return cudaGetLastError();
}

size_t tc_chol_bytes(int64_t n) {
  const int64_t np = (n + kDp - 1) / kDp, n_pad = np * kDp;
  int64_t units = 0;
  for (int64_t k = 0; k + 1 < np; ++k) {
    const int64_t m = np - 1 - k;
    units += m * (m + 1) / 2 + m * (k + 1);
  }
  return round256(8 * sizeof(CUtensorMap)) + 8 * round256((size_t)n_pad * kDp * 4) +
         round256((size_t)np * kDp * kDp * 4) + round256((size_t)units * sizeof(CholUnit));
}

void tc_chol_release(TcCholPlan *P) {
  if (P->side) cudaStreamDestroy(P->side);
  for (cudaEvent_t *e : {&P->ev_start, &P->ev_next, &P->ev_panel})
    if (*e) cudaEventDestroy(*e);
  P->side = nullptr;
  P->ev_start = P->ev_next = P->ev_panel = nullptr;
  P->ready = false;
}

cudaError_t tc_chol_prepare(int64_t n, void *ws, int num_sms, TcCholPlan *P) {
  P->ready = false;
  P->n = n;
  P->np = (int)((n + kDp - 1) / kDp);
  P->n_pad = (int64_t)P->np * kDp;
  P->ws = ws;
  unsigned char *w = static_cast<unsigned char *>(ws);
  size_t o = 0;
  P->maps = reinterpret_cast<CUtensorMap *>(w + o); o += round256(8 * sizeof(CUtensorMap));
  float **bufs[8] = {&P->Ph[0], &P->Pl[0], &P->Rh[0], &P->Rl[0], &P->Ph[1], &P->Pl[1], &P->Rh[1], &P->Rl[1]};
  for (float **b : bufs) { *b = reinterpret_cast<float *>(w + o); o += round256((size_t)P->n_pad * kDp * 4); }
  P->InvT = reinterpret_cast<float *>(w + o); o += round256((size_t)P->np * kDp * kDp * 4);
  P->units = reinterpret_cast<CholUnit *>(w + o);
  // Per panel k: first the units that the diagonal and panel steps of panel k + 1
  // read (tile column k + 1 of the factor, tile row k + 1 of the inverse), then the rest.
  std::vector<CholUnit> u;
  P->unit_off.assign(1, 0);
  P->unit_mid.clear();
  for (int k = 0; k + 1 < P->np; ++k) {
    const int k1 = k + 1;
    for (int ti = k1; ti < P->np; ++ti) u.push_back(CholUnit{ti, k1, 0, 0, ti == k1 ? 1 : 0, 0});
    for (int tj = 0; tj <= k; ++tj) u.push_back(CholUnit{k1, tj, 1, 1, 0, 0});
    P->unit_mid.push_back((int)u.size());
    for (int ti = k1 + 1; ti < P->np; ++ti)
      for (int tj = k1 + 1; tj <= ti; ++tj) u.push_back(CholUnit{ti, tj, 0, 0, ti == tj ? 1 : 0, 0});
    for (int ti = k1 + 1; ti < P->np; ++ti)
      for (int tj = 0; tj <= k; ++tj) u.push_back(CholUnit{ti, tj, 1, 1, 0, 0});
    P->unit_off.push_back((int)u.size());
  }
  CUtensorMap hm[8];
  cudaError_t e;
  for (int i = 0; i < 8; ++i)
    if ((e = encode_rows_map(*bufs[i], P->n_pad, kDp, &hm[i])) != cudaSuccess) return e;
  if ((e = cudaMemcpy(P->maps, hm, sizeof(hm), cudaMemcpyHostToDevice)) != cudaSuccess) return e;
  if (!u.empty() && (e = cudaMemcpy(P->units, u.data(), u.size() * sizeof(CholUnit), cudaMemcpyHostToDevice)) !=
                        cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(chol_diag128_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kDiag128Smem)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(chol_panel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kPanelSmem)) != cudaSuccess)
    return e;
  if ((e = chol_update_tc_setup()) != cudaSuccess) return e;
  if ((e = cudaStreamCreateWithFlags(&P->side, cudaStreamNonBlocking)) != cudaSuccess) return e;
  for (cudaEvent_t *ev : {&P->ev_start, &P->ev_next, &P->ev_panel})
    if ((e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming)) != cudaSuccess) return e;
  P->grid = num_sms;
  P->reserve = std::min(kCholReserve, num_sms / 4);
  P->ready = true;
  return cudaSuccess;
}

cudaError_t launch_mixed_solve_tc(const TcCholPlan &P, const double *F, float *F32, const double *g, double *delta,
                                  void *work, int *status, int *err, int iters, uint64_t wait_ns, cudaStream_t st,
                                  int *launches) {
  if (!P.ready) return cudaErrorInvalidValue;
  const int64_t n = P.n;
  const MixedLayout L = mixed_layout(n);
  unsigned char *w = static_cast<unsigned char *>(work);
  float *Li = reinterpret_cast<float *>(w + L.li), *y = reinterpret_cast<float *>(w + L.y);
  float *z = reinterpret_cast<float *>(w + L.z);
  double *r = reinterpret_cast<double *>(w + L.r), *ref = reinterpret_cast<double *>(w + L.ref);
  cudaError_t e;
  if ((e = cudaMemsetAsync(Li, 0, (size_t)n * n * 4, st)) != cudaSuccess) return e;
  int cnt = 0;
  // Diagonal and panel steps of panel k on stream s, into the buffers of parity k & 1.
  auto diag_panel = [&](int k, cudaStream_t s) {
    const int b = k & 1;
    chol_diag128_kernel<<<1, 256, kDiag128Smem, s>>>(F32, n, n, k, Li, P.InvT, P.Rh[b], P.Rl[b], status, 8);
    const int64_t j0 = (int64_t)k * kDp;
    const int items = (int)((P.n_pad - j0 - kDp) / kPr + j0 / kPr);
    if (items > 0)
      chol_panel_kernel<<<std::min(items, 2 * P.grid), 256, kPanelSmem, s>>>(F32, n, n, P.n_pad, k, Li, P.InvT,
                                                                            P.Ph[b], P.Pl[b], P.Rh[b], P.Rl[b]);
    cnt += items > 0 ? 2 : 1;
  };
  // Look-ahead: while the bulk of panel k's trailing update runs on st (on all
  // but `reserve` SMs), the side stream factors the diagonal block of panel
  // k + 1 and forms its panel, as soon as the few update tiles they read are
  // done.  The panel buffers alternate between two sets so that panel k + 1's
  // are written while panel k's are still read.
  if ((e = cudaEventRecord(P.ev_start, st)) != cudaSuccess) return e;
  if ((e = cudaStreamWaitEvent(P.side, P.ev_start, 0)) != cudaSuccess) return e;
  diag_panel(0, P.side);
  if ((e = cudaEventRecord(P.ev_panel, P.side)) != cudaSuccess) return e;
  for (int k = 0; k + 1 < P.np; ++k) {
    const CUtensorMap *maps = P.maps + 4 * (k & 1);
    const int u0 = P.unit_off[(size_t)k], um = P.unit_mid[(size_t)k], u1 = P.unit_off[(size_t)k + 1];
    if ((e = cudaStreamWaitEvent(st, P.ev_panel, 0)) != cudaSuccess) return e;
    if ((e = launch_chol_update_tc(maps, P.units + u0, um - u0, std::min(um - u0, P.grid), F32, Li, n, n, err,
                                   wait_ns, st)) != cudaSuccess)
      return e;
    if ((e = cudaEventRecord(P.ev_next, st)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(P.side, P.ev_next, 0)) != cudaSuccess) return e;
    diag_panel(k + 1, P.side);
    if ((e = cudaEventRecord(P.ev_panel, P.side)) != cudaSuccess) return e;
    if (u1 > um) {
      if ((e = launch_chol_update_tc(maps, P.units + um, u1 - um, std::max(1, std::min(u1 - um, P.grid - P.reserve)),
                                     F32, Li, n, n, err, wait_ns, st)) != cudaSuccess)
        return e;
      ++cnt;
    }
    ++cnt;
  }
  if ((e = cudaStreamWaitEvent(st, P.ev_panel, 0)) != cudaSuccess) return e;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  cnt += refine_with_inverse(n, F, Li, g, delta, y, z, r, ref, status, iters, st);
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
