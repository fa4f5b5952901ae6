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
__device__ bool grid_sync(GridBarrier *b, int w, unsigned nblocks, int *err, bool wait = true) {
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
template <typename T>
__device__ __forceinline__ bool warp_chol_inv32(T *Bc, T *Xb, T *Lt, T *rinv) {
  constexpr int kUnroll = sizeof(T) == 4 ? kCholUnroll : 1;  // float64: registers are short
  const int lane = threadIdx.x & 31;
  T a[32], x[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    a[j] = j <= lane ? Bc[j * kDs + lane] : (T)0;
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
    Bc[c * kDs + lane] = lane >= c ? v : (T)0;
    const T xc = x[0] * ri;
    Xb[lane * kDs + c] = xc;
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
  if (!grid_sync(a.bar, 1, G, a.err)) return;
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
    if (!grid_sync(a.bar, 0, G, a.err, !arrive_only)) return;
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
    if (!grid_sync(a.bar, 1, G, a.err)) return;
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

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

int64_t panels(int64_t n) { return (n + kCb - 1) / kCb; }

template <typename T, bool INV>
cudaError_t launch_coop(int64_t n, T *A, T *Li, T *Dinv, T *dinv, GridBarrier *bar, int *status, int bad_bit,
                        int *err, cudaStream_t st) {
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
                               int *status, int *err, int iters, cudaStream_t st, int *launches, bool f32_ready) {
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
  if ((e = launch_coop<float, true>(n, F32, Li, Dblk, dinv, bar, status, 8, err, st)) != cudaSuccess) return e;
  const unsigned nt = (unsigned)((n + 31) / 32);
  mirror_lower_kernel<float><<<dim3(nt, nt), dim3(32, 8), 0, st>>>(n, Li);
  const unsigned gb = (unsigned)((n + 7) / 8);
  // delta_0 = L^{-T} (L^{-1} g)
  gemv_col_kernel<float, double, float, 0><<<gb, 256, 0, st>>>(n, Li, g, y, nullptr, nullptr);
  gemv_col_kernel<float, float, float, 1><<<gb, 256, 0, st>>>(n, Li, y, z, nullptr, nullptr);
  refine_update_kernel<<<1, 1024, 0, st>>>(n, z, delta, ref, status, 1);
  int cnt = f32_ready ? 6 : 7;
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
