// Structured negative Hessian F = -H (Sec. 3.3, eq. "hessian block"; App. A).
//
// With W_nm = diag(P_n (delta_nm - P_m)) and M_k = [X, Y_k] (q = p + d columns):
//   class blocks, n != m:  F_nm = (P_n o M_n)^T (P_m o M_m)       -> one SYRK over
//                          A = [P_1 o M_1 | ... | P_{K-1} o M_{K-1}]  (N x (K-1)q)
//   class blocks, n == m:  F_nn = M_n^T diag(P_n (1 - P_n)) M_n   -> the same SYRK over
//                          Ad = [sqrt(P_k (1-P_k)) o M_k], restricted to the diagonal
//                          class blocks (no cancellation when P_nk is close to 1)
//   cross blocks:          F_{n,alpha} = sum_i P_in m_in (z_in - zbar_i)^T
//   alpha block:           F_aa = sum_i sum_k P_ik (z_ik - zbar_i)(z_ik - zbar_i)^T
// with zbar_i = sum_k P_ik z_ik from the pass (the centred form of App. A's
// alpha-alpha derivation, with raw Z: a per-row shift of Z cancels).
#include <cuda_bf16.h>

#include "mnl_internal.cuh"

namespace mnl {
namespace {

// ---------------------------------------------------------------------------
// Operand builder: At[c][i] = P_ik m_ik[l], Ad[c][i] = sqrt(P_ik(1-P_ik)) m_ik[l]
// ---------------------------------------------------------------------------

// Rounding of the operands.  TF32 rounds to nearest (cvt.rna).  BF16 rounds
// stochastically: the 16 discarded bits of the float32 value are replaced by
// a uniform random draw before truncation, so the rounded value is unbiased.
// With round-to-nearest, designs in which many observations share the same
// P_ik (an intercept-only model, indicator columns) would give every product
// the same rounding error; unbiased rounding turns that into independent
// errors that average out over the observations.  The random bits are a hash
// of (operand, column, observation pair), so results are reproducible.
template <OpType OT>
struct OpStore;
template <>
struct OpStore<OpType::F64> {
  using CT = double;
  __device__ static void put(void *base, int64_t idx, double a, double b, uint32_t) {
    *reinterpret_cast<double2 *>(reinterpret_cast<double *>(base) + idx) = make_double2(a, b);
  }
};
__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}
template <>
struct OpStore<OpType::TF32> {
  using CT = float;
  __device__ static void put(void *base, int64_t idx, float a, float b, uint32_t) {
    *reinterpret_cast<float2 *>(reinterpret_cast<float *>(base) + idx) = make_float2(to_tf32(a), to_tf32(b));
  }
};
template <>
struct OpStore<OpType::BF16> {
  using CT = float;
  // r: 32 random bits, 16 for each of the two values.
  __device__ static void put(void *base, int64_t idx, float a, float b, uint32_t r) {
    const uint32_t ua = __float_as_uint(a) + (r & 0xFFFFu);
    const uint32_t ub = __float_as_uint(b) + (r >> 16);
    *reinterpret_cast<uint32_t *>(reinterpret_cast<__nv_bfloat16 *>(base) + idx) = (ua >> 16) | (ub & 0xFFFF0000u);
  }
};

// 32 random bits from (salt, column, observation).
__device__ __forceinline__ uint32_t mix3(uint32_t s, uint32_t c, uint32_t i) {
  uint32_t h = (i * 0x9E3779B1u) ^ (c * 0x85EBCA77u) ^ (s * 0xC2B2AE3Du);
  h = (h ^ (h >> 16)) * 0x7FEB352Du;
  return h ^ (h >> 15);
}

struct BuildDims {
  int64_t N, ldn;
  int K, p, d, q;
  int ob;  // observations per CTA (even)
  int kc;  // classes per Y staging chunk
};

// Shared memory (row strides made odd so that lanes reading every other row
// hit distinct banks): Ps[ob][K|1], Ws[ob][K|1] (P and sqrt(P(1-P)), compute
// type), Xs[ob][p|1], Ys[ob][(kc*d)|1] (float32).
template <OpType OT, typename PT>
__device__ __forceinline__ void build_block(const BuildDims &D, const float *__restrict__ X,
                                            const float *__restrict__ Y, const PT *__restrict__ P, void *At,
                                            void *Ad, int64_t blk) {
  using CT = typename OpStore<OT>::CT;
  extern __shared__ __align__(16) unsigned char smem[];
  const int K = D.K, p = D.p, d = D.d, q = D.q, OB = D.ob;
  const int SP = K | 1, SX = p | 1;
  CT *Ps = reinterpret_cast<CT *>(smem);
  CT *Ws = Ps + (size_t)OB * SP;
  float *Xs = reinterpret_cast<float *>(smem + ((2 * (size_t)OB * SP * sizeof(CT) + 15) & ~(size_t)15));
  float *Ys = Xs + (((size_t)OB * SX + 3) & ~(size_t)3);
  const int64_t i0 = blk * OB;
  const int nobs = (int)min((int64_t)OB, D.N - i0);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;

  for (int e = tid; e < OB * K; e += blockDim.x) {
    const int r = e / K, k = e % K;
    const CT pk = r < nobs ? (CT)P[i0 * K + e] : (CT)0;
    const CT w = pk * ((CT)1 - pk);
    Ps[r * SP + k] = pk;
    Ws[r * SP + k] = w > (CT)0 ? sqrt(w) : (CT)0;
  }
  for (int e = tid; e < OB * p; e += blockDim.x) {
    const int r = e / p, l = e % p;
    Xs[r * SX + l] = r < nobs ? X[i0 * p + e] : 0.f;
  }

  for (int k0 = 1; k0 < K; k0 += D.kc) {
    const int k1 = min(K, k0 + D.kc);
    const int w = (k1 - k0) * d, SY = w | 1;
    __syncthreads();
    if (d) {
      for (int e = tid; e < OB * w; e += blockDim.x) {
        const int r = e / w, c = e % w;
        Ys[r * SY + c] = r < nobs ? Y[((i0 + r) * K + k0) * d + c] : 0.f;
      }
    }
    __syncthreads();
    const int ncols = (k1 - k0) * q;
    for (int cc = warp; cc < ncols; cc += nw) {
      const int k = k0 + cc / q, l = cc % q;
      const int64_t c = (int64_t)(k - 1) * q + l;
      const float *mcol = l < p ? Xs + l : Ys + (k - k0) * d + (l - p);
      const int mstride = l < p ? SX : SY;
      for (int r = 2 * lane; r < OB; r += 64) {
        const CT m0 = (CT)mcol[r * mstride], m1 = (CT)mcol[(r + 1) * mstride];
        const CT p0 = Ps[r * SP + k], p1 = Ps[(r + 1) * SP + k];
        const CT w0 = Ws[r * SP + k], w1 = Ws[(r + 1) * SP + k];
        const uint32_t ii = (uint32_t)(i0 + r), c32 = (uint32_t)c;
        OpStore<OT>::put(At, c * D.ldn + i0 + r, p0 * m0, p1 * m1, mix3(1u, c32, ii));
        OpStore<OT>::put(Ad, c * D.ldn + i0 + r, w0 * m0, w1 * m1, mix3(2u, c32, ii));
      }
    }
  }
}

template <OpType OT, typename PT>
__global__ void __launch_bounds__(256) build_operands_kernel(BuildDims D, const float *__restrict__ X,
                                                             const float *__restrict__ Y,
                                                             const PT *__restrict__ P, void *At, void *Ad) {
  build_block<OT, PT>(D, X, Y, P, At, Ad, blockIdx.x);
}

template <OpType OT, typename PT>
__global__ void __launch_bounds__(256) grouped_build_kernel(const GroupProblem *__restrict__ probs,
                                                            const GroupItem *__restrict__ items,
                                                            const int *__restrict__ active) {
  const GroupItem it = items[blockIdx.x];
  if (active[it.problem] == 0) return;
  const GroupProblem &g = probs[it.problem];
  BuildDims D;
  D.N = g.N; D.ldn = g.ldn; D.K = g.K; D.p = g.p; D.d = g.d; D.q = g.p + g.d;
  D.ob = g.build_ob; D.kc = g.build_kc;
  build_block<OT, PT>(D, g.X, g.Y, reinterpret_cast<const PT *>(g.P), g.At, g.Ad, it.idx);
}

// ---------------------------------------------------------------------------
// FP64 CUDA-core SYRK tile: C[a][b] = sum_i At[a0+a][i] At[b0+b][i], 128 x 128,
// stored transposed (out[b][a]) like the tensor-core tiles.  256 threads,
// 8 x 8 outputs per thread (strided by 16 for conflict-free reads and
// coalesced stores).
// ---------------------------------------------------------------------------

constexpr int kKc = 16;  // observations per shared-memory chunk

// One 128 x 128 tile (ti, tj) over observation chunks [c0, c1) into o (transposed).
__device__ __forceinline__ void syrk_f64_tile(const double *__restrict__ At, int64_t ldn, int ti, int tj, int64_t c0,
                                              int64_t c1, double *__restrict__ o) {
  __shared__ double As[kKc][kTile + 1];
  __shared__ double Bs[kKc][kTile + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t a0 = (int64_t)ti * kTile, b0 = (int64_t)tj * kTile;
  double acc[8][8];
#pragma unroll
  for (int v = 0; v < 8; ++v)
#pragma unroll
    for (int u = 0; u < 8; ++u) acc[v][u] = 0.0;
  const bool diag = ti == tj;
  for (int64_t ch = c0; ch < c1; ++ch) {
    const int64_t i = ch * kKc;
    __syncthreads();
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int idx = tid + 256 * e;
      const int row = idx >> 4, kk = idx & 15;
      As[kk][row] = At[(a0 + row) * ldn + i + kk];
      if (!diag) Bs[kk][row] = At[(b0 + row) * ldn + i + kk];
    }
    __syncthreads();
    const double(*Bp)[kTile + 1] = diag ? As : Bs;
#pragma unroll 4
    for (int kk = 0; kk < kKc; ++kk) {
      double av[8], bv[8];
#pragma unroll
      for (int v = 0; v < 8; ++v) av[v] = As[kk][tx + 16 * v];
#pragma unroll
      for (int u = 0; u < 8; ++u) bv[u] = Bp[kk][ty + 16 * u];
#pragma unroll
      for (int v = 0; v < 8; ++v)
#pragma unroll
        for (int u = 0; u < 8; ++u) acc[v][u] = fma(av[v], bv[u], acc[v][u]);
    }
  }
#pragma unroll
  for (int v = 0; v < 8; ++v)
#pragma unroll
    for (int u = 0; u < 8; ++u) o[(ty + 16 * u) * kTile + tx + 16 * v] = acc[v][u];
}

__global__ void __launch_bounds__(256, 1) syrk_f64_kernel(const double *__restrict__ At, int64_t ldn, int64_t nchunks,
                                                          const int2 *__restrict__ tiles, int ntiles, int nsplit,
                                                          double *__restrict__ out) {
  const int s = blockIdx.x / ntiles, t = blockIdx.x % ntiles;
  const int2 tl = tiles[t];
  syrk_f64_tile(At, ldn, tl.x, tl.y, nchunks * s / nsplit, nchunks * (s + 1) / nsplit,
                out + ((int64_t)s * ntiles + t) * kTile * kTile);
}

// Grouped float64 contraction: one CTA per unit; map 0 selects the problem's
// At operand, map 1 its Ad operand; kb0/kb1 count chunks of kKc observations.
__global__ void __launch_bounds__(256, 1) grouped_syrk_f64_kernel(const GroupProblem *__restrict__ probs,
                                                                  const SyrkUnit *__restrict__ units,
                                                                  const int *__restrict__ active,
                                                                  double *__restrict__ out) {
  const SyrkUnit w = units[blockIdx.x];
  if (active[w.problem] == 0) return;
  const GroupProblem &g = probs[w.problem];
  const double *At = reinterpret_cast<const double *>(w.map == 0 ? g.At : g.Ad);
  syrk_f64_tile(At, g.ldn, w.ti, w.tj, w.kb0, w.kb1, out + w.out_off);
}

// ---------------------------------------------------------------------------
// Z blocks.  With W_ikj = P_ik (z_ikj - zbar_ij) (a centred, probability
// weighted Z), the cross and alpha-alpha blocks are
//   C_X[l][k f + j] = sum_i x_il W_ikj                 (beta_k x alpha)
//   C_Y[k][l][j]    = sum_i y_ikl W_ikj                (gamma_k x alpha)
//   A[j1][j2]       = sum_i sum_k W_ikj1 (z_ikj2 - zbar_ij2)
// Output vector per split: [C_X: p*K*f | C_Y: K*d*f | A: f*f] (k = 0 entries
// of C_X and C_Y are computed but not used).  A CTA stages a tile of rows
// (X, Y, Z, P, zbar contiguous in memory), forms W and z - zbar in shared
// memory and adds the tile to the outputs it owns; grid.y splits the output
// vector when one CTA cannot own all of it.
// ---------------------------------------------------------------------------

constexpr int kZSlots = 16;   // outputs per thread
constexpr int kZThreads = 512;

struct ZDims {
  int64_t N;
  int K, p, d, f;
  int rows;     // rows per tile
  int nsplit;   // row splits (grid.x)
  int64_t nzt;  // outputs per split
};

template <typename T>
__device__ __forceinline__ void zblocks_item(const ZDims &D, const float *__restrict__ X,
                                             const float *__restrict__ Y, const float *__restrict__ Z,
                                             const T *__restrict__ P, const T *__restrict__ zbar, int split,
                                             int chunk, T *__restrict__ out_row) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int K = D.K, p = D.p, d = D.d, f = D.f, R = D.rows;
  const int Kf = K * f, Kd = K * d;
  T *Ws = reinterpret_cast<T *>(smem);          // [R][K f]
  T *Zc = Ws + (size_t)R * Kf;                   // [R][K f]
  float *Xs = reinterpret_cast<float *>(Zc + (size_t)R * Kf);  // [R][p]
  float *Ys = Xs + (size_t)R * p;                // [R][K d]
  const int tid = threadIdx.x;
  const int64_t r0 = D.N * split / D.nsplit, r1 = D.N * (split + 1) / D.nsplit;
  const int64_t obase = (int64_t)chunk * kZThreads * kZSlots;
  const int64_t nx = (int64_t)p * Kf, ny = (int64_t)Kd * f;
  // Slot decoding, once: kind (0 C_X, 1 C_Y, 2 A, 3 none), the two operand
  // offsets inside a staged row, and their row strides.
  int kind[kZSlots], ou[kZSlots], ov[kZSlots];
#pragma unroll
  for (int sl = 0; sl < kZSlots; ++sl) {
    const int64_t o = obase + tid + (int64_t)sl * blockDim.x;
    if (o >= D.nzt) { kind[sl] = 3; ou[sl] = ov[sl] = 0; }
    else if (o < nx) { kind[sl] = 0; ou[sl] = (int)(o / Kf); ov[sl] = (int)(o % Kf); }
    else if (o < nx + ny) {
      const int e = (int)(o - nx), k = e / (d * f), l = (e / f) % d, j = e % f;
      kind[sl] = 1; ou[sl] = k * d + l; ov[sl] = k * f + j;
    } else {
      const int e = (int)(o - nx - ny);
      kind[sl] = 2; ou[sl] = e / f; ov[sl] = e % f;
    }
  }
  T acc[kZSlots];
#pragma unroll
  for (int sl = 0; sl < kZSlots; ++sl) acc[sl] = 0;
  for (int64_t rb = r0; rb < r1; rb += R) {
    const int nr = (int)min((int64_t)R, r1 - rb);
    __syncthreads();
    for (int e = tid; e < nr * K; e += blockDim.x) {
      const int r = e / K, k = e % K;
      const int64_t i = rb + r;
      const T pk = P[i * K + k];
      const float *z = Z + i * Kf + k * f;
      const T *zb = zbar + i * f;
      T *zc = Zc + r * Kf + k * f, *ws = Ws + r * Kf + k * f;
      for (int j = 0; j < f; ++j) {
        const T c = (T)z[j] - zb[j];
        zc[j] = c;
        ws[j] = pk * c;
      }
    }
    for (int e = tid; e < nr * p; e += blockDim.x) Xs[e] = X[rb * p + e];
    for (int e = tid; e < nr * Kd; e += blockDim.x) Ys[e] = Y[rb * Kd + e];
    __syncthreads();
#pragma unroll
    for (int sl = 0; sl < kZSlots; ++sl) {
      T a = 0;
      if (kind[sl] == 0) {
        const float *u = Xs + ou[sl];
        const T *v = Ws + ov[sl];
        for (int r = 0; r < nr; ++r) a = fma((T)u[r * p], v[r * Kf], a);
      } else if (kind[sl] == 1) {
        const float *u = Ys + ou[sl];
        const T *v = Ws + ov[sl];
        for (int r = 0; r < nr; ++r) a = fma((T)u[r * Kd], v[r * Kf], a);
      } else if (kind[sl] == 2) {
        for (int r = 0; r < nr; ++r)
          for (int k = 0; k < K; ++k) a = fma(Ws[r * Kf + k * f + ou[sl]], Zc[r * Kf + k * f + ov[sl]], a);
      }
      acc[sl] += a;
    }
  }
#pragma unroll
  for (int sl = 0; sl < kZSlots; ++sl) {
    const int64_t oo = obase + tid + (int64_t)sl * blockDim.x;
    if (oo < D.nzt) out_row[oo] = acc[sl];
  }
}

template <typename T>
__global__ void __launch_bounds__(kZThreads) zblocks_kernel(ZDims D, const float *__restrict__ X,
                                                            const float *__restrict__ Y, const float *__restrict__ Z,
                                                            const T *__restrict__ P, const T *__restrict__ zbar,
                                                            T *__restrict__ out) {
  zblocks_item<T>(D, X, Y, Z, P, zbar, blockIdx.x, blockIdx.y, out + (int64_t)blockIdx.x * D.nzt);
}

template <typename T>
__global__ void __launch_bounds__(kZThreads) grouped_zblocks_kernel(const GroupProblem *__restrict__ probs,
                                                                    const GroupItem *__restrict__ items,
                                                                    const int *__restrict__ active,
                                                                    T *__restrict__ zpart) {
  const GroupItem it = items[blockIdx.x];
  if (active[it.problem] == 0) return;
  const GroupProblem &g = probs[it.problem];
  ZDims D;
  D.N = g.N; D.K = g.K; D.p = g.p; D.d = g.d; D.f = g.f;
  D.rows = g.zrows;
  D.nsplit = g.zsplit;
  D.nzt = (int64_t)g.p * g.K * g.f + (int64_t)g.K * g.d * g.f + (int64_t)g.f * g.f;
  const int chunks = (int)((D.nzt + (int64_t)kZThreads * kZSlots - 1) / ((int64_t)kZThreads * kZSlots));
  const int split = it.idx / chunks, chunk = it.idx % chunks;
  zblocks_item<T>(D, g.X, g.Y, g.Z, reinterpret_cast<const T *>(g.P), reinterpret_cast<const T *>(g.zbar), split,
                  chunk, zpart + g.z_off + (int64_t)split * D.nzt);
}

// ---------------------------------------------------------------------------
// Assembly of F (lower triangle, column-major) in theta order.
// ---------------------------------------------------------------------------

// F(r, c), r >= c, from the partial sums.
template <typename CT, typename ZT>
__device__ __forceinline__ double assemble_entry(const Shape &S, const CT *__restrict__ mainp, int msplit, int nmain,
                                                 const CT *__restrict__ bandp, int bsplit, int nband,
                                                 const int *__restrict__ band_of, int nt1d,
                                                 const ZT *__restrict__ zp, int zsplit, int64_t r, int64_t c) {
  const int q = S.q, f = S.f, K = S.K;
  const int64_t nx = (int64_t)S.p * K * f, ny = (int64_t)K * S.d * f, nzt = nx + ny + (int64_t)f * f;
  double v = 0.0;
  if (r < S.mc) {
    int kr, lr, kc, lc;
    theta_class_local(S, r, kr, lr);
    theta_class_local(S, c, kc, lc);
    const int64_t ar = (int64_t)(kr - 1) * q + lr, ac = (int64_t)(kc - 1) * q + lc;
    const int64_t ahi = ar > ac ? ar : ac, alo = ar > ac ? ac : ar;
    const int ti = (int)(ahi / kTile), tj = (int)(alo / kTile);
    const int64_t within = (alo % kTile) * kTile + (ahi % kTile);  // tiles are stored [b][a]
    if (kr != kc) {
      const int64_t idx = (int64_t)ti * (ti + 1) / 2 + tj;
      for (int s = 0; s < msplit; ++s) v -= (double)mainp[((int64_t)s * nmain + idx) * kTile * kTile + within];
    } else {
      const int b = band_of[ti * nt1d + tj];
      for (int s = 0; s < bsplit; ++s) v += (double)bandp[((int64_t)s * nband + b) * kTile * kTile + within];
    }
  } else if (c < S.mc) {
    const int j = (int)(r - S.mc);
    int kc, lc;
    theta_class_local(S, c, kc, lc);
    const int64_t off = lc < S.p ? (int64_t)lc * K * f + (int64_t)kc * f + j
                                 : nx + (int64_t)kc * S.d * f + (int64_t)(lc - S.p) * f + j;
    for (int s = 0; s < zsplit; ++s) v += (double)zp[s * nzt + off];
  } else {
    const int j1 = (int)(r - S.mc), j2 = (int)(c - S.mc);
    const int64_t off = nx + ny + (int64_t)j1 * f + j2;
    for (int s = 0; s < zsplit; ++s) v += (double)zp[s * nzt + off];
  }
  return v;
}

template <typename CT, typename ZT>
__global__ void assemble_kernel(Shape S, const CT *__restrict__ mainp, int msplit, int nmain,
                                const CT *__restrict__ bandp, int bsplit, int nband, const int *__restrict__ band_of,
                                int nt1d, const ZT *__restrict__ zp, int zsplit, double *__restrict__ F) {
  const int64_t n = S.n;
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t c = blockIdx.y + (int64_t)gridDim.y * blockIdx.z;
  if (r >= n || c >= n || r < c) return;  // (r, c) in the lower triangle; both mirror entries are written
  const double v = assemble_entry<CT, ZT>(S, mainp, msplit, nmain, bandp, bsplit, nband, band_of, nt1d, zp, zsplit,
                                          r, c);
  F[c * n + r] = v;
  F[r * n + c] = v;
}

// Grouped assembly: item = (problem, block of kAssembleCols columns); the
// batched contractions use one observation split (msplit = bsplit = 1).
template <typename CT, typename ZT>
__global__ void __launch_bounds__(256) grouped_assemble_kernel(const GroupProblem *__restrict__ probs,
                                                               const GroupItem *__restrict__ items,
                                                               const int *__restrict__ active,
                                                               const CT *__restrict__ mainp,
                                                               const CT *__restrict__ bandp,
                                                               const ZT *__restrict__ zpart) {
  const GroupItem it = items[blockIdx.x];
  if (active[it.problem] == 0) return;
  const GroupProblem &g = probs[it.problem];
  const Shape S = shape_of(g.N, g.K, g.p, g.d, g.f);
  const int64_t n = S.n;
  const int nmain = g.nt1d * (g.nt1d + 1) / 2;
  for (int cc = 0; cc < kAssembleCols; ++cc) {
    const int64_t c = (int64_t)it.idx * kAssembleCols + cc;
    if (c >= n) break;
    for (int64_t r = c + threadIdx.x; r < n; r += blockDim.x) {
      const double v = assemble_entry<CT, ZT>(S, mainp + g.main_off, 1, nmain, bandp + g.band_off, 1, 0, g.band_of,
                                              g.nt1d, zpart + g.z_off, g.zsplit, r, c);
      g.F[c * n + r] = v;
      g.F[r * n + c] = v;
    }
  }
}

__global__ void export_hessian_kernel(int64_t n, const double *__restrict__ F, double *__restrict__ H) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t c = blockIdx.y + (int64_t)gridDim.y * blockIdx.z;
  if (r >= n || c >= n) return;
  H[c * n + r] = r >= c ? -F[c * n + r] : -F[r * n + c];
}

void grid_2d(int64_t rows, int64_t cols, dim3 &grid, dim3 &block) {
  block = dim3(256);
  grid.x = (unsigned)((rows + 255) / 256);
  const int64_t ymax = 65535;
  grid.y = (unsigned)std::min<int64_t>(cols, ymax);
  grid.z = (unsigned)((cols + ymax - 1) / ymax);
}

}  // namespace

size_t build_smem_bytes(const Shape &s, OpType t, int ob, int kc) {
  const size_t csz = t == OpType::F64 ? 8 : 4;
  return ((2 * (size_t)ob * (s.K | 1) * csz + 15) & ~(size_t)15) + (((size_t)ob * (s.p | 1) + 3) & ~(size_t)3) * 4 +
         (size_t)ob * ((kc * s.d) | 1) * 4;
}

void build_blocking(const Shape &s, OpType t, int *ob, int *kc) {
  *ob = 64;
  *kc = std::max(1, s.K - 1);
  while (*kc > 1 && build_smem_bytes(s, t, *ob, *kc) > 160 * 1024) *kc = (*kc + 1) / 2;
  while (*ob > 16 && build_smem_bytes(s, t, *ob, *kc) > 160 * 1024) *ob /= 2;
}

cudaError_t launch_build_operands(const Shape &s, OpType t, const float *X, const float *Y, const void *P, void *At,
                                  void *Ad, int64_t ldn, cudaStream_t st) {
  BuildDims D;
  D.N = s.N; D.ldn = ldn; D.K = s.K; D.p = s.p; D.d = s.d; D.q = s.q;
  build_blocking(s, t, &D.ob, &D.kc);
  const size_t smem = build_smem_bytes(s, t, D.ob, D.kc);
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  const int blocks = (int)((s.N + D.ob - 1) / D.ob);
  cudaError_t e;
  switch (t) {
    case OpType::F64: {
      auto k = build_operands_kernel<OpType::F64, double>;
      if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return e;
      k<<<blocks, 256, smem, st>>>(D, X, Y, reinterpret_cast<const double *>(P), At, Ad);
      break;
    }
    case OpType::TF32: {
      auto k = build_operands_kernel<OpType::TF32, float>;
      if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return e;
      k<<<blocks, 256, smem, st>>>(D, X, Y, reinterpret_cast<const float *>(P), At, Ad);
      break;
    }
    case OpType::BF16: {
      auto k = build_operands_kernel<OpType::BF16, float>;
      if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return e;
      k<<<blocks, 256, smem, st>>>(D, X, Y, reinterpret_cast<const float *>(P), At, Ad);
      break;
    }
  }
  return cudaGetLastError();
}

cudaError_t launch_grouped_build(OpType t, const GroupProblem *probs, const GroupItem *items, int nitems,
                                 const int *active, size_t smem, cudaStream_t st) {
  if (nitems <= 0) return cudaSuccess;
  cudaError_t e;
  switch (t) {
    case OpType::F64: {
      auto k = grouped_build_kernel<OpType::F64, double>;
      if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return e;
      k<<<nitems, 256, smem, st>>>(probs, items, active);
      break;
    }
    case OpType::TF32: {
      auto k = grouped_build_kernel<OpType::TF32, float>;
      if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return e;
      k<<<nitems, 256, smem, st>>>(probs, items, active);
      break;
    }
    case OpType::BF16: {
      auto k = grouped_build_kernel<OpType::BF16, float>;
      if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return e;
      k<<<nitems, 256, smem, st>>>(probs, items, active);
      break;
    }
  }
  return cudaGetLastError();
}

cudaError_t launch_grouped_zblocks(bool fp64, const GroupProblem *probs, const GroupItem *items, int nitems,
                                   const int *active, size_t smem, void *zpart, cudaStream_t st) {
  if (nitems <= 0) return cudaSuccess;
  cudaError_t e;
  if (fp64) {
    if ((e = cudaFuncSetAttribute(grouped_zblocks_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem)))
      return e;
    grouped_zblocks_kernel<double><<<nitems, kZThreads, smem, st>>>(probs, items, active,
                                                                     reinterpret_cast<double *>(zpart));
  } else {
    if ((e = cudaFuncSetAttribute(grouped_zblocks_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem)))
      return e;
    grouped_zblocks_kernel<float><<<nitems, kZThreads, smem, st>>>(probs, items, active,
                                                                    reinterpret_cast<float *>(zpart));
  }
  return cudaGetLastError();
}

cudaError_t launch_grouped_assemble(bool fp64, const GroupProblem *probs, const GroupItem *items, int nitems,
                                    const int *active, const void *mainp, const void *bandp, const void *zpart,
                                    cudaStream_t st) {
  if (nitems <= 0) return cudaSuccess;
  if (fp64)
    grouped_assemble_kernel<double, double><<<nitems, 256, 0, st>>>(
        probs, items, active, reinterpret_cast<const double *>(mainp), reinterpret_cast<const double *>(bandp),
        reinterpret_cast<const double *>(zpart));
  else
    grouped_assemble_kernel<float, float><<<nitems, 256, 0, st>>>(
        probs, items, active, reinterpret_cast<const float *>(mainp), reinterpret_cast<const float *>(bandp),
        reinterpret_cast<const float *>(zpart));
  return cudaGetLastError();
}

cudaError_t launch_syrk_f64(const double *At, int64_t ldn, int64_t N, const int2 *tiles, int ntiles, int nsplit,
                            double *out, cudaStream_t st) {
  (void)N;
  const int64_t nchunks = ldn / kKc;
  syrk_f64_kernel<<<ntiles * nsplit, 256, 0, st>>>(At, ldn, nchunks, tiles, ntiles, nsplit, out);
  return cudaGetLastError();
}

int64_t zblocks_outputs(const Shape &s) {
  return (int64_t)s.p * s.K * s.f + (int64_t)s.K * s.d * s.f + (int64_t)s.f * s.f;
}

size_t zblocks_smem(const Shape &s, int rows, bool fp64) {
  const size_t tsz = fp64 ? 8 : 4;
  return (size_t)rows * (2 * (size_t)s.K * s.f * tsz + ((size_t)s.p + (size_t)s.K * s.d) * 4);
}

int zblocks_rows(const Shape &s, bool fp64) {
  int rows = 32;
  while (rows > 1 && zblocks_smem(s, rows, fp64) > 110 * 1024) rows /= 2;
  return rows;
}

cudaError_t launch_grouped_syrk_f64(const GroupProblem *probs, const SyrkUnit *units, int nunits, const int *active,
                                    double *out, cudaStream_t st) {
  if (nunits <= 0) return cudaSuccess;
  grouped_syrk_f64_kernel<<<nunits, 256, 0, st>>>(probs, units, active, out);
  return cudaGetLastError();
}

int f64_chunk_rows() { return kKc; }

cudaError_t launch_zblocks(const Shape &s, bool fp64, const float *X, const float *Y, const float *Z, const void *P,
                           const void *zbar, int nsplit, void *out, cudaStream_t st) {
  ZDims D;
  D.N = s.N; D.K = s.K; D.p = s.p; D.d = s.d; D.f = s.f;
  D.rows = zblocks_rows(s, fp64);
  D.nsplit = nsplit;
  D.nzt = zblocks_outputs(s);
  const size_t smem = zblocks_smem(s, D.rows, fp64);
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  const int chunks = (int)((D.nzt + (int64_t)kZThreads * kZSlots - 1) / ((int64_t)kZThreads * kZSlots));
  dim3 grid(nsplit, chunks);
  cudaError_t e;
  if (fp64) {
    if ((e = cudaFuncSetAttribute(zblocks_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
      return e;
    zblocks_kernel<double><<<grid, kZThreads, smem, st>>>(D, X, Y, Z, reinterpret_cast<const double *>(P),
                                                          reinterpret_cast<const double *>(zbar),
                                                          reinterpret_cast<double *>(out));
  } else {
    if ((e = cudaFuncSetAttribute(zblocks_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
      return e;
    zblocks_kernel<float><<<grid, kZThreads, smem, st>>>(D, X, Y, Z, reinterpret_cast<const float *>(P),
                                                         reinterpret_cast<const float *>(zbar),
                                                         reinterpret_cast<float *>(out));
  }
  return cudaGetLastError();
}

cudaError_t launch_assemble(const Shape &s, const AssembleIO &io, int nmain, double *F, cudaStream_t st) {
  dim3 grid, block;
  grid_2d(s.n, s.n, grid, block);
  const TileLists &tl = *io.tl;
  const int nt1d = (int)((s.mc + kTile - 1) / kTile);
  if (io.fp64) {
    assemble_kernel<double, double><<<grid, block, 0, st>>>(
        s, reinterpret_cast<const double *>(io.main_part), io.main_split, nmain,
        reinterpret_cast<const double *>(io.band_part), io.band_split, tl.nband, tl.band_of, nt1d,
        reinterpret_cast<const double *>(io.z_part), io.z_split, F);
  } else {
    assemble_kernel<float, float><<<grid, block, 0, st>>>(
        s, reinterpret_cast<const float *>(io.main_part), io.main_split, nmain,
        reinterpret_cast<const float *>(io.band_part), io.band_split, tl.nband, tl.band_of, nt1d,
        reinterpret_cast<const float *>(io.z_part), io.z_split, F);
  }
  return cudaGetLastError();
}

cudaError_t launch_export_hessian(int64_t n, const double *F, double *H, cudaStream_t st) {
  dim3 grid, block;
  grid_2d(n, n, grid, block);
  export_hessian_kernel<<<grid, block, 0, st>>>(n, F, H);
  return cudaGetLastError();
}

}  // namespace mnl
