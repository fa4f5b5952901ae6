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
// of (operand, column, observation), so results are reproducible.
template <OpType OT>
struct OpStore;
template <>
struct OpStore<OpType::F64> {
  __device__ static void put(void *base, int64_t idx, double a, double b, uint32_t, uint32_t) {
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
  __device__ static void put(void *base, int64_t idx, double a, double b, uint32_t, uint32_t) {
    *reinterpret_cast<float2 *>(reinterpret_cast<float *>(base) + idx) =
        make_float2(to_tf32((float)a), to_tf32((float)b));
  }
};
__device__ __forceinline__ uint16_t bf16_stochastic(float x, uint32_t r) {
  const uint32_t u = __float_as_uint(x) + (r & 0xFFFFu);
  return (uint16_t)(u >> 16);
}
template <>
struct OpStore<OpType::BF16> {
  __device__ static void put(void *base, int64_t idx, double a, double b, uint32_t ra, uint32_t rb) {
    const uint32_t lo = bf16_stochastic((float)a, ra), hi = bf16_stochastic((float)b, rb);
    *reinterpret_cast<uint32_t *>(reinterpret_cast<__nv_bfloat16 *>(base) + idx) = lo | (hi << 16);
  }
};

// 32-bit mix of (salt, column, observation) (a murmur3-style finaliser).
__device__ __forceinline__ uint32_t mix3(uint32_t s, uint32_t c, uint32_t i) {
  uint32_t h = s * 0x9E3779B9u ^ c * 0x85EBCA6Bu ^ i * 0xC2B2AE35u;
  h ^= h >> 16; h *= 0x7FEB352Du;
  h ^= h >> 15; h *= 0x846CA68Bu;
  h ^= h >> 16;
  return h;
}

struct BuildDims {
  int64_t N, ldn;
  int K, p, d, q;
  int ob;  // observations per CTA (even)
  int kc;  // classes per Y staging chunk
};

// P is float64 in FP64 mode, float32 otherwise.
template <OpType OT, typename PT>
__global__ void __launch_bounds__(256) build_operands_kernel(BuildDims D, const float *__restrict__ X,
                                                             const float *__restrict__ Y,
                                                             const PT *__restrict__ P, void *At, void *Ad) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int K = D.K, p = D.p, d = D.d, q = D.q, OB = D.ob;
  PT *Ps = reinterpret_cast<PT *>(smem);
  float *Xs = reinterpret_cast<float *>(smem + (((size_t)OB * K * sizeof(PT) + 15) & ~(size_t)15));
  float *Ys = Xs + (((size_t)OB * p + 3) & ~(size_t)3);
  const int64_t i0 = (int64_t)blockIdx.x * OB;
  const int nobs = (int)min((int64_t)OB, D.N - i0);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;

  for (int e = tid; e < nobs * K; e += blockDim.x) Ps[e] = P[i0 * K + e];
  for (int e = tid; e < nobs * p; e += blockDim.x) Xs[e] = X[i0 * p + e];

  for (int k0 = 1; k0 < K; k0 += D.kc) {
    const int k1 = min(K, k0 + D.kc);
    __syncthreads();
    if (d) {
      const int w = (k1 - k0) * d;
      for (int e = tid; e < nobs * w; e += blockDim.x) {
        const int r = e / w, c = e % w;
        Ys[(size_t)r * w + c] = Y[((i0 + r) * K + k0) * d + c];
      }
    }
    __syncthreads();
    const int w = (k1 - k0) * d;
    const int ncols = (k1 - k0) * q;
    for (int cc = warp; cc < ncols; cc += nw) {
      const int k = k0 + cc / q, l = cc % q;
      const int64_t c = (int64_t)(k - 1) * q + l;
      for (int r = 2 * lane; r < OB; r += 64) {
        double av[2] = {0.0, 0.0}, dv[2] = {0.0, 0.0};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int rr = r + h;
          if (rr < nobs) {
            const double pk = (double)Ps[(size_t)rr * K + k];
            const double m = l < p ? (double)Xs[(size_t)rr * p + l] : (double)Ys[(size_t)rr * w + (k - k0) * d + (l - p)];
            av[h] = pk * m;
            const double wv = pk * (1.0 - pk);
            dv[h] = (wv > 0.0 ? sqrt(wv) : 0.0) * m;
          }
        }
        const uint32_t ii = (uint32_t)(i0 + r), cc32 = (uint32_t)c;
        OpStore<OT>::put(At, c * D.ldn + i0 + r, av[0], av[1], mix3(1u, cc32, ii), mix3(1u, cc32, ii + 1));
        OpStore<OT>::put(Ad, c * D.ldn + i0 + r, dv[0], dv[1], mix3(2u, cc32, ii), mix3(2u, cc32, ii + 1));
      }
    }
  }
}

// ---------------------------------------------------------------------------
// FP64 CUDA-core SYRK tile: C[a][b] = sum_i At[a0+a][i] At[b0+b][i], 128 x 128,
// stored transposed (out[b][a]) like the tensor-core tiles.  256 threads,
// 8 x 8 outputs per thread (strided by 16 for conflict-free reads and
// coalesced stores).
// ---------------------------------------------------------------------------

constexpr int kKc = 16;  // observations per shared-memory chunk

__global__ void __launch_bounds__(256, 1) syrk_f64_kernel(const double *__restrict__ At, int64_t ldn, int64_t nchunks,
                                                          const int2 *__restrict__ tiles, int ntiles, int nsplit,
                                                          double *__restrict__ out) {
  __shared__ double As[kKc][kTile + 1];
  __shared__ double Bs[kKc][kTile + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int unit = blockIdx.x;
  const int s = unit / ntiles, t = unit % ntiles;
  const int2 tl = tiles[t];
  const int64_t a0 = (int64_t)tl.x * kTile, b0 = (int64_t)tl.y * kTile;
  const int64_t c0 = nchunks * s / nsplit, c1 = nchunks * (s + 1) / nsplit;
  double acc[8][8];
#pragma unroll
  for (int v = 0; v < 8; ++v)
#pragma unroll
    for (int u = 0; u < 8; ++u) acc[v][u] = 0.0;
  const bool diag = tl.x == tl.y;
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
  double *o = out + ((int64_t)s * ntiles + t) * kTile * kTile;
#pragma unroll
  for (int v = 0; v < 8; ++v)
#pragma unroll
    for (int u = 0; u < 8; ++u) o[(ty + 16 * u) * kTile + tx + 16 * v] = acc[v][u];
}

// ---------------------------------------------------------------------------
// Z blocks: per (split, class) partial sums of the cross and alpha-alpha terms.
// ---------------------------------------------------------------------------

constexpr int kZRows = 32;
constexpr int kZSlots = 16;  // outputs per thread (q f + f f <= 4096)

template <typename T>
__global__ void __launch_bounds__(256) zblocks_kernel(int64_t N, int K, int p, int d, int f, int nsplit,
                                                      const float *__restrict__ X, const float *__restrict__ Y,
                                                      const float *__restrict__ Z, const T *__restrict__ P,
                                                      const T *__restrict__ zbar, T *__restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int q = p + d, nz = q * f + f * f;
  T *ms = reinterpret_cast<T *>(smem);      // [kZRows][q]
  T *zs = ms + (size_t)kZRows * q;          // [kZRows][f]
  T *ws = zs + (size_t)kZRows * f;          // [kZRows]
  const int s = blockIdx.x, k = blockIdx.y, tid = threadIdx.x;
  const int64_t r0 = N * s / nsplit, r1 = N * (s + 1) / nsplit;
  T acc[kZSlots];
#pragma unroll
  for (int sl = 0; sl < kZSlots; ++sl) acc[sl] = 0;
  for (int64_t rb = r0; rb < r1; rb += kZRows) {
    const int nr = (int)min((int64_t)kZRows, r1 - rb);
    __syncthreads();
    for (int e = tid; e < nr * q; e += blockDim.x) {
      const int r = e / q, l = e % q;
      const int64_t i = rb + r;
      ms[e] = l < p ? (T)X[i * p + l] : (T)Y[(i * K + k) * d + (l - p)];
    }
    for (int e = tid; e < nr * f; e += blockDim.x) {
      const int r = e / f, j = e % f;
      const int64_t i = rb + r;
      zs[e] = (T)Z[(i * K + k) * f + j] - zbar[i * f + j];
    }
    for (int r = tid; r < nr; r += blockDim.x) ws[r] = P[(rb + r) * K + k];
    __syncthreads();
#pragma unroll
    for (int sl = 0; sl < kZSlots; ++sl) {
      const int o = tid + sl * blockDim.x;
      if (o < nz) {
        T a = 0;
        if (o < q * f) {
          if (k > 0) {
            const int l = o / f, j = o % f;
            for (int r = 0; r < nr; ++r) a = fma(ws[r] * ms[r * q + l], zs[r * f + j], a);
          }
        } else {
          const int e = o - q * f, j1 = e / f, j2 = e % f;
          for (int r = 0; r < nr; ++r) a = fma(ws[r] * zs[r * f + j1], zs[r * f + j2], a);
        }
        acc[sl] += a;
      }
    }
  }
  T *o = out + ((int64_t)s * K + k) * nz;
#pragma unroll
  for (int sl = 0; sl < kZSlots; ++sl) {
    const int oo = tid + sl * blockDim.x;
    if (oo < nz) o[oo] = acc[sl];
  }
}

// ---------------------------------------------------------------------------
// Assembly of F (lower triangle, column-major) in theta order.
// ---------------------------------------------------------------------------

template <typename CT, typename ZT>
__global__ void assemble_kernel(Shape S, const CT *__restrict__ mainp, int msplit, int nmain,
                                const CT *__restrict__ bandp, int bsplit, int nband, const int *__restrict__ band_of,
                                int nt1d, const ZT *__restrict__ zp, int zsplit, double *__restrict__ F) {
  const int64_t n = S.n;
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t c = blockIdx.y + (int64_t)gridDim.y * blockIdx.z;
  if (r >= n || c >= n || r < c) return;
  const int q = S.q, f = S.f, K = S.K;
  const int nz = q * f + f * f;
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
    for (int s = 0; s < zsplit; ++s) v += (double)zp[((int64_t)s * K + kc) * nz + lc * f + j];
  } else {
    const int j1 = (int)(r - S.mc), j2 = (int)(c - S.mc);
    for (int k = 0; k < K; ++k) {
      double vk = 0.0;
      for (int s = 0; s < zsplit; ++s) vk += (double)zp[((int64_t)s * K + k) * nz + q * f + j1 * f + j2];
      v += vk;
    }
  }
  F[c * n + r] = v;
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

cudaError_t launch_build_operands(const Shape &s, OpType t, const float *X, const float *Y, const void *P, void *At,
                                  void *Ad, int64_t ldn, cudaStream_t st) {
  BuildDims D;
  D.N = s.N; D.ldn = ldn; D.K = s.K; D.p = s.p; D.d = s.d; D.q = s.q;
  const size_t psz = t == OpType::F64 ? 8 : 4;
  D.ob = 64;
  auto smem_for = [&](int ob, int kc) {
    return (((size_t)ob * s.K * psz + 15) & ~(size_t)15) + (((size_t)ob * s.p + 3) & ~(size_t)3) * 4 +
           (size_t)ob * kc * s.d * 4;
  };
  D.kc = s.K - 1;
  while (D.kc > 1 && smem_for(D.ob, D.kc) > 160 * 1024) D.kc = (D.kc + 1) / 2;
  while (D.ob > 16 && smem_for(D.ob, D.kc) > 160 * 1024) D.ob /= 2;
  const size_t smem = smem_for(D.ob, D.kc);
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

cudaError_t launch_syrk_f64(const double *At, int64_t ldn, int64_t N, const int2 *tiles, int ntiles, int nsplit,
                            double *out, cudaStream_t st) {
  (void)N;
  const int64_t nchunks = ldn / kKc;
  syrk_f64_kernel<<<ntiles * nsplit, 256, 0, st>>>(At, ldn, nchunks, tiles, ntiles, nsplit, out);
  return cudaGetLastError();
}

cudaError_t launch_zblocks(const Shape &s, bool fp64, const float *X, const float *Y, const float *Z, const void *P,
                           const void *zbar, int nsplit, void *out, cudaStream_t st) {
  const int nz = s.q * s.f + s.f * s.f;
  if (nz > 256 * kZSlots) return cudaErrorInvalidValue;
  const size_t tsz = fp64 ? 8 : 4;
  const size_t smem = ((size_t)kZRows * (s.q + s.f) + kZRows) * tsz;
  dim3 grid(nsplit, s.K);
  if (fp64) {
    zblocks_kernel<double><<<grid, 256, smem, st>>>(s.N, s.K, s.p, s.d, s.f, nsplit, X, Y, Z,
                                                    reinterpret_cast<const double *>(P),
                                                    reinterpret_cast<const double *>(zbar),
                                                    reinterpret_cast<double *>(out));
  } else {
    zblocks_kernel<float><<<grid, 256, smem, st>>>(s.N, s.K, s.p, s.d, s.f, nsplit, X, Y, Z,
                                                   reinterpret_cast<const float *>(P),
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
