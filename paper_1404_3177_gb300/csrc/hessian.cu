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

#include <algorithm>

#include "mnl_internal.cuh"

namespace mnl {
namespace {

// ---------------------------------------------------------------------------
// Operand builder: At[c][i] = P_ik m_ik[l], Ad[c][i] = sqrt(P_ik(1-P_ik)) m_ik[l]
// ---------------------------------------------------------------------------

// Rounding of the operands.  TF32 rounds to nearest (cvt.rna).  BF16 rounds
// stochastically (the conversion instruction with random bits, 16 per value):
// the rounded value is unbiased.  With round-to-nearest, designs in which many
// observations share the same P_ik (an intercept-only model, indicator
// columns) would give every product the same rounding error; unbiased rounding
// turns that into independent errors that average out over the observations.
// The random bits are a hash of (operand, row, observation), so results are
// reproducible.
//
// put8 stores 8 consecutive observations of one operand row (16-byte stores);
// r holds the random words of the BF16 conversion (one per pair of values).
template <OpType OT>
struct OpStore;
template <>
struct OpStore<OpType::F64> {
  using CT = double;
  __device__ __forceinline__ static void put8(void *row, const double v[8], uint4) {
    double2 *d = reinterpret_cast<double2 *>(row);
#pragma unroll
    for (int u = 0; u < 4; ++u) d[u] = make_double2(v[2 * u], v[2 * u + 1]);
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
  __device__ __forceinline__ static void put8(void *row, const float v[8], uint4) {
    float4 *d = reinterpret_cast<float4 *>(row);
    d[0] = make_float4(to_tf32(v[0]), to_tf32(v[1]), to_tf32(v[2]), to_tf32(v[3]));
    d[1] = make_float4(to_tf32(v[4]), to_tf32(v[5]), to_tf32(v[6]), to_tf32(v[7]));
  }
};
template <>
struct OpStore<OpType::BF16> {
  using CT = float;
  __device__ __forceinline__ static void put8(void *row, const float v[8], uint4 r) {
    const uint32_t rr[4] = {r.x, r.y, r.z, r.w};
    uint32_t o[4];
#pragma unroll
    for (int u = 0; u < 4; ++u)  // o[u] = bf16(v[2u + 1]) << 16 | bf16(v[2u])
      asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(o[u]) : "f"(v[2 * u + 1]), "f"(v[2 * u]), "r"(rr[u]));
    *reinterpret_cast<uint4 *>(row) = make_uint4(o[0], o[1], o[2], o[3]);
  }
};

// 32 random bits from (salt, column, observation).
__device__ __forceinline__ uint32_t mix3(uint32_t s, uint32_t c, uint32_t i) {
  uint32_t h = (i * 0x9E3779B1u) ^ (c * 0x85EBCA77u) ^ (s * 0xC2B2AE3Du);
  h = (h ^ (h >> 16)) * 0x7FEB352Du;
  return h ^ (h >> 15);
}
// Four random words (for 8 BF16 conversions) from one hash value.
__device__ __forceinline__ uint32_t word_of(uint32_t h, uint32_t u) {
  const uint32_t w = (h + u * 0x9E3779B9u) * 0x85EBCA6Bu;
  return w ^ (w >> 15);
}
__device__ __forceinline__ uint4 words4(uint32_t h) {
  return make_uint4(word_of(h, 0u), word_of(h, 1u), word_of(h, 2u), word_of(h, 3u));
}

// Exact x / d (x + d < 2^32) by a multiply-high and one correction step.
struct FastDiv {
  uint32_t d, m;
  __device__ explicit FastDiv(uint32_t dd) : d(dd), m(0xFFFFFFFFu / (dd ? dd : 1u)) {}
  __device__ __forceinline__ uint32_t div(uint32_t x) const {
    const uint32_t t = __umulhi(x, m);
    return t + ((t + 1u) * d <= x ? 1u : 0u);
  }
};

// 8 consecutive shared-memory values (16-byte aligned).
__device__ __forceinline__ void lds8(const float *p, float v[8]) {
  const float4 a = reinterpret_cast<const float4 *>(p)[0], b = reinterpret_cast<const float4 *>(p)[1];
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}
__device__ __forceinline__ void lds8(const double *p, double v[8]) {
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const double2 a = reinterpret_cast<const double2 *>(p)[u];
    v[2 * u] = a.x;
    v[2 * u + 1] = a.y;
  }
}

constexpr int kBob = 64;        // observations per builder block (8 lanes x 8)
constexpr int kBs = kBob + 4;   // shared row stride (16-byte aligned rows)
constexpr int kStage = 16;      // staging loads in flight per thread

struct ZopDims {
  int64_t N, ldn, oY, oW, oZ;
  int K, p, d, f, kc;
};

struct BuildDims {
  int64_t N, ldn;
  int K, p, d, q;
  int ob;  // observations per block (kBob)
  int kc;  // classes per Y (and Z) staging chunk
  int f;   // Z operand (Az != nullptr): generic columns and its row-block offsets
  int64_t oY, oW, oZ;
  int64_t rpA, rpZ;  // padded row counts of At / Ad and of Az (K-blocked layout)
  const float *w;    // [N] observation weights (every operand row scaled by sqrt(w_i)), or nullptr
};

// Element offset of operand row `row`, observation i.  float64 operands are
// row-major ([rows][ldn]).  TF32 / BF16 operands, which the tensor cores read
// through TMA, are K-blocked: [ldn / BK][rows_pad][BK] with BK = 32 (TF32) or
// 64 (BF16) observations = 128 bytes, so that the 128-row box of one K-block
// is 16 KB of contiguous memory (no strided rows: DRAM pages and TLB entries
// stay few however large N is).
template <OpType OT>
__device__ __forceinline__ int64_t op_off(int64_t row, int64_t i, int64_t ldn, int64_t rows_pad) {
  if (OT == OpType::F64) return row * ldn + i;
  constexpr int BK = OT == OpType::TF32 ? kBkTf32 : kBkBf16;
  return ((i / BK) * rows_pad + row) * BK + (i % BK);
}

// Shared memory, transposed so that observations are contiguous:
//   PsT[K][kBs], WsT[K][kBs] (P and sqrt(P(1-P)), compute type),
//   XsT[p][kBs], YsT[kc*d][kBs] (float32), and with the Z operand
//   ZcT[kc*f][kBs], zbT[f][kBs] (z - zbar, zbar; compute type).
// A warp writes 4 operand rows at a time: lanes 8c..8c+7 take row c of the
// group, 8 observations each (one 16-byte store per lane and operand for BF16).
// With Az, the same staged block also gives the rows of the Z-block operand
// (X, Y, W = P (z - zbar), Zc = z - zbar; see the Z-block section below).
template <OpType OT, typename PT>
__device__ __forceinline__ void build_block(const BuildDims &D, const float *__restrict__ X,
                                            const float *__restrict__ Y, const PT *__restrict__ P, void *At,
                                            void *Ad, int64_t blk, const float *__restrict__ Z = nullptr,
                                            const PT *__restrict__ zbar = nullptr, void *Az = nullptr) {
  using CT = typename OpStore<OT>::CT;
  constexpr int esz = OT == OpType::F64 ? 8 : OT == OpType::TF32 ? 4 : 2;
  extern __shared__ __align__(16) unsigned char smem[];
  const int K = D.K, p = D.p, d = D.d, q = D.q, f = Az ? D.f : 0;
  CT *PsT = reinterpret_cast<CT *>(smem);
  CT *WsT = PsT + (size_t)K * kBs;
  float *XsT = reinterpret_cast<float *>(WsT + (size_t)K * kBs);
  float *YsT = XsT + (size_t)p * kBs;
  CT *ZcT = reinterpret_cast<CT *>(YsT + (size_t)D.kc * d * kBs);
  CT *zbT = ZcT + (size_t)D.kc * f * kBs;
  CT *swT = zbT + (size_t)f * kBs;  // sqrt(w_i) of the block's observations (weights only)
  const int64_t i0 = blk * kBob;
  const int nobs = (int)min((int64_t)kBob, D.N - i0);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const FastDiv divK((uint32_t)K), divp((uint32_t)p), divq((uint32_t)q), divd((uint32_t)d), divf((uint32_t)f);
  // Case weights: -H = sum_i w_i [...] is the SYRK of operand rows scaled by sqrt(w_i).
  if (D.w) {
    for (int r = tid; r < kBob; r += 256) swT[r] = r < nobs ? (CT)sqrt((double)D.w[i0 + r]) : (CT)0;
    __syncthreads();
  }
  auto sw = [&](int r) { return D.w ? swT[r] : (CT)1; };

  // staging, kStage loads in flight per thread
  for (int e0 = 0; e0 < kBob * K; e0 += kStage * 256) {
    PT v[kStage];
#pragma unroll
    for (int u = 0; u < kStage; ++u) {
      const int e = e0 + tid + u * 256;
      v[u] = (e < kBob * K && (int)divK.div(e) < nobs) ? P[i0 * K + e] : (PT)0;
    }
#pragma unroll
    for (int u = 0; u < kStage; ++u) {
      const int e = e0 + tid + u * 256;
      if (e < kBob * K) {
        const int r = divK.div(e), k = e - r * K;
        const CT pk = (CT)v[u], w = pk * ((CT)1 - pk), s = sw(r);
        PsT[k * kBs + r] = pk * s;
        WsT[k * kBs + r] = w > (CT)0 ? sqrt(w) * s : (CT)0;
      }
    }
  }
  for (int e0 = 0; e0 < kBob * p; e0 += kStage * 256) {
    float v[kStage];
#pragma unroll
    for (int u = 0; u < kStage; ++u) {
      const int e = e0 + tid + u * 256;
      v[u] = (e < kBob * p && (int)divp.div(e) < nobs) ? __ldg(X + i0 * p + e) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < kStage; ++u) {
      const int e = e0 + tid + u * 256;
      if (e < kBob * p) {
        const int r = divp.div(e), l = e - r * p;
        XsT[l * kBs + r] = v[u];
      }
    }
  }
  for (int e = tid; e < kBob * f; e += 256) {
    const int r = divf.div(e), j = e - r * f;
    zbT[j * kBs + r] = r < nobs ? (CT)zbar[i0 * f + e] : (CT)0;
  }

  const int cl = lane >> 3, oc = (lane & 7) * 8;
  const uint32_t iobs = (uint32_t)(i0 + oc);
  constexpr bool kRand = OT == OpType::BF16;
  auto put_z = [&](int64_t row, const CT v[8]) {  // one row of the Z-block operand
    const uint4 rw = kRand ? words4(mix3(5u, (uint32_t)row, iobs)) : make_uint4(0u, 0u, 0u, 0u);
    OpStore<OT>::put8(reinterpret_cast<unsigned char *>(Az) + op_off<OT>(row, i0 + oc, D.ldn, D.rpZ) * esz, v, rw);
  };
  if (Az) {
    __syncthreads();
    for (int cg = warp * 4; cg < p; cg += nw * 4) {  // X rows
      const int l = cg + cl;
      if (l >= p) continue;
      float m[8];
      CT v[8];
      lds8(XsT + l * kBs + oc, m);
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = (CT)m[u] * sw(oc + u);
      put_z(l, v);
    }
  }
  for (int k0 = Az ? 0 : 1; k0 < K; k0 += D.kc) {
    const int k1 = min(K, k0 + D.kc), nk = k1 - k0;
    const int w = nk * d;
    const FastDiv divw((uint32_t)w), divwz((uint32_t)(nk * f));
    __syncthreads();
    if (d) {
      for (int e0 = 0; e0 < kBob * w; e0 += kStage * 256) {
        float v[kStage];
#pragma unroll
        for (int u = 0; u < kStage; ++u) {
          const int e = e0 + tid + u * 256;
          const int r = divw.div(e);
          v[u] = (e < kBob * w && r < nobs) ? __ldg(Y + ((i0 + r) * K + k0) * d + (e - r * w)) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < kStage; ++u) {
          const int e = e0 + tid + u * 256;
          if (e < kBob * w) {
            const int r = divw.div(e);
            YsT[(e - r * w) * kBs + r] = v[u];
          }
        }
      }
    }
    if (f) {
      const int wz = nk * f;
      for (int e0 = 0; e0 < kBob * wz; e0 += kStage * 256) {
        float v[kStage];
#pragma unroll
        for (int u = 0; u < kStage; ++u) {
          const int e = e0 + tid + u * 256;
          const int r = divwz.div(e);
          v[u] = (e < kBob * wz && r < nobs) ? __ldg(Z + ((i0 + r) * K + k0) * f + (e - r * wz)) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < kStage; ++u) {
          const int e = e0 + tid + u * 256;
          if (e < kBob * wz) {
            const int r = divwz.div(e), c = e - r * wz;
            ZcT[c * kBs + r] = r < nobs ? (CT)v[u] - zbT[(c - (int)divf.div(c) * f) * kBs + r] : (CT)0;
          }
        }
      }
    }
    __syncthreads();
    const int ks = k0 == 0 ? 1 : k0;  // the class operands start at class 1
    const int ncols = (k1 - ks) * q;
    // each warp takes a contiguous range of columns, so that a lane keeps the
    // P and sqrt(P(1-P)) values of its class in registers until the class changes
    const int per = ((ncols + nw - 1) / nw + 3) & ~3;
    const int cbeg = warp * per, cend = min(ncols, cbeg + per);
    int kcur = -1;
    CT pk[8], wk[8];
    for (int cg = cbeg; cg < cend; cg += 4) {
      const int cc = cg + cl;
      if (cc >= cend) continue;
      const int kq = divq.div(cc), l = cc - kq * q, k = ks + kq, kk = k - k0;
      const int64_t c = (int64_t)(k - 1) * q + l;
      const float *mrow = l < p ? XsT + l * kBs : YsT + (kk * d + (l - p)) * kBs;
      float m[8];
      CT pv[8], wv[8];
      lds8(mrow + oc, m);
      if (k != kcur) {
        lds8(PsT + k * kBs + oc, pk);
        lds8(WsT + k * kBs + oc, wk);
        kcur = k;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        pv[u] = pk[u] * (CT)m[u];
        wv[u] = wk[u] * (CT)m[u];
      }
      uint4 ra = make_uint4(0u, 0u, 0u, 0u), rd = ra;
      if (kRand) {
        ra = words4(mix3(1u, (uint32_t)c, iobs));
        // Ad takes the other halves of the same words
        rd = make_uint4(__funnelshift_l(ra.x, ra.x, 16), __funnelshift_l(ra.y, ra.y, 16),
                        __funnelshift_l(ra.z, ra.z, 16), __funnelshift_l(ra.w, ra.w, 16));
      }
      const int64_t off = op_off<OT>(c, i0 + oc, D.ldn, D.rpA) * esz;
      unsigned char *rowA = reinterpret_cast<unsigned char *>(At) + off;
      unsigned char *rowD = reinterpret_cast<unsigned char *>(Ad) + off;
      OpStore<OT>::put8(rowA, pv, ra);
      OpStore<OT>::put8(rowD, wv, rd);
    }
    if (Az) {  // Y rows (classes >= 1), W and Zc rows of this chunk's classes
      const int ny = (k1 - ks) * d, nwz = nk * f, rows = ny + 2 * nwz;
      for (int cg = warp * 4; cg < rows; cg += nw * 4) {
        const int c = cg + cl;
        if (c >= rows) continue;
        CT v[8];
        int64_t row;
        if (c < ny) {
          const int kq = divd.div(c), l = c - kq * d, kk = ks + kq - k0;
          float m[8];
          lds8(YsT + (kk * d + l) * kBs + oc, m);
#pragma unroll
          for (int u = 0; u < 8; ++u) v[u] = (CT)m[u] * sw(oc + u);
          row = D.oY + (int64_t)(ks + kq - 1) * d + l;
        } else if (c < ny + nwz) {
          const int c2 = c - ny, kk = divf.div(c2);
          CT pk[8], zc[8];
          lds8(PsT + (k0 + kk) * kBs + oc, pk);
          lds8(ZcT + c2 * kBs + oc, zc);
#pragma unroll
          for (int u = 0; u < 8; ++u) v[u] = pk[u] * zc[u];
          row = D.oW + (int64_t)k0 * f + c2;
        } else {
          const int c2 = c - ny - nwz;
          lds8(ZcT + c2 * kBs + oc, v);
#pragma unroll
          for (int u = 0; u < 8; ++u) v[u] *= sw(oc + u);
          row = D.oZ + (int64_t)k0 * f + c2;
        }
        put_z(row, v);
      }
    }
  }
}

template <OpType OT, typename PT>
__global__ void __launch_bounds__(256, 3) build_operands_z_kernel(BuildDims D, const float *__restrict__ X,
                                                               const float *__restrict__ Y, const PT *__restrict__ P,
                                                               void *At, void *Ad, const float *__restrict__ Z,
                                                               const PT *__restrict__ zbar, void *Az) {
  build_block<OT, PT>(D, X, Y, P, At, Ad, blockIdx.x, Z, zbar, Az);
}

template <OpType OT, typename PT>
__global__ void __launch_bounds__(256, 3) build_operands_kernel(BuildDims D, const float *__restrict__ X,
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
  BuildDims D{};
  D.N = g.N; D.ldn = g.ldn; D.K = g.K; D.p = g.p; D.d = g.d; D.q = g.p + g.d;
  D.ob = g.build_ob; D.kc = g.build_kc;
  D.rpA = g.mc_pad; D.rpZ = 0;
  D.w = nullptr;
  build_block<OT, PT>(D, g.X, g.Y, reinterpret_cast<const PT *>(g.P), g.At, g.Ad, it.idx);
}

// ---------------------------------------------------------------------------
// Z-block operand for the tensor-core contraction (TF32 / BF16 modes).  Rows,
// in blocks that start on 128-row tiles, observations contiguous:
//   X  rows l          x_il                      (oX = 0)
//   Y  rows (k-1) d + l  y_ikl, k >= 1             (oY)
//   W  rows k f + j    P_ik (z_ikj - zbar_ij)     (oW)
//   Zc rows k f + j    z_ikj - zbar_ij            (oZ)
// so that C_X = X W^T, C_Y = the class-diagonal blocks of Y W^T and
// A = sum_k W_k Zc_k^T are tiles of the Gram matrix of this operand.  Its rows
// are written by the class-operand builder from the same staged block.
// ---------------------------------------------------------------------------

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
// Output vector per observation split: [C_X: p*K*f | C_Y: K*d*f | A: f*f]
// (k = 0 entries of C_X and C_Y are computed but not used).
//
// The work of one split is cut into parts, one CTA each:
//   * C_X tiles of 64 (l) x 64 (c = k f + j): X and W rows are staged in a
//     double-buffered shared tile (the next tile's loads are in flight while
//     the current one is used) and every thread accumulates a 4 x 4 block of
//     Xᵀ W in registers (two 16-byte shared loads per 16 FMAs);
//   * C_Y chunks of kZyOut outputs, a thread per output;
//   * the alpha block: the (observation, alternative) pairs of a staged tile
//     are dealt to thread subsets, each thread accumulating a 4 x 4 block of
//     the f x f result; the subsets are added in a fixed order at the end.
// ---------------------------------------------------------------------------

constexpr int kZThreads = 256;
constexpr int kZxTile = 64;    // C_X tile edge (l and c)
constexpr int kZxRows = 32;    // observations per staged C_X tile
constexpr int kZxStride = 68;  // shared row stride of the C_X tiles (multiple of 4)
constexpr int kZySlots = 8;
constexpr int kZyOut = kZThreads * kZySlots;  // C_Y outputs per part
constexpr size_t kZBudget = 96 * 1024;        // shared bytes of a C_Y or alpha tile
constexpr int kZBatch = 8;                    // rows staged per batch of loads

struct ZPlan {
  int nl, nc;  // C_X tiles over l (p) and c (K f)
  int ny;      // C_Y parts
  int kspan;   // classes a C_Y part spans at most
  int ry, ra;  // observations per staged tile of a C_Y / alpha part
  int fs;      // f rounded up to a multiple of 4
  __host__ __device__ int parts() const { return nl * nc + ny + 1; }
};

__host__ __device__ inline size_t zmin(size_t a, size_t b) { return a < b ? a : b; }
__host__ __device__ inline size_t zmax(size_t a, size_t b) { return a > b ? a : b; }

__host__ __device__ inline ZPlan make_zplan(int K, int p, int d, int f, int tsz) {
  ZPlan z;
  const int Kf = K * f;
  z.nl = (p + kZxTile - 1) / kZxTile;
  z.nc = (Kf + kZxTile - 1) / kZxTile;
  const int64_t ny = (int64_t)K * d * f;
  z.ny = (int)((ny + kZyOut - 1) / kZyOut);
  z.fs = (f + 3) & ~3;
  z.kspan = d ? (int)zmin((size_t)K, (size_t)(kZyOut / (d * f) + 2)) : 0;
  const size_t yrow = (size_t)z.kspan * ((size_t)d * 4 + (size_t)f * tsz);
  z.ry = yrow ? (int)zmin(32, zmax(1, kZBudget / yrow)) : 1;
  const size_t arow = (size_t)2 * K * z.fs * tsz, red = (size_t)kZThreads * 16 * tsz;
  z.ra = (int)zmin(32, zmax(1, (kZBudget - red) / arow));
  return z;
}

struct ZDims {
  int64_t N;
  int K, p, d, f;
  int nsplit;   // observation splits
  int64_t nzt;  // outputs per split
  ZPlan zp;
  const float *w;  // [N] observation weights (they scale P_ik in W = P (z - zbar)), or nullptr
};

template <typename T>
struct Vec4;
template <>
struct Vec4<float> {
  __device__ static void load(const float *p, float v[4]) {
    const float4 a = *reinterpret_cast<const float4 *>(p);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  }
};
template <>
struct Vec4<double> {
  __device__ static void load(const double *p, double v[4]) {
    const double2 a = reinterpret_cast<const double2 *>(p)[0], b = reinterpret_cast<const double2 *>(p)[1];
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  }
};

// C_X tile (lb, cb) over observations [r0, r1).
template <typename T>
__device__ __forceinline__ void zx_part(const ZDims &D, const float *__restrict__ X, const float *__restrict__ Z,
                                        const T *__restrict__ P, const T *__restrict__ zbar, int64_t r0, int64_t r1,
                                        int lb, int cb, T *__restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int kBuf = kZxRows * kZxStride;
  float *Xs = reinterpret_cast<float *>(smem);  // [2][kZxRows][kZxStride]
  T *Ws = reinterpret_cast<T *>(Xs + 2 * kBuf);  // [2][kZxRows][kZxStride]
  const int K = D.K, p = D.p, f = D.f, Kf = K * f;
  const int l0 = lb * kZxTile, c0 = cb * kZxTile;
  const int nlw = min(kZxTile, p - l0), ncw = min(kZxTile, Kf - c0);
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  // Staging: this thread moves column cc of rows rr, rr + 4, ..., rr + 28.
  const int cc = tid & 63, rr = tid >> 6;
  const bool xcol = cc < nlw, zcol = cc < ncw;
  const int c = c0 + cc, k = zcol ? c / f : 0, j = zcol ? c - k * f : 0;
  constexpr int kPer = kZxRows / 4;
  float xv[kPer], zv[kPer];
  T pv[kPer], bv[kPer];
  auto fetch = [&](int64_t rb) {
#pragma unroll
    for (int s = 0; s < kPer; ++s) {
      const int64_t i = rb + rr + 4 * s;
      const bool in = i < r1;
      xv[s] = (in && xcol) ? __ldg(X + i * p + l0 + cc) : 0.f;
      if (in && zcol) {
        zv[s] = __ldg(Z + i * Kf + c);
        pv[s] = P[i * K + k] * (D.w ? (T)D.w[i] : (T)1);
        bv[s] = zbar[i * f + j];
      } else {
        zv[s] = 0.f; pv[s] = (T)0; bv[s] = (T)0;
      }
    }
  };
  auto put = [&](int buf) {
#pragma unroll
    for (int s = 0; s < kPer; ++s) {
      const int o = buf * kBuf + (rr + 4 * s) * kZxStride + cc;
      Xs[o] = xv[s];
      Ws[o] = pv[s] * ((T)zv[s] - bv[s]);
    }
  };
  T acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = (T)0;
  fetch(r0);
  put(0);
  __syncthreads();
  int buf = 0;
  for (int64_t rb = r0; rb < r1; rb += kZxRows) {
    const bool more = rb + kZxRows < r1;
    if (more) fetch(rb + kZxRows);
    const float *xs = Xs + buf * kBuf + ty * 4;
    const T *ws = Ws + buf * kBuf + tx * 4;
#pragma unroll 8
    for (int r = 0; r < kZxRows; ++r) {
      const float4 a4 = *reinterpret_cast<const float4 *>(xs + r * kZxStride);
      const T a[4] = {(T)a4.x, (T)a4.y, (T)a4.z, (T)a4.w};
      T b[4];
      Vec4<T>::load(ws + r * kZxStride, b);
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
    }
    if (more) put(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int l = l0 + ty * 4 + u;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int cw = c0 + tx * 4 + v;
      if (l < p && cw < Kf) out[(int64_t)l * Kf + cw] = acc[u][v];
    }
  }
}

// C_Y outputs [o0, o0 + kZyOut) over observations [r0, r1).
template <typename T>
__device__ __forceinline__ void zy_part(const ZDims &D, const float *__restrict__ Y, const float *__restrict__ Z,
                                        const T *__restrict__ P, const T *__restrict__ zbar, int64_t r0, int64_t r1,
                                        int yc, T *__restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int K = D.K, d = D.d, f = D.f, Kf = K * f, df = d * f;
  const int64_t ny = (int64_t)K * df;
  const int64_t o0 = (int64_t)yc * kZyOut, o1 = o0 + kZyOut < ny ? o0 + kZyOut : ny;
  const int kb = (int)(o0 / df), ku = (int)((o1 - 1) / df) - kb + 1;
  const int YW = ku * d, WW = ku * f, R = D.zp.ry;
  float *Ys = reinterpret_cast<float *>(smem);                                   // [R][YW]
  T *Wy = reinterpret_cast<T *>(smem + (((size_t)R * YW * 4 + 15) & ~(size_t)15));  // [R][WW]
  const int tid = threadIdx.x;
  int yo[kZySlots], wo[kZySlots];
#pragma unroll
  for (int s = 0; s < kZySlots; ++s) {
    const int64_t o = o0 + tid + (int64_t)s * kZThreads;
    if (o < o1) {
      const int k = (int)(o / df), l = (int)((o / f) % d), j = (int)(o % f);
      yo[s] = (k - kb) * d + l;
      wo[s] = (k - kb) * f + j;
    } else {
      yo[s] = -1; wo[s] = 0;
    }
  }
  T acc[kZySlots];
#pragma unroll
  for (int s = 0; s < kZySlots; ++s) acc[s] = (T)0;
  for (int64_t rb = r0; rb < r1; rb += R) {
    const int nr = (int)(r1 - rb < R ? r1 - rb : R);
    __syncthreads();
    // Each thread owns fixed columns and moves kZBatch rows at a time, so that
    // kZBatch loads per operand are in flight.
    for (int c = tid; c < YW; c += kZThreads) {
      const float *src = Y + (rb * K + kb) * d + c;
      for (int q0 = 0; q0 < nr; q0 += kZBatch) {
        float v[kZBatch];
#pragma unroll
        for (int u = 0; u < kZBatch; ++u) v[u] = q0 + u < nr ? __ldg(src + (int64_t)(q0 + u) * K * d) : 0.f;
#pragma unroll
        for (int u = 0; u < kZBatch; ++u)
          if (q0 + u < nr) Ys[(q0 + u) * YW + c] = v[u];
      }
    }
    for (int c = tid; c < WW; c += kZThreads) {
      const int kk = c / f, j = c - kk * f;
      for (int q0 = 0; q0 < nr; q0 += kZBatch) {
        float zv[kZBatch];
        T pv[kZBatch], bv[kZBatch];
#pragma unroll
        for (int u = 0; u < kZBatch; ++u) {
          const int64_t i = rb + q0 + u;
          const bool in = q0 + u < nr;
          zv[u] = in ? __ldg(Z + i * Kf + (int64_t)kb * f + c) : 0.f;
          pv[u] = in ? P[i * K + kb + kk] * (D.w ? (T)D.w[i] : (T)1) : (T)0;
          bv[u] = in ? zbar[i * f + j] : (T)0;
        }
#pragma unroll
        for (int u = 0; u < kZBatch; ++u)
          if (q0 + u < nr) Wy[(q0 + u) * WW + c] = pv[u] * ((T)zv[u] - bv[u]);
      }
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < kZySlots; ++s) {
      if (yo[s] < 0) continue;
      T a0 = (T)0, a1 = (T)0;
      int r = 0;
      for (; r + 1 < nr; r += 2) {
        a0 = fma((T)Ys[r * YW + yo[s]], Wy[r * WW + wo[s]], a0);
        a1 = fma((T)Ys[(r + 1) * YW + yo[s]], Wy[(r + 1) * WW + wo[s]], a1);
      }
      if (r < nr) a0 = fma((T)Ys[r * YW + yo[s]], Wy[r * WW + wo[s]], a0);
      acc[s] += a0 + a1;
    }
  }
  const int64_t nx = (int64_t)D.p * Kf;
#pragma unroll
  for (int s = 0; s < kZySlots; ++s)
    if (yo[s] >= 0) out[nx + o0 + tid + (int64_t)s * kZThreads] = acc[s];
}

// Alpha block over observations [r0, r1).
template <typename T>
__device__ __forceinline__ void za_part(const ZDims &D, const float *__restrict__ Z, const T *__restrict__ P,
                                        const T *__restrict__ zbar, int64_t r0, int64_t r1, T *__restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int K = D.K, f = D.f, Kf = K * f, fs = D.zp.fs, R = D.zp.ra;
  const int nm4 = fs / 4, nm = nm4 * nm4;  // 4 x 4 micro-tiles of the f x f block
  T *Wa = reinterpret_cast<T *>(smem);      // [R*K][fs]
  T *Za = Wa + (size_t)R * K * fs;          // [R*K][fs]
  T *red = Za + (size_t)R * K * fs;         // [kZThreads][16]
  const int tid = threadIdx.x;
  const int64_t nx = (int64_t)D.p * Kf, ny = (int64_t)K * D.d * f;
  for (int m0 = 0; m0 < nm; m0 += kZThreads) {  // more than one pass only when f > 64
    const int nmp = nm - m0 < kZThreads ? nm - m0 : kZThreads;  // micro-tiles of this pass
    const int S = kZThreads / nmp;                               // thread subsets
    const int m = m0 + tid % nmp, s = tid / nmp;
    const bool act = s < S;
    const int mi = m / nm4, mj = m - mi * nm4;
    T acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[u][v] = (T)0;
    for (int64_t rb = r0; rb < r1; rb += R) {
      const int nr = (int)(r1 - rb < R ? r1 - rb : R);
      __syncthreads();
      for (int c = tid; c < K * fs; c += kZThreads) {  // fixed columns, kZBatch rows in flight
        const int kk = c / fs, j = c - kk * fs;
        const bool jin = j < f;
        for (int q0 = 0; q0 < nr; q0 += kZBatch) {
          float zv[kZBatch];
          T pv[kZBatch], bv[kZBatch];
#pragma unroll
          for (int u = 0; u < kZBatch; ++u) {
            const int64_t i = rb + q0 + u;
            const bool in = jin && q0 + u < nr;
            zv[u] = in ? __ldg(Z + i * Kf + kk * f + j) : 0.f;
            pv[u] = in ? P[i * K + kk] * (D.w ? (T)D.w[i] : (T)1) : (T)0;
            bv[u] = in ? zbar[i * f + j] : (T)0;
          }
#pragma unroll
          for (int u = 0; u < kZBatch; ++u) {
            if (q0 + u >= nr) continue;
            const T zc = (T)zv[u] - bv[u];
            Wa[((size_t)(q0 + u) * K) * fs + c] = pv[u] * zc;
            Za[((size_t)(q0 + u) * K) * fs + c] = zc;
          }
        }
      }
      __syncthreads();
      if (act) {
        const int ne = nr * K;
        for (int e = s; e < ne; e += S) {
          T a[4], b[4];
          Vec4<T>::load(Wa + (size_t)e * fs + mi * 4, a);
          Vec4<T>::load(Za + (size_t)e * fs + mj * 4, b);
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
        }
      }
    }
    // fixed-order sum over the subsets
    __syncthreads();
    if (act)
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) red[(size_t)tid * 16 + u * 4 + v] = acc[u][v];
    __syncthreads();
    for (int o = tid; o < f * f; o += kZThreads) {
      const int j1 = o / f, j2 = o - (o / f) * f;
      const int mo = (j1 / 4) * nm4 + j2 / 4;
      if (mo < m0 || mo >= m0 + nmp) continue;
      const int uv = (j1 & 3) * 4 + (j2 & 3);
      T v = (T)0;
      for (int ss = 0; ss < S; ++ss) v += red[(size_t)(ss * nmp + (mo - m0)) * 16 + uv];
      out[nx + ny + o] = v;
    }
  }
}

template <typename T>
__device__ __forceinline__ void zblocks_item(const ZDims &D, const float *__restrict__ X,
                                             const float *__restrict__ Y, const float *__restrict__ Z,
                                             const T *__restrict__ P, const T *__restrict__ zbar, int split,
                                             int part, T *__restrict__ out_row) {
  const int64_t r0 = D.N * split / D.nsplit, r1 = D.N * (split + 1) / D.nsplit;
  const int nxp = D.zp.nl * D.zp.nc;
  if (part < nxp) zx_part<T>(D, X, Z, P, zbar, r0, r1, part / D.zp.nc, part % D.zp.nc, out_row);
  else if (part < nxp + D.zp.ny) zy_part<T>(D, Y, Z, P, zbar, r0, r1, part - nxp, out_row);
  else za_part<T>(D, Z, P, zbar, r0, r1, out_row);
}

template <typename T>
__global__ void __launch_bounds__(kZThreads) zblocks_kernel(ZDims D, const float *__restrict__ X,
                                                            const float *__restrict__ Y, const float *__restrict__ Z,
                                                            const T *__restrict__ P, const T *__restrict__ zbar,
                                                            T *__restrict__ out) {
  zblocks_item<T>(D, X, Y, Z, P, zbar, blockIdx.y, blockIdx.x, out + (int64_t)blockIdx.y * D.nzt);
}

template <typename T>
__global__ void __launch_bounds__(kZThreads) grouped_zblocks_kernel(const GroupProblem *__restrict__ probs,
                                                                    const GroupItem *__restrict__ items,
                                                                    const int *__restrict__ active,
                                                                    T *__restrict__ zpart) {
  const GroupItem it = items[blockIdx.x];
  if (active[it.problem] == 0) return;
  const GroupProblem &g = probs[it.problem];
  ZDims D{};
  D.N = g.N; D.K = g.K; D.p = g.p; D.d = g.d; D.f = g.f;
  D.nsplit = g.zsplit;
  D.nzt = (int64_t)g.p * g.K * g.f + (int64_t)g.K * g.d * g.f + (int64_t)g.f * g.f;
  D.w = nullptr;
  D.zp = make_zplan(g.K, g.p, g.d, g.f, (int)sizeof(T));
  const int parts = D.zp.parts();
  const int split = it.idx / parts, part = it.idx % parts;
  zblocks_item<T>(D, g.X, g.Y, g.Z, reinterpret_cast<const T *>(g.P), reinterpret_cast<const T *>(g.zbar), split,
                  part, zpart + g.z_off + (int64_t)split * D.nzt);
}

// ---------------------------------------------------------------------------
// Assembly of F (lower triangle, column-major) in theta order.
// ---------------------------------------------------------------------------

// F(r, c), r >= c, from the partial sums.
// Entry (a, b) of the Gram matrix of the Z-block operand, summed over the splits.
__device__ __forceinline__ double zop_entry(const ZTileView &zv, int64_t a, int64_t b) {
  const int pair = zv.index[(a / kTile) * zv.nt + (b / kTile)];
  const int64_t within = (b % kTile) * kTile + (a % kTile);  // tiles are stored [b][a]
  float v = 0.f;
  for (int s = 0; s < zv.split; ++s) v += zv.part[((int64_t)s * zv.npairs + pair) * kTile * kTile + within];
  return (double)v;
}

// Class and local index of a class coefficient (theta index a < mc), 32-bit.
__device__ __forceinline__ void class_local32(const Shape &S, int a, int &k, int &l) {
  if (a < (int)S.nb) {
    k = a / S.p;
    l = a - k * S.p;
    ++k;
  } else {
    const int r = a - (int)S.nb;
    k = r / S.d;
    l = S.p + (r - k * S.d);
    ++k;
  }
}

// Sum over the splits of one partial entry: float32 partials are summed in
// float32 (a few terms; relative error ~1e-7), float64 ones in float64.
template <typename CT>
__device__ __forceinline__ double split_sum(const CT *__restrict__ base, int nsplit, int64_t stride) {
  CT v = (CT)0;
  for (int s = 0; s < nsplit; ++s) v += base[(int64_t)s * stride];
  return (double)v;
}

template <typename CT, typename ZT>
__device__ __forceinline__ double assemble_entry(const Shape &S, const CT *__restrict__ mainp, int msplit, int nmain,
                                                 const CT *__restrict__ bandp, int bsplit, int nband,
                                                 const int *__restrict__ band_of, int nt1d,
                                                 const ZT *__restrict__ zp, int zsplit, int64_t r, int64_t c,
                                                 const ZTileView &zv = ZTileView()) {
  const int q = S.q, f = S.f, K = S.K;
  const int64_t nx = (int64_t)S.p * K * f, ny = (int64_t)K * S.d * f, nzt = nx + ny + (int64_t)f * f;
  double v = 0.0;
  if (r < S.mc) {
    int kr, lr, kc, lc;
    class_local32(S, (int)r, kr, lr);
    class_local32(S, (int)c, kc, lc);
    const int ar = (kr - 1) * q + lr, ac = (kc - 1) * q + lc;
    const int ahi = ar > ac ? ar : ac, alo = ar > ac ? ac : ar;
    const int ti = ahi / kTile, tj = alo / kTile;
    const int within = (alo % kTile) * kTile + (ahi % kTile);  // tiles are stored [b][a]
    if (kr != kc) {
      const int64_t idx = (int64_t)ti * (ti + 1) / 2 + tj;
      return -split_sum<CT>(mainp + idx * kTile * kTile + within, msplit, (int64_t)nmain * kTile * kTile);
    }
    const int b = band_of[ti * nt1d + tj];
    return split_sum<CT>(bandp + (int64_t)b * kTile * kTile + within, bsplit, (int64_t)nband * kTile * kTile);
  } else if (c < S.mc) {
    const int j = (int)(r - S.mc);
    int kc, lc;
    theta_class_local(S, c, kc, lc);
    if (zv.part) {  // C_X = X W^T, C_Y = Y W^T (class kc)
      const int64_t a = lc < S.p ? (int64_t)lc : zv.oY + (int64_t)(kc - 1) * S.d + (lc - S.p);
      return zop_entry(zv, a, zv.oW + (int64_t)kc * f + j);
    }
    const int64_t off = lc < S.p ? (int64_t)lc * K * f + (int64_t)kc * f + j
                                 : nx + (int64_t)kc * S.d * f + (int64_t)(lc - S.p) * f + j;
    for (int s = 0; s < zsplit; ++s) v += (double)zp[s * nzt + off];
  } else {
    const int j1 = (int)(r - S.mc), j2 = (int)(c - S.mc);
    if (zv.part) {  // A = sum_k W_k Zc_k^T
      for (int k = 0; k < K; ++k) v += zop_entry(zv, zv.oW + (int64_t)k * f + j1, zv.oZ + (int64_t)k * f + j2);
      return v;
    }
    const int64_t off = nx + ny + (int64_t)j1 * f + j2;
    for (int s = 0; s < zsplit; ++s) v += (double)zp[s * nzt + off];
  }
  return v;
}

// Tiled assembly: one CTA per 32 x 32 tile (ti >= tj) of the lower triangle,
// one entry per thread.  The entries are written column by column (coalesced)
// and, through a transpose in shared memory, into the mirror tile row by row
// (coalesced too).
template <typename CT, typename ZT>
__global__ void __launch_bounds__(1024, 2) assemble_tiles_kernel(Shape S, const CT *__restrict__ mainp, int msplit,
                                                                 int nmain, const CT *__restrict__ bandp, int bsplit,
                                                                 int nband, const int *__restrict__ band_of, int nt1d,
                                                                 const ZT *__restrict__ zp, int zsplit, ZTileView zv,
                                                                 double *__restrict__ F, float *__restrict__ F32) {
  __shared__ double tile[32][33];  // tile[c - c0][r - r0]
  const int64_t n = S.n;
  const int t = (int)blockIdx.x;
  int ti = (int)((sqrtf(8.f * (float)t + 1.f) - 1.f) * 0.5f);
  while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
  while (ti * (ti + 1) / 2 > t) --ti;
  const int tj = t - ti * (ti + 1) / 2;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t r0 = (int64_t)ti * 32, c0 = (int64_t)tj * 32, r = r0 + tx, c = c0 + ty;
  double v = 0.0;
  if (r < n && c < n && r >= c) {
    v = assemble_entry<CT, ZT>(S, mainp, msplit, nmain, bandp, bsplit, nband, band_of, nt1d, zp, zsplit, r, c, zv);
    F[c * n + r] = v;
    if (F32) F32[c * n + r] = (float)v;
  }
  tile[ty][tx] = v;
  __syncthreads();
  const int64_t rr = r0 + ty, cc = c0 + tx;  // F(c, r) = F(r, c) for r > c: row r0 + ty, columns c0 + tx
  if (rr < n && cc < n && rr > cc) F[rr * n + cc] = tile[tx][ty];
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

size_t build_smem_bytes(const Shape &s, OpType t, int ob, int kc, bool with_z) {
  (void)ob;
  const size_t csz = t == OpType::F64 ? 8 : 4;
  return (size_t)2 * s.K * kBs * csz + ((size_t)s.p + (size_t)kc * s.d) * kBs * 4 +
         (with_z ? ((size_t)kc * s.f + s.f) * kBs * csz : 0) + (size_t)kBs * csz;  // + sqrt(w) of the block
}

// Classes per staging chunk: the most that keep three blocks on an SM (so that
// one block's staging overlaps the others' stores), else two, else one.
void build_blocking(const Shape &s, OpType t, int *ob, int *kc, bool with_z) {
  *ob = kBob;
  const int kmax = std::max(1, with_z ? s.K : s.K - 1);
  for (const size_t cap : {(size_t)74 * 1024, (size_t)112 * 1024, (size_t)200 * 1024}) {
    *kc = kmax;
    while (*kc > 1 && build_smem_bytes(s, t, *ob, *kc, with_z) > cap) --*kc;
    if (build_smem_bytes(s, t, *ob, *kc, with_z) <= cap) return;
  }
}

cudaError_t launch_build_operands(const Shape &s, OpType t, const float *X, const float *Y, const void *P, void *At,
                                  void *Ad, int64_t ldn, cudaStream_t st, const float *Z, const void *zbar, void *Az,
                                  const float *w) {
  BuildDims D{};
  D.w = w;
  D.N = s.N; D.ldn = ldn; D.K = s.K; D.p = s.p; D.d = s.d; D.q = s.q;
  D.rpA = (s.mc + kTile - 1) / kTile * kTile;
  D.rpZ = 0;
  const bool with_z = Az != nullptr && s.f > 0;
  build_blocking(s, t, &D.ob, &D.kc, with_z);
  D.f = with_z ? s.f : 0;
  D.oY = D.oW = D.oZ = 0;
  if (with_z) {
    const ZopLayout L = zop_layout(s);
    D.oY = L.oY; D.oW = L.oW; D.oZ = L.oZ;
    D.rpZ = L.rows_pad;
  }
  const size_t smem = build_smem_bytes(s, t, D.ob, D.kc, with_z);
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
      if (with_z) {
        auto k = build_operands_z_kernel<OpType::TF32, float>;
        if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return e;
        k<<<blocks, 256, smem, st>>>(D, X, Y, reinterpret_cast<const float *>(P), At, Ad, Z,
                                     reinterpret_cast<const float *>(zbar), Az);
      } else {
        auto k = build_operands_kernel<OpType::TF32, float>;
        if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return e;
        k<<<blocks, 256, smem, st>>>(D, X, Y, reinterpret_cast<const float *>(P), At, Ad);
      }
      break;
    }
    case OpType::BF16: {
      if (with_z) {
        auto k = build_operands_z_kernel<OpType::BF16, float>;
        if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return e;
        k<<<blocks, 256, smem, st>>>(D, X, Y, reinterpret_cast<const float *>(P), At, Ad, Z,
                                     reinterpret_cast<const float *>(zbar), Az);
      } else {
        auto k = build_operands_kernel<OpType::BF16, float>;
        if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return e;
        k<<<blocks, 256, smem, st>>>(D, X, Y, reinterpret_cast<const float *>(P), At, Ad);
      }
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

int zblocks_parts(const Shape &s, bool fp64) { return make_zplan(s.K, s.p, s.d, s.f, fp64 ? 8 : 4).parts(); }

size_t zblocks_smem(const Shape &s, bool fp64) {
  const size_t tsz = fp64 ? 8 : 4;
  const ZPlan z = make_zplan(s.K, s.p, s.d, s.f, (int)tsz);
  const size_t x = (size_t)2 * kZxRows * kZxStride * (4 + tsz);
  const size_t y = z.kspan ? (((size_t)z.ry * z.kspan * s.d * 4 + 15) & ~(size_t)15) + (size_t)z.ry * z.kspan * s.f * tsz
                           : 0;
  const size_t a = (size_t)2 * z.ra * s.K * z.fs * tsz + (size_t)kZThreads * 16 * tsz;
  return std::max(x, std::max(y, a));
}

cudaError_t launch_grouped_syrk_f64(const GroupProblem *probs, const SyrkUnit *units, int nunits, const int *active,
                                    double *out, cudaStream_t st) {
  if (nunits <= 0) return cudaSuccess;
  grouped_syrk_f64_kernel<<<nunits, 256, 0, st>>>(probs, units, active, out);
  return cudaGetLastError();
}

int f64_chunk_rows() { return kKc; }

cudaError_t launch_zblocks(const Shape &s, bool fp64, const float *X, const float *Y, const float *Z, const void *P,
                           const void *zbar, int nsplit, void *out, cudaStream_t st, const float *w) {
  ZDims D{};
  D.N = s.N; D.K = s.K; D.p = s.p; D.d = s.d; D.f = s.f;
  D.w = w;
  D.nsplit = nsplit;
  D.nzt = zblocks_outputs(s);
  D.zp = make_zplan(s.K, s.p, s.d, s.f, fp64 ? 8 : 4);
  const size_t smem = zblocks_smem(s, fp64);
  if (smem > 220 * 1024) return cudaErrorInvalidValue;
  dim3 grid(D.zp.parts(), nsplit);  // the parts of one split are dispatched together
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
  const int64_t nt = (s.n + 31) / 32;
  const unsigned grid = (unsigned)(nt * (nt + 1) / 2);
  const int block = 1024;
  const TileLists &tl = *io.tl;
  const int nt1d = (int)((s.mc + kTile - 1) / kTile);
  if (io.fp64) {
    assemble_tiles_kernel<double, double><<<grid, block, 0, st>>>(
        s, reinterpret_cast<const double *>(io.main_part), io.main_split, nmain,
        reinterpret_cast<const double *>(io.band_part), io.band_split, tl.nband, tl.band_of, nt1d,
        reinterpret_cast<const double *>(io.z_part), io.z_split, io.zt, F, io.f32);
  } else {
    assemble_tiles_kernel<float, float><<<grid, block, 0, st>>>(
        s, reinterpret_cast<const float *>(io.main_part), io.main_split, nmain,
        reinterpret_cast<const float *>(io.band_part), io.band_split, tl.nband, tl.band_of, nt1d,
        reinterpret_cast<const float *>(io.z_part), io.z_split, io.zt, F, io.f32);
  }
  return cudaGetLastError();
}

ZopLayout zop_layout(const Shape &s) {
  auto r128 = [](int64_t v) { return (v + kTile - 1) / kTile * kTile; };
  ZopLayout L;
  L.oY = r128(s.p);
  L.oW = L.oY + r128((int64_t)(s.K - 1) * s.d);
  L.oZ = L.oW + r128((int64_t)s.K * s.f);
  L.rows_pad = L.oZ + r128((int64_t)s.K * s.f);
  return L;
}

ZTiles zop_tiles(const Shape &s, const ZopLayout &L) {
  ZTiles z;
  z.nt = (int)(L.rows_pad / kTile);
  z.index.assign((size_t)z.nt * z.nt, -1);
  auto add = [&](int64_t ti, int64_t tj) {
    int &slot = z.index[(size_t)ti * z.nt + tj];
    if (slot < 0) { slot = (int)z.pairs.size(); z.pairs.push_back(make_int2((int)ti, (int)tj)); }
  };
  const int f = s.f, d = s.d;
  if (f == 0) return z;
  // C_X: every X tile with every W tile
  for (int64_t ti = 0; ti * kTile < s.p; ++ti)
    for (int64_t tj = L.oW / kTile; tj * kTile < L.oW + (int64_t)s.K * f; ++tj) add(ti, tj);
  // C_Y and A: tiles that hold rows of the same class
  for (int k = 0; k < s.K; ++k) {
    const int64_t w0 = (L.oW + (int64_t)k * f) / kTile, w1 = (L.oW + (int64_t)k * f + f - 1) / kTile;
    if (k >= 1 && d > 0) {
      const int64_t y0 = (L.oY + (int64_t)(k - 1) * d) / kTile, y1 = (L.oY + (int64_t)(k - 1) * d + d - 1) / kTile;
      for (int64_t a = y0; a <= y1; ++a)
        for (int64_t b = w0; b <= w1; ++b) add(a, b);
    }
    const int64_t z0 = (L.oZ + (int64_t)k * f) / kTile, z1 = (L.oZ + (int64_t)k * f + f - 1) / kTile;
    for (int64_t a = w0; a <= w1; ++a)
      for (int64_t b = z0; b <= z1; ++b) add(a, b);
  }
  return z;
}


namespace {
__global__ void export_probs_kernel(int64_t count, const void *__restrict__ P, int fp64, double *__restrict__ out) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = fp64 ? reinterpret_cast<const double *>(P)[e] : (double)reinterpret_cast<const float *>(P)[e];
}
}  // namespace

namespace {
// Packed lower triangle, column by column: entry (r, c), r >= c, at c n - c (c - 1) / 2 + (r - c).
__device__ __forceinline__ int64_t packed_index(int64_t n, int64_t r, int64_t c) { return c * n - c * (c - 1) / 2 + (r - c); }

__global__ void pack_lower_kernel(int64_t n, const double *__restrict__ F, double *__restrict__ out) {
  const int64_t c = blockIdx.y + (int64_t)gridDim.y * blockIdx.z;
  if (c >= n) return;
  for (int64_t r = c + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
    out[packed_index(n, r, c)] = F[c * n + r];
}

__global__ void unpack_lower_kernel(int64_t n, const double *__restrict__ in, double *__restrict__ F) {
  const int64_t c = blockIdx.y + (int64_t)gridDim.y * blockIdx.z;
  if (c >= n) return;
  for (int64_t r = c + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    const double v = in[packed_index(n, r, c)];
    F[c * n + r] = v;
    F[r * n + c] = v;
  }
}
}  // namespace

cudaError_t launch_pack_lower(int64_t n, const double *F, double *out, cudaStream_t st) {
  const dim3 grid((unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 32)),
                  (unsigned)std::min<int64_t>(n, 65535), (unsigned)((n + 65534) / 65535));
  pack_lower_kernel<<<grid, 256, 0, st>>>(n, F, out);
  return cudaGetLastError();
}

cudaError_t launch_unpack_lower(int64_t n, const double *in, double *F, cudaStream_t st) {
  const dim3 grid((unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 32)),
                  (unsigned)std::min<int64_t>(n, 65535), (unsigned)((n + 65534) / 65535));
  unpack_lower_kernel<<<grid, 256, 0, st>>>(n, in, F);
  return cudaGetLastError();
}

cudaError_t launch_export_probs(int64_t count, const void *P, bool fp64, double *out, cudaStream_t st) {
  const int64_t blocks = std::min<int64_t>((count + 255) / 256, 4096);
  export_probs_kernel<<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, st>>>(count, P, fp64 ? 1 : 0, out);
  return cudaGetLastError();
}

cudaError_t launch_export_hessian(int64_t n, const double *F, double *H, cudaStream_t st) {
  dim3 grid, block;
  grid_2d(n, n, grid, block);
  export_hessian_kernel<<<grid, block, 0, st>>>(n, F, H);
  return cudaGetLastError();
}

}  // namespace mnl
