// Fused float32 pass over the observations with asynchronous row-tile copies
// (Sec. 2.1 eqs. "unormalized utility", "probability", "base probability";
// Sec. 3.1 eq. "log-lik function"; Sec. 3.3 eq. "loglik gradient").
//
// Same results as the pass of pass.cu (utilities over all K alternatives from
// raw data, row softmax, l, P, zbar and g), organised for bandwidth:
//   * one or two CTAs per SM walk tiles of R = 8 * RPW consecutive observations; the
//     X, Y, Z and choice rows of a tile are contiguous in memory and arrive by
//     bulk asynchronous copies (cp.async.bulk, completion counted on an
//     mbarrier) into a ring of 2-3 shared-memory stages, so the next tiles
//     load while the current one is used (the last, partial tile is loaded
//     with plain loads);
//   * X is transposed in shared memory (column l at Xt + xcol(l), rows
//     contiguous; groups of 4 columns padded so that the gradient's 16-byte
//     reads of 8 column groups hit distinct banks) so that a warp reads RPW
//     rows of one column in one broadcast load; warp w forms the utilities of
//     rows RPW w .. RPW w + RPW - 1 with lanes over alternatives;
//   * the residuals r_ik = I(y_i = k) - P_ik are kept transposed (Rt[k][r]) and
//     the beta gradient X^T r of the tile is a register tile of 2 classes x 4
//     columns per thread fed by 16-byte loads; gamma and alpha entries are
//     owned by threads; every per-tile float32 sum is folded into a
//     Kahan-compensated running sum;
//   * each CTA writes its float64 partial row [l, sum |l_i|, g] for the fixed
//     order reduction (pass_reduce_kernel).
// The wait on a stage is bounded (2 s on %globaltimer); a wait that runs out
// sets *err and the CTA stops after waiting (bounded) for its copies in flight.
#include <cfloat>

#include "mnl_internal.cuh"

namespace mnl {
namespace {

constexpr int kPT = 256;          // threads per CTA
constexpr int kBetaItems = 2;     // beta-gradient register tiles per warp
// gamma / alpha outputs per thread: YZS (a template parameter) = 2, or 4 when (K-1) d + K f > 512
constexpr int kRegYZ = 8;         // d, f up to this: gamma and alpha coefficients in registers
constexpr uint64_t kTileWaitNs = 2000000000ull;
constexpr int kGbRows = 32;   // beta-gradient kernel: observations per tile
constexpr int kGbStages = 3;  // and stages of its copy ring
constexpr int kGbMaxJ = 8, kGbMaxK = 8;  // its register tile: up to 16 * 8 columns x 16 * 8 classes

struct TileDims {
  int64_t N, ntiles;
  int K, p, d, f, Kpad, R, R4, S, pp;
  int xq;  // Xt: columns in groups of 4 rows of R4, groups xq = 4 R4 + 4 apart (conflict-free 16-byte reads)
  int nb, mc, n;
  int stage_bytes, off_x, off_y, off_z, off_c;                       // within a stage
  int off_bt, off_gt, off_al, off_xt, off_rt, off_red, off_bar, off_stage;
  int kp2, lq, wk, wl, nyz;                                          // gradient work
  int beta_ext;  // the beta gradient is left to grad_beta_kernel (too many outputs for the register tiles)
  int ux;        // the X-block utilities come precomputed (io.ux): the stage holds their rows instead of X's
};

struct KahanF {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float v) {
    const float y = v - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

__device__ __forceinline__ uint32_t sa(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t gclock() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void bulk_copy(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(sa(dst)),
      "l"(src), "r"(bytes), "r"(sa(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_done(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(sa(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for phase `parity` of a stage barrier.
// bound_ns = 0: kTileWaitNs.  Waits for copies already issued before a CTA
// stops (the drain) always use kTileWaitNs.
__device__ __forceinline__ bool stage_wait(uint64_t *bar, uint32_t parity, uint64_t bound_ns = 0) {
  if (mbar_done(bar, parity)) return true;
  const uint64_t lim = bound_ns ? bound_ns : kTileWaitNs;
  const uint64_t t0 = gclock();
  while (!mbar_done(bar, parity))
    if (gclock() - t0 > lim) return false;
  return true;
}

__device__ __forceinline__ float wmax(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ float wsum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <int RPW>
__device__ __forceinline__ void load_rows(const float *p, float v[RPW]) {
  if (RPW == 4) {
    const float4 a = *reinterpret_cast<const float4 *>(p);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  } else if (RPW == 2) {
    const float2 a = *reinterpret_cast<const float2 *>(p);
    v[0] = a.x; v[1] = a.y;
  } else {
    v[0] = p[0];
  }
}

// kYZSlots = 4 is the wide-shape variant (one CTA per SM: its ring fills the shared memory).
template <int RPW, int CS, bool FULL, int kYZSlots>
__global__ void __launch_bounds__(kPT, kYZSlots == 4 ? 1 : 2) pass_tile_kernel(TileDims D, PassIO io) {
  extern __shared__ __align__(128) unsigned char sm[];
  float *Bt = reinterpret_cast<float *>(sm + D.off_bt);  // [p][Kpad]
  float *Gt = reinterpret_cast<float *>(sm + D.off_gt);  // [d][Kpad]
  float *al = reinterpret_cast<float *>(sm + D.off_al);  // [f]
  float *Xt = reinterpret_cast<float *>(sm + D.off_xt);  // column l at xcol(l)
  float *Rt = reinterpret_cast<float *>(sm + D.off_rt);  // [Kpad][R4] (FULL)
  double *red = reinterpret_cast<double *>(sm + D.off_red);
  uint64_t *bar = reinterpret_cast<uint64_t *>(sm + D.off_bar);
  __shared__ int s_abort;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int K = D.K, p = D.p, d = D.d, f = D.f, Kpad = D.Kpad, R = D.R, R4 = D.R4;
  const int64_t N = D.N;
  auto xcol = [&](int l) { return (l >> 2) * D.xq + (l & 3) * R4; };
  constexpr int kR = 8 * RPW, kRsh = RPW == 4 ? 5 : RPW == 2 ? 4 : 3;  // rows per tile, log2

  // coefficients theta (+ t delta), zero for the base alternative and the padding
  const double tsc = io.delta ? *io.tscale : 0.0;
  auto coef = [&](int64_t a) { return io.theta[a] + (io.delta ? tsc * io.delta[a] : 0.0); };
  if (!D.ux)
    for (int e = tid; e < p * Kpad; e += kPT) {
      const int j = e / Kpad, k = e - j * Kpad;
      Bt[e] = (k >= 1 && k < K) ? (float)coef((int64_t)(k - 1) * p + j) : 0.f;
    }
  for (int e = tid; e < d * Kpad; e += kPT) {
    const int j = e / Kpad, k = e - j * Kpad;
    Gt[e] = (k >= 1 && k < K) ? (float)coef(D.nb + (int64_t)(k - 1) * d + j) : 0.f;
  }
  for (int j = tid; j < f; j += kPT) al[j] = (float)coef(D.mc + j);
  if (!D.ux)
    for (int e = p * R4 + tid; e < D.pp * R4; e += kPT) Xt[xcol(e / R4) + e % R4] = 0.f;  // padding columns
  if (FULL)
    for (int e = tid; e < R4; e += kPT) Rt[Kpad * R4 + e] = 0.f;       // row read by the last class pair
  if (tid == 0) {
    s_abort = 0;
    for (int s = 0; s < D.S; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sa(&bar[s])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  const int px = D.ux ? K : p;  // floats per observation in the stage's first block (U_x or X)
  const float *xsrc = D.ux ? io.ux : io.X;
  const uint32_t tile_bytes = (uint32_t)(R * (px + K * d + K * f + 1) * 4);
  auto full_tile = [&](int64_t tl) { return (tl + 1) * R <= N; };
  auto issue = [&](int64_t tl, int s) {  // one thread
    const int64_t row0 = tl * R;
    unsigned char *st = sm + D.off_stage + s * D.stage_bytes;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sa(&bar[s])), "r"(tile_bytes)
                 : "memory");
    bulk_copy(st + D.off_x, xsrc + row0 * px, (uint32_t)(R * px * 4), &bar[s]);
    if (d) bulk_copy(st + D.off_y, io.Y + row0 * K * d, (uint32_t)(R * K * d * 4), &bar[s]);
    if (f) bulk_copy(st + D.off_z, io.Z + row0 * K * f, (uint32_t)(R * K * f * 4), &bar[s]);
    bulk_copy(st + D.off_c, io.choice + row0, (uint32_t)(R * 4), &bar[s]);
  };
  int pend[3] = {-1, -1, -1};  // thread 0: per stage, parity of a copy not yet waited for
  if (tid == 0)
    for (int s = 0; s < D.S; ++s) {
      const int64_t tl = blockIdx.x + (int64_t)s * gridDim.x;
      if (tl < D.ntiles && full_tile(tl)) { issue(tl, s); pend[s] = 0; }
    }

  KahanF lsum, labs;                   // lane 0 of each warp
  KahanF bs[kBetaItems][8];            // beta gradient: 2 classes x 4 columns per item
  KahanF yz[kYZSlots];                 // gamma entries and alpha partials per class
  int yz_k[kYZSlots], yz_j[kYZSlots];  // decoded once: class and column, yz_j < 0 for alpha
#pragma unroll
  for (int q = 0; q < kYZSlots; ++q) {
    const int e = tid + q * kPT;
    yz_k[q] = -1; yz_j[q] = 0;
    if (FULL && e < D.nyz) {
      const int ng = (K - 1) * d;
      if (e < ng) { yz_k[q] = 1 + e / d; yz_j[q] = e - (e / d) * d; }
      else { const int e2 = e - ng; yz_k[q] = e2 / f; yz_j[q] = -1 - (e2 - (e2 / f) * f); }
    }
  }

  // this lane's gamma coefficients (classes lane + 32 c) and alpha, in
  // registers when d, f <= kRegYZ (they do not change during the pass)
  const bool yz_reg = d <= kRegYZ && f <= kRegYZ;
  float gr[CS][kRegYZ], ar[kRegYZ];
#pragma unroll
  for (int j = 0; j < kRegYZ; ++j) {
    ar[j] = (yz_reg && j < f) ? al[j] : 0.f;
#pragma unroll
    for (int c = 0; c < CS; ++c) gr[c][j] = (yz_reg && j < d) ? Gt[j * Kpad + lane + 32 * c] : 0.f;
  }

  int it = 0;
  for (int64_t tl = blockIdx.x; tl < D.ntiles; tl += gridDim.x, ++it) {
    const int s = it % D.S;
    const uint32_t par = (uint32_t)((it / D.S) & 1);
    unsigned char *st = sm + D.off_stage + s * D.stage_bytes;
    float *Xs = reinterpret_cast<float *>(st + D.off_x);
    float *Ys = reinterpret_cast<float *>(st + D.off_y);
    float *Zs = reinterpret_cast<float *>(st + D.off_z);
    int *cs = reinterpret_cast<int *>(st + D.off_c);
    const int64_t row0 = tl * R;
    const int nrows = (int)(N - row0 < R ? N - row0 : R);
    if (nrows == R) {
      if (!stage_wait(&bar[s], par, io.wait_ns)) s_abort = 1;
      else if (tid == 0) pend[s] = -1;
    } else {  // the partial last tile: plain loads, zero padding
      for (int e = tid; e < R * px; e += kPT) Xs[e] = e < nrows * px ? xsrc[row0 * px + e] : 0.f;
      for (int e = tid; e < R * K * d; e += kPT) Ys[e] = e < nrows * K * d ? io.Y[row0 * K * d + e] : 0.f;
      for (int e = tid; e < R * K * f; e += kPT) Zs[e] = e < nrows * K * f ? io.Z[row0 * K * f + e] : 0.f;
      for (int e = tid; e < R; e += kPT) cs[e] = e < nrows ? io.choice[row0 + e] : -1;
    }
    __syncthreads();
    if (s_abort) break;
    if (!D.ux) {
      for (int e = tid; e < kR * p; e += kPT) {  // lanes over rows: no division, conflict-free
        const int r = e & (kR - 1), l = e >> kRsh;
        Xt[xcol(l) + r] = Xs[r * p + l];
      }
      __syncthreads();
    }

    // ---- utilities, softmax, l (and P, residuals, zbar) ----
    {
      const int r0 = warp * RPW;
      float u[RPW][CS];
#pragma unroll
      for (int r = 0; r < RPW; ++r)
#pragma unroll
        for (int c = 0; c < CS; ++c) u[r][c] = 0.f;
      if (D.ux) {  // precomputed x_i . beta_k
#pragma unroll
        for (int c = 0; c < CS; ++c) {
          const int k = lane + 32 * c;
#pragma unroll
          for (int r = 0; r < RPW; ++r) u[r][c] = k < K ? Xs[(r0 + r) * K + k] : 0.f;
        }
      } else {
#pragma unroll 2
        for (int j = 0; j < p; ++j) {
          float xv[RPW];
          load_rows<RPW>(Xt + xcol(j) + r0, xv);
#pragma unroll
          for (int c = 0; c < CS; ++c) {
            const float b = Bt[j * Kpad + lane + 32 * c];
#pragma unroll
            for (int r = 0; r < RPW; ++r) u[r][c] = fmaf(xv[r], b, u[r][c]);
          }
        }
      }
#pragma unroll
      for (int c = 0; c < CS; ++c) {
        const int k = lane + 32 * c;
        if (k >= K) continue;
#pragma unroll
        for (int r = 0; r < RPW; ++r) {
          const float *y = Ys + ((size_t)(r0 + r) * K + k) * d;
          const float *z = Zs + ((size_t)(r0 + r) * K + k) * f;
          if (yz_reg) {
#pragma unroll
            for (int j = 0; j < kRegYZ; ++j) {
              if (j < d) u[r][c] = fmaf(y[j], gr[c][j], u[r][c]);
              if (j < f) u[r][c] = fmaf(z[j], ar[j], u[r][c]);
            }
          } else {
            for (int j = 0; j < d; ++j) u[r][c] = fmaf(y[j], Gt[j * Kpad + k], u[r][c]);
            for (int j = 0; j < f; ++j) u[r][c] = fmaf(z[j], al[j], u[r][c]);
          }
        }
      }
      float res[CS][RPW];  // residuals of this lane's classes for the warp's rows
#pragma unroll
      for (int r = 0; r < RPW; ++r) {
        const int rr = r0 + r;
        const bool vr = rr < nrows;
        const int yi = cs[rr];
        const float wr = (io.w && vr) ? __ldg(io.w + row0 + rr) : 1.f;  // case weight
        if (FULL && io.Pin) {  // Hessian-vector product: r_ik = w_i P_ik (u_ik - ubar_i)
          const float *Pr = reinterpret_cast<const float *>(io.Pin) + (row0 + rr) * K;
          float pk[CS], ub = 0.f;
#pragma unroll
          for (int c = 0; c < CS; ++c) {
            const int k = lane + 32 * c;
            pk[c] = (k < K && vr) ? __ldg(Pr + k) : 0.f;
            ub = fmaf(pk[c], u[r][c], ub);
          }
          ub = wsum(ub);
#pragma unroll
          for (int c = 0; c < CS; ++c) {
            const int k = lane + 32 * c;
            res[c][r] = wr * pk[c] * (u[r][c] - ub);
            if (io.Wout && k < K && vr) io.Wout[(row0 + rr) * K + k] = res[c][r];
          }
          continue;
        }
        float m = -FLT_MAX;
#pragma unroll
        for (int c = 0; c < CS; ++c)
          if (lane + 32 * c < K) m = fmaxf(m, u[r][c]);
        m = wmax(m);
        float sum = 0.f, uy = 0.f;
#pragma unroll
        for (int c = 0; c < CS; ++c) {
          const int k = lane + 32 * c;
          if (k < K) {
            if (k == yi) uy = u[r][c];
            u[r][c] = expf(u[r][c] - m);
            sum += u[r][c];
          } else {
            u[r][c] = 0.f;
          }
        }
        sum = wsum(sum);
        uy = wsum(uy);
        if (vr && lane == 0) {
          const float li = uy - (m + logf(sum));
          lsum.add(wr * li);
          labs.add(wr * fabsf(li));
        }
        if (FULL) {
          const float inv = 1.f / sum;
          float *Pg = reinterpret_cast<float *>(io.P) + (row0 + rr) * K;
#pragma unroll
          for (int c = 0; c < CS; ++c) {
            const int k = lane + 32 * c;
            const float P = u[r][c] * inv;
            u[r][c] = P;
            if (k < K && vr) Pg[k] = P;
            res[c][r] = (k < K && vr) ? wr * ((k == yi ? 1.f : 0.f) - P) : 0.f;
          }
          for (int j = 0; j < f; ++j) {
            float zb = 0.f;
#pragma unroll
            for (int c = 0; c < CS; ++c) {
              const int k = lane + 32 * c;
              if (k < K) zb = fmaf(u[r][c], Zs[((size_t)rr * K + k) * f + j], zb);
            }
            zb = wsum(zb);
            if (vr && lane == 0) reinterpret_cast<float *>(io.zbar)[(row0 + rr) * f + j] = zb;
          }
        }
      }
      if (FULL) {
#pragma unroll
        for (int c = 0; c < CS; ++c) {
          float *dst = Rt + (lane + 32 * c) * R4 + r0;
          if (RPW == 4) *reinterpret_cast<float4 *>(dst) = make_float4(res[c][0], res[c][1], res[c][2], res[c][3]);
          else if (RPW == 2) *reinterpret_cast<float2 *>(dst) = make_float2(res[c][0], res[c][1]);
          else dst[0] = res[c][0];
        }
      }
    }

    if (FULL) {
      __syncthreads();  // residuals of every row are in Rt
      // ---- beta gradient: warp item (wkp, wlq) covers classes 1 + 2 kp, 2 + 2 kp and columns 4 lq .. 4 lq + 3 ----
      const int nitems = D.beta_ext ? 0 : D.wk * D.wl;
#pragma unroll
      for (int ii = 0; ii < kBetaItems; ++ii) {
        const int item = warp + 8 * ii;
        if (item >= nitems) break;
        const int kp = (item / D.wl) * 4 + (lane >> 3), lq = (item % D.wl) * 8 + (lane & 7);
        if (kp >= D.kp2 || lq >= D.lq) continue;
        const int k1 = 1 + 2 * kp, l0 = 4 * lq;
        float a[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) a[q] = 0.f;
        for (int r = 0; r < R; r += 4) {
          const float4 ra = *reinterpret_cast<const float4 *>(Rt + k1 * R4 + r);
          const float4 rb = *reinterpret_cast<const float4 *>(Rt + (k1 + 1) * R4 + r);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float4 x = *reinterpret_cast<const float4 *>(Xt + xcol(l0 + q) + r);
            a[q] = fmaf(ra.x, x.x, fmaf(ra.y, x.y, fmaf(ra.z, x.z, fmaf(ra.w, x.w, a[q]))));
            a[4 + q] = fmaf(rb.x, x.x, fmaf(rb.y, x.y, fmaf(rb.z, x.z, fmaf(rb.w, x.w, a[4 + q]))));
          }
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) bs[ii][q].add(a[q]);
      }
      // ---- gamma entries and per-class alpha partials ----
#pragma unroll
      for (int q = 0; q < kYZSlots; ++q) {
        const int k = yz_k[q];
        if (k < 0) continue;
        const int j = yz_j[q];
        const float *src = j >= 0 ? Ys + (size_t)k * d + j : Zs + (size_t)k * f + (-1 - j);
        const int stride = j >= 0 ? K * d : K * f;
        float a0 = 0.f, a1 = 0.f;
        for (int r = 0; r < R; r += 2) {
          a0 = fmaf(Rt[k * R4 + r], src[(size_t)r * stride], a0);
          a1 = fmaf(Rt[k * R4 + r + 1], src[(size_t)(r + 1) * stride], a1);
        }
        yz[q].add(a0 + a1);
      }
    }
    __syncthreads();  // the stage, Xt and Rt are free
    if (tid == 0) {
      const int64_t nx = tl + (int64_t)D.S * gridDim.x;
      if (nx < D.ntiles && full_tile(nx)) { issue(nx, s); pend[s] = (int)(((it + D.S) / D.S) & 1); }
    }
  }
  if (s_abort) {
    if (tid == 0) {
      atomicOr(io.err, 16);
      // no copy may still be writing into shared memory when the CTA exits
      for (int s = 0; s < D.S; ++s)
        if (pend[s] >= 0) stage_wait(&bar[s], (uint32_t)pend[s]);
    }
    __syncthreads();
    return;
  }

  // ---- CTA partial row: [l, sum |l_i|, g (theta order)] ----
  double *out = io.partials + (int64_t)blockIdx.x * (FULL ? 2 + D.n : 2);
  if (lane == 0) {
    red[2 * warp] = lsum.value();
    red[2 * warp + 1] = labs.value();
  }
  __syncthreads();
  if (tid == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < kPT / 32; ++w) { a += red[2 * w]; b += red[2 * w + 1]; }
    out[0] = a;
    out[1] = b;
  }
  if (!FULL) return;
  const int nitems = D.beta_ext ? 0 : D.wk * D.wl;
#pragma unroll
  for (int ii = 0; ii < kBetaItems; ++ii) {
    const int item = warp + 8 * ii;
    if (item >= nitems) break;
    const int kp = (item / D.wl) * 4 + (lane >> 3), lq = (item % D.wl) * 8 + (lane & 7);
    if (kp >= D.kp2 || lq >= D.lq) continue;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int k = 1 + 2 * kp + h;
      if (k >= K) continue;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int l = 4 * lq + q;
        if (l < p) out[2 + (int64_t)(k - 1) * p + l] = bs[ii][4 * h + q].value();
      }
    }
  }
  // gamma directly; alpha partials per class through shared memory, summed over k in fixed order
  __syncthreads();
#pragma unroll
  for (int q = 0; q < kYZSlots; ++q) {
    const int k = yz_k[q];
    if (k < 0) continue;
    const int j = yz_j[q];
    if (j >= 0) out[2 + D.nb + (int64_t)(k - 1) * d + j] = yz[q].value();
    else red[k * f + (-1 - j)] = yz[q].value();
  }
  __syncthreads();
  for (int j = tid; j < f; j += kPT) {
    double sa2 = 0.0;
    for (int k = 0; k < K; ++k) sa2 += red[k * f + j];
    out[2 + D.mc + j] = sa2;
  }
}

// ---------------------------------------------------------------------------
// beta gradient for shapes whose (K - 1) p outputs do not fit the pass's
// register tiles (eq. "loglik gradient"):  g_beta_k[j] = sum_i x_ij (I(y_i = k) - P_ik).
// A tall-skinny product X^T R over the observations, R = onehot(y) - P, run
// after the pass on the same grid: CTA b takes the tiles of kGbRows
// observations b, b + grid, ... (X, P and choice rows by bulk asynchronous
// copies into a 3-stage ring, bounded waits) and writes the beta entries of
// its own partial row.  Thread (tx, ty) of a 16 x 16 grid owns the outputs
// j = tx + 16 a (a < JA), k = ty + 16 b (b < KB); per tile the float32 sums
// are folded into Kahan-compensated running sums.
// ---------------------------------------------------------------------------
template <int JA, int KB>
__global__ void __launch_bounds__(256, 1) grad_beta_kernel(int64_t N, int K, int p, int64_t n,
                                                           const float *__restrict__ X, const float *__restrict__ P,
                                                           const int *__restrict__ choice, const float *w,
                                                           double *partials, int *err, uint64_t wait_ns,
                                                           int p_is_residual) {
  extern __shared__ __align__(128) unsigned char sm[];
  const int sx = ((kGbRows * p * 4) + 127) & ~127, sp = ((kGbRows * K * 4) + 127) & ~127;
  const int stage_bytes = sx + sp + 256;
  uint64_t *bar = reinterpret_cast<uint64_t *>(sm + kGbStages * stage_bytes);
  __shared__ int s_abort;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t ntiles = (N + kGbRows - 1) / kGbRows;
  if (tid == 0) {
    s_abort = 0;
    for (int st = 0; st < kGbStages; ++st)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sa(&bar[st])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const uint32_t tile_bytes = (uint32_t)(kGbRows * (p + K + 1 + (w ? 1 : 0)) * 4);
  auto full_tile = [&](int64_t tl) { return (tl + 1) * kGbRows <= N; };
  auto issue = [&](int64_t tl, int st) {
    const int64_t r0 = tl * kGbRows;
    unsigned char *b = sm + st * stage_bytes;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sa(&bar[st])), "r"(tile_bytes)
                 : "memory");
    bulk_copy(b, X + r0 * p, (uint32_t)(kGbRows * p * 4), &bar[st]);
    bulk_copy(b + sx, P + r0 * K, (uint32_t)(kGbRows * K * 4), &bar[st]);
    bulk_copy(b + sx + sp, choice + r0, (uint32_t)(kGbRows * 4), &bar[st]);
    if (w) bulk_copy(b + sx + sp + 128, w + r0, (uint32_t)(kGbRows * 4), &bar[st]);
  };
  int pend[kGbStages];
  for (int st = 0; st < kGbStages; ++st) pend[st] = -1;
  if (tid == 0)
    for (int st = 0; st < kGbStages; ++st) {
      const int64_t tl = blockIdx.x + (int64_t)st * gridDim.x;
      if (tl < ntiles && full_tile(tl)) { issue(tl, st); pend[st] = 0; }
    }
  KahanF ks[JA][KB];
  int it = 0;
  for (int64_t tl = blockIdx.x; tl < ntiles; tl += gridDim.x, ++it) {
    const int st = it % kGbStages;
    const uint32_t par = (uint32_t)((it / kGbStages) & 1);
    unsigned char *b = sm + st * stage_bytes;
    float *Xs = reinterpret_cast<float *>(b);
    float *Ps = reinterpret_cast<float *>(b + sx);
    int *cs = reinterpret_cast<int *>(b + sx + sp);
    float *ws = reinterpret_cast<float *>(b + sx + sp + 128);
    const int64_t r0 = tl * kGbRows;
    const int nrows = (int)(N - r0 < kGbRows ? N - r0 : kGbRows);
    if (nrows == kGbRows) {
      if (!stage_wait(&bar[st], par, wait_ns)) s_abort = 1;
      else if (tid == 0) pend[st] = -1;
    } else {  // the partial last tile: plain loads, zero padding
      for (int e = tid; e < kGbRows * p; e += 256) Xs[e] = e < nrows * p ? X[r0 * p + e] : 0.f;
      for (int e = tid; e < kGbRows * K; e += 256) Ps[e] = e < nrows * K ? P[r0 * K + e] : 0.f;
      for (int e = tid; e < kGbRows; e += 256) cs[e] = e < nrows ? choice[r0 + e] : -1;
      if (w)
        for (int e = tid; e < kGbRows; e += 256) ws[e] = e < nrows ? w[r0 + e] : 0.f;
    }
    __syncthreads();
    if (s_abort) break;
    if (!p_is_residual) {  // residuals w_i (I(y_i = k) - P_ik) of the tile, in place of P (once per tile)
      for (int e = tid; e < kGbRows * K; e += 256) {
        const int r = e / K, k = e - r * K;
        const float wr = w ? ws[r] : 1.f;
        Ps[e] = wr * ((k == cs[r] ? 1.f : 0.f) - Ps[e]);
      }
      __syncthreads();
    }
    float acc[JA][KB];
#pragma unroll
    for (int a = 0; a < JA; ++a)
#pragma unroll
      for (int c = 0; c < KB; ++c) acc[a][c] = 0.f;
#pragma unroll 2
    for (int r = 0; r < kGbRows; ++r) {
      float x[JA], rr[KB];
#pragma unroll
      for (int a = 0; a < JA; ++a) {
        const int j = tx + 16 * a;
        x[a] = j < p ? Xs[r * p + j] : 0.f;
      }
#pragma unroll
      for (int c = 0; c < KB; ++c) {
        const int k = ty + 16 * c;
        rr[c] = k < K ? Ps[r * K + k] : 0.f;
      }
#pragma unroll
      for (int a = 0; a < JA; ++a)
#pragma unroll
        for (int c = 0; c < KB; ++c) acc[a][c] = fmaf(x[a], rr[c], acc[a][c]);
    }
#pragma unroll
    for (int a = 0; a < JA; ++a)
#pragma unroll
      for (int c = 0; c < KB; ++c) ks[a][c].add(acc[a][c]);
    __syncthreads();  // the stage is free
    if (tid == 0) {
      const int64_t nx = tl + (int64_t)kGbStages * gridDim.x;
      if (nx < ntiles && full_tile(nx)) { issue(nx, st); pend[st] = (int)(((it + kGbStages) / kGbStages) & 1); }
    }
  }
  if (s_abort) {
    if (tid == 0) {
      atomicOr(err, 16);
      for (int st = 0; st < kGbStages; ++st)
        if (pend[st] >= 0) stage_wait(&bar[st], (uint32_t)pend[st]);
    }
    __syncthreads();
    return;
  }
  double *out = partials + (int64_t)blockIdx.x * (2 + n);
#pragma unroll
  for (int a = 0; a < JA; ++a)
#pragma unroll
    for (int c = 0; c < KB; ++c) {
      const int j = tx + 16 * a, k = ty + 16 * c;
      if (j < p && k >= 1 && k < K) out[2 + (int64_t)(k - 1) * p + j] = ks[a][c].value();
    }
}

size_t grad_beta_smem(int K, int p) {
  const int sx = ((kGbRows * p * 4) + 127) & ~127, sp = ((kGbRows * K * 4) + 127) & ~127;
  return (size_t)kGbStages * (sx + sp + 256) + kGbStages * 8;
}

template <int JA, int KB>
cudaError_t launch_gb(const Shape &s, int grid, const PassIO &io, cudaStream_t st) {
  auto kern = grad_beta_kernel<JA, KB>;
  const size_t smem = grad_beta_smem(s.K, s.p);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // Hessian-vector mode: the residuals w_i P_ik (u_ik - ubar_i) written by the pass stand in for P
  const bool hv = io.Pin != nullptr;
  kern<<<grid, 256, smem, st>>>(s.N, s.K, s.p, s.n, io.X, hv ? io.Wout : reinterpret_cast<const float *>(io.P),
                                io.choice, hv ? nullptr : io.w, io.partials, io.err, io.wait_ns, hv ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_grad_beta(const Shape &s, int grid, const PassIO &io, cudaStream_t st) {
  const int ja = (s.p + 15) / 16, kb = (s.K + 15) / 16;
  // register tiles of 4, 7 or 8 (columns) x 4, 7 or 8 (classes)
  const int JA = ja <= 4 ? 4 : ja <= 7 ? 7 : 8, KBv = kb <= 4 ? 4 : kb <= 7 ? 7 : 8;
  if (ja > 8 || kb > 8) return cudaErrorInvalidValue;
#define MNL_GB(a, b) if (JA == a && KBv == b) return launch_gb<a, b>(s, grid, io, st);
  MNL_GB(4, 4) MNL_GB(4, 7) MNL_GB(4, 8) MNL_GB(7, 4) MNL_GB(7, 7) MNL_GB(7, 8) MNL_GB(8, 4) MNL_GB(8, 7) MNL_GB(8, 8)
#undef MNL_GB
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// Utilities of the individual-specific block for wide shapes (eq. "unormalized
// utility"): U_x[i][k] = x_i . beta_k (beta_0 = 0) as the float32 product
// U_x = X B, B[l][k] = beta_k[l] rounded to float32 as in the fused pass.
// For these shapes the product is most of the pass's arithmetic; as a
// register-tiled GEMM (CTA tile 128 observations x 128 classes, 16 columns of
// X per step through shared memory, 8 x 8 outputs per thread) it runs at the
// FMA rate instead of the shared-memory load rate of the fused loop.
// ---------------------------------------------------------------------------
constexpr int kUgM = 128, kUgN = 128, kUgK = 16;

__global__ void __launch_bounds__(256) ux_coef_kernel(int p, int K, int ldb, const double *__restrict__ theta,
                                                      const double *__restrict__ delta,
                                                      const double *__restrict__ tscale, float *__restrict__ Bf) {
  const double t = delta ? *tscale : 0.0;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < p * ldb; e += gridDim.x * blockDim.x) {
    const int l = e / ldb, k = e - l * ldb;
    float v = 0.f;
    if (k >= 1 && k < K) {
      const int64_t a = (int64_t)(k - 1) * p + l;
      v = (float)(theta[a] + (delta ? t * delta[a] : 0.0));
    }
    Bf[e] = v;
  }
}

__global__ void __launch_bounds__(256, 2) ux_gemm_kernel(int64_t N, int p, int K, int ldb,
                                                         const float *__restrict__ X, const float *__restrict__ Bf,
                                                         float *__restrict__ U) {
  __shared__ __align__(16) float As[kUgK][kUgM + 4];  // As[l][r] = X[row0 + r][l0 + l]
  __shared__ __align__(16) float Bs[kUgK][kUgN];      // Bs[l][c] = B[l0 + l][col0 + c]
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t row0 = (int64_t)blockIdx.x * kUgM;
  const int col0 = blockIdx.y * kUgN;
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
  float xa[8], xb[8];
  auto load = [&](int l0) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = tid + 256 * u, r = e >> 4, l = e & 15;
      xa[u] = (row0 + r < N && l0 + l < p) ? X[(row0 + r) * p + l0 + l] : 0.f;
      const int lb = e >> 7, c = e & 127;
      xb[u] = (l0 + lb < p) ? Bf[(int64_t)(l0 + lb) * ldb + col0 + c] : 0.f;
    }
  };
  load(0);
  for (int l0 = 0; l0 < p; l0 += kUgK) {
    __syncthreads();  // the previous step is done with As, Bs
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = tid + 256 * u;
      As[e & 15][e >> 4] = xa[u];
      Bs[e >> 7][e & 127] = xb[u];
    }
    __syncthreads();
    if (l0 + kUgK < p) load(l0 + kUgK);  // in flight during the products below
#pragma unroll
    for (int l = 0; l < kUgK; ++l) {
      const float4 a0 = *reinterpret_cast<const float4 *>(&As[l][4 * ty]);
      const float4 a1 = *reinterpret_cast<const float4 *>(&As[l][64 + 4 * ty]);
      const float4 b0 = *reinterpret_cast<const float4 *>(&Bs[l][4 * tx]);
      const float4 b1 = *reinterpret_cast<const float4 *>(&Bs[l][64 + 4 * tx]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int64_t r = row0 + (i < 4 ? 4 * ty + i : 64 + 4 * ty + i - 4);
    if (r >= N) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int c = col0 + (j < 4 ? 4 * tx + j : 64 + 4 * tx + j - 4);
      if (c < K) U[r * K + c] = acc[i][j];
    }
  }
}

cudaError_t launch_ux(const Shape &s, const PassIO &io, cudaStream_t st) {
  const int ldb = ux_ldb(s.K);
  ux_coef_kernel<<<(unsigned)std::min((s.p * ldb + 255) / 256, 1024), 256, 0, st>>>(s.p, s.K, ldb, io.theta, io.delta,
                                                                                   io.tscale, io.bf);
  const dim3 grid((unsigned)((s.N + kUgM - 1) / kUgM), (unsigned)((s.K + kUgN - 1) / kUgN));
  ux_gemm_kernel<<<grid, 256, 0, st>>>(s.N, s.p, s.K, ldb, io.X, io.bf, io.ux);
  return cudaGetLastError();
}

int round_up_int(int v, int m) { return (v + m - 1) / m * m; }

bool make_tile_dims(const Shape &s, bool full, int rpw, TileDims &D, size_t &smem, bool ux = false) {
  if (s.K < 2 || s.K > 256) return false;
  const int cs = (s.K + 31) / 32;
  D.N = s.N; D.K = s.K; D.p = s.p; D.d = s.d; D.f = s.f;
  D.Kpad = 32 * (cs <= 1 ? 1 : cs <= 2 ? 2 : cs <= 4 ? 4 : 8);
  D.R = 8 * rpw;
  D.R4 = D.R + 4;
  D.pp = round_up_int(std::max(s.p, 1), 4);
  D.xq = 4 * D.R4 + 4;
  D.nb = (int)s.nb; D.mc = (int)s.mc; D.n = (int)s.n;
  D.ntiles = (s.N + D.R - 1) / D.R;
  int o = 0;
  D.ux = ux ? 1 : 0;
  D.off_x = o; o += round_up_int(D.R * (ux ? s.K : s.p) * 4, 128);
  D.off_y = o; o += round_up_int(D.R * s.K * s.d * 4, 128);
  D.off_z = o; o += round_up_int(D.R * s.K * s.f * 4, 128);
  D.off_c = o; o += round_up_int(D.R * 4, 128);
  D.stage_bytes = o;
  o = 0;
  D.off_bt = o; o += ux ? 0 : round_up_int(s.p * D.Kpad * 4, 128);
  D.off_gt = o; o += round_up_int(s.d * D.Kpad * 4, 128);
  D.off_al = o; o += round_up_int(std::max(s.f, 1) * 4, 128);
  D.off_xt = o; o += ux ? 0 : round_up_int(D.pp / 4 * D.xq * 4, 128);
  D.off_rt = o; o += full ? round_up_int((D.Kpad + 1) * D.R4 * 4, 128) : 0;
  D.off_red = o; o += round_up_int(std::max(2 * kPT / 32, s.K * s.f) * 8, 128);
  D.off_bar = o; o += 128;
  D.off_stage = o;
  // beta-gradient items and gamma/alpha entries
  D.kp2 = (s.K - 1 + 1) / 2;
  D.lq = (s.p + 3) / 4;
  D.wk = (D.kp2 + 3) / 4;
  D.wl = (D.lq + 7) / 8;
  D.nyz = (s.K - 1) * s.d + s.K * s.f;
  D.beta_ext = full && (ux || D.wk * D.wl > 8 * kBetaItems);
  if (D.beta_ext && (s.p > 16 * kGbMaxJ || s.K > 16 * kGbMaxK)) return false;
  if (full && D.nyz > kPT * 4) return false;
  // two CTAs per SM when a 2-stage ring fits in half of the shared memory, else one
  for (size_t budget : {(size_t)110 * 1024, (size_t)224 * 1024})
    for (int S = 3; S >= 2; --S) {
      const size_t b = (size_t)o + (size_t)S * D.stage_bytes;
      if (b <= budget) { D.S = S; smem = b; return true; }
    }
  return false;
}

template <int RPW, int CS, bool FULL, int YZS>
cudaError_t launch_t(const TileDims &D, int grid, size_t smem, const PassIO &io, cudaStream_t st) {
  auto kern = pass_tile_kernel<RPW, CS, FULL, YZS>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, kPT, smem, st>>>(D, io);
  return cudaGetLastError();
}

template <int RPW, bool FULL>
cudaError_t launch_cs(const TileDims &D, int grid, size_t smem, const PassIO &io, cudaStream_t st) {
  const bool wide = FULL && D.nyz > kPT * 2;
  switch (D.Kpad / 32) {
    case 1: return wide ? launch_t<RPW, 1, FULL, 4>(D, grid, smem, io, st) : launch_t<RPW, 1, FULL, 2>(D, grid, smem, io, st);
    case 2: return wide ? launch_t<RPW, 2, FULL, 4>(D, grid, smem, io, st) : launch_t<RPW, 2, FULL, 2>(D, grid, smem, io, st);
    case 4: return wide ? launch_t<RPW, 4, FULL, 4>(D, grid, smem, io, st) : launch_t<RPW, 4, FULL, 2>(D, grid, smem, io, st);
    case 8: return wide ? launch_t<RPW, 8, FULL, 4>(D, grid, smem, io, st) : launch_t<RPW, 8, FULL, 2>(D, grid, smem, io, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

bool plan_pass_beta_ext(const Shape &s) {
  TileDims D{};
  size_t smem = 0;
  return make_tile_dims(s, true, 2, D, smem) && D.beta_ext;
}

bool plan_pass_tiled(const Shape &s, bool full, int num_sms, PassPlan &pl) {
  TileDims D{};
  size_t smem = 0;
  // Wide shapes (the full pass's beta gradient does not fit its register
  // tiles): the X-block utilities from the separate GEMM, in both passes.
  const bool ux = plan_pass_beta_ext(s);
  // the log-likelihood-only pass of a wide shape: 8-row tiles, whose ring fits two CTAs per SM
  const int rpw_first = ux && !full ? 1 : 2;
  for (int rpw = rpw_first; rpw <= 2; ++rpw) {
    if (!make_tile_dims(s, full, rpw, D, smem, ux)) continue;
    pl.tiled = true;
    pl.ux = ux;
    pl.rows = D.R;
    pl.block = kPT;
    pl.npt = 0;
    pl.smem = smem;
    pl.grid = (int)std::min<int64_t>(D.ntiles, (int64_t)num_sms * (smem <= 110 * 1024 ? 2 : 1));
    if (pl.grid < 1) pl.grid = 1;
    pl.ok = true;
    return true;
  }
  return false;
}

cudaError_t launch_pass_tiled(const Shape &s, const PassPlan &pl, bool full, const PassIO &io, cudaStream_t st) {
  TileDims D{};
  size_t smem = 0;
  if (!make_tile_dims(s, full, pl.rows / 8, D, smem, pl.ux) || smem != pl.smem || io.err == nullptr)
    return cudaErrorInvalidValue;
  if (pl.ux && (!io.ux || !io.bf || (reinterpret_cast<uintptr_t>(io.ux) & 15))) return cudaErrorInvalidValue;
  const bool aligned = ((reinterpret_cast<uintptr_t>(io.X) | reinterpret_cast<uintptr_t>(io.choice) |
                         reinterpret_cast<uintptr_t>(io.w) |
                         (s.d ? reinterpret_cast<uintptr_t>(io.Y) : 0) | (s.f ? reinterpret_cast<uintptr_t>(io.Z) : 0)) &
                        15) == 0;
  if (!aligned) return cudaErrorInvalidValue;
  if (pl.rows != 16 && !(pl.rows == 8 && pl.ux && !full)) return cudaErrorInvalidValue;
  if (pl.ux) {
    cudaError_t e = launch_ux(s, io, st);
    if (e != cudaSuccess) return e;
  }
  if (!full) return pl.rows == 8 ? launch_cs<1, false>(D, pl.grid, smem, io, st) : launch_cs<2, false>(D, pl.grid, smem, io, st);
  if (io.Pin && D.beta_ext && !io.Wout) return cudaErrorInvalidValue;
  cudaError_t e = launch_cs<2, true>(D, pl.grid, smem, io, st);
  if (e == cudaSuccess && D.beta_ext) e = launch_grad_beta(s, pl.grid, io, st);
  return e;
}

}  // namespace mnl
