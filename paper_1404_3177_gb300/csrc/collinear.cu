// Collinearity check of the data blocks (Sec. 2.3 `linDepTol`; App. B, the
// necessary conditions for a non-singular Hessian) and the masks that hold the
// coefficients of dropped columns at zero.
//
// The paper asks for X and every Y_k to have full column rank, and for the
// generic variables' normalized columns (the stacked Z_ik - Z_i0, k >= 1) to
// be linearly independent; the package tests this by a rank-revealing QR with
// tolerance linDepTol and drops the columns of a collinear set one by one.
// Column j of a block is dropped when the part of it orthogonal to the kept
// earlier columns has a norm of at most tol * ||column j||.  In terms of the
// Gram matrix G = M^T M that residual norm squared is the pivot of an in-order
// Cholesky factorisation of G restricted to the kept columns, so the check is:
//   1. every Gram matrix in float64 from one pass over the data (products of
//      float32 values are exact in float64; sums in a fixed order);
//   2. per block, an in-order (left-looking) Cholesky that drops column j when
//      its pivot is at most tol^2 G_jj (or G_jj = 0); a dropped column keeps a
//      zero column in the factor, so it leaves the span of the later ones.
#include <algorithm>
#include <cmath>
#include <vector>

#include "mnl_internal.cuh"

namespace mnl {
namespace {

constexpr int kGramThreads = 256;

// Rows of a block: row r is sub-row j = r % nk of observation i = r / nk, its
// column c at src[i * row_stride + (k0 + j) * sub_stride + c], minus the
// observation's sub-row 0 (src[i * row_stride + c]) when diff.
struct GramGroup {
  const float *src;
  int64_t rows, row_stride;
  int nk, k0, sub_stride, diff;
  int cols, nblk;  // nblk = ceil(cols / B)
  int64_t g_off;   // cols x cols Gram (column-major) in G
  int flag_off;    // first flag of this block
};

// One CTA: block pair (a >= b) of group g over rows [r0, r1); B x B partial at part + out.
struct GramJob {
  int g, a, b, pad;
  int64_t r0, r1, out;
};

// Fixed-order sum of the jobs [j0, j0 + nj) of one block pair into G.
struct GramSlot {
  int g, a, b, nj;
  int64_t j0;
};

template <int B>
__device__ __forceinline__ void load_block(const GramGroup &g, int64_t r, int blk, double (&v)[B]) {
  const int64_t i = r / g.nk;
  const int j = (int)(r - i * g.nk);
  const float *row = g.src + i * g.row_stride + (int64_t)(g.k0 + j) * g.sub_stride;
  const float *row0 = g.src + i * g.row_stride;
#pragma unroll
  for (int u = 0; u < B; ++u) {
    const int c = blk * B + u;
    double x = 0.0;
    if (c < g.cols) {
      x = (double)row[c];
      if (g.diff) x -= (double)row0[c];
    }
    v[u] = x;
  }
}

// Partial Gram block of one job: each thread sums its rows (stride blockDim)
// into a B x B register tile; the tiles are added warp by warp (shuffles, a
// fixed tree) and then over the warps in order.
template <int B>
__global__ void __launch_bounds__(kGramThreads) gram_partial_kernel(const GramGroup *__restrict__ groups,
                                                                   const GramJob *__restrict__ jobs,
                                                                   double *__restrict__ part) {
  __shared__ double red[kGramThreads / 32][B * B];
  const GramJob jb = jobs[blockIdx.x];
  const GramGroup g = groups[jb.g];
  double acc[B][B];
#pragma unroll
  for (int u = 0; u < B; ++u)
#pragma unroll
    for (int v = 0; v < B; ++v) acc[u][v] = 0.0;
  for (int64_t r = jb.r0 + threadIdx.x; r < jb.r1; r += kGramThreads) {
    double va[B], vb[B];
    load_block<B>(g, r, jb.a, va);
    if (jb.a == jb.b) {
#pragma unroll
      for (int u = 0; u < B; ++u) vb[u] = va[u];
    } else {
      load_block<B>(g, r, jb.b, vb);
    }
#pragma unroll
    for (int u = 0; u < B; ++u)
#pragma unroll
      for (int v = 0; v < B; ++v) acc[u][v] = fma(va[u], vb[v], acc[u][v]);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int u = 0; u < B; ++u)
#pragma unroll
    for (int v = 0; v < B; ++v) {
      double s = acc[u][v];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) red[warp][u * B + v] = s;
    }
  __syncthreads();
  if (threadIdx.x < B * B) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < kGramThreads / 32; ++w) s += red[w][threadIdx.x];
    part[jb.out + threadIdx.x] = s;
  }
}

// G entries of every slot: thread per (slot, entry u * B + v); writes (a B + u,
// b B + v) and its mirror.
__global__ void gram_reduce_kernel(const GramGroup *__restrict__ groups, const GramSlot *__restrict__ slots,
                                   int nslots, int B, const double *__restrict__ part, double *__restrict__ G) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int bb = B * B;
  if (t >= (int64_t)nslots * bb) return;
  const GramSlot s = slots[t / bb];
  const int e = (int)(t % bb), u = e / B, v = e % B;
  const GramGroup g = groups[s.g];
  const int r = s.a * B + u, c = s.b * B + v;
  if (r >= g.cols || c >= g.cols) return;
  double sum = 0.0;
  for (int j = 0; j < s.nj; ++j) sum += part[(s.j0 + j) * bb + e];
  double *Gg = G + g.g_off;
  Gg[(int64_t)c * g.cols + r] = sum;
  Gg[(int64_t)r * g.cols + c] = sum;
}

// In-order Cholesky of one group's Gram matrix with dropping (left-looking:
// column j is formed from the original G(:, j) and the finished columns
// k < j of the factor, which replace G's lower triangle).  flags[j] = 1 for a
// dropped column, whose factor column is set to zero.
__global__ void __launch_bounds__(256) drop_chol_kernel(const GramGroup *__restrict__ groups, double *__restrict__ G,
                                                       double tol2, int32_t *__restrict__ flags) {
  const GramGroup g = groups[blockIdx.x];
  const int c = g.cols;
  double *A = G + g.g_off;
  __shared__ double orig, piv;
  __shared__ int drop;
  for (int j = 0; j < c; ++j) {
    if (threadIdx.x == 0) orig = A[(int64_t)j * c + j];
    __syncthreads();
    for (int i = j + threadIdx.x; i < c; i += blockDim.x) {
      double s = A[(int64_t)j * c + i];
      for (int k = 0; k < j; ++k) s = fma(-A[(int64_t)k * c + i], A[(int64_t)k * c + j], s);
      A[(int64_t)j * c + i] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      const double d = A[(int64_t)j * c + j];
      drop = (orig > 0.0 && d > tol2 * orig) ? 0 : 1;
      piv = drop ? 0.0 : sqrt(d);
      flags[g.flag_off + j] = drop;
    }
    __syncthreads();
    for (int i = j + threadIdx.x; i < c; i += blockDim.x)
      A[(int64_t)j * c + i] = drop ? 0.0 : A[(int64_t)j * c + i] / piv;
    __syncthreads();
  }
}

__global__ void mask_vec_kernel(int m, const int64_t *__restrict__ idx, double *__restrict__ v, double val) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < m) v[idx[t]] = val;
}

// Rows and columns idx[0 .. m) of F (both triangles) and of the lower
// triangle of F32 (when given) become those of the identity.
__global__ void mask_matrix_kernel(int64_t n, int m, const int64_t *__restrict__ idx, double *__restrict__ F,
                                   float *__restrict__ F32) {
  for (int t = blockIdx.y; t < m; t += gridDim.y) {
    const int64_t j = idx[t];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
      const double e = i == j ? 1.0 : 0.0;
      F[j * n + i] = e;
      F[i * n + j] = e;
      if (F32) {
        if (i >= j) F32[j * n + i] = (float)e;
        if (i <= j) F32[i * n + j] = (float)e;
      }
    }
  }
}

template <typename T>
cudaError_t dmalloc(T **p, size_t bytes) {
  return cudaMalloc(reinterpret_cast<void **>(p), std::max<size_t>(bytes, 256));
}

}  // namespace

int collinear_flags_size(const mnl_dims &d) { return d.p + d.K * d.d + d.f; }

cudaError_t collinear_check(const mnl_dims &d, const float *X, const float *Y, const float *Z, double tol,
                            int nsm, cudaStream_t st, int32_t *flags_host, CollinearStats *stats) {
  const int nflags = collinear_flags_size(d);
  std::vector<GramGroup> groups;
  auto add = [&](const float *src, int64_t rows, int64_t rs, int nk, int k0, int ss, int diff, int cols,
                 int flag_off) {
    if (cols <= 0 || rows <= 0) return;
    GramGroup g{};
    g.src = src; g.rows = rows; g.row_stride = rs; g.nk = nk; g.k0 = k0; g.sub_stride = ss; g.diff = diff;
    g.cols = cols; g.flag_off = flag_off;
    groups.push_back(g);
  };
  add(X, d.N, d.p, 1, 0, 0, 0, d.p, 0);
  if (d.d > 0)
    for (int k = d.gamma_base ? 0 : 1; k < d.K; ++k) add(Y, d.N, (int64_t)d.K * d.d, 1, k, d.d, 0, d.d, d.p + k * d.d);
  if (d.f > 0 && d.K > 1) add(Z, d.N * (int64_t)(d.K - 1), (int64_t)d.K * d.f, d.K - 1, 1, d.f, 1, d.f, d.p + d.K * d.d);
  std::vector<int32_t> flags(nflags, 0);
  if (groups.empty()) {
    std::copy(flags.begin(), flags.end(), flags_host);
    if (stats) *stats = CollinearStats{};
    return cudaSuccess;
  }
  // Register tile edge B: the least work over the groups (rows x block pairs x B^2).
  int B = 8;
  double best = 1e300;
  for (int b = 4; b <= 8; ++b) {
    double w = 0.0;
    for (const GramGroup &g : groups) {
      const double nb = (g.cols + b - 1) / b;
      w += (double)g.rows * nb * (nb + 1) / 2 * b * b;
    }
    if (w < best) { best = w; B = b; }
  }
  int64_t goff = 0;
  double total = 0.0;
  for (GramGroup &g : groups) {
    g.nblk = (g.cols + B - 1) / B;
    g.g_off = goff;
    goff += (int64_t)g.cols * g.cols;
    total += (double)g.rows * g.nblk * (g.nblk + 1) / 2;
  }
  // Row chunks: about 8 jobs per SM in all, at least 2048 rows per job.
  const double per_job = std::max(2048.0, total / (8.0 * std::max(nsm, 1)));
  std::vector<GramJob> jobs;
  std::vector<GramSlot> slots;
  for (int gi = 0; gi < (int)groups.size(); ++gi) {
    const GramGroup &g = groups[gi];
    const int64_t chunk = std::max<int64_t>(2048, (int64_t)std::ceil(per_job));
    const int64_t nch = (g.rows + chunk - 1) / chunk;
    for (int a = 0; a < g.nblk; ++a)
      for (int b = 0; b <= a; ++b) {
        GramSlot s{gi, a, b, (int)nch, (int64_t)jobs.size()};
        slots.push_back(s);
        for (int64_t c = 0; c < nch; ++c) {
          GramJob j{};
          j.g = gi; j.a = a; j.b = b;
          j.r0 = c * chunk;
          j.r1 = std::min(g.rows, (c + 1) * chunk);
          j.out = (int64_t)jobs.size() * B * B;
          jobs.push_back(j);
        }
      }
  }
  GramGroup *d_groups = nullptr;
  GramJob *d_jobs = nullptr;
  GramSlot *d_slots = nullptr;
  double *d_part = nullptr, *d_G = nullptr;
  int32_t *d_flags = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaSuccess;
  auto cleanup = [&]() {
    cudaFree(d_groups); cudaFree(d_jobs); cudaFree(d_slots); cudaFree(d_part); cudaFree(d_G); cudaFree(d_flags);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  };
#define CC(x)                                  \
  do {                                         \
    if ((e = (x)) != cudaSuccess) {            \
      cleanup();                               \
      return e;                                \
    }                                          \
  } while (0)
  CC(dmalloc(&d_groups, groups.size() * sizeof(GramGroup)));
  CC(dmalloc(&d_jobs, jobs.size() * sizeof(GramJob)));
  CC(dmalloc(&d_slots, slots.size() * sizeof(GramSlot)));
  CC(dmalloc(&d_part, jobs.size() * (size_t)B * B * sizeof(double)));
  CC(dmalloc(&d_G, (size_t)goff * sizeof(double)));
  CC(dmalloc(&d_flags, (size_t)nflags * sizeof(int32_t)));
  CC(cudaEventCreate(&e0));
  CC(cudaEventCreate(&e1));
  CC(cudaMemcpyAsync(d_groups, groups.data(), groups.size() * sizeof(GramGroup), cudaMemcpyHostToDevice, st));
  CC(cudaMemcpyAsync(d_jobs, jobs.data(), jobs.size() * sizeof(GramJob), cudaMemcpyHostToDevice, st));
  CC(cudaMemcpyAsync(d_slots, slots.data(), slots.size() * sizeof(GramSlot), cudaMemcpyHostToDevice, st));
  CC(cudaMemsetAsync(d_flags, 0, (size_t)nflags * sizeof(int32_t), st));
  CC(cudaEventRecord(e0, st));
  const unsigned nj = (unsigned)jobs.size();
  switch (B) {
    case 4: gram_partial_kernel<4><<<nj, kGramThreads, 0, st>>>(d_groups, d_jobs, d_part); break;
    case 5: gram_partial_kernel<5><<<nj, kGramThreads, 0, st>>>(d_groups, d_jobs, d_part); break;
    case 6: gram_partial_kernel<6><<<nj, kGramThreads, 0, st>>>(d_groups, d_jobs, d_part); break;
    case 7: gram_partial_kernel<7><<<nj, kGramThreads, 0, st>>>(d_groups, d_jobs, d_part); break;
    default: gram_partial_kernel<8><<<nj, kGramThreads, 0, st>>>(d_groups, d_jobs, d_part); break;
  }
  CC(cudaGetLastError());
  const int64_t nt = (int64_t)slots.size() * B * B;
  gram_reduce_kernel<<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(d_groups, d_slots, (int)slots.size(), B, d_part,
                                                                    d_G);
  CC(cudaGetLastError());
  drop_chol_kernel<<<(unsigned)groups.size(), 256, 0, st>>>(d_groups, d_G, tol * tol, d_flags);
  CC(cudaGetLastError());
  CC(cudaEventRecord(e1, st));
  CC(cudaMemcpyAsync(flags.data(), d_flags, (size_t)nflags * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  CC(cudaStreamSynchronize(st));
  if (stats) {
    float ms = 0.f;
    CC(cudaEventElapsedTime(&ms, e0, e1));
    stats->ms = ms;
    stats->groups = (int)groups.size();
    stats->jobs = (int)jobs.size();
    stats->tile = B;
    stats->gram_fma = 0.0;
    for (const GramGroup &g : groups) stats->gram_fma += (double)g.rows * g.cols * (g.cols + 1) / 2;
    stats->bytes = 0.0;
    for (const GramGroup &g : groups) stats->bytes += (double)g.rows * g.cols * 4.0;
  }
#undef CC
  cleanup();
  std::copy(flags.begin(), flags.end(), flags_host);
  return cudaSuccess;
}

cudaError_t launch_mask_vec(int m, const int64_t *idx, double *v, double val, cudaStream_t st) {
  if (m <= 0) return cudaSuccess;
  mask_vec_kernel<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(m, idx, v, val);
  return cudaGetLastError();
}

cudaError_t launch_mask_matrix(int64_t n, int m, const int64_t *idx, double *F, float *F32, cudaStream_t st) {
  if (m <= 0) return cudaSuccess;
  const unsigned gx = (unsigned)std::min<int64_t>((n + 255) / 256, 64);
  mask_matrix_kernel<<<dim3(gx, (unsigned)std::min(m, 65535)), 256, 0, st>>>(n, m, idx, F, F32);
  return cudaGetLastError();
}

}  // namespace mnl
