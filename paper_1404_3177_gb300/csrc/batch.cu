// Batched fits: many independent multinomial-logit problems of uneven size,
// each Newton-Raphson phase one grouped launch over all problems still
// iterating (Sec. 3.1 eq. "NR update" with step halving, applied per problem).
//
// One iteration = grouped pass (l, g, P, zbar) -> per-problem reduction and
// gradient test -> operand build -> tensor-core (or FP64) contractions of the
// class blocks -> Z blocks -> assembly of -H -> one CTA per problem for the
// Cholesky solve -> line search (grouped log-likelihood pass at theta + t delta,
// per-problem accept / halve) -> coefficient update and step test.
// The launch sequence of one iteration is captured once as a CUDA graph and
// replayed; problems that converged (or failed) are skipped by every kernel
// through the device-side `active` flags, so the graph never changes.
//
// Autotuning: the row-tile height of the grouped pass is chosen among a few
// candidates by timing the log-likelihood pass over the whole batch when the
// batch is created; the choice is cached per distinct batch shape summary in
// the process, and in the file named by MNL_TUNE_CACHE when that is set.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "mnl_internal.cuh"

using namespace mnl;

namespace {

__global__ void gtol_check_kernel(int nprob, const GroupProblem *__restrict__ probs, int *__restrict__ active,
                                  int *__restrict__ status, int *__restrict__ stop, double gtol) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nprob || active[b] == 0) return;
  double *sc = probs[b].scal;
  const double l = sc[kGsL], ginf = sc[kGsGinf];
  if (!isfinite(l) || !isfinite(ginf)) { status[b] = MNL_ERR_NONFINITE; active[b] = 0; return; }
  sc[kGsLold] = l;
  if (gtol > 0 && ginf < gtol) { stop[b] = MNL_STOP_GTOL; active[b] = 0; }
}

// After the solve: problems with an error leave; the rest start a line search at t = 1.
__global__ void ls_init_kernel(int nprob, const GroupProblem *__restrict__ probs, int *__restrict__ active,
                               int *__restrict__ pending, const int *__restrict__ status) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nprob) return;
  pending[b] = 0;
  if (active[b] == 0) return;
  if (status[b] != MNL_OK) { active[b] = 0; return; }
  probs[b].scal[kGsT] = 1.0;
  pending[b] = 1;
}

// One line-search round: accept when l(theta + t delta) >= l(theta) - tau, else halve t.
__global__ void ls_update_kernel(int nprob, const GroupProblem *__restrict__ probs, int *__restrict__ pending,
                                 int *__restrict__ accepted, int *__restrict__ active, int *__restrict__ status,
                                 double u_round, int max_halvings) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nprob || pending[b] == 0) return;
  double *sc = probs[b].scal;
  sc[kGsLsEvals] += 1.0;
  const double lt = sc[kGsLt], l0 = sc[kGsLold], tau = 8.0 * u_round * sc[kGsLabs];
  if (isfinite(lt) && lt >= l0 - tau) {
    pending[b] = 0;
    accepted[b] = 1;
    return;
  }
  const double t = sc[kGsT] * 0.5;
  if (t < ldexp(1.0, -max_halvings)) {
    pending[b] = 0;
    active[b] = 0;
    status[b] = MNL_ERR_LINESEARCH;
    return;
  }
  sc[kGsT] = t;
}

// theta += t delta for accepted problems, step test, iteration count.
__global__ void __launch_bounds__(256) theta_update_kernel(const GroupProblem *__restrict__ probs,
                                                           int *__restrict__ accepted, int *__restrict__ active,
                                                           int *__restrict__ stop, double steptol, double ftol) {
  __shared__ double red[2][8];
  const int b = blockIdx.x;
  if (accepted[b] == 0) return;
  const GroupProblem &g = probs[b];
  double *sc = g.scal;
  const double t = sc[kGsT];
  double m1 = 0.0, m2 = 0.0;
  for (int64_t i = threadIdx.x; i < g.n; i += blockDim.x) {
    const double s = t * g.delta[i];
    const double th = g.theta[i] + s;
    g.theta[i] = th;
    m1 = fmax(m1, fabs(s));
    m2 = fmax(m2, fabs(th));
  }
  for (int o = 16; o > 0; o >>= 1) {
    m1 = fmax(m1, __shfl_xor_sync(0xffffffffu, m1, o));
    m2 = fmax(m2, __shfl_xor_sync(0xffffffffu, m2, o));
  }
  if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = m1; red[1][threadIdx.x >> 5] = m2; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, c = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { a = fmax(a, red[0][w]); c = fmax(c, red[1][w]); }
    sc[kGsStepInf] = a;
    sc[kGsThetaInf] = c;
    sc[kGsIters] += 1.0;
    const double dl = sc[kGsLt] - sc[kGsLold];
    sc[kGsL] = sc[kGsLt];
    accepted[b] = 0;
    if (ftol > 0 && fabs(dl) < ftol) { stop[b] = MNL_STOP_FTOL; active[b] = 0; }
    else if (steptol > 0 && a <= steptol * fmax(1.0, c)) { stop[b] = MNL_STOP_STEPTOL; active[b] = 0; }
  }
}

__global__ void count_kernel(int nprob, const int *__restrict__ a, const int *__restrict__ b, int *__restrict__ out) {
  __shared__ int sa, sb;
  if (threadIdx.x == 0) { sa = 0; sb = 0; }
  __syncthreads();
  int ca = 0, cb = 0;
  for (int i = threadIdx.x; i < nprob; i += blockDim.x) { ca += a[i] != 0; cb += b[i] != 0; }
  atomicAdd(&sa, ca);
  atomicAdd(&sb, cb);
  __syncthreads();
  if (threadIdx.x == 0) { out[0] = sa; out[1] = sb; }
}

int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

// Cached autotuning choices: key -> rows per pass tile.
std::mutex g_tune_mutex;
std::map<std::string, int> g_tune;
bool g_tune_loaded = false;

void tune_load() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char *path = std::getenv("MNL_TUNE_CACHE");
  if (!path) return;
  FILE *fh = std::fopen(path, "r");
  if (!fh) return;
  char key[512];
  int v;
  while (std::fscanf(fh, "%511s %d", key, &v) == 2) g_tune[key] = v;
  std::fclose(fh);
}

void tune_store(const std::string &key, int v) {
  g_tune[key] = v;
  const char *path = std::getenv("MNL_TUNE_CACHE");
  if (!path) return;
  FILE *fh = std::fopen(path, "a");
  if (!fh) return;
  std::fprintf(fh, "%s %d\n", key.c_str(), v);
  std::fclose(fh);
}

}  // namespace

struct mnl_batch {
  int count, prec;
  OpType op;
  bool fp64, mixed;
  cudaStream_t user_st, st;
  cudaEvent_t ev_user, ev_done, t0, t1;
  int dev, nsm;
  std::vector<Shape> shapes;
  std::vector<GroupProblem> hp;   // host copy of the descriptors
  std::vector<int64_t> theta_off;
  int64_t theta_total;
  GroupProblem *probs;
  int *active, *pending, *accepted, *status, *stop, *counts, *h_counts;
  int *err;
  // grouped pass
  GroupedPassPlan pfull, pll;
  PassSeg *segs;
  int *seg_start, *slot_start, *slot_segs;
  double *partials;
  // contractions
  GroupItem *build_items, *z_items, *asm_items;
  int n_build, n_z, n_asm;
  size_t build_smem, z_smem, chol_smem;
  CUtensorMap *maps;
  SyrkUnit *units_main, *units_band;
  int nunits_main, nunits_band;
  void *main_part, *band_part, *z_part;
  int64_t nmax;
  // graph of one iteration (without the extra line-search rounds)
  cudaGraphExec_t graph;
  bool have_graph;
  double graph_gtol;      // options baked into the captured graph
  int graph_halvings;
  std::vector<void *> allocs;
};

namespace {

#define BCK(x)                                           \
  do {                                                   \
    cudaError_t e_ = (x);                                \
    if (e_ != cudaSuccess) { cudaGetLastError(); return e_ == cudaErrorMemoryAllocation ? MNL_ERR_OOM : MNL_ERR_CUDA; } \
  } while (0)

template <typename T>
int balloc(mnl_batch *b, T **p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) return MNL_OK;
  void *q = nullptr;
  cudaError_t e = cudaMalloc(&q, bytes);
  if (e != cudaSuccess) { cudaGetLastError(); return e == cudaErrorMemoryAllocation ? MNL_ERR_OOM : MNL_ERR_CUDA; }
  b->allocs.push_back(q);
  *p = reinterpret_cast<T *>(q);
  return MNL_OK;
}

void bfree(mnl_batch *b) {
  if (b->have_graph) cudaGraphExecDestroy(b->graph);
  for (void *p : b->allocs) cudaFree(p);
  b->allocs.clear();
  if (b->h_counts) cudaFreeHost(b->h_counts);
  if (b->st) cudaStreamDestroy(b->st);
  for (cudaEvent_t e : {b->ev_user, b->ev_done, b->t0, b->t1})
    if (e) cudaEventDestroy(e);
}

// Pass segments: the tiles of all problems in order, cut into one contiguous
// range per CTA of about equal cost, then at problem boundaries.
int build_pass_lists(mnl_batch *b, int rows, int grid, std::vector<PassSeg> &segs, std::vector<int> &seg_start,
                     std::vector<int> &slot_start, std::vector<int> &slot_segs, int64_t *partial_len) {
  struct TileRun { int problem; int64_t ntiles; double cost; };
  std::vector<TileRun> runs;
  double total = 0.0;
  for (int i = 0; i < b->count; ++i) {
    const Shape &s = b->shapes[i];
    const int64_t nt = (s.N + rows - 1) / rows;
    const double c = (double)rows * s.K * (s.p + s.d + s.f + 1) + (double)s.nout;
    runs.push_back({i, nt, c});
    total += c * nt;
  }
  segs.clear();
  seg_start.assign(grid + 1, 0);
  std::vector<std::vector<int>> per_prob(b->count);
  int64_t off_full = 0, off_ll = 0;
  double acc = 0.0;
  size_t ri = 0;
  int64_t ti = 0;  // next tile within runs[ri]
  for (int c = 0; c < grid; ++c) {
    seg_start[c] = (int)segs.size();
    const double target = total * (c + 1) / grid;
    while (ri < runs.size() && (acc < target - 1e-9 || c == grid - 1)) {
      const TileRun &r = runs[ri];
      // tiles of this run that fit below the target
      int64_t take = r.ntiles - ti;
      if (c < grid - 1) {
        const int64_t fit = (int64_t)std::ceil((target - acc) / r.cost - 1e-9);
        take = std::max<int64_t>(1, std::min(take, fit));
      }
      PassSeg sg;
      sg.problem = r.problem;
      sg.tile0 = ti;
      sg.tile1 = ti + take;
      sg.slot_full = off_full;
      sg.slot_ll = off_ll;
      off_full += 2 + b->shapes[r.problem].n;
      off_ll += 2;
      per_prob[r.problem].push_back((int)segs.size());
      segs.push_back(sg);
      acc += take * r.cost;
      ti += take;
      if (ti >= r.ntiles) { ++ri; ti = 0; }
      if (c < grid - 1 && acc >= target - 1e-9) break;
    }
  }
  seg_start[grid] = (int)segs.size();
  slot_start.assign(b->count + 1, 0);
  slot_segs.clear();
  for (int i = 0; i < b->count; ++i) {
    slot_start[i] = (int)slot_segs.size();
    for (int s : per_prob[i]) slot_segs.push_back(s);
  }
  slot_start[b->count] = (int)slot_segs.size();
  *partial_len = std::max(off_full, off_ll);
  return MNL_OK;
}

int upload_pass_lists(mnl_batch *b, const std::vector<PassSeg> &segs, const std::vector<int> &seg_start,
                      const std::vector<int> &slot_start, const std::vector<int> &slot_segs, int64_t plen) {
  int rc;
  if ((rc = balloc(b, &b->segs, segs.size() * sizeof(PassSeg))) ||
      (rc = balloc(b, &b->seg_start, seg_start.size() * sizeof(int))) ||
      (rc = balloc(b, &b->slot_start, slot_start.size() * sizeof(int))) ||
      (rc = balloc(b, &b->slot_segs, slot_segs.size() * sizeof(int))) ||
      (rc = balloc(b, &b->partials, (size_t)plen * sizeof(double))))
    return rc;
  BCK(cudaMemcpy(b->segs, segs.data(), segs.size() * sizeof(PassSeg), cudaMemcpyHostToDevice));
  BCK(cudaMemcpy(b->seg_start, seg_start.data(), seg_start.size() * sizeof(int), cudaMemcpyHostToDevice));
  BCK(cudaMemcpy(b->slot_start, slot_start.data(), slot_start.size() * sizeof(int), cudaMemcpyHostToDevice));
  if (!slot_segs.empty())
    BCK(cudaMemcpy(b->slot_segs, slot_segs.data(), slot_segs.size() * sizeof(int), cudaMemcpyHostToDevice));
  return MNL_OK;
}

// Grouped log-likelihood pass over all problems at theta (delta ignored: t = 0
// is not used; the pass reads theta + t delta, so set t = 0 first) - used to
// time tile heights.
int autotune_rows(mnl_batch *b, int *rows_out) {
  std::string key = std::string(b->fp64 ? "f64" : "f32") + ":";
  {
    int64_t sN = 0, sK = 0, sq = 0;
    for (const Shape &s : b->shapes) { sN += s.N; sK += s.K; sq += s.p + s.d + s.f; }
    key += std::to_string(b->count) + "," + std::to_string(sN) + "," + std::to_string(sK) + "," + std::to_string(sq);
  }
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    tune_load();
    auto it = g_tune.find(key);
    if (it != g_tune.end()) { *rows_out = it->second; return MNL_OK; }
  }
  static const int cands[] = {8, 16, 32};
  float best = 1e30f;
  int best_rows = 16;
  for (int rows : cands) {
    GroupedPassPlan pl = plan_grouped_pass(b->shapes, b->fp64, rows, b->nsm);
    if (!pl.ok) continue;
    std::vector<PassSeg> segs;
    std::vector<int> ss, sl, sls;
    int64_t plen = 0;
    build_pass_lists(b, rows, pl.grid, segs, ss, sl, sls, &plen);
    PassSeg *d_segs = nullptr;
    int *d_ss = nullptr;
    double *d_part = nullptr;
    if (cudaMalloc(&d_segs, segs.size() * sizeof(PassSeg)) != cudaSuccess ||
        cudaMalloc(&d_ss, ss.size() * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&d_part, (size_t)plen * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(d_segs); cudaFree(d_ss); cudaFree(d_part);
      continue;
    }
    cudaMemcpy(d_segs, segs.data(), segs.size() * sizeof(PassSeg), cudaMemcpyHostToDevice);
    cudaMemcpy(d_ss, ss.data(), ss.size() * sizeof(int), cudaMemcpyHostToDevice);
    float ms = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
      cudaEventRecord(b->t0, b->st);
      launch_grouped_pass(pl, b->fp64, false, b->probs, d_segs, d_ss, b->active, d_part, b->st);
      cudaEventRecord(b->t1, b->st);
      cudaEventSynchronize(b->t1);
      float m = 0.f;
      cudaEventElapsedTime(&m, b->t0, b->t1);
      if (rep > 0) ms = std::min(ms, m);
    }
    cudaFree(d_segs); cudaFree(d_ss); cudaFree(d_part);
    if (cudaGetLastError() != cudaSuccess) continue;
    if (ms < best) { best = ms; best_rows = rows; }
  }
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    tune_store(key, best_rows);
  }
  *rows_out = best_rows;
  return MNL_OK;
}

int enqueue_iteration(mnl_batch *b, const mnl_fit_opts &o) {
  const int np = b->count;
  const int tb = 256, nb = (np + tb - 1) / tb;
  BCK(launch_grouped_pass(b->pfull, b->fp64, true, b->probs, b->segs, b->seg_start, b->active, b->partials, b->st));
  BCK(launch_grouped_reduce(np, true, b->probs, b->slot_start, b->segs, b->slot_segs, b->active, b->partials, kGsL,
                            b->st));
  gtol_check_kernel<<<nb, tb, 0, b->st>>>(np, b->probs, b->active, b->status, b->stop, o.gtol);
  BCK(cudaGetLastError());
  BCK(launch_grouped_build(b->op, b->probs, b->build_items, b->n_build, b->active, b->build_smem, b->st));
  if (b->fp64) {
    BCK(launch_grouped_syrk_f64(b->probs, b->units_main, b->nunits_main, b->active,
                                reinterpret_cast<double *>(b->main_part), b->st));
    BCK(launch_grouped_syrk_f64(b->probs, b->units_band, b->nunits_band, b->active,
                                reinterpret_cast<double *>(b->band_part), b->st));
  } else {
    BCK(launch_syrk_tc(b->op, b->maps, b->units_main, b->nunits_main, b->active, b->nsm,
                       reinterpret_cast<float *>(b->main_part), b->err, b->st));
    BCK(launch_syrk_tc(b->op, b->maps, b->units_band, b->nunits_band, b->active, b->nsm,
                       reinterpret_cast<float *>(b->band_part), b->err, b->st));
  }
  BCK(launch_grouped_zblocks(b->fp64, b->probs, b->z_items, b->n_z, b->active, b->z_smem, b->z_part, b->st));
  BCK(launch_grouped_assemble(b->fp64, b->probs, b->asm_items, b->n_asm, b->active, b->main_part, b->band_part,
                              b->z_part, b->st));
  BCK(launch_grouped_chol_solve(b->mixed, b->probs, np, b->active, 5, b->status, b->chol_smem, b->st));
  ls_init_kernel<<<nb, tb, 0, b->st>>>(np, b->probs, b->active, b->pending, b->status);
  BCK(cudaGetLastError());
  return MNL_OK;
}

int enqueue_ls_round(mnl_batch *b, const mnl_fit_opts &o) {
  const int np = b->count;
  const int tb = 256, nb = (np + tb - 1) / tb;
  BCK(launch_grouped_pass(b->pll, b->fp64, false, b->probs, b->segs, b->seg_start, b->pending, b->partials, b->st));
  BCK(launch_grouped_reduce(np, false, b->probs, b->slot_start, b->segs, b->slot_segs, b->pending, b->partials, kGsLt,
                            b->st));
  const double u = b->fp64 ? std::ldexp(1.0, -53) : std::ldexp(1.0, -24);
  ls_update_kernel<<<nb, tb, 0, b->st>>>(np, b->probs, b->pending, b->accepted, b->active, b->status, u,
                                         o.max_halvings);
  BCK(cudaGetLastError());
  count_kernel<<<1, 256, 0, b->st>>>(np, b->active, b->pending, b->counts);
  BCK(cudaGetLastError());
  return MNL_OK;
}

}  // namespace

extern "C" {

int mnl_batch_create(int count, const mnl_dims *dims, const mnl_data *data, int precision, void *stream,
                     mnl_batch **out) {
  if (!out) return MNL_ERR_INVALID_ARG;
  *out = nullptr;
  if (count < 1 || !dims || !data || precision < MNL_FP64 || precision > MNL_BF16) return MNL_ERR_INVALID_ARG;
  for (int i = 0; i < count; ++i) {
    const mnl_dims &d = dims[i];
    if (d.N < 1 || d.K < 2 || d.p < 0 || d.d < 0 || d.f < 0 || d.p + d.d + d.f < 1) return MNL_ERR_INVALID_ARG;
    if (d.gamma_base != 0) return MNL_ERR_UNSUPPORTED;
    if (!data[i].choice || (d.p > 0 && !data[i].X) || (d.d > 0 && !data[i].Y) || (d.f > 0 && !data[i].Z))
      return MNL_ERR_INVALID_ARG;
  }
  mnl_batch *b = new (std::nothrow) mnl_batch();
  if (!b) return MNL_ERR_OOM;
  auto fail = [&](int rc) { bfree(b); delete b; return rc; };
  b->count = count;
  b->prec = precision;
  b->fp64 = precision == MNL_FP64;
  b->op = precision == MNL_FP64 ? OpType::F64 : precision == MNL_TF32 ? OpType::TF32 : OpType::BF16;
  b->mixed = !b->fp64;
  b->user_st = reinterpret_cast<cudaStream_t>(stream);
  if (cudaGetDevice(&b->dev) != cudaSuccess) { cudaGetLastError(); return fail(MNL_ERR_CUDA); }
  cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, b->dev);
  if (cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_user, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_done, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreate(&b->t0) != cudaSuccess || cudaEventCreate(&b->t1) != cudaSuccess ||
      cudaMallocHost(&b->h_counts, 4 * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return fail(MNL_ERR_CUDA);
  }
  int rc;
  const size_t tsz = b->fp64 ? 8 : 4;
  const size_t esz = b->fp64 ? 8 : b->op == OpType::TF32 ? 4 : 2;
  // shapes, offsets and the per-problem arena
  b->theta_total = 0;
  b->nmax = 0;
  size_t bytes = 0;
  struct Off { size_t P, zbar, At, Ad, F, F32, grad, delta, scal, rwork, band_of; };
  std::vector<Off> offs(count);
  std::vector<std::vector<int2>> bands(count);
  std::vector<std::vector<int>> band_maps(count);
  int64_t main_elems = 0, band_elems = 0, z_elems = 0;
  b->hp.resize(count);
  for (int i = 0; i < count; ++i) {
    const Shape s = make_shape(dims[i]);
    b->shapes.push_back(s);
    b->theta_off.push_back(b->theta_total);
    b->theta_total += s.n;
    b->nmax = std::max(b->nmax, s.n);
    GroupProblem &g = b->hp[i];
    std::memset(&g, 0, sizeof(g));
    g.N = s.N; g.K = s.K; g.p = s.p; g.d = s.d; g.f = s.f; g.n = s.n; g.mc = s.mc;
    g.X = data[i].X; g.Y = data[i].Y; g.Z = data[i].Z; g.choice = data[i].choice;
    g.ldn = round_up(s.N, 64);
    g.mc_pad = round_up(s.mc, kTile);
    g.nt1d = (int)(g.mc_pad / kTile);
    build_blocking(s, b->op, &g.build_ob, &g.build_kc);
    g.zrows = zblocks_rows(s, b->fp64);
    g.zsplit = (int)std::max<int64_t>(1, s.N / 4096);
    // band tiles of this problem
    band_maps[i].assign((size_t)g.nt1d * g.nt1d, -1);
    if (s.q > 0)
      for (int k = 1; k < s.K; ++k) {
        const int lo = (int)((int64_t)(k - 1) * s.q / kTile), hi = (int)(((int64_t)k * s.q - 1) / kTile);
        for (int ti = lo; ti <= hi; ++ti)
          for (int tj = lo; tj <= ti; ++tj)
            if (band_maps[i][(size_t)ti * g.nt1d + tj] < 0) {
              band_maps[i][(size_t)ti * g.nt1d + tj] = (int)bands[i].size();
              bands[i].push_back(make_int2(ti, tj));
            }
      }
    g.main_off = main_elems;
    main_elems += (int64_t)g.nt1d * (g.nt1d + 1) / 2 * kTile * kTile;
    g.band_off = band_elems;
    band_elems += (int64_t)bands[i].size() * kTile * kTile;
    g.z_off = z_elems;
    if (s.f > 0) z_elems += (int64_t)g.zsplit * zblocks_outputs(s);
    Off &o = offs[i];
    auto take = [&](size_t nbytes) { size_t at = bytes; bytes += (nbytes + 255) & ~(size_t)255; return at; };
    o.P = take((size_t)s.N * s.K * tsz);
    o.zbar = take((size_t)s.N * s.f * tsz);
    o.At = take((size_t)g.mc_pad * g.ldn * esz);
    o.Ad = take((size_t)g.mc_pad * g.ldn * esz);
    o.F = take((size_t)s.n * s.n * 8);
    o.F32 = b->mixed ? take((size_t)s.n * s.n * 4) : 0;
    o.grad = take((size_t)s.n * 8);
    o.delta = take((size_t)s.n * 8);
    o.scal = take(kGsCount * 8);
    o.rwork = take((size_t)2 * s.n * 8);
    o.band_of = take(band_maps[i].size() * sizeof(int));
  }
  if (b->nmax > 1400) return fail(MNL_ERR_UNSUPPORTED);  // per-problem solve keeps 128 n bytes in shared memory
  unsigned char *arena = nullptr;
  if ((rc = balloc(b, &arena, bytes))) return fail(rc);
  if (cudaMemsetAsync(arena, 0, bytes, b->st) != cudaSuccess) { cudaGetLastError(); return fail(MNL_ERR_CUDA); }
  for (int i = 0; i < count; ++i) {
    GroupProblem &g = b->hp[i];
    const Off &o = offs[i];
    g.P = arena + o.P;
    g.zbar = arena + o.zbar;
    g.At = arena + o.At;
    g.Ad = arena + o.Ad;
    g.F = reinterpret_cast<double *>(arena + o.F);
    g.F32 = b->mixed ? reinterpret_cast<float *>(arena + o.F32) : nullptr;
    g.grad = reinterpret_cast<double *>(arena + o.grad);
    g.delta = reinterpret_cast<double *>(arena + o.delta);
    g.scal = reinterpret_cast<double *>(arena + o.scal);
    g.rwork = reinterpret_cast<double *>(arena + o.rwork);
    g.band_of = reinterpret_cast<int *>(arena + o.band_of);
    if (!band_maps[i].empty() && cudaMemcpy(g.band_of, band_maps[i].data(), band_maps[i].size() * sizeof(int),
                                            cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaGetLastError();
      return fail(MNL_ERR_CUDA);
    }
  }
  const size_t csz = b->fp64 ? 8 : 4;
  if ((rc = balloc(b, &b->main_part, (size_t)main_elems * csz)) ||
      (rc = balloc(b, &b->band_part, (size_t)band_elems * csz)) || (rc = balloc(b, &b->z_part, (size_t)z_elems * tsz)) ||
      (rc = balloc(b, &b->probs, (size_t)count * sizeof(GroupProblem))) ||
      (rc = balloc(b, &b->active, (size_t)count * sizeof(int))) ||
      (rc = balloc(b, &b->pending, (size_t)count * sizeof(int))) ||
      (rc = balloc(b, &b->accepted, (size_t)count * sizeof(int))) ||
      (rc = balloc(b, &b->status, (size_t)count * sizeof(int))) ||
      (rc = balloc(b, &b->stop, (size_t)count * sizeof(int))) || (rc = balloc(b, &b->counts, 4 * sizeof(int))) ||
      (rc = balloc(b, &b->err, sizeof(int))))
    return fail(rc);
  // work items
  std::vector<GroupItem> bi, zi, ai;
  size_t bsm = 0, zsm = 0;
  for (int i = 0; i < count; ++i) {
    const Shape &s = b->shapes[i];
    const GroupProblem &g = b->hp[i];
    if (s.mc > 0) {
      const int nblk = (int)((s.N + g.build_ob - 1) / g.build_ob);
      for (int k = 0; k < nblk; ++k) bi.push_back({i, k});
      bsm = std::max(bsm, build_smem_bytes(s, b->op, g.build_ob, g.build_kc));
    }
    if (s.f > 0) {
      const int64_t nzt = zblocks_outputs(s);
      const int chunks = (int)((nzt + 8191) / 8192);
      for (int k = 0; k < g.zsplit * chunks; ++k) zi.push_back({i, k});
      zsm = std::max(zsm, zblocks_smem(s, g.zrows, b->fp64));
    }
    const int ncb = (int)((s.n + kAssembleCols - 1) / kAssembleCols);
    for (int k = 0; k < ncb; ++k) ai.push_back({i, k});
  }
  b->n_build = (int)bi.size();
  b->n_z = (int)zi.size();
  b->n_asm = (int)ai.size();
  b->build_smem = bsm;
  b->z_smem = zsm;
  b->chol_smem = grouped_chol_smem(b->nmax);
  if (bsm > 200 * 1024 || zsm > 200 * 1024 || b->chol_smem > 220 * 1024) return fail(MNL_ERR_UNSUPPORTED);
  if ((rc = balloc(b, &b->build_items, bi.size() * sizeof(GroupItem))) ||
      (rc = balloc(b, &b->z_items, zi.size() * sizeof(GroupItem))) ||
      (rc = balloc(b, &b->asm_items, ai.size() * sizeof(GroupItem))))
    return fail(rc);
  if ((!bi.empty() && cudaMemcpy(b->build_items, bi.data(), bi.size() * sizeof(GroupItem), cudaMemcpyHostToDevice)) ||
      (!zi.empty() && cudaMemcpy(b->z_items, zi.data(), zi.size() * sizeof(GroupItem), cudaMemcpyHostToDevice)) ||
      (!ai.empty() && cudaMemcpy(b->asm_items, ai.data(), ai.size() * sizeof(GroupItem), cudaMemcpyHostToDevice))) {
    cudaGetLastError();
    return fail(MNL_ERR_CUDA);
  }
  // contraction units: per-problem maps (tensor-core modes), tiles in
  // decreasing K-length (longest first, round-robin over the CTAs)
  {
    std::vector<CUtensorMap> maps(b->fp64 ? 1 : 2 * (size_t)count);
    std::vector<SyrkUnit> um, ub;
    for (int i = 0; i < count; ++i) {
      const GroupProblem &g = b->hp[i];
      if (b->shapes[i].mc == 0) continue;
      if (!b->fp64 && (encode_operand_map(b->op, g.At, g.mc_pad, g.ldn, &maps[2 * i]) != cudaSuccess ||
                       encode_operand_map(b->op, g.Ad, g.mc_pad, g.ldn, &maps[2 * i + 1]) != cudaSuccess))
        return fail(MNL_ERR_CUDA);
      const int kb = b->fp64 ? (int)(g.ldn / f64_chunk_rows()) : tc_kblocks(b->op, g.ldn);
      const int mA = b->fp64 ? 0 : 2 * i, mD = b->fp64 ? 1 : 2 * i + 1;
      int t = 0;
      for (int ti = 0; ti < g.nt1d; ++ti)
        for (int tj = 0; tj <= ti; ++tj, ++t)
          um.push_back({mA, i, ti, tj, 0, kb, g.main_off + (int64_t)t * kTile * kTile});
      for (size_t k = 0; k < bands[i].size(); ++k)
        ub.push_back({mD, i, bands[i][k].x, bands[i][k].y, 0, kb, g.band_off + (int64_t)k * kTile * kTile});
    }
    auto by_len = [](const SyrkUnit &a, const SyrkUnit &c) { return (a.kb1 - a.kb0) > (c.kb1 - c.kb0); };
    std::stable_sort(um.begin(), um.end(), by_len);
    std::stable_sort(ub.begin(), ub.end(), by_len);
    b->nunits_main = (int)um.size();
    b->nunits_band = (int)ub.size();
    if ((rc = balloc(b, &b->maps, maps.size() * sizeof(CUtensorMap))) ||
        (rc = balloc(b, &b->units_main, um.size() * sizeof(SyrkUnit))) ||
        (rc = balloc(b, &b->units_band, ub.size() * sizeof(SyrkUnit))))
      return fail(rc);
    if (cudaMemcpy(b->maps, maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice) ||
        (!um.empty() && cudaMemcpy(b->units_main, um.data(), um.size() * sizeof(SyrkUnit), cudaMemcpyHostToDevice)) ||
        (!ub.empty() && cudaMemcpy(b->units_band, ub.data(), ub.size() * sizeof(SyrkUnit), cudaMemcpyHostToDevice))) {
      cudaGetLastError();
      return fail(MNL_ERR_CUDA);
    }
  }
  // descriptors (theta pointers are set by each fit), then autotune the pass tile height
  if (cudaMemcpy(b->probs, b->hp.data(), (size_t)count * sizeof(GroupProblem), cudaMemcpyHostToDevice) ||
      cudaMemsetAsync(b->active, 0, (size_t)count * sizeof(int), b->st)) {
    cudaGetLastError();
    return fail(MNL_ERR_CUDA);
  }
  cudaStreamSynchronize(b->st);
  int rows = 16;
  if (b->fp64) {
    rows = 16;
  } else {
    // timing needs the probabilities' inputs only: theta = 0 everywhere (the arena is zeroed)
    std::vector<int> ones(count, 1);
    double *th0 = nullptr;
    if ((rc = balloc(b, &th0, (size_t)b->theta_total * 8))) return fail(rc);
    cudaMemset(th0, 0, (size_t)b->theta_total * 8);
    std::vector<GroupProblem> tmp = b->hp;
    for (int i = 0; i < count; ++i) { tmp[i].theta = th0 + b->theta_off[i]; tmp[i].delta = th0 + b->theta_off[i]; }
    cudaMemcpy(b->probs, tmp.data(), (size_t)count * sizeof(GroupProblem), cudaMemcpyHostToDevice);
    cudaMemcpy(b->active, ones.data(), (size_t)count * sizeof(int), cudaMemcpyHostToDevice);
    autotune_rows(b, &rows);
    cudaMemset(b->active, 0, (size_t)count * sizeof(int));
  }
  b->pfull = plan_grouped_pass(b->shapes, b->fp64, rows, b->nsm);
  b->pll = plan_grouped_pass(b->shapes, b->fp64, rows, b->nsm);
  if (!b->pfull.ok) return fail(MNL_ERR_UNSUPPORTED);
  b->pll.grid = b->pfull.grid;
  std::vector<PassSeg> segs;
  std::vector<int> ss, sl, sls;
  int64_t plen = 0;
  build_pass_lists(b, rows, b->pfull.grid, segs, ss, sl, sls, &plen);
  if ((rc = upload_pass_lists(b, segs, ss, sl, sls, plen))) return fail(rc);
  if (cudaStreamSynchronize(b->st) != cudaSuccess) { cudaGetLastError(); return fail(MNL_ERR_CUDA); }
  *out = b;
  return MNL_OK;
}

int64_t mnl_batch_num_params(const mnl_batch *b, int64_t *offsets) {
  if (!b) return -1;
  if (offsets)
    for (int i = 0; i < b->count; ++i) offsets[i] = b->theta_off[i];
  return b->theta_total;
}

int mnl_batch_fit(mnl_batch *b, const mnl_fit_opts *opts, double *theta, mnl_batch_info *info) {
  if (!b || !theta) return MNL_ERR_INVALID_ARG;
  mnl_fit_opts o;
  mnl_fit_opts_default(&o);
  if (opts) o = *opts;
  if (o.maxiter < 0 || o.max_halvings < 0) return MNL_ERR_INVALID_ARG;
  const double steptol = o.steptol >= 0 ? o.steptol : (b->fp64 ? 1e-10 : 1e-7);
  const int np = b->count;
  const auto wall0 = std::chrono::steady_clock::now();
  // order after the caller's prior work on its stream
  BCK(cudaEventRecord(b->ev_user, b->user_st));
  BCK(cudaStreamWaitEvent(b->st, b->ev_user, 0));
  for (int i = 0; i < np; ++i) b->hp[i].theta = theta + b->theta_off[i];
  BCK(cudaMemcpyAsync(b->probs, b->hp.data(), (size_t)np * sizeof(GroupProblem), cudaMemcpyHostToDevice, b->st));
  {
    std::vector<int> ones(np, 1);
    BCK(cudaMemcpyAsync(b->active, ones.data(), (size_t)np * sizeof(int), cudaMemcpyHostToDevice, b->st));
    BCK(cudaMemsetAsync(b->status, 0, (size_t)np * sizeof(int), b->st));
    BCK(cudaMemsetAsync(b->stop, 0, (size_t)np * sizeof(int), b->st));
    BCK(cudaMemsetAsync(b->accepted, 0, (size_t)np * sizeof(int), b->st));
    BCK(cudaMemsetAsync(b->err, 0, sizeof(int), b->st));
    for (int i = 0; i < np; ++i) BCK(cudaMemsetAsync(b->hp[i].scal, 0, kGsCount * sizeof(double), b->st));
    BCK(cudaStreamSynchronize(b->st));
  }
  // one iteration + first line-search round, captured once per set of options
  if (b->have_graph && (b->graph_gtol != o.gtol || b->graph_halvings != o.max_halvings)) {
    cudaGraphExecDestroy(b->graph);
    b->have_graph = false;
  }
  if (!b->have_graph) {
    cudaGraph_t g;
    BCK(cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal));
    int rc1 = enqueue_iteration(b, o);
    int rc2 = rc1 == MNL_OK ? enqueue_ls_round(b, o) : rc1;
    cudaError_t ec = cudaStreamEndCapture(b->st, &g);
    if (rc2 != MNL_OK) return rc2;
    BCK(ec);
    BCK(cudaGraphInstantiate(&b->graph, g, 0));
    cudaGraphDestroy(g);
    b->have_graph = true;
    b->graph_gtol = o.gtol;
    b->graph_halvings = o.max_halvings;
  }
  const int tb = 256, nb = (np + tb - 1) / tb;
  int iters = 0;
  float t_graph = 0.f;
  for (int it = 0; it < o.maxiter; ++it) {
    BCK(cudaEventRecord(b->t0, b->st));
    BCK(cudaGraphLaunch(b->graph, b->st));
    BCK(cudaEventRecord(b->t1, b->st));
    BCK(cudaMemcpyAsync(b->h_counts, b->counts, 2 * sizeof(int), cudaMemcpyDeviceToHost, b->st));
    BCK(cudaStreamSynchronize(b->st));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, b->t0, b->t1);
    t_graph += ms;
    int rounds = 1;
    while (b->h_counts[1] > 0 && rounds <= o.max_halvings) {
      int rc = enqueue_ls_round(b, o);
      if (rc) return rc;
      BCK(cudaMemcpyAsync(b->h_counts, b->counts, 2 * sizeof(int), cudaMemcpyDeviceToHost, b->st));
      BCK(cudaStreamSynchronize(b->st));
      ++rounds;
    }
    theta_update_kernel<<<np, 256, 0, b->st>>>(b->probs, b->accepted, b->active, b->stop, steptol, o.ftol);
    count_kernel<<<1, 256, 0, b->st>>>(np, b->active, b->pending, b->counts);
    BCK(cudaGetLastError());
    BCK(cudaMemcpyAsync(b->h_counts, b->counts, 2 * sizeof(int), cudaMemcpyDeviceToHost, b->st));
    BCK(cudaMemcpyAsync(b->h_counts + 2, b->err, sizeof(int), cudaMemcpyDeviceToHost, b->st));
    BCK(cudaStreamSynchronize(b->st));
    ++iters;
    if (b->h_counts[2]) return MNL_ERR_TIMEOUT;
    if (b->h_counts[0] == 0) break;
  }
  (void)nb;
  // results
  std::vector<int> st(np), sp(np);
  std::vector<double> sc((size_t)np * kGsCount);
  BCK(cudaMemcpyAsync(st.data(), b->status, np * sizeof(int), cudaMemcpyDeviceToHost, b->st));
  BCK(cudaMemcpyAsync(sp.data(), b->stop, np * sizeof(int), cudaMemcpyDeviceToHost, b->st));
  for (int i = 0; i < np; ++i)
    BCK(cudaMemcpyAsync(sc.data() + (size_t)i * kGsCount, b->hp[i].scal, kGsCount * sizeof(double),
                        cudaMemcpyDeviceToHost, b->st));
  BCK(cudaStreamSynchronize(b->st));
  BCK(cudaEventRecord(b->ev_done, b->st));
  BCK(cudaStreamWaitEvent(b->user_st, b->ev_done, 0));
  int nconv = 0, nerr = 0;
  for (int i = 0; i < np; ++i) {
    if (st[i] != MNL_OK) ++nerr;
    else if (sp[i] != 0) ++nconv;
    if (info && info->problems) {
      mnl_batch_problem_info &pi = info->problems[i];
      pi.status = st[i] != MNL_OK ? st[i] : (sp[i] != 0 ? MNL_OK : MNL_MAXITER);
      pi.stop_reason = sp[i] != 0 ? sp[i] : (st[i] == MNL_OK ? MNL_STOP_MAXITER : 0);
      pi.iters = (int)sc[(size_t)i * kGsCount + kGsIters];
      pi.ls_evals = (int)sc[(size_t)i * kGsCount + kGsLsEvals];
      pi.loglik = sc[(size_t)i * kGsCount + kGsL];
      pi.grad_inf = sc[(size_t)i * kGsCount + kGsGinf];
    }
  }
  if (info) {
    info->iterations = iters;
    info->converged = nconv;
    info->failed = nerr;
    info->t_total_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - wall0).count();
    info->t_graph_ms = t_graph;
    info->pass_rows = b->pfull.rows;
  }
  if (nconv == np) return MNL_OK;
  for (int i = 0; i < np; ++i)
    if (st[i] != MNL_OK) return st[i];
  return MNL_MAXITER;
}

int mnl_batch_destroy(mnl_batch *b) {
  if (!b) return MNL_OK;
  cudaStreamSynchronize(b->st);
  cudaGetLastError();
  bfree(b);
  delete b;
  return MNL_OK;
}

}  // extern "C"
