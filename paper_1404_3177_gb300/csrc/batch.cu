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
#include <deque>
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
                                                           int *__restrict__ stop, double steptol, double ftol,
                                                           double noise_step) {
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
    const double rel = a / fmax(1.0, c);
    const double prev = sc[kGsIters] > 1.0 ? sc[kGsPrevStep] : 1e300;
    sc[kGsPrevStep] = rel;
    if (ftol > 0 && fabs(dl) < ftol) { stop[b] = MNL_STOP_FTOL; active[b] = 0; }
    else if (steptol > 0 && rel <= steptol) { stop[b] = MNL_STOP_STEPTOL; active[b] = 0; }
    else if (noise_step > 0 && rel > 0.5 * prev && rel <= noise_step) { stop[b] = MNL_STOP_NOISE; active[b] = 0; }
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


namespace {

#define BCK(x)                                                                              \
  do {                                                                                      \
    cudaError_t e_ = (x);                                                                   \
    if (e_ != cudaSuccess) {                                                                \
      cudaGetLastError();                                                                   \
      return e_ == cudaErrorMemoryAllocation ? MNL_ERR_OOM : MNL_ERR_CUDA;                  \
    }                                                                                       \
  } while (0)

// Stream, events and device properties shared by a batch or a server.
struct Engine {
  int prec = 0;
  OpType op = OpType::BF16;
  bool fp64 = false, mixed = true;
  cudaStream_t user_st = nullptr, st = nullptr;
  cudaEvent_t ev_user = nullptr, ev_done = nullptr, t0 = nullptr, t1 = nullptr;
  int dev = 0, nsm = 148;
  int *h_counts = nullptr;  // pinned: [0] active, [1] pending, [2] error word
  int init(int precision, void *stream) {
    prec = precision;
    fp64 = precision == MNL_FP64;
    op = fp64 ? OpType::F64 : precision == MNL_TF32 ? OpType::TF32 : OpType::BF16;
    mixed = !fp64;
    user_st = reinterpret_cast<cudaStream_t>(stream);
    BCK(cudaGetDevice(&dev));
    BCK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    BCK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    BCK(cudaEventCreateWithFlags(&ev_user, cudaEventDisableTiming));
    BCK(cudaEventCreateWithFlags(&ev_done, cudaEventDisableTiming));
    BCK(cudaEventCreate(&t0));
    BCK(cudaEventCreate(&t1));
    BCK(cudaMallocHost(&h_counts, 4 * sizeof(int)));
    return MNL_OK;
  }
  void release() {
    if (h_counts) cudaFreeHost(h_counts);
    if (st) cudaStreamDestroy(st);
    for (cudaEvent_t e : {ev_user, ev_done, t0, t1})
      if (e) cudaEventDestroy(e);
    h_counts = nullptr;
    st = nullptr;
    ev_user = ev_done = t0 = t1 = nullptr;
  }
};

// Persistent device state of one problem, laid out in one chunk.
struct ProbLayout {
  Shape s;
  int64_t ldn = 0, mc_pad = 0;
  int nt1d = 0, build_ob = 64, build_kc = 1, zsplit = 1;
  std::vector<int2> bands;
  std::vector<int> band_map;
  size_t P = 0, zbar = 0, At = 0, Ad = 0, F = 0, F32 = 0, grad = 0, delta = 0, scal = 0, rwork = 0, band_of = 0;
  size_t theta = 0, X = 0, Y = 0, Z = 0, choice = 0;  // owned copies (server requests)
  // multi-CTA solve workspace (problems with n_theta > kCtaSolveMaxN)
  size_t dinv = 0, mwork = 0, cwork = 0, sstat = 0;
  bool large = false;
  size_t bytes = 0;
};

ProbLayout layout_problem(const mnl_dims &d, OpType op, bool fp64, bool mixed, bool own) {
  ProbLayout L;
  const Shape s = make_shape(d);
  L.s = s;
  const size_t tsz = fp64 ? 8 : 4;
  const size_t esz = fp64 ? 8 : op == OpType::TF32 ? 4 : 2;
  L.ldn = round_up(s.N, 64);
  L.mc_pad = round_up(s.mc, kTile);
  L.nt1d = (int)(L.mc_pad / kTile);
  build_blocking(s, op, &L.build_ob, &L.build_kc);
  L.zsplit = (int)std::max<int64_t>(1, s.N / 4096);
  L.band_map.assign((size_t)L.nt1d * L.nt1d, -1);
  if (s.q > 0)
    for (int k = 1; k < s.K; ++k) {
      const int lo = (int)((int64_t)(k - 1) * s.q / kTile), hi = (int)(((int64_t)k * s.q - 1) / kTile);
      for (int ti = lo; ti <= hi; ++ti)
        for (int tj = lo; tj <= ti; ++tj)
          if (L.band_map[(size_t)ti * L.nt1d + tj] < 0) {
            L.band_map[(size_t)ti * L.nt1d + tj] = (int)L.bands.size();
            L.bands.push_back(make_int2(ti, tj));
          }
    }
  size_t b = 0;
  auto take = [&](size_t nbytes) { const size_t at = b; b += (nbytes + 255) & ~(size_t)255; return at; };
  L.P = take((size_t)s.N * s.K * tsz);
  L.zbar = take((size_t)s.N * s.f * tsz);
  L.At = take((size_t)L.mc_pad * L.ldn * esz);
  L.Ad = take((size_t)L.mc_pad * L.ldn * esz);
  L.F = take((size_t)s.n * s.n * 8);
  L.F32 = mixed ? take((size_t)s.n * s.n * 4) : 0;
  L.grad = take((size_t)s.n * 8);
  L.delta = take((size_t)s.n * 8);
  L.scal = take(kGsCount * 8);
  L.rwork = take((size_t)2 * s.n * 8);
  L.band_of = take(L.band_map.size() * sizeof(int));
  L.large = s.n > kCtaSolveMaxN;
  if (L.large) {
    L.dinv = take((size_t)s.n * 8);
    L.mwork = mixed ? take(mixed_solve_bytes(s.n)) : 0;
    L.cwork = take(chol_work_bytes(s.n));
    L.sstat = take(16);
    if (!mixed) L.F32 = 0;
  }
  if (own) {
    L.theta = take((size_t)s.n * 8);
    L.X = take((size_t)s.N * s.p * 4);
    L.Y = take((size_t)s.N * s.K * s.d * 4);
    L.Z = take((size_t)s.N * s.K * s.f * 4);
    L.choice = take((size_t)s.N * 4);
  }
  L.bytes = b;
  return L;
}

// Descriptor of a problem whose chunk starts at `base`; data and theta either
// given (batch) or inside the chunk (server).
void bind_problem(const ProbLayout &L, unsigned char *base, const mnl_data *data, double *theta, GroupProblem &g) {
  std::memset(&g, 0, sizeof(g));
  const Shape &s = L.s;
  g.N = s.N; g.K = s.K; g.p = s.p; g.d = s.d; g.f = s.f; g.n = s.n; g.mc = s.mc;
  if (data) {
    g.X = data->X; g.Y = data->Y; g.Z = data->Z; g.choice = data->choice;
  } else {
    g.X = reinterpret_cast<const float *>(base + L.X);
    g.Y = reinterpret_cast<const float *>(base + L.Y);
    g.Z = reinterpret_cast<const float *>(base + L.Z);
    g.choice = reinterpret_cast<const int32_t *>(base + L.choice);
  }
  g.theta = theta ? theta : reinterpret_cast<double *>(base + L.theta);
  g.grad = reinterpret_cast<double *>(base + L.grad);
  g.delta = reinterpret_cast<double *>(base + L.delta);
  g.P = base + L.P;
  g.zbar = base + L.zbar;
  g.At = base + L.At;
  g.Ad = base + L.Ad;
  g.ldn = L.ldn;
  g.mc_pad = L.mc_pad;
  g.nt1d = L.nt1d;
  g.zsplit = L.zsplit;
  g.build_ob = L.build_ob;
  g.build_kc = L.build_kc;
  g.band_of = reinterpret_cast<int *>(base + L.band_of);
  g.F = reinterpret_cast<double *>(base + L.F);
  g.F32 = L.F32 ? reinterpret_cast<float *>(base + L.F32) : nullptr;
  g.rwork = reinterpret_cast<double *>(base + L.rwork);
  g.scal = reinterpret_cast<double *>(base + L.scal);
}

// Grow-only device buffer.
struct DBuf {
  void *p = nullptr;
  size_t cap = 0;
  int ensure(size_t bytes) {
    if (bytes <= cap) return MNL_OK;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    const size_t want = std::max(bytes, cap + cap / 2);
    if (cudaMalloc(&p, want) != cudaSuccess) { cudaGetLastError(); return MNL_ERR_OOM; }
    cap = want;
    return MNL_OK;
  }
  void release() { if (p) cudaFree(p); p = nullptr; cap = 0; }
  template <typename T> T *as() const { return reinterpret_cast<T *>(p); }
};

// Descriptors, flags and work lists of the problems being iterated together.
struct WorkSet {
  int count = 0;
  int rows = 16;
  std::vector<GroupProblem> hp;     // host copy of the descriptors
  std::vector<Shape> shapes;
  DBuf probs, flags, counts, err, segs, seg_start, slot_start, slot_segs, partials;
  DBuf build_items, z_items, asm_items, maps, units_main, units_band, main_part, band_part, z_part, chol_list;
  GroupedPassPlan pfull{}, pll{};
  // per-problem solves by size class (each launch sizes its shared memory for its largest member)
  struct CholBucket {
    int offset, count;
    size_t smem;
  };
  std::vector<CholBucket> chol_buckets;
  int n_build = 0, n_z = 0, n_asm = 0, nunits_main = 0, nunits_band = 0;
  size_t build_smem = 0, z_smem = 0, chol_smem = 0;
  int64_t nmax = 0;
  int *active() const { return flags.as<int>(); }
  int *pending() const { return flags.as<int>() + count; }
  int *accepted() const { return flags.as<int>() + 2 * count; }
  int *status() const { return flags.as<int>() + 3 * count; }
  int *stop() const { return flags.as<int>() + 4 * count; }
  void release() {
    for (DBuf *d : {&probs, &flags, &counts, &err, &segs, &seg_start, &slot_start, &slot_segs, &partials, &build_items,
                    &z_items, &asm_items, &maps, &units_main, &units_band, &main_part, &band_part, &z_part,
                    &chol_list})
      d->release();
  }
};

// Pass segments: the tiles of all problems in order, cut into one contiguous
// range per CTA of about equal cost, then at problem boundaries.
void build_pass_lists(const std::vector<Shape> &shapes, int rows, int grid, std::vector<PassSeg> &segs,
                      std::vector<int> &seg_start, std::vector<int> &slot_start, std::vector<int> &slot_segs,
                      int64_t *partial_len) {
  struct TileRun { int problem; int64_t ntiles; double cost; };
  std::vector<TileRun> runs;
  double total = 0.0;
  const int count = (int)shapes.size();
  for (int i = 0; i < count; ++i) {
    const Shape &s = shapes[i];
    const int64_t nt = (s.N + rows - 1) / rows;
    // modelled cost of one tile: its arithmetic, its outputs, and a fixed part (staging latency, barriers)
    const double c = (double)rows * s.K * (s.p + s.d + s.f + 1) + (double)s.nout + 4096.0;
    runs.push_back({i, nt, c});
    total += c * nt;
  }
  segs.clear();
  seg_start.assign(grid + 1, 0);
  std::vector<std::vector<int>> per_prob(count);
  int64_t off_full = 0, off_ll = 0;
  double acc = 0.0;
  size_t ri = 0;
  int64_t ti = 0;  // next tile within runs[ri]
  for (int c = 0; c < grid; ++c) {
    seg_start[c] = (int)segs.size();
    const double target = total * (c + 1) / grid;
    while (ri < runs.size() && (acc < target - 1e-9 || c == grid - 1)) {
      const TileRun &r = runs[ri];
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
      off_full += 2 + shapes[r.problem].n;
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
  slot_start.assign(count + 1, 0);
  slot_segs.clear();
  for (int i = 0; i < count; ++i) {
    slot_start[i] = (int)slot_segs.size();
    for (int s : per_prob[i]) slot_segs.push_back(s);
  }
  slot_start[count] = (int)slot_segs.size();
  *partial_len = std::max(off_full, off_ll);
}

template <typename T>
int upload(DBuf &d, const std::vector<T> &v, cudaStream_t st) {
  int rc = d.ensure(std::max<size_t>(1, v.size()) * sizeof(T));
  if (rc) return rc;
  if (!v.empty()) BCK(cudaMemcpyAsync(d.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st));
  return MNL_OK;
}

// (Re)build a work set over the descriptors W.hp (persistent pointers already
// bound) with layouts L; fills the per-set partial offsets and work lists.
int ws_build(Engine &E, WorkSet &W, const std::vector<const ProbLayout *> &L, int rows) {
  const int count = W.count = (int)W.hp.size();
  W.rows = rows;
  W.shapes.clear();
  for (const ProbLayout *l : L) W.shapes.push_back(l->s);
  int rc;
  // contraction partials: per-set offsets
  const size_t csz = E.fp64 ? 8 : 4, tsz = E.fp64 ? 8 : 4;
  int64_t main_elems = 0, band_elems = 0, z_elems = 0;
  W.nmax = 0;
  for (int i = 0; i < count; ++i) {
    GroupProblem &g = W.hp[i];
    const ProbLayout &l = *L[i];
    g.main_off = main_elems;
    main_elems += (int64_t)l.nt1d * (l.nt1d + 1) / 2 * kTile * kTile;
    g.band_off = band_elems;
    band_elems += (int64_t)l.bands.size() * kTile * kTile;
    g.z_off = z_elems;
    if (l.s.f > 0) z_elems += (int64_t)l.zsplit * zblocks_outputs(l.s);
    if (!l.large) W.nmax = std::max(W.nmax, l.s.n);
  }
  if ((rc = W.main_part.ensure(std::max<int64_t>(1, main_elems) * csz)) ||
      (rc = W.band_part.ensure(std::max<int64_t>(1, band_elems) * csz)) ||
      (rc = W.z_part.ensure(std::max<int64_t>(1, z_elems) * tsz)))
    return rc;
  // items
  std::vector<GroupItem> bi, zi, ai;
  size_t bsm = 0, zsm = 0;
  for (int i = 0; i < count; ++i) {
    const ProbLayout &l = *L[i];
    const Shape &s = l.s;
    if (s.mc > 0) {
      const int nblk = (int)((s.N + l.build_ob - 1) / l.build_ob);
      for (int k = 0; k < nblk; ++k) bi.push_back({i, k});
      bsm = std::max(bsm, build_smem_bytes(s, E.op, l.build_ob, l.build_kc));
    }
    if (s.f > 0) {
      const int parts = zblocks_parts(s, E.fp64);
      for (int k = 0; k < l.zsplit * parts; ++k) zi.push_back({i, k});
      zsm = std::max(zsm, zblocks_smem(s, E.fp64));
    }
    const int ncb = (int)((s.n + kAssembleCols - 1) / kAssembleCols);
    for (int k = 0; k < ncb; ++k) ai.push_back({i, k});
  }
  W.n_build = (int)bi.size();
  W.n_z = (int)zi.size();
  W.n_asm = (int)ai.size();
  W.build_smem = bsm;
  W.z_smem = zsm;
  W.chol_smem = grouped_chol_smem(W.nmax);
  if (bsm > 200 * 1024 || zsm > 200 * 1024 || W.chol_smem > 220 * 1024) return MNL_ERR_UNSUPPORTED;
  {  // size classes of the per-problem solves, largest first within a class
    std::vector<int> order;
    for (int i = 0; i < count; ++i)
      if (!L[i]->large) order.push_back(i);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return L[a]->s.n > L[b]->s.n; });
    static const int64_t bounds[] = {128, 256, 512, kCtaSolveMaxN};
    W.chol_buckets.clear();
    size_t at = order.size();  // walk from the smallest
    for (int64_t hi : bounds) {
      size_t from = at;
      while (from > 0 && L[order[from - 1]]->s.n <= hi) --from;
      if (from < at) W.chol_buckets.push_back({(int)from, (int)(at - from), grouped_chol_smem(L[order[from]]->s.n)});
      at = from;
    }
    if ((rc = upload(W.chol_list, order, E.st))) return rc;
  }
  if ((rc = upload(W.build_items, bi, E.st)) || (rc = upload(W.z_items, zi, E.st)) ||
      (rc = upload(W.asm_items, ai, E.st)))
    return rc;
  // contraction units (longest K range first, dealt round-robin over the CTAs)
  std::vector<CUtensorMap> maps(E.fp64 ? 1 : 2 * (size_t)count);
  std::vector<SyrkUnit> um, ub;
  for (int i = 0; i < count; ++i) {
    const GroupProblem &g = W.hp[i];
    const ProbLayout &l = *L[i];
    if (l.s.mc == 0) continue;
    if (!E.fp64 && (encode_operand_map(E.op, g.At, g.mc_pad, g.ldn, &maps[2 * i]) != cudaSuccess ||
                    encode_operand_map(E.op, g.Ad, g.mc_pad, g.ldn, &maps[2 * i + 1]) != cudaSuccess))
      return MNL_ERR_CUDA;
    const int kb = E.fp64 ? (int)(g.ldn / f64_chunk_rows()) : tc_kblocks(E.op, g.ldn);
    const int mA = E.fp64 ? 0 : 2 * i, mD = E.fp64 ? 1 : 2 * i + 1;
    int t = 0;
    for (int ti = 0; ti < l.nt1d; ++ti)
      for (int tj = 0; tj <= ti; ++tj, ++t)
        um.push_back({mA, i, ti, tj, 0, kb, g.main_off + (int64_t)t * kTile * kTile, 0, -1});
    for (size_t k = 0; k < l.bands.size(); ++k)
      ub.push_back({mD, i, l.bands[k].x, l.bands[k].y, 0, kb, g.band_off + (int64_t)k * kTile * kTile, 0, -1});
  }
  if (E.fp64) {
    auto by_len = [](const SyrkUnit &a, const SyrkUnit &c) { return (a.kb1 - a.kb0) > (c.kb1 - c.kb0); };
    std::stable_sort(um.begin(), um.end(), by_len);
    std::stable_sort(ub.begin(), ub.end(), by_len);
  } else {  // bounded accumulation chunks, one CTA per job (the kernel runs on E.nsm CTAs)
    um = schedule_syrk_units(um, E.nsm, tc_chunk_kblocks(E.op));
    ub = schedule_syrk_units(ub, E.nsm, tc_chunk_kblocks(E.op));
  }
  W.nunits_main = (int)um.size();
  W.nunits_band = (int)ub.size();
  if ((rc = upload(W.maps, maps, E.st)) || (rc = upload(W.units_main, um, E.st)) || (rc = upload(W.units_band, ub, E.st)))
    return rc;
  // grouped pass
  W.pfull = plan_grouped_pass(W.shapes, E.fp64, rows, E.nsm);
  if (!W.pfull.ok) return MNL_ERR_UNSUPPORTED;
  W.pll = W.pfull;
  std::vector<PassSeg> segs;
  std::vector<int> ss, sl, sls;
  int64_t plen = 0;
  build_pass_lists(W.shapes, rows, W.pfull.grid, segs, ss, sl, sls, &plen);
  if ((rc = upload(W.segs, segs, E.st)) || (rc = upload(W.seg_start, ss, E.st)) || (rc = upload(W.slot_start, sl, E.st)) ||
      (rc = upload(W.slot_segs, sls, E.st)) || (rc = W.partials.ensure(std::max<int64_t>(1, plen) * sizeof(double))))
    return rc;
  // descriptors and flags
  if ((rc = upload(W.probs, W.hp, E.st)) || (rc = W.flags.ensure(5 * (size_t)count * sizeof(int))) ||
      (rc = W.counts.ensure(4 * sizeof(int))) || (rc = W.err.ensure(sizeof(int))))
    return rc;
  BCK(cudaMemsetAsync(W.flags.p, 0, 5 * (size_t)count * sizeof(int), E.st));
  return MNL_OK;
}

const GroupProblem *dprobs(const WorkSet &W) { return W.probs.as<GroupProblem>(); }

int enqueue_iteration(Engine &E, WorkSet &W, const mnl_fit_opts &o, bool with_ls_init = true) {
  const int np = W.count;
  const int tb = 256, nb = (np + tb - 1) / tb;
  const GroupProblem *P = dprobs(W);
  BCK(launch_grouped_pass(W.pfull, E.fp64, true, P, W.segs.as<PassSeg>(), W.seg_start.as<int>(), W.active(),
                          W.partials.as<double>(), E.st));
  BCK(launch_grouped_reduce(np, true, P, W.slot_start.as<int>(), W.segs.as<PassSeg>(), W.slot_segs.as<int>(),
                            W.active(), W.partials.as<double>(), kGsL, E.st));
  gtol_check_kernel<<<nb, tb, 0, E.st>>>(np, P, W.active(), W.status(), W.stop(), o.gtol);
  BCK(cudaGetLastError());
  BCK(launch_grouped_build(E.op, P, W.build_items.as<GroupItem>(), W.n_build, W.active(), W.build_smem, E.st));
  if (E.fp64) {
    BCK(launch_grouped_syrk_f64(P, W.units_main.as<SyrkUnit>(), W.nunits_main, W.active(), W.main_part.as<double>(),
                                E.st));
    BCK(launch_grouped_syrk_f64(P, W.units_band.as<SyrkUnit>(), W.nunits_band, W.active(), W.band_part.as<double>(),
                                E.st));
  } else {
    BCK(launch_syrk_tc(E.op, W.maps.as<CUtensorMap>(), W.units_main.as<SyrkUnit>(), W.nunits_main, W.active(), E.nsm,
                       W.main_part.as<float>(), W.err.as<int>(), E.st));
    BCK(launch_syrk_tc(E.op, W.maps.as<CUtensorMap>(), W.units_band.as<SyrkUnit>(), W.nunits_band, W.active(), E.nsm,
                       W.band_part.as<float>(), W.err.as<int>(), E.st));
  }
  BCK(launch_grouped_zblocks(E.fp64, P, W.z_items.as<GroupItem>(), W.n_z, W.active(), W.z_smem, W.z_part.p, E.st));
  BCK(launch_grouped_assemble(E.fp64, P, W.asm_items.as<GroupItem>(), W.n_asm, W.active(), W.main_part.p,
                              W.band_part.p, W.z_part.p, E.st));
  // up to 30 refinement steps: each gains a factor of about cond(F) * 2^-24, so ill-conditioned problems need
  // more than a few; the float64 fallback is kept for stagnation and failed float32 factors
  for (const auto &cb : W.chol_buckets)
    BCK(launch_grouped_chol_solve(E.mixed, P, W.chol_list.as<int>() + cb.offset, cb.count, W.active(), 30,
                                  W.status(), cb.smem, kCtaSolveMaxN, E.st));
  if (!with_ls_init) return MNL_OK;
  ls_init_kernel<<<nb, tb, 0, E.st>>>(np, P, W.active(), W.pending(), W.status());
  BCK(cudaGetLastError());
  return MNL_OK;
}

int enqueue_ls_init(Engine &E, WorkSet &W) {
  const int np = W.count;
  ls_init_kernel<<<(np + 255) / 256, 256, 0, E.st>>>(np, dprobs(W), W.active(), W.pending(), W.status());
  BCK(cudaGetLastError());
  return MNL_OK;
}

int enqueue_ls_round(Engine &E, WorkSet &W, const mnl_fit_opts &o) {
  const int np = W.count;
  const int tb = 256, nb = (np + tb - 1) / tb;
  const GroupProblem *P = dprobs(W);
  BCK(launch_grouped_pass(W.pll, E.fp64, false, P, W.segs.as<PassSeg>(), W.seg_start.as<int>(), W.pending(),
                          W.partials.as<double>(), E.st));
  BCK(launch_grouped_reduce(np, false, P, W.slot_start.as<int>(), W.segs.as<PassSeg>(), W.slot_segs.as<int>(),
                            W.pending(), W.partials.as<double>(), kGsLt, E.st));
  const double u = E.fp64 ? std::ldexp(1.0, -53) : std::ldexp(1.0, -24);
  ls_update_kernel<<<nb, tb, 0, E.st>>>(np, P, W.pending(), W.accepted(), W.active(), W.status(), u, o.max_halvings);
  BCK(cudaGetLastError());
  count_kernel<<<1, 256, 0, E.st>>>(np, W.active(), W.pending(), W.counts.as<int>());
  BCK(cudaGetLastError());
  return MNL_OK;
}

// After enqueue_iteration + one enqueue_ls_round: the remaining line-search
// rounds (host loop), the coefficient update and the count of problems still
// iterating (E.h_counts[0]).
int finish_iteration(Engine &E, WorkSet &W, const mnl_fit_opts &o, double steptol) {
  BCK(cudaMemcpyAsync(E.h_counts, W.counts.p, 2 * sizeof(int), cudaMemcpyDeviceToHost, E.st));
  BCK(cudaStreamSynchronize(E.st));
  int rounds = 1;
  while (E.h_counts[1] > 0 && rounds <= o.max_halvings) {
    int rc = enqueue_ls_round(E, W, o);
    if (rc) return rc;
    BCK(cudaMemcpyAsync(E.h_counts, W.counts.p, 2 * sizeof(int), cudaMemcpyDeviceToHost, E.st));
    BCK(cudaStreamSynchronize(E.st));
    ++rounds;
  }
  const int np = W.count;
  theta_update_kernel<<<np, 256, 0, E.st>>>(dprobs(W), W.accepted(), W.active(), W.stop(), steptol, o.ftol,
                                            E.fp64 ? 0.0 : 1e-5);
  count_kernel<<<1, 256, 0, E.st>>>(np, W.active(), W.pending(), W.counts.as<int>());
  BCK(cudaGetLastError());
  BCK(cudaMemcpyAsync(E.h_counts, W.counts.p, 2 * sizeof(int), cudaMemcpyDeviceToHost, E.st));
  BCK(cudaMemcpyAsync(E.h_counts + 2, W.err.p, sizeof(int), cudaMemcpyDeviceToHost, E.st));
  BCK(cudaStreamSynchronize(E.st));
  if (E.h_counts[2]) return MNL_ERR_TIMEOUT;
  return MNL_OK;
}

// Time the grouped log-likelihood pass for a few tile heights (theta = 0).
int autotune_rows(Engine &E, WorkSet &W, const std::vector<const ProbLayout *> &L, double *theta0, int *rows_out) {
  std::string key = std::string(E.fp64 ? "f64" : "f32") + ":";
  {
    int64_t sN = 0, sK = 0, sq = 0;
    for (const ProbLayout *l : L) { sN += l->s.N; sK += l->s.K; sq += l->s.p + l->s.d + l->s.f; }
    key += std::to_string(L.size()) + "," + std::to_string(sN) + "," + std::to_string(sK) + "," + std::to_string(sq);
  }
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    tune_load();
    auto it = g_tune.find(key);
    if (it != g_tune.end()) { *rows_out = it->second; return MNL_OK; }
  }
  // a scratch copy of the descriptors with theta = delta = 0 and every problem pending
  std::vector<GroupProblem> saved = W.hp;
  for (size_t i = 0; i < W.hp.size(); ++i) { W.hp[i].theta = theta0; W.hp[i].delta = theta0; }
  static const int cands[] = {16, 32, 64};
  float best = 1e30f;
  int best_rows = 16;
  for (int rows : cands) {
    int rc = ws_build(E, W, L, rows);
    if (rc) continue;
    std::vector<int> ones(W.count, 1);
    BCK(cudaMemcpyAsync(W.pending(), ones.data(), ones.size() * sizeof(int), cudaMemcpyHostToDevice, E.st));
    for (const GroupProblem &g : W.hp) BCK(cudaMemsetAsync(g.scal, 0, kGsCount * sizeof(double), E.st));
    float ms = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
      BCK(cudaEventRecord(E.t0, E.st));
      BCK(launch_grouped_pass(W.pll, E.fp64, false, dprobs(W), W.segs.as<PassSeg>(), W.seg_start.as<int>(),
                              W.pending(), W.partials.as<double>(), E.st));
      BCK(cudaEventRecord(E.t1, E.st));
      BCK(cudaEventSynchronize(E.t1));
      float m = 0.f;
      cudaEventElapsedTime(&m, E.t0, E.t1);
      if (rep > 0) ms = std::min(ms, m);
    }
    if (ms < best) { best = ms; best_rows = rows; }
  }
  W.hp = saved;
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    tune_store(key, best_rows);
  }
  *rows_out = best_rows;
  return MNL_OK;
}

}  // namespace

// ===========================================================================
// Batched fits over a fixed set of problems (one CUDA graph per iteration).
// ===========================================================================

struct mnl_batch {
  Engine E;
  WorkSet W;
  std::vector<ProbLayout> layouts;
  std::vector<const ProbLayout *> lp;
  std::vector<int64_t> theta_off;
  int64_t theta_total = 0;
  unsigned char *arena = nullptr;
  double *theta0 = nullptr;
  cudaGraphExec_t graph = nullptr;
  bool have_graph = false;
  double graph_gtol = 0.0;
  int graph_halvings = 0;
  void release() {
    if (have_graph) cudaGraphExecDestroy(graph);
    W.release();
    if (arena) cudaFree(arena);
    if (theta0) cudaFree(theta0);
    E.release();
  }
};

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
  auto fail = [&](int rc) { b->release(); delete b; return rc; };
  int rc;
  if ((rc = b->E.init(precision, stream))) return fail(rc);
  Engine &E = b->E;
  size_t bytes = 0;
  std::vector<size_t> base(count);
  for (int i = 0; i < count; ++i) {
    b->layouts.push_back(layout_problem(dims[i], E.op, E.fp64, E.mixed, false));
    if (b->layouts.back().large) return fail(MNL_ERR_UNSUPPORTED);
    base[i] = bytes;
    bytes += b->layouts.back().bytes;
    b->theta_off.push_back(b->theta_total);
    b->theta_total += b->layouts.back().s.n;
  }
  for (const ProbLayout &l : b->layouts) b->lp.push_back(&l);
  if (cudaMalloc(&b->arena, bytes) != cudaSuccess || cudaMalloc(&b->theta0, b->theta_total * sizeof(double))) {
    cudaGetLastError();
    return fail(MNL_ERR_OOM);
  }
  if (cudaMemsetAsync(b->arena, 0, bytes, E.st) || cudaMemsetAsync(b->theta0, 0, b->theta_total * 8, E.st)) {
    cudaGetLastError();
    return fail(MNL_ERR_CUDA);
  }
  b->W.hp.resize(count);
  for (int i = 0; i < count; ++i) {
    const ProbLayout &l = b->layouts[i];
    bind_problem(l, b->arena + base[i], &data[i], b->theta0 + b->theta_off[i], b->W.hp[i]);
    if (!l.band_map.empty() && cudaMemcpyAsync(b->W.hp[i].band_of, l.band_map.data(), l.band_map.size() * sizeof(int),
                                               cudaMemcpyHostToDevice, E.st)) {
      cudaGetLastError();
      return fail(MNL_ERR_CUDA);
    }
  }
  int rows = 16;
  if ((rc = autotune_rows(E, b->W, b->lp, b->theta0, &rows))) return fail(rc);
  if ((rc = ws_build(E, b->W, b->lp, rows))) return fail(rc);
  if (cudaStreamSynchronize(E.st) != cudaSuccess) { cudaGetLastError(); return fail(MNL_ERR_CUDA); }
  *out = b;
  return MNL_OK;
}

int64_t mnl_batch_num_params(const mnl_batch *b, int64_t *offsets) {
  if (!b) return -1;
  if (offsets)
    for (size_t i = 0; i < b->theta_off.size(); ++i) offsets[i] = b->theta_off[i];
  return b->theta_total;
}

int mnl_batch_fit(mnl_batch *b, const mnl_fit_opts *opts, double *theta, mnl_batch_info *info) {
  if (!b || !theta) return MNL_ERR_INVALID_ARG;
  mnl_fit_opts o;
  mnl_fit_opts_default(&o);
  if (opts) o = *opts;
  if (o.maxiter < 0 || o.max_halvings < 0) return MNL_ERR_INVALID_ARG;
  Engine &E = b->E;
  WorkSet &W = b->W;
  const double steptol = o.steptol >= 0 ? o.steptol : (E.fp64 ? 1e-10 : 1e-7);
  const int np = W.count;
  const auto wall0 = std::chrono::steady_clock::now();
  BCK(cudaEventRecord(E.ev_user, E.user_st));
  BCK(cudaStreamWaitEvent(E.st, E.ev_user, 0));
  for (int i = 0; i < np; ++i) W.hp[i].theta = theta + b->theta_off[i];
  BCK(cudaMemcpyAsync(W.probs.p, W.hp.data(), (size_t)np * sizeof(GroupProblem), cudaMemcpyHostToDevice, E.st));
  std::vector<int> ones(np, 1);
  BCK(cudaMemcpyAsync(W.active(), ones.data(), (size_t)np * sizeof(int), cudaMemcpyHostToDevice, E.st));
  BCK(cudaMemsetAsync(W.pending(), 0, 4 * (size_t)np * sizeof(int), E.st));  // pending, accepted, status, stop
  BCK(cudaMemsetAsync(W.err.p, 0, sizeof(int), E.st));
  for (int i = 0; i < np; ++i) BCK(cudaMemsetAsync(W.hp[i].scal, 0, kGsCount * sizeof(double), E.st));
  BCK(cudaStreamSynchronize(E.st));
  if (b->have_graph && (b->graph_gtol != o.gtol || b->graph_halvings != o.max_halvings)) {
    cudaGraphExecDestroy(b->graph);
    b->have_graph = false;
  }
  if (!b->have_graph) {
    cudaGraph_t g;
    BCK(cudaStreamBeginCapture(E.st, cudaStreamCaptureModeThreadLocal));
    int rc1 = enqueue_iteration(E, W, o);
    int rc2 = rc1 == MNL_OK ? enqueue_ls_round(E, W, o) : rc1;
    cudaError_t ec = cudaStreamEndCapture(E.st, &g);
    if (rc2 != MNL_OK) return rc2;
    BCK(ec);
    BCK(cudaGraphInstantiate(&b->graph, g, 0));
    cudaGraphDestroy(g);
    b->have_graph = true;
    b->graph_gtol = o.gtol;
    b->graph_halvings = o.max_halvings;
  }
  int iters = 0;
  float t_graph = 0.f;
  for (int it = 0; it < o.maxiter; ++it) {
    BCK(cudaEventRecord(E.t0, E.st));
    BCK(cudaGraphLaunch(b->graph, E.st));
    BCK(cudaEventRecord(E.t1, E.st));
    int rc = finish_iteration(E, W, o, steptol);
    if (rc) return rc;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, E.t0, E.t1);
    t_graph += ms;
    ++iters;
    if (E.h_counts[0] == 0) break;
  }
  std::vector<int> st(np), sp(np);
  std::vector<double> sc((size_t)np * kGsCount);
  BCK(cudaMemcpyAsync(st.data(), W.status(), np * sizeof(int), cudaMemcpyDeviceToHost, E.st));
  BCK(cudaMemcpyAsync(sp.data(), W.stop(), np * sizeof(int), cudaMemcpyDeviceToHost, E.st));
  for (int i = 0; i < np; ++i)
    BCK(cudaMemcpyAsync(sc.data() + (size_t)i * kGsCount, W.hp[i].scal, kGsCount * sizeof(double),
                        cudaMemcpyDeviceToHost, E.st));
  BCK(cudaStreamSynchronize(E.st));
  BCK(cudaEventRecord(E.ev_done, E.st));
  BCK(cudaStreamWaitEvent(E.user_st, E.ev_done, 0));
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
    info->pass_rows = W.rows;
  }
  if (nconv == np) return MNL_OK;
  for (int i = 0; i < np; ++i)
    if (st[i] != MNL_OK) return st[i];
  return MNL_MAXITER;
}

int mnl_batch_destroy(mnl_batch *b) {
  if (!b) return MNL_OK;
  cudaStreamSynchronize(b->E.st);
  cudaGetLastError();
  b->release();
  delete b;
  return MNL_OK;
}

}  // extern "C"

// ===========================================================================
// Serving: continuous batching of fit requests under a device-memory budget.
// Each tick admits queued requests whose state fits in the remaining budget
// (FIFO; a request skipped too often blocks later ones so large requests are
// not starved), runs one Newton iteration for every admitted request in the
// same grouped launches, and retires the requests that finished.  A request's
// data, coefficients, P, gradient and Hessian stay resident in its chunk of
// the pool from admission to retirement.
// ===========================================================================

namespace {

struct Pool {
  unsigned char *base = nullptr;
  size_t size = 0, used = 0;
  std::map<size_t, size_t> free_;  // offset -> bytes
  int init(size_t bytes) {
    size = (bytes + 255) & ~(size_t)255;
    if (cudaMalloc(&base, size) != cudaSuccess) { cudaGetLastError(); base = nullptr; return MNL_ERR_OOM; }
    free_[0] = size;
    return MNL_OK;
  }
  bool alloc(size_t bytes, size_t *off) {
    bytes = (bytes + 255) & ~(size_t)255;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      *off = it->first;
      const size_t rem = it->second - bytes, o2 = it->first + bytes;
      free_.erase(it);
      if (rem) free_[o2] = rem;
      used += bytes;
      return true;
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = (bytes + 255) & ~(size_t)255;
    used -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  void destroy() { if (base) cudaFree(base); base = nullptr; }
};

struct Request {
  mnl_dims dims{};
  ProbLayout L;
  std::vector<float> X, Y, Z;
  std::vector<int32_t> choice;
  std::vector<double> theta0, theta_out;
  size_t off = 0;
  bool admitted = false, done = false;
  int skipped = 0;
  GroupProblem g{};
  mnl_request_result res{};
  std::chrono::steady_clock::time_point t_submit, t_admit;
};

}  // namespace

struct mnl_server {
  Engine E;
  WorkSet W;
  Pool pool;
  mnl_server_opts opts{};
  double steptol = 1e-7;
  uint64_t next_ticket = 1;
  std::deque<uint64_t> queue;
  std::vector<uint64_t> members;
  std::map<uint64_t, Request> reqs;
  std::vector<uint64_t> finished;  // retired, not yet reported by mnl_server_finished
  bool dirty = true;
  std::mutex mu;
  int ticks = 0;
  void release() {
    W.release();
    pool.destroy();
    E.release();
  }
};

// Members too large for the one-CTA solve: the multi-CTA mixed solve (float64
// Cholesky for MNL_FP64, or as the fallback), then their status code.
int solve_large_members(mnl_server *s, int np) {
  Engine &E = s->E;
  WorkSet &W = s->W;
  std::vector<int> large;
  for (int i = 0; i < np; ++i)
    if (s->reqs.at(s->members[i]).L.large) large.push_back(i);
  if (large.empty()) return MNL_OK;
  std::vector<int> act(np);
  BCK(cudaMemcpyAsync(act.data(), W.active(), np * sizeof(int), cudaMemcpyDeviceToHost, E.st));
  BCK(cudaStreamSynchronize(E.st));
  std::vector<int> flags(large.size(), 0);
  for (size_t j = 0; j < large.size(); ++j) {
    const int i = large[j];
    if (!act[i]) continue;
    Request &r = s->reqs.at(s->members[i]);
    unsigned char *base = s->pool.base + r.off;
    const int64_t n = r.L.s.n;
    int *sst = reinterpret_cast<int *>(base + r.L.sstat);
    int nl = 0;
    BCK(cudaMemsetAsync(sst, 0, sizeof(int), E.st));
    if (E.mixed) {
      void *mw = base + r.L.mwork;
      BCK(cudaMemsetAsync(mixed_solve_ref(mw, n), 0, 4 * 8, E.st));
      BCK(launch_mixed_solve(n, r.g.F, r.g.F32, r.g.grad, r.g.delta, mw, sst, W.err.as<int>(), 5, E.st, &nl));
    } else
      BCK(cudaMemsetAsync(sst, 0xff, sizeof(int), E.st));  // straight to the float64 path
    BCK(cudaMemcpyAsync(&flags[j], sst, sizeof(int), cudaMemcpyDeviceToHost, E.st));
  }
  BCK(cudaStreamSynchronize(E.st));
  for (size_t j = 0; j < large.size(); ++j) {
    const int i = large[j];
    if (!act[i]) continue;
    Request &r = s->reqs.at(s->members[i]);
    if (E.mixed && (flags[j] & (8 | 16 | 4)) == 0) continue;
    unsigned char *base = s->pool.base + r.off;
    int *sst = reinterpret_cast<int *>(base + r.L.sstat);
    double *dinv = reinterpret_cast<double *>(base + r.L.dinv);
    int nl = 0;
    BCK(cudaMemsetAsync(sst, 0, sizeof(int), E.st));
    BCK(launch_cholesky(r.L.s.n, r.g.F, dinv, base + r.L.cwork, sst, W.err.as<int>(), E.st));
    BCK(launch_cholesky_solve(r.L.s.n, r.g.F, dinv, r.g.grad, r.g.delta, sst, E.st, &nl));
    int st = 0;
    BCK(cudaMemcpyAsync(&st, sst, sizeof(int), cudaMemcpyDeviceToHost, E.st));
    BCK(cudaStreamSynchronize(E.st));
    if (st & 4) {
      const int code = MNL_ERR_NOT_PD;
      BCK(cudaMemcpy(W.status() + i, &code, sizeof(int), cudaMemcpyHostToDevice));
    }
  }
  return MNL_OK;
}

extern "C" {

void mnl_server_opts_default(mnl_server_opts *o) {
  if (!o) return;
  o->mem_budget = (size_t)80 << 30;
  o->precision = MNL_BF16;
  o->max_active = 4096;
  o->max_skips = 8;
  mnl_fit_opts_default(&o->fit);
}

int mnl_server_create(const mnl_server_opts *opts, void *stream, mnl_server **out) {
  if (!out) return MNL_ERR_INVALID_ARG;
  *out = nullptr;
  mnl_server_opts o;
  mnl_server_opts_default(&o);
  if (opts) o = *opts;
  if (o.precision < MNL_FP64 || o.precision > MNL_BF16 || o.mem_budget < ((size_t)1 << 20) || o.max_active < 1)
    return MNL_ERR_INVALID_ARG;
  mnl_server *s = new (std::nothrow) mnl_server();
  if (!s) return MNL_ERR_OOM;
  int rc;
  if ((rc = s->E.init(o.precision, stream)) || (rc = s->pool.init(o.mem_budget))) {
    s->release();
    delete s;
    return rc;
  }
  s->opts = o;
  s->steptol = o.fit.steptol >= 0 ? o.fit.steptol : (s->E.fp64 ? 1e-10 : 1e-7);
  *out = s;
  return MNL_OK;
}

int mnl_server_submit(mnl_server *s, const mnl_dims *dims, const mnl_data *host, const double *theta0,
                      uint64_t *ticket) {
  if (!s || !dims || !host || !ticket) return MNL_ERR_INVALID_ARG;
  const mnl_dims &d = *dims;
  if (d.N < 1 || d.K < 2 || d.p < 0 || d.d < 0 || d.f < 0 || d.p + d.d + d.f < 1) return MNL_ERR_INVALID_ARG;
  if (d.gamma_base != 0) return MNL_ERR_UNSUPPORTED;
  if (!host->choice || (d.p > 0 && !host->X) || (d.d > 0 && !host->Y) || (d.f > 0 && !host->Z))
    return MNL_ERR_INVALID_ARG;
  for (int64_t i = 0; i < d.N; ++i)
    if (host->choice[i] < 0 || host->choice[i] >= d.K) return MNL_ERR_INVALID_ARG;
  Request r;
  r.dims = d;
  r.L = layout_problem(d, s->E.op, s->E.fp64, s->E.mixed, true);
  if (r.L.s.K > 256 || r.L.s.nout > 16384) return MNL_ERR_UNSUPPORTED;
  if (r.L.bytes > s->pool.size) return MNL_ERR_OOM;
  r.X.assign(host->X, host->X + (size_t)d.N * d.p);
  if (d.d) r.Y.assign(host->Y, host->Y + (size_t)d.N * d.K * d.d);
  if (d.f) r.Z.assign(host->Z, host->Z + (size_t)d.N * d.K * d.f);
  r.choice.assign(host->choice, host->choice + d.N);
  r.theta0.assign((size_t)r.L.s.n, 0.0);
  if (theta0) std::copy(theta0, theta0 + r.L.s.n, r.theta0.begin());
  r.t_submit = std::chrono::steady_clock::now();
  std::lock_guard<std::mutex> lock(s->mu);
  const uint64_t t = s->next_ticket++;
  s->reqs.emplace(t, std::move(r));
  s->queue.push_back(t);
  *ticket = t;
  return MNL_OK;
}

int mnl_server_step(mnl_server *s, int32_t *n_active, int32_t *n_queued) {
  if (!s) return MNL_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(s->mu);
  Engine &E = s->E;
  WorkSet &W = s->W;
  // admission
  for (auto it = s->queue.begin(); it != s->queue.end();) {
    if ((int)s->members.size() >= s->opts.max_active) break;
    Request &r = s->reqs.at(*it);
    size_t off = 0;
    if (!s->pool.alloc(r.L.bytes, &off)) {
      if (++r.skipped > s->opts.max_skips) break;  // keep its place: later requests wait
      ++it;
      continue;
    }
    r.off = off;
    r.admitted = true;
    r.t_admit = std::chrono::steady_clock::now();
    unsigned char *base = s->pool.base + off;
    bind_problem(r.L, base, nullptr, nullptr, r.g);
    const Shape &sh = r.L.s;
    BCK(cudaMemsetAsync(base, 0, r.L.bytes, E.st));
    if (sh.p) BCK(cudaMemcpyAsync(base + r.L.X, r.X.data(), r.X.size() * 4, cudaMemcpyHostToDevice, E.st));
    if (sh.d) BCK(cudaMemcpyAsync(base + r.L.Y, r.Y.data(), r.Y.size() * 4, cudaMemcpyHostToDevice, E.st));
    if (sh.f) BCK(cudaMemcpyAsync(base + r.L.Z, r.Z.data(), r.Z.size() * 4, cudaMemcpyHostToDevice, E.st));
    BCK(cudaMemcpyAsync(base + r.L.choice, r.choice.data(), r.choice.size() * 4, cudaMemcpyHostToDevice, E.st));
    BCK(cudaMemcpyAsync(base + r.L.theta, r.theta0.data(), r.theta0.size() * 8, cudaMemcpyHostToDevice, E.st));
    if (!r.L.band_map.empty())
      BCK(cudaMemcpyAsync(r.g.band_of, r.L.band_map.data(), r.L.band_map.size() * sizeof(int),
                          cudaMemcpyHostToDevice, E.st));
    s->members.push_back(*it);
    s->dirty = true;
    it = s->queue.erase(it);
  }
  if (!s->members.empty()) {
    const int np = (int)s->members.size();
    if (s->dirty) {
      std::vector<const ProbLayout *> lp;
      W.hp.clear();
      for (uint64_t t : s->members) {
        Request &r = s->reqs.at(t);
        W.hp.push_back(r.g);
        lp.push_back(&r.L);
      }
      int rc = ws_build(E, W, lp, 16);
      if (rc) return rc;
      s->dirty = false;
    }
    std::vector<int> ones(np, 1);
    BCK(cudaMemcpyAsync(W.active(), ones.data(), (size_t)np * sizeof(int), cudaMemcpyHostToDevice, E.st));
    BCK(cudaMemsetAsync(W.pending(), 0, 4 * (size_t)np * sizeof(int), E.st));
    BCK(cudaMemsetAsync(W.err.p, 0, sizeof(int), E.st));
    int rc = enqueue_iteration(E, W, s->opts.fit, false);
    if (!rc) rc = solve_large_members(s, np);
    if (!rc) rc = enqueue_ls_init(E, W);
    if (!rc) rc = enqueue_ls_round(E, W, s->opts.fit);
    if (!rc) rc = finish_iteration(E, W, s->opts.fit, s->steptol);
    if (rc) return rc;
    ++s->ticks;
    // retire
    std::vector<int> st(np), sp(np);
    BCK(cudaMemcpyAsync(st.data(), W.status(), np * sizeof(int), cudaMemcpyDeviceToHost, E.st));
    BCK(cudaMemcpyAsync(sp.data(), W.stop(), np * sizeof(int), cudaMemcpyDeviceToHost, E.st));
    std::vector<double> sc((size_t)np * kGsCount);
    for (int i = 0; i < np; ++i)
      BCK(cudaMemcpyAsync(sc.data() + (size_t)i * kGsCount, W.hp[i].scal, kGsCount * 8, cudaMemcpyDeviceToHost, E.st));
    BCK(cudaStreamSynchronize(E.st));
    std::vector<uint64_t> keep;
    for (int i = 0; i < np; ++i) {
      Request &r = s->reqs.at(s->members[i]);
      const double *c = sc.data() + (size_t)i * kGsCount;
      const int iters = (int)c[kGsIters];
      const bool fin = st[i] != MNL_OK || sp[i] != 0 || iters >= s->opts.fit.maxiter;
      if (!fin) { keep.push_back(s->members[i]); continue; }
      r.theta_out.resize((size_t)r.L.s.n);
      BCK(cudaMemcpy(r.theta_out.data(), r.g.theta, r.theta_out.size() * 8, cudaMemcpyDeviceToHost));
      r.res.status = st[i] != MNL_OK ? st[i] : (sp[i] != 0 ? MNL_OK : MNL_MAXITER);
      r.res.stop_reason = sp[i] != 0 ? sp[i] : (st[i] == MNL_OK ? MNL_STOP_MAXITER : 0);
      r.res.iters = iters;
      r.res.ls_evals = (int)c[kGsLsEvals];
      r.res.loglik = c[kGsL];
      r.res.grad_inf = c[kGsGinf];
      const auto now = std::chrono::steady_clock::now();
      r.res.latency_ms = std::chrono::duration<double, std::milli>(now - r.t_submit).count();
      r.res.queue_ms = std::chrono::duration<double, std::milli>(r.t_admit - r.t_submit).count();
      r.done = true;
      s->finished.push_back(s->members[i]);
      s->pool.release(r.off, r.L.bytes);
      r.X.clear(); r.X.shrink_to_fit();
      r.Y.clear(); r.Y.shrink_to_fit();
      r.Z.clear(); r.Z.shrink_to_fit();
      r.choice.clear(); r.choice.shrink_to_fit();
      s->dirty = true;
    }
    s->members.swap(keep);
  }
  if (n_active) *n_active = (int32_t)s->members.size();
  if (n_queued) *n_queued = (int32_t)s->queue.size();
  return MNL_OK;
}

int mnl_server_poll(mnl_server *s, uint64_t ticket, double *theta, mnl_request_result *res) {
  if (!s) return MNL_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return MNL_ERR_INVALID_ARG;
  if (!it->second.done) return MNL_PENDING;
  if (theta) std::copy(it->second.theta_out.begin(), it->second.theta_out.end(), theta);
  if (res) *res = it->second.res;
  s->reqs.erase(it);
  return MNL_OK;
}

int mnl_server_finished(mnl_server *s, uint64_t *tickets, int32_t cap, int32_t *count) {
  if (!s || !count || cap < 0 || (cap > 0 && !tickets)) return MNL_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(s->mu);
  const int32_t k = (int32_t)std::min<size_t>((size_t)cap, s->finished.size());
  std::copy(s->finished.begin(), s->finished.begin() + k, tickets);
  s->finished.erase(s->finished.begin(), s->finished.begin() + k);
  *count = k;
  return MNL_OK;
}

size_t mnl_server_memory_in_use(const mnl_server *s) { return s ? s->pool.used : 0; }

int mnl_server_destroy(mnl_server *s) {
  if (!s) return MNL_OK;
  cudaStreamSynchronize(s->E.st);
  cudaGetLastError();
  s->release();
  delete s;
  return MNL_OK;
}

}  // extern "C"
