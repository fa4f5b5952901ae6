// C ABI of libmnl: handle lifetime, workspaces and the Newton-Raphson driver
// (Sec. 3.1 eq. "NR update" with step halving; stopping rules of Sec. 2.3).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <new>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "mnl_internal.cuh"

using namespace mnl;

struct mnl_handle {
  mnl_dims dims;  // as given (gamma_base 0 or 1)
  Shape S;        // of the problem the kernels solve (gamma_base = 1: f + d generic columns)
  int prec;
  OpType op;
  bool fp64;
  cudaStream_t st;
  int dev, nsm;
  // data
  const float *X, *Y, *Z;  // Z: the kernels' generic columns (Zaug when gamma_base = 1)
  const int32_t *choice;
  const float *Zu;         // the caller's Z
  const float *w;          // observation weights (device [N]) or nullptr
  // gamma_base = 1: augmented Z, theta permutation and internal-order vectors
  bool gb1;
  float *Zaug;
  int64_t *perm;
  double *th_int, *vec_int;
  bool owns_data, data_ready;
  void *owned[4];
  // pass
  PassPlan pfull, pll;
  double *part_full, *part_ll;
  void *P, *zbar;
  double *scal;    // device scalars
  double *grad, *delta, *tscale;
  int *status, *err;
  // Hessian
  int64_t ldn, mc_pad;
  int nt1d;
  void *At, *Ad;
  size_t op_bytes;
  TileLists tl;
  std::vector<int2> h_main, h_band;
  void *main_part, *band_part, *z_part;
  int main_split, band_split, z_split;
  CUtensorMap *maps;       // device: [0] At, [1] Ad, [2] Az (tensor-core modes)
  SyrkUnit *units_main, *units_band;
  int nunits_main, nunits_band, grid_main, grid_band;
  // Z blocks on the tensor cores (TF32 / BF16 with f > 0): operand Az, contracted tile pairs
  bool tcz;
  void *Az;
  ZopLayout zl;
  float *zt_part;
  int *zt_index;
  int zt_split, zt_npairs, zt_nt;
  SyrkUnit *units_z;
  int nunits_z, grid_z;
  double *F;
  // solve
  int solve_mode;  // MNL_SOLVE_FP64 or MNL_SOLVE_MIXED (resolved)
  double *dinv, *ref;  // ref points into mwork
  float *F32;
  void *mwork, *cwork;  // mixed-solve and float64-factor workspaces
  void *tcwork;         // tensor-core factorisation (n_theta >= the threshold)
  double *Binv;         // inverse of the float64 factor (standard errors; allocated at the first call)
  TcCholPlan tcp;
  uint64_t wait_ns;     // bound of the kernels' device waits (0: their defaults)
  // Hessian-free handle (truncated Newton): no Hessian, factor or solve workspaces
  bool hfree;
  int cg_max;           // conjugate-gradient iterations per Newton step at most
  double *cg;           // [3 n]: CG residual, direction, product (also scratch of mnl_hessian_vec)
  float *wbuf;          // [N][K] Hessian-vector residuals for the separate beta kernel (wide shapes)
  float *ux, *bf;       // wide shapes: X-block utilities [N][K] and float32 coefficients of their GEMM
  // coefficients of dropped data columns (mnl_drop_columns), in the kernels' order
  int nmask;
  int64_t *mask_idx;    // device [n_theta] (the first nmask entries are used)
  // host mirrors (pinned)
  double *h_scal;
  int *h_flags;
  cudaEvent_t ev[12];
  // host uploads (handles that own their data): chunks spread over several
  // copy streams, joined to st by events
  static constexpr int kUp = 4;
  cudaStream_t ust[kUp];
  cudaEvent_t uev[kUp + 1];
  bool up_ready;
  int launches;
  std::vector<void *> allocs;
};

namespace {

enum Scal { kL = 0, kLabs = 1, kGinf = 2, kLt = 4, kLtabs = 5, kStepInf = 6, kThetaInf = 7, kNscal = 16 };

#define CK(x)                                   \
  do {                                          \
    cudaError_t e_ = (x);                       \
    if (e_ != cudaSuccess) return cuda_fail(e_); \
  } while (0)

int cuda_fail(cudaError_t e) {
  if (e == cudaErrorMemoryAllocation) return MNL_ERR_OOM;
  if (e == cudaErrorNotSupported) return MNL_ERR_UNSUPPORTED;
  return MNL_ERR_CUDA;
}

int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

// n_theta from which the mixed solve factors on the tensor cores; the
// environment variable MNL_TC_CHOL_MIN_N (read when a handle is created)
// overrides it.
int64_t tc_chol_min_n() {
  const char *v = std::getenv("MNL_TC_CHOL_MIN_N");
  if (v && *v) {
    char *end = nullptr;
    const long long x = std::strtoll(v, &end, 10);
    if (end && *end == 0 && x > 0) return (int64_t)x;
  }
  return kTcCholMinN;
}

// Below this many observations MNL_BF16 forms the Hessian operands in TF32.
constexpr int64_t kBf16MinRows = 1024;
// Refinement steps of a mixed solve at most (each skipped once converged).
constexpr int kRefineIters = 5;   // refinement steps per round of launches
constexpr int kRefineMax = 30;    // refinement steps in all
// Relative step below which a non-shrinking step means the float32 noise floor.
constexpr double kNoiseStep = 1e-5;

bool dims_ok(const mnl_dims *d) {
  return d && d->N >= 1 && d->K >= 2 && d->p >= 0 && d->d >= 0 && d->f >= 0 && (d->p + d->d + d->f) >= 1 &&
         (d->gamma_base == 0 || d->gamma_base == 1);
}

struct Sizes {
  size_t P, zbar, part_full, part_ll, ops, main_part, band_part, z_part, F, owned, solve, zop, zt_part, ux;
  size_t total() const {
    return P + zbar + part_full + part_ll + ux + 2 * ops + main_part + band_part + z_part + F + owned + solve + zop +
           zt_part;
  }
};

void band_tiles(const Shape &S, int nt1d, std::vector<int2> &band, std::vector<int> &band_of) {
  band.clear();
  band_of.assign((size_t)nt1d * nt1d, -1);
  if (S.q == 0 || nt1d == 0) return;  // no class coefficients, no class blocks
  for (int k = 1; k < S.K; ++k) {
    const int64_t c0 = (int64_t)(k - 1) * S.q, c1 = (int64_t)k * S.q - 1;
    const int lo = (int)(c0 / kTile), hi = (int)(c1 / kTile);
    for (int ti = lo; ti <= hi; ++ti)
      for (int tj = lo; tj <= ti; ++tj)
        if (band_of[(size_t)ti * nt1d + tj] < 0) {
          band_of[(size_t)ti * nt1d + tj] = (int)band.size();
          band.push_back(make_int2(ti, tj));
        }
  }
}

int simt_split(int ntiles, int64_t nchunks, int nsm) {
  int s = (int)((2 * nsm + ntiles - 1) / ntiles);
  s = std::max(1, std::min<int>(s, (int)std::max<int64_t>(1, nchunks / 64)));
  return std::min(s, 64);
}

Sizes plan_sizes(const mnl_dims &d, int prec_in, bool owned, int nsm, int *main_split, int *band_split, int *z_split,
                 PassPlan *pf, PassPlan *pl, int64_t *ldn, int64_t *mc_pad, int *nt1d, int *nband, int *zt_split,
                 bool hfree = false) {
  const Shape S = make_shape(d);
  const int prec = (prec_in == MNL_BF16 && d.N < kBf16MinRows) ? MNL_TF32 : prec_in;
  const bool fp64 = prec == MNL_FP64;
  const size_t tsz = fp64 ? 8 : 4;
  const size_t esz = prec == MNL_FP64 ? 8 : prec == MNL_TF32 ? 4 : 2;
  Sizes z{};
  *pf = plan_pass(S, fp64, true, nsm);
  *pl = plan_pass(S, fp64, false, nsm);
  z.P = (size_t)S.N * S.K * tsz;
  z.zbar = (size_t)S.N * S.f * tsz;
  z.part_full = (size_t)pf->grid * (2 + S.n) * 8;
  z.part_ll = (size_t)pl->grid * 2 * 8;
  // wide shapes: utilities of the X block ([N][K] float32) and float32 coefficients ([p][ux_ldb(K)])
  z.ux = (pf->ux || pl->ux) ? (size_t)S.N * S.K * 4 + (size_t)S.p * ux_ldb(S.K) * 4 : 0;
  *ldn = round_up(S.N, 64);
  *mc_pad = round_up(S.mc, kTile);
  *nt1d = (int)(*mc_pad / kTile);
  z.ops = (size_t)(*mc_pad) * (*ldn) * esz;
  const int nmain = (*nt1d) * (*nt1d + 1) / 2;
  std::vector<int2> band;
  std::vector<int> band_of;
  band_tiles(S, *nt1d, band, band_of);
  *nband = (int)band.size();
  const size_t csz = fp64 ? 8 : 4;
  if (fp64) {
    *main_split = simt_split(nmain, *ldn / 16, nsm);
    *band_split = simt_split(*nband, *ldn / 16, nsm);
  } else {
    const int kb = tc_kblocks(prec == MNL_TF32 ? OpType::TF32 : OpType::BF16, *ldn);
    int nmain256 = 0;  // 256-wide main tiles (rows ti, columns tj, tj + 1 with tj even, tj <= ti)
    for (int ti = 0; ti < *nt1d; ++ti) nmain256 += ti / 2 + 1;
    *main_split = nmain ? tc_pick_split(nmain256, kb, nsm) : 1;
    *band_split = *nband ? tc_pick_split(*nband, kb, nsm) : 1;
  }
  z.main_part = (size_t)(*main_split) * nmain * kTile * kTile * csz;
  z.band_part = (size_t)(*band_split) * (*nband) * kTile * kTile * csz;
  const int64_t nzt = zblocks_outputs(S);
  *zt_split = 1;
  *z_split = 1;
  if (!fp64 && S.f > 0) {  // Z blocks on the tensor cores
    const OpType op = prec == MNL_TF32 ? OpType::TF32 : OpType::BF16;
    const ZopLayout L = zop_layout(S);
    const ZTiles zt = zop_tiles(S, L);
    *zt_split = tc_pick_split((int)zt.pairs.size(), tc_kblocks(op, *ldn), nsm);
    z.zop = (size_t)L.rows_pad * (*ldn) * esz;
    z.zt_part = (size_t)(*zt_split) * zt.pairs.size() * kTile * kTile * 4;
    z.z_part = 0;
  } else {
    // observation splits of the Z blocks: about 1024 observations each, at least four CTAs per SM,
    // at least 256 observations each, and at most 64 MB of partial sums
    const int64_t zparts = S.f ? zblocks_parts(S, fp64) : 1;
    int64_t zs = std::max<int64_t>((4 * nsm + zparts - 1) / zparts, S.N / 1024);
    zs = std::min<int64_t>(zs, std::max<int64_t>(1, ((int64_t)64 << 20) / std::max<int64_t>(1, nzt * (int64_t)tsz)));
    *z_split = (int)std::max<int64_t>(1, std::min<int64_t>(zs, S.N / 256));
    z.z_part = S.f ? (size_t)(*z_split) * nzt * tsz : 0;
  }
  z.F = (size_t)S.n * S.n * 8;
  // dinv (float64), F32 (float32), the mixed-solve and float64-factor workspaces
  z.solve = (size_t)S.n * 8 + (size_t)S.n * S.n * 4 + mixed_solve_bytes(S.n) + chol_work_bytes(S.n) +
            (S.n >= tc_chol_min_n() ? tc_chol_bytes(S.n) : 0);
  z.owned = owned ? ((size_t)S.N * S.p + (size_t)S.N * S.K * (S.d + S.f)) * 4 + (size_t)S.N * 4 : 0;
  if (hfree)  // truncated Newton: no Hessian operands, partials, F or factor workspaces; CG vectors instead
  {
    z.ops = z.main_part = z.band_part = z.z_part = z.zop = z.zt_part = z.F = 0;
    z.solve = (size_t)3 * S.n * 8;
  }
  return z;
}

template <typename T>
int dalloc(mnl_handle *h, T **p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) return MNL_OK;
  void *q = nullptr;
  cudaError_t e = cudaMalloc(&q, bytes);
  if (e != cudaSuccess) { cudaGetLastError(); return e == cudaErrorMemoryAllocation ? MNL_ERR_OOM : MNL_ERR_CUDA; }
  h->allocs.push_back(q);
  *p = reinterpret_cast<T *>(q);
  return MNL_OK;
}

void free_all(mnl_handle *h) {
  tc_chol_release(&h->tcp);
  for (void *p : h->allocs) cudaFree(p);
  h->allocs.clear();
  if (h->h_scal) cudaFreeHost(h->h_scal);
  if (h->h_flags) cudaFreeHost(h->h_flags);
  for (auto &e : h->ev) if (e) cudaEventDestroy(e);
  if (h->up_ready) {
    for (auto &s2 : h->ust) cudaStreamDestroy(s2);
    for (auto &e : h->uev) cudaEventDestroy(e);
    h->up_ready = false;
  }
  h->h_scal = nullptr;
  h->h_flags = nullptr;
}

int validate(mnl_handle *h) {
  CK(cudaMemsetAsync(h->status, 0, sizeof(int), h->st));
  const Shape U = shape_of(h->dims.N, h->dims.K, h->dims.p, h->dims.d, h->dims.f);  // the caller's arrays
  CK(launch_validate(U, h->X, h->Y, h->Zu, h->choice, h->status, h->st));
  if (h->gb1) CK(launch_augment_z(U.N, U.K, U.d, U.f, h->Y, h->Zu, h->Zaug, h->st));
  CK(cudaMemcpyAsync(h->h_flags, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  if (h->h_flags[0] & 1) return MNL_ERR_INVALID_ARG;
  if (h->h_flags[0] & 2) return MNL_ERR_NONFINITE;
  h->data_ready = true;
  return MNL_OK;
}

// l (and g, P, zbar when full) at theta (+ t delta when delta given) -> scal[base], scal[base+1], grad.
int run_pass(mnl_handle *h, const double *theta, bool full, const double *delta, int base) {
  PassIO io{};
  io.X = h->X; io.Y = h->Y; io.Z = h->Z; io.choice = h->choice;
  io.theta = theta; io.delta = delta; io.tscale = h->tscale;
  io.P = h->P; io.zbar = h->zbar;
  const PassPlan &pl = full ? h->pfull : h->pll;
  io.partials = full ? h->part_full : h->part_ll;
  io.err = h->err;
  io.wait_ns = h->wait_ns;
  io.w = h->w;
  io.ux = h->ux;
  io.bf = h->bf;
  CK(launch_pass(h->S, pl, h->fp64, full, io, h->st));
  CK(launch_pass_reduce(h->S, pl.grid, full, io.partials, h->scal + base, full ? h->grad : nullptr, h->st));
  h->launches += 2;
  return MNL_OK;
}

// Optional event between kernels (per-kernel timing of a step).
int mark(mnl_handle *h, cudaEvent_t *ev) {
  if (ev) CK(cudaEventRecord(*ev, h->st));
  return MNL_OK;
}

// F = -H from P, zbar (the last full pass).  ev: 4 events recorded after the
// operand build, the A^T A contraction, the diagonal class blocks and the Z blocks.
int run_hessian(mnl_handle *h, cudaEvent_t *ev = nullptr) {
  const Shape &S = h->S;
  const int nmain = (int)h->h_main.size();
  int rc;
  // class operands (and the Z-block operand's rows, from the same staged blocks)
  if (S.mc > 0 || h->tcz) {
    CK(launch_build_operands(S, h->op, h->X, h->Y, h->P, h->At, h->Ad, h->ldn, h->st, h->tcz ? h->Z : nullptr,
                             h->zbar, h->tcz ? h->Az : nullptr, h->w));
    h->launches += 1;
  }
  if ((rc = mark(h, ev ? ev + 0 : nullptr))) return rc;
  if (S.mc > 0) {
    if (h->fp64) {
      CK(launch_syrk_f64(reinterpret_cast<const double *>(h->At), h->ldn, S.N, h->tl.main, nmain, h->main_split,
                         reinterpret_cast<double *>(h->main_part), h->st));
      if ((rc = mark(h, ev ? ev + 1 : nullptr))) return rc;
      CK(launch_syrk_f64(reinterpret_cast<const double *>(h->Ad), h->ldn, S.N, h->tl.band, h->tl.nband,
                         h->band_split, reinterpret_cast<double *>(h->band_part), h->st));
    } else {
      CK(launch_syrk_tc(h->op, h->maps, h->units_main, h->nunits_main, nullptr, h->grid_main,
                        reinterpret_cast<float *>(h->main_part), h->err, h->st, 256, h->wait_ns));
      if ((rc = mark(h, ev ? ev + 1 : nullptr))) return rc;
      CK(launch_syrk_tc(h->op, h->maps, h->units_band, h->nunits_band, nullptr, h->grid_band,
                        reinterpret_cast<float *>(h->band_part), h->err, h->st, 128, h->wait_ns));
    }
    h->launches += 2;
  } else {
    if ((rc = mark(h, ev ? ev + 1 : nullptr))) return rc;
  }
  if ((rc = mark(h, ev ? ev + 2 : nullptr))) return rc;
  if (S.f > 0 && h->tcz) {
    CK(launch_syrk_tc(h->op, h->maps, h->units_z, h->nunits_z, nullptr, h->grid_z, h->zt_part, h->err, h->st, 128,
                      h->wait_ns));
    h->launches += 1;
  } else if (S.f > 0) {
    CK(launch_zblocks(S, h->fp64, h->X, h->Y, h->Z, h->P, h->zbar, h->z_split, h->z_part, h->st, h->w));
    h->launches += 1;
  }
  if ((rc = mark(h, ev ? ev + 3 : nullptr))) return rc;
  AssembleIO io{};
  io.main_part = h->main_part; io.main_split = h->main_split;
  io.band_part = h->band_part; io.band_split = h->band_split;
  io.z_part = h->z_part; io.z_split = h->z_split;
  io.tl = &h->tl;
  io.fp64 = h->fp64;
  io.f32 = h->solve_mode == MNL_SOLVE_MIXED ? h->F32 : nullptr;  // the mixed solve's input, written on the way
  if (h->tcz) {
    io.zt.part = h->zt_part;
    io.zt.split = h->zt_split;
    io.zt.npairs = h->zt_npairs;
    io.zt.nt = h->zt_nt;
    io.zt.index = h->zt_index;
    io.zt.oY = h->zl.oY;
    io.zt.oW = h->zl.oW;
    io.zt.oZ = h->zl.oZ;
  }
  CK(launch_assemble(S, io, nmain, h->F, h->st));
  h->launches += 1;
  return MNL_OK;
}

double noise_tol(const mnl_handle *h, double labs) {
  const double u = h->fp64 ? std::ldexp(1.0, -53) : std::ldexp(1.0, -24);
  return 8.0 * u * labs;
}

float elapsed(cudaEvent_t a, cudaEvent_t b) {
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) { cudaGetLastError(); return 0.f; }
  return ms;
}

// Per-phase device times of a step from its events.
void fill_times(mnl_handle *h, mnl_step_info &loc, float t_fallback) {
  loc.t_pass_ms = elapsed(h->ev[0], h->ev[1]);
  loc.t_hess_ms = elapsed(h->ev[1], h->ev[2]);
  loc.t_chol_ms = elapsed(h->ev[2], h->ev[3]) + t_fallback;
  loc.t_ls_ms = elapsed(h->ev[3], h->ev[4]);
  loc.t_build_ms = elapsed(h->ev[1], h->ev[5]);
  loc.t_syrk_ms = elapsed(h->ev[5], h->ev[6]);
  loc.t_band_ms = elapsed(h->ev[6], h->ev[7]);
  loc.t_zblk_ms = elapsed(h->ev[7], h->ev[8]);
  loc.t_asm_ms = elapsed(h->ev[8], h->ev[2]);
  loc.t_factor_ms = elapsed(h->ev[2], h->ev[9]);
  loc.t_solve_ms = elapsed(h->ev[9], h->ev[3]);
  loc.t_fallback_ms = t_fallback;
  loc.launches = h->launches;
}

// One Newton iteration.  With gtol > 0 the gradient is checked before the
// Hessian is formed; *converged is set and theta left unchanged if it is met.
int step_impl(mnl_handle *h, double *theta, mnl_step_info *info, double gtol, bool *converged, int max_halvings) {
  const int64_t n = h->S.n;
  mnl_step_info loc{};
  if (converged) *converged = false;
  h->launches = 0;
  CK(cudaMemsetAsync(h->status, 0, sizeof(int), h->st));
  CK(cudaMemsetAsync(h->err, 0, sizeof(int), h->st));
  CK(cudaMemsetAsync(h->scal, 0, kNscal * sizeof(double), h->st));
  CK(cudaMemsetAsync(h->ref, 0, 4 * sizeof(double), h->st));
  CK(cudaEventRecord(h->ev[0], h->st));
  int rc = run_pass(h, theta, true, nullptr, kL);
  if (rc) return rc;
  CK(launch_mask_vec(h->nmask, h->mask_idx, h->grad, 0.0, h->st));
  CK(launch_vec_absmax(n, h->grad, h->scal + kGinf, h->st));
  h->launches += 1;
  CK(cudaEventRecord(h->ev[1], h->st));
  if (gtol > 0) {
    CK(cudaMemcpyAsync(h->h_scal, h->scal, 4 * sizeof(double), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    if (!std::isfinite(h->h_scal[kL]) || !std::isfinite(h->h_scal[kGinf])) return MNL_ERR_NONFINITE;
    if (h->h_scal[kGinf] < gtol) {
      loc.loglik_old = loc.loglik_new = h->h_scal[kL];
      loc.grad_inf = h->h_scal[kGinf];
      loc.t_pass_ms = elapsed(h->ev[0], h->ev[1]);
      if (info) *info = loc;
      if (converged) *converged = true;
      return MNL_OK;
    }
  }
  rc = run_hessian(h, h->ev + 5);
  if (rc) return rc;
  const bool mixed = h->solve_mode == MNL_SOLVE_MIXED;
  CK(launch_mask_matrix(n, h->nmask, h->mask_idx, h->F, mixed ? h->F32 : nullptr, h->st));
  CK(cudaEventRecord(h->ev[2], h->st));
  int nl = 0;
  if (mixed && h->tcp.ready) {
    CK(launch_mixed_solve_tc(h->tcp, h->F, h->F32, h->grad, h->delta, h->mwork, h->status, h->err, kRefineIters,
                             h->wait_ns, h->st, &nl));
    h->launches += nl;
    CK(cudaEventRecord(h->ev[9], h->st));
  } else if (mixed) {
    CK(launch_mixed_solve(n, h->F, h->F32, h->grad, h->delta, h->mwork, h->status, h->err, kRefineIters, h->st,
                          &nl, true, h->wait_ns));
    h->launches += nl;
    CK(cudaEventRecord(h->ev[9], h->st));
  } else {
    CK(launch_cholesky(n, h->F, h->dinv, h->cwork, h->status, h->err, h->st, h->wait_ns));
    h->launches += cholesky_launches(n);
    CK(cudaEventRecord(h->ev[9], h->st));
    CK(launch_cholesky_solve(n, h->F, h->dinv, h->grad, h->delta, h->status, h->st, &nl));
    h->launches += nl;
  }
  CK(cudaEventRecord(h->ev[3], h->st));
  // The first trial of the step halving (t = 1) and, when it is acceptable, the
  // update of theta are enqueued behind the solve, so that the common case needs
  // one host round trip; otherwise theta is unchanged and the steps below decide.
  const double u8 = 8.0 * (h->fp64 ? std::ldexp(1.0, -53) : std::ldexp(1.0, -24));
  h->h_scal[8] = 1.0;
  CK(cudaMemcpyAsync(h->tscale, h->h_scal + 8, sizeof(double), cudaMemcpyHostToDevice, h->st));
  rc = run_pass(h, theta, false, h->delta, kLt);
  if (rc) return rc;
  CK(cudaEventRecord(h->ev[4], h->st));
  CK(launch_try_full_step(n, theta, h->delta, h->scal + kL, h->scal + kLabs, h->scal + kLt, h->status, h->err, u8,
                          h->scal + kStepInf, h->st));
  h->launches += 1;
  CK(cudaMemcpyAsync(h->h_scal, h->scal, 8 * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  CK(cudaMemcpyAsync(h->h_flags, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  CK(cudaMemcpyAsync(h->h_flags + 1, h->err, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  if (mixed) CK(cudaMemcpyAsync(h->h_scal + 12, h->ref, 4 * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  if (h->h_flags[1]) {
    loc.wait_errors = h->h_flags[1];
    if (info) *info = loc;
    return MNL_ERR_TIMEOUT;
  }
  const double l0 = h->h_scal[kL], labs = h->h_scal[kLabs], ginf = h->h_scal[kGinf];
  if (!std::isfinite(l0) || !std::isfinite(ginf)) return MNL_ERR_NONFINITE;
  loc.solve_mode = h->solve_mode;
  loc.factor_kind = (mixed && h->tcp.ready) ? MNL_FACTOR_TENSOR : MNL_FACTOR_COOP;
  if (mixed) loc.refine_steps = (int)h->h_scal[14];
  if (h->h_flags[0] & 32) {  // the full step was taken
    loc.loglik_old = l0;
    loc.loglik_new = h->h_scal[kLt];
    loc.grad_inf = ginf;
    loc.step_inf = h->h_scal[kStepInf];
    loc.theta_inf = h->h_scal[kThetaInf];
    loc.step_scale = 1.0;
    loc.ls_noise = noise_tol(h, labs);
    loc.halvings = 0;
    loc.ls_evals = 1;
    fill_times(h, loc, 0.f);
    if (info) *info = loc;
    return MNL_OK;
  }
  // A refinement that is still converging (ref[1] == 0) continues, 5 steps at a time, up to kRefineMax.
  for (int done = kRefineIters; mixed && (h->h_flags[0] & 16) && !(h->h_flags[0] & 8) && h->h_scal[13] == 0.0 &&
                                done < kRefineMax;
       done += kRefineIters) {
    const int clear = ~16;
    CK(launch_status_and(h->status, clear, h->st));
    CK(launch_mixed_refine(n, h->F, h->grad, h->delta, h->mwork, h->status, kRefineIters, h->st, &nl));
    h->launches += nl + 1;
    CK(cudaMemcpyAsync(h->h_flags, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->st));
    CK(cudaMemcpyAsync(h->h_scal + 12, h->ref, 4 * sizeof(double), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
  }
  if (mixed) loc.refine_steps = (int)h->h_scal[14];
  float t_fallback = 0.f;
  if (mixed && (h->h_flags[0] & (8 | 16))) {
    // float32 factor or refinement failed: float64 Cholesky of the intact F
    loc.fallback = 1;
    CK(cudaEventRecord(h->ev[10], h->st));
    CK(launch_cholesky(n, h->F, h->dinv, h->cwork, h->status, h->err, h->st, h->wait_ns));
    CK(launch_cholesky_solve(n, h->F, h->dinv, h->grad, h->delta, h->status, h->st, &nl));
    h->launches += cholesky_launches(n) + nl;
    CK(cudaEventRecord(h->ev[11], h->st));
    CK(cudaMemcpyAsync(h->h_flags, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->st));
    CK(cudaMemcpyAsync(h->h_flags + 1, h->err, sizeof(int), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    if (h->h_flags[1]) {
      loc.wait_errors = h->h_flags[1];
      if (info) *info = loc;
      return MNL_ERR_TIMEOUT;
    }
    t_fallback = elapsed(h->ev[10], h->ev[11]);
  }
  if (h->h_flags[0] & 4) return MNL_ERR_NOT_PD;
  const double tau = noise_tol(h, labs);
  // Step halving (Sec. 3.1).
  double t = 1.0, lt = 0.0;
  int j = 0, evals = 0;
  bool accepted = false;
  for (j = 0; j <= max_halvings; ++j) {
    h->h_scal[8] = t;
    CK(cudaMemcpyAsync(h->tscale, h->h_scal + 8, sizeof(double), cudaMemcpyHostToDevice, h->st));
    rc = run_pass(h, theta, false, h->delta, kLt);
    if (rc) return rc;
    CK(cudaMemcpyAsync(h->h_scal + kLt, h->scal + kLt, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    ++evals;
    lt = h->h_scal[kLt];
    if (std::isfinite(lt) && lt >= l0 - tau) { accepted = true; break; }
    t *= 0.5;
  }
  CK(cudaEventRecord(h->ev[4], h->st));
  if (!accepted) return MNL_ERR_LINESEARCH;
  CK(launch_axpy_theta(n, theta, h->delta, h->tscale, h->scal + kStepInf, h->st));
  h->launches += 1;
  CK(cudaMemcpyAsync(h->h_scal + kStepInf, h->scal + kStepInf, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  loc.loglik_old = l0;
  loc.loglik_new = lt;
  loc.grad_inf = ginf;
  loc.step_inf = h->h_scal[kStepInf];
  loc.theta_inf = h->h_scal[kThetaInf];
  loc.step_scale = t;
  loc.ls_noise = tau;
  loc.halvings = j;
  loc.ls_evals = evals;
  fill_times(h, loc, t_fallback);
  if (info) *info = loc;
  return MNL_OK;
}

// theta in the caller's order -> the order of the kernels (gamma_base = 1:
// gamma_0 after alpha), in h->th_int; the caller's pointer otherwise.
const double *theta_in(mnl_handle *h, const double *theta, int *rc) {
  *rc = MNL_OK;
  if (!h->gb1) return theta;
  const cudaError_t e = launch_perm_to_internal(h->S.n, h->perm, theta, h->th_int, h->st);
  if (e != cudaSuccess) *rc = cuda_fail(e);
  return h->th_int;
}

// F v = -H v at the theta of the last full pass (whose P it reuses), into out:
// the pass with v as its coefficients and the residuals P_ik (u_ik - ubar_i).
int hv_pass(mnl_handle *h, const double *v, double *out) {
  PassIO io{};
  io.X = h->X; io.Y = h->Y; io.Z = h->Z; io.choice = h->choice;
  io.theta = v;
  io.P = h->P; io.zbar = h->zbar;
  io.partials = h->part_full;
  io.err = h->err;
  io.wait_ns = h->wait_ns;
  io.w = h->w;
  io.Pin = h->P;
  io.Wout = h->wbuf;
  io.ux = h->ux;
  io.bf = h->bf;
  CK(launch_pass(h->S, h->pfull, h->fp64, true, io, h->st));
  CK(launch_pass_reduce(h->S, h->pfull.grid, true, io.partials, h->scal + 10, out, h->st));
  h->launches += 2;
  return MNL_OK;
}

// Truncated (inexact) Newton iteration (Sec. 3.1 eq. "NR update" with the
// Newton system solved only approximately): conjugate gradients on
// F delta = g with products F v from hv_pass (no Hessian is formed or stored),
// stopped when ||r|| <= eta ||g||, eta = min(0.1, sqrt(||g||)) (a forcing
// sequence that tends to 0 as g does, so convergence stays superlinear), then
// the same step halving as the exact step.
int step_truncated(mnl_handle *h, double *theta, mnl_step_info *info, double gtol, bool *converged,
                   int max_halvings) {
  const int64_t n = h->S.n;
  mnl_step_info loc{};
  if (converged) *converged = false;
  h->launches = 0;
  double *r = h->cg, *pv = h->cg + n, *ap = h->cg + 2 * n;
  CK(cudaMemsetAsync(h->err, 0, sizeof(int), h->st));
  CK(cudaMemsetAsync(h->scal, 0, kNscal * sizeof(double), h->st));
  CK(cudaEventRecord(h->ev[0], h->st));
  int rc = run_pass(h, theta, true, nullptr, kL);
  if (rc) return rc;
  CK(launch_mask_vec(h->nmask, h->mask_idx, h->grad, 0.0, h->st));
  CK(launch_vec_absmax(n, h->grad, h->scal + kGinf, h->st));
  CK(launch_dot(n, h->grad, h->grad, h->scal + 3, h->st));
  CK(cudaEventRecord(h->ev[1], h->st));
  CK(cudaMemcpyAsync(h->h_scal, h->scal, 4 * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  CK(cudaMemcpyAsync(h->h_flags + 1, h->err, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  if (h->h_flags[1]) { loc.wait_errors = h->h_flags[1]; if (info) *info = loc; return MNL_ERR_TIMEOUT; }
  const double l0 = h->h_scal[kL], labs = h->h_scal[kLabs], ginf = h->h_scal[kGinf], gg = h->h_scal[3];
  if (!std::isfinite(l0) || !std::isfinite(ginf)) return MNL_ERR_NONFINITE;
  loc.loglik_old = loc.loglik_new = l0;
  loc.grad_inf = ginf;
  loc.factor_kind = MNL_FACTOR_NONE;
  if (gtol > 0 && ginf < gtol) {
    if (converged) *converged = true;
    if (info) *info = loc;
    return MNL_OK;
  }
  // conjugate gradients, delta_0 = 0
  const double eta = std::min(0.1, std::sqrt(std::sqrt(gg)));
  const double target = eta * eta * gg;
  CK(cudaMemsetAsync(h->delta, 0, (size_t)n * 8, h->st));
  CK(cudaMemcpyAsync(r, h->grad, (size_t)n * 8, cudaMemcpyDeviceToDevice, h->st));
  CK(cudaMemcpyAsync(pv, h->grad, (size_t)n * 8, cudaMemcpyDeviceToDevice, h->st));
  double rs = gg;
  int it = 0;
  for (; it < h->cg_max && rs > target; ++it) {
    if ((rc = hv_pass(h, pv, ap))) return rc;
    CK(launch_mask_vec(h->nmask, h->mask_idx, ap, 0.0, h->st));  // CG stays in the free coefficients
    CK(launch_dot(n, pv, ap, h->scal + 13, h->st));
    CK(cudaMemcpyAsync(h->h_scal + 13, h->scal + 13, sizeof(double), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    const double pap = h->h_scal[13];
    if (!(pap > 0.0) || !std::isfinite(pap)) {
      if (it == 0) return MNL_ERR_NOT_PD;  // a direction of zero or negative curvature: -H is singular
      break;
    }
    const double alpha = rs / pap;
    CK(launch_axpby(n, alpha, pv, 1.0, h->delta, h->st));
    CK(launch_axpby(n, -alpha, ap, 1.0, r, h->st));
    CK(launch_dot(n, r, r, h->scal + 14, h->st));
    CK(cudaMemcpyAsync(h->h_scal + 14, h->scal + 14, sizeof(double), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    const double rs_new = h->h_scal[14];
    CK(launch_axpby(n, 1.0, r, rs_new / rs, pv, h->st));
    rs = rs_new;
    h->launches += 6;
  }
  CK(cudaEventRecord(h->ev[3], h->st));
  loc.cg_iters = it;
  // step halving (Sec. 3.1)
  const double tau = noise_tol(h, labs);
  double t = 1.0, lt = 0.0;
  int j = 0;
  bool accepted = false;
  for (j = 0; j <= max_halvings; ++j) {
    h->h_scal[8] = t;
    CK(cudaMemcpyAsync(h->tscale, h->h_scal + 8, sizeof(double), cudaMemcpyHostToDevice, h->st));
    if ((rc = run_pass(h, theta, false, h->delta, kLt))) return rc;
    CK(cudaMemcpyAsync(h->h_scal + kLt, h->scal + kLt, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->st));
    CK(cudaMemcpyAsync(h->h_flags + 1, h->err, sizeof(int), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    if (h->h_flags[1]) { loc.wait_errors = h->h_flags[1]; if (info) *info = loc; return MNL_ERR_TIMEOUT; }
    lt = h->h_scal[kLt];
    if (std::isfinite(lt) && lt >= l0 - tau) { accepted = true; break; }
    t *= 0.5;
  }
  CK(cudaEventRecord(h->ev[4], h->st));
  if (!accepted) return MNL_ERR_LINESEARCH;
  CK(launch_axpy_theta(n, theta, h->delta, h->tscale, h->scal + kStepInf, h->st));
  CK(cudaMemcpyAsync(h->h_scal + kStepInf, h->scal + kStepInf, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  loc.loglik_new = lt;
  loc.step_inf = h->h_scal[kStepInf];
  loc.theta_inf = h->h_scal[kThetaInf];
  loc.step_scale = t;
  loc.ls_noise = tau;
  loc.halvings = j;
  loc.ls_evals = j + 1;
  loc.t_pass_ms = elapsed(h->ev[0], h->ev[1]);
  loc.t_chol_ms = loc.t_solve_ms = elapsed(h->ev[1], h->ev[3]);
  loc.t_ls_ms = elapsed(h->ev[3], h->ev[4]);
  loc.launches = h->launches;
  if (info) *info = loc;
  return MNL_OK;
}

// (-H) delta = g from h->F (both triangles) and h->grad, synchronously, with the
// handle's solve mode: refinement continued while it converges, the float64
// factorisation when a mixed solve fails.  The sharded Newton step's solve.
int solve_system(mnl_handle *h, mnl_step_info &loc) {
  const int64_t n = h->S.n;
  int nl = 0;
  const bool mixed = h->solve_mode == MNL_SOLVE_MIXED;
  CK(cudaMemsetAsync(h->status, 0, sizeof(int), h->st));
  CK(cudaMemsetAsync(h->err, 0, sizeof(int), h->st));
  CK(cudaMemsetAsync(h->ref, 0, 4 * sizeof(double), h->st));
  if (mixed) {
    if (h->tcp.ready) {
      CK(launch_f64_to_f32_lower(n, h->F, h->F32, h->st));
      CK(launch_mixed_solve_tc(h->tcp, h->F, h->F32, h->grad, h->delta, h->mwork, h->status, h->err, kRefineIters,
                               h->wait_ns, h->st, &nl));
    } else {
      CK(launch_mixed_solve(n, h->F, h->F32, h->grad, h->delta, h->mwork, h->status, h->err, kRefineIters, h->st,
                            &nl, false, h->wait_ns));
    }
    loc.factor_kind = h->tcp.ready ? MNL_FACTOR_TENSOR : MNL_FACTOR_COOP;
    for (int done = 0;; done += kRefineIters) {
      CK(cudaMemcpyAsync(h->h_flags, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->st));
      CK(cudaMemcpyAsync(h->h_flags + 1, h->err, sizeof(int), cudaMemcpyDeviceToHost, h->st));
      CK(cudaMemcpyAsync(h->h_scal + 12, h->ref, 4 * sizeof(double), cudaMemcpyDeviceToHost, h->st));
      CK(cudaStreamSynchronize(h->st));
      if (h->h_flags[1]) { loc.wait_errors = h->h_flags[1]; return MNL_ERR_TIMEOUT; }
      const bool cont = (h->h_flags[0] & 16) && !(h->h_flags[0] & 8) && h->h_scal[13] == 0.0 &&
                        done + kRefineIters < kRefineMax;
      if (!cont) break;
      CK(launch_status_and(h->status, ~16, h->st));
      CK(launch_mixed_refine(n, h->F, h->grad, h->delta, h->mwork, h->status, kRefineIters, h->st, &nl));
    }
    loc.refine_steps = (int)h->h_scal[14];
    if (!(h->h_flags[0] & (8 | 16))) return MNL_OK;
    loc.fallback = 1;
    CK(cudaMemsetAsync(h->status, 0, sizeof(int), h->st));
  }
  CK(launch_cholesky(n, h->F, h->dinv, h->cwork, h->status, h->err, h->st, h->wait_ns));
  CK(launch_cholesky_solve(n, h->F, h->dinv, h->grad, h->delta, h->status, h->st, &nl));
  CK(cudaMemcpyAsync(h->h_flags, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  CK(cudaMemcpyAsync(h->h_flags + 1, h->err, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  if (h->h_flags[1]) { loc.wait_errors = h->h_flags[1]; return MNL_ERR_TIMEOUT; }
  if (!mixed) loc.factor_kind = MNL_FACTOR_COOP;
  return (h->h_flags[0] & 4) ? MNL_ERR_NOT_PD : MNL_OK;
}

int step_any(mnl_handle *h, double *theta, mnl_step_info *info, double gtol, bool *converged, int max_halvings) {
  return h->hfree ? step_truncated(h, theta, info, gtol, converged, max_halvings)
                  : step_impl(h, theta, info, gtol, converged, max_halvings);
}

int check_handle(const mnl_handle *h) {
  if (!h) return MNL_ERR_INVALID_ARG;
  if (!h->data_ready) return MNL_ERR_INVALID_ARG;
  return MNL_OK;
}

int set_device(const mnl_handle *h) {
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) { cudaGetLastError(); return MNL_ERR_CUDA; }
  if (cur != h->dev && cudaSetDevice(h->dev) != cudaSuccess) { cudaGetLastError(); return MNL_ERR_CUDA; }
  return MNL_OK;
}

}  // namespace

extern "C" {

int64_t mnl_num_params(const mnl_dims *d) {
  if (!dims_ok(d)) return -1;
  return (int64_t)(d->K - 1) * d->p + (int64_t)(d->gamma_base ? d->K : d->K - 1) * d->d + d->f;
}

const char *mnl_status_string(int s) {
  switch (s) {
    case MNL_OK: return "ok";
    case MNL_ERR_INVALID_ARG: return "invalid argument";
    case MNL_ERR_OOM: return "device allocation failed";
    case MNL_ERR_CUDA: return "CUDA error";
    case MNL_ERR_NOT_PD: return "negative Hessian not positive definite (singular design)";
    case MNL_ERR_NONFINITE: return "non-finite value in data, log-likelihood or gradient";
    case MNL_ERR_LINESEARCH: return "line search found no non-decreasing step";
    case MNL_MAXITER: return "maximum number of iterations reached";
    case MNL_ERR_TIMEOUT: return "a bounded device wait timed out";
    case MNL_ERR_UNSUPPORTED: return "unsupported configuration";
    case MNL_PENDING: return "request still pending";
    default: return "unknown status";
  }
}

void mnl_fit_opts_default(mnl_fit_opts *o) {
  if (!o) return;
  o->maxiter = 50;
  o->max_halvings = 30;
  o->gtol = 1e-8;
  o->ftol = 0.0;
  o->steptol = -1.0;
}

size_t mnl_workspace_bytes(const mnl_dims *d, int precision) {
  if (!dims_ok(d) || precision < 0 || precision > 2) return 0;
  int nsm = 148, dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  else cudaGetLastError();
  int ms, bs, zs, nt1d, nband;
  PassPlan pf, pl;
  int64_t ldn, mcp;
  int zts = 1;
  mnl_dims di = *d;  // gamma_base = 1: the equivalent problem with d more generic columns
  if (d->gamma_base == 1) { di.gamma_base = 0; di.f = d->f + d->d; }
  Sizes z = plan_sizes(di, precision, false, nsm, &ms, &bs, &zs, &pf, &pl, &ldn, &mcp, &nt1d, &nband, &zts);
  if (d->gamma_base == 1) z.owned += (size_t)d->N * d->K * di.f * 4 + 3 * (size_t)mnl_num_params(d) * 8;
  return z.total();
}

int mnl_create(const mnl_dims *dims, const mnl_data *data, int precision, void *stream, mnl_handle **out) {
  return mnl_create_ex(dims, data, precision, 0, stream, out);
}

int mnl_create_ex(const mnl_dims *dims, const mnl_data *data, int precision, int flags, void *stream,
                  mnl_handle **out) {
  if (!out) return MNL_ERR_INVALID_ARG;
  *out = nullptr;
  if (!dims_ok(dims) || precision < 0 || precision > 2 || (flags & ~MNL_CREATE_TRUNCATED)) return MNL_ERR_INVALID_ARG;
  const bool hfree = (flags & MNL_CREATE_TRUNCATED) != 0;
  if (dims->gamma_base == 1 && dims->d == 0) return MNL_ERR_INVALID_ARG;  // no gamma_0 to estimate
  // gamma_base = 1 is solved as gamma_base = 0 with the d columns of Y's base rows as generic columns
  mnl_dims di = *dims;
  if (dims->gamma_base == 1) { di.gamma_base = 0; di.f = dims->f + dims->d; }
  if (data) {
    if (!data->choice || (dims->p > 0 && !data->X) || (dims->d > 0 && !data->Y) || (dims->f > 0 && !data->Z))
      return MNL_ERR_INVALID_ARG;
  }
  mnl_handle *h = new (std::nothrow) mnl_handle();
  if (!h) return MNL_ERR_OOM;
  h->dims = *dims;
  h->S = make_shape(di);
  h->gb1 = dims->gamma_base == 1;
  h->prec = precision;
  h->op = precision == MNL_FP64 ? OpType::F64 : precision == MNL_TF32 ? OpType::TF32 : OpType::BF16;
  // Too few observations for unbiased BF16 rounding to average out: TF32 operands.
  if (h->op == OpType::BF16 && dims->N < kBf16MinRows) h->op = OpType::TF32;
  h->fp64 = precision == MNL_FP64;
  h->hfree = hfree;
  h->cg_max = 500;
  h->st = reinterpret_cast<cudaStream_t>(stream);
  int rc = MNL_OK;
  auto fail = [&](int code) {
    free_all(h);
    delete h;
    return code;
  };
  if (cudaGetDevice(&h->dev) != cudaSuccess) { cudaGetLastError(); return fail(MNL_ERR_CUDA); }
  cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, h->dev);
  int nband = 0;
  Sizes z = plan_sizes(di, precision, data == nullptr, h->nsm, &h->main_split, &h->band_split, &h->z_split,
                       &h->pfull, &h->pll, &h->ldn, &h->mc_pad, &h->nt1d, &nband, &h->zt_split, hfree);
  if (!h->pfull.ok || !h->pll.ok) return fail(MNL_ERR_UNSUPPORTED);

  for (auto &e : h->ev)
    if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return fail(MNL_ERR_CUDA); }
  if (cudaMallocHost(&h->h_scal, 32 * sizeof(double)) != cudaSuccess ||
      cudaMallocHost(&h->h_flags, 4 * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return fail(MNL_ERR_OOM);
  }
  const Shape &S = h->S;
  const size_t tsz = h->fp64 ? 8 : 4;
  if ((rc = dalloc(h, &h->P, z.P)) || (rc = dalloc(h, &h->zbar, z.zbar)) ||
      (rc = dalloc(h, &h->part_full, z.part_full)) || (rc = dalloc(h, &h->part_ll, z.part_ll)) ||
      (rc = dalloc(h, &h->scal, kNscal * sizeof(double))) || (rc = dalloc(h, &h->grad, S.n * 8)) ||
      (rc = dalloc(h, &h->delta, S.n * 8)) || (rc = dalloc(h, &h->tscale, 8)) ||
      (rc = dalloc(h, &h->status, 16)) || (rc = dalloc(h, &h->err, 16)) || (rc = dalloc(h, &h->At, z.ops)) ||
      (rc = dalloc(h, &h->Ad, z.ops)) || (rc = dalloc(h, &h->main_part, z.main_part)) ||
      (rc = dalloc(h, &h->band_part, z.band_part)) || (rc = dalloc(h, &h->z_part, z.z_part)) ||
      (rc = dalloc(h, &h->F, z.F)) || (rc = dalloc(h, &h->dinv, hfree ? 0 : S.n * 8)) ||
      (rc = dalloc(h, &h->F32, hfree ? 0 : (size_t)S.n * S.n * 4)) ||
      (rc = dalloc(h, &h->mwork, hfree ? 0 : mixed_solve_bytes(S.n))) ||
      (rc = dalloc(h, &h->cwork, hfree ? 0 : chol_work_bytes(S.n))) || (rc = dalloc(h, &h->cg, (size_t)3 * S.n * 8)))
    return fail(rc);
  // Hessian-vector residuals for the separate beta kernel of the wide tiled pass
  if (!h->fp64 && h->pfull.tiled && plan_pass_beta_ext(S) && (rc = dalloc(h, &h->wbuf, (size_t)S.N * S.K * 4)))
    return fail(rc);
  if ((h->pfull.ux || h->pll.ux) && ((rc = dalloc(h, &h->ux, (size_t)S.N * S.K * 4)) ||
                                     (rc = dalloc(h, &h->bf, (size_t)S.p * ux_ldb(S.K) * 4))))
    return fail(rc);
  h->ref = hfree ? nullptr : mixed_solve_ref(h->mwork, S.n);
  if (!hfree && S.n >= tc_chol_min_n()) {
    if ((rc = dalloc(h, &h->tcwork, tc_chol_bytes(S.n)))) return fail(rc);
    const cudaError_t e = tc_chol_prepare(S.n, h->tcwork, h->nsm, &h->tcp);
    if (e != cudaSuccess) { cudaGetLastError(); return fail(cuda_fail(e)); }
  }
  h->solve_mode = h->fp64 ? MNL_SOLVE_FP64 : MNL_SOLVE_MIXED;
  (void)tsz;
  h->op_bytes = z.ops;
  if (z.ops) {
    if (cudaMemsetAsync(h->At, 0, z.ops, h->st) != cudaSuccess || cudaMemsetAsync(h->Ad, 0, z.ops, h->st) != cudaSuccess) {
      cudaGetLastError();
      return fail(MNL_ERR_CUDA);
    }
  }
  // tile lists
  for (int ti = 0; ti < h->nt1d; ++ti)
    for (int tj = 0; tj <= ti; ++tj) h->h_main.push_back(make_int2(ti, tj));
  std::vector<int> band_of;
  band_tiles(S, h->nt1d, h->h_band, band_of);
  h->tl.nmain = (int)h->h_main.size();
  h->tl.nband = (int)h->h_band.size();
  if ((rc = dalloc(h, &h->tl.main, h->h_main.size() * sizeof(int2))) ||
      (rc = dalloc(h, &h->tl.band, h->h_band.size() * sizeof(int2))) ||
      (rc = dalloc(h, &h->tl.band_of, band_of.size() * sizeof(int))))
    return fail(rc);
  if ((!h->h_main.empty() && cudaMemcpy(h->tl.main, h->h_main.data(), h->h_main.size() * sizeof(int2),
                                        cudaMemcpyHostToDevice) != cudaSuccess) ||
      (!h->h_band.empty() && cudaMemcpy(h->tl.band, h->h_band.data(), h->h_band.size() * sizeof(int2),
                                        cudaMemcpyHostToDevice) != cudaSuccess) ||
      (!band_of.empty() &&
       cudaMemcpy(h->tl.band_of, band_of.data(), band_of.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)) {
    cudaGetLastError();
    return fail(MNL_ERR_CUDA);
  }
  h->tcz = !h->fp64 && S.f > 0 && !hfree;
  if (!h->fp64 && !hfree && (S.mc > 0 || h->tcz)) {
    CUtensorMap hm[3];
    std::memset(hm, 0, sizeof(hm));
    cudaError_t e = cudaSuccess;
    if (S.mc > 0) {
      e = encode_operand_map(h->op, h->At, h->mc_pad, h->ldn, &hm[0]);
      if (e == cudaSuccess) e = encode_operand_map(h->op, h->Ad, h->mc_pad, h->ldn, &hm[1]);
    }
    ZTiles zt;
    if (e == cudaSuccess && h->tcz) {
      h->zl = zop_layout(S);
      zt = zop_tiles(S, h->zl);
      h->zt_npairs = (int)zt.pairs.size();
      h->zt_nt = zt.nt;
      const size_t zbytes = (size_t)h->zl.rows_pad * h->ldn * (h->op == OpType::TF32 ? 4 : 2);
      if ((rc = dalloc(h, &h->Az, zbytes)) ||
          (rc = dalloc(h, &h->zt_part, (size_t)h->zt_split * zt.pairs.size() * kTile * kTile * 4)) ||
          (rc = dalloc(h, &h->zt_index, zt.index.size() * sizeof(int))))
        return fail(rc);
      if (cudaMemsetAsync(h->Az, 0, zbytes, h->st) != cudaSuccess ||
          cudaMemcpy(h->zt_index, zt.index.data(), zt.index.size() * sizeof(int), cudaMemcpyHostToDevice) !=
              cudaSuccess) {
        cudaGetLastError();
        return fail(MNL_ERR_CUDA);
      }
      e = encode_operand_map(h->op, h->Az, h->zl.rows_pad, h->ldn, &hm[2]);
    }
    if (e != cudaSuccess) return fail(cuda_fail(e));
    // Units: split-major, so CTAs running at the same time read the same observation range (L2 reuse).
    const int kb = tc_kblocks(h->op, h->ldn);
    auto make_units = [&](const std::vector<int2> &tiles, int nsplit, int map) {
      std::vector<SyrkUnit> u;
      for (int sp = 0; sp < nsplit; ++sp)
        for (size_t t = 0; t < tiles.size(); ++t) {
          SyrkUnit w;
          w.map = map; w.problem = 0; w.ti = tiles[t].x; w.tj = tiles[t].y;
          w.kb0 = (int)((int64_t)kb * sp / nsplit);
          w.kb1 = (int)((int64_t)kb * (sp + 1) / nsplit);
          w.out_off = ((int64_t)sp * (int64_t)tiles.size() + (int64_t)t) * kTile * kTile;
          w.flags = 0;
          w.out_off2 = -1;
          u.push_back(w);
        }
      return u;
    };
    // main contraction with 256-wide tiles: B = tiles (2c, 2c + 1), the second half stored when below the diagonal
    auto make_main_units = [&](int nsplit) {
      std::vector<SyrkUnit> u;
      const int64_t nmain = (int64_t)h->h_main.size();
      auto slot = [](int ti, int tj) { return (int64_t)ti * (ti + 1) / 2 + tj; };
      // Tiles in square blocks of kSuper x kSuper (block rows I >= block columns J, J fastest): the
      // persistent CTAs take consecutive jobs at the same time and walk the observations in step, so
      // a block keeps the operand rows read at once to 2 kSuper tile rows instead of a whole band of
      // the triangle (which does not fit in L2 when there are many tile rows).
      constexpr int kSuper = 16;
      const int nsb = (h->nt1d + kSuper - 1) / kSuper;
      for (int sp = 0; sp < nsplit; ++sp)
        for (int I = 0; I < nsb; ++I)
          for (int J = 0; J <= I; ++J)
            for (int ti = I * kSuper; ti < std::min(h->nt1d, (I + 1) * kSuper); ++ti)
              for (int tj = J * kSuper; tj <= std::min(ti, (J + 1) * kSuper - 1); tj += 2) {
                SyrkUnit w;
                w.map = 0; w.problem = 0; w.ti = ti; w.tj = tj;
                w.kb0 = (int)((int64_t)kb * sp / nsplit);
                w.kb1 = (int)((int64_t)kb * (sp + 1) / nsplit);
                w.out_off = ((int64_t)sp * nmain + slot(ti, tj)) * kTile * kTile;
                w.out_off2 = tj + 1 <= ti ? ((int64_t)sp * nmain + slot(ti, tj + 1)) * kTile * kTile : -1;
                w.flags = 0;
                u.push_back(w);
              }
      return u;
    };
    const std::vector<SyrkUnit> jm = S.mc > 0 ? make_main_units(h->main_split) : std::vector<SyrkUnit>();
    const std::vector<SyrkUnit> jb = S.mc > 0 ? make_units(h->h_band, h->band_split, 1) : std::vector<SyrkUnit>();
    const std::vector<SyrkUnit> jz = h->tcz ? make_units(zt.pairs, h->zt_split, 2) : std::vector<SyrkUnit>();
    h->grid_main = std::min((int)jm.size(), h->nsm);
    h->grid_band = std::min((int)jb.size(), h->nsm);
    h->grid_z = std::min((int)jz.size(), h->nsm);
    const std::vector<SyrkUnit> um = schedule_syrk_units(jm, h->grid_main, tc_chunk_kblocks(h->op));
    const std::vector<SyrkUnit> ub = schedule_syrk_units(jb, h->grid_band, tc_chunk_kblocks(h->op));
    const std::vector<SyrkUnit> uz = schedule_syrk_units(jz, h->grid_z, tc_chunk_kblocks(h->op));
    h->nunits_main = (int)um.size();
    h->nunits_band = (int)ub.size();
    h->nunits_z = (int)uz.size();
    if ((rc = dalloc(h, &h->maps, sizeof(hm))) || (rc = dalloc(h, &h->units_main, um.size() * sizeof(SyrkUnit))) ||
        (rc = dalloc(h, &h->units_band, ub.size() * sizeof(SyrkUnit))) ||
        (rc = dalloc(h, &h->units_z, uz.size() * sizeof(SyrkUnit))))
      return fail(rc);
    auto up = [&](SyrkUnit *dst, const std::vector<SyrkUnit> &v) {
      return v.empty() || cudaMemcpy(dst, v.data(), v.size() * sizeof(SyrkUnit), cudaMemcpyHostToDevice) == cudaSuccess;
    };
    if (cudaMemcpy(h->maps, hm, sizeof(hm), cudaMemcpyHostToDevice) != cudaSuccess || !up(h->units_main, um) ||
        !up(h->units_band, ub) || !up(h->units_z, uz)) {
      cudaGetLastError();
      return fail(MNL_ERR_CUDA);
    }
  }
  if (h->gb1) {  // augmented Z, theta permutation (user order <-> kernels' order), internal-order vectors
    const int64_t nb = (int64_t)(S.K - 1) * S.p, dd = dims->d, nn = S.n;
    std::vector<int64_t> perm((size_t)nn);
    for (int64_t u = 0; u < nn; ++u)
      perm[(size_t)u] = u < nb ? u : u < nb + dd ? nn - dd + (u - nb) : u - dd;
    if ((rc = dalloc(h, &h->Zaug, (size_t)S.N * S.K * S.f * 4)) || (rc = dalloc(h, &h->perm, (size_t)nn * 8)) ||
        (rc = dalloc(h, &h->th_int, (size_t)nn * 8)) || (rc = dalloc(h, &h->vec_int, (size_t)nn * 8)))
      return fail(rc);
    if (cudaMemcpy(h->perm, perm.data(), (size_t)nn * 8, cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaGetLastError();
      return fail(MNL_ERR_CUDA);
    }
  }
  // data (the caller's shapes: Z has dims->f columns)
  if (data) {
    h->X = data->X; h->Y = data->Y; h->Zu = data->Z; h->choice = data->choice;
    h->Z = h->gb1 ? h->Zaug : h->Zu;
    h->owns_data = false;
    if ((rc = validate(h))) return fail(rc);
  } else {
    h->owns_data = true;
    float *X = nullptr, *Y = nullptr, *Z = nullptr;
    int32_t *c = nullptr;
    if ((rc = dalloc(h, &X, (size_t)S.N * S.p * 4)) || (rc = dalloc(h, &Y, (size_t)S.N * S.K * S.d * 4)) ||
        (rc = dalloc(h, &Z, (size_t)S.N * S.K * dims->f * 4)) || (rc = dalloc(h, &c, (size_t)S.N * 4)))
      return fail(rc);
    h->X = X; h->Y = Y; h->Zu = Z; h->choice = c;
    h->Z = h->gb1 ? h->Zaug : h->Zu;
    h->data_ready = false;
  }
  if (cudaStreamSynchronize(h->st) != cudaSuccess) { cudaGetLastError(); return fail(MNL_ERR_CUDA); }
  *out = h;
  return MNL_OK;
}

int mnl_upload(mnl_handle *h, const mnl_data *hd) {
  if (!h || !hd || !h->owns_data) return MNL_ERR_INVALID_ARG;
  const Shape &S = h->S;
  if (!hd->choice || (S.p > 0 && !hd->X) || (S.d > 0 && !hd->Y) || (h->dims.f > 0 && !hd->Z))
    return MNL_ERR_INVALID_ARG;
  int rc = set_device(h);
  if (rc) return rc;
  if (!h->up_ready) {
    for (auto &s2 : h->ust) CK(cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking));
    for (auto &e : h->uev) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    h->up_ready = true;
  }
  // The copies start after the work already queued on st (which may still
  // read the previous data) and st waits for all of them.  Chunks of 32 MiB
  // are dealt to the copy streams in turn, so several copy engines run.
  CK(cudaEventRecord(h->uev[mnl_handle::kUp], h->st));
  for (auto &s2 : h->ust) CK(cudaStreamWaitEvent(s2, h->uev[mnl_handle::kUp], 0));
  constexpr size_t kChunk = (size_t)32 << 20;
  int next = 0;
  auto copy = [&](void *dst, const void *src, size_t bytes) -> cudaError_t {
    for (size_t o = 0; o < bytes; o += kChunk) {
      const size_t b = bytes - o < kChunk ? bytes - o : kChunk;
      const cudaError_t e = cudaMemcpyAsync(static_cast<char *>(dst) + o, static_cast<const char *>(src) + o, b,
                                            cudaMemcpyHostToDevice, h->ust[next]);
      if (e != cudaSuccess) return e;
      next = (next + 1) % mnl_handle::kUp;
    }
    return cudaSuccess;
  };
  if (S.p) CK(copy(const_cast<float *>(h->X), hd->X, (size_t)S.N * S.p * 4));
  if (S.d) CK(copy(const_cast<float *>(h->Y), hd->Y, (size_t)S.N * S.K * S.d * 4));
  if (h->dims.f) CK(copy(const_cast<float *>(h->Zu), hd->Z, (size_t)S.N * S.K * h->dims.f * 4));
  CK(copy(const_cast<int32_t *>(h->choice), hd->choice, (size_t)S.N * 4));
  for (int i = 0; i < mnl_handle::kUp; ++i) {
    CK(cudaEventRecord(h->uev[i], h->ust[i]));
    CK(cudaStreamWaitEvent(h->st, h->uev[i], 0));
  }
  return validate(h);
}

int mnl_loglik_grad(mnl_handle *h, const double *theta, double *loglik, double *grad) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!theta) return MNL_ERR_INVALID_ARG;
  if ((rc = set_device(h))) return rc;
  CK(cudaMemsetAsync(h->err, 0, sizeof(int), h->st));
  const double *th = theta_in(h, theta, &rc);
  if (rc) return rc;
  rc = run_pass(h, th, grad != nullptr, nullptr, kL);
  if (rc) return rc;
  if (grad && h->gb1) CK(launch_perm_to_user(h->S.n, h->perm, h->grad, grad, h->st));
  else if (grad) CK(cudaMemcpyAsync(grad, h->grad, h->S.n * 8, cudaMemcpyDeviceToDevice, h->st));
  if (loglik) {
    CK(cudaMemcpyAsync(h->h_scal, h->scal, sizeof(double), cudaMemcpyDeviceToHost, h->st));
    CK(cudaMemcpyAsync(h->h_flags + 1, h->err, sizeof(int), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    if (h->h_flags[1]) return MNL_ERR_TIMEOUT;
    *loglik = h->h_scal[0];
  }
  return MNL_OK;
}

int mnl_hessian(mnl_handle *h, const double *theta, double *H) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!theta || !H) return MNL_ERR_INVALID_ARG;
  if (h->hfree) return MNL_ERR_UNSUPPORTED;
  if ((rc = set_device(h))) return rc;
  CK(cudaMemsetAsync(h->err, 0, sizeof(int), h->st));
  const double *th = theta_in(h, theta, &rc);
  if (rc) return rc;
  if ((rc = run_pass(h, th, true, nullptr, kL))) return rc;
  if ((rc = run_hessian(h))) return rc;
  if (h->gb1) CK(launch_export_hessian_perm(h->S.n, h->F, h->perm, H, h->st));
  else CK(launch_export_hessian(h->S.n, h->F, H, h->st));
  return MNL_OK;
}

int mnl_newton_step(mnl_handle *h, double *theta, mnl_step_info *info) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!theta) return MNL_ERR_INVALID_ARG;
  if ((rc = set_device(h))) return rc;
  if (!h->gb1) return step_any(h, theta, info, 0.0, nullptr, 30);
  double *th = const_cast<double *>(theta_in(h, theta, &rc));
  if (rc) return rc;
  rc = step_any(h, th, info, 0.0, nullptr, 30);
  if (rc == MNL_OK) CK(launch_perm_to_user(h->S.n, h->perm, th, theta, h->st));
  if (rc == MNL_OK) CK(cudaStreamSynchronize(h->st));
  return rc;
}

int mnl_fit(mnl_handle *h, const mnl_fit_opts *opts, double *theta, mnl_fit_info *info) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!theta) return MNL_ERR_INVALID_ARG;
  if ((rc = set_device(h))) return rc;
  mnl_fit_opts o;
  mnl_fit_opts_default(&o);
  if (opts) o = *opts;
  if (o.maxiter < 0 || o.max_halvings < 0) return MNL_ERR_INVALID_ARG;
  const double steptol = o.steptol >= 0 ? o.steptol : (h->fp64 ? 1e-10 : 1e-7);
  double *const theta_user = theta;
  theta = const_cast<double *>(theta_in(h, theta_user, &rc));  // gamma_base = 1: the kernels' order
  if (rc) return rc;
  mnl_fit_info fi{};
  const auto t0 = std::chrono::steady_clock::now();
  rc = MNL_MAXITER;
  double prev_step_rel = 1e300;
  for (int it = 0; it < o.maxiter; ++it) {
    mnl_step_info si{};
    bool conv = false;
    int s = step_any(h, theta, &si, o.gtol, &conv, o.max_halvings);
    fi.t_pass_ms += si.t_pass_ms;
    fi.t_hess_ms += si.t_hess_ms;
    fi.t_chol_ms += si.t_chol_ms;
    fi.t_ls_ms += si.t_ls_ms;
    if (s != MNL_OK) { rc = s; break; }
    fi.grad_inf = si.grad_inf;
    if (conv) {
      fi.loglik = si.loglik_old;
      fi.stop_reason = MNL_STOP_GTOL;
      rc = MNL_OK;
      break;
    }
    fi.iters = it + 1;
    fi.ls_evals += si.ls_evals;
    fi.loglik = si.loglik_new;
    fi.dloglik = si.loglik_new - si.loglik_old;
    fi.step_rel = si.step_inf / std::max(1.0, si.theta_inf);
    if (o.ftol > 0 && std::fabs(fi.dloglik) < o.ftol) { fi.stop_reason = MNL_STOP_FTOL; rc = MNL_OK; break; }
    if (steptol > 0 && fi.step_rel <= steptol) { fi.stop_reason = MNL_STOP_STEPTOL; rc = MNL_OK; break; }
    if (!h->fp64 && it > 0 && fi.step_rel > 0.5 * prev_step_rel && fi.step_rel <= kNoiseStep) {
      fi.stop_reason = MNL_STOP_NOISE;
      rc = MNL_OK;
      break;
    }
    prev_step_rel = fi.step_rel;
  }
  if (rc == MNL_MAXITER) fi.stop_reason = MNL_STOP_MAXITER;
  if (h->gb1) {
    CK(launch_perm_to_user(h->S.n, h->perm, theta, theta_user, h->st));
    CK(cudaStreamSynchronize(h->st));
  }
  fi.status = rc;
  fi.t_total_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (info) *info = fi;
  return rc;
}

int mnl_hessian_vec(mnl_handle *h, const double *theta, const double *v, double *Hv) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!theta || !v || !Hv) return MNL_ERR_INVALID_ARG;
  if ((rc = set_device(h))) return rc;
  const int64_t n = h->S.n;
  CK(cudaMemsetAsync(h->err, 0, sizeof(int), h->st));
  const double *th = theta_in(h, theta, &rc);
  if (rc) return rc;
  if ((rc = run_pass(h, th, true, nullptr, kL))) return rc;  // P at theta
  const double *vi = v;
  if (h->gb1) {
    CK(launch_perm_to_internal(n, h->perm, v, h->cg, h->st));
    vi = h->cg;
  }
  if ((rc = hv_pass(h, vi, h->cg + n))) return rc;
  if (h->gb1) {
    CK(launch_axpby(n, -1.0, h->cg + n, 0.0, h->cg + 2 * n, h->st));  // H v = -(F v)
    CK(launch_perm_to_user(n, h->perm, h->cg + 2 * n, Hv, h->st));
  } else {
    CK(launch_axpby(n, -1.0, h->cg + n, 0.0, Hv, h->st));
  }
  CK(cudaMemcpyAsync(h->h_flags + 1, h->err, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  return h->h_flags[1] ? MNL_ERR_TIMEOUT : MNL_OK;
}

int mnl_set_cg_max(mnl_handle *h, int32_t iters) {
  if (!h || iters < 1) return MNL_ERR_INVALID_ARG;
  h->cg_max = iters;
  return MNL_OK;
}

int mnl_std_errors(mnl_handle *h, const double *theta, double *se) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!theta || !se) return MNL_ERR_INVALID_ARG;
  if (h->hfree) return MNL_ERR_UNSUPPORTED;
  if ((rc = set_device(h))) return rc;
  const int64_t n = h->S.n;
  if (!h->Binv && (rc = dalloc(h, &h->Binv, (size_t)n * n * 8))) return rc;
  CK(cudaMemsetAsync(h->status, 0, sizeof(int), h->st));
  CK(cudaMemsetAsync(h->err, 0, sizeof(int), h->st));
  const double *th = theta_in(h, theta, &rc);
  if (rc) return rc;
  if ((rc = run_pass(h, th, true, nullptr, kL))) return rc;
  if ((rc = run_hessian(h))) return rc;
  CK(launch_mask_matrix(n, h->nmask, h->mask_idx, h->F, nullptr, h->st));
  CK(launch_std_errors(n, h->F, h->Binv, h->dinv, h->cwork, h->status, h->err, h->gb1 ? h->vec_int : se, h->st,
                       h->wait_ns));
  CK(launch_mask_vec(h->nmask, h->mask_idx, h->gb1 ? h->vec_int : se, std::nan(""), h->st));
  if (h->gb1) CK(launch_perm_to_user(n, h->perm, h->vec_int, se, h->st));
  CK(cudaMemcpyAsync(h->h_flags, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  CK(cudaMemcpyAsync(h->h_flags + 1, h->err, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  if (h->h_flags[1]) return MNL_ERR_TIMEOUT;
  if (h->h_flags[0] & 4) return MNL_ERR_NOT_PD;
  return MNL_OK;
}

int mnl_predict(mnl_handle *h, const double *theta, double *P, double *loglik) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!theta || !P) return MNL_ERR_INVALID_ARG;
  if ((rc = set_device(h))) return rc;
  CK(cudaMemsetAsync(h->err, 0, sizeof(int), h->st));
  const double *th = theta_in(h, theta, &rc);
  if (rc) return rc;
  if ((rc = run_pass(h, th, true, nullptr, kL))) return rc;
  CK(launch_export_probs(h->S.N * (int64_t)h->S.K, h->P, h->fp64, P, h->st));
  if (loglik) {
    CK(cudaMemcpyAsync(h->h_scal, h->scal, sizeof(double), cudaMemcpyDeviceToHost, h->st));
    CK(cudaMemcpyAsync(h->h_flags + 1, h->err, sizeof(int), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    if (h->h_flags[1]) return MNL_ERR_TIMEOUT;
    *loglik = h->h_scal[0];
  }
  return MNL_OK;
}

int64_t mnl_shard_sums_size(const mnl_dims *d) {
  const int64_t n = mnl_num_params(d);
  return n < 0 ? -1 : 2 + n + n * (n + 1) / 2;
}

int mnl_shard_grad_hess(mnl_handle *h, const double *theta, double *sums) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!theta || !sums) return MNL_ERR_INVALID_ARG;
  if (h->gb1 || h->hfree) return MNL_ERR_UNSUPPORTED;
  if ((rc = set_device(h))) return rc;
  const int64_t n = h->S.n;
  CK(cudaMemsetAsync(h->err, 0, sizeof(int), h->st));
  if ((rc = run_pass(h, theta, true, nullptr, kL))) return rc;
  if ((rc = run_hessian(h))) return rc;
  CK(cudaMemcpyAsync(sums, h->scal + kL, 2 * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
  CK(cudaMemcpyAsync(sums + 2, h->grad, (size_t)n * 8, cudaMemcpyDeviceToDevice, h->st));
  CK(launch_pack_lower(n, h->F, sums + 2 + n, h->st));
  CK(cudaMemcpyAsync(h->h_flags + 1, h->err, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  return h->h_flags[1] ? MNL_ERR_TIMEOUT : MNL_OK;
}

int mnl_shard_solve(mnl_handle *h, const double *sums, double *delta, mnl_step_info *info) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!sums || !delta) return MNL_ERR_INVALID_ARG;
  if (h->gb1 || h->hfree) return MNL_ERR_UNSUPPORTED;
  if ((rc = set_device(h))) return rc;
  const int64_t n = h->S.n;
  mnl_step_info loc{};
  CK(cudaEventRecord(h->ev[2], h->st));
  CK(cudaMemcpyAsync(h->grad, sums + 2, (size_t)n * 8, cudaMemcpyDeviceToDevice, h->st));
  CK(launch_unpack_lower(n, sums + 2 + n, h->F, h->st));
  CK(launch_mask_vec(h->nmask, h->mask_idx, h->grad, 0.0, h->st));
  CK(launch_mask_matrix(n, h->nmask, h->mask_idx, h->F, nullptr, h->st));
  rc = solve_system(h, loc);
  CK(cudaEventRecord(h->ev[3], h->st));
  if (rc == MNL_OK) CK(cudaMemcpyAsync(delta, h->delta, (size_t)n * 8, cudaMemcpyDeviceToDevice, h->st));
  CK(cudaStreamSynchronize(h->st));
  loc.solve_mode = h->solve_mode;
  loc.t_chol_ms = loc.t_factor_ms = elapsed(h->ev[2], h->ev[3]);
  if (info) *info = loc;
  return rc;
}

int mnl_shard_loglik(mnl_handle *h, const double *theta, const double *delta, double t, double *l2) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!theta || !l2) return MNL_ERR_INVALID_ARG;
  if (h->gb1) return MNL_ERR_UNSUPPORTED;
  if ((rc = set_device(h))) return rc;
  CK(cudaMemsetAsync(h->err, 0, sizeof(int), h->st));
  if (delta) {
    h->h_scal[8] = t;
    CK(cudaMemcpyAsync(h->tscale, h->h_scal + 8, sizeof(double), cudaMemcpyHostToDevice, h->st));
  }
  if ((rc = run_pass(h, theta, false, delta, kLt))) return rc;
  CK(cudaMemcpyAsync(l2, h->scal + kLt, 2 * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
  CK(cudaMemcpyAsync(h->h_flags + 1, h->err, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  return h->h_flags[1] ? MNL_ERR_TIMEOUT : MNL_OK;
}

double mnl_loglik_roundoff(const mnl_handle *h) {
  return h ? (h->fp64 ? std::ldexp(1.0, -53) : std::ldexp(1.0, -24)) : 0.0;
}

int mnl_set_weights(mnl_handle *h, const float *w) {
  if (!h) return MNL_ERR_INVALID_ARG;
  if (!w) { h->w = nullptr; return MNL_OK; }
  if ((reinterpret_cast<uintptr_t>(w) & 15) != 0) return MNL_ERR_INVALID_ARG;
  int rc = set_device(h);
  if (rc) return rc;
  CK(cudaMemsetAsync(h->status, 0, sizeof(int), h->st));
  CK(launch_validate_weights(h->S.N, w, h->status, h->st));
  CK(cudaMemcpyAsync(h->h_flags, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  if (h->h_flags[0] & 2) return MNL_ERR_NONFINITE;
  if (h->h_flags[0] & 1) return MNL_ERR_INVALID_ARG;
  h->w = w;
  return MNL_OK;
}

int mnl_check_collinear(mnl_handle *h, double tol, int32_t *flags, int32_t *ndropped) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!flags || !(tol > 0.0) || !std::isfinite(tol)) return MNL_ERR_INVALID_ARG;
  if ((rc = set_device(h))) return rc;
  CK(collinear_check(h->dims, h->X, h->Y, h->Zu, tol, h->nsm, h->st, flags, nullptr));
  if (ndropped) {
    int32_t c = 0;
    for (int i = 0; i < collinear_flags_size(h->dims); ++i) c += flags[i] != 0;
    *ndropped = c;
  }
  return MNL_OK;
}

int mnl_drop_columns(mnl_handle *h, const int32_t *flags) {
  if (!h) return MNL_ERR_INVALID_ARG;
  if (!flags) { h->nmask = 0; return MNL_OK; }
  const mnl_dims &d = h->dims;
  const int nf = collinear_flags_size(d);
  for (int i = 0; i < nf; ++i)
    if (flags[i] != 0 && flags[i] != 1) return MNL_ERR_INVALID_ARG;
  // The coefficients of the flagged columns in the caller's order (eq. "theta vec"), then in the kernels'.
  const int64_t n = h->S.n, nb = (int64_t)(d.K - 1) * d.p, dd = d.d;
  std::vector<int64_t> idx;
  auto internal = [&](int64_t u) { return !h->gb1 ? u : u < nb ? u : u < nb + dd ? n - dd + (u - nb) : u - dd; };
  for (int k = 1; k < d.K; ++k)
    for (int j = 0; j < d.p; ++j)
      if (flags[j]) idx.push_back(internal((int64_t)(k - 1) * d.p + j));
  int64_t u = nb;
  for (int k = h->gb1 ? 0 : 1; k < d.K; ++k)
    for (int j = 0; j < d.d; ++j, ++u)
      if (flags[d.p + k * d.d + j]) idx.push_back(internal(u));
  for (int j = 0; j < d.f; ++j, ++u)
    if (flags[d.p + d.K * d.d + j]) idx.push_back(internal(u));
  if (u != n) return MNL_ERR_INVALID_ARG;
  int rc = set_device(h);
  if (rc) return rc;
  if (!h->mask_idx && (rc = dalloc(h, &h->mask_idx, (size_t)n * sizeof(int64_t)))) return rc;
  if (!idx.empty()) {
    CK(cudaMemcpyAsync(h->mask_idx, idx.data(), idx.size() * sizeof(int64_t), cudaMemcpyHostToDevice, h->st));
    CK(cudaStreamSynchronize(h->st));
  }
  h->nmask = (int)idx.size();
  return MNL_OK;
}

int mnl_set_wait_bound(mnl_handle *h, uint64_t ns) {
  if (!h) return MNL_ERR_INVALID_ARG;
  h->wait_ns = ns;
  return MNL_OK;
}

int mnl_set_solve(mnl_handle *h, int mode) {
  if (!h || mode < MNL_SOLVE_AUTO || mode > MNL_SOLVE_MIXED) return MNL_ERR_INVALID_ARG;
  if (h->hfree) return mode == MNL_SOLVE_AUTO ? MNL_OK : MNL_ERR_UNSUPPORTED;
  h->solve_mode = mode == MNL_SOLVE_AUTO ? (h->fp64 ? MNL_SOLVE_FP64 : MNL_SOLVE_MIXED) : mode;
  return MNL_OK;
}

int mnl_destroy(mnl_handle *h) {
  if (!h) return MNL_OK;
  set_device(h);
  cudaStreamSynchronize(h->st);
  cudaGetLastError();
  free_all(h);
  delete h;
  return MNL_OK;
}

}  // extern "C"
