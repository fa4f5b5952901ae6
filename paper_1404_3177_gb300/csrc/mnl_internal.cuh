// Internal declarations shared by the CUDA translation units of libmnl.
//
// Coefficient layout (eq. "theta vec", gamma_0 fixed at 0):
//   theta = [beta_1..beta_{K-1} (p each) | gamma_1..gamma_{K-1} (d each) | alpha (f)]
// Hessian operand layout ("class-major"): the class columns of
//   A = [P_1 o M_1 | ... | P_{K-1} o M_{K-1}],  M_k = [X, Y_k]  (q = p + d columns per class)
// are numbered c = (k-1) q + l, l < p for X columns, l >= p for Y columns.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "../../include/mnl.h"

namespace mnl {

// Element type of the Hessian operands: double (FP64), float rounded to TF32,
// or bf16.
enum class OpType { F64 = 0, TF32 = 1, BF16 = 2 };

// Operand / output tile edge of every Hessian contraction.
constexpr int kTile = 128;
// Rows of the N dimension consumed per pipeline stage by the tensor-core SYRK
// (one 128-byte swizzle row per operand row).
constexpr int kBkBf16 = 64;
constexpr int kBkTf32 = 32;

struct Shape {
  int64_t N;
  int K, p, d, f;
  int q;        // p + d
  int64_t nb;   // (K-1) p
  int64_t ng;   // (K-1) d
  int64_t mc;   // (K-1) q  : class coefficients
  int64_t n;    // n_theta = mc + f
  int64_t nout; // raw gradient accumulators: (K-1) q + K f
};

__host__ __device__ inline Shape shape_of(int64_t N, int K, int p, int d, int f) {
  Shape s;
  s.N = N; s.K = K; s.p = p; s.d = d; s.f = f;
  s.q = p + d;
  s.nb = (int64_t)(K - 1) * p;
  s.ng = (int64_t)(K - 1) * d;
  s.mc = s.nb + s.ng;
  s.n = s.mc + f;
  s.nout = s.mc + (int64_t)K * f;
  return s;
}
inline Shape make_shape(const mnl_dims &d) { return shape_of(d.N, d.K, d.p, d.d, d.f); }

// A unit of the tiled contractions: operand (tensor map index, or 0 = At /
// 1 = Ad for the float64 path), problem, output tile (ti, tj), K-block range
// [kb0, kb1) and the offset of its 128 x 128 output tile.
// One contraction work unit: tile (ti, tj) of operand map `map` over the
// K-blocks [kb0, kb1), written at out_off (with 256-wide tiles, rows tj and
// tj + 1 of the B operand, the second half at out_off2).  flags: kUnitAcc adds into the
// output instead of storing it; kUnitEmpty is a placeholder that every role
// skips.
constexpr int kUnitAcc = 1, kUnitEmpty = 2;
struct SyrkUnit {
  int map, problem, ti, tj, kb0, kb1;
  int64_t out_off;
  int flags;
  int64_t out_off2;  // 256-wide tiles: offset of the second 128 x 128 half (tile tj + 1), < 0 when not stored
};

// theta index (class part) -> class k (1..K-1) and local column l (0..q-1).
__host__ __device__ inline void theta_class_local(const Shape &s, int64_t a, int &k, int &l) {
  if (a < s.nb) { k = (int)(a / s.p) + 1; l = (int)(a % s.p); }
  else { const int64_t r = a - s.nb; k = (int)(r / s.d) + 1; l = s.p + (int)(r % s.d); }
}

// ---------------------------------------------------------------------------
// Launchers (each defined in the .cu file that owns the kernel).
// ---------------------------------------------------------------------------

struct PassIO {
  const float *X, *Y, *Z;
  const int32_t *choice;
  const double *theta;   // [n]
  const double *delta;   // [n] or nullptr: coefficients are theta + (*tscale) * delta
  const double *tscale;  // device scalar (used when delta != nullptr)
  void *P;               // [N][K] T, FULL mode only
  void *zbar;            // [N][f] T, FULL mode only
  double *partials;      // [grid][2 + n] (FULL) or [grid][2] (loglik only)
  int *err;              // error word (bit 16: a tile copy did not complete in time); tiled pass only
  uint64_t wait_ns;      // bound of the tile-copy waits (0: the default, 2 s)
  const float *w;        // [N] observation weights, or nullptr (all ones)
  // Hessian-vector mode (FULL pass only): theta holds v, Pin the probabilities
  // of the last full pass ([N][K], T); the residual r_ik becomes
  // w_i P_ik (u_ik - sum_k P_ik u_ik) with u = J v, so the gradient slots
  // accumulate F v = -H v.  Wout ([N][K] float32, tiled pass with the
  // separate beta kernel only) receives those residuals.
  const void *Pin;
  float *Wout;
  // Wide shapes (PassPlan::ux): the utilities of the X block, U_x = X B, come
  // from a float32 GEMM into ux ([N][K] float32) before the pass, with the
  // coefficients as float32 in bf ([p][ux_ldb(K)]); both are scratch of the caller.
  float *ux;
  float *bf;
};
// Leading dimension of the float32 coefficient matrix of the utility GEMM.
inline int ux_ldb(int K) { return (K + 127) / 128 * 128; }

// Bits of the device error word: which kernel's bounded wait gave up.
constexpr int kWaitSyrk = 1 | 2 | 4 | 8;  // tensor-core contraction (producer, MMA, epilogue, drain)
constexpr int kWaitPass = 16;             // tiled pass / beta-gradient tile copies
constexpr int kWaitCoop = 32;             // cooperative factorisation's grid barrier
constexpr int kWaitPanel = 64;            // tensor-core trailing updates of the panel factorisation

// Configuration of the fused utility/softmax/log-likelihood/gradient pass.
struct PassPlan {
  int grid, block, rows, npt;   // CTAs, threads, rows per tile, outputs per thread
  size_t smem;
  bool ok;
  bool tiled;                   // float32 pass with asynchronous tile copies (pass_tile.cu)
  bool ux;                      // tiled, with the X-block utilities from a separate GEMM (wide shapes)
};
// allow_tiled: the float32 path may use the tiled pass (needs io.err and
// 16-byte aligned X, Y, Z, choice).
PassPlan plan_pass(const Shape &s, bool fp64, bool full, int num_sms, bool allow_tiled = true);
bool plan_pass_tiled(const Shape &s, bool full, int num_sms, PassPlan &pl);
// The tiled full pass leaves the beta gradient to its separate kernel (wide shapes).
bool plan_pass_beta_ext(const Shape &s);
cudaError_t launch_pass_tiled(const Shape &s, const PassPlan &pl, bool full, const PassIO &io, cudaStream_t st);
cudaError_t launch_pass(const Shape &s, const PassPlan &pl, bool fp64, bool full, const PassIO &io, cudaStream_t st);

// ---------------------------------------------------------------------------
// Grouped (batched) path: many independent problems, one launch per phase.
// ---------------------------------------------------------------------------

// Per-problem float64 scalars of a batched fit (GroupProblem::scal).
enum GroupScal {
  kGsL = 0, kGsLabs = 1, kGsGinf = 2, kGsLt = 3, kGsLtabs = 4, kGsT = 5, kGsStepInf = 6, kGsThetaInf = 7,
  kGsLold = 8, kGsLsEvals = 9, kGsIters = 10, kGsRefine = 11, kGsPrevStep = 12, kGsCount = 16
};

// Everything a grouped kernel needs to know about one problem (device memory).
struct GroupProblem {
  int64_t N;
  int K, p, d, f;
  int64_t n, mc;                 // n_theta, class coefficients
  const float *X, *Y, *Z;
  const int32_t *choice;
  double *theta, *grad, *delta;  // [n]
  void *P, *zbar;                // [N][K], [N][f] (float64 in FP64 mode, else float32)
  void *At, *Ad;                 // Hessian operands [mc_pad][ldn]
  int64_t ldn, mc_pad;
  int nt1d, zsplit;
  int build_ob, build_kc;        // operand-builder blocking
  int64_t main_off, band_off, z_off;  // offsets of this problem's contraction partials (elements)
  int *band_of;                  // [nt1d][nt1d]
  double *F;                     // [n][n]
  float *F32;                    // [n][n] (mixed solve)
  double *rwork;                 // [2 n] (mixed solve)
  double *scal;                  // [kGsCount]
};

// One CTA's run of consecutive row tiles of one problem in the grouped pass,
// with the offsets of its partial row (full pass / log-likelihood-only pass).
struct PassSeg {
  int problem;
  int64_t tile0, tile1;
  int64_t slot_full, slot_ll;
};

// A generic grouped work item: (problem, index within the problem).
struct GroupItem {
  int problem;
  int idx;
};

// Grouped Hessian pieces (one CTA per item; items of inactive problems exit).
cudaError_t launch_grouped_build(OpType t, const GroupProblem *probs, const GroupItem *items, int nitems,
                                 const int *active, size_t smem, cudaStream_t st);
cudaError_t launch_grouped_zblocks(bool fp64, const GroupProblem *probs, const GroupItem *items, int nitems,
                                   const int *active, size_t smem, void *zpart, cudaStream_t st);
cudaError_t launch_grouped_assemble(bool fp64, const GroupProblem *probs, const GroupItem *items, int nitems,
                                    const int *active, const void *mainp, const void *bandp, const void *zpart,
                                    cudaStream_t st);
size_t build_smem_bytes(const Shape &s, OpType t, int ob, int kc, bool with_z = false);
void build_blocking(const Shape &s, OpType t, int *ob, int *kc, bool with_z = false);
int zblocks_parts(const Shape &s, bool fp64);  // CTAs per observation split
size_t zblocks_smem(const Shape &s, bool fp64);
constexpr int kAssembleCols = 8;  // columns per grouped-assembly item

// Grouped float64 contraction (FP64 mode): one CTA per unit, map 0 = At, 1 = Ad,
// K range in chunks of f64_chunk_rows() observations.
cudaError_t launch_grouped_syrk_f64(const GroupProblem *probs, const SyrkUnit *units, int nunits, const int *active,
                                    double *out, cudaStream_t st);
int f64_chunk_rows();

// One CTA per active problem: delta = (-H)^{-1} g (mixed or float64), see cholesky.cu.
// Problems with n_theta above max_n are skipped (solved by the multi-CTA path).
constexpr int64_t kCtaSolveMaxN = 1400;
size_t grouped_chol_smem(int64_t nmax);
// One CTA per listed problem (plist[0 .. nprob)), shared memory `smem` sized for the largest listed n.
cudaError_t launch_grouped_chol_solve(bool mixed, const GroupProblem *probs, const int *plist, int nprob,
                                      const int *active, int iters, int *status, size_t smem, int64_t max_n,
                                      cudaStream_t st);

struct GroupedPassPlan {
  int grid, block, rows, npt;
  size_t smem;
  bool ok;
};
GroupedPassPlan plan_grouped_pass(const std::vector<Shape> &shapes, bool fp64, int rows, int num_sms);
cudaError_t launch_grouped_pass(const GroupedPassPlan &pl, bool fp64, bool full, const GroupProblem *probs,
                                const PassSeg *segs, const int *seg_start, const int *active, double *partials,
                                cudaStream_t st);
// Per problem (one CTA each): l, sum|l| -> scal[base..]; full: g -> grad, max|g| -> scal[kGsGinf].
cudaError_t launch_grouped_reduce(int nprob, bool full, const GroupProblem *probs, const int *slot_start,
                                  const PassSeg *segs, const int *slot_segs, const int *active,
                                  const double *partials, int base, cudaStream_t st);

// Fixed-order FP64 reduction of the pass partials.
//   out: [0] l, [1] sum |l_i|, [2] max|g|; grad (θ order) when full.
cudaError_t launch_pass_reduce(const Shape &s, int grid, bool full, const double *partials, double *scal,
                               double *grad, cudaStream_t st);

// Data validation: status bits |= 1 (choice out of range), 2 (non-finite data).
cudaError_t launch_validate(const Shape &s, const float *X, const float *Y, const float *Z, const int32_t *choice,
                            int *status, cudaStream_t st);

// Hessian operands At [mc_pad][ldn] (class-major rows, observation columns):
//   At  [c][i] = P_ik m_ik[l]                   (c = (k-1)q + l)
//   Ad  [c][i] = sqrt(P_ik (1 - P_ik)) m_ik[l]
// T = double (FP64), float rounded to TF32 (TF32), or bf16 (BF16).
// Class operands At, Ad (and, when Az != nullptr, the rows of the Z-block operand from the same staged block).
cudaError_t launch_build_operands(const Shape &s, OpType t, const float *X, const float *Y, const void *P, void *At,
                                  void *Ad, int64_t ldn, cudaStream_t st, const float *Z = nullptr,
                                  const void *zbar = nullptr, void *Az = nullptr, const float *w = nullptr);

// Tile lists (pairs (ti, tj), ti >= tj) of the two contractions.
struct TileLists {
  int nmain, nband;
  int2 *main;      // all lower-triangle tiles, index ti(ti+1)/2 + tj
  int2 *band;      // tiles meeting a diagonal class block
  int *band_of;    // [nt1d][nt1d]: index in `band` of tile (ti, tj), or -1
};

// FP64 CUDA-core SYRK: out[(s * ntiles + t)][128][128] = sum over split s of At[a] At[b]^T.
cudaError_t launch_syrk_f64(const double *At, int64_t ldn, int64_t N, const int2 *tiles, int ntiles, int nsplit,
                            double *out, cudaStream_t st);

// tcgen05 tensor-core SYRK (BF16 or TF32 operands, FP32 accumulation in TMEM)
// over a list of work units: unit = (tensor map, problem, output tile (ti, tj),
// K-block range [kb0, kb1)), writing out[out_off .. + 128*128) transposed.
// Units of problems with active[problem] == 0 are skipped (active may be null).
// TF32 / BF16 operands in the K-blocked layout [ldn / BK][rows_pad][BK] (BK
// observations = 128 bytes per row of a block; see op_off in hessian.cu).
cudaError_t encode_operand_map(OpType t, const void *At, int64_t rows_pad, int64_t ldn, CUtensorMap *out);
// A row-major float32 [rows][cols] matrix read as TF32 boxes of 128 rows x 32 columns.
cudaError_t encode_rows_map(const float *A, int64_t rows, int64_t cols, CUtensorMap *out);
int tc_kblocks(OpType t, int64_t ldn);
int tc_pick_split(int ntiles, int kblocks, int num_sms);
// K-blocks of one accumulation chunk of the tensor-core SYRK (16384 observations):
// the FP32 accumulator in TMEM never sums more observations than that.
int tc_chunk_kblocks(OpType t);
// Lay out SYRK jobs for a persistent grid: each job is cut into chunks of at
// most max_kb K-blocks that one CTA runs back to back (the first stores the
// tile, the rest add into it, a fixed order), jobs go longest first to the
// least-loaded CTA, and the per-CTA sequences are interleaved (unit u runs on
// CTA u % grid) with empty units as padding.
std::vector<SyrkUnit> schedule_syrk_units(const std::vector<SyrkUnit> &jobs, int grid, int max_kb);
size_t tc_smem_bytes();
cudaError_t launch_syrk_tc(OpType t, const CUtensorMap *maps, const SyrkUnit *units, int nunits, const int *active,
                           int grid, float *out, int *err, cudaStream_t st, int bn = 128, uint64_t wait_ns = 0);

// Z blocks (FP32 or FP64 accumulation) per observation split s:
// out[s][zblocks_outputs()] = [C_X: p*K*f | C_Y: K*d*f | A: f*f] (see hessian.cu).
int64_t zblocks_outputs(const Shape &s);
cudaError_t launch_zblocks(const Shape &s, bool fp64, const float *X, const float *Y, const float *Z, const void *P,
                           const void *zbar, int nsplit, void *out, cudaStream_t st, const float *w = nullptr);
// Data validation of observation weights: status bits |= 1 (negative), 2 (non-finite).
cudaError_t launch_validate_weights(int64_t N, const float *w, int *status, cudaStream_t st);

// Assemble F = -H (n x n, column-major, both triangles) from the contraction
// partials.  main/band partials are FP32 (tensor path) or FP64.
// Z blocks from the tensor-core contraction of the Z-block operand (TF32 /
// BF16 modes): row offsets of its blocks (X at 0), and the tile pairs that are
// contracted (index[ti * nt + tj] = pair or -1; partial tiles [split][pair]).
struct ZopLayout {
  int64_t oY, oW, oZ, rows_pad;
};
ZopLayout zop_layout(const Shape &s);
struct ZTiles {
  std::vector<int2> pairs;
  std::vector<int> index;  // [nt * nt]
  int nt = 0;
};
ZTiles zop_tiles(const Shape &s, const ZopLayout &L);
struct ZTileView {
  const float *part = nullptr;  // nullptr: Z blocks come from z_part (CUDA-core kernel)
  int split = 0, npairs = 0, nt = 0;
  const int *index = nullptr;
  int64_t oY = 0, oW = 0, oZ = 0;
};

struct AssembleIO {
  const void *main_part; int main_split;
  const void *band_part; int band_split;
  const void *z_part;    int z_split;
  const TileLists *tl;   // device pointers inside
  bool fp64;
  ZTileView zt;
  float *f32 = nullptr;  // when given, the lower triangle of F in float32 too (the mixed solve's input)
};
cudaError_t launch_assemble(const Shape &s, const AssembleIO &io, int nmain, double *F, cudaStream_t st);

// Mirror the lower triangle of F into a full symmetric matrix H = -F (column-major).
cudaError_t launch_export_hessian(int64_t n, const double *F, double *H, cudaStream_t st);

// Blocked Cholesky of F (lower, column-major, ld = n) in place by one
// cooperative kernel, dinv[j] = 1/L_jj; work: chol_work_bytes(n) bytes.
// status |= 4 when a pivot is not positive or not finite; *err != 0 when a
// grid barrier wait ran out (the kernel then returns early).
size_t chol_work_bytes(int64_t n);
int cholesky_launches(int64_t n);
cudaError_t launch_cholesky(int64_t n, double *F, double *dinv, void *work, int *status, int *err, cudaStream_t st,
                            uint64_t wait_ns = 0);
// Standard errors sqrt(diag(F^{-1})): float64 factor of F (in place) with the
// inverse of the factor Binv (n x n scratch), then the column norms of Binv.
// status |= 4 when F is not positive definite (se is then NaN).
cudaError_t launch_std_errors(int64_t n, double *F, double *Binv, double *dinv, void *work, int *status, int *err,
                              double *se, cudaStream_t st, uint64_t wait_ns = 0);
// Probabilities [N][K] in float64 from the pass's P (float32 or float64).
cudaError_t launch_export_probs(int64_t count, const void *P, bool fp64, double *out, cudaStream_t st);
// Solve L L^T x = b with the factor above (FP64; skipped when status & 4).
cudaError_t launch_cholesky_solve(int64_t n, const double *L, const double *dinv, const double *b, double *x,
                                  const int *status, cudaStream_t st, int *launches);
// Mixed solve: float32 factor and inverse of the factor (F kept intact, both
// triangles; F32: n*n floats of scratch) and float64 iterative refinement of
// F delta = g.  status |= 8 when the float32 factor fails, 16 when the
// refinement does not converge (use the FP64 path then).  work:
// mixed_solve_bytes(n); mixed_solve_ref(work, n) holds 4 doubles of
// refinement state ([2] = refinement steps taken), zeroed by the caller.
size_t mixed_solve_bytes(int64_t n);
double *mixed_solve_ref(void *work, int64_t n);
// f32_ready: F32 already holds the float32 lower triangle of F (written by the assembly).
cudaError_t launch_mixed_solve(int64_t n, const double *F, float *F32, const double *g, double *delta, void *work,
                               int *status, int *err, int iters, cudaStream_t st, int *launches,
                               bool f32_ready = false, uint64_t wait_ns = 0);
// status &= mask (device word).
cudaError_t launch_status_and(int *status, int mask, cudaStream_t st);
// `iters` more refinement steps after launch_mixed_solve (the caller first clears status bit 16).
cudaError_t launch_mixed_refine(int64_t n, const double *F, const double *g, double *delta, void *work, int *status,
                                int iters, cudaStream_t st, int *launches);

// ---------------------------------------------------------------------------
// Mixed solve with a tensor-core factorisation (large n): blocked right-looking
// float32 Cholesky of F and the inverse of the factor, panels of kCholPanel
// columns; per panel one CTA factors and inverts the diagonal block, a panel
// kernel forms the panel rows of L (and of L^{-1}) and their TF32 hi/lo
// copies, and the trailing updates run as 3xTF32 tcgen05 tiles.
// ---------------------------------------------------------------------------
constexpr int kCholPanel = 128;
// One 128 x 128 tile of a trailing update: C(ti, tj) -= A(ti) B(tj)^T, with
// A = panel rows (maps 0, 1), B = rows of maps (2 bmap, 2 bmap + 1), C the
// factor (cbuf 0) or the inverse (cbuf 1); tri: only the lower triangle of
// the tile.
struct CholUnit {
  int ti, tj, bmap, cbuf, tri, pad;
};
size_t chol_update_smem_bytes();
// Sets the kernel's shared-memory attribute on the current device.
cudaError_t chol_update_tc_setup();
cudaError_t launch_chol_update_tc(const CUtensorMap *maps, const CholUnit *units, int nunits, int grid, float *C0,
                                  float *C1, int64_t ld, int64_t n, int *err, uint64_t wait_ns, cudaStream_t st);

// Host-side plan (built once per handle; holds device pointers into `ws`).
struct TcCholPlan {
  int64_t n = 0, n_pad = 0;
  int np = 0, grid = 0;
  int reserve = 0;                    // SMs left to the side stream while the rest of an update runs
  void *ws = nullptr;                 // tc_chol_bytes(n) bytes of device memory
  CUtensorMap *maps = nullptr;        // device: two sets (panel parity) of Ph, Pl, Rh, Rl
  CholUnit *units = nullptr;          // device: all panels' units
  // host: panel k's units are [unit_off[k], unit_off[k + 1]); those that the next
  // panel's diagonal and panel steps wait for come first, [unit_off[k], unit_mid[k])
  std::vector<int> unit_off, unit_mid;
  float *Ph[2] = {}, *Pl[2] = {}, *Rh[2] = {}, *Rl[2] = {};  // [n_pad][128] hi / lo, per panel parity
  float *InvT = nullptr;             // [np][128][128]: inverse of each diagonal block, transposed
  cudaStream_t side = nullptr;       // the diagonal and panel steps of the next panel (look-ahead)
  cudaEvent_t ev_start = nullptr, ev_next = nullptr, ev_panel = nullptr;
  bool ready = false;
};
// Destroys the plan's stream and events (the device memory belongs to the caller).
void tc_chol_release(TcCholPlan *plan);
// Use the tensor-core factorisation for n_theta at or above this.
constexpr int64_t kTcCholMinN = 4096;
size_t tc_chol_bytes(int64_t n);
// Encodes the tensor maps and uploads the unit lists (synchronous; call at set-up).
cudaError_t tc_chol_prepare(int64_t n, void *ws, int num_sms, TcCholPlan *plan);
// As launch_mixed_solve (F32 holds the float32 lower triangle of F), with the
// tensor-core factorisation and inverse.
cudaError_t launch_mixed_solve_tc(const TcCholPlan &plan, const double *F, float *F32, const double *g, double *delta,
                                  void *work, int *status, int *err, int iters, uint64_t wait_ns, cudaStream_t st,
                                  int *launches);

// Paper-literal gamma_0 (gamma_base = 1): the model equals a gamma_base = 0
// model with d more generic (Z-type) columns z'_ikj = (k == 0 ? y_i0j : 0),
// whose coefficients are gamma_0 (only differences against alternative 0
// enter: z'_ik - z'_i0 = -y_i0 for k >= 1, the paper's -Y_i0 gamma_0 term).
// Zaug [N][K][f + d] = [Z | that block].
cudaError_t launch_augment_z(int64_t N, int K, int d, int f, const float *Y, const float *Z, float *Zaug,
                             cudaStream_t st);
// theta orders: user (gamma_0 before gamma_1) and internal (gamma_0 after alpha);
// perm[u] = internal index of user coefficient u.
cudaError_t launch_perm_to_internal(int64_t n, const int64_t *perm, const double *user, double *internal,
                                    cudaStream_t st);
cudaError_t launch_perm_to_user(int64_t n, const int64_t *perm, const double *internal, double *user,
                                cudaStream_t st);
// H[u][v] = -F[perm[u]][perm[v]] (column-major, both triangles of F present).
cudaError_t launch_export_hessian_perm(int64_t n, const double *F, const int64_t *perm, double *H, cudaStream_t st);

// Observation sharding: -H's lower triangle packed column by column
// (n (n + 1) / 2 doubles) and back into both triangles of F.
cudaError_t launch_pack_lower(int64_t n, const double *F, double *out, cudaStream_t st);
cudaError_t launch_unpack_lower(int64_t n, const double *in, double *F, cudaStream_t st);
cudaError_t launch_f64_to_f32_lower(int64_t n, const double *F, float *F32, cudaStream_t st);

// Collinearity check (collinear.cu): flags of the dependent data columns in the
// layout [X (p) | Y_0 .. Y_{K-1} (K d) | Z (f)] (Y_0 only with gamma_base = 1),
// written to flags_host; synchronous, allocates and frees its own scratch.
struct CollinearStats {
  float ms;          // device time of the Gram pass and the decisions
  int groups, jobs, tile;
  double gram_fma;   // sum over the blocks of rows x cols (cols + 1) / 2
  double bytes;      // sum over the blocks of rows x cols x 4 (data read once per block pair at least)
};
int collinear_flags_size(const mnl_dims &d);
cudaError_t collinear_check(const mnl_dims &d, const float *X, const float *Y, const float *Z, double tol, int nsm,
                            cudaStream_t st, int32_t *flags_host, CollinearStats *stats);
// v[idx[t]] = val for t < m.
cudaError_t launch_mask_vec(int m, const int64_t *idx, double *v, double val, cudaStream_t st);
// Rows and columns idx[0 .. m) of F (n x n, both triangles) and of F32's lower
// triangle (when not NULL) set to those of the identity.
cudaError_t launch_mask_matrix(int64_t n, int m, const int64_t *idx, double *F, float *F32, cudaStream_t st);

// Small FP64 vector kernels.
cudaError_t launch_dot(int64_t n, const double *a, const double *b, double *out, cudaStream_t st);  // out = a.b
cudaError_t launch_axpby(int64_t n, double a, const double *x, double b, double *y, cudaStream_t st);  // y = ax+by
cudaError_t launch_axpy_theta(int64_t n, double *theta, const double *delta, const double *tscale, double *scal_out,
                              cudaStream_t st);
cudaError_t launch_vec_absmax(int64_t n, const double *v, double *out, cudaStream_t st);
// theta += delta when l(theta + delta) = *lt >= *l0 - u8 * *labs and status / err show no failure; then status |= 32.
cudaError_t launch_try_full_step(int64_t n, double *theta, const double *delta, const double *l0, const double *labs,
                                 const double *lt, int *status, const int *err, double u8, double *scal_out,
                                 cudaStream_t st);

}  // namespace mnl
