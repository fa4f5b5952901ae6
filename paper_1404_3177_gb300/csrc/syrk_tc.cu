// Tensor-core SYRK for the class blocks of the negative Hessian (Sec. 3.3,
// eq. "hessian block"):  C = A^T A  over the observations, A = At^T.
//
// At is stored class-major, [rows_pad][ldn], one operand row per Hessian
// column, observations contiguous ("K-major" for the MMA).  A job is one
// 128 x 128 output tile (ti, tj), ti >= tj, over one contiguous range ("split")
// of the observations; partial tiles are written in float32 and reduced in
// fixed order by the assembly kernel (no float atomics).  A job runs as units
// of at most 16384 observations on one CTA, one after the other: the first
// stores the tile and the others add into it, so no FP32 accumulator in TMEM
// sums more than 16384 products (the rounding of long accumulations otherwise
// grows with N).
//
// Per CTA (one per SM, persistent, 6 warps):
//   warp 0 (one lane): TMA producer, 128-row x 128-byte boxes with the
//                      128-byte swizzle into a 6-stage shared-memory ring;
//                      a diagonal tile loads its single operand once.
//   warp 1:            TMEM allocation (256 columns = two 128-column FP32
//                      accumulators); one lane issues tcgen05.mma
//                      (M = N = 128, K = 16 for BF16 or 8 for TF32) and frees
//                      ring slots / publishes accumulators with tcgen05.commit.
//   warps 2-5:         epilogue, tcgen05.ld of 32 TMEM lanes each, written
//                      transposed so each store instruction covers 128
//                      contiguous bytes; overlaps the next tile's main loop.
// Every wait is bounded (2 s on %globaltimer).  A wait that gives up raises a
// shared abort flag and the error word; every role then leaves its loop,
// in-flight TMA loads and MMAs are waited for (again bounded), TMEM is freed
// and the kernel returns.
#include <algorithm>
#include <queue>

#include "mnl_internal.cuh"

namespace mnl {
namespace {

constexpr int kOpBytes = kTile * 128;        // one operand box: 128 rows x 128 bytes
constexpr uint64_t kTimeoutNs = 2000000000ull;

// Tile width BN (the MMA's N): 128, or 256 for the main contraction (the B
// operand is two adjacent 128-row tiles), which halves the shared-memory
// operand traffic of A per flop.
template <int BN>
struct TcCfg {
  static constexpr int kStages = BN == 128 ? 6 : 4;
  static constexpr int kStageBytes = kOpBytes * (1 + BN / kTile);  // A and B operands
  static constexpr int kSmemBytes = kStages * kStageBytes + 256 + 1024;
  static constexpr int kTmemCols = 2 * BN;                         // two FP32 accumulators
};

// Instruction descriptors (kind::f16 with BF16 inputs / kind::tf32): FP32
// accumulator, both operands K-major, N = BN, M = 128.
template <bool TF32, int BN>
constexpr uint32_t idesc() {
  return (1u << 4) | (TF32 ? (2u << 7) | (2u << 10) : (1u << 7) | (1u << 10)) | ((uint32_t)(BN >> 3) << 17) |
         ((uint32_t)(kTile >> 4) << 24);
}

__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(saddr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the phase of `parity` to complete.  Returns false when another role
// raised the abort flag (if honour_abort) or after kTimeoutNs (then raises the
// abort flag and records `code` in the error word).
// Waits that drain copies or MMAs already issued (honour_abort = false) always
// use the full bound, so that nothing is left writing into shared memory or
// TMEM when the CTA exits.
__device__ bool wait_bounded(uint64_t *bar, uint32_t parity, volatile int *abort_flag, int *err, int code,
                             bool honour_abort = true, uint64_t bound_ns = kTimeoutNs) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = gtimer();
  const uint64_t lim = honour_abort ? bound_ns : kTimeoutNs;
  for (uint32_t it = 1;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 31u) == 0) {
      if (honour_abort && *abort_flag) return false;
      if (gtimer() - t0 > lim) {
        *abort_flag = 1;
        atomicOr(err, code);
        return false;
      }
    }
  }
}

__device__ __forceinline__ void tma_load_2d(const CUtensorMap *map, uint64_t *bar, void *dst, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::
          "r"(saddr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(saddr(bar)), "r"(x), "r"(y)
      : "memory");
}

// Box (0, y, z) of a 3-D map: the K-blocked operands (K-block z, rows y ..).
__device__ __forceinline__ void tma_load_3d(const CUtensorMap *map, uint64_t *bar, void *dst, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];" ::
          "r"(saddr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(saddr(bar)), "r"(0), "r"(y), "r"(z)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
               : "memory");
}

// Shared-memory matrix descriptor: K-major operand in the 128-byte swizzle
// layout written by TMA (8-row x 128-byte atoms, 1024 bytes apart).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);  // start address
  d |= (uint64_t)1 << 16;                   // leading byte offset (not used by this layout)
  d |= (uint64_t)(1024 >> 4) << 32;         // stride byte offset: next 8-row group
  d |= (uint64_t)1 << 46;                   // descriptor version
  d |= (uint64_t)2 << 61;                   // 128-byte swizzle
  return d;
}

template <bool TF32, int BN>
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
  if (TF32) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc<true, BN>()), "r"(accumulate)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc<false, BN>()), "r"(accumulate)
        : "memory");
  }
}

__device__ __forceinline__ void tmem_ld_32x32b_x32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
        "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
        "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Error word bits.
constexpr int kErrProducer = 1, kErrMma = 2, kErrEpilogue = 4, kErrDrain = 8;

template <bool TF32, int BN>
__global__ void __launch_bounds__(192, 1) syrk_tc_kernel(const CUtensorMap *__restrict__ maps,
                                                         const SyrkUnit *__restrict__ units, int nunits,
                                                         const int *__restrict__ active, float *__restrict__ out,
                                                         int *__restrict__ err, uint64_t wait_ns) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  constexpr int kStages = TcCfg<BN>::kStages, kStageBytes = TcCfg<BN>::kStageBytes;
  constexpr int kTmemCols = TcCfg<BN>::kTmemCols;
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + kStages * kStageBytes);
  uint64_t *empty = full + kStages;
  uint64_t *tfull = empty + kStages;
  uint64_t *tempty = tfull + 2;
  uint64_t *drain = tempty + 2;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drain + 1);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int kBk = TF32 ? kBkTf32 : kBkBf16;
  // A unit is skipped by every role alike when its problem is inactive.
  auto skip = [&](const SyrkUnit &w) {
    return (w.flags & kUnitEmpty) != 0 || (active != nullptr && active[w.problem] == 0);
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(&tfull[b], 1); mbar_init(&tempty[b], 4); }
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer ----------------
      int stage = 0;
      uint32_t phase = 0;
      int last_par[kStages];
      for (int s = 0; s < kStages; ++s) last_par[s] = -1;
      bool ok = true;
      for (int u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
        const SyrkUnit w = units[u];
        if (skip(w)) continue;
        const CUtensorMap *map = maps + w.map;
        const bool diag = BN == kTile && w.ti == w.tj;  // a 128-wide diagonal tile loads its operand once
        for (int kb = w.kb0; kb < w.kb1; ++kb) {
          if (!wait_bounded(&empty[stage], phase ^ 1u, abort_flag, err, kErrProducer, true, wait_ns)) {
            ok = false;
            break;
          }
          uint8_t *dst = smem + stage * kStageBytes;
          mbar_arrive_expect_tx(&full[stage], diag ? kOpBytes : (1 + BN / kTile) * kOpBytes);
          tma_load_3d(map, &full[stage], dst, w.ti * kTile, kb);
          if (!diag)
#pragma unroll
            for (int h = 0; h < BN / kTile; ++h)  // B: BN / 128 consecutive tiles (zero-filled past the last row)
              tma_load_3d(map, &full[stage], dst + (1 + h) * kOpBytes, (w.tj + h) * kTile, kb);
          last_par[stage] = (int)phase;
          if (++stage == kStages) { stage = 0; phase ^= 1u; }
        }
      }
      // No TMA write may still be pending when the CTA exits.
      for (int s = 0; s < kStages; ++s)
        if (last_par[s] >= 0) wait_bounded(&full[s], (uint32_t)last_par[s], abort_flag, err, kErrDrain, false);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer ----------------
      int stage = 0;
      uint32_t phase = 0;
      uint32_t acc_ph[2] = {0u, 0u};
      int local = 0;
      bool ok = true;
      for (int u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
        const SyrkUnit w = units[u];
        if (skip(w)) continue;
        const int kb0 = w.kb0, kb1 = w.kb1;
        const bool diag = BN == kTile && w.ti == w.tj;
        const int b = local & 1;
        ++local;
        if (!wait_bounded(&tempty[b], acc_ph[b] ^ 1u, abort_flag, err, kErrMma, true, wait_ns)) break;
        acc_ph[b] ^= 1u;
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + (uint32_t)(b * BN);
        for (int kb = kb0; kb < kb1; ++kb) {
          if (!wait_bounded(&full[stage], phase, abort_flag, err, kErrMma, true, wait_ns)) { ok = false; break; }
          tc_fence_after();
          const uint32_t a_addr = saddr(smem + stage * kStageBytes);
          const uint32_t b_addr = diag ? a_addr : a_addr + kOpBytes;
          const uint64_t ad = sw128_desc(a_addr), bd = sw128_desc(b_addr);
#pragma unroll
          for (int k = 0; k < 4; ++k)  // 4 x 32 bytes along K inside the 128-byte row
            tc_mma<TF32, BN>(d_tmem, ad + (uint64_t)(2 * k), bd + (uint64_t)(2 * k), (kb > kb0 || k > 0) ? 1u : 0u);
          tc_commit(&empty[stage]);
          if (++stage == kStages) { stage = 0; phase ^= 1u; }
        }
        if (!ok) break;
        tc_commit(&tfull[b]);
      }
      // Every MMA issued by this thread has completed before TMEM is freed.
      tc_commit(drain);
      wait_bounded(drain, 0u, abort_flag, err, kErrDrain, false);
    }
  } else {
    // ---------------- epilogue (warps 2..5) ----------------
    const int quarter = warp & 3;  // this warp may access TMEM lanes 32*quarter .. +31
    uint32_t acc_ph[2] = {0u, 0u};
    int local = 0;
    for (int u = blockIdx.x; u < nunits; u += gridDim.x) {
      const SyrkUnit w = units[u];
      if (skip(w)) continue;
      const int b = local & 1;
      ++local;
      int ok = 0;
      if (lane == 0) ok = wait_bounded(&tfull[b], acc_ph[b], abort_flag, err, kErrEpilogue, true, wait_ns) ? 1 : 0;
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) break;
      acc_ph[b] ^= 1u;
      tc_fence_after();
      // Tile stored transposed: out[col][row], row = MMA M index (operand tile ti).
      // A later chunk of the same job adds into what this thread stored before.
      // A BN = 256 tile is two 128 x 128 output tiles (out_off, out_off2; out_off2 < 0: not stored).
      const bool acc = (w.flags & kUnitAcc) != 0;
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 32) {
        const int64_t o = c0 < kTile ? w.out_off : w.out_off2;
        uint32_t v[32];
        tmem_ld_32x32b_x32(tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * BN + c0), v);
        if (o < 0) continue;
        const int cl = c0 < kTile ? c0 : c0 - kTile;  // column within its 128 x 128 output tile
        float *dst = out + o + quarter * 32 + lane;
        if (acc) {
          float prev[32];
#pragma unroll
          for (int j = 0; j < 32; ++j) prev[j] = dst[(int64_t)(cl + j) * kTile];
#pragma unroll
          for (int j = 0; j < 32; ++j) dst[(int64_t)(cl + j) * kTile] = prev[j] + __uint_as_float(v[j]);
        } else {
#pragma unroll
          for (int j = 0; j < 32; ++j) dst[(int64_t)(cl + j) * kTile] = __uint_as_float(v[j]);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[b]);
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(kTmemCols)
                 : "memory");
  }
}

// ---------------------------------------------------------------------------
// Trailing updates of the blocked float32 Cholesky factorisation (and of the
// inverse of the factor carried along with it), C -= A B^T over one panel of
// kCholPanel = 128 columns, on the tensor cores in three TF32 passes:
// every operand is held as hi + lo (hi = TF32 rounding of the float32 value,
// lo = TF32 rounding of the remainder) and A B^T = Ah Bh^T + Ah Bl^T + Al Bh^T
// up to the Al Bl^T term, about 2^-21 relative: float32 accuracy from the
// TF32 datapath.  The operands are the panel buffers written by the panel
// kernel (rows contiguous along the 128 panel columns, i.e. K-major), so
// every TMA box is 128 rows x 32 floats.
// A unit is one 128 x 128 output tile of C (column-major, leading dimension
// ld), A = rows ti of maps (0, 1), B = rows tj of maps (2 bmap, 2 bmap + 1);
// tri: only entries on or below the diagonal of the tile are written.
// Roles as in the SYRK kernel: warp 0 TMA producer, warp 1 MMA issuer (one
// lane) and TMEM owner, warps 2-9 the epilogue (read C, subtract, write C,
// 128 contiguous bytes per store instruction across the warp): two warps per
// TMEM lane quarter, each taking half of the tile's columns, so that twice as
// many C loads are in flight (the epilogue's load latency sets the pace).
// ---------------------------------------------------------------------------
constexpr int kCuStages = 3;
constexpr int kCuEpiWarps = 8;                    // epilogue warps: two per TMEM lane quarter
constexpr int kCuThreads = 64 + 32 * kCuEpiWarps;  // + the producer and MMA warps
constexpr int kCuStageBytes = 4 * kOpBytes;  // Ah, Al, Bh, Bl
constexpr int kCuSmemBytes = kCuStages * kCuStageBytes + 256 + 1024;

__global__ void __launch_bounds__(kCuThreads, 1) chol_update_tc_kernel(const CUtensorMap *__restrict__ maps,
                                                                const CholUnit *__restrict__ units, int nunits,
                                                                float *__restrict__ C0, float *__restrict__ C1,
                                                                int64_t ld, int64_t n, int *__restrict__ err,
                                                                uint64_t wait_ns) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + kCuStages * kCuStageBytes);
  uint64_t *empty = full + kCuStages;
  uint64_t *tfull = empty + kCuStages;
  uint64_t *tempty = tfull + 2;
  uint64_t *drain = tempty + 2;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drain + 1);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
  constexpr int kTmemCols = 2 * kTile;
  constexpr int kKb = kCholPanel / kBkTf32;  // K-blocks per unit
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kCuStages; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(&tfull[b], 1); mbar_init(&tempty[b], kCuEpiWarps); }
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int last_par[kCuStages];
      for (int s = 0; s < kCuStages; ++s) last_par[s] = -1;
      bool ok = true;
      for (int u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
        const CholUnit w = units[u];
        const bool same = w.bmap == 0 && w.ti == w.tj;  // B = A: one pair of boxes
        const CUtensorMap *ma = maps, *mb = maps + 2 * w.bmap;
        for (int kb = 0; kb < kKb; ++kb) {
          if (!wait_bounded(&empty[stage], phase ^ 1u, abort_flag, err, kWaitPanel, true, wait_ns)) {
            ok = false;
            break;
          }
          uint8_t *dst = smem + stage * kCuStageBytes;
          mbar_arrive_expect_tx(&full[stage], (same ? 2 : 4) * kOpBytes);
          tma_load_2d(ma, &full[stage], dst, kb * kBkTf32, w.ti * kTile);
          tma_load_2d(ma + 1, &full[stage], dst + kOpBytes, kb * kBkTf32, w.ti * kTile);
          if (!same) {
            tma_load_2d(mb, &full[stage], dst + 2 * kOpBytes, kb * kBkTf32, w.tj * kTile);
            tma_load_2d(mb + 1, &full[stage], dst + 3 * kOpBytes, kb * kBkTf32, w.tj * kTile);
          }
          last_par[stage] = (int)phase;
          if (++stage == kCuStages) { stage = 0; phase ^= 1u; }
        }
      }
      for (int s = 0; s < kCuStages; ++s)
        if (last_par[s] >= 0) wait_bounded(&full[s], (uint32_t)last_par[s], abort_flag, err, kWaitPanel, false);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      uint32_t acc_ph[2] = {0u, 0u};
      int local = 0;
      bool ok = true;
      for (int u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
        const CholUnit w = units[u];
        const bool same = w.bmap == 0 && w.ti == w.tj;
        const int b = local & 1;
        ++local;
        if (!wait_bounded(&tempty[b], acc_ph[b] ^ 1u, abort_flag, err, kWaitPanel, true, wait_ns)) break;
        acc_ph[b] ^= 1u;
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + (uint32_t)(b * kTile);
        for (int kb = 0; kb < kKb; ++kb) {
          if (!wait_bounded(&full[stage], phase, abort_flag, err, kWaitPanel, true, wait_ns)) { ok = false; break; }
          tc_fence_after();
          const uint32_t a0 = saddr(smem + stage * kCuStageBytes);
          const uint64_t ah = sw128_desc(a0), al = sw128_desc(a0 + kOpBytes);
          const uint64_t bh = same ? ah : sw128_desc(a0 + 2 * kOpBytes);
          const uint64_t bl = same ? al : sw128_desc(a0 + 3 * kOpBytes);
#pragma unroll
          for (int k = 0; k < 4; ++k) {  // 4 x 8 TF32 values along K inside the 128-byte row
            const uint64_t o = (uint64_t)(2 * k);
            tc_mma<true, kTile>(d_tmem, al + o, bh + o, (kb > 0 || k > 0) ? 1u : 0u);
            tc_mma<true, kTile>(d_tmem, ah + o, bl + o, 1u);
            tc_mma<true, kTile>(d_tmem, ah + o, bh + o, 1u);
          }
          tc_commit(&empty[stage]);
          if (++stage == kCuStages) { stage = 0; phase ^= 1u; }
        }
        if (!ok) break;
        tc_commit(&tfull[b]);
      }
      tc_commit(drain);
      wait_bounded(drain, 0u, abort_flag, err, kWaitPanel, false);
    }
  } else {
    // Epilogue: C -= accumulator, 32 columns (one chunk) at a time.  While a
    // chunk is written back the old C values of the next chunk (of this unit or
    // of the CTA's next unit) are already in flight, in the other of two
    // register buffers: the loads, not the tensor cores, set the pace of this
    // kernel.  Whole tiles strictly below the diagonal and inside the matrix
    // (all but the diagonal and last tiles) take a path without per-element
    // checks and with 32-bit offsets.
    const int quarter = warp & 3;          // TMEM lanes 32 quarter .. + 31 (the rows of this warp)
    const int cbase = 2 * ((warp - 2) >> 2);  // two warps per quarter: chunks cbase, cbase + 1 of each tile
    uint32_t acc_ph[2] = {0u, 0u};
    int local = 0;
    const int ldi = (int)ld;
    auto interior = [&](const CholUnit &w) {
      return !w.tri && (int64_t)(w.ti + 1) * kTile <= n && (int64_t)(w.tj + 1) * kTile <= n;
    };
    auto load_chunk = [&](const CholUnit &w, int c, float(&dst)[32]) {
      const float *C = w.cbuf ? C1 : C0;
      const int64_t row = (int64_t)w.ti * kTile + quarter * 32 + lane;
      const int64_t col0 = (int64_t)w.tj * kTile + 32 * c;
      const float *src = C + col0 * ld + row;
      if (interior(w)) {
#pragma unroll
        for (int j = 0; j < 32; ++j) dst[j] = src[j * ldi];
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int64_t col = col0 + j;
          dst[j] = (row < n && col < n && (!w.tri || col <= row)) ? src[(int64_t)j * ld] : 0.f;
        }
      }
    };
    auto store_chunk = [&](const CholUnit &w, int b, int c, const float(&old)[32]) {
      uint32_t v[32];
      tmem_ld_32x32b_x32(tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * kTile + 32 * c), v);
      float *C = w.cbuf ? C1 : C0;
      const int64_t row = (int64_t)w.ti * kTile + quarter * 32 + lane;
      const int64_t col0 = (int64_t)w.tj * kTile + 32 * c;
      float *dst = C + col0 * ld + row;
      if (interior(w)) {
#pragma unroll
        for (int j = 0; j < 32; ++j) dst[j * ldi] = old[j] - __uint_as_float(v[j]);
      } else if (row < n) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int64_t col = col0 + j;
          if (col < n && (!w.tri || col <= row)) dst[(int64_t)j * ld] = old[j] - __uint_as_float(v[j]);
        }
      }
    };
    float bufA[32], bufB[32];
    int u = blockIdx.x;
    CholUnit wc{};
    if (u < nunits) {
      wc = units[u];
      load_chunk(wc, cbase, bufA);
    }
    for (; u < nunits; u += gridDim.x) {
      const int un = u + gridDim.x;
      CholUnit wn{};
      if (un < nunits) wn = units[un];
      const int b = local & 1;
      ++local;
      int ok = 0;
      if (lane == 0) ok = wait_bounded(&tfull[b], acc_ph[b], abort_flag, err, kWaitPanel, true, wait_ns) ? 1 : 0;
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) break;
      acc_ph[b] ^= 1u;
      tc_fence_after();
      load_chunk(wc, cbase + 1, bufB);
      store_chunk(wc, b, cbase, bufA);
      if (un < nunits) load_chunk(wn, cbase, bufA);
      store_chunk(wc, b, cbase + 1, bufB);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[b]);
      wc = wn;
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(kTmemCols)
                 : "memory");
  }
}

using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled get_encoder() {
  static EncodeTiled fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
  }
  return fn;
}

}  // namespace

cudaError_t encode_operand_map(OpType t, const void *At, int64_t rows_pad, int64_t ldn, CUtensorMap *out) {
  if (t == OpType::F64) return cudaErrorInvalidValue;
  EncodeTiled enc = get_encoder();
  if (!enc) return cudaErrorNotSupported;
  const bool tf32 = t == OpType::TF32;
  const int bk = tf32 ? kBkTf32 : kBkBf16;
  const size_t esz = tf32 ? 4 : 2;
  if (ldn % bk != 0 || rows_pad % kTile != 0 || (reinterpret_cast<uintptr_t>(At) & 15) != 0)
    return cudaErrorInvalidValue;
  // K-blocked layout [ldn / bk][rows_pad][bk]: one box = 128 rows x 128 bytes, contiguous
  cuuint64_t dims[3] = {(cuuint64_t)bk, (cuuint64_t)rows_pad, (cuuint64_t)(ldn / bk)};
  cuuint64_t strides[2] = {(cuuint64_t)(bk * esz), (cuuint64_t)(rows_pad * bk * esz)};
  cuuint32_t box[3] = {(cuuint32_t)bk, (cuuint32_t)kTile, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(out, tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3,
                   const_cast<void *>(At), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t encode_rows_map(const float *A, int64_t rows, int64_t cols, CUtensorMap *out) {
  EncodeTiled enc = get_encoder();
  if (!enc) return cudaErrorNotSupported;
  if (cols % kBkTf32 != 0 || rows % kTile != 0 || (reinterpret_cast<uintptr_t>(A) & 15) != 0)
    return cudaErrorInvalidValue;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(cols * sizeof(float))};
  cuuint32_t box[2] = {(cuuint32_t)kBkTf32, (cuuint32_t)kTile};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(A), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

int tc_kblocks(OpType t, int64_t ldn) { return (int)(ldn / (t == OpType::TF32 ? kBkTf32 : kBkBf16)); }

int tc_pick_split(int ntiles, int kblocks, int num_sms) {
  // balance the units over the SMs, keep >= 8 K-blocks per split
  int best = 1;
  double best_eff = -1.0;
  const int max_split = std::max(1, std::min(16, kblocks / 8));
  for (int s = 1; s <= max_split; ++s) {
    const int units = ntiles * s;
    const int g = std::min(units, num_sms);
    const int waves = (units + g - 1) / g;
    const double eff = (double)units / ((double)g * waves) * (g / (double)num_sms);
    if (eff > best_eff + 0.02) { best_eff = eff; best = s; }
  }
  return best;
}

int tc_chunk_kblocks(OpType t) { return 16384 / (t == OpType::TF32 ? kBkTf32 : kBkBf16); }

std::vector<SyrkUnit> schedule_syrk_units(const std::vector<SyrkUnit> &jobs, int grid, int max_kb) {
  std::vector<SyrkUnit> out;
  if (jobs.empty() || grid < 1) return out;
  std::vector<size_t> order(jobs.size());
  for (size_t j = 0; j < jobs.size(); ++j) order[j] = j;
  std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) {
    return (jobs[a].kb1 - jobs[a].kb0) > (jobs[b].kb1 - jobs[b].kb0);
  });
  std::vector<std::vector<SyrkUnit>> per((size_t)grid);
  // least-loaded CTA first, lowest index on ties (equal jobs go round-robin)
  using Item = std::pair<int64_t, int>;
  std::priority_queue<Item, std::vector<Item>, std::greater<Item>> heap;
  for (int b = 0; b < grid; ++b) heap.push({0, b});
  for (size_t j : order) {
    const SyrkUnit &w = jobs[j];
    const Item top = heap.top();
    heap.pop();
    const int len = w.kb1 - w.kb0;
    const int nch = std::max(1, (len + max_kb - 1) / max_kb);
    for (int c = 0; c < nch; ++c) {
      SyrkUnit u = w;
      u.kb0 = w.kb0 + (int)((int64_t)len * c / nch);
      u.kb1 = w.kb0 + (int)((int64_t)len * (c + 1) / nch);
      u.flags = c > 0 ? kUnitAcc : 0;
      per[(size_t)top.second].push_back(u);
    }
    heap.push({top.first + len + 8, top.second});  // 8 K-blocks of fixed cost per job
  }
  // Within a CTA, the chunks of its jobs are taken chunk-major (the first chunk of
  // every job, then the second, ...; a job's chunks keep their order, so stores
  // still precede adds): all CTAs then walk the same observation range at the
  // same time however long the jobs are, which keeps the operand rows in L2.
  for (auto &v : per) {
    std::vector<std::vector<SyrkUnit>> jobs_of;
    for (const SyrkUnit &u : v) {
      if (!(u.flags & kUnitAcc)) jobs_of.emplace_back();
      jobs_of.back().push_back(u);
    }
    std::vector<SyrkUnit> out2;
    for (size_t c = 0;; ++c) {
      bool any = false;
      for (const auto &j : jobs_of)
        if (c < j.size()) { out2.push_back(j[c]); any = true; }
      if (!any) break;
    }
    v.swap(out2);
  }
  size_t depth = 0;
  for (const auto &v : per) depth = std::max(depth, v.size());
  SyrkUnit empty{};
  empty.flags = kUnitEmpty;
  out.assign(depth * (size_t)grid, empty);
  for (int b = 0; b < grid; ++b)
    for (size_t i = 0; i < per[(size_t)b].size(); ++i) out[i * (size_t)grid + (size_t)b] = per[(size_t)b][i];
  return out;
}

size_t tc_smem_bytes() { return TcCfg<kTile>::kSmemBytes; }

template <bool TF32, int BN>
cudaError_t launch_tc(const CUtensorMap *maps, const SyrkUnit *units, int nunits, const int *active, int grid,
                      float *out, int *err, cudaStream_t st, uint64_t wait_ns) {
  auto kern = syrk_tc_kernel<TF32, BN>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, TcCfg<BN>::kSmemBytes);
  if (e != cudaSuccess) return e;
  kern<<<grid, 192, TcCfg<BN>::kSmemBytes, st>>>(maps, units, nunits, active, out, err,
                                                 wait_ns ? wait_ns : kTimeoutNs);
  return cudaGetLastError();
}

cudaError_t launch_syrk_tc(OpType t, const CUtensorMap *maps, const SyrkUnit *units, int nunits, const int *active,
                           int grid, float *out, int *err, cudaStream_t st, int bn, uint64_t wait_ns) {
  if (nunits <= 0) return cudaSuccess;
  if (bn == 256)
    return t == OpType::TF32 ? launch_tc<true, 256>(maps, units, nunits, active, grid, out, err, st, wait_ns)
                             : launch_tc<false, 256>(maps, units, nunits, active, grid, out, err, st, wait_ns);
  return t == OpType::TF32 ? launch_tc<true, 128>(maps, units, nunits, active, grid, out, err, st, wait_ns)
                           : launch_tc<false, 128>(maps, units, nunits, active, grid, out, err, st, wait_ns);
}

size_t chol_update_smem_bytes() { return kCuSmemBytes; }

cudaError_t chol_update_tc_setup() {
  return cudaFuncSetAttribute(chol_update_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kCuSmemBytes);
}

cudaError_t launch_chol_update_tc(const CUtensorMap *maps, const CholUnit *units, int nunits, int grid, float *C0,
                                  float *C1, int64_t ld, int64_t n, int *err, uint64_t wait_ns, cudaStream_t st) {
  if (nunits <= 0) return cudaSuccess;
  chol_update_tc_kernel<<<grid, kCuThreads, kCuSmemBytes, st>>>(maps, units, nunits, C0, C1, ld, n, err,
                                                         wait_ns ? wait_ns : kTimeoutNs);
  return cudaGetLastError();
}

}  // namespace mnl
