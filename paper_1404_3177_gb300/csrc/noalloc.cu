// mnl_loglik_grad_noalloc: the log-likelihood / gradient pass for callers that
// must not allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they need l and g:
// code running inside a memory pool or arena that owns all device memory,
// plug-ins of a host application that forbids allocation after start-up, and
// real-time loops where an allocation (which can synchronise the device or
// fail when memory is fragmented) is not allowed.  This entry point takes all
// of its inputs and outputs from the caller and keeps the only scratch it
// needs - the per-CTA partial sums of the pass - in a fixed array that is part
// of the library image on every GPU that loads it.
#include <mutex>

#include "mnl_internal.cuh"

namespace {

// Scratch: [0] l, [1] sum |l_i| (reduction outputs), then the CTA partials.
constexpr size_t kScratchDoubles = size_t(1) << 19;  // 4 MiB per GPU
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

// Largest raw gradient count (K-1)(p+d) + K f of the pass this entry point runs
// (512 threads x 32 accumulators), and its largest K.
constexpr int64_t kMaxOutputs = 16384;
constexpr int kMaxK = 256;

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
// Per device: the array's device address and the context it was looked up in.
// A device reset (or a new primary context) changes the context, and the
// address is then looked up again instead of being reused.
double *g_scratch_addr[kMaxDevices] = {};
CUcontext g_scratch_ctx[kMaxDevices] = {};

using CtxGetCurrent = CUresult (*)(CUcontext *);
CtxGetCurrent ctx_get_current() {
  static CtxGetCurrent fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<CtxGetCurrent>(p);
  }
  return fn;
}

// Device address of the scratch array on the current device (looked up once per
// device and context, with that device current).
cudaError_t scratch_address(int dev, double **out) {
  std::lock_guard<std::mutex> lock(g_mutex);
  CUcontext ctx = nullptr;
  CtxGetCurrent get = ctx_get_current();
  if (!get || get(&ctx) != CUDA_SUCCESS || !ctx) return cudaErrorInitializationError;
  if (!g_scratch_addr[dev] || g_scratch_ctx[dev] != ctx) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<double *>(p);
    g_scratch_ctx[dev] = ctx;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

__global__ void copy_scalar_kernel(const double *src, double *dst) { *dst = *src; }

}  // namespace

extern "C" MNL_API int mnl_loglik_grad_noalloc(const mnl_dims *dims, const mnl_data *data, int precision,
                                               const double *theta, double *loglik, double *grad, void *P,
                                               void *zbar, void *stream) {
  using namespace mnl;
  if (!dims || !data || !theta || !loglik || !grad || !P) return MNL_ERR_INVALID_ARG;
  if (dims->N < 1 || dims->K < 2 || dims->p < 0 || dims->d < 0 || dims->f < 0 || dims->p + dims->d + dims->f < 1)
    return MNL_ERR_INVALID_ARG;
  if (dims->gamma_base != 0) return MNL_ERR_UNSUPPORTED;
  if (precision < MNL_FP64 || precision > MNL_BF16) return MNL_ERR_INVALID_ARG;
  if (!data->choice || (dims->p > 0 && !data->X) || (dims->d > 0 && !data->Y) || (dims->f > 0 && !data->Z) ||
      (dims->f > 0 && !zbar))
    return MNL_ERR_INVALID_ARG;
  const Shape S = make_shape(*dims);
  const bool fp64 = precision == MNL_FP64;
  // sizes beyond the limits are refused before any CUDA call
  if (S.nout > kMaxOutputs || S.K > kMaxK) return MNL_ERR_UNSUPPORTED;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) { cudaGetLastError(); return MNL_ERR_CUDA; }
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return MNL_ERR_CUDA;
  }
  PassPlan pl = plan_pass(S, fp64, true, nsm, false);
  if (!pl.ok) return MNL_ERR_UNSUPPORTED;
  // Fit the CTA partials into the fixed scratch: fewer CTAs when needed.
  const size_t per_cta = 2 + (size_t)S.n;
  if (2 + per_cta > kScratchDoubles) return MNL_ERR_UNSUPPORTED;
  const size_t max_grid = (kScratchDoubles - 2) / per_cta;
  if ((size_t)pl.grid > max_grid) pl.grid = (int)max_grid;
  double *scratch = nullptr;
  if (scratch_address(dev, &scratch) != cudaSuccess) { cudaGetLastError(); return MNL_ERR_CUDA; }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  PassIO io{};
  io.X = data->X; io.Y = data->Y; io.Z = data->Z; io.choice = data->choice;
  io.theta = theta; io.delta = nullptr; io.tscale = nullptr;
  io.P = P; io.zbar = zbar;
  io.partials = scratch + 2;
  if (launch_pass(S, pl, fp64, true, io, st) != cudaSuccess ||
      launch_pass_reduce(S, pl.grid, true, io.partials, scratch, grad, st) != cudaSuccess) {
    cudaGetLastError();
    return MNL_ERR_CUDA;
  }
  copy_scalar_kernel<<<1, 1, 0, st>>>(scratch, loglik);
  if (cudaGetLastError() != cudaSuccess) return MNL_ERR_CUDA;
  return MNL_OK;
}
