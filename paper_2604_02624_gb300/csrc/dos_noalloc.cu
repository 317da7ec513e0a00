// dos_noalloc.cu - scoring entry point that allocates no memory.
//
// dos_loss keeps its per-channel statistics in workspace that dos_create
// allocates.  Some callers cannot allocate device memory at all: code that
// runs inside a host framework owning every byte of the device through its
// own pool, code with a fixed memory budget decided at start-up, or code on a
// path where a cudaMalloc would synchronise the device.  dos_loss_noalloc
// serves them: the same statistics kernels, with their scratch in a
// file-scope __device__ array of fixed size that every GPU loading this
// library holds until the process exits.
#include <cuda.h>

#include <mutex>
#include <string>

#include "../../include/dos.h"
#include "dos_internal.h"

namespace dos {
namespace {

// Scratch shared by every call on a device: per-channel statistics and the
// loss scalar.  The kernels write every entry they later read, so nothing
// has to be cleared between calls.
static __device__ __align__(256) LossStats g_noalloc_stats[DOS_NOALLOC_MAX_LAMBDA];
static __device__ __align__(256) double g_noalloc_loss;

constexpr int kThreads = 256;

__device__ __forceinline__ double block_sum_na(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

// Same statistics as the context's loss kernel, read from intensities.
__global__ void __launch_bounds__(kThreads) k_stats_from_intensity(const float* __restrict__ I,
                                                                   const float* __restrict__ T,
                                                                   LossStats* __restrict__ st,
                                                                   int fov2) {
  __shared__ double sh[kThreads];
  const int w = blockIdx.x;
  const float* iw = I + (size_t)w * fov2;
  const float* tw = T + (size_t)w * fov2;
  double sse = 0, sit = 0, sii = 0;
  for (int p = threadIdx.x; p < fov2; p += kThreads) {
    const double i = iw[p];
    const double t = tw[p];
    sse += (i - t) * (i - t);
    sit += i * t;
    sii += i * i;
  }
  sse = block_sum_na(sse, sh);
  sit = block_sum_na(sit, sh);
  sii = block_sum_na(sii, sh);
  const double sigma = sii > 0.0 ? sit / sii : 0.0;
  double ssc = 0;
  for (int p = threadIdx.x; p < fov2; p += kThreads) {
    const double d = sigma * (double)iw[p] - (double)tw[p];
    ssc += d * d;
  }
  ssc = block_sum_na(ssc, sh);
  if (threadIdx.x == 0) {
    LossStats s;
    s.sse = sse;
    s.sigma = sigma;
    s.sse_sc = ssc;
    s.pad = 0;
    st[w] = s;
  }
}

__global__ void k_dldi_from_intensity(const float* __restrict__ I, const float* __restrict__ T,
                                      const LossStats* __restrict__ st, float* __restrict__ dLdI,
                                      size_t total, int fov2, double norm, int mode) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const double v = I[i];
  double g;
  if (mode == DOS_LOSS_MSE_SCALED) {
    const double sg = st[i / fov2].sigma;
    g = 2.0 * sg * (sg * v - (double)T[i]) / norm;
  } else {
    g = 2.0 * (v - (double)T[i]) / norm;
  }
  dLdI[i] = (float)g;
}

// Device addresses of the scratch, looked up with the device current (host
// code cannot use the symbols' names as addresses).  The addresses belong to
// the context the module was loaded in, so each device's entry remembers that
// context's process-unique id and is looked up again under another one (a
// primary context recreated after cudaDeviceReset, a caller's own driver
// context).
constexpr int kMaxDevices = 64;
struct Scratch {
  LossStats* stats = nullptr;
  double* loss = nullptr;
  unsigned long long ctx_id = 0;
};
Scratch g_scratch[kMaxDevices];
std::mutex g_scratch_mu;

int na_fail(int code, const std::string& msg) {
  set_last_error(msg.c_str());
  return code;
}

// Process-unique id of the calling thread's current context (cuCtxGetId,
// found through the runtime's driver entry points); 0 when it cannot be told,
// and then the addresses are looked up on every call.
unsigned long long current_context_id() {
  using GetCurrent = CUresult (*)(CUcontext*);
  using GetId = CUresult (*)(CUcontext, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<GetCurrent>(fn);
    fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<GetId>(fn);
    (void)cudaGetLastError();
  });
  if (!get_current || !get_id) return 0;
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

int scratch_for_current_device(Scratch* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return na_fail(DOS_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return na_fail(DOS_ERR_UNSUPPORTED, "device index beyond 63");
  // 0 also when no context is current yet: the lookup below binds the
  // runtime's context to the thread, and the entry records that one
  const unsigned long long ctx_id = current_context_id();
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  Scratch& s = g_scratch[dev];
  if (!s.stats || ctx_id == 0 || s.ctx_id != ctx_id) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_stats);
    if (e != cudaSuccess)
      return na_fail(DOS_ERR_CUDA, std::string("cudaGetSymbolAddress(stats): ") + cudaGetErrorString(e));
    void* q = nullptr;
    e = cudaGetSymbolAddress(&q, g_noalloc_loss);
    if (e != cudaSuccess)
      return na_fail(DOS_ERR_CUDA, std::string("cudaGetSymbolAddress(loss): ") + cudaGetErrorString(e));
    s.stats = static_cast<LossStats*>(p);
    s.loss = static_cast<double*>(q);
    s.ctx_id = current_context_id();
  }
  *out = s;
  return DOS_OK;
}

}  // namespace
}  // namespace dos

extern "C" {

DOS_API int dos_loss_noalloc(const float* d_I, const float* d_T, int n_lambda, int fov,
                             int n_lambda_total, int loss, double* h_loss, float* d_psnr,
                             float* d_dLdI, void* cuda_stream) {
  using namespace dos;
  if (!d_I || !d_T) return na_fail(DOS_ERR_ARG, "d_I and d_T are required");
  if (n_lambda < 1 || n_lambda > DOS_NOALLOC_MAX_LAMBDA)
    return na_fail(DOS_ERR_ARG, "n_lambda must be in [1, " + std::to_string(DOS_NOALLOC_MAX_LAMBDA) +
                                    "] for dos_loss_noalloc (its scratch has a fixed size)");
  if (fov < 1 || fov > 16384) return na_fail(DOS_ERR_ARG, "fov must be in [1, 16384]");
  if (n_lambda_total != 0 && n_lambda_total < n_lambda)
    return na_fail(DOS_ERR_ARG, "n_lambda_total must be 0 or >= n_lambda");
  if (loss != DOS_LOSS_MSE && loss != DOS_LOSS_MSE_SCALED)
    return na_fail(DOS_ERR_ARG, "loss must be DOS_LOSS_MSE or DOS_LOSS_MSE_SCALED");
  Scratch s;
  int rc = scratch_for_current_device(&s);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int fov2 = fov * fov;
  const double norm = (double)(n_lambda_total ? n_lambda_total : n_lambda) * fov2;
  k_stats_from_intensity<<<n_lambda, kThreads, 0, st>>>(d_I, d_T, s.stats, fov2);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = launch_loss_final(s.stats, n_lambda, fov2, norm, loss, s.loss, d_psnr, st);
  if (e == cudaSuccess && d_dLdI) {
    const size_t total = (size_t)n_lambda * fov2;
    k_dldi_from_intensity<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(d_I, d_T, s.stats, d_dLdI, total,
                                                                          fov2, norm, loss);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && h_loss) {
    e = cudaMemcpyAsync(h_loss, s.loss, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  if (e != cudaSuccess) return na_fail(DOS_ERR_CUDA, std::string("dos_loss_noalloc: ") + cudaGetErrorString(e));
  return DOS_OK;
}

}  // extern "C"
