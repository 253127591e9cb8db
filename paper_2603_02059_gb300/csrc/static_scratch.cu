// static_scratch.cu -- a forward entry point that allocates no device memory.
//
// Some callers cannot call cudaMalloc: their device memory is owned by another
// allocator or held to a fixed budget, or they cannot accept the device-wide
// synchronisation that cudaMalloc/cudaFree may cause. traknn_knn_scores needs a
// handle whose workspace grows with cudaMalloc; this entry point needs neither.
// Its scratch is one file-scope __device__ array of kStaticScratchBytes that every
// GPU loading the library keeps until the process exits. It runs the FP32
// CUDA-core path with the same kernels and work split as the handle-based call.
//
// In host code the array's name is only a host-side stand-in, never a device
// address. Its device address is looked up with cudaGetSymbolAddress (with the
// device current) and cached per device and CUDA context: after the device's primary
// context is torn down (cudaDeviceReset) the module is loaded again and the array can
// move, so a new context means a new lookup.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "../../include/traknn.h"
#include "internal.h"

namespace traknn {
namespace {

constexpr size_t kStaticScratchBytes = size_t(32) << 20;  // 32 MiB
constexpr int kMaxDevices = 128;

__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

std::mutex g_addr_mutex;
void* g_addr[kMaxDevices] = {};
unsigned long long g_ctx_id[kMaxDevices] = {};

// Identity of the calling thread's current CUDA context (0 when there is none or the
// driver entry points are unavailable).
unsigned long long current_context_id() {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {
    looked_up = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<CtxGetCurrentFn>(p);
    p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<CtxGetIdFn>(p);
    cudaGetLastError();
  }
  if (!get_current || !get_id) return 0;
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr) return 0;
  if (get_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

// Device address of g_static_scratch on `dev` (the current device). Cached per device
// and context; looked up on every call when the context cannot be identified.
traknn_status scratch_address(int dev, char** out) {
  std::lock_guard<std::mutex> lock(g_addr_mutex);
  if (dev < 0 || dev >= kMaxDevices) return TRAKNN_ERR_INVALID_ARG;
  const unsigned long long id = current_context_id();
  if (!g_addr[dev] || id == 0 || id != g_ctx_id[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      g_addr[dev] = nullptr;
      return TRAKNN_ERR_CUDA;
    }
    g_addr[dev] = p;
    // the lookup makes the primary context current if it was not yet
    g_ctx_id[dev] = id != 0 ? id : current_context_id();
  }
  *out = static_cast<char*>(g_addr[dev]);
  return TRAKNN_OK;
}

}  // namespace
}  // namespace traknn

using namespace traknn;

extern "C" traknn_status traknn_knn_scores_static(const float* X, int64_t N, int64_t D, int L,
                                                  int k, int exclusion, int32_t* nbr_idx,
                                                  float* nbr_dist, float* score, void* stream) {
  if (!X || !nbr_idx || !nbr_dist || !score) return TRAKNN_ERR_INVALID_ARG;
  traknn_status st = traknn_check_problem(N, D, L, k, exclusion);
  if (st != TRAKNN_OK) return st;
  int dev = 0, major = 0, minor = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return TRAKNN_ERR_CUDA;
  }
  if (major != 10 || minor != 3) return TRAKNN_ERR_UNSUPPORTED_DEVICE;

  // work split and scratch layout: those of the handle-based FP32 call with
  // automatic column chunks, plus the status word after the layout
  const int M = (int)(N - L + 1);
  const Schedule s = make_schedule(M, L, k, exclusion, sms, 0);
  const Fp32Layout lay = make_layout(N, D, s);
  const size_t o_err = (lay.total + 255) / 256 * 256;
  if (o_err + 256 > kStaticScratchBytes) return TRAKNN_ERR_SCRATCH_LIMIT;

  char* base = nullptr;
  st = scratch_address(dev, &base);
  if (st != TRAKNN_OK) return st;
  cudaStream_t cs = static_cast<cudaStream_t>(stream);

  FusedArgs a;
  a.sch = s;
  a.N = (int)N;
  a.Dp = lay.Dp;
  float* W = reinterpret_cast<float*>(base + lay.W);
  a.W = W;
  a.part_d = reinterpret_cast<float*>(base + lay.pd);
  a.part_i = reinterpret_cast<int32_t*>(base + lay.pi);
  a.err = reinterpret_cast<int*>(base + o_err);
  a.wait_limit_ns = 2000000000LL;
  a.debug_withhold = 0;
  float* partial = reinterpret_cast<float*>(base + lay.partial);
  float* mu = reinterpret_cast<float*>(base + lay.mu);
  double* norms = reinterpret_cast<double*>(base + lay.norms);
  float* Xc = reinterpret_cast<float*>(base + lay.ops);

  // the status word is the only scratch that must start at zero; every other
  // byte a kernel reads is written earlier in this same call
  if (cudaMemsetAsync(a.err, 0, sizeof(int), cs) != cudaSuccess ||
      launch_col_mean(X, (int)N, (int)D, partial, mu, true, cs) != cudaSuccess ||
      launch_prep_fp32(X, (int)N, (int)D, lay.Dp, mu, nullptr, Xc, norms, cs) != cudaSuccess ||
      launch_window(norms, M, L, W, cs) != cudaSuccess ||
      launch_fused_fp32(Xc, a, sms, cs) != cudaSuccess ||
      launch_merge(a, nbr_idx, nbr_dist, score, cs) != cudaSuccess) {
    cudaGetLastError();
    return TRAKNN_ERR_CUDA;
  }
  return TRAKNN_OK;
}
