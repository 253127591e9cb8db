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
// address: the device address is looked up once per device with
// cudaGetSymbolAddress (with that device current) and cached.
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

std::mutex g_addr_mutex;
void* g_addr[kMaxDevices] = {};

// Device address of g_static_scratch on `dev` (the current device), cached.
traknn_status scratch_address(int dev, char** out) {
  std::lock_guard<std::mutex> lock(g_addr_mutex);
  if (dev < 0 || dev >= kMaxDevices) return TRAKNN_ERR_INVALID_ARG;
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return TRAKNN_ERR_CUDA;
    }
    g_addr[dev] = p;
  }
  *out = static_cast<char*>(g_addr[dev]);
  return TRAKNN_OK;
}

inline size_t up256(size_t v) { return (v + 255) / 256 * 256; }

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

  // work split: the same rule as the handle-based call with automatic chunks
  const int M = (int)(N - L + 1);
  Schedule s;
  s.M = M;
  s.L = L;
  s.k = k;
  s.e = exclusion;
  s.rows_out = kTileRows - (L - 1);
  s.strips = (M + s.rows_out - 1) / s.rows_out;
  const int chunks = std::max(1, std::min(8, M));
  s.chunk_cols = (M + chunks - 1) / chunks;
  s.chunks = (M + s.chunk_cols - 1) / s.chunk_cols;
  s.group_strips = std::max(1, sms / s.chunks);
  s.units = ((s.strips + s.group_strips - 1) / s.group_strips) * s.group_strips * s.chunks;

  // scratch layout inside the static array
  const int Dp = (int)((D + 31) / 32 * 32);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = up256(off + bytes);
    return o;
  };
  const size_t o_err = take(sizeof(int));
  const size_t o_partial = take((size_t)kMeanSlices * D * sizeof(float));
  const size_t o_mu = take((size_t)D * sizeof(float));
  const size_t o_norms = take((size_t)N * sizeof(double));
  const size_t o_W = take((size_t)M * sizeof(float));
  const size_t o_Xc = take((size_t)N * Dp * sizeof(float));
  const size_t o_pd = take((size_t)M * s.chunks * k * sizeof(float));
  const size_t o_pi = take((size_t)M * s.chunks * k * sizeof(int32_t));
  if (off > kStaticScratchBytes) return TRAKNN_ERR_SCRATCH_LIMIT;

  char* base = nullptr;
  st = scratch_address(dev, &base);
  if (st != TRAKNN_OK) return st;
  cudaStream_t cs = static_cast<cudaStream_t>(stream);

  FusedArgs a;
  a.sch = s;
  a.N = (int)N;
  a.Dp = Dp;
  float* W = reinterpret_cast<float*>(base + o_W);
  a.W = W;
  a.part_d = reinterpret_cast<float*>(base + o_pd);
  a.part_i = reinterpret_cast<int32_t*>(base + o_pi);
  a.err = reinterpret_cast<int*>(base + o_err);
  a.wait_limit_ns = 2000000000LL;
  a.debug_withhold = 0;
  float* partial = reinterpret_cast<float*>(base + o_partial);
  float* mu = reinterpret_cast<float*>(base + o_mu);
  double* norms = reinterpret_cast<double*>(base + o_norms);
  float* Xc = reinterpret_cast<float*>(base + o_Xc);

  // the status word is the only scratch that must start at zero; every other
  // byte a kernel reads is written earlier in this same call
  if (cudaMemsetAsync(a.err, 0, sizeof(int), cs) != cudaSuccess ||
      launch_col_mean(X, (int)N, (int)D, partial, mu, true, cs) != cudaSuccess ||
      launch_prep_fp32(X, (int)N, (int)D, Dp, mu, nullptr, Xc, norms, cs) != cudaSuccess ||
      launch_window(norms, M, L, W, cs) != cudaSuccess ||
      launch_fused_fp32(Xc, a, sms, cs) != cudaSuccess ||
      launch_merge(a, nbr_idx, nbr_dist, score, cs) != cudaSuccess) {
    cudaGetLastError();
    return TRAKNN_ERR_CUDA;
  }
  return TRAKNN_OK;
}
