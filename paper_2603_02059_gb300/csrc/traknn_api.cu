// traknn_api.cu -- the C ABI declared in include/traknn.h: argument checks,
// workspace management and the launch sequence of the forward and backward
// passes. All arithmetic runs in the kernels of the other translation units.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdint>
#include <cstring>
#include <new>

#include "../../include/traknn.h"
#include "internal.h"

using namespace traknn;

struct traknn_ctx {
  int device = 0;
  int sm_count = 0;
  traknn_precision precision = TRAKNN_PREC_SPLIT_BF16;
  int center = 1;
  int col_chunks = 0;
  int wait_limit_ms = 2000;
  int debug_withhold = 0;
  // library-owned buffers, grown on demand
  void* ws = nullptr;
  size_t ws_bytes = 0;
  void* io = nullptr;  // device staging for the host-buffer entry point
  size_t io_bytes = 0;
  void* adj = nullptr;  // reverse neighbour index of the adjoint
  size_t adj_bytes = 0;
  int* err = nullptr;  // device status word
  // profiling of the fused kernel
  int profile = 0;
  static constexpr int kRing = 256;
  cudaEvent_t ev_start[kRing] = {};
  cudaEvent_t ev_stop[kRing] = {};
  int ev_head = 0, ev_count = 0;
  int64_t launches = 0;
};

namespace {

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }


#define TRY_CUDA(expr)                              \
  do {                                              \
    cudaError_t e_ = (expr);                        \
    if (e_ != cudaSuccess) return TRAKNN_ERR_CUDA;  \
  } while (0)

traknn_status ensure_buffer(void** buf, size_t* have, size_t need) {
  if (*have >= need) return TRAKNN_OK;
  if (*buf) {
    cudaDeviceSynchronize();
    cudaFree(*buf);
    *buf = nullptr;
    *have = 0;
  }
  size_t bytes = align_up(need + need / 8, 1 << 20);
  if (cudaMalloc(buf, bytes) != cudaSuccess) {
    cudaGetLastError();
    *buf = nullptr;
    return TRAKNN_ERR_ALLOC;
  }
  *have = bytes;
  return TRAKNN_OK;
}

// Work split of the M x M pair space (see Schedule in internal.h).
Schedule make_schedule(int M, int L, int k, int e, int sm_count, int chunks_opt) {
  Schedule s;
  s.M = M;
  s.L = L;
  s.k = k;
  s.e = e;
  s.rows_out = kTileRows - (L - 1);
  s.strips = (M + s.rows_out - 1) / s.rows_out;
  int chunks = chunks_opt > 0 ? chunks_opt : 8;
  chunks = std::min(chunks, 32);
  chunks = std::max(1, std::min(chunks, M));
  s.chunk_cols = (M + chunks - 1) / chunks;
  s.chunks = (M + s.chunk_cols - 1) / s.chunk_cols;  // every chunk non-empty
  s.group_strips = std::max(1, sm_count / s.chunks);
  const int groups = (s.strips + s.group_strips - 1) / s.group_strips;
  s.units = groups * s.group_strips * s.chunks;
  return s;
}

struct Layout {
  size_t partial, mu, norms, W, ops, pd, pi, total;
  int Dp;
};

Layout make_layout(int64_t N, int64_t D, const Schedule& s) {
  Layout l;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    off = align_up(off, 256);
    size_t o = off;
    off += bytes;
    return o;
  };
  l.Dp = (int)align_up((size_t)D, 32);
  l.partial = take((size_t)kMeanSlices * D * sizeof(float));
  l.mu = take((size_t)D * sizeof(float));
  l.norms = take((size_t)N * sizeof(double));
  l.W = take((size_t)s.M * sizeof(float));
  // FP32 centred copy, or hi and lo BF16 copies: 4 bytes per element either way
  l.ops = take((size_t)N * l.Dp * 4);
  l.pd = take((size_t)s.M * s.chunks * s.k * sizeof(float));
  l.pi = take((size_t)s.M * s.chunks * s.k * sizeof(int32_t));
  l.total = off;
  return l;
}

traknn_status check_handle(traknn_handle h) {
  if (!h) return TRAKNN_ERR_INVALID_ARG;
  if (cudaSetDevice(h->device) != cudaSuccess) return TRAKNN_ERR_CUDA;
  return TRAKNN_OK;
}

}  // namespace

extern "C" {

const char* traknn_status_string(traknn_status s) {
  switch (s) {
    case TRAKNN_OK: return "ok";
    case TRAKNN_ERR_INVALID_ARG: return "invalid argument";
    case TRAKNN_ERR_TOO_FEW_CANDIDATES: return "k exceeds the candidate count of some row";
    case TRAKNN_ERR_ALLOC: return "workspace allocation failed";
    case TRAKNN_ERR_CUDA: return "CUDA runtime error";
    case TRAKNN_ERR_TIMEOUT: return "a bounded device-side wait ran out";
    case TRAKNN_ERR_UNSUPPORTED_DEVICE: return "device is not sm_103";
    case TRAKNN_ERR_UNSUPPORTED: return "L or k above the compiled limits";
    case TRAKNN_ERR_SCRATCH_LIMIT: return "problem exceeds the fixed scratch array of the static entry point";
  }
  return "unknown status";
}

traknn_status traknn_check_problem(int64_t N, int64_t D, int L, int k, int exclusion) {
  if (N < 1 || D < 1 || L < 1 || k < 1 || exclusion < 0) return TRAKNN_ERR_INVALID_ARG;
  if (L > N) return TRAKNN_ERR_INVALID_ARG;
  if (N > INT_MAX / 2 || D > INT_MAX / 2) return TRAKNN_ERR_INVALID_ARG;
  if (L > TRAKNN_MAX_L || k > TRAKNN_MAX_K) return TRAKNN_ERR_UNSUPPORTED;
  const int64_t M = N - L + 1;
  // the tightest row (away from both ends) has M - (2e+1) candidates
  if ((int64_t)k > M - (2 * (int64_t)exclusion + 1)) return TRAKNN_ERR_TOO_FEW_CANDIDATES;
  return TRAKNN_OK;
}

traknn_status traknn_create(traknn_handle* out, int device) {
  if (!out) return TRAKNN_ERR_INVALID_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
    cudaGetLastError();
    return TRAKNN_ERR_CUDA;
  }
  if (device < 0 || device >= ndev) return TRAKNN_ERR_INVALID_ARG;
  cudaDeviceProp prop;
  TRY_CUDA(cudaGetDeviceProperties(&prop, device));
  if (prop.major != 10 || prop.minor != 3) return TRAKNN_ERR_UNSUPPORTED_DEVICE;
  TRY_CUDA(cudaSetDevice(device));
  traknn_ctx* h = new (std::nothrow) traknn_ctx();
  if (!h) return TRAKNN_ERR_ALLOC;
  h->device = device;
  h->sm_count = prop.multiProcessorCount;
  if (cudaMalloc(&h->err, 256) != cudaSuccess) {
    delete h;
    return TRAKNN_ERR_ALLOC;
  }
  cudaMemset(h->err, 0, 256);
  *out = h;
  return TRAKNN_OK;
}

traknn_status traknn_destroy(traknn_handle h) {
  if (!h) return TRAKNN_ERR_INVALID_ARG;
  cudaSetDevice(h->device);
  cudaDeviceSynchronize();
  if (h->ws) cudaFree(h->ws);
  if (h->io) cudaFree(h->io);
  if (h->adj) cudaFree(h->adj);
  if (h->err) cudaFree(h->err);
  for (int i = 0; i < traknn_ctx::kRing; ++i) {
    if (h->ev_start[i]) cudaEventDestroy(h->ev_start[i]);
    if (h->ev_stop[i]) cudaEventDestroy(h->ev_stop[i]);
  }
  delete h;
  return TRAKNN_OK;
}

traknn_status traknn_set_option(traknn_handle h, traknn_option opt, int64_t v) {
  if (!h) return TRAKNN_ERR_INVALID_ARG;
  switch (opt) {
    case TRAKNN_OPT_PRECISION:
      if (v < TRAKNN_PREC_FP32 || v > TRAKNN_PREC_BF16) return TRAKNN_ERR_INVALID_ARG;
      h->precision = (traknn_precision)v;
      return TRAKNN_OK;
    case TRAKNN_OPT_CENTER:
      h->center = v ? 1 : 0;
      return TRAKNN_OK;
    case TRAKNN_OPT_COL_CHUNKS:
      if (v < 0 || v > 32) return TRAKNN_ERR_INVALID_ARG;
      h->col_chunks = (int)v;
      return TRAKNN_OK;
    case TRAKNN_OPT_WAIT_LIMIT_MS:
      if (v < 1 || v > 600000) return TRAKNN_ERR_INVALID_ARG;
      h->wait_limit_ms = (int)v;
      return TRAKNN_OK;
    case TRAKNN_OPT_DEBUG_WITHHOLD:
      h->debug_withhold = v ? 1 : 0;
      return TRAKNN_OK;
    case TRAKNN_OPT_PROFILE:
      if (v && !h->ev_start[0]) {
        if (cudaSetDevice(h->device) != cudaSuccess) return TRAKNN_ERR_CUDA;
        for (int i = 0; i < traknn_ctx::kRing; ++i) {
          TRY_CUDA(cudaEventCreate(&h->ev_start[i]));
          TRY_CUDA(cudaEventCreate(&h->ev_stop[i]));
        }
      }
      h->profile = v ? 1 : 0;
      h->ev_head = h->ev_count = 0;
      return TRAKNN_OK;
  }
  return TRAKNN_ERR_INVALID_ARG;
}

traknn_status traknn_knn_scores(traknn_handle h, const float* X, int64_t N, int64_t D, int L,
                                int k, int e, int32_t* nbr_idx, float* nbr_dist, float* score,
                                void* stream) {
  traknn_status st = check_handle(h);
  if (st != TRAKNN_OK) return st;
  if (!X || !nbr_idx || !nbr_dist || !score) return TRAKNN_ERR_INVALID_ARG;
  st = traknn_check_problem(N, D, L, k, e);
  if (st != TRAKNN_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int M = (int)(N - L + 1);

  const Schedule sch = make_schedule(M, L, k, e, h->sm_count, h->col_chunks);
  const Layout lay = make_layout(N, D, sch);
  st = ensure_buffer(&h->ws, &h->ws_bytes, lay.total);
  if (st != TRAKNN_OK) return st;
  char* ws = static_cast<char*>(h->ws);
  float* partial = reinterpret_cast<float*>(ws + lay.partial);
  float* mu = reinterpret_cast<float*>(ws + lay.mu);
  double* norms = reinterpret_cast<double*>(ws + lay.norms);
  float* W = reinterpret_cast<float*>(ws + lay.W);
  void* ops = ws + lay.ops;

  FusedArgs fa;
  fa.sch = sch;
  fa.N = (int)N;
  fa.Dp = lay.Dp;
  fa.W = W;
  fa.part_d = reinterpret_cast<float*>(ws + lay.pd);
  fa.part_i = reinterpret_cast<int32_t*>(ws + lay.pi);
  fa.err = h->err;
  fa.wait_limit_ns = (long long)h->wait_limit_ms * 1000000LL;
  fa.debug_withhold = h->debug_withhold;

  if (h->precision != TRAKNN_PREC_FP32 && !tc_available()) return TRAKNN_ERR_UNSUPPORTED;
  TRY_CUDA(launch_col_mean(X, (int)N, (int)D, partial, mu, h->center != 0, s));
  h->launches += h->center ? 2 : 1;
  const int slot = h->ev_head;
  void* hi = ops;
  void* lo = static_cast<char*>(ops) + (size_t)N * lay.Dp * 2;
  if (h->precision == TRAKNN_PREC_FP32)
    TRY_CUDA(launch_prep_fp32(X, (int)N, (int)D, lay.Dp, mu, static_cast<float*>(ops), norms, s));
  else
    TRY_CUDA(launch_prep_split(X, (int)N, (int)D, lay.Dp, mu, hi, lo, norms, s));
  TRY_CUDA(launch_window(norms, M, L, W, s));
  if (h->profile) TRY_CUDA(cudaEventRecord(h->ev_start[slot], s));
  if (h->precision == TRAKNN_PREC_FP32)
    TRY_CUDA(launch_fused_fp32(static_cast<float*>(ops), fa, h->sm_count, s));
  else
    TRY_CUDA(launch_fused_tc(hi, lo, h->precision == TRAKNN_PREC_SPLIT_BF16, fa, h->sm_count, s));
  if (h->profile) {
    TRY_CUDA(cudaEventRecord(h->ev_stop[slot], s));
    h->ev_head = (h->ev_head + 1) % traknn_ctx::kRing;
    h->ev_count = std::min(h->ev_count + 1, traknn_ctx::kRing);
  }
  TRY_CUDA(launch_merge(fa, nbr_idx, nbr_dist, score, s));
  h->launches += 4;
  return TRAKNN_OK;
}

traknn_status traknn_knn_scores_host(traknn_handle h, const float* Xh, int64_t N, int64_t D,
                                     int L, int k, int e, int32_t* idx_h, float* dist_h,
                                     float* score_h, void* stream) {
  traknn_status st = check_handle(h);
  if (st != TRAKNN_OK) return st;
  if (!Xh || !idx_h || !dist_h || !score_h) return TRAKNN_ERR_INVALID_ARG;
  st = traknn_check_problem(N, D, L, k, e);
  if (st != TRAKNN_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t M = N - L + 1;
  const size_t xb = align_up((size_t)N * D * sizeof(float), 256);
  const size_t ib = align_up((size_t)M * k * sizeof(int32_t), 256);
  const size_t db = align_up((size_t)M * k * sizeof(float), 256);
  const size_t sb = align_up((size_t)M * sizeof(float), 256);
  st = ensure_buffer(&h->io, &h->io_bytes, xb + ib + db + sb);
  if (st != TRAKNN_OK) return st;
  char* io = static_cast<char*>(h->io);
  float* Xd = reinterpret_cast<float*>(io);
  int32_t* idx_d = reinterpret_cast<int32_t*>(io + xb);
  float* dist_d = reinterpret_cast<float*>(io + xb + ib);
  float* score_d = reinterpret_cast<float*>(io + xb + ib + db);
  TRY_CUDA(cudaMemcpyAsync(Xd, Xh, (size_t)N * D * sizeof(float), cudaMemcpyHostToDevice, s));
  st = traknn_knn_scores(h, Xd, N, D, L, k, e, idx_d, dist_d, score_d, stream);
  if (st != TRAKNN_OK) return st;
  TRY_CUDA(cudaMemcpyAsync(idx_h, idx_d, (size_t)M * k * sizeof(int32_t),
                           cudaMemcpyDeviceToHost, s));
  TRY_CUDA(cudaMemcpyAsync(dist_h, dist_d, (size_t)M * k * sizeof(float),
                           cudaMemcpyDeviceToHost, s));
  TRY_CUDA(cudaMemcpyAsync(score_h, score_d, (size_t)M * sizeof(float), cudaMemcpyDeviceToHost,
                           s));
  TRY_CUDA(cudaStreamSynchronize(s));
  return traknn_sync_status(h, stream);
}

traknn_status traknn_score_backward(traknn_handle h, const float* X, int64_t N, int64_t D, int L,
                                    int k, const int32_t* nbr_idx, const float* grad_score,
                                    float* dX, void* stream) {
  traknn_status st = check_handle(h);
  if (st != TRAKNN_OK) return st;
  if (!X || !nbr_idx || !grad_score || !dX) return TRAKNN_ERR_INVALID_ARG;
  if (N < 1 || D < 1 || L < 1 || L > N || k < 1) return TRAKNN_ERR_INVALID_ARG;
  if (N > INT_MAX / 2 || D > INT_MAX / 2) return TRAKNN_ERR_INVALID_ARG;
  if (L > TRAKNN_MAX_L || k > TRAKNN_MAX_K) return TRAKNN_ERR_UNSUPPORTED;
  const int M = (int)(N - L + 1);
  st = ensure_buffer(&h->adj, &h->adj_bytes, adjoint_workspace_bytes(M, k));
  if (st != TRAKNN_OK) return st;
  int launches = 0;
  TRY_CUDA(launch_adjoint(X, (int)N, (int)D, L, k, nbr_idx, grad_score, dX, h->adj, h->err,
                          static_cast<cudaStream_t>(stream), &launches));
  h->launches += launches;
  return TRAKNN_OK;
}

traknn_status traknn_sync_status(traknn_handle h, void* stream) {
  traknn_status st = check_handle(h);
  if (st != TRAKNN_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  TRY_CUDA(cudaStreamSynchronize(s));
  int flag = 0;
  TRY_CUDA(cudaMemcpy(&flag, h->err, sizeof(int), cudaMemcpyDeviceToHost));
  if (flag != 0) {
    TRY_CUDA(cudaMemset(h->err, 0, sizeof(int)));
    return (traknn_status)flag;
  }
  return TRAKNN_OK;
}

traknn_status traknn_profile_read(traknn_handle h, float* ms, int max_n, int* n_out) {
  traknn_status st = check_handle(h);
  if (st != TRAKNN_OK) return st;
  if (!n_out || (max_n > 0 && !ms)) return TRAKNN_ERR_INVALID_ARG;
  TRY_CUDA(cudaDeviceSynchronize());
  const int n = std::min(h->ev_count, std::max(max_n, 0));
  const int first = (h->ev_head - h->ev_count + traknn_ctx::kRing) % traknn_ctx::kRing;
  for (int i = 0; i < n; ++i) {
    const int slot = (first + i) % traknn_ctx::kRing;
    TRY_CUDA(cudaEventElapsedTime(&ms[i], h->ev_start[slot], h->ev_stop[slot]));
  }
  *n_out = n;
  h->ev_head = h->ev_count = 0;
  return TRAKNN_OK;
}

traknn_status traknn_launch_count(traknn_handle h, int64_t* count) {
  if (!h || !count) return TRAKNN_ERR_INVALID_ARG;
  *count = h->launches;
  return TRAKNN_OK;
}

}  // extern "C"
