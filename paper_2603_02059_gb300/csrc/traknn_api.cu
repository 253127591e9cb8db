// traknn_api.cu -- the C ABI declared in include/traknn.h: argument checks,
// workspace management and the launch sequence of the forward and backward
// passes. All arithmetic runs in the kernels of the other translation units.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

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
  // tensor-core work split
  int sym = 1;
  int unit_cols = 0;
  int stats = 0;
  unsigned long long* stats_dev = nullptr;
  struct {
    int M = -1, L = -1, k = -1, e = -1, sym = -1, cols = -1;
    int strips = 0, slots = 0, nunits = 0, nband = 0;
    long long col_lists = 0;
    size_t bytes = 0;
  } plan;
  void* plan_dev = nullptr;  // units, col_off, slot_lo
  size_t plan_dev_bytes = 0;
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

// Tensor-core work list. Units (strip, column range) are ordered in groups of
// strips that run side by side (sharing A and B tiles in L2); with the symmetric
// split the groups go from the last strip upwards, so the rows whose own lists
// bound the column side of a strip have mostly been processed before it.
static_assert(sizeof(WorkUnit) == 16, "work unit layout");

struct TcPlan {
  std::vector<WorkUnit> units;
  std::vector<WorkUnit> band;  // threshold pre-pass: one unit around each strip's diagonal
  std::vector<long long> col_off;
  std::vector<int> slot_lo;
  int strips = 0, slots = 0;
  long long col_lists = 0;
};

TcPlan make_tc_plan(int M, int L, int k, int sym, int cols_opt, int sm_count) {
  TcPlan p;
  const int R = kTileRows - (L - 1);
  const int ng = tc_groups(k);  // row-side lists per unit and row
  p.strips = (M + R - 1) / R;
  // a tile yields 256 - (L-1) output columns; units are whole numbers of tiles
  const int cols = cols_opt > 0 ? cols_opt : 16 * (256 - (L - 1));
  const int chunks = (M + cols - 1) / cols;
  p.slots = chunks * ng;
  const int group = std::max(1, std::min(p.strips, 19));
  (void)sm_count;
  p.col_off.resize(p.strips);
  p.slot_lo.resize(p.strips);
  long long off = 0;
  for (int s = 0; s < p.strips; ++s) {
    p.col_off[s] = off;
    const long long first_col = (long long)(s + 1) * R;  // column side starts here
    if (sym && first_col < M) off += M - first_col;
    p.slot_lo[s] = sym ? ((s * R) / cols) * ng : 0;
  }
  p.col_lists = off;
  const int ngroups = (p.strips + group - 1) / group;
  for (int gi = 0; gi < ngroups; ++gi) {
    const int g = sym ? ngroups - 1 - gi : gi;
    const int s_lo = g * group, s_hi = std::min(p.strips, s_lo + group);
    for (int c = 0; c < chunks; ++c)
      for (int s = s_lo; s < s_hi; ++s) {
        const int T0 = s * R;
        int jlo = c * cols;
        const int jhi = std::min(M, (c + 1) * cols);
        if (sym) jlo = std::max(jlo, T0);
        if (jlo >= jhi) continue;
        p.units.push_back(WorkUnit{s, jlo, jhi, c});
      }
  }
  // Band pre-pass: two tiles of columns centred on each strip's own rows. Its
  // row-side lists are not kept; their k-th distances seed the row bounds that
  // prune both sides of the main pass (candidates near in time first).
  const int bw = std::max(0, (2 * 256 - (L - 1) - R) / 2);
  for (int s = 0; s < p.strips; ++s) {
    const int T0 = s * R;
    const int jlo = std::max(0, T0 - bw), jhi = std::min(M, T0 + R + bw);
    if (jlo < jhi) p.band.push_back(WorkUnit{s, jlo, jhi, 0});
  }
  return p;
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
  if (h->plan_dev) cudaFree(h->plan_dev);
  if (h->stats_dev) cudaFree(h->stats_dev);
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
    case TRAKNN_OPT_SYMMETRIC:
      h->sym = v ? 1 : 0;
      return TRAKNN_OK;
    case TRAKNN_OPT_UNIT_COLS:
      if (v < 0 || v > (1 << 24)) return TRAKNN_ERR_INVALID_ARG;
      h->unit_cols = (int)v;
      return TRAKNN_OK;
    case TRAKNN_OPT_STATS:
      if (v && !h->stats_dev) {
        if (cudaSetDevice(h->device) != cudaSuccess) return TRAKNN_ERR_CUDA;
        if (cudaMalloc(&h->stats_dev, kStatCount * sizeof(unsigned long long)) != cudaSuccess)
          return TRAKNN_ERR_ALLOC;
        TRY_CUDA(cudaMemset(h->stats_dev, 0, kStatCount * sizeof(unsigned long long)));
      }
      h->stats = v ? 1 : 0;
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

  const bool tc = h->precision != TRAKNN_PREC_FP32;
  if (tc && !tc_available()) return TRAKNN_ERR_UNSUPPORTED;
  Schedule sch = make_schedule(M, L, k, e, h->sm_count, h->col_chunks);

  // tensor-core work list (rebuilt when the shape changes)
  auto& pl = h->plan;
  if (tc && (pl.M != M || pl.L != L || pl.k != k || pl.e != e || pl.sym != h->sym ||
             pl.cols != h->unit_cols)) {
    TcPlan tp = make_tc_plan(M, L, k, h->sym, h->unit_cols, h->sm_count);
    const size_t nb = tp.band.size();
    tp.units.insert(tp.units.end(), tp.band.begin(), tp.band.end());  // band units last
    const size_t ub = align_up(tp.units.size() * sizeof(WorkUnit), 256);
    const size_t cb = align_up(tp.col_off.size() * sizeof(long long), 256);
    const size_t sb = align_up(tp.slot_lo.size() * sizeof(int), 256);
    if (h->plan_dev && h->plan_dev_bytes < ub + cb + sb) TRY_CUDA(cudaStreamSynchronize(s));
    st = ensure_buffer(&h->plan_dev, &h->plan_dev_bytes, ub + cb + sb);
    if (st != TRAKNN_OK) return st;
    char* pd = static_cast<char*>(h->plan_dev);
    TRY_CUDA(cudaMemcpyAsync(pd, tp.units.data(), tp.units.size() * sizeof(WorkUnit),
                             cudaMemcpyHostToDevice, s));
    TRY_CUDA(cudaMemcpyAsync(pd + ub, tp.col_off.data(), tp.col_off.size() * sizeof(long long),
                             cudaMemcpyHostToDevice, s));
    TRY_CUDA(cudaMemcpyAsync(pd + ub + cb, tp.slot_lo.data(), tp.slot_lo.size() * sizeof(int),
                             cudaMemcpyHostToDevice, s));
    pl.M = M;
    pl.L = L;
    pl.k = k;
    pl.e = e;
    pl.sym = h->sym;
    pl.cols = h->unit_cols;
    pl.strips = tp.strips;
    pl.slots = tp.slots;
    pl.nunits = (int)(tp.units.size() - nb);
    pl.nband = (int)nb;
    pl.col_lists = tp.col_lists;
    pl.bytes = ub;  // device layout: units | col_off | slot_lo
  }
  if (tc) sch.chunks = pl.slots;  // partial lists: one slot per column range

  Layout lay = make_layout(N, D, sch);
  size_t thr_off = 0, coln_off = 0, cold_off = 0, coli_off = 0, cnt_off = 0;
  if (tc) {
    auto take = [&](size_t bytes) {
      lay.total = align_up(lay.total, 256);
      size_t o = lay.total;
      lay.total += bytes;
      return o;
    };
    thr_off = take((size_t)M * sizeof(unsigned int));
    coln_off = take((size_t)pl.col_lists * sizeof(int32_t));
    cold_off = take((size_t)pl.col_lists * k * sizeof(float));
    coli_off = take((size_t)pl.col_lists * k * sizeof(int32_t));
    cnt_off = take(256);
  }
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

  TcWork tw;
  if (tc) {
    char* pd = static_cast<char*>(h->plan_dev);
    const size_t ub = pl.bytes;
    const size_t cb = align_up((size_t)pl.strips * sizeof(long long), 256);
    tw.units = reinterpret_cast<const WorkUnit*>(pd);
    tw.nunits = pl.nunits;
    tw.slots = pl.slots;
    tw.col_off = reinterpret_cast<const long long*>(pd + ub);
    tw.slot_lo = reinterpret_cast<const int*>(pd + ub + cb);
    tw.sym = h->sym;
    tw.thr = reinterpret_cast<unsigned int*>(ws + thr_off);
    tw.col_n = reinterpret_cast<int32_t*>(ws + coln_off);
    tw.col_d = reinterpret_cast<float*>(ws + cold_off);
    tw.col_i = reinterpret_cast<int32_t*>(ws + coli_off);
    tw.counter = reinterpret_cast<int*>(ws + cnt_off);
    tw.write_lists = 1;
    tw.stats = h->stats ? h->stats_dev : nullptr;
  }

  TRY_CUDA(launch_col_mean(X, (int)N, (int)D, partial, mu, h->center != 0, s));
  h->launches += h->center ? 2 : 1;
  const int slot = h->ev_head;
  void* hi = ops;
  void* lo = static_cast<char*>(ops) + (size_t)N * lay.Dp * 2;
  if (!tc)
    TRY_CUDA(launch_prep_fp32(X, (int)N, (int)D, lay.Dp, mu, static_cast<float*>(ops), norms, s));
  else
    TRY_CUDA(launch_prep_split(X, (int)N, (int)D, lay.Dp, mu, hi, lo, norms, s));
  TRY_CUDA(launch_window(norms, M, L, W, s));
  if (tc) {
    TRY_CUDA(cudaMemsetAsync(tw.thr, 0x7F, (size_t)M * sizeof(unsigned int), s));
    TRY_CUDA(cudaMemsetAsync(tw.counter, 0, 2 * sizeof(int), s));
  }
  if (h->profile) TRY_CUDA(cudaEventRecord(h->ev_start[slot], s));
  if (!tc) {
    TRY_CUDA(launch_fused_fp32(static_cast<float*>(ops), fa, h->sm_count, s));
  } else {
    const bool split = h->precision == TRAKNN_PREC_SPLIT_BF16;
    if (pl.nband > 0) {
      // threshold pre-pass over the band units (stored after the main units)
      TcWork bw = tw;
      bw.units = tw.units + pl.nunits;
      bw.nunits = pl.nband;
      bw.sym = 0;
      bw.write_lists = 0;
      bw.counter = tw.counter + 1;
      TRY_CUDA(launch_fused_tc(hi, lo, split, fa, bw, h->sm_count, s));
      h->launches += 1;
    }
    TRY_CUDA(launch_fused_tc(hi, lo, split, fa, tw, h->sm_count, s));
  }
  if (h->profile) {
    TRY_CUDA(cudaEventRecord(h->ev_stop[slot], s));
    h->ev_head = (h->ev_head + 1) % traknn_ctx::kRing;
    h->ev_count = std::min(h->ev_count + 1, traknn_ctx::kRing);
  }
  if (!tc)
    TRY_CUDA(launch_merge(fa, nbr_idx, nbr_dist, score, s));
  else
    TRY_CUDA(launch_merge_tc(fa, tw, nbr_idx, nbr_dist, score, s));
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

traknn_status traknn_stats_read(traknn_handle h, uint64_t* counters, int n) {
  traknn_status st = check_handle(h);
  if (st != TRAKNN_OK) return st;
  if (!counters || n < 0) return TRAKNN_ERR_INVALID_ARG;
  unsigned long long buf[kStatCount] = {};
  if (h->stats_dev) {
    TRY_CUDA(cudaDeviceSynchronize());
    TRY_CUDA(cudaMemcpy(buf, h->stats_dev, sizeof(buf), cudaMemcpyDeviceToHost));
    TRY_CUDA(cudaMemset(h->stats_dev, 0, sizeof(buf)));
  }
  for (int i = 0; i < n && i < kStatCount; ++i) counters[i] = buf[i];
  return TRAKNN_OK;
}

traknn_status traknn_launch_count(traknn_handle h, int64_t* count) {
  if (!h || !count) return TRAKNN_ERR_INVALID_ARG;
  *count = h->launches;
  return TRAKNN_OK;
}

}  // extern "C"
