// traknn_api.cu -- the C ABI declared in include/traknn.h: argument checks,
// workspace management, work planning and the launch sequences of the forward
// (single series and batched) and backward passes. All arithmetic runs in the
// kernels of the other translation units.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/traknn.h"
#include "internal.h"

using namespace traknn;

namespace {

// One series of a tensor-core call as the caller describes it.
struct HostSeries {
  const float* X;
  int64_t N;
  int L, k, e;
  int32_t* idx;
  float* dist;
  float* score;
};

// Work list and layout of one tensor-core call (all series of a batch).
struct TcPlan {
  std::vector<int64_t> key;     // D, options and per-series shapes the plan was built for
  SeriesTable table;            // output and input pointers filled per call
  std::vector<WorkUnit> units;  // main units, then the band units
  int nunits = 0, nband = 0;
  std::vector<long long> col_off;
  std::vector<int> slot_lo;
  int rows = 0, out_rows = 0, kmax = 0, Lmax = 0;
  long long part_lists = 0, col_lists = 0;
  int emb = 1;  // days per operand row (trajectory-embedded operands when > 1)
  int part_lo = 0, part_hi = INT_MAX;  // strips evaluated (one part of a split series)
  // Host-buffer calls in phases (one series): phase q runs the strips
  // [pstrip[q+1], pstrip[q]) (pstrip[0] = strips, the last 0), the later strips first,
  // each as soon as the days it reads (from pstrip[q+1] * R on: upper triangle) are in.
  // Its main units are units[pu[q] .. pu[q+1]), its band units units[pb[q] .. pb[q+1])
  // (stored after every main unit). One phase: pstrip empty, pu = {0, nunits},
  // pb = {nunits, nunits + nband}.
  std::vector<int> pstrip, pu, pb;
  int egroups = 1;  // epilogue groups of the fused kernel; each writes its own row lists
  int mask_words = 1;  // 32-bit words per row of the non-empty column-list masks
};

constexpr size_t kMaxGraphs = 16;  // captured launch sequences kept per handle
constexpr int kMaxPhases = 8;      // phases of a host-buffer call

struct GraphEntry {
  std::vector<int64_t> key;  // plan key, pointers and options
  cudaGraphExec_t exec = nullptr;
};

}  // namespace

struct traknn_ctx {
  int device = 0;
  int sm_count = 0;
  traknn_precision precision = TRAKNN_PREC_SPLIT_BF16;
  int center = 1;
  int col_chunks = 0;
  int wait_limit_ms = 2000;
  int debug_withhold = 0;
  // library-owned buffers, grown on demand
  void* ws = nullptr;  // FP32 path
  size_t ws_bytes = 0;
  void* tcws = nullptr;  // tensor-core path
  size_t tcws_bytes = 0;
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
  int autotune = 0;
  int seg_k = kSegmentK;
  int group_strips = 0;
  int l2_keep_a = 0;
  int embed = 0;  // 0: automatic, 1: always, 2: never (TRAKNN_OPT_EMBED)
  int epi_groups = 0;  // 0: automatic, 1: one epilogue group (TRAKNN_OPT_EPI_GROUPS)
  const float* weights = nullptr;  // [weights_D] grid-point weights (caller-owned), or null
  int64_t weights_D = 0;
  int stats = 0;
  unsigned long long* stats_dev = nullptr;
  TcPlan plan;
  void* plan_dev = nullptr;  // units, col_off, slot_lo of `plan`
  size_t plan_dev_bytes = 0;
  // shape key -> (tiles per unit, strips side by side) chosen by the autotuner
  std::vector<std::pair<std::vector<int64_t>, std::pair<int, int>>> tuned;
  int last_tiles = 0, last_group = 0;  // work-unit shape of the last tensor-core call
  std::vector<GraphEntry> graphs;
  cudaStream_t cap_stream = nullptr;
  // host-buffer calls: copy stream and its events (created on first use)
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_io_free = nullptr;
  cudaEvent_t ev_in[kMaxPhases] = {};  // the days of phase q are in
};

namespace {

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

#define TRY_CUDA(expr)                              \
  do {                                              \
    cudaError_t e_ = (expr);                        \
    if (e_ != cudaSuccess) return TRAKNN_ERR_CUDA;  \
  } while (0)

#define TRY_ST(expr)                  \
  do {                                \
    traknn_status s_ = (expr);        \
    if (s_ != TRAKNN_OK) return s_;   \
  } while (0)

void drop_graphs(traknn_ctx* h) {
  for (auto& g : h->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  h->graphs.clear();
}

// Grow a library buffer. Captured graphs refer to the old buffers, so they go too.
traknn_status ensure_buffer(traknn_ctx* h, void** buf, size_t* have, size_t need) {
  if (*have >= need) return TRAKNN_OK;
  drop_graphs(h);
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

static_assert(sizeof(WorkUnit) == 32, "work unit layout");

// Pitch of the candidate lists: k rounded up to 4 entries, so that every list starts
// on a 16-byte boundary and is read four entries at a time.
inline int list_pitch(int kmax) { return (kmax + 3) / 4 * 4; }

// Tensor-core work list of a batch. For each series: strips of 128 - (L-1) output
// rows; units of `tiles` Gram tiles (tiles * kTileCols - (L-1) output columns: the
// epilogue carries the last L-1 Gram columns of a tile into the next); with the
// symmetric split only columns from each strip's own block on. Units
// are ordered per series in groups of strips that run side by side (sharing A and
// B tiles in L2), the groups from the last strip upwards. The band units (two
// tiles of columns centred on each strip's rows) seed the row bounds first.
//
// With `shared` set the B series are several (L, k, exclusion) settings of one record
// (same X and N, sorted by ascending L): they share one set of operand rows and every
// Gram tile, so the strip height and the tile step are those of the largest L, every
// unit is one tile long and carries all B series (pad[0] = B), and the first series
// (smallest L, most trajectories) defines the units' column ranges.
void build_plan(const HostSeries* sd, int B, int64_t D, int sym, int cols_opt, int tiles,
                int group_opt, bool shared, int part_lo, int part_hi,
                const std::vector<int>& pstrip, int egroups, int band_tiles, TcPlan& p) {
  p.units.clear();
  p.col_off.clear();
  p.slot_lo.clear();
  const int K = pstrip.empty() ? 1 : (int)pstrip.size() - 1;  // phases
  auto phase_of = [&](int s) {
    int q = 0;
    while (q + 1 < K && s < pstrip[q + 1]) ++q;
    return q;
  };
  std::vector<std::vector<WorkUnit>> mainq(K), bandq(K);  // units of each phase
  int row_base = 0, out_base = 0, strip_base = 0;
  long long part_base = 0, col_base = 0;
  p.kmax = 0;
  p.Lmax = 1;
  p.mask_words = 1;
  p.table.n = B;
  int Lshare = 1;
  for (int b = 0; b < B; ++b) Lshare = std::max(Lshare, sd[b].L);
  for (int b = 0; b < B; ++b) {
    const int N = (int)sd[b].N, L = sd[b].L, k = sd[b].k;
    const int M = N - L + 1;
    const int Lg = shared ? Lshare : L;  // geometry: strip height and tile step
    const int R = kTileRows - (Lg - 1);
    const int step = kTileCols - (Lg - 1);
    const int strips = (M + R - 1) / R;
    p.mask_words = std::max(p.mask_words, (strips + 31) / 32);
    const int cols = shared ? step : cols_opt > 0 ? cols_opt : tiles * kTileCols - (Lg - 1);
    // row-side list slots per trajectory row: one per column range and epilogue group
    const int slots = (M + cols - 1) / cols * egroups;
    SeriesInfo& si = p.table.s[b];
    si.N = N;
    si.M = M;
    si.L = L;
    si.k = k;
    si.e = sd[b].e;
    si.rows_out = R;
    si.step = step;
    si.row_base = row_base;
    si.out_base = out_base;
    si.slots = slots;
    si.strip_base = strip_base;
    si.part_base = part_base;
    si.col_base = col_base;
    long long off = 0;
    for (int s = 0; s < strips; ++s) {
      p.col_off.push_back(off);
      const long long first_col = (long long)(s + 1) * R;
      if (sym && first_col < M) off += M - first_col;
      p.slot_lo.push_back(sym ? (s * R) / cols * egroups : 0);
    }
    const int nser = shared ? B : 1;
    if (!shared || b == 0) {
      const int group = std::max(1, std::min(strips, group_opt > 0 ? group_opt : 19));
      const int ngroups = (strips + group - 1) / group;
      for (int gi = 0; gi < ngroups; ++gi) {
        const int g = sym ? ngroups - 1 - gi : gi;
        const int s_lo = g * group, s_hi = std::min(strips, s_lo + group);
        for (int c = 0; c < slots; ++c)
          for (int s = std::max(s_lo, part_lo); s < std::min(s_hi, part_hi); ++s) {
            int jlo = c * cols;
            const int jhi = std::min(M, (c + 1) * cols);
            if (sym) jlo = std::max(jlo, s * R);
            if (jlo < jhi) mainq[phase_of(s)].push_back(WorkUnit{b, s, jlo, jhi, c, {nser, 0, 0}});
          }
      }
      // band: band_tiles tiles of columns (band_tiles kTileCols - (L-1) outputs) centred on
      // the strip's rows
      const int bw = std::max(0, (band_tiles * kTileCols - (Lg - 1) - R) / 2);
      for (int s = std::max(0, part_lo); s < std::min(strips, part_hi); ++s) {
        const int T0 = s * R;
        int jlo = std::max(0, T0 - bw);
        const int jhi = std::min(M, T0 + R + bw);
        // a phase's band units stay clear of the days still being copied (a band only
        // seeds bounds, from whatever candidates it holds)
        const int q = phase_of(s);
        if (K > 1) jlo = std::max(jlo, pstrip[q + 1] * R);
        if (jlo < jhi) bandq[q].push_back(WorkUnit{b, s, jlo, jhi, 0, {nser, 0, 0}});
      }
    }
    if (!shared || b == B - 1) row_base += N;
    out_base += M;
    strip_base += strips;
    part_base += (long long)M * slots;
    col_base += off;
    p.kmax = std::max(p.kmax, k);
    p.Lmax = std::max(p.Lmax, L);
  }
  p.pstrip = pstrip;
  p.egroups = egroups;
  p.pu.assign(1, 0);
  for (int q = 0; q < K; ++q) {
    p.units.insert(p.units.end(), mainq[q].begin(), mainq[q].end());
    p.pu.push_back((int)p.units.size());
  }
  p.nunits = (int)p.units.size();
  p.pb.assign(1, p.nunits);
  for (int q = 0; q < K; ++q) {
    p.units.insert(p.units.end(), bandq[q].begin(), bandq[q].end());
    p.pb.push_back((int)p.units.size());
  }
  p.nband = (int)p.units.size() - p.nunits;
  p.rows = row_base;
  p.out_rows = out_base;
  p.part_lists = part_base;
  p.col_lists = col_base;
}

traknn_status check_handle(traknn_handle h) {
  if (!h) return TRAKNN_ERR_INVALID_ARG;
  if (cudaSetDevice(h->device) != cudaSuccess) return TRAKNN_ERR_CUDA;
  return TRAKNN_OK;
}

std::vector<int64_t> shape_key(const HostSeries* sd, int B, int64_t D, const traknn_ctx* h) {
  std::vector<int64_t> key = {D, h->sym, h->unit_cols, (int64_t)h->precision, h->center, B,
                              h->seg_k, h->group_strips, h->l2_keep_a};
  for (int b = 0; b < B; ++b) {
    key.push_back(sd[b].N);
    key.push_back(sd[b].L);
    key.push_back(sd[b].k);
    key.push_back(sd[b].e);
  }
  return key;
}

// Device pointers of the tensor-core workspace for plan `p`.
struct TcBuffers {
  float* partial;
  float* mu;
  double* norms;
  float* cval;
  float* W;
  void* hi;
  void* lo;
  float* part_d;
  int32_t* part_i;
  unsigned int* thr;
  int32_t* col_rec;
  unsigned int* col_mask;
  int* counter;
  float* scratch;
  float* pscore;  // [out_rows] scores of partial lists (split series), not returned
  int Dp;
  size_t total;
};

TcBuffers tc_layout(const TcPlan& p, int64_t D, int num_ctas, char* base) {
  TcBuffers b;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    off = align_up(off, 256);
    const size_t o = off;
    off += bytes;
    return base + o;
  };
  b.Dp = tc_groups((int)D * p.emb) * 64;
  const int B = p.table.n;
  const size_t ks = (size_t)list_pitch(p.kmax);
  b.partial = reinterpret_cast<float*>(take((size_t)B * kMeanSlices * D * sizeof(float)));
  b.mu = reinterpret_cast<float*>(take((size_t)B * D * sizeof(float)));
  b.norms = reinterpret_cast<double*>(take((size_t)p.rows * sizeof(double)));
  b.cval = reinterpret_cast<float*>(take((size_t)p.rows * sizeof(float)));
  b.W = reinterpret_cast<float*>(take((size_t)p.out_rows * sizeof(float)));
  b.hi = take((size_t)p.rows * b.Dp * 2);
  b.lo = take((size_t)p.rows * b.Dp * 2);
  b.part_d = reinterpret_cast<float*>(take((size_t)p.part_lists * ks * sizeof(float)));
  b.part_i = reinterpret_cast<int32_t*>(take((size_t)p.part_lists * ks * sizeof(int32_t)));
  b.thr = reinterpret_cast<unsigned int*>(take((size_t)p.out_rows * sizeof(unsigned int)));
  b.col_rec = reinterpret_cast<int32_t*>(
      take((size_t)p.col_lists * col_pitch((int)ks) * sizeof(int32_t)));
  b.col_mask = reinterpret_cast<unsigned int*>(
      take((size_t)p.out_rows * p.mask_words * sizeof(unsigned int)));
  b.counter = reinterpret_cast<int*>(take(256));
  b.scratch = reinterpret_cast<float*>(take(tc_scratch_bytes(num_ctas)));
  b.pscore = reinterpret_cast<float*>(take((size_t)p.out_rows * sizeof(float)));
  b.total = off;
  return b;
}

// Make h->plan the plan for these series (built and uploaded when the shape changes)
// and size the workspace. Must not run during a stream capture.
traknn_status prepare_tc(traknn_ctx* h, const HostSeries* sd, int B, int64_t D, int tiles,
                         bool shared, int emb, cudaStream_t s, TcBuffers* out,
                         int part_lo = 0, int part_hi = INT_MAX,
                         const std::vector<int>& pstrip = {}, int group = 0) {
  if (group <= 0) group = h->group_strips;  // 0: the planner's default
  std::vector<int64_t> key = shape_key(sd, B, D, h);
  key.push_back(tiles);
  key.push_back(group);
  key.push_back(shared ? 1 : 0);
  key.push_back(emb);
  key.push_back(part_lo);
  key.push_back(part_hi);
  key.push_back((int64_t)pstrip.size());
  key.insert(key.end(), pstrip.begin(), pstrip.end());
  // two epilogue groups for L = 1 (small grids through embedded operands) when the
  // tile has one accumulation segment and the lists are short
  int Lmax = 1, kmax = 1;
  for (int b = 0; b < B; ++b) {
    Lmax = std::max(Lmax, sd[b].L);
    kmax = std::max(kmax, sd[b].k);
  }
  const int egroups = (h->epi_groups != 1 && !shared && Lmax == 1 && kmax <= 32 &&
                       tc_groups((int)D * emb) * 64 <= h->seg_k)
                          ? 2
                          : 1;
  key.push_back(egroups);
  // Band pre-pass width: two tiles per strip when the contraction dominates a tile's
  // cost; with short operand rows (small grids) a tile's contraction is cheap and the
  // epilogue decides, and eight tiles give bounds tight enough to save more list
  // inserts in the main pass than the band costs (D = 32, L = 5: 1.91 -> 1.69 ms; at
  // D = 3,726 four tiles already cost 6 %)
  const int band_tiles = tc_groups((int)D * emb) * 64 <= 768 ? 8 : 2;
  key.push_back(band_tiles);
  TcPlan& p = h->plan;
  if (p.key != key) {
    build_plan(sd, B, D, h->sym, h->unit_cols, tiles, group, shared, part_lo, part_hi, pstrip,
               egroups, band_tiles, p);
    p.key = key;
    p.emb = emb;
    p.part_lo = part_lo;
    p.part_hi = part_hi;
    const size_t ub = align_up(p.units.size() * sizeof(WorkUnit), 256);
    const size_t cb = align_up(p.col_off.size() * sizeof(long long), 256);
    const size_t sb = align_up(p.slot_lo.size() * sizeof(int), 256);
    TRY_CUDA(cudaStreamSynchronize(s));  // earlier work may still read the old list
    TRY_ST(ensure_buffer(h, &h->plan_dev, &h->plan_dev_bytes, ub + cb + sb));
    char* pd = static_cast<char*>(h->plan_dev);
    TRY_CUDA(cudaMemcpy(pd, p.units.data(), p.units.size() * sizeof(WorkUnit),
                        cudaMemcpyHostToDevice));
    TRY_CUDA(cudaMemcpy(pd + ub, p.col_off.data(), p.col_off.size() * sizeof(long long),
                        cudaMemcpyHostToDevice));
    TRY_CUDA(cudaMemcpy(pd + ub + cb, p.slot_lo.data(), p.slot_lo.size() * sizeof(int),
                        cudaMemcpyHostToDevice));
    drop_graphs(h);  // graphs captured the previous work list
  }
  for (int b = 0; b < B; ++b) {
    p.table.s[b].X = sd[b].X;
    p.table.s[b].idx = sd[b].idx;
    p.table.s[b].dist = sd[b].dist;
    p.table.s[b].score = sd[b].score;
  }
  const TcBuffers probe = tc_layout(p, D, h->sm_count, nullptr);
  TRY_ST(ensure_buffer(h, &h->tcws, &h->tcws_bytes, probe.total));
  *out = tc_layout(p, D, h->sm_count, static_cast<char*>(h->tcws));
  for (int b = 0; b < B; ++b)  // partial lists: their scores go to the workspace
    if (!p.table.s[b].score) p.table.s[b].score = out->pscore + p.table.s[b].out_base;
  return TRAKNN_OK;
}

// The band pre-pass only seeds upper bounds of the rows' k-th distances, from whatever
// candidates it holds. For split-BF16 calls with long operand rows (more than 768 K
// entries, where the contraction sets a tile's cost) it runs in one BF16 product (hi
// only: a third of its tensor work) and raises every distance by a bound of that
// product's error before it enters a list. For operands a, b (hi = bf16(x), unit
// roundoff u = 2^-8): |a.b - hi_a.hi_b| <= (2u + u^2) ||a|| ||b||; the FP32
// accumulation of Dp products and correction terms (sum of magnitudes at most about
// 2 ||a|| ||b||) adds at most 2.1 Dp 2^-23 ||a|| ||b||, allowing for truncating adds;
// so each day pair's distance n_a + n_b - 2 G moves by at most
// (2u + u^2 + 2.1 Dp 2^-23) (n_a + n_b), and a window's by that times W_t + W_j, plus
// a few FP32 roundings of the epilogue (2^-19). The k-th of the raised distances is
// then an upper bound of the row's exact k-th distance.
// (One epilogue group only: the kernel with two groups, which short operand rows use,
// has no raised-distance path.)
bool band_single_product(const traknn_ctx* h, const TcPlan& p, int Dp) {
  return h->precision == TRAKNN_PREC_SPLIT_BF16 && Dp > 768 && p.egroups == 1;
}
float band_error_margin(int Dp) {
  const double u = 1.0 / 256.0;
  return (float)(2.0 * u + u * u + 2.1 * Dp * std::ldexp(1.0, -23) + std::ldexp(1.0, -19));
}

// The launch sequence of one tensor-core call (also what a graph captures).
traknn_status enqueue_tc(traknn_ctx* h, const TcBuffers& b, int64_t D,
                         cudaStream_t s, bool record_events) {
  const TcPlan& p = h->plan;
  const SeriesTable& sr = p.table;
  const size_t ub = align_up(p.units.size() * sizeof(WorkUnit), 256);
  const size_t cb = align_up(p.col_off.size() * sizeof(long long), 256);
  char* pd = static_cast<char*>(h->plan_dev);

  TcArgs a;
  a.Dp = b.Dp;
  a.rows = p.rows;
  a.out_rows = p.out_rows;
  a.Lmax = p.Lmax;
  a.kmax = p.kmax;
  a.W = b.W;
  a.part_d = b.part_d;
  a.part_i = b.part_i;
  a.err = h->err;
  a.wait_limit_ns = (long long)h->wait_limit_ms * 1000000LL;
  a.debug_withhold = h->debug_withhold;
  a.seg_k = h->seg_k;
  a.scratch = b.scratch;
  a.groups = b.Dp / 64;
  a.cval = b.cval;
  a.l2_keep_a = h->l2_keep_a;
  a.egroups = p.egroups;
  a.corr_neg = 0;
  a.band_margin = 0.f;

  TcWork w;
  w.units = reinterpret_cast<const WorkUnit*>(pd);
  w.nunits = p.nunits;
  w.kstride = list_pitch(p.kmax);
  w.col_off = reinterpret_cast<const long long*>(pd + ub);
  w.slot_lo = reinterpret_cast<const int*>(pd + ub + cb);
  w.sym = h->sym;
  w.col_rec = b.col_rec;
  w.col_ints = p.col_lists * col_pitch(w.kstride);
  w.col_mask = b.col_mask;
  w.mask_words = p.mask_words;
  w.part_ints = p.part_lists * w.kstride;
  w.thr = b.thr;
  w.counter = b.counter;
  w.write_lists = 1;
  w.stats = h->stats ? h->stats_dev : nullptr;
  w.part_lo = p.part_lo;
  w.part_hi = p.part_hi;

  const bool split = h->precision == TRAKNN_PREC_SPLIT_BF16;
  TRY_CUDA(launch_col_mean_series(sr, (int)D, b.partial, b.mu, h->center != 0, s));
  TRY_CUDA(launch_prep_split_series(sr, p.rows, (int)D, p.emb, b.Dp / 64, split, b.mu,
                                    h->weights,
                                    b.hi, b.lo,
                                    b.norms, b.cval, s));
  TRY_CUDA(launch_window_series(sr, p.out_rows, b.norms, b.W, s));
  TRY_CUDA(cudaMemsetAsync(b.thr, 0x7F, (size_t)p.out_rows * sizeof(unsigned int), s));
  TRY_CUDA(cudaMemsetAsync(b.col_mask, 0,
                           (size_t)p.out_rows * p.mask_words * sizeof(unsigned int), s));
  TRY_CUDA(cudaMemsetAsync(b.counter, 0, 2 * sizeof(int), s));
  const int slot = h->ev_head;
  if (record_events) TRY_CUDA(cudaEventRecord(h->ev_start[slot], s));
  if (p.nband > 0) {
    // threshold pre-pass over the band units (stored after the main units)
    TcWork bw = w;
    bw.units = w.units + p.nunits;
    bw.nunits = p.nband;
    bw.sym = 0;
    bw.write_lists = 0;
    bw.counter = w.counter + 1;
    TcArgs ab = a;
    const bool one = band_single_product(h, p, b.Dp);
    if (one) {
      ab.corr_neg = 1;
      ab.band_margin = band_error_margin(b.Dp);
    }
    TRY_CUDA(launch_fused_tc(b.hi, b.lo, one ? false : split, ab, bw, sr, h->sm_count, s));
  }
  TRY_CUDA(launch_fused_tc(b.hi, b.lo, split, a, w, sr, h->sm_count, s));
  if (record_events) {
    TRY_CUDA(cudaEventRecord(h->ev_stop[slot], s));
    h->ev_head = (h->ev_head + 1) % traknn_ctx::kRing;
    h->ev_count = std::min(h->ev_count + 1, traknn_ctx::kRing);
  }
  TRY_CUDA(launch_merge_tc(a, w, sr, s));
  h->launches += (h->center ? 2 : 1) + 2 + (p.nband > 0 ? 1 : 0) + 2;
  return TRAKNN_OK;
}


// Phases of a host-buffer call (tensor-core path, one series): strip boundaries
// pstrip[0] = strips > pstrip[1] > ... > pstrip[K] = 0, phase q reading the days from
// pstrip[q+1] R on; phase q starts once the fraction kPhaseDays[q] of the days (the
// last ones) is in. Phase 0 holds at least the days the centring mean reads. With the
// upper triangle the work a fraction F of the days unlocks is F^2 of the call, and it
// is concentrated in few strips with few units each, so every phase ends with a tail
// of idle SMs: a few large phases overlap the copy better than many small ones.
// Empty when the series is too short to split.
constexpr double kPhaseDays[] = {0.35};
std::vector<int> phase_plan(int strips, int R, int64_t N) {
  std::vector<int> ps;
  if (strips < 8) return ps;
  const int first = mean_first((int)N) / R;  // last boundary that keeps the mean's days
  ps.push_back(strips);
  for (double f : kPhaseDays) {
    const int sb = std::min(first, (int)std::floor((1.0 - f) * (double)N / R));
    if (sb < 2 || sb > ps.back() - 2) break;
    ps.push_back(sb);
  }
  ps.push_back(0);
  if (ps.size() <= 2) ps.clear();
  return ps;
}

// The launch sequence of a host-buffer call in phases (plan built with phase
// boundaries, one series). The days of phase q, [pstrip[q+1] R, pstrip[q] R) (phase 0:
// up to N, including the days the centring mean reads), are copied in on the copy
// stream in phase order, event in[q] after each. Phase q waits for its days, prepares
// their operand rows and window sums, and runs its band and main units: strips from
// pstrip[q+1] on read only days >= pstrip[q+1] R (upper triangle: columns j >= T0 of
// the strip), so each phase runs while the copy of the earlier days continues. One
// merge follows. The operands, and so every distance, are those of the one-phase
// sequence; only the order of the work units differs.
traknn_status enqueue_tc_phased(traknn_ctx* h, const TcBuffers& b, int64_t D, cudaStream_t s,
                                const cudaEvent_t* in) {
  const TcPlan& p = h->plan;
  const SeriesTable& sr = p.table;
  const SeriesInfo& si = sr.s[0];
  const int R = kTileRows - (si.L - 1);
  const int K = (int)p.pstrip.size() - 1;
  const size_t ub = align_up(p.units.size() * sizeof(WorkUnit), 256);
  const size_t cb = align_up(p.col_off.size() * sizeof(long long), 256);
  char* pd = static_cast<char*>(h->plan_dev);
  TcArgs a;
  a.Dp = b.Dp;
  a.rows = p.rows;
  a.out_rows = p.out_rows;
  a.Lmax = p.Lmax;
  a.kmax = p.kmax;
  a.W = b.W;
  a.part_d = b.part_d;
  a.part_i = b.part_i;
  a.err = h->err;
  a.wait_limit_ns = (long long)h->wait_limit_ms * 1000000LL;
  a.debug_withhold = h->debug_withhold;
  a.seg_k = h->seg_k;
  a.scratch = b.scratch;
  a.groups = b.Dp / 64;
  a.cval = b.cval;
  a.l2_keep_a = h->l2_keep_a;
  a.egroups = p.egroups;
  a.corr_neg = 0;
  a.band_margin = 0.f;
  TcWork w;
  w.units = reinterpret_cast<const WorkUnit*>(pd);
  w.kstride = list_pitch(p.kmax);
  w.col_off = reinterpret_cast<const long long*>(pd + ub);
  w.slot_lo = reinterpret_cast<const int*>(pd + ub + cb);
  w.sym = h->sym;
  w.col_rec = b.col_rec;
  w.col_ints = p.col_lists * col_pitch(w.kstride);
  w.col_mask = b.col_mask;
  w.mask_words = p.mask_words;
  w.part_ints = p.part_lists * w.kstride;
  w.thr = b.thr;
  w.write_lists = 1;
  w.stats = h->stats ? h->stats_dev : nullptr;
  w.part_lo = 0;
  w.part_hi = INT_MAX;
  const bool split = h->precision == TRAKNN_PREC_SPLIT_BF16;
  auto fused = [&](int u0, int nu, int ctr, bool band) -> cudaError_t {
    if (nu <= 0) return cudaSuccess;
    TcWork x = w;
    x.units = w.units + u0;
    x.nunits = nu;
    x.counter = b.counter + ctr;
    TcArgs ax = a;
    bool sp = split;
    if (band) {
      x.sym = 0;
      x.write_lists = 0;
      if (band_single_product(h, p, b.Dp)) {  // see band_error_margin
        ax.corr_neg = 1;
        ax.band_margin = band_error_margin(b.Dp);
        sp = false;
      }
    }
    ++h->launches;
    return launch_fused_tc(b.hi, b.lo, sp, ax, x, sr, h->sm_count, s);
  };
  for (int q = 0; q < K; ++q) {
    const int lo = p.pstrip[q + 1] * R;                      // first day (and row) of phase q
    const int hi = q == 0 ? p.rows : p.pstrip[q] * R;        // rows prepared by phase q
    const int ohi = q == 0 ? p.out_rows : std::min(hi, p.out_rows);
    TRY_CUDA(cudaStreamWaitEvent(s, in[q], 0));
    if (q == 0) {
      TRY_CUDA(launch_col_mean_series(sr, (int)D, b.partial, b.mu, h->center != 0, s));
      TRY_CUDA(cudaMemsetAsync(b.thr, 0x7F, (size_t)p.out_rows * sizeof(unsigned int), s));
      TRY_CUDA(cudaMemsetAsync(b.col_mask, 0,
                               (size_t)p.out_rows * p.mask_words * sizeof(unsigned int), s));
      TRY_CUDA(cudaMemsetAsync(b.counter, 0, 2 * K * sizeof(int), s));
      h->launches += h->center ? 2 : 1;
    }
    // window sums of rows [lo, ohi) read day norms up to ohi + L - 2: prepared now or
    // by an earlier phase
    TRY_CUDA(launch_prep_split_series(sr, hi, (int)D, 1, b.Dp / 64, split, b.mu, h->weights,
                                      b.hi, b.lo, b.norms, b.cval, s, lo));
    TRY_CUDA(launch_window_series(sr, ohi, b.norms, b.W, s, lo));
    h->launches += (hi > lo ? 1 : 0) + (ohi > lo ? 1 : 0);
    TRY_CUDA(fused(p.pb[q], p.pb[q + 1] - p.pb[q], 2 * q + 1, true));
    TRY_CUDA(fused(p.pu[q], p.pu[q + 1] - p.pu[q], 2 * q, false));
  }
  w.nunits = p.nunits;
  w.counter = b.counter;
  TRY_CUDA(launch_merge_tc(a, w, sr, s));
  h->launches += 1;
  return TRAKNN_OK;
}

// Trajectory-embedded operands for a single-series tensor-core call: automatic for
// small grids, where the fixed per-chunk cost of the epilogue (staging, window sums)
// and not the contraction decides the time, so L times the Gram work costs little.
constexpr int64_t kEmbedAutoMaxLD = 1536;    // automatic: L * D at most this
constexpr int64_t kEmbedMaxLD = 1 << 20;     // forced: L * D at most this
bool use_embedding(const traknn_ctx* h, int64_t D, int L) {
  if (L < 2 || h->embed == 2) return false;
  if (h->embed == 1) return (int64_t)L * D <= kEmbedMaxLD;
  return (int64_t)L * D <= kEmbedAutoMaxLD;
}

traknn_status validate_series(const HostSeries* sd, int B, int64_t D) {
  if (B < 1) return TRAKNN_ERR_INVALID_ARG;
  int64_t rows = 0;
  for (int b = 0; b < B; ++b) {
    if (!sd[b].X || !sd[b].idx || !sd[b].dist || !sd[b].score) return TRAKNN_ERR_INVALID_ARG;
    TRY_ST(traknn_check_problem(sd[b].N, D, sd[b].L, sd[b].k, sd[b].e));
    rows += sd[b].N;
  }
  if (rows > INT_MAX / 2) return TRAKNN_ERR_INVALID_ARG;
  return TRAKNN_OK;
}

// Work-unit shape for this batch: Gram tiles per unit and row strips whose units run
// side by side (sharing operand tiles in L2). With tuning on (and neither set by an
// option) every pair of {4, 8, 16} tiles and {10, 19, 38} strips is timed once after a
// warm-up launch and the fastest is kept per shape; else 8 tiles and the default
// grouping (19 strips, or the option's value).
traknn_status pick_shape(traknn_ctx* h, const HostSeries* sd, int B, int64_t D, cudaStream_t s,
                         int* tiles, int* group) {
  *tiles = 8;
  *group = 0;
  if (!h->autotune || h->unit_cols > 0) return TRAKNN_OK;
  const std::vector<int64_t> key = shape_key(sd, B, D, h);
  for (auto& t : h->tuned)
    if (t.first == key) {
      *tiles = t.second.first;
      *group = t.second.second;
      return TRAKNN_OK;
    }
  cudaEvent_t e0, e1;
  TRY_CUDA(cudaEventCreate(&e0));
  TRY_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  int best_t = 8, best_g = 0;
  const std::vector<int> groups = h->group_strips > 0 ? std::vector<int>{h->group_strips}
                                                      : std::vector<int>{10, 19, 38};
  for (int cand_g : groups)
    for (int cand_t : {4, 8, 16}) {
      TcBuffers buf;
      TRY_ST(prepare_tc(h, sd, B, D, cand_t, false, 1, s, &buf, 0, INT_MAX, {}, cand_g));
      TRY_ST(enqueue_tc(h, buf, D, s, false));  // warm-up
      TRY_CUDA(cudaEventRecord(e0, s));
      TRY_ST(enqueue_tc(h, buf, D, s, false));
      TRY_CUDA(cudaEventRecord(e1, s));
      TRY_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      TRY_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best) {
        best = ms;
        best_t = cand_t;
        best_g = cand_g;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->tuned.emplace_back(key, std::make_pair(best_t, best_g));
  *tiles = best_t;
  *group = best_g;
  return TRAKNN_OK;
}

// Work-unit shape when neither the autotuner nor an option sets it: Gram tiles per
// unit and row strips side by side (0 = the planner's default). Short operand rows
// (small grids): the epilogue sets the pace, and units of 16 tiles keep fewer partial
// lists per row, so fewer list inserts (D = 32, L = 5, embedded: 1.70 -> 1.61 ms;
// longer units lose more at the launch's tail than they save), with 38 strips side by
// side (1.61 -> 1.58 ms). Otherwise the unit length follows the Gram tiles per SM of
// an average series of the call (strips [part_lo, part_hi)): eight tiles from 64
// (the 75-year series has 78), four from 16, two below (L = 5, D = 3,726:
// N = 10,957 1.31 -> 1.21 ms with two; N = 13,697 1.87 -> 1.83 ms and N = 20,546
// 3.84 -> 3.72 ms with four; at N = 27,394 the three lengths time alike; 64 series of
// 3,650 to 27,394 days in one call: four tiles 1.04x faster than eight). Shorter
// units let the persistent CTAs run out of work together and keep more of a
// series' operand tiles in L2 while its strips run side by side. Long operand rows
// make every tile long too, so a unit also holds at most 65,536 K entries x tiles
// (Dp x tiles), two tiles at least: at the 0.25-degree grid (Dp = 59,072, N = 27,394,
// L = 5) 8 / 4 / 2 tiles took 106.0-108.8 / 99.8-100.7 / 98.9-99.9 ms, while at
// Dp = 3,840 eight tiles stay within the cap; between the two the cap is a choice.
void default_shape(const traknn_ctx* h, const HostSeries* sd, int B, int64_t D, int emb,
                   int part_lo, int part_hi, int* tiles, int* group) {
  if (tc_groups((int)D * emb) * 64 <= 768) {
    *tiles = 16;
    if (*group == 0 && h->group_strips == 0) *group = 38;
    return;
  }
  double t = 0.0;  // Gram tiles of the call
  for (int b = 0; b < B; ++b) {
    const int64_t M = sd[b].N - sd[b].L + 1;
    const int R = emb > 1 ? kTileRows : kTileRows - (sd[b].L - 1);
    const int strips = (int)((M + R - 1) / R);
    for (int st = std::max(0, part_lo); st < std::min(strips, part_hi); ++st)
      t += (double)(h->sym ? M - (int64_t)st * R : M) / kTileCols;
  }
  const double per_sm = t / B / std::max(1, h->sm_count);
  *tiles = per_sm >= 64.0 ? 8 : per_sm >= 16.0 ? 4 : 2;
  const int64_t Dp = (int64_t)tc_groups((int)D * emb) * 64;
  while (*tiles > 2 && *tiles * Dp > 65536) *tiles /= 2;
}

// Forward pass of B series on the tensor cores. With `graph` set the launch
// sequence is captured once per (shape, pointers, options) and replayed.
traknn_status run_tc(traknn_ctx* h, const HostSeries* sd, int B, int64_t D, cudaStream_t s,
                     bool graph, bool shared = false, int emb = 1, int part_lo = 0,
                     int part_hi = INT_MAX) {
  if (!tc_available()) return TRAKNN_ERR_UNSUPPORTED;
  int tiles = 8, group = 0;
  const bool whole = part_lo == 0 && part_hi == INT_MAX;
  if (!shared && emb == 1 && whole) TRY_ST(pick_shape(h, sd, B, D, s, &tiles, &group));
  if (!h->autotune && !shared) default_shape(h, sd, B, D, emb, part_lo, part_hi, &tiles, &group);
  TcBuffers buf;
  TRY_ST(prepare_tc(h, sd, B, D, tiles, shared, emb, s, &buf, part_lo, part_hi, {}, group));
  h->last_tiles = tiles;
  h->last_group = group > 0 ? group : (h->group_strips > 0 ? h->group_strips : 19);
  if (!graph) return enqueue_tc(h, buf, D, s, h->profile != 0);

  std::vector<int64_t> key = h->plan.key;
  for (int b = 0; b < B; ++b) {
    key.push_back((int64_t)reinterpret_cast<uintptr_t>(sd[b].X));
    key.push_back((int64_t)reinterpret_cast<uintptr_t>(sd[b].idx));
    key.push_back((int64_t)reinterpret_cast<uintptr_t>(sd[b].dist));
    key.push_back((int64_t)reinterpret_cast<uintptr_t>(sd[b].score));
  }
  key.push_back(h->stats);
  key.push_back((int64_t)reinterpret_cast<uintptr_t>(h->weights));
  key.push_back(h->debug_withhold);
  key.push_back(h->wait_limit_ms);
  for (auto& g : h->graphs)
    if (g.key == key) {
      TRY_CUDA(cudaGraphLaunch(g.exec, s));
      h->launches += (h->center ? 2 : 1) + 2 + (h->plan.nband > 0 ? 1 : 0) + 2;
      return TRAKNN_OK;
    }
  if (!h->cap_stream) TRY_CUDA(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  // run once outside the capture (kernel attributes, first-use costs), then capture
  TRY_ST(enqueue_tc(h, buf, D, s, false));
  TRY_CUDA(cudaStreamSynchronize(s));
  const int64_t l0 = h->launches;
  TRY_CUDA(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
  const traknn_status st = enqueue_tc(h, buf, D, h->cap_stream, false);
  cudaGraph_t g = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(h->cap_stream, &g);
  if (st != TRAKNN_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  TRY_CUDA(ce);
  cudaGraphExec_t exec = nullptr;
  const cudaError_t ie = cudaGraphInstantiate(&exec, g, 0);
  cudaGraphDestroy(g);
  TRY_CUDA(ie);
  h->launches = l0;  // the capture enqueued nothing
  if (h->graphs.size() >= kMaxGraphs) {
    // keep the cache bounded: drop the oldest graph (after its launches have finished)
    TRY_CUDA(cudaStreamSynchronize(s));
    cudaGraphExecDestroy(h->graphs.front().exec);
    h->graphs.erase(h->graphs.begin());
  }
  h->graphs.push_back(GraphEntry{key, exec});
  TRY_CUDA(cudaGraphLaunch(exec, s));
  h->launches += (h->center ? 2 : 1) + 2 + (h->plan.nband > 0 ? 1 : 0) + 2;
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
    case TRAKNN_ERR_BOUNDS: return "a device-side index check failed (debug build)";
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
  drop_graphs(h);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
  if (h->ev_io_free) cudaEventDestroy(h->ev_io_free);
  for (cudaEvent_t ev : h->ev_in)
    if (ev) cudaEventDestroy(ev);
  if (h->ws) cudaFree(h->ws);
  if (h->tcws) cudaFree(h->tcws);
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
    case TRAKNN_OPT_AUTOTUNE:
      h->autotune = v ? 1 : 0;
      return TRAKNN_OK;
    case TRAKNN_OPT_L2_KEEP_A:
      h->l2_keep_a = v ? 1 : 0;
      return TRAKNN_OK;
    case TRAKNN_OPT_EMBED:
      if (v < 0 || v > 2) return TRAKNN_ERR_INVALID_ARG;
      h->embed = (int)v;
      return TRAKNN_OK;
    case TRAKNN_OPT_EPI_GROUPS:
      if (v < 0 || v > 1) return TRAKNN_ERR_INVALID_ARG;
      h->epi_groups = (int)v;
      return TRAKNN_OK;
    case TRAKNN_OPT_GROUP_STRIPS:
      if (v < 0 || v > 4096) return TRAKNN_ERR_INVALID_ARG;
      h->group_strips = (int)v;
      return TRAKNN_OK;
    case TRAKNN_OPT_SEGMENT_K:
      if (v != 0 && (v < 32 || v % 32 != 0 || v > (1 << 20))) return TRAKNN_ERR_INVALID_ARG;
      h->seg_k = v ? (int)v : kSegmentK;
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
  TRY_ST(check_handle(h));
  if (!X || !nbr_idx || !nbr_dist || !score) return TRAKNN_ERR_INVALID_ARG;
  TRY_ST(traknn_check_problem(N, D, L, k, e));
  if (h->weights && h->weights_D != D) return TRAKNN_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (h->precision != TRAKNN_PREC_FP32) {
    if (use_embedding(h, D, L)) {
      // trajectory-embedded operands: one row per trajectory (L days, contiguous in
      // X), whose Gram is the window sum itself; the kernels see M rows and L = 1
      const HostSeries sd{X, N - L + 1, 1, k, e, nbr_idx, nbr_dist, score};
      return run_tc(h, &sd, 1, D, s, false, false, L);
    }
    const HostSeries sd{X, N, L, k, e, nbr_idx, nbr_dist, score};
    return run_tc(h, &sd, 1, D, s, false);
  }

  // plain FP32 CUDA-core path
  const int M = (int)(N - L + 1);
  const Schedule sch = make_schedule(M, L, k, e, h->sm_count, h->col_chunks);
  const Fp32Layout lay = make_layout(N, D, sch);
  TRY_ST(ensure_buffer(h, &h->ws, &h->ws_bytes, lay.total));
  char* ws = static_cast<char*>(h->ws);
  float* partial = reinterpret_cast<float*>(ws + lay.partial);
  float* mu = reinterpret_cast<float*>(ws + lay.mu);
  double* norms = reinterpret_cast<double*>(ws + lay.norms);
  float* W = reinterpret_cast<float*>(ws + lay.W);
  float* Xc = reinterpret_cast<float*>(ws + lay.ops);
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
  TRY_CUDA(launch_col_mean(X, (int)N, (int)D, partial, mu, h->center != 0, s));
  TRY_CUDA(launch_prep_fp32(X, (int)N, (int)D, lay.Dp, mu, h->weights, Xc, norms, s));
  TRY_CUDA(launch_window(norms, M, L, W, s));
  const int slot = h->ev_head;
  if (h->profile) TRY_CUDA(cudaEventRecord(h->ev_start[slot], s));
  TRY_CUDA(launch_fused_fp32(Xc, fa, h->sm_count, s));
  if (h->profile) {
    TRY_CUDA(cudaEventRecord(h->ev_stop[slot], s));
    h->ev_head = (h->ev_head + 1) % traknn_ctx::kRing;
    h->ev_count = std::min(h->ev_count + 1, traknn_ctx::kRing);
  }
  TRY_CUDA(launch_merge(fa, nbr_idx, nbr_dist, score, s));
  h->launches += (h->center ? 2 : 1) + 4;
  return TRAKNN_OK;
}

traknn_status traknn_knn_scores_batched(traknn_handle h, const traknn_series* series, int B,
                                        int64_t D, void* stream) {
  TRY_ST(check_handle(h));
  if (!series || B < 1 || D < 1) return TRAKNN_ERR_INVALID_ARG;
  std::vector<HostSeries> sd(B);
  for (int b = 0; b < B; ++b)
    sd[b] = HostSeries{series[b].X, series[b].N, series[b].L, series[b].k, series[b].exclusion,
                       series[b].nbr_idx, series[b].nbr_dist, series[b].score};
  TRY_ST(validate_series(sd.data(), B, D));
  if (h->weights && h->weights_D != D) return TRAKNN_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (h->precision == TRAKNN_PREC_FP32) {
    for (int b = 0; b < B; ++b)
      TRY_ST(traknn_knn_scores(h, sd[b].X, sd[b].N, D, sd[b].L, sd[b].k, sd[b].e, sd[b].idx,
                               sd[b].dist, sd[b].score, stream));
    return TRAKNN_OK;
  }
  for (int b0 = 0; b0 < B; b0 += kMaxSeries)
    TRY_ST(run_tc(h, sd.data() + b0, std::min(kMaxSeries, B - b0), D, s, true));
  return TRAKNN_OK;
}

traknn_status traknn_knn_scores_multi(traknn_handle h, const traknn_series* settings, int nset,
                                      int64_t D, void* stream) {
  TRY_ST(check_handle(h));
  if (!settings || nset < 1 || nset > kMaxSeries || D < 1) return TRAKNN_ERR_INVALID_ARG;
  std::vector<HostSeries> sd(nset);
  for (int b = 0; b < nset; ++b) {
    sd[b] = HostSeries{settings[b].X, settings[b].N, settings[b].L, settings[b].k,
                       settings[b].exclusion, settings[b].nbr_idx, settings[b].nbr_dist,
                       settings[b].score};
    if (sd[b].X != sd[0].X || sd[b].N != sd[0].N) return TRAKNN_ERR_INVALID_ARG;
  }
  TRY_ST(validate_series(sd.data(), nset, D));
  if (h->weights && h->weights_D != D) return TRAKNN_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (h->precision == TRAKNN_PREC_FP32) {
    for (int b = 0; b < nset; ++b)
      TRY_ST(traknn_knn_scores(h, sd[b].X, sd[b].N, D, sd[b].L, sd[b].k, sd[b].e, sd[b].idx,
                               sd[b].dist, sd[b].score, stream));
    return TRAKNN_OK;
  }
  // the shared geometry takes the smallest L (most trajectories) first
  std::stable_sort(sd.begin(), sd.end(),
                   [](const HostSeries& x, const HostSeries& y) { return x.L < y.L; });
  return run_tc(h, sd.data(), nset, D, s, false, true);
}

traknn_status traknn_partition(int64_t M, int L, int nparts, int part, int64_t* row_lo,
                               int64_t* row_hi) {
  if (!row_lo || !row_hi || M < 1 || M > INT_MAX / 2 || L < 1 || L > TRAKNN_MAX_L ||
      nparts < 1 || nparts > TRAKNN_MAX_PARTS || part < 0 || part >= nparts)
    return TRAKNN_ERR_INVALID_ARG;
  int s_lo = 0, s_hi = 0;
  split_strips(M, L, nparts, part, &s_lo, &s_hi);
  const int64_t R = kTileRows - (L - 1);
  *row_lo = std::min<int64_t>(M, s_lo * R);
  *row_hi = std::min<int64_t>(M, s_hi * R);
  return TRAKNN_OK;
}

traknn_status traknn_knn_partial(traknn_handle h, const float* X, int64_t N, int64_t D, int L,
                                 int k, int e, int part, int nparts, int32_t* part_idx,
                                 float* part_dist, void* stream) {
  TRY_ST(check_handle(h));
  if (!X || !part_idx || !part_dist) return TRAKNN_ERR_INVALID_ARG;
  TRY_ST(traknn_check_problem(N, D, L, k, e));
  if (nparts < 1 || nparts > TRAKNN_MAX_PARTS || part < 0 || part >= nparts)
    return TRAKNN_ERR_INVALID_ARG;
  if (h->weights && h->weights_D != D) return TRAKNN_ERR_INVALID_ARG;
  if (h->precision == TRAKNN_PREC_FP32 || !h->sym) return TRAKNN_ERR_UNSUPPORTED;
  int s_lo = 0, s_hi = 0;
  split_strips(N - L + 1, L, nparts, part, &s_lo, &s_hi);
  const HostSeries sd{X, N, L, k, e, part_idx, part_dist, nullptr};
  return run_tc(h, &sd, 1, D, static_cast<cudaStream_t>(stream), false, false, 1, s_lo, s_hi);
}

traknn_status traknn_merge_partials(traknn_handle h, const int32_t* idx_parts,
                                    const float* dist_parts, int nparts, int64_t M, int k,
                                    int32_t* nbr_idx, float* nbr_dist, float* score,
                                    void* stream) {
  TRY_ST(check_handle(h));
  if (!idx_parts || !dist_parts || !nbr_idx || !nbr_dist || !score) return TRAKNN_ERR_INVALID_ARG;
  if (nparts < 1 || nparts > TRAKNN_MAX_PARTS || M < 1 || M > INT_MAX / 2 || k < 1 ||
      k > TRAKNN_MAX_K)
    return TRAKNN_ERR_INVALID_ARG;
  TRY_CUDA(launch_merge_parts(idx_parts, dist_parts, nparts, (int)M, k, nbr_idx, nbr_dist, score,
                              static_cast<cudaStream_t>(stream)));
  h->launches += 1;
  return TRAKNN_OK;
}

traknn_status traknn_set_grid_weights(traknn_handle h, const float* weights, int64_t D) {
  if (!h) return TRAKNN_ERR_INVALID_ARG;
  if (weights && (D < 1 || D > INT_MAX / 2)) return TRAKNN_ERR_INVALID_ARG;
  h->weights = weights;
  h->weights_D = weights ? D : 0;
  return TRAKNN_OK;
}

traknn_status traknn_knn_stats(traknn_handle h, const float* nbr_dist, int64_t M, int k,
                               float* prefix_scores, int k_id, float* local_id, void* stream) {
  TRY_ST(check_handle(h));
  if (!nbr_dist || M < 1 || M > INT_MAX / 2 || k < 1 || k > TRAKNN_MAX_K)
    return TRAKNN_ERR_INVALID_ARG;
  if (!prefix_scores && !local_id) return TRAKNN_ERR_INVALID_ARG;
  if (local_id && (k_id < 2 || k_id > k)) return TRAKNN_ERR_INVALID_ARG;
  TRY_CUDA(launch_knn_stats(nbr_dist, (int)M, k, prefix_scores, k_id, local_id,
                            static_cast<cudaStream_t>(stream)));
  h->launches += 1;
  return TRAKNN_OK;
}

traknn_status traknn_knn_scores_host(traknn_handle h, const float* Xh, int64_t N, int64_t D,
                                     int L, int k, int e, int32_t* idx_h, float* dist_h,
                                     float* score_h, void* stream) {
  TRY_ST(check_handle(h));
  if (!Xh || !idx_h || !dist_h || !score_h) return TRAKNN_ERR_INVALID_ARG;
  TRY_ST(traknn_check_problem(N, D, L, k, e));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t M = N - L + 1;
  const size_t xb = align_up((size_t)N * D * sizeof(float), 256);
  const size_t ib = align_up((size_t)M * k * sizeof(int32_t), 256);
  const size_t db = align_up((size_t)M * k * sizeof(float), 256);
  const size_t sb = align_up((size_t)M * sizeof(float), 256);
  TRY_ST(ensure_buffer(h, &h->io, &h->io_bytes, xb + ib + db + sb));
  char* io = static_cast<char*>(h->io);
  float* Xd = reinterpret_cast<float*>(io);
  int32_t* idx_d = reinterpret_cast<int32_t*>(io + xb);
  float* dist_d = reinterpret_cast<float*>(io + xb + ib);
  float* score_d = reinterpret_cast<float*>(io + xb + ib + db);
  // Phases when the series has enough strips: its days are copied in on the copy
  // stream from the last ones back, and the strips whose days are in start while the
  // copy of the earlier days continues (see phase_plan and enqueue_tc_phased)
  const int R = kTileRows - (L - 1);
  const int strips = (int)((M + R - 1) / R);
  const bool tc_form = h->precision != TRAKNN_PREC_FP32 && h->sym && !use_embedding(h, D, L) &&
                       (!h->weights || h->weights_D == D) && tc_available();
  const std::vector<int> ps = tc_form ? phase_plan(strips, R, N) : std::vector<int>();
  if (ps.empty()) {
    TRY_CUDA(cudaMemcpyAsync(Xd, Xh, (size_t)N * D * sizeof(float), cudaMemcpyHostToDevice, s));
    TRY_ST(traknn_knn_scores(h, Xd, N, D, L, k, e, idx_d, dist_d, score_d, stream));
  } else {
    if (!h->copy_stream) {
      TRY_CUDA(cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking));
      TRY_CUDA(cudaEventCreateWithFlags(&h->ev_io_free, cudaEventDisableTiming));
      for (cudaEvent_t& ev : h->ev_in)
        TRY_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    }
    const HostSeries sd{Xd, N, L, k, e, idx_d, dist_d, score_d};
    int tiles = 8, group = 0;
    default_shape(h, &sd, 1, D, 1, 0, INT_MAX, &tiles, &group);
    TcBuffers buf;
    TRY_ST(prepare_tc(h, &sd, 1, D, tiles, false, 1, s, &buf, 0, INT_MAX, ps, group));
    const size_t row = (size_t)D * sizeof(float);
    const cudaStream_t cs = h->copy_stream;
    // the staging buffer is rewritten only after earlier work on `stream` is done
    TRY_CUDA(cudaEventRecord(h->ev_io_free, s));
    TRY_CUDA(cudaStreamWaitEvent(cs, h->ev_io_free, 0));
    for (int q = 0; q + 1 < (int)ps.size(); ++q) {
      const int64_t lo = (int64_t)ps[q + 1] * R, hi = q == 0 ? N : (int64_t)ps[q] * R;
      TRY_CUDA(cudaMemcpyAsync(Xd + lo * D, Xh + lo * D, (size_t)(hi - lo) * row,
                               cudaMemcpyHostToDevice, cs));
      TRY_CUDA(cudaEventRecord(h->ev_in[q], cs));
    }
    TRY_ST(enqueue_tc_phased(h, buf, D, s, h->ev_in));
  }
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
  TRY_ST(check_handle(h));
  if (!X || !nbr_idx || !grad_score || !dX) return TRAKNN_ERR_INVALID_ARG;
  if (N < 1 || D < 1 || L < 1 || L > N || k < 1) return TRAKNN_ERR_INVALID_ARG;
  if (N > INT_MAX / 2 || D > INT_MAX / 2) return TRAKNN_ERR_INVALID_ARG;
  if (L > TRAKNN_MAX_L || k > TRAKNN_MAX_K) return TRAKNN_ERR_UNSUPPORTED;
  TRY_ST(ensure_buffer(h, &h->adj, &h->adj_bytes, adjoint_workspace_bytes((int)N, L, k)));
  int launches = 0;
  if (h->weights && h->weights_D != D) return TRAKNN_ERR_INVALID_ARG;
  TRY_CUDA(launch_adjoint(X, (int)N, (int)D, L, k, nbr_idx, grad_score, h->weights, dX, h->adj,
                          h->err,
                          static_cast<cudaStream_t>(stream), &launches));
  h->launches += launches;
  return TRAKNN_OK;
}

traknn_status traknn_sync_status(traknn_handle h, void* stream) {
  TRY_ST(check_handle(h));
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
  TRY_ST(check_handle(h));
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
  TRY_ST(check_handle(h));
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

traknn_status traknn_work_shape(traknn_handle h, int* tiles_per_unit, int* group_strips) {
  if (!h || !tiles_per_unit || !group_strips) return TRAKNN_ERR_INVALID_ARG;
  *tiles_per_unit = h->last_tiles;
  *group_strips = h->last_group;
  return TRAKNN_OK;
}

traknn_status traknn_launch_count(traknn_handle h, int64_t* count) {
  if (!h || !count) return TRAKNN_ERR_INVALID_ARG;
  *count = h->launches;
  return TRAKNN_OK;
}

}  // extern "C"
