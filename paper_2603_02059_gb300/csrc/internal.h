// internal.h -- parameters and launchers shared by the CUDA translation units
// of libtraknn (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace traknn {

// Rows of one Gram tile (the tcgen05 accumulator height and the FP32 SIMT tile).
constexpr int kTileRows = 128;
// Columns of one tensor-core Gram tile (one TMEM accumulator).
constexpr int kTileCols = 256;
// Default length (elements of K) of one tensor-core accumulation segment: the
// tensor cores accumulate at most this many products per output before the
// partial sum is added, in FP32 on the CUDA cores, to the tile's running total.
constexpr int kSegmentK = 8192;
// Left halo kept beside each G tile in shared memory: the diagonal window of
// Eq. 2 reaches L-1 <= kHalo columns to the right of an output column.
constexpr int kHalo = 16;
constexpr int kMaxL = kHalo + 1;
constexpr int kMaxK = 64;
// Status word value a kernel records when one of its bounded waits runs out
// (matches TRAKNN_ERR_TIMEOUT of the public header).
constexpr int kErrTimeout = 5;
// ... and when an input it reads is out of range (TRAKNN_ERR_INVALID_ARG).
constexpr int kErrInvalidArg = 1;
// Column-mean partial sums use this many row slices (fixed order => deterministic).
constexpr int kMeanSlices = 64;
// Centring: the per-grid-point mean over the last kMeanDays days (all days when there
// are fewer): days [mean_first(N), N). A host-buffer call copies those days in first.
constexpr int kMeanDays = 4096;
__host__ __device__ inline int mean_days(int N) { return N < kMeanDays ? N : kMeanDays; }
__host__ __device__ inline int mean_first(int N) { return N - mean_days(N); }
// Status word value of the debug build's index checks (TRAKNN_ERR_BOUNDS).
constexpr int kErrBounds = 9;

// Index check of the debug build (compiled with -DTRAKNN_BOUNDS_CHECK): an index i
// outside [0, n) records kErrBounds in the status word and the caller skips the
// access, so a wrong index is reported by traknn_sync_status instead of touching
// memory it does not own. In the regular build the check compiles to nothing.
#ifdef TRAKNN_BOUNDS_CHECK
__device__ __forceinline__ bool tk_in(long long i, long long n, int* err) {
  if (i >= 0 && i < n) return true;
  atomicCAS(err, 0, kErrBounds);
  return false;
}
#else
__device__ __forceinline__ bool tk_in(long long, long long, int*) { return true; }
#endif

// Work decomposition of the M x M trajectory-pair space shared by the fused
// Gram/top-k kernels and the merge.
//   strip s : output rows t in [s*rows_out, (s+1)*rows_out), rows_out = 128 - (L-1);
//             its Gram tiles start at day row s*rows_out and span 128 day rows.
//   chunk c : output columns j in [c*chunk_cols, min(M, (c+1)*chunk_cols)).
//   unit    : one (strip, chunk); a CTA walks the unit's Gram tiles left to right,
//             carrying the last L-1 Gram columns from tile to tile.
// Units are numbered in groups of `group_strips` strips x all chunks so that the
// CTAs running at the same time share strips and column ranges in L2.
struct Schedule {
  int M, L, k, e;
  int rows_out;      // output rows per strip
  int strips;        // ceil(M / rows_out)
  int chunks;        // column chunks
  int chunk_cols;    // output columns per chunk
  int group_strips;  // strips per scheduling group
  int units;         // ceil(strips/group_strips) * group_strips * chunks (some empty)
};

struct UnitCoord {
  int strip, chunk;
};

__host__ __device__ inline UnitCoord unit_coord(const Schedule& s, int u) {
  int per_group = s.group_strips * s.chunks;
  int g = u / per_group;
  int r = u - g * per_group;
  UnitCoord c;
  c.chunk = r / s.group_strips;
  c.strip = g * s.group_strips + (r - c.chunk * s.group_strips);
  return c;
}

// Work split of the M x M pair space of the FP32 path (see Schedule above);
// chunks_opt = 0 takes 8 column chunks (at most 32, at most M).
inline Schedule make_schedule(int M, int L, int k, int e, int sm_count, int chunks_opt) {
  Schedule s;
  s.M = M;
  s.L = L;
  s.k = k;
  s.e = e;
  s.rows_out = kTileRows - (L - 1);
  s.strips = (M + s.rows_out - 1) / s.rows_out;
  int chunks = chunks_opt > 0 ? chunks_opt : 8;
  chunks = chunks < 32 ? chunks : 32;
  chunks = chunks < M ? chunks : M;
  chunks = chunks > 1 ? chunks : 1;
  s.chunk_cols = (M + chunks - 1) / chunks;
  s.chunks = (M + s.chunk_cols - 1) / s.chunk_cols;  // every chunk non-empty
  s.group_strips = sm_count / s.chunks > 1 ? sm_count / s.chunks : 1;
  const int groups = (s.strips + s.group_strips - 1) / s.group_strips;
  s.units = groups * s.group_strips * s.chunks;
  return s;
}

// Byte offsets of the FP32 path's workspace (each piece starts on a 256-byte
// boundary): column partial sums, mean, FP64 day norms, window sums, the centred
// FP32 copy (row pitch Dp = D rounded up to 32) and the partial neighbour lists.
struct Fp32Layout {
  size_t partial, mu, norms, W, ops, pd, pi, total;
  int Dp;
};

inline Fp32Layout make_layout(int64_t N, int64_t D, const Schedule& s) {
  Fp32Layout l;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    off = (off + 255) / 256 * 256;
    const size_t o = off;
    off += bytes;
    return o;
  };
  l.Dp = (int)((D + 31) / 32 * 32);
  l.partial = take((size_t)kMeanSlices * D * sizeof(float));
  l.mu = take((size_t)D * sizeof(float));
  l.norms = take((size_t)N * sizeof(double));
  l.W = take((size_t)s.M * sizeof(float));
  l.ops = take((size_t)N * l.Dp * 4);
  l.pd = take((size_t)s.M * s.chunks * s.k * sizeof(float));
  l.pi = take((size_t)s.M * s.chunks * s.k * sizeof(int32_t));
  l.total = off;
  return l;
}

struct FusedArgs {
  Schedule sch;
  int N;              // days
  int Dp;             // padded row pitch of the operand copies (elements), multiple of 32
  const float* W;     // [M] window sums of day norms, FP32
  float* part_d;      // [M][chunks][k] partial neighbour distances (sorted per list)
  int32_t* part_i;    // [M][chunks][k] partial neighbour indices (-1 = empty)
  int* err;           // device status word (0 = ok, else a traknn_status)
  long long wait_limit_ns;
  int debug_withhold;
};

// One series of a tensor-core call. A call processes one or more independent
// series (same D, own N, L, k, exclusion); their operand copies are stacked in one
// buffer and their trajectory rows in one index space.
struct SeriesInfo {
  int N, M, L, k;
  int e;
  int rows_out;         // output rows per strip: 128 - (L-1), or less when series share tiles
  int step;             // output columns of a one-tile unit: 256 - (L-1), or less likewise
  int row_base;         // first stacked operand row (day 0 of the series)
  int out_base;         // first stacked trajectory row
  int slots;            // row-side list slots per trajectory row
  int strip_base;       // index of the series' strip 0 in col_off / slot_lo
  long long part_base;  // first row-side list of the series
  long long col_base;   // first column list of the series
  const float* X;       // input [N][D]
  int32_t* idx;         // outputs [M][k], [M][k], [M]
  float* dist;
  float* score;
};

// Series of one tensor-core launch, passed by value as a kernel parameter.
constexpr int kMaxSeries = 64;
struct SeriesTable {
  int n;
  int pad[3];
  SeriesInfo s[kMaxSeries];
};

// Work list of the tensor-core kernel. A unit is one row strip of one series and
// one column range; its Gram tiles are walked left to right. With `sym` set only
// the upper triangle of each series' pair space is evaluated: strip s covers
// columns j >= T0_s; inside its own block [T0_s, T0_s + rows_out) only the rows
// collect candidates, beyond it every tile also gives each column j the strip's
// rows as candidates (the column side), so every unordered pair is evaluated once.
struct WorkUnit {
  int series;  // first (or only) series of the unit
  int strip;   // row strip; output rows [strip*rows_out, (strip+1)*rows_out)
  int jlo;     // first output column
  int jhi;     // one past the last output column (clipped to each series' M)
  int slot;    // slot of the row-side partial lists written by this unit
  int pad[3];  // pad[0]: number of consecutive series sharing the unit's Gram tiles
};

struct TcWork {
  const WorkUnit* units;
  int nunits;
  int kstride;              // list pitch: largest k of the call rounded up to 4
  const long long* col_off; // [stacked strips] column-list offset within the series
  const int* slot_lo;       // [stacked strips] first slot written for the strip's rows
  int sym;                  // 1: upper triangle + column side
  // Column-side candidate lists, one record of col_pitch() ints per list:
  // [n, unused, row_0, dist_0, row_1, dist_1, ...] (distances as FP32 bit patterns,
  // entries in row order or, for a full list, the k best), 16-byte aligned, so that
  // one 16-byte load gives the count and the first entry.
  int32_t* col_rec;
  long long col_ints;       // ints of col_rec (index checks of the debug build)
  // [stacked rows][mask_words] bit s of a row's mask: the column list of strip s for
  // that row (as a column) is non-empty; only those lists have a record written
  unsigned int* col_mask;
  int mask_words;
  long long part_ints;      // entries of each row-side list array (likewise)
  unsigned int* thr;        // [stacked rows] bit patterns of an upper bound of each row's k-th distance
  int* counter;             // next unit to hand out (zero before the launch)
  int write_lists;          // 0: only publish row bounds (band pre-pass)
  unsigned long long* stats;  // optional event counters (see kStat*), nullptr = off
  // Strips [part_lo, part_hi) of the (single) series were evaluated by this call (one
  // part of a series split across processes); the merge reads only their lists.
  // Every other call: 0 and INT_MAX.
  int part_lo, part_hi;
};

// Ints per column-list record for list pitch kstride (a multiple of 4).
__host__ __device__ inline int col_pitch(int kstride) { return 4 + 2 * kstride; }

struct TcArgs {
  int Dp;              // padded row pitch of the stacked operand copies
  int rows;            // stacked operand rows
  int out_rows;        // stacked trajectory rows
  int Lmax, kmax;      // largest L and k of the call (shared-memory sizing)
  const float* W;      // [out_rows] window sums of day norms
  float* part_d;       // [lists][kstride] row-side partial lists
  int32_t* part_i;
  int* err;
  long long wait_limit_ns;
  int debug_withhold;
  int seg_k;           // elements of K per accumulation segment (multiple of 32)
  int groups;          // K groups of the operand layout (see tc_groups)
  const float* cval;   // [rows] correction value c of every stacked operand row
  int l2_keep_a;       // 1: load the strip operand with an L2 evict-last policy
  float* scratch;      // [CTAs][2][128 x 256] running tile totals (more than one segment)
  int egroups;         // epilogue groups of the tensor-core kernel (1, or 2 at L = 1)
  // Band pre-pass in one BF16 product (hi only) on split operands: the correction
  // entries then add +groups c_a c_b, which the epilogue subtracts (corr_neg = 1), and
  // every distance is raised by band_margin (W_t + W_j), a bound of its error, before
  // it enters a list, so that the bounds it publishes stay upper bounds. 0 and 0.0f
  // for every other launch.
  int corr_neg;
  float band_margin;
};

// Bytes of TcArgs::scratch for a launch of `num_ctas` CTAs.
inline size_t tc_scratch_bytes(int num_ctas) {
  return (size_t)num_ctas * 2 * kTileRows * kTileCols * sizeof(float);
}

// Event counters of the tensor-core kernel (diagnostics, TRAKNN_OPT_STATS).
enum : int {
  kStatRowInserts = 0,     // row-side list insertions
  kStatColEmits = 1,       // column-side candidates handed to a column
  kStatColFull = 2,        // column lists with more than k candidates (k best kept)
  kStatColLists = 3,       // non-empty column lists written
  kStatChunks = 4,         // 32-column chunks processed
  kStatMmaWaitTmem = 5,    // MMA-thread cycles spent waiting for a free accumulator
  kStatMmaWaitFull = 6,    // MMA-thread cycles spent waiting for a filled stage
  kStatMmaCycles = 7,      // MMA-thread cycles from start to end, summed over CTAs
  // epilogue phases, timed by its first thread (cycles, summed over CTAs)
  kStatEpiWaitAcc = 8,     // waiting for a filled accumulator
  kStatEpiTileHead = 9,    // per-tile loads of window sums and column bounds
  kStatEpiStage = 10,      // TMEM read-out and staging of a chunk
  kStatEpiBar1 = 11,       // barrier after staging (waits for the slowest thread)
  kStatEpiScan = 12,       // row-side scan and emissions, to the barrier after them
  kStatEpiCol = 13,        // column-side lists (and dense recomputation)
  kStatEpiCycles = 14,     // epilogue first thread from start to end
  kStatCount = 15
};

// ----------------------------------------------------------------- launchers
cudaError_t launch_col_mean(const float* X, int N, int D, float* partial, float* mu,
                            bool center, cudaStream_t st);
// wts: optional [D] grid-point weights (the values are scaled by sqrt(w_p)), or null.
cudaError_t launch_prep_fp32(const float* X, int N, int D, int Dp, const float* mu,
                             const float* wts, float* Xc, double* norms, cudaStream_t st);
cudaError_t launch_window(const double* norms, int M, int L, float* W, cudaStream_t st);
cudaError_t launch_fused_fp32(const float* Xc, const FusedArgs& a, int num_ctas,
                              cudaStream_t st);
// Tensor-core path; `split` selects the 3-product split-BF16 form.
cudaError_t launch_fused_tc(const void* hi, const void* lo, bool split, const TcArgs& a,
                            const TcWork& w, const SeriesTable& sr, int num_ctas, cudaStream_t st);
// Final neighbour sets of the tensor-core path: candidates of every row's partial
// lists (and column lists) that do not exceed its bound, then an exact top-k,
// written to each series' output buffers.
cudaError_t launch_merge_tc(const TcArgs& a, const TcWork& w, const SeriesTable& sr,
                            cudaStream_t st);
// Series-aware preparation for the tensor-core path (stacked operands).
cudaError_t launch_col_mean_series(const SeriesTable& sr, int D, float* partial, float* mu,
                                   bool center, cudaStream_t st);
// Operand layout of the tensor-core path: groups = ceil(D / 63) groups of 64 K
// entries (63 permuted grid points + 1 correction entry); pitch groups * 64.
inline int tc_groups(int D) { return (D + 62) / 63; }

// Split of one series' upper-triangle work over `nparts` processes: contiguous ranges
// of row strips (strip height R = 128 - (L-1)) with about equal work, strip s holding
// (M - s R) R of the M (M+1)/2 unordered pairs. Strips [*s_lo, *s_hi) go to `part`;
// an unordered pair {a, b} is evaluated in the part whose strips hold min(a, b).
inline void split_strips(long long M, int L, int nparts, int part, int* s_lo, int* s_hi) {
  const long long R = kTileRows - (L - 1);
  const long long S = (M + R - 1) / R;
  long long total = 0;
  for (long long s = 0; s < S; ++s) total += M - s * R;
  auto first = [&](int p) -> int {  // first strip of part p: cumulative work >= p/nparts
    if (p <= 0) return 0;
    if (p >= nparts) return (int)S;
    long long cum = 0, s = 0;
    while (s < S && cum * nparts < (long long)p * total) cum += M - (s++) * R;
    return (int)s;
  };
  *s_lo = first(part);
  *s_hi = first(part + 1);
}
// emb > 1: each operand row is the emb-day trajectory starting at that day (emb * D
// values, contiguous in X); the series table then describes trajectories (N = M, L = 1).
// Rows [r_lo, rows) of the stacked operands (all rows with r_lo = 0).
cudaError_t launch_prep_split_series(const SeriesTable& sr, int rows, int D, int emb, int groups,
                                     bool correct, const float* mu, const float* wts, void* hi,
                                     void* lo, double* norms, float* cval, cudaStream_t st,
                                     int r_lo = 0);
// Window sums of the stacked trajectory rows [r_lo, out_rows).
cudaError_t launch_window_series(const SeriesTable& sr, int out_rows, const double* norms,
                                 float* W, cudaStream_t st, int r_lo = 0);
cudaError_t launch_merge(const FusedArgs& a, int32_t* idx, float* dist, float* score,
                         cudaStream_t st);
// Exact top-k of the union of nparts sorted candidate lists per row ([nparts][M][k],
// index -1 = empty entry), with the rarity score (FP64 mean); nparts <= 32.
cudaError_t launch_merge_parts(const int32_t* idx_parts, const float* dist_parts, int nparts,
                               int M, int k, int32_t* idx, float* dist, float* score,
                               cudaStream_t st);
// Adjoint of the summed weighted score (kernels_adjoint.cu); `ws` must hold
// adjoint_workspace_bytes(N, L, k) bytes. Adds the number of launches to *launches.
size_t adjoint_workspace_bytes(int N, int L, int k);
// wts: optional [D] grid-point weights (dX is multiplied by w_p), or null.
cudaError_t launch_adjoint(const float* X, int N, int D, int L, int k, const int32_t* idx,
                           const float* g, const float* wts, float* dX, void* ws, int* err,
                           cudaStream_t st, int* launches);
// Scores for every k' <= k (prefix means of each sorted row, FP64 sums) and the
// Levina-Bickel local intrinsic dimension for k_id <= k; either output may be null.
cudaError_t launch_knn_stats(const float* dist, int M, int k, float* prefix, int k_id,
                             float* local_id, cudaStream_t st);
size_t fused_fp32_smem_bytes(int k);
// False until the tensor-core kernel is compiled in.
bool tc_available();

size_t fused_tc_smem_bytes(bool split, int kmax, int Lmax, int G);

}  // namespace traknn
