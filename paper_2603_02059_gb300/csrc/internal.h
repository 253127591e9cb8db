// internal.h -- parameters and launchers shared by the CUDA translation units
// of libtraknn (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace traknn {

// Rows of one Gram tile (the tcgen05 accumulator height and the FP32 SIMT tile).
constexpr int kTileRows = 128;
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

// Work list of the tensor-core kernel. A unit is one row strip and one column
// range; its Gram tiles are walked left to right with the diagonal carry.
// With `sym` set only the upper triangle of the pair space is evaluated: strip s
// covers columns j >= T0_s; inside its own block [T0_s, T0_s + rows_out) only the
// rows collect candidates, beyond it every tile also gives each column j the
// strip's rows as candidates (the column side), so every unordered pair is
// evaluated once.
struct WorkUnit {
  int strip;  // row strip; output rows [strip*rows_out, (strip+1)*rows_out)
  int jlo;    // first output column
  int jhi;    // one past the last output column
  int slot;   // slot of the row-side partial lists written by this unit
};

struct TcWork {
  const WorkUnit* units;
  int nunits;
  int slots;                // row-side partial list slots per row
  const int* slot_lo;       // [strips] first slot written for the strip's rows
  int sym;                  // 1: upper triangle + column side
  const long long* col_off; // [strips] first column-list of strip s (sym only)
  float* col_d;             // [lists][k] column-side candidate distances (sorted)
  int32_t* col_i;           // [lists][k] column-side candidate rows
  int32_t* col_n;           // [lists] number of valid entries of each column list
  unsigned int* thr;        // [M] bit patterns of an upper bound of each row's k-th distance
  int* counter;             // next unit to hand out (zero before the launch)
  int write_lists;          // 0: only publish row bounds (band pre-pass)
  unsigned long long* stats;  // optional event counters (see kStat*), nullptr = off
};

// Event counters of the tensor-core kernel (diagnostics, TRAKNN_OPT_STATS).
enum : int {
  kStatRowInserts = 0,     // row-side list insertions
  kStatColEmits = 1,       // column-side candidates handed to a column
  kStatColDense = 2,       // columns recomputed densely after a buffer overflow
  kStatColLists = 3,       // non-empty column lists written
  kStatChunks = 4,         // 32-column chunks processed
  kStatMmaWaitTmem = 5,    // MMA-thread cycles spent waiting for a free accumulator
  kStatMmaWaitFull = 6,    // MMA-thread cycles spent waiting for a filled stage
  kStatMmaCycles = 7,      // MMA-thread cycles from start to end, summed over CTAs
  kStatCount = 8
};

// ----------------------------------------------------------------- launchers
cudaError_t launch_col_mean(const float* X, int N, int D, float* partial, float* mu,
                            bool center, cudaStream_t st);
cudaError_t launch_prep_fp32(const float* X, int N, int D, int Dp, const float* mu,
                             float* Xc, double* norms, cudaStream_t st);
cudaError_t launch_prep_split(const float* X, int N, int D, int Dp, const float* mu,
                              void* hi, void* lo, double* norms, cudaStream_t st);
cudaError_t launch_window(const double* norms, int M, int L, float* W, cudaStream_t st);
cudaError_t launch_fused_fp32(const float* Xc, const FusedArgs& a, int num_ctas,
                              cudaStream_t st);
// Tensor-core path; `split` selects the 3-product split-BF16 form.
cudaError_t launch_fused_tc(const void* hi, const void* lo, bool split, const FusedArgs& a,
                            const TcWork& w, int num_ctas, cudaStream_t st);
// Final neighbour sets of the tensor-core path: candidates of every row's partial
// lists (and column lists) that do not exceed its bound, then an exact top-k.
cudaError_t launch_merge_tc(const FusedArgs& a, const TcWork& w, int32_t* idx, float* dist,
                            float* score, cudaStream_t st);
cudaError_t launch_merge(const FusedArgs& a, int32_t* idx, float* dist, float* score,
                         cudaStream_t st);
// Adjoint of the summed weighted score (kernels_adjoint.cu); `ws` must hold
// adjoint_workspace_bytes(M, k) bytes. Adds the number of launches to *launches.
size_t adjoint_workspace_bytes(int M, int k);
cudaError_t launch_adjoint(const float* X, int N, int D, int L, int k, const int32_t* idx,
                           const float* g, float* dX, void* ws, int* err, cudaStream_t st,
                           int* launches);
size_t fused_fp32_smem_bytes(int k);
// False until the tensor-core kernel is compiled in.
bool tc_available();
// Epilogue groups the tensor-core kernel runs with for k neighbours; each group
// keeps its own row-side partial list per work unit.
int tc_groups(int k);
size_t fused_tc_smem_bytes(bool split, int k, int L);

}  // namespace traknn
