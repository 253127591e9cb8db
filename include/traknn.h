/*
 * traknn.h -- C ABI of the GB300 (sm_103a) trajectory-kNN rarity library.
 *
 * The library computes, for a sequence of N daily fields X (row-major N x D,
 * float32, one row per day), the exact k nearest neighbours of every L-day
 * trajectory and its rarity score, as defined in TRAKNN (arXiv 2603.02059):
 *
 *   trajectory      T_t = (X_t, ..., X_{t+L-1}),  t = 0 .. M-1,  M = N - L + 1
 *                                                   (Sec. 3.2, Eq. 1)
 *   distance        D(t,j) = sum_{m<L} ||X_{t+m} - X_{j+m}||^2   (Sec. 3.2, Eq. 2)
 *   candidates      j with |t - j| > exclusion                   (Sec. 3.2)
 *   neighbour set   the k candidates with smallest D(t,j); ties go to the
 *                   smaller index                                (Algorithm 1, kNN step)
 *   rarity score    s_t = (1/k) sum_{j in N_t} D(t,j)             (Sec. 3.2, Eq. 3)
 *
 * Distances are squared (no square root), as in Eq. 2-3. Indices are 0-based.
 *
 * Conventions for every entry point:
 *   - Pointers named X, nbr_*, score, grad_score, dX are DEVICE pointers on the
 *     handle's device unless the function name ends in _host. The caller owns
 *     every buffer; the library owns only the workspaces cached in the handle.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream). Device work is enqueued asynchronously on it.
 *   - Argument errors are detected on the host and returned before anything is
 *     enqueued. Device-side failures (a bounded wait that ran out) are recorded
 *     in the handle and reported by traknn_sync_status().
 *   - X must hold finite values. NaN or infinite entries make the affected distances
 *     NaN, which compare false against every bound: their rows' neighbour lists and
 *     scores are then unspecified (entries may be missing, index -1).
 *   - A handle is not thread-safe: serialise calls that share one handle.
 *     Calls on one handle share its workspace, so two calls on different
 *     streams must not overlap on the GPU.
 */
#ifndef TRAKNN_H
#define TRAKNN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Opaque library context: device, options, cached workspaces and tensor maps. */
typedef struct traknn_ctx* traknn_handle;

typedef enum {
  TRAKNN_OK = 0,
  TRAKNN_ERR_INVALID_ARG = 1,        /* null pointer, non-positive size, L > N, k < 1, ... */
  TRAKNN_ERR_TOO_FEW_CANDIDATES = 2, /* k > M - (2*exclusion + 1): some row has < k candidates */
  TRAKNN_ERR_ALLOC = 3,              /* workspace allocation failed */
  TRAKNN_ERR_CUDA = 4,               /* a CUDA runtime call failed */
  TRAKNN_ERR_TIMEOUT = 5,            /* a bounded device-side wait ran out */
  TRAKNN_ERR_UNSUPPORTED_DEVICE = 6, /* the device is not sm_103 */
  TRAKNN_ERR_UNSUPPORTED = 7,        /* L or k above the compiled limits below */
  TRAKNN_ERR_SCRATCH_LIMIT = 8,      /* traknn_knn_scores_static: the problem needs more scratch
                                        than the library's fixed device array holds */
  TRAKNN_ERR_BOUNDS = 9              /* debug build (libtraknn_bounds.so) only: a device-side
                                        index check failed; the access was skipped */
} traknn_status;

/* Arithmetic of the snapshot Gram contraction (the dominant step, Sec. 3.3,
 * "Optimized Spatial Distance Computation"). Day norms, window sums and
 * scores are accumulated in FP64 in every mode. */
typedef enum {
  TRAKNN_PREC_FP32 = 0,       /* CUDA-core FP32 FMA Gram */
  TRAKNN_PREC_SPLIT_BF16 = 1, /* tensor cores: x = hi + lo (two BF16), G = hi.hi + hi.lo + lo.hi, FP32 accumulate */
  TRAKNN_PREC_BF16 = 2        /* tensor cores: single BF16 product, FP32 accumulate (lower accuracy) */
} traknn_precision;

typedef enum {
  TRAKNN_OPT_PRECISION = 0,          /* a traknn_precision value (default SPLIT_BF16) */
  TRAKNN_OPT_CENTER = 1,             /* 1: subtract the per-grid-point mean over days before the
                                        Gram (the last 4,096 days, or all when fewer; exact by the
                                        offset invariance of Eq. 2 whatever the mean; default 1) */
  TRAKNN_OPT_COL_CHUNKS = 2,         /* column chunks per row strip, 0 = automatic */
  TRAKNN_OPT_WAIT_LIMIT_MS = 3,      /* limit of every device spin-wait in ms (default 2000) */
  TRAKNN_OPT_DEBUG_WITHHOLD = 4,     /* test hook: 1 makes the tensor-core kernel's producer withhold
                                        the first stage of work unit 0, so that the consumer's bounded
                                        wait runs out and the call reports TRAKNN_ERR_TIMEOUT
                                        (default 0) */
  TRAKNN_OPT_PROFILE = 5,            /* 1: record CUDA events around the fused Gram/top-k kernel of
                                        every forward call (read with traknn_profile_read) */
  TRAKNN_OPT_SYMMETRIC = 6,          /* tensor-core paths: 1 evaluates each unordered pair once
                                        (upper triangle, Sec. 3.3), 0 both triangles (default 1) */
  TRAKNN_OPT_UNIT_COLS = 7,          /* tensor-core paths: output columns per work unit; 0 = auto:
                                        units of 2, 4 or 8 Gram tiles of 256 columns, by the Gram
                                        tiles per SM of an average series of the call (8 from
                                        64, 4 from 16) and at most 65,536 operand K entries x
                                        tiles; 16 tiles for operand rows of at most 768 K
                                        entries (the results are the same) */
  TRAKNN_OPT_STATS = 8,              /* 1: count kernel events (read with traknn_stats_read) */
  TRAKNN_OPT_AUTOTUNE = 9,           /* tensor-core paths: 1 times every work-unit shape of
                                        {4, 8, 16} Gram tiles per unit x {10, 19, 38} row strips
                                        run side by side (the strips only while
                                        TRAKNN_OPT_GROUP_STRIPS is 0) on the first call of each
                                        problem shape and keeps the fastest (ignored while
                                        TRAKNN_OPT_UNIT_COLS is set; default 0) */
  TRAKNN_OPT_SEGMENT_K = 10,         /* tensor-core paths: the tensor cores accumulate at most this
                                        many grid points (a multiple of 32) of a Gram entry before
                                        the partial sum is added in FP32 to the entry's running
                                        total; shorter segments bound the error of the tensor-core
                                        accumulation over large D (0 = default 8192) */
  TRAKNN_OPT_GROUP_STRIPS = 11,      /* tensor-core paths: row strips whose work units are handed
                                        out side by side (sharing operand tiles in L2; 0 = 19) */
  TRAKNN_OPT_L2_KEEP_A = 12,         /* tensor-core paths: 1 loads a unit's row-strip operand with
                                        an L2 evict-last policy (it is re-read for every tile of
                                        the unit; default 0) */
  TRAKNN_OPT_EMBED = 13,             /* tensor-core traknn_knn_scores with L > 1: 1 builds one
                                        operand row per trajectory (its L days, Eq. 1, L*D values)
                                        so that one Gram entry is the whole window sum of Eq. 2
                                        (L times the contraction, no diagonal sums); 2 never;
                                        0 (default) when L*D <= 1536, the small-grid form (Sec. 5:
                                        fields reduced to a few dozen principal components) */
  TRAKNN_OPT_EPI_GROUPS = 14         /* tensor-core paths: 1 keeps one epilogue warpgroup; 0
                                        (default) uses two at L = 1 (embedded operands included)
                                        when the grid fits one accumulation segment and k <= 32,
                                        each reading half of every tile's columns (the results
                                        are the same) */
} traknn_option;

#define TRAKNN_MAX_L 17  /* longest trajectory (days) supported */
#define TRAKNN_MAX_K 64  /* largest neighbour count supported */
#define TRAKNN_MAX_PARTS 32  /* most parts of one series split across processes */

/* Create a handle on CUDA device `device` (must be compute capability 10.3).
 * Returns TRAKNN_ERR_UNSUPPORTED_DEVICE on any other device. */
traknn_status traknn_create(traknn_handle* handle, int device);

/* Free the handle and its workspaces. Synchronises the handle's device. */
traknn_status traknn_destroy(traknn_handle handle);

/* Set an option (see traknn_option). Takes effect at the next call. */
traknn_status traknn_set_option(traknn_handle handle, traknn_option option, int64_t value);

/* Pure host check of a problem shape; returns the status a compute call would
 * return for these sizes (no device needed). */
traknn_status traknn_check_problem(int64_t N, int64_t D, int L, int k, int exclusion);

/* Forward pass (Sec. 3.2 Eq. 2-3, Algorithm 1):
 *   X         [N x D] float32, row-major, leading dimension D (device)
 *   L         trajectory length in days, 1 <= L <= min(N, TRAKNN_MAX_L)
 *   k         neighbours, 1 <= k <= min(TRAKNN_MAX_K, M - (2*exclusion + 1))
 *   exclusion e >= 0; j is a candidate of t only if |t - j| > e
 *   nbr_idx   [M x k] int32 out: neighbour trajectory indices, each row sorted by
 *             ascending (distance, index)
 *   nbr_dist  [M x k] float32 out: the matching D(t, j)
 *   score     [M] float32 out: s_t, the mean of the row's k distances (summed in FP64)
 * Workspace grows on demand (a cudaMalloc on the first call of a larger size). */
traknn_status traknn_knn_scores(traknn_handle handle, const float* X, int64_t N, int64_t D,
                                int L, int k, int exclusion, int32_t* nbr_idx, float* nbr_dist,
                                float* score, void* stream);

/* Same as traknn_knn_scores with HOST buffers: copies X to the device, runs,
 * copies the results back and synchronises the stream before returning.
 * Page-locked host buffers give the fastest copies. */
traknn_status traknn_knn_scores_host(traknn_handle handle, const float* X_host, int64_t N,
                                     int64_t D, int L, int k, int exclusion,
                                     int32_t* nbr_idx_host, float* nbr_dist_host,
                                     float* score_host, void* stream);

/* Adjoint of the summed weighted score with the neighbour sets held fixed:
 *   dX = d( sum_t grad_score[t] * s_t ) / dX          (derived from Eq. 2-3)
 *   nbr_idx    [M x k] int32 neighbour sets (as returned by the forward pass)
 *   grad_score [M] float32 weights g_t (all ones gives d(sum_t s_t)/dX)
 *   dX         [N x D] float32 out, overwritten (not accumulated) */
traknn_status traknn_score_backward(traknn_handle handle, const float* X, int64_t N, int64_t D,
                                    int L, int k, const int32_t* nbr_idx,
                                    const float* grad_score, float* dX, void* stream);

/* One series of a batched forward call: the arguments of traknn_knn_scores for
 * one sequence of daily fields (device pointers). */
typedef struct {
  const float* X;     /* [N x D] float32, row-major */
  int64_t N;          /* days */
  int L;              /* trajectory length */
  int k;              /* neighbours */
  int exclusion;      /* temporal exclusion e */
  int32_t* nbr_idx;   /* [M x k] out */
  float* nbr_dist;    /* [M x k] out */
  float* score;       /* [M] out */
} traknn_series;

/* Forward pass over B independent series that share the grid size D (each with
 * its own N, L, k and exclusion; the method of Sec. 3.2 applied to each series
 * separately, as when a study scores several regions, variables or ensemble
 * members). Every series' outputs equal those of traknn_knn_scores on it alone.
 * With a tensor-core precision up to 64 series run in one persistent launch
 * sequence, which is captured as a CUDA graph on first use and replayed on later
 * calls with the same shapes, pointers and options (the handle keeps one graph
 * per such signature, the 16 most recent; a change of shape or a larger workspace
 * drops them; evicting the oldest synchronises `stream` once).
 * With TRAKNN_PREC_FP32 the series run one after another. Each series is
 * checked as traknn_check_problem would check it; the first failing series'
 * status is returned before anything is enqueued. */
traknn_status traknn_knn_scores_batched(traknn_handle handle, const traknn_series* series, int B,
                                        int64_t D, void* stream);

/* Several (L, k, exclusion) settings of ONE record in one Gram sweep (Sec. 6: the
 * "what-if" analyses over trajectory lengths). All nset entries must share X and N
 * (the same device pointer and day count; D as given) and differ in L, k, exclusion
 * and their output buffers (layouts as in traknn_knn_scores). With a tensor-core
 * precision the Gram tiles are computed once (strip height and tile step sized for
 * the largest L) and every tile is scanned once per setting, so the cost is close to
 * that of one setting when the contraction dominates (large D). Each setting's
 * outputs equal those of traknn_knn_scores on it alone except that, as in that call,
 * D(t,j) may be evaluated from either operand order: distances agree to a few ulp
 * and neighbour sets may differ only at near ties. With TRAKNN_PREC_FP32 the settings
 * run one after another. 1 <= nset <= 64; each entry is checked as
 * traknn_check_problem would check it; entries with another X or N are refused
 * (TRAKNN_ERR_INVALID_ARG). */
traknn_status traknn_knn_scores_multi(traknn_handle handle, const traknn_series* settings,
                                      int nset, int64_t D, void* stream);

/* ---- One series split across processes (one GPU each) ------------------------
 * The unordered trajectory pairs of a series are independent (the upper-triangle
 * Gram tiles of Sec. 3.3, "Symmetric Batched GeMM"), so P processes can share one
 * series: each evaluates the pairs of its part (traknn_knn_partial), the per-row
 * candidate lists are exchanged once (for example an all-gather over the processes),
 * and every process merges them (traknn_merge_partials) into the exact result of
 * traknn_knn_scores on the whole series, up to distances evaluated in the other
 * operand order (a few ulp; neighbour sets may then differ at near ties). */

/* Host-only: the trajectory rows [*row_lo, *row_hi) whose pairs part `part` of
 * `nparts` evaluates. Rows are cut into strips of 128 - (L-1) rows; each part gets a
 * contiguous range of strips carrying about 1/nparts of the M(M+1)/2 unordered
 * pairs (strip s holds the pairs {a, b} with min(a, b) in the strip, b >= a). A part
 * may be empty (*row_lo == *row_hi) when nparts exceeds the number of strips.
 * 1 <= L <= TRAKNN_MAX_L, 1 <= nparts <= TRAKNN_MAX_PARTS, 0 <= part < nparts. */
traknn_status traknn_partition(int64_t M, int L, int nparts, int part, int64_t* row_lo,
                               int64_t* row_hi);

/* The candidate lists of one part of a split series (tensor-core precisions with the
 * symmetric evaluation; TRAKNN_ERR_UNSUPPORTED with TRAKNN_PREC_FP32 or
 * TRAKNN_OPT_SYMMETRIC = 0). Arguments as traknn_knn_scores plus the part:
 *   part_idx  [M x k] int32 out (device): for every trajectory row t, candidates j of t
 *             whose pair {t, j} this part evaluates, sorted by (distance, index), at
 *             least every one of t's k nearest neighbours among them; entries beyond
 *             the row's candidates hold index -1 and distance +inf
 *   part_dist [M x k] float32 out (device): their distances D(t, j)
 * Rows outside the part's strips receive candidates only from pairs whose smaller
 * index lies in the part (possibly none). */
traknn_status traknn_knn_partial(traknn_handle handle, const float* X, int64_t N, int64_t D,
                                 int L, int k, int exclusion, int part, int nparts,
                                 int32_t* part_idx, float* part_dist, void* stream);

/* Merge the parts' candidate lists (Algorithm 1, kNN step over the union) into the
 * neighbour sets and rarity scores of Eq. 3:
 *   idx_parts  [nparts x M x k] int32 (device), part-major: the part_idx of every part
 *   dist_parts [nparts x M x k] float32 (device): the matching part_dist
 *   nbr_idx, nbr_dist [M x k], score [M] out (device), as traknn_knn_scores returns them
 * Each row takes the k smallest (distance, index) entries of the union of its lists;
 * the score is their FP64 mean. 1 <= nparts <= TRAKNN_MAX_PARTS. */
traknn_status traknn_merge_partials(traknn_handle handle, const int32_t* idx_parts,
                                    const float* dist_parts, int nparts, int64_t M, int k,
                                    int32_t* nbr_idx, float* nbr_dist, float* score,
                                    void* stream);

/* Grid-point weights: with weights w (D values >= 0, DEVICE pointer, caller-owned,
 * read by every later call on this handle until cleared) the snapshot distance of
 * Eq. 2 becomes sum_p w_p (X[a,p] - X[b,p])^2 in every forward path of the handle
 * (tensor-core and FP32) and in traknn_score_backward (dX carries the factor w_p).
 * Area weights proportional to the cosine of latitude (Sec. 5, composite analysis)
 * are the intended use. weights = NULL clears them. Calls whose D differs from
 * the D given here return TRAKNN_ERR_INVALID_ARG. traknn_knn_scores_static ignores
 * weights (it has no handle). */
traknn_status traknn_set_grid_weights(traknn_handle handle, const float* weights, int64_t D);

/* Statistics of sorted neighbour distance lists (DEVICE pointers, asynchronous):
 *   nbr_dist      [M x k] float32, each row ascending (as traknn_knn_scores returns it)
 *   prefix_scores [M x k] float32 out, or NULL: prefix_scores[t][k'-1] = the rarity
 *                 score of Eq. 3 with k' neighbours, for every k' = 1..k (the neighbour
 *                 set for k' is the first k' of the list for k: Sec. 6 notes that the
 *                 top-k results of a larger k contain those of every smaller k);
 *                 summed in FP64
 *   local_id      [M] float32 out, or NULL: the local intrinsic dimension of every
 *                 trajectory by the maximum-likelihood kNN estimator of Levina and
 *                 Bickel with k_id neighbours (2 <= k_id <= k), as in the intrinsic
 *                 dimension study of Sec. 4: [ (1/(k_id-1)) sum_{j<k_id} log(T_k_id/T_j) ]^-1
 *                 with T_j = sqrt(nbr_dist[t][j-1]); NaN when one of the first k_id
 *                 distances is zero or all of them are equal
 * At least one output must be given. */
traknn_status traknn_knn_stats(traknn_handle handle, const float* nbr_dist, int64_t M, int k,
                               float* prefix_scores, int k_id, float* local_id, void* stream);

/* Forward pass for callers that cannot allocate device memory. There is no
 * counterpart in the paper: this is an interface addition of this library.
 *
 * Who needs it: code whose device memory belongs to another allocator or is held
 * to a fixed budget, and code that must not cause the device-wide
 * synchronisation a cudaMalloc or cudaFree can trigger. traknn_knn_scores needs
 * a handle whose workspace grows by cudaMalloc; this call needs no handle and
 * allocates nothing (no cudaMalloc, cudaFree or allocating library routine).
 *
 * Its scratch is one fixed 32 MiB array of device memory inside the library,
 * which every GPU that loads the library holds until the process exits. A
 * problem needs exactly
 *     a(256*D) + a(4*D) + a(8*N) + a(4*M) + a(4*N*Dp) + 2*a(4*M*C*k) + 256  bytes,
 * with a(x) = x rounded up to a multiple of 256, Dp = D rounded up to a multiple
 * of 32, and C the number of column chunks: c = min(8, M), C = ceil(M / ceil(M / c)).
 * Larger problems return TRAKNN_ERR_SCRATCH_LIMIT before any work is enqueued.
 * It runs the FP32 CUDA-core path on the current device. Arguments, layouts and
 * outputs are those of traknn_knn_scores (X, nbr_idx, nbr_dist and score are
 * device pointers; `stream` is a cudaStream_t).
 *
 * The array's device address is looked up on the first call on a device and
 * cached for that device's current CUDA context; the lookup can also load the
 * library's device code, so make the first call before any stream capture. If
 * the context is destroyed (cudaDeviceReset) and a new one created, the next call
 * looks the address up again (the array may have moved). Every call reuses the
 * same array and leaves its contents behind; nothing in it needs to be cleared by
 * the caller (the call clears its own status word). Calls that overlap on the GPU
 * (for example on two streams without an ordering between them) race on the array
 * and corrupt each other's results: serialise them. */
traknn_status traknn_knn_scores_static(const float* X, int64_t N, int64_t D, int L, int k,
                                       int exclusion, int32_t* nbr_idx, float* nbr_dist,
                                       float* score, void* stream);

/* Synchronise `stream` and return the first device-side failure recorded since
 * the last call to this function (TRAKNN_ERR_TIMEOUT), or TRAKNN_OK. */
traknn_status traknn_sync_status(traknn_handle handle, void* stream);

/* Durations in ms of the fused Gram/top-k kernel of the forward calls made
 * since the last read while TRAKNN_OPT_PROFILE was on (oldest first, at most
 * max_n; at most 256 are kept). Synchronises the handle's device.
 * *n_out receives the number written. */
traknn_status traknn_profile_read(traknn_handle handle, float* ms, int max_n, int* n_out);

/* Event counters of the tensor-core kernel accumulated while TRAKNN_OPT_STATS was on
 * (diagnostics): [0] row-side list insertions, [1] column-side candidates,
 * [2] column lists with more than k candidates (the column's own thread keeps the
 * k best), [3] non-empty column lists,
 * [4] 32-column chunks processed, [5] MMA-thread cycles waiting for a free
 * accumulator, [6] MMA-thread cycles waiting for operands, [7] MMA-thread cycles
 * in total; cycles of the first epilogue thread [8] waiting for a filled
 * accumulator, [9] loading a tile's window sums and column bounds, [10] reading
 * out and staging chunks, [11] in the barrier after staging, [12] in the row-side
 * scan up to the barrier after it, [13] in the column side, [14] in total (all
 * summed over CTAs). Synchronises the device and resets them. */
traknn_status traknn_stats_read(traknn_handle handle, uint64_t* counters, int n);

/* Work-unit shape of the handle's last tensor-core forward call (the autotuner's
 * choice when TRAKNN_OPT_AUTOTUNE is on): Gram tiles per work unit and row strips
 * whose units run side by side. Both 0 before the first such call. */
traknn_status traknn_work_shape(traknn_handle handle, int* tiles_per_unit, int* group_strips);

/* Total number of kernels this handle has launched (all entry points). */
traknn_status traknn_launch_count(traknn_handle handle, int64_t* count);

/* Static description of a status code. */
const char* traknn_status_string(traknn_status status);

#ifdef __cplusplus
}
#endif

#endif /* TRAKNN_H */
