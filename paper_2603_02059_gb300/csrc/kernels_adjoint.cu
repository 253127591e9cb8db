// kernels_adjoint.cu -- gradient of the weighted summed rarity score with respect to
// every grid-point value, the neighbour sets held fixed. From Eq. 2-3:
//   F(X) = sum_t g_t s_t = sum_t (g_t/k) sum_{j in N_t} sum_{m<L} ||X_{t+m} - X_{j+m}||^2
//   dF/dX_a = sum over incidences (t, j, m) with t+m = a or j+m = a of
//             w_t (X_a - X_b),   w_t = 2 g_t / k,   b the other day of the pair.
// The incidences of day a are
//   forward:  t in [a-L+1, a], j in N_t,             b = j + (a - t)
//   reverse:  j in [a-L+1, a], t with j in N_t,       b = t + (a - j)
// With grid-point weights w_p (distance sum_p w_p (x_p - y_p)^2) every term carries
// the factor w_p, applied once to the finished sum.
//
// Neighbouring trajectories have neighbouring neighbours (j in N_t makes j+1 in
// N_{t+1} likely), so the incidences of a run of consecutive days share many partner
// rows. The gradient is therefore taken per block of kAdjR consecutive days:
//   build:  the block's incidences are listed in shared memory as keys (partner b,
//           day in block, kind, window slot), sorted, and every run with the same
//           (b, day) is merged into one entry (b, day, summed weight);
//   gather: one CTA per (day block, 256 grid points) applies the block's entries in
//           list order, so that every partner row segment is read once per block,
//           and all CTAs of one 256-point tile run first (that tile of X, 1 KB per
//           day, stays in L2 while it is re-read).
// No floating-point atomics are used: every sum is taken in a fixed order (sorted
// keys, then list order), so the result is bitwise reproducible. A single day with
// more incidences than the sort buffer lists them unmerged in a fixed order (its
// forward incidences by (t, rank), then its reverse ones by (j, t), from reverse
// lists sorted by t).
#include <cuda_runtime.h>

#include "internal.h"

namespace traknn {
namespace {

__global__ void adj_count_kernel(const int32_t* __restrict__ idx, int M, int k, int* count,
                                 int* err) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (long long)M * k) return;
  const int j = idx[q];
  if (j < 0 || j >= M) {
    atomicCAS(err, 0, kErrInvalidArg);
    return;
  }
  atomicAdd(count + j, 1);
}

// Exclusive scan of count[0..M) into off[0..M]; one block of 1024 threads.
__global__ void adj_scan_kernel(const int* __restrict__ count, int M, int* off) {
  __shared__ int part[1024];
  const int tid = threadIdx.x;
  const int per = (M + 1023) / 1024;
  const int lo = min(M, tid * per), hi = min(M, lo + per);
  int s = 0;
  for (int i = lo; i < hi; ++i) s += count[i];
  part[tid] = s;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const int v = tid >= o ? part[tid - o] : 0;
    __syncthreads();
    part[tid] += v;
    __syncthreads();
  }
  int run = tid > 0 ? part[tid - 1] : 0;
  for (int i = lo; i < hi; ++i) {
    off[i] = run;
    run += count[i];
  }
  if (tid == 1023) off[M] = part[1023];
}

__global__ void adj_fill_kernel(const int32_t* __restrict__ idx, int M, int k,
                                const int* __restrict__ off, int* cursor, int* rev) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (long long)M * k) return;
  const int j = idx[q];
  if (j < 0 || j >= M) return;
  const int t = (int)(q / k);
  const int pos = atomicAdd(cursor + j, 1);
  rev[off[j] + pos] = t;
}

__device__ void sift_down(int* a, int root, int n) {
  for (;;) {
    int c = 2 * root + 1;
    if (c >= n) return;
    if (c + 1 < n && a[c + 1] > a[c]) ++c;
    if (a[root] >= a[c]) return;
    const int tmp = a[root];
    a[root] = a[c];
    a[c] = tmp;
    root = c;
  }
}

constexpr int kAdjR = 16;         // output days per block
constexpr int kKeyCap = 4096;     // incidences sorted at once in shared memory
constexpr int kBuildThreads = 256;
constexpr int kGatherThreads = 256;

// One merged entry of a block's gradient list: partner day b and summed weight w
// (as FP32 bits). A block's entries are in order of output day (blk_day gives each
// day's first entry), then partner.
typedef int2 AdjEntry;

// Incidences of day a: the forward ones (k per trajectory t of its window) and the
// reverse segments of the days j of its window, [max(0, a-L+1), min(a, M-1)].
__device__ __forceinline__ int day_incidences(const int* off, int a, int L, int M, int k) {
  const int t_lo = max(0, a - L + 1), t_hi = min(a, M - 1);
  if (t_hi < t_lo) return 0;
  return (t_hi - t_lo + 1) * k + (off[t_hi + 1] - off[t_lo]);
}

// Sort ascending (heap sort, in place) every reverse segment read by a day with more
// incidences than the sort buffer holds; that day lists its incidences unmerged, in
// an order that must not depend on the order the fill kernel produced. Other days
// order their incidences by key in the build kernel and need no sorted segments.
__global__ void adj_sort_kernel(const int* __restrict__ off, int N, int L, int M, int k,
                                int* rev) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= M) return;
  bool needed = false;
  for (int d = j; d < min(N, j + L); ++d) needed |= day_incidences(off, d, L, M, k) > kKeyCap;
  if (!needed) return;
  int* a = rev + off[j];
  const int n = off[j + 1] - off[j];
  for (int r = n / 2 - 1; r >= 0; --r) sift_down(a, r, n);
  for (int end = n - 1; end > 0; --end) {
    const int tmp = a[0];
    a[0] = a[end];
    a[end] = tmp;
    sift_down(a, 0, end);
  }
}

// Exclusive scan of the blocks' incidence totals (upper bounds of their entry counts)
// into blk_off[0..nblk]; one block of 1024 threads.
__global__ void adj_block_scan_kernel(const int* __restrict__ off, int N, int L, int M, int k,
                                      int nblk, long long* blk_off) {
  __shared__ long long part[1024];
  const int tid = threadIdx.x;
  const int per = (nblk + 1023) / 1024;
  const int lo = min(nblk, tid * per), hi = min(nblk, lo + per);
  auto total = [&](int blk) {
    long long s = 0;
    for (int a = blk * kAdjR; a < min(N, (blk + 1) * kAdjR); ++a)
      s += day_incidences(off, a, L, M, k);
    return s;
  };
  long long s = 0;
  for (int i = lo; i < hi; ++i) s += total(i);
  part[tid] = s;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const long long v = tid >= o ? part[tid - o] : 0;
    __syncthreads();
    part[tid] += v;
    __syncthreads();
  }
  long long run = tid > 0 ? part[tid - 1] : 0;
  for (int i = lo; i < hi; ++i) {
    blk_off[i] = run;
    run += total(i);
  }
  if (tid == 1023) blk_off[nblk] = part[1023];
}

// The merged entry list of one block of kAdjR days (one CTA per block). The days are
// cut into segments of consecutive days whose incidences fit the key buffer. A
// segment's keys are (day d << 58) | (partner b << 24) | (kind << 23) | slot: kind 0
// is a forward incidence (trajectory t = t_lo + slot of day a0 + d), kind 1 a reverse
// one (window day j = t_lo + slot, trajectory t = b - a + j). Every key is unique, so
// the sorted order is fixed whatever order the reverse lists were filled in; each run
// of equal (d, b) becomes one entry whose weight is summed in key order. blk_day
// receives the first entry of every day (kAdjR + 1 offsets per block).
__global__ void __launch_bounds__(kBuildThreads)
    adj_build_kernel(const int32_t* __restrict__ idx, const float* __restrict__ g, int N, int L,
                     int M, int k, const int* __restrict__ off, const int* __restrict__ rev,
                     const long long* __restrict__ blk_off, int* __restrict__ blk_day,
                     AdjEntry* __restrict__ ent, int* err) {
  __shared__ unsigned long long key[kKeyCap];
  __shared__ int dayoff[kAdjR + 1];  // first position of each day in the block
  __shared__ int daycnt[kAdjR];      // entries written for each day
  __shared__ int soff[kAdjR + kMaxL + 1];  // off[j] for the window days j of the block
  __shared__ int scan[kBuildThreads];
  const int tid = threadIdx.x;
  const int a0 = blockIdx.x * kAdjR;
  const int nd = min(kAdjR, N - a0);
  const float inv_k2 = 2.0f / (float)k;
  // window days of the block's days: [jb, je]; their reverse-list offsets off[jb..je+1]
  const int jb = max(0, a0 - L + 1), je = min(a0 + nd - 1, M - 1);
  for (int i = tid; i <= je - jb + 1; i += kBuildThreads) soff[i] = off[jb + i];
  if (tid < kAdjR) daycnt[tid] = 0;
  __syncthreads();
  auto offj = [&](int j) { return soff[j - jb]; };  // off[j], jb <= j <= je + 1
  if (tid == 0) {
    int pos = 0;
    for (int d = 0; d < nd; ++d) {
      dayoff[d] = pos;
      const int a = a0 + d;
      const int t_lo = max(0, a - L + 1), t_hi = min(a, M - 1);
      if (t_hi >= t_lo) pos += (t_hi - t_lo + 1) * k + (offj(t_hi + 1) - offj(t_lo));
    }
    dayoff[nd] = pos;
  }
  __syncthreads();
  AdjEntry* out = ent + blk_off[blockIdx.x];
  const long long cap = blk_off[blockIdx.x + 1] - blk_off[blockIdx.x];  // entries of the block
  int nout = 0;
  // incidence q (0 <= q < day_incidences) of day a: its partner and trajectory
  auto incidence = [&](int a, int q, int& b, int& t, int& kind, int& slot) -> bool {
    const int t_lo = max(0, a - L + 1), t_hi = min(a, M - 1);
    const int nfwd = (t_hi - t_lo + 1) * k;
    if (q < nfwd) {
      slot = q / k;
      t = t_lo + slot;
      kind = 0;
      const int j = idx[(size_t)t * k + q % k];
      b = j + a - t;
      return j >= 0 && j < M;
    }
    const int r = offj(t_lo) + (q - nfwd);  // reverse lists of t_lo..t_hi are contiguous
    int j = t_lo;
    while (offj(j + 1) <= r) ++j;
    t = rev[r];
    kind = 1;
    slot = j - t_lo;
    b = t + a - j;
    return true;
  };
  int d = 0;
  while (d < nd) {
    int dh = d + 1;
    while (dh < nd && dayoff[dh + 1] - dayoff[d] <= kKeyCap) ++dh;
    const int base = dayoff[d];
    const int n = dayoff[dh] - base;
    if (n > kKeyCap) {
      // one day with more incidences than the buffer: unmerged, in the fixed order of
      // its lists (forward by (t, rank), reverse by (j, t) from sorted segments)
      const int a = a0 + d;
      for (int q = tid; q < n; q += kBuildThreads) {
        int b, t, kind, slot;
        const bool ok = incidence(a, q, b, t, kind, slot);
        if (tk_in(nout + q, cap, err))
          out[nout + q] = ok ? make_int2(b, __float_as_int(inv_k2 * g[t])) : make_int2(a, 0);
      }
      if (tid == 0) daycnt[d] = n;
      nout += n;
      d = dh;
      continue;
    }
    int n2 = 1;
    while (n2 < n) n2 <<= 1;
    for (int q = tid; q < n2; q += kBuildThreads) {
      unsigned long long kq = ~0ull;  // padding and invalid incidences sort last
      if (q < n) {
        int dd = d;
        while (dayoff[dd + 1] <= base + q) ++dd;
        int b, t, kind, slot;
        if (incidence(a0 + dd, base + q - dayoff[dd], b, t, kind, slot))
          kq = ((unsigned long long)dd << 58) | ((unsigned long long)(unsigned)b << 24) |
               ((unsigned long long)kind << 23) | (unsigned long long)slot;
      }
      key[q] = kq;
    }
    __syncthreads();
    for (int size = 2; size <= n2; size <<= 1) {
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        for (int q = tid; q < n2; q += kBuildThreads) {
          const int r = q ^ stride;
          if (r > q) {
            const bool up = (q & size) == 0;
            const unsigned long long x = key[q], y = key[r];
            if ((x > y) == up) {
              key[q] = y;
              key[r] = x;
            }
          }
        }
        __syncthreads();
      }
    }
    // run heads (first position of each distinct (b, day)), numbered by an exclusive
    // prefix sum over each thread's consecutive positions
    const int per = (n + kBuildThreads - 1) / kBuildThreads;
    auto head = [&](int q) {
      if (q >= n || key[q] == ~0ull) return 0;
      return (q == 0 || (key[q - 1] >> 24) != (key[q] >> 24)) ? 1 : 0;
    };
    const int q0 = tid * per;
    int cnt = 0;
    for (int i = 0; i < per; ++i) cnt += head(q0 + i);
    scan[tid] = cnt;
    __syncthreads();
    for (int o = 1; o < kBuildThreads; o <<= 1) {
      const int v = tid >= o ? scan[tid - o] : 0;
      __syncthreads();
      scan[tid] += v;
      __syncthreads();
    }
    int u = nout + scan[tid] - cnt;
    for (int i = 0; i < per; ++i) {
      const int q = q0 + i;
      if (!head(q)) continue;
      const unsigned long long run = key[q] >> 24;
      const int b = (int)((key[q] >> 24) & 0x3FFFFFFFull);
      const int dd = (int)(key[q] >> 58);
      const int a = a0 + dd;
      const int t_lo = max(0, a - L + 1);
      float w = 0.f;
      for (int r = q; r < n && key[r] != ~0ull && (key[r] >> 24) == run; ++r) {
        const int kind = (int)((key[r] >> 23) & 1);
        const int slot = (int)(key[r] & 0x7F);
        const int t = kind ? b - a + t_lo + slot : t_lo + slot;
        w += inv_k2 * g[t];
      }
      if (tk_in(u, cap, err)) out[u] = make_int2(b, __float_as_int(w));
      ++u;
      atomicAdd(&daycnt[dd], 1);
    }
    nout += scan[kBuildThreads - 1];
    __syncthreads();  // the key buffer is refilled by the next segment
    d = dh;
  }
  __syncthreads();
  if (tid == 0) {
    int pos = 0;
    for (int dd = 0; dd < kAdjR; ++dd) {
      blk_day[blockIdx.x * (kAdjR + 1) + dd] = pos;
      pos += dd < nd ? daycnt[dd] : 0;
    }
    blk_day[blockIdx.x * (kAdjR + 1) + kAdjR] = pos;
  }
}

// Values of V adjacent grid points (V = 2: one 8-byte load; rows are 8-byte aligned
// when D is even) and the update acc += w (xa - xb) on them, with V = 2 as two packed
// FP32 operations (xa - xb exactly as xb * -1 + xa, then one fused multiply-add).
template <int V> struct Vec;
template <> struct Vec<1> {
  typedef float T;
  static __device__ __forceinline__ T load(const float* p) { return __ldg(p); }
  static __device__ __forceinline__ T zero() { return 0.f; }
  static __device__ __forceinline__ void update(T& acc, float w, T xa, T xb) {
    acc = fmaf(w, xa - xb, acc);
  }
  static __device__ __forceinline__ float get(T v, int) { return v; }
};
template <> struct Vec<2> {
  typedef float2 T;
  static __device__ __forceinline__ T load(const float* p) {
    return __ldg(reinterpret_cast<const float2*>(p));
  }
  static __device__ __forceinline__ T zero() { return make_float2(0.f, 0.f); }
  static __device__ __forceinline__ void update(T& acc, float w, T xa, T xb) {
    const float2 d = __ffma2_rn(xb, make_float2(-1.f, -1.f), xa);
    acc = __ffma2_rn(make_float2(w, w), d, acc);
  }
  static __device__ __forceinline__ float get(T v, int i) { return i ? v.y : v.x; }
};

// dX for one block of kAdjR days and kGatherThreads * V grid points: for each day
// a0 + d, every entry (b, w) of the day adds w (X[a0+d] - X[b]), in list order. Each
// thread owns V adjacent grid points and keeps the block's values of X and sums for
// them in registers; one entry (read from shared memory, the same for every thread)
// serves all of them. Partner values are loaded kU entries at a time (kU loads per
// thread in flight). blockIdx.x is the day block and blockIdx.y the grid-point tile:
// CTAs are scheduled with x fastest, so the CTAs running at one time share a tile of
// X, which stays in L2 while the entries re-read its rows (consecutive days of a
// block share many partner rows, which then also come from L1).
constexpr int kU = 16;
constexpr int kStage = 2048;
template <int V>
__global__ void __launch_bounds__(kGatherThreads, 2)
    adj_gather_kernel(const float* __restrict__ X, int N, int D,
                      const long long* __restrict__ blk_off, const int* __restrict__ blk_day,
                      const AdjEntry* __restrict__ ent, const float* __restrict__ wts,
                      float* __restrict__ dX, int* err) {
  typedef Vec<V> Op;
  typedef typename Op::T T;
  constexpr int kCols = kGatherThreads * V;
  __shared__ AdjEntry se[kStage];
  __shared__ int sday[kAdjR + 1];
  const int tid = threadIdx.x;
  const int a0 = blockIdx.x * kAdjR;
  const int nd = min(kAdjR, N - a0);
  const AdjEntry* e2 = ent + blk_off[blockIdx.x];
  if (tid <= kAdjR) sday[tid] = blk_day[blockIdx.x * (kAdjR + 1) + tid];
  __syncthreads();
  const int ntot = sday[kAdjR];
  const int tiles = (D + kCols - 1) / kCols;
  for (int tile = blockIdx.y; tile < tiles; tile += gridDim.y) {
    const int p = tile * kCols + V * tid;  // first of the thread's V grid points
    const bool pin = p < D;                // (D is a multiple of V)
    const float* xp = X + (pin ? p : 0);
    T xa[kAdjR], acc[kAdjR];
#pragma unroll
    for (int d = 0; d < kAdjR; ++d) {
      xa[d] = (pin && d < nd) ? Op::load(xp + (size_t)(a0 + d) * D) : Op::zero();
      acc[d] = Op::zero();
    }
    for (int c0 = 0; c0 < ntot; c0 += kStage) {
      const int c1 = min(ntot, c0 + kStage);
      __syncthreads();  // the previous pass has read its entries
      for (int i = tid; i < c1 - c0; i += kGatherThreads) {
        AdjEntry e = __ldg(e2 + c0 + i);
        if (!tk_in(e.x, N, err)) e = make_int2(a0, 0);  // debug build: adds 0
        se[i] = e;
      }
      __syncthreads();
#pragma unroll
      for (int d = 0; d < kAdjR; ++d) {
        const int q1 = min(sday[d + 1], c1);
        int q = max(sday[d], c0);
        // whole groups of kU entries, then the remainder with predicated loads
        for (; q + kU <= q1; q += kU) {
          T xb[kU];
#pragma unroll
          for (int u = 0; u < kU; ++u)
            xb[u] = pin ? Op::load(xp + (size_t)se[q + u - c0].x * D) : Op::zero();
#pragma unroll
          for (int u = 0; u < kU; ++u)
            Op::update(acc[d], __int_as_float(se[q + u - c0].y), xa[d], xb[u]);
        }
        if (q < q1) {
          T xb[kU];
#pragma unroll
          for (int u = 0; u < kU; ++u)
            xb[u] = (pin && q + u < q1) ? Op::load(xp + (size_t)se[q + u - c0].x * D)
                                        : Op::zero();
#pragma unroll
          for (int u = 0; u < kU; ++u)
            if (q + u < q1) Op::update(acc[d], __int_as_float(se[q + u - c0].y), xa[d], xb[u]);
        }
      }
    }
    if (pin) {
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const float wp = wts ? wts[p + v] : 1.f;
#pragma unroll
        for (int d = 0; d < kAdjR; ++d)
          if (d < nd) dX[(size_t)(a0 + d) * D + p + v] = wts ? Op::get(acc[d], v) * wp
                                                             : Op::get(acc[d], v);
      }
    }
  }
}

}  // namespace

namespace {

inline size_t up256(size_t v) { return (v + 255) / 256 * 256; }

// Workspace layout: merged entries (at most one per incidence, 2 L k M in all), block
// offsets and counts, then the reverse neighbour index (count, cursor, off, rev).
struct AdjLayout {
  size_t ent, blk_off, blk_day, count, total;
};

AdjLayout adj_layout(int N, int L, int k) {
  const size_t M = (size_t)(N - L + 1);
  const size_t nblk = ((size_t)N + kAdjR - 1) / kAdjR;
  AdjLayout l;
  l.ent = 0;
  l.blk_off = up256(2 * (size_t)L * k * M * sizeof(AdjEntry));
  l.blk_day = l.blk_off + up256((nblk + 1) * sizeof(long long));
  l.count = l.blk_day + up256(nblk * (kAdjR + 1) * sizeof(int));
  l.total = l.count + up256((3 * M + 1 + M * (size_t)k) * sizeof(int));
  return l;
}

}  // namespace

size_t adjoint_workspace_bytes(int N, int L, int k) { return adj_layout(N, L, k).total; }

cudaError_t launch_adjoint(const float* X, int N, int D, int L, int k, const int32_t* idx,
                           const float* g, const float* wts, float* dX, void* ws, int* err,
                           cudaStream_t st, int* launches) {
  const int M = N - L + 1;
  const AdjLayout lay = adj_layout(N, L, k);
  char* base = static_cast<char*>(ws);
  AdjEntry* ent = reinterpret_cast<AdjEntry*>(base + lay.ent);
  long long* blk_off = reinterpret_cast<long long*>(base + lay.blk_off);
  int* blk_day = reinterpret_cast<int*>(base + lay.blk_day);
  int* count = reinterpret_cast<int*>(base + lay.count);
  int* cursor = count + M;
  int* off = cursor + M;
  int* rev = off + M + 1;
  const int nblk = (N + kAdjR - 1) / kAdjR;
  cudaError_t e = cudaMemsetAsync(count, 0, (size_t)2 * M * sizeof(int), st);
  if (e != cudaSuccess) return e;
  const long long nq = (long long)M * k;
  const int blocks = (int)((nq + 255) / 256);
  adj_count_kernel<<<blocks, 256, 0, st>>>(idx, M, k, count, err);
  adj_scan_kernel<<<1, 1024, 0, st>>>(count, M, off);
  adj_fill_kernel<<<blocks, 256, 0, st>>>(idx, M, k, off, cursor, rev);
  adj_sort_kernel<<<(M + 127) / 128, 128, 0, st>>>(off, N, L, M, k, rev);
  adj_block_scan_kernel<<<1, 1024, 0, st>>>(off, N, L, M, k, nblk, blk_off);
  adj_build_kernel<<<nblk, kBuildThreads, 0, st>>>(idx, g, N, L, M, k, off, rev, blk_off,
                                                    blk_day, ent, err);
  // two adjacent grid points per thread when rows are 8-byte aligned (D even)
  const int V = D % 2 == 0 ? 2 : 1;
  const int tiles = (D + kGatherThreads * V - 1) / (kGatherThreads * V);
  const dim3 grid(nblk, tiles < 65535 ? tiles : 65535);
  if (V == 2)
    adj_gather_kernel<2><<<grid, kGatherThreads, 0, st>>>(X, N, D, blk_off, blk_day, ent, wts,
                                                          dX, err);
  else
    adj_gather_kernel<1><<<grid, kGatherThreads, 0, st>>>(X, N, D, blk_off, blk_day, ent, wts,
                                                          dX, err);
  *launches += 7;
  return cudaGetLastError();
}

}  // namespace traknn
