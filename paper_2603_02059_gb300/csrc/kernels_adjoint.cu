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
// Every incidence of day a with the same partner b adds to one entry (b, summed
// weight), so the gradient is taken in two steps:
//   build:  one warp per day lists the day's incidences in shared memory as keys
//           (partner b, kind, window slot), sorts them, and merges every run with the
//           same b into one entry (b, summed weight); days with more incidences than
//           a warp's buffer are merged by the whole CTA afterwards;
//   gather: one CTA per (block of consecutive days, tile of grid points) walks its
//           days in order, applying each day's entries in list order with four
//           adjacent grid points per thread, and all CTAs of one tile run first
//           (that tile of X stays in L2 while the partner rows are re-read).
// No floating-point atomics are used: every sum is taken in a fixed order (sorted
// keys, then list order), so the result is bitwise reproducible. A single day with
// more incidences than the CTA's key buffer lists them unmerged in a fixed order (its
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

constexpr int kDayWarps = 8;     // days per CTA of the build kernel, one warp each
constexpr int kWarpKeys = 256;   // incidences one warp merges
constexpr int kBuildThreads = kDayWarps * 32;
constexpr int kKeyCap = 4096;    // incidences one CTA merges for one day (days beyond a warp)
constexpr int kBigThreads = 256;

// One merged entry of a day's gradient list: partner day b and summed weight w (as
// FP32 bits). A day's entries are in order of partner.
typedef int2 AdjEntry;

// Incidences of day a: the forward ones (k per trajectory t of its window) and the
// reverse segments of the days j of its window, [max(0, a-L+1), min(a, M-1)].
__device__ __forceinline__ int day_incidences(const int* off, int a, int L, int M, int k) {
  const int t_lo = max(0, a - L + 1), t_hi = min(a, M - 1);
  if (t_hi < t_lo) return 0;
  return (t_hi - t_lo + 1) * k + (off[t_hi + 1] - off[t_lo]);
}

// Sort ascending (heap sort, in place) every reverse segment read by a day with more
// incidences than the key buffer holds; that day lists its incidences unmerged, in an
// order that must not depend on the order the fill kernel produced. Other days order
// their incidences by key in the build kernel and need no sorted segments.
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

// Exclusive scan of the days' incidence counts (upper bounds of their merged entry
// counts) into inc_off[0..N]; one block of 1024 threads.
__global__ void adj_day_scan_kernel(const int* __restrict__ off, int N, int L, int M, int k,
                                    long long* inc_off) {
  __shared__ long long part[1024];
  const int tid = threadIdx.x;
  const int per = (N + 1023) / 1024;
  const int lo = min(N, tid * per), hi = min(N, lo + per);
  long long s = 0;
  for (int a = lo; a < hi; ++a) s += day_incidences(off, a, L, M, k);
  part[tid] = s;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const long long v = tid >= o ? part[tid - o] : 0;
    __syncthreads();
    part[tid] += v;
    __syncthreads();
  }
  long long run = tid > 0 ? part[tid - 1] : 0;
  for (int a = lo; a < hi; ++a) {
    inc_off[a] = run;
    run += day_incidences(off, a, L, M, k);
  }
  if (tid == 1023) inc_off[N] = part[1023];
}

// The window of day a: trajectories [t_lo, t_lo + nw) contain it; its forward
// incidences are the nw k neighbour entries idx[t_lo k ..) (trajectory t_lo + q / k,
// contiguous), its reverse ones the reverse lists of the window days, rev[r0 ..)
// (contiguous as well). Incidence q (0 <= q < n) is forward for q < nfwd.
struct DayWindow {
  int a, t_lo, nw, nfwd, r0;
};

__device__ __forceinline__ DayWindow day_window(const int* off, int a, int L, int M, int k) {
  DayWindow w;
  w.a = a;
  w.t_lo = max(0, a - L + 1);
  w.nw = max(0, min(a, M - 1) - w.t_lo + 1);
  w.nfwd = w.nw * k;
  w.r0 = off[w.t_lo];
  return w;
}

// Sort keys: (partner b << 24) | (kind << 23) | slot, kind 0 for a forward incidence
// (slot: trajectory t = t_lo + slot) and 1 for a reverse one (slot: window day j =
// t_lo + slot, t from j's reverse list). Every key of a day is unique, so the sorted
// order is fixed whatever order the reverse lists were filled in; invalid incidences
// (a neighbour index out of range, flagged by the count kernel) and padding are all
// ones and sort last.
__device__ __forceinline__ unsigned long long fwd_key(const DayWindow& w, int q, int j, int M,
                                                      int k) {
  if (j < 0 || j >= M) return ~0ull;
  const int slot = q / k;
  const int b = j + w.a - (w.t_lo + slot);
  return ((unsigned long long)(unsigned)b << 24) | (unsigned long long)slot;
}
__device__ __forceinline__ unsigned long long rev_key(const DayWindow& w, int slot, int t) {
  const int b = t + w.a - (w.t_lo + slot);
  return ((unsigned long long)(unsigned)b << 24) | (1ull << 23) | (unsigned long long)slot;
}
// Partner b and trajectory t of a (valid) key.
__device__ __forceinline__ void key_pair(const DayWindow& w, unsigned long long key, int& b,
                                         int& t) {
  b = (int)((key >> 24) & 0x3FFFFFFFull);
  const int slot = (int)(key & 0x7F);
  t = (key >> 23) & 1 ? b - w.a + w.t_lo + slot : w.t_lo + slot;
}

// Summed weight of the run of equal partners starting at sorted position q, in key
// order: w = sum over the run of (2 / k) g_t.
__device__ __forceinline__ float run_weight(const unsigned long long* key, int q, int n,
                                            const DayWindow& w, const float* g, float inv_k2) {
  const unsigned long long run = key[q] >> 24;
  float s = 0.f;
  for (int r = q; r < n && key[r] != ~0ull && (key[r] >> 24) == run; ++r) {
    int b, t;
    key_pair(w, key[r], b, t);
    s += inv_k2 * g[t];
  }
  return s;
}

// Merged entries of one day with n <= kWarpKeys incidences, by one warp: the keys from
// coalesced loads of the day's two contiguous lists (the window day of a reverse
// position found from the window's list offsets, one per lane, by shuffles), sorted
// by a bitonic network in the warp's part of shared memory, run heads numbered with a
// ballot per 32 positions.
__device__ void merge_day_warp(const DayWindow& w, int n, unsigned long long* key,
                               const int32_t* idx, const float* g, const int* off,
                               const int* rev, int M, int k, AdjEntry* out, long long cap,
                               int* cnt_a, int* err) {
  const int lane = threadIdx.x & 31;
  const float inv_k2 = 2.0f / (float)k;
  const int woff = lane <= w.nw ? off[w.t_lo + lane] : 0;  // off[t_lo + lane]
  int n2 = 32;
  while (n2 < n) n2 <<= 1;
  constexpr int kIt = kWarpKeys / 32;
  int v[kIt];  // neighbour j (forward) or trajectory t (reverse) of each own position
#pragma unroll
  for (int it = 0; it < kIt; ++it) {
    const int q = it * 32 + lane;
    v[it] = 0;
    if (q < n)
      v[it] = q < w.nfwd ? __ldg(idx + (size_t)w.t_lo * k + q) : __ldg(rev + w.r0 + (q - w.nfwd));
  }
#pragma unroll
  for (int it = 0; it < kIt; ++it) {
    const int q = it * 32 + lane;
    // window slot of a reverse position: the number of later window days whose lists
    // start at or before it
    int slot = 0;
    if (__any_sync(0xffffffffu, q >= w.nfwd && q < n)) {
      const int r = w.r0 + (q - w.nfwd);
      for (int i = 1; i < w.nw; ++i) slot += __shfl_sync(0xffffffffu, woff, i) <= r;
    }
    unsigned long long kq = ~0ull;
    if (q < n) kq = q < w.nfwd ? fwd_key(w, q, v[it], M, k) : rev_key(w, slot, v[it]);
    if (q < n2) key[q] = kq;
  }
  __syncwarp();
  for (int size = 2; size <= n2; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int q = lane; q < n2; q += 32) {
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
      __syncwarp();
    }
  }
  int nout = 0;
  for (int q0 = 0; q0 < n; q0 += 32) {
    const int q = q0 + lane;
    const bool head =
        q < n && key[q] != ~0ull && (q == 0 || (key[q - 1] >> 24) != (key[q] >> 24));
    const unsigned bal = __ballot_sync(0xffffffffu, head);
    if (head) {
      const int u = nout + __popc(bal & ((1u << lane) - 1u));
      const int b = (int)((key[q] >> 24) & 0x3FFFFFFFull);
      const float s = run_weight(key, q, n, w, g, inv_k2);
      if (tk_in(u, cap, err)) out[u] = make_int2(b, __float_as_int(s));
    }
    nout += __popc(bal);
  }
  if (lane == 0) *cnt_a = nout;
}

// Merged entries of one day with more than kWarpKeys incidences, by the whole CTA (a
// bitonic sort of up to kKeyCap keys; run heads numbered by an exclusive prefix sum
// over each thread's consecutive positions). A day with more than kKeyCap incidences
// lists them unmerged, in the fixed order of its lists (forward by (t, rank), reverse
// by (j, t) from sorted segments). Ends with a CTA barrier.
__device__ void merge_day_block(const DayWindow& w, int n, unsigned long long* key, int* scan,
                                int* swoff, const int32_t* idx, const float* g, const int* off,
                                const int* rev, int M, int k, AdjEntry* out, long long cap,
                                int* cnt_a, int* err) {
  const int tid = threadIdx.x;
  const float inv_k2 = 2.0f / (float)k;
  for (int i = tid; i <= w.nw; i += kBigThreads) swoff[i] = off[w.t_lo + i];
  __syncthreads();
  auto key_of = [&](int q) -> unsigned long long {
    if (q < w.nfwd) return fwd_key(w, q, __ldg(idx + (size_t)w.t_lo * k + q), M, k);
    const int r = w.r0 + (q - w.nfwd);
    int slot = 0;
    while (slot + 1 < w.nw && swoff[slot + 1] <= r) ++slot;
    return rev_key(w, slot, __ldg(rev + r));
  };
  if (n > kKeyCap) {
    for (int q = tid; q < n; q += kBigThreads) {
      const unsigned long long kq = key_of(q);
      int b = w.a, t = 0;
      if (kq != ~0ull) key_pair(w, kq, b, t);
      if (tk_in(q, cap, err))
        out[q] = kq != ~0ull ? make_int2(b, __float_as_int(inv_k2 * g[t])) : make_int2(w.a, 0);
    }
    if (tid == 0) *cnt_a = n;
    __syncthreads();
    return;
  }
  int n2 = 1;
  while (n2 < n) n2 <<= 1;
  for (int q = tid; q < n2; q += kBigThreads) key[q] = q < n ? key_of(q) : ~0ull;
  __syncthreads();
  for (int size = 2; size <= n2; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int q = tid; q < n2; q += kBigThreads) {
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
  const int per = (n + kBigThreads - 1) / kBigThreads;
  auto head = [&](int q) {
    if (q >= n || key[q] == ~0ull) return 0;
    return (q == 0 || (key[q - 1] >> 24) != (key[q] >> 24)) ? 1 : 0;
  };
  const int q0 = tid * per;
  int cnt = 0;
  for (int i = 0; i < per; ++i) cnt += head(q0 + i);
  scan[tid] = cnt;
  __syncthreads();
  for (int o = 1; o < kBigThreads; o <<= 1) {
    const int v = tid >= o ? scan[tid - o] : 0;
    __syncthreads();
    scan[tid] += v;
    __syncthreads();
  }
  int u = scan[tid] - cnt;
  for (int i = 0; i < per; ++i) {
    const int q = q0 + i;
    if (!head(q)) continue;
    const int b = (int)((key[q] >> 24) & 0x3FFFFFFFull);
    const float s = run_weight(key, q, n, w, g, inv_k2);
    if (tk_in(u, cap, err)) out[u] = make_int2(b, __float_as_int(s));
    ++u;
  }
  if (tid == kBigThreads - 1) *cnt_a = scan[kBigThreads - 1];
  __syncthreads();  // the buffers are refilled by the next day
}

// The merged entry list of every day with at most kWarpKeys incidences, one warp per
// day (CTA x holds days [x kDayWarps, (x+1) kDayWarps)); a day with more is appended
// to the list `big` for adj_build_big_kernel. Day a's entries go to ent[inc_off[a] ..)
// (room for all its incidences) and their number to cnt[a].
__global__ void __launch_bounds__(kBuildThreads)
    adj_build_kernel(const int32_t* __restrict__ idx, const float* __restrict__ g, int N, int L,
                     int M, int k, const int* __restrict__ off, const int* __restrict__ rev,
                     const long long* __restrict__ inc_off, int* __restrict__ cnt,
                     AdjEntry* __restrict__ ent, int* big, int* nbig, int* err) {
  __shared__ unsigned long long key[kDayWarps * kWarpKeys];
  const int warp = threadIdx.x >> 5;
  const int a = blockIdx.x * kDayWarps + warp;
  if (a >= N) return;  // no CTA barrier in this kernel
  const DayWindow w = day_window(off, a, L, M, k);
  const int n = w.nfwd + (off[w.t_lo + w.nw] - w.r0);
  if (n > kWarpKeys) {
    if ((threadIdx.x & 31) == 0) big[atomicAdd(nbig, 1)] = a;
    return;
  }
  const long long o = inc_off[a];
  merge_day_warp(w, n, key + warp * kWarpKeys, idx, g, off, rev, M, k, ent + o,
                 inc_off[a + 1] - o, cnt + a, err);
}

// The days listed by adj_build_kernel, one CTA each (grid-stride over the list; the
// order in which they are taken does not matter: every day's list is its own).
__global__ void __launch_bounds__(kBigThreads)
    adj_build_big_kernel(const int32_t* __restrict__ idx, const float* __restrict__ g, int N,
                         int L, int M, int k, const int* __restrict__ off,
                         const int* __restrict__ rev, const long long* __restrict__ inc_off,
                         int* __restrict__ cnt, AdjEntry* __restrict__ ent,
                         const int* __restrict__ big, const int* __restrict__ nbig, int* err) {
  __shared__ unsigned long long key[kKeyCap];
  __shared__ int scan[kBigThreads];
  __shared__ int swoff[kMaxL + 1];
  const int nb = *nbig;
  for (int i = blockIdx.x; i < nb; i += gridDim.x) {
    const int d = big[i];
    if (!tk_in(d, N, err)) continue;
    const DayWindow w = day_window(off, d, L, M, k);
    const int n = w.nfwd + (off[w.t_lo + w.nw] - w.r0);
    const long long o = inc_off[d];
    merge_day_block(w, n, key, scan, swoff, idx, g, off, rev, M, k, ent + o, inc_off[d + 1] - o,
                    cnt + d, err);
  }
}

// The points of one thread in the gather: each warp covers 128 consecutive grid
// points [128 w, 128 w + 128), and every load instruction of the warp reads whole
// 128-byte lines (contiguous across the lanes). Form 2: lane l owns the four points
// 128 w + 4 l + [0, 4), one 16-byte load (D a multiple of 4, 16-byte aligned X and
// dX); form 1: two pairs 128 w + 2 l + [0, 2) and 128 w + 64 + 2 l + [0, 2), two
// 8-byte loads (D even, 8-byte aligned X and dX); form 0: four points 128 w + l +
// 32 i, four 4-byte loads (any D). A part of a thread's points at or beyond D is
// loaded from point 0 and not stored. The update acc += w (xa - xb) is taken per
// point as xa - xb (exactly xb * -1 + xa) and one fused multiply-add, as packed FP32
// pairs in forms 1 and 2: the same arithmetic in every form.
struct Quad {
  float2 lo, hi;
};
__device__ __forceinline__ void update_pair(float2& acc, float w, float2 xa, float2 xb) {
  const float2 d = __ffma2_rn(xb, make_float2(-1.f, -1.f), xa);
  acc = __ffma2_rn(make_float2(w, w), d, acc);
}
template <int F> struct Pts;
template <> struct Pts<2> {
  typedef Quad T;
  static constexpr int kParts = 1, kPart = 4;  // parts per thread, points per part
  struct O {  // first point of each part (held in registers)
    int v[1];
  };
  static __device__ __forceinline__ int part(int base, int lane, int) { return base + 4 * lane; }
  static __device__ __forceinline__ T load(const float* row, O o) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(row + o.v[0]));
    return Quad{make_float2(v.x, v.y), make_float2(v.z, v.w)};
  }
  static __device__ __forceinline__ T zero() {
    return Quad{make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
  }
  static __device__ __forceinline__ void update(T& acc, float w, const T& xa, const T& xb) {
    update_pair(acc.lo, w, xa.lo, xb.lo);
    update_pair(acc.hi, w, xa.hi, xb.hi);
  }
  // value of point j (0 <= j < kPart) of part i
  static __device__ __forceinline__ float get(const T& v, int, int j) {
    return j == 0 ? v.lo.x : j == 1 ? v.lo.y : j == 2 ? v.hi.x : v.hi.y;
  }
};
template <> struct Pts<1> : Pts<2> {
  static constexpr int kParts = 2, kPart = 2;
  struct O {
    int v[2];
  };
  static __device__ __forceinline__ int part(int base, int lane, int i) {
    return base + 64 * i + 2 * lane;
  }
  static __device__ __forceinline__ T load(const float* row, O o) {
    return Quad{__ldg(reinterpret_cast<const float2*>(row + o.v[0])),
                __ldg(reinterpret_cast<const float2*>(row + o.v[1]))};
  }
  static __device__ __forceinline__ float get(const T& v, int i, int j) {
    return i == 0 ? (j == 0 ? v.lo.x : v.lo.y) : (j == 0 ? v.hi.x : v.hi.y);
  }
};
template <> struct Pts<0> {
  struct T {
    float v[4];
  };
  static constexpr int kParts = 4, kPart = 1;
  struct O {
    int v[4];
  };
  static __device__ __forceinline__ int part(int base, int lane, int i) {
    return base + 32 * i + lane;
  }
  static __device__ __forceinline__ T load(const float* row, O o) {
    T t;
#pragma unroll
    for (int i = 0; i < 4; ++i) t.v[i] = __ldg(row + o.v[i]);
    return t;
  }
  static __device__ __forceinline__ T zero() { return T{{0.f, 0.f, 0.f, 0.f}}; }
  static __device__ __forceinline__ void update(T& acc, float w, const T& xa, const T& xb) {
#pragma unroll
    for (int i = 0; i < 4; ++i) acc.v[i] = fmaf(w, xa.v[i] - xb.v[i], acc.v[i]);
  }
  static __device__ __forceinline__ float get(const T& v, int i, int) { return v.v[i]; }
};

constexpr int kAdjR = 2;              // days per gather CTA
constexpr int kStage = 2048;          // entries staged in shared memory at a time
constexpr int kU = 16;                 // partner loads in flight per thread (a power of 2)
constexpr int kGatherMaxThreads = 256;

// acc += w (xa - X[b]) over the staged entries [q, q + U), partner loads first.
template <int F, int U>
__device__ __forceinline__ void gather_group(typename Pts<F>::T& acc,
                                             const typename Pts<F>::T& xa, const float* X,
                                             typename Pts<F>::O o, int D, const AdjEntry* se) {
  typedef Pts<F> P;
  typename P::T xb[U];
#pragma unroll
  for (int u = 0; u < U; ++u) xb[u] = P::load(X + (size_t)se[u].x * D, o);
#pragma unroll
  for (int u = 0; u < U; ++u) P::update(acc, __int_as_float(se[u].y), xa, xb[u]);
}

// The rest of a day's entries after the groups of kU (staged entries from position
// c0 on): groups of S, S/2, ..., 1 (S = kU/2), so that every count below kU is covered.
template <int F, int S>
__device__ __forceinline__ void gather_rest(typename Pts<F>::T& acc,
                                            const typename Pts<F>::T& xa, const float* X,
                                            typename Pts<F>::O o, int D, const AdjEntry* se,
                                            int c0, int& q, int q1) {
  if constexpr (S >= 1) {
    if (q + S <= q1) {
      gather_group<F, S>(acc, xa, X, o, D, se + (q - c0));
      q += S;
    }
    gather_rest<F, S / 2>(acc, xa, X, o, D, se, c0, q, q1);
  }
}
static_assert((kU & (kU - 1)) == 0, "the rest of a day is split in powers of 2 below kU");

// dX for kAdjR consecutive days and one tile of grid points (blockIdx.x the day block,
// blockIdx.y the tile: CTAs are scheduled with x fastest, so the CTAs running at one
// time share a tile of X, which stays in L2 while the entries re-read its rows). The
// days' entries are staged in shared memory (the same for every thread); each thread
// owns four grid points and walks the days in order with one accumulator,
// adding w (X[a] - X[b]) for every entry (b, w) of day a in list order, partner
// values loaded kU entries at a time (then kU/2, ..., 1 for the rest of a day).
template <int F>
__global__ void __launch_bounds__(kGatherMaxThreads)
    adj_gather_kernel(const float* __restrict__ X, int N, int D,
                      const long long* __restrict__ inc_off, const int* __restrict__ cnt,
                      const AdjEntry* __restrict__ ent, const float* __restrict__ wts,
                      float* __restrict__ dX, int tiles, int* err) {
  typedef Pts<F> P;
  typedef typename P::T T;
  __shared__ AdjEntry se[kStage];
  __shared__ int sday[kAdjR + 1];  // first staged position of each day
  const int a0 = blockIdx.x * kAdjR;
  const int nd = min(kAdjR, N - a0);
  if (threadIdx.x < 32) {  // exclusive scan of the days' entry counts
    const int lane = threadIdx.x;
    const int c = lane < nd ? cnt[a0 + lane] : 0;
    int s = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += v;
    }
    if (lane <= kAdjR) sday[lane] = s - c;
  }
  __syncthreads();
  const int ntot = sday[kAdjR];
  for (int tile = blockIdx.y; tile < tiles; tile += gridDim.y) {
    const int slot = tile * blockDim.x + threadIdx.x;
    const int base = 128 * (slot >> 5), lane = slot & 31;
    typename P::O o;      // first point of each part (0 for a part beyond D)
    bool own[P::kParts];  // the part lies within the row
#pragma unroll
    for (int i = 0; i < P::kParts; ++i) {
      const int pi = P::part(base, lane, i);
      own[i] = pi < D;
      o.v[i] = own[i] ? pi : 0;
    }
    int d = 0, q = 0;
    T acc = P::zero();
    T xa = nd > 0 ? P::load(X + (size_t)a0 * D, o) : P::zero();
    for (int c0 = 0;; c0 += kStage) {
      const int c1 = min(ntot, c0 + kStage);
      __syncthreads();  // the staged entries of the previous chunk (or tile) have been read
      for (int dd = 0; dd < nd; ++dd) {
        const int s0 = max(sday[dd], c0), s1 = min(sday[dd + 1], c1);
        const long long base = inc_off[a0 + dd] - sday[dd];
        for (int i = s0 + threadIdx.x; i < s1; i += blockDim.x) {
          AdjEntry e = __ldg(ent + base + i);
          if (!tk_in(e.x, N, err)) e = make_int2(a0 + dd, 0);  // debug build: adds 0
          se[i - c0] = e;
        }
      }
      __syncthreads();
      while (d < nd) {
        const int q1 = min(sday[d + 1], c1);
        for (; q + kU <= q1; q += kU) gather_group<F, kU>(acc, xa, X, o, D, se + q - c0);
        gather_rest<F, kU / 2>(acc, xa, X, o, D, se, c0, q, q1);
        if (q1 < sday[d + 1]) break;  // the day continues in the next chunk
        float* dp = dX + (size_t)(a0 + d) * D;
#pragma unroll
        for (int i = 0; i < P::kParts; ++i)
#pragma unroll
          for (int j = 0; j < P::kPart; ++j)
            if (own[i]) dp[o.v[i] + j] = wts ? P::get(acc, i, j) * wts[o.v[i] + j] : P::get(acc, i, j);
        ++d;
        acc = P::zero();
        if (d < nd) xa = P::load(X + (size_t)(a0 + d) * D, o);
      }
      if (c1 >= ntot) break;
    }
  }
}

}  // namespace

namespace {

inline size_t up256(size_t v) { return (v + 255) / 256 * 256; }

// Workspace layout: merged entries (room for every incidence, 2 L k M in all), the
// days' entry offsets and counts, then the reverse neighbour index (count, cursor),
// the number of days left to adj_build_big_kernel (zeroed with count and cursor),
// off, rev, and the list of those days.
struct AdjLayout {
  size_t ent, inc_off, cnt, count, total;
};

AdjLayout adj_layout(int N, int L, int k) {
  const size_t M = (size_t)(N - L + 1);
  AdjLayout l;
  l.ent = 0;
  l.inc_off = up256(2 * (size_t)L * k * M * sizeof(AdjEntry));
  l.cnt = l.inc_off + up256(((size_t)N + 1) * sizeof(long long));
  l.count = l.cnt + up256((size_t)N * sizeof(int));
  l.total = l.count + up256((3 * M + 2 + M * (size_t)k + (size_t)N) * sizeof(int));
  return l;
}

// Threads per gather CTA for `quads` thread slots along a row: whole warps, at most
// kGatherMaxThreads, tiles chosen to leave the fewest idle warps.
int gather_threads(int quads, int* tiles) {
  const int warps = (quads + 31) / 32;
  int best_t = 0, best_w = 0;
  for (int per = kGatherMaxThreads / 32; per >= 4; --per) {
    const int t = (warps + per - 1) / per;
    if (best_t == 0 || t * per - warps < best_t * best_w - warps) {
      best_t = t;
      best_w = per;
    }
  }
  if (warps < 4) {
    best_t = 1;
    best_w = warps;
  }
  *tiles = best_t;
  return best_w * 32;
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
  long long* inc_off = reinterpret_cast<long long*>(base + lay.inc_off);
  int* cnt = reinterpret_cast<int*>(base + lay.cnt);
  int* count = reinterpret_cast<int*>(base + lay.count);
  int* cursor = count + M;
  int* nbig = cursor + M;
  int* off = nbig + 1;
  int* rev = off + M + 1;
  int* big = rev + (size_t)M * k;
  cudaError_t e = cudaMemsetAsync(count, 0, ((size_t)2 * M + 1) * sizeof(int), st);
  if (e != cudaSuccess) return e;
  const long long nq = (long long)M * k;
  const int blocks = (int)((nq + 255) / 256);
  adj_count_kernel<<<blocks, 256, 0, st>>>(idx, M, k, count, err);
  adj_scan_kernel<<<1, 1024, 0, st>>>(count, M, off);
  adj_fill_kernel<<<blocks, 256, 0, st>>>(idx, M, k, off, cursor, rev);
  adj_sort_kernel<<<(M + 127) / 128, 128, 0, st>>>(off, N, L, M, k, rev);
  adj_day_scan_kernel<<<1, 1024, 0, st>>>(off, N, L, M, k, inc_off);
  adj_build_kernel<<<(N + kDayWarps - 1) / kDayWarps, kBuildThreads, 0, st>>>(
      idx, g, N, L, M, k, off, rev, inc_off, cnt, ent, big, nbig, err);
  int dev = 0, sms = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return e;
  adj_build_big_kernel<<<2 * sms, kBigThreads, 0, st>>>(idx, g, N, L, M, k, off, rev, inc_off,
                                                        cnt, ent, big, nbig, err);
  // 16-byte loads where D is a multiple of 4 and X, dX 16-byte aligned; 8-byte loads
  // where D is even and they are 8-byte aligned; else 4-byte loads
  const uintptr_t al = reinterpret_cast<uintptr_t>(X) | reinterpret_cast<uintptr_t>(dX);
  const int form = D < 4 || D % 2 != 0 || al % 8 != 0 ? 0 : (D % 4 == 0 && al % 16 == 0 ? 2 : 1);
  const int slots = (D + 3) / 4;  // four points per thread in every form
  int tiles = 1;
  const int threads = gather_threads(slots, &tiles);
  const dim3 grid((N + kAdjR - 1) / kAdjR, tiles < 65535 ? tiles : 65535);
  if (form == 2)
    adj_gather_kernel<2><<<grid, threads, 0, st>>>(X, N, D, inc_off, cnt, ent, wts, dX,
                                                    tiles, err);
  else if (form == 1)
    adj_gather_kernel<1><<<grid, threads, 0, st>>>(X, N, D, inc_off, cnt, ent, wts, dX,
                                                    tiles, err);
  else
    adj_gather_kernel<0><<<grid, threads, 0, st>>>(X, N, D, inc_off, cnt, ent, wts, dX,
                                                    tiles, err);
  *launches += 8;
  return cudaGetLastError();
}

}  // namespace traknn
