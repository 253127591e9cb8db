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
// Each output row is owned by one CTA that sums its incidences in a fixed order,
// so no floating-point atomics are used and the result is bitwise reproducible.
// The reverse lists (who has j as a neighbour) come from a counting sort whose
// segments are then sorted by t (heap sort, one thread per segment).
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

constexpr int kMaxInc = 2048;  // incidences of one day merged in the gather's shared memory

// Incidences of day a: the forward ones (k per trajectory t of its window) and the
// reverse segments of the days j of its window, [max(0, a-L+1), min(a, M-1)].
__device__ __forceinline__ int day_incidences(const int* off, int a, int L, int M, int k) {
  const int t_lo = max(0, a - L + 1), t_hi = min(a, M - 1);
  if (t_hi < t_lo) return 0;
  return (t_hi - t_lo + 1) * k + (off[t_hi + 1] - off[t_lo]);
}

// Sort ascending (heap sort, in place) every reverse segment that some day reads one
// incidence at a time: a day with more incidences than the gather's buffer, whose
// summation order must not depend on the order the fill kernel produced. The other
// days order their incidences by key in the gather and need no sorted segments.
__global__ void adj_sort_kernel(const int* __restrict__ off, int N, int L, int M, int k,
                                int* rev) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= M) return;
  bool needed = false;
  for (int d = j; d < min(N, j + L); ++d) needed |= day_incidences(off, d, L, M, k) > kMaxInc;
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

constexpr int kGatherThreads = 256;
constexpr int kPerThread = kMaxInc / kGatherThreads;  // consecutive positions per thread

// One CTA per day a: dX[a] = sum over incidences w (X[a] - X[b]).
//
// The incidences are listed in shared memory as keys (partner day b, kind, window
// slot): a forward incidence (trajectory t, neighbour j, b = j + a - t) has kind 0
// and slot t - t_lo, a reverse one (j in the window, t with j among its neighbours,
// b = t + a - j) kind 1 and slot j - t_lo. For one partner no two incidences share
// kind and slot, so the sorted order does not depend on the order the lists were
// built in. The weights of each partner are summed in key order and the partners
// are visited in increasing day order, so every partner row X[b] is read once
// (consecutive days tend to have consecutive neighbours, so a day's incidences have
// about half as many distinct partners). A day with more incidences than the buffer
// holds sums them one by one, forward then reverse in sorted segments. Both ways the
// order is fixed, so the result is bitwise reproducible.
__global__ void __launch_bounds__(kGatherThreads)
    adj_gather_kernel(const float* __restrict__ X, int N, int D, int L, int M, int k,
                      const int32_t* __restrict__ idx, const float* __restrict__ g,
                      const int* __restrict__ off, const int* __restrict__ rev,
                      const float* __restrict__ wts, float* __restrict__ dX) {
  __shared__ unsigned long long key[kMaxInc];  // (partner << 32) | position
  __shared__ float wsum[kMaxInc];              // merged weight of each distinct partner
  __shared__ int part[kMaxInc];                // distinct partners, increasing
  __shared__ int scan[kGatherThreads];
  __shared__ int rstart[kMaxL + 1];            // first position of each reverse segment
  const int a = blockIdx.x;
  const int tid = threadIdx.x;
  const float* xa = X + (size_t)a * D;
  const int t_lo = max(0, a - L + 1), t_hi = min(a, M - 1);
  const int nt = max(0, t_hi - t_lo + 1);
  const float inv_k2 = 2.0f / (float)k;
  const int nfwd = nt * k;
  if (tid == 0) {
    int pos = nfwd;
    for (int j = t_lo; j <= t_hi; ++j) {
      rstart[j - t_lo] = pos;
      pos += off[j + 1] - off[j];
    }
    rstart[nt] = pos;
  }
  __syncthreads();
  const int ninc = rstart[nt];
  const bool merged = ninc <= kMaxInc;
  int nu = 0;
  if (merged) {
    int n2 = 1;
    while (n2 < ninc) n2 <<= 1;
    for (int q = tid; q < n2; q += kGatherThreads) {
      unsigned long long kq = ~0ull;  // padding and invalid entries sort last
      if (q < nfwd) {
        const int ts = q / k;
        const int t = t_lo + ts;
        const int j = idx[(size_t)t * k + q % k];
        if (j >= 0 && j < M) kq = ((unsigned long long)(unsigned)(j + a - t) << 32) | (unsigned)ts;
      } else if (q < ninc) {
        int sg = 0;
        while (rstart[sg + 1] <= q) ++sg;  // reverse segment of day j = t_lo + sg
        const int j = t_lo + sg;
        const int t = rev[off[j] + (q - rstart[sg])];
        kq = ((unsigned long long)(unsigned)(t + a - j) << 32) | (1u << 16) | (unsigned)sg;
      }
      key[q] = kq;
    }
    __syncthreads();
    // bitonic sort of the n2 keys (ascending)
    for (int size = 2; size <= n2; size <<= 1) {
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        for (int q = tid; q < n2; q += kGatherThreads) {
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
    // run heads (first position of each distinct valid partner), numbered by an
    // exclusive prefix sum over the thread's kPerThread consecutive positions
    auto head = [&](int q) {
      if (q >= ninc || key[q] == ~0ull) return 0;
      return (q == 0 || (key[q - 1] >> 32) != (key[q] >> 32)) ? 1 : 0;
    };
    const int q0 = tid * kPerThread;
    int cnt = 0;
    for (int i = 0; i < kPerThread; ++i) cnt += head(q0 + i);
    scan[tid] = cnt;
    __syncthreads();
    for (int o = 1; o < kGatherThreads; o <<= 1) {
      const int v = tid >= o ? scan[tid - o] : 0;
      __syncthreads();
      scan[tid] += v;
      __syncthreads();
    }
    int u = scan[tid] - cnt;
    for (int i = 0; i < kPerThread; ++i) {
      const int q = q0 + i;
      if (!head(q)) continue;
      const unsigned long long b = key[q] >> 32;
      float w = 0.f;
      for (int r = q; r < ninc && key[r] != ~0ull && (key[r] >> 32) == b; ++r) {
        // the incidence's trajectory t, recovered from its kind and slot
        const unsigned lo = (unsigned)key[r];
        const int slot = (int)(lo & 0xFFFFu);
        const int t = (lo >> 16) ? (int)b - a + t_lo + slot : t_lo + slot;
        w += inv_k2 * g[t];
      }
      part[u] = (int)b;
      wsum[u] = w;
      ++u;
    }
    nu = scan[kGatherThreads - 1];
    __syncthreads();
  }
  for (int p0 = 0; p0 < D; p0 += kGatherThreads * 4) {
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    float xv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int p = p0 + u * kGatherThreads + tid;
      xv[u] = p < D ? xa[p] : 0.f;
    }
    if (merged) {
      for (int v = 0; v < nu; ++v) {
        const float w = wsum[v];
        const float* xb = X + (size_t)part[v] * D;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int p = p0 + u * kGatherThreads + tid;
          if (p < D) acc[u] = fmaf(w, xv[u] - xb[p], acc[u]);
        }
      }
    } else {
      for (int t = t_lo; t <= t_hi; ++t) {
        const float w = inv_k2 * g[t];
        for (int i = 0; i < k; ++i) {
          const int j = idx[(size_t)t * k + i];
          if (j < 0 || j >= M) continue;
          const float* xb = X + (size_t)(j + a - t) * D;
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int p = p0 + u * kGatherThreads + tid;
            if (p < D) acc[u] = fmaf(w, xv[u] - xb[p], acc[u]);
          }
        }
      }
      for (int j = t_lo; j <= t_hi; ++j) {
        for (int r = off[j]; r < off[j + 1]; ++r) {
          const int t = rev[r];
          const float w = inv_k2 * g[t];
          const float* xb = X + (size_t)(t + a - j) * D;
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int p = p0 + u * kGatherThreads + tid;
            if (p < D) acc[u] = fmaf(w, xv[u] - xb[p], acc[u]);
          }
        }
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int p = p0 + u * kGatherThreads + tid;
      if (p < D) dX[(size_t)a * D + p] = wts ? acc[u] * wts[p] : acc[u];
    }
  }
}

}  // namespace

size_t adjoint_workspace_bytes(int M, int k) {
  return ((size_t)3 * M + 1 + (size_t)M * k) * sizeof(int) + 1024;
}

cudaError_t launch_adjoint(const float* X, int N, int D, int L, int k, const int32_t* idx,
                           const float* g, const float* wts, float* dX, void* ws, int* err,
                           cudaStream_t st, int* launches) {
  const int M = N - L + 1;
  int* count = static_cast<int*>(ws);
  int* cursor = count + M;
  int* off = cursor + M;
  int* rev = off + M + 1;
  cudaError_t e = cudaMemsetAsync(count, 0, (size_t)2 * M * sizeof(int), st);
  if (e != cudaSuccess) return e;
  const long long nq = (long long)M * k;
  const int blocks = (int)((nq + 255) / 256);
  adj_count_kernel<<<blocks, 256, 0, st>>>(idx, M, k, count, err);
  adj_scan_kernel<<<1, 1024, 0, st>>>(count, M, off);
  adj_fill_kernel<<<blocks, 256, 0, st>>>(idx, M, k, off, cursor, rev);
  adj_sort_kernel<<<(M + 127) / 128, 128, 0, st>>>(off, N, L, M, k, rev);
  adj_gather_kernel<<<N, kGatherThreads, 0, st>>>(X, N, D, L, M, k, idx, g, off, rev, wts, dX);
  *launches += 5;
  return cudaGetLastError();
}

}  // namespace traknn
