// kernels_aux.cu -- the light kernels around the fused Gram/top-k kernels:
//   column means (optional centring, exact by the offset invariance of Eq. 2),
//   operand preparation with FP64 day norms (Algorithm 1, norm precomputation),
//   window sums of the norms, and the final merge of partial neighbour lists
//   into sorted neighbour sets and rarity scores (Eq. 3).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math_constants.h>

#include <climits>
#include <cstdint>

#include "internal.h"

namespace traknn {
namespace {

// The centring offset only has to be one fixed field subtracted from every day (any
// value keeps Eq. 2 exact); the mean over the last kMeanDays days is close enough to
// the full mean to shrink the Gram values as well, costs a small fraction of a pass
// over X, and lies in the first part of X a host-buffer call copies in.

// Column sums of the centring days (the last kMeanDays) over fixed slices (fixed
// summation order: deterministic).
__global__ void col_partial_kernel(const float* __restrict__ X, int N, int D, float* partial) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= D) return;
  const int first = mean_first(N), ns = mean_days(N);
  const int per = (ns + kMeanSlices - 1) / kMeanSlices;
  const int r0 = blockIdx.y * per, r1 = min(ns, r0 + per);
  float acc = 0.f;
  for (int i = r0; i < r1; ++i) acc += X[(size_t)(first + i) * D + p];
  partial[(size_t)blockIdx.y * D + p] = acc;
}

// FP32 sums suffice for the offset (see above).
__global__ void col_final_kernel(const float* __restrict__ partial, int N, int D, float* mu,
                                 int center) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= D) return;
  if (!center) {
    mu[p] = 0.f;
    return;
  }
  float acc = 0.f;
  for (int s = 0; s < kMeanSlices; ++s) acc += partial[(size_t)s * D + p];
  mu[p] = acc / (float)mean_days(N);
}

__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
  return s;
}

// One block per day: centred FP32 copy (row pitch Dp, zero padded) and the
// FP64 squared norm of the centred row.
__global__ void prep_fp32_kernel(const float* __restrict__ X, int D, int Dp,
                                 const float* __restrict__ mu, const float* __restrict__ wts,
                                 float* __restrict__ Xc, double* __restrict__ norms) {
  __shared__ double red[32];
  const int a = blockIdx.x;
  const float* x = X + (size_t)a * D;
  float* y = Xc + (size_t)a * Dp;
  double acc = 0.0;
  for (int p = threadIdx.x; p < Dp; p += blockDim.x) {
    float v = p < D ? x[p] - mu[p] : 0.f;
    if (wts && p < D) v *= sqrtf(wts[p]);  // grid-point weight w_p enters as sqrt(w_p)
    y[p] = v;
    acc = fma((double)v, (double)v, acc);
  }
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) norms[a] = s;
}

// Index of the series whose [base, base + count) range of stacked rows holds r.
__device__ __forceinline__ int find_series(const SeriesInfo* sr, int ns, int r, bool traj) {
  int lo = 0, hi = ns - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    const int base = traj ? sr[mid].out_base : sr[mid].row_base;
    if (base <= r) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Column sums of every series' centring days over fixed slices (grid.z = series).
__global__ void col_partial_series_kernel(const __grid_constant__ SeriesTable st, int D,
                                          float* partial) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= D) return;
  const SeriesInfo& si = st.s[blockIdx.z];
  const int first = mean_first(si.N), ns = mean_days(si.N);
  const int per = (ns + kMeanSlices - 1) / kMeanSlices;
  const int r0 = blockIdx.y * per, r1 = min(ns, r0 + per);
  float acc = 0.f;
  for (int i = r0; i < r1; ++i) acc += si.X[(size_t)(first + i) * D + p];
  partial[((size_t)blockIdx.z * kMeanSlices + blockIdx.y) * D + p] = acc;
}

__global__ void col_final_series_kernel(const __grid_constant__ SeriesTable st,
                                        const float* partial, int D, float* mu, int center) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= D) return;
  const int b = blockIdx.y;
  if (!center) {
    mu[(size_t)b * D + p] = 0.f;
    return;
  }
  float acc = 0.f;
  for (int s = 0; s < kMeanSlices; ++s) acc += partial[((size_t)b * kMeanSlices + s) * D + p];
  mu[(size_t)b * D + p] = acc / (float)mean_days(st.s[b].N);
}

// One warp per stacked day: the centred row x - mu(series) as two BF16 copies hi + lo
// (split form; the BF16 form uses hi alone) in the tensor-core operand layout, its
// FP64 norm, and its correction value.
//
// Layout: `groups` = ceil(D / 63) groups of 64 K entries. Group b holds the grid
// points b, b + groups, b + 2 groups, ... (63 at most), so that every group samples
// the whole grid and carries about 1/groups of the row's energy; entry 63 of every
// group holds c = bf16(sqrt(n / groups)) in hi and -c in lo. The three split
// products of that entry add hi_a hi_b + hi_a lo_b + lo_a hi_b = -c_a c_b to the
// Gram accumulator once per group, so the tensor cores accumulate
// G_ab - groups c_a c_b, which stays near zero for the close pairs that decide the
// neighbour sets, instead of G_ab itself; the epilogue adds groups c_a c_b back in
// FP32. A permutation of the grid points (the same for every row) leaves the Gram
// unchanged. With kCorr false (BF16 form) the correction entries and c are zero.
//
// With emb > 1 operand row a is the trajectory of emb consecutive days a .. a+emb-1
// (Eq. 1): its emb * D values are X[a][0..D), X[a+1][0..D), ..., which in the
// row-major input are the contiguous values X + a*D .. X + (a+emb)*D. The Gram of
// such rows is the diagonal window sum of Eq. 2 (sum over m of <x_{a+m}, x_{b+m}>),
// and the norm of a row is the window sum of the day norms.
template <bool kCorr, bool kEmb>
__global__ void __launch_bounds__(256)
    prep_split_series_kernel(const __grid_constant__ SeriesTable st, int r_lo, int rows, int D,
                             int emb, int groups, const float* __restrict__ mu,
                             const float* __restrict__ wts, __nv_bfloat16* __restrict__ hi,
                             __nv_bfloat16* __restrict__ lo, double* __restrict__ norms,
                             float* __restrict__ cval) {
  // per warp: 32 finished groups of one copy (36-word rows: 16-byte aligned)
  __shared__ __align__(16) uint32_t stage[8][32 * 36];
  const int r = r_lo + blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (r >= rows) return;
  uint32_t* sh = stage[threadIdx.x >> 5];
  const int b = find_series(st.s, st.n, r, false);
  const SeriesInfo& si = st.s[b];
  const int a = r - si.row_base;
  const int Dp = groups * 64;
  __nv_bfloat162* h2 = reinterpret_cast<__nv_bfloat162*>(hi + (size_t)r * Dp);
  __nv_bfloat162* l2 = reinterpret_cast<__nv_bfloat162*>(lo + (size_t)r * Dp);
  if (a >= si.N) {  // padding row between series: zeros
    const __nv_bfloat162 z = __floats2bfloat162_rn(0.f, 0.f);
    for (int q = lane; q < Dp / 2; q += 32) {
      h2[q] = z;
      l2[q] = z;
    }
    if (lane == 0) {
      norms[r] = 0.0;
      cval[r] = 0.f;
    }
    return;
  }
  const float* x = si.X + (size_t)a * D;
  const float* m = mu + (size_t)b * D;
  const int Dlen = emb * D;  // values of one operand row
  // grid-point weights w_p enter the distance as sqrt(w_p) scalings of the values
  auto val = [&](int i) {
    const int pnt = kEmb ? i % D : i;  // grid point of value i
    return wts ? (x[i] - m[pnt]) * sqrtf(wts[pnt]) : x[i] - m[pnt];
  };
  // One read of the row. Lane g0 + lane builds group g0 + lane: its entry pos is grid
  // point pos * groups + g, so for each pos the warp reads 32 consecutive grid points
  // (coalesced). The warp's 32 groups, contiguous in the output row, are staged in
  // shared memory (one copy at a time) and written with contiguous 16-byte stores;
  // entry 63 (the correction) is written once the row's norm is known. The FP64 norm
  // sums each group's FP32 squares.
  double acc = 0.0;
  for (int g0 = 0; g0 < groups; g0 += 32) {
    const int g = g0 + lane;
    const int ng = min(32, groups - g0);  // groups of this pass
    uint32_t hv[32], lv[32];  // 64 BF16 entries per copy, in pairs
    float part = 0.f;
#pragma unroll
    for (int pp = 0; pp < 32; ++pp) {
      const int i0 = (2 * pp) * groups + g, i1 = (2 * pp + 1) * groups + g;
      const float v0 = i0 < Dlen ? val(i0) : 0.f;
      const float v1 = (pp < 31 && i1 < Dlen) ? val(i1) : 0.f;  // entry 63 filled later
      part = fmaf(v0, v0, part);
      part = fmaf(v1, v1, part);
      const __nv_bfloat16 h0 = __float2bfloat16_rn(v0);
      const __nv_bfloat16 q0 = __float2bfloat16_rn(v0 - __bfloat162float(h0));
      const __nv_bfloat16 h1 = __float2bfloat16_rn(v1);
      const __nv_bfloat16 q1 = __float2bfloat16_rn(v1 - __bfloat162float(h1));
      const __nv_bfloat162 hp = __halves2bfloat162(h0, h1);
      const __nv_bfloat162 lp = __halves2bfloat162(q0, q1);
      hv[pp] = *reinterpret_cast<const uint32_t*>(&hp);
      lv[pp] = *reinterpret_cast<const uint32_t*>(&lp);
    }
    if (g < groups) acc += (double)part;
    // hi, then lo: 16-byte chunk c of the pass is chunk c % 8 of group g0 + c / 8
#pragma unroll
    for (int copy = 0; copy < 2; ++copy) {
      const uint32_t* v = copy == 0 ? hv : lv;
      if (g < groups) {
        uint4* st4 = reinterpret_cast<uint4*>(sh + lane * 36);
#pragma unroll
        for (int q4 = 0; q4 < 8; ++q4)
          st4[q4] = make_uint4(v[4 * q4], v[4 * q4 + 1], v[4 * q4 + 2], v[4 * q4 + 3]);
      }
      __syncwarp();
      uint4* dst = reinterpret_cast<uint4*>((copy == 0 ? h2 : l2) + (size_t)g0 * 32);
      for (int c = lane; c < ng * 8; c += 32)
        dst[c] = *reinterpret_cast<const uint4*>(sh + (c >> 3) * 36 + (c & 7) * 4);
      __syncwarp();
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  const float c = kCorr ? __bfloat162float(__float2bfloat16_rn((float)sqrt(acc / groups))) : 0.f;
  // the correction entries of this lane's groups (same thread as the stores above)
  __nv_bfloat16* hrow = hi + (size_t)r * Dp;
  __nv_bfloat16* lrow = lo + (size_t)r * Dp;
  for (int g = lane; g < groups; g += 32) {
    hrow[g * 64 + 63] = __float2bfloat16_rn(c);
    lrow[g * 64 + 63] = __float2bfloat16_rn(-c);
  }
  if (lane == 0) {
    norms[r] = acc;
    cval[r] = c;
  }
}

// The same operand preparation for rows of few groups (groups <= 16, e.g. the
// trajectory-embedded rows of a small grid): a warp takes 32 / groups rows at once,
// lane (r, g) = (lane / groups, lane % groups) building group g of row r, so that no
// lane idles; the row's FP64 norm is summed over its lanes in a fixed order. The grid
// point of value i (i mod D) is stepped along with i instead of divided.
template <bool kCorr>
__global__ void __launch_bounds__(256)
    prep_split_small_kernel(const __grid_constant__ SeriesTable st, int r_lo, int rows, int D,
                            int emb, int groups, const float* __restrict__ mu,
                            const float* __restrict__ wts, __nv_bfloat16* __restrict__ hi,
                            __nv_bfloat16* __restrict__ lo, double* __restrict__ norms,
                            float* __restrict__ cval) {
  const int lane = threadIdx.x & 31;
  const int per_warp = 32 / groups;
  const int rl = lane / groups, g = lane - rl * groups;  // row of the warp, group of the row
  const int r = r_lo + (blockIdx.x * 8 + (threadIdx.x >> 5)) * per_warp + rl;
  const bool act = rl < per_warp && r < rows;
  const int Dp = groups * 64;
  double part = 0.0;
  int b = 0;
  bool pad = true;
  if (act) {
    b = find_series(st.s, st.n, r, false);
    const SeriesInfo& si = st.s[b];
    const int a = r - si.row_base;
    pad = a >= si.N;
    uint4* hd = reinterpret_cast<uint4*>(hi + (size_t)r * Dp + g * 64);
    uint4* ld = reinterpret_cast<uint4*>(lo + (size_t)r * Dp + g * 64);
    uint32_t hv[32], lv[32];
    float fp = 0.f;
    if (!pad) {
      const float* x = si.X + (size_t)a * D;
      const float* m = mu + (size_t)b * D;
      const int Dlen = emb * D;
      int pnt = g % D;  // grid point of value i = pos * groups + g, stepped with pos
#pragma unroll
      for (int pp = 0; pp < 32; ++pp) {
        float v[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int pos = 2 * pp + h, i = pos * groups + g;
          float val = 0.f;
          if (i < Dlen && pos < 63) {
            val = x[i] - m[pnt];
            if (wts) val *= sqrtf(wts[pnt]);
          }
          v[h] = val;
          pnt += groups;  // groups <= D (emb <= 17 < 63), so one subtraction suffices
          if (pnt >= D) pnt -= D;
        }
        fp = fmaf(v[0], v[0], fp);
        fp = fmaf(v[1], v[1], fp);
        const __nv_bfloat16 h0 = __float2bfloat16_rn(v[0]);
        const __nv_bfloat16 q0 = __float2bfloat16_rn(v[0] - __bfloat162float(h0));
        const __nv_bfloat16 h1 = __float2bfloat16_rn(v[1]);
        const __nv_bfloat16 q1 = __float2bfloat16_rn(v[1] - __bfloat162float(h1));
        const __nv_bfloat162 hp = __halves2bfloat162(h0, h1);
        const __nv_bfloat162 lp = __halves2bfloat162(q0, q1);
        hv[pp] = *reinterpret_cast<const uint32_t*>(&hp);
        lv[pp] = *reinterpret_cast<const uint32_t*>(&lp);
      }
    } else {
#pragma unroll
      for (int pp = 0; pp < 32; ++pp) hv[pp] = lv[pp] = 0u;
    }
    part = (double)fp;
#pragma unroll
    for (int q4 = 0; q4 < 8; ++q4) {
      hd[q4] = make_uint4(hv[4 * q4], hv[4 * q4 + 1], hv[4 * q4 + 2], hv[4 * q4 + 3]);
      ld[q4] = make_uint4(lv[4 * q4], lv[4 * q4 + 1], lv[4 * q4 + 2], lv[4 * q4 + 3]);
    }
  }
  // the row's norm: its groups' FP32 sums added in group order by the row's first lane
  double acc = 0.0;
  const int first = rl * groups;
  for (int j = 0; j < groups; ++j) {
    const double pj = __shfl_sync(0xffffffffu, part, min(31, first + j));
    acc += pj;
  }
  if (!act) return;
  const float c = (kCorr && !pad)
                      ? __bfloat162float(__float2bfloat16_rn((float)sqrt(acc / groups)))
                      : 0.f;
  hi[(size_t)r * Dp + g * 64 + 63] = __float2bfloat16_rn(c);
  lo[(size_t)r * Dp + g * 64 + 63] = __float2bfloat16_rn(-c);
  if (g == 0) {
    norms[r] = pad ? 0.0 : acc;
    cval[r] = c;
  }
}

// W of every stacked trajectory row: an explicit L-term FP64 sum of its series' norms.
__global__ void window_series_kernel(const __grid_constant__ SeriesTable st, int r_lo,
                                     int out_rows, const double* __restrict__ norms, float* W) {
  const int r = r_lo + blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= out_rows) return;
  const int b = find_series(st.s, st.n, r, true);
  const SeriesInfo& si = st.s[b];
  const int t = r - si.out_base;
  if (t >= si.M) {
    W[r] = 0.f;
    return;
  }
  double s = 0.0;
  for (int m = 0; m < si.L; ++m) s += norms[si.row_base + t + m];
  W[r] = (float)s;
}

// W_t = sum_{m<L} n_{t+m}: an explicit L-term FP64 sum per trajectory.
__global__ void window_kernel(const double* __restrict__ norms, int M, int L, float* W) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= M) return;
  double s = 0.0;
  for (int m = 0; m < L; ++m) s += norms[t + m];
  W[t] = (float)s;
}

// One warp per trajectory row: a P-way merge of the row's sorted partial lists
// (lane p walks list p), k rounds of a warp arg-min on (distance, index).
// The score is the FP64 mean of the k selected distances (Eq. 3).
__global__ void merge_kernel(const float* __restrict__ part_d, const int32_t* __restrict__ part_i,
                             int M, int P, int k, int32_t* __restrict__ idx,
                             float* __restrict__ dist, float* __restrict__ score) {
  const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (t >= M) return;
  const float* pd = part_d + (size_t)t * P * k;
  const int32_t* pi = part_i + (size_t)t * P * k;
  int cur = 0;
  double sum = 0.0;
  for (int r = 0; r < k; ++r) {
    float hd = CUDART_INF_F;
    int hidx = INT_MAX;
    if (lane < P && cur < k) {
      const int ii = pi[lane * k + cur];
      if (ii >= 0) {
        hd = pd[lane * k + cur];
        hidx = ii;
      }
    }
    float bd = hd;
    int bi = hidx, bl = lane;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float od = __shfl_xor_sync(0xffffffffu, bd, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      const int ol = __shfl_xor_sync(0xffffffffu, bl, o);
      if (od < bd || (od == bd && (oi < bi || (oi == bi && ol < bl)))) {
        bd = od;
        bi = oi;
        bl = ol;
      }
    }
    if (lane == bl) ++cur;
    if (lane == 0) {
      idx[(size_t)t * k + r] = bi == INT_MAX ? -1 : bi;
      dist[(size_t)t * k + r] = bd;
      sum += (double)bd;
    }
  }
  if (lane == 0) score[t] = (float)(sum / (double)k);
}

// One warp per trajectory row: the exact top-k of the union of the row's candidate
// lists from the parts of a split series ([nparts][M][k], each sorted by (distance,
// index), index -1 = empty). Every unordered pair was evaluated by exactly one part,
// so the lists are disjoint; lane p walks list p and k rounds of a warp arg-min on
// (distance, index) take the smallest. The score is the FP64 mean (Eq. 3).
__global__ void merge_parts_kernel(const int32_t* __restrict__ pidx,
                                   const float* __restrict__ pdist, int P, int M, int k,
                                   int32_t* __restrict__ idx, float* __restrict__ dist,
                                   float* __restrict__ score) {
  const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (t >= M) return;
  const size_t base = ((size_t)lane * M + t) * k;
  int cur = 0;
  double sum = 0.0;
  for (int r = 0; r < k; ++r) {
    float hd = CUDART_INF_F;
    int hidx = INT_MAX;
    if (lane < P && cur < k) {
      const int ii = pidx[base + cur];
      if (ii >= 0) {
        hd = pdist[base + cur];
        hidx = ii;
      }
    }
    float bd = hd;
    int bi = hidx, bl = lane;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float od = __shfl_xor_sync(0xffffffffu, bd, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      const int ol = __shfl_xor_sync(0xffffffffu, bl, o);
      if (od < bd || (od == bd && (oi < bi || (oi == bi && ol < bl)))) {
        bd = od;
        bi = oi;
        bl = ol;
      }
    }
    if (lane == bl) ++cur;
    if (lane == 0) {
      idx[(size_t)t * k + r] = bi == INT_MAX ? -1 : bi;
      dist[(size_t)t * k + r] = bd;
      sum += (double)bd;
    }
  }
  if (lane == 0) score[t] = (float)(sum / (double)k);
}

constexpr int kMergeWarps = 8;
constexpr int kMergeCap = 256;

// Bits [lo, hi) of a 32-bit word (empty when hi <= lo).
__device__ __forceinline__ uint32_t bit_range32(int lo, int hi) {
  lo = max(lo, 0);
  hi = min(hi, 32);
  if (hi <= lo) return 0u;
  const uint32_t w = (hi - lo >= 32) ? 0xffffffffu : ((1u << (hi - lo)) - 1u);
  return w << lo;
}

__device__ __forceinline__ bool key_less(float d1, int i1, float d2, int i2) {
  return d1 < d2 || (d1 == d2 && i1 < i2);
}

// One warp per trajectory row of the tensor-core path. Every true neighbour of
// row t has a distance <= thr[t] (an upper bound of its k-th distance taken from
// some complete candidate list), so the candidates at or below the bound are
// gathered from the row's partial lists and, with the symmetric work split,
// from the column lists of the strips above; k rounds of a warp arg-min on
// (distance, index) then give the exact neighbour set in order. If the gathered
// set overflows the buffer, the rounds scan the lists directly.
__global__ void __launch_bounds__(32 * kMergeWarps)
    merge_tc_kernel(const float* __restrict__ part_d, const int32_t* __restrict__ part_i,
                    int out_rows, TcWork w, const __grid_constant__ SeriesTable st, int* err) {
  __shared__ float bd[kMergeWarps][kMergeCap];
  __shared__ int bi[kMergeWarps][kMergeCap];
  __shared__ int bn[kMergeWarps];
  __shared__ float sorted_d[kMergeWarps][kMaxK];  // the row's k distances in order
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r = blockIdx.x * kMergeWarps + wid;
  if (r >= out_rows) return;
  const int sidx = find_series(st.s, st.n, r, true);
  const SeriesInfo& si = st.s[sidx];
  const int t = r - si.out_base;
  if (t >= si.M) return;
  const int k = si.k, ks = w.kstride;
  const long long cp = col_pitch(ks);  // ints per column-list record
  const int strip = t / si.rows_out;
  float thr = __uint_as_float(w.thr[r]);
  const int c_lo = w.slot_lo[si.strip_base + strip];
  const long long plist = si.part_base + (long long)t * si.slots;  // first row-side list
  auto collist = [&](int s2) {
    return si.col_base + w.col_off[si.strip_base + s2] + (t - (s2 + 1) * si.rows_out);
  };
  auto push = [&](float d, int i) {
    const int pos = atomicAdd(&bn[wid], 1);
    if (pos < kMergeCap) {
      bd[wid][pos] = d;
      bi[wid][pos] = i;
    }
  };
  // The k smallest (distance, index) keys among the n <= kMergeCap buffered
  // candidates (distinct keys): a binary search on the distance bits (distances are
  // >= 0, so their bit patterns order like the values) finds the k-th distance T;
  // among candidates tied at T the smallest indices are taken (a second search on the
  // index, only when there are more ties than places). Returns T; with `out` the k
  // keys are written to the row's outputs in (distance, index) order (index -1,
  // distance +inf for missing ones) with the FP64 mean of the k distances, summed in
  // that order.
  auto select_k = [&](int n, bool out) -> float {
    constexpr int kPer = kMergeCap / 32;
    unsigned db[kPer];
    int ib[kPer];
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int q = lane + 32 * u;
      db[u] = q < n ? (__float_as_uint(bd[wid][q]) & 0x7FFFFFFFu) : 0xFFFFFFFFu;
      ib[u] = q < n ? bi[wid][q] : INT_MAX;
    }
    auto count_le = [&](unsigned x) {
      unsigned c = 0;
#pragma unroll
      for (int u = 0; u < kPer; ++u) c += db[u] <= x ? 1u : 0u;
      return (int)__reduce_add_sync(0xffffffffu, c);
    };
    const unsigned kInf = 0x7F800000u;
    const int kk = min(k, count_le(kInf));  // candidates with a distance (not NaN)
    unsigned T = kInf;
    int I = INT_MAX;
    if (kk > 0) {
      unsigned lo = 0, hi = kInf;
      while (lo < hi) {
        const unsigned mid = lo + ((hi - lo) >> 1);
        if (count_le(mid) >= kk) hi = mid;
        else lo = mid + 1;
      }
      T = lo;
      const int less = T > 0 ? count_le(T - 1) : 0;
      const int need = kk - less;  // places for candidates at distance T (>= 1)
      unsigned ceq = 0;
#pragma unroll
      for (int u = 0; u < kPer; ++u) ceq += db[u] == T ? 1u : 0u;
      if ((int)__reduce_add_sync(0xffffffffu, ceq) > need) {
        int lo2 = 0, hi2 = INT_MAX;
        while (lo2 < hi2) {
          const int mid = lo2 + ((hi2 - lo2) >> 1);
          unsigned c = 0;
#pragma unroll
          for (int u = 0; u < kPer; ++u) c += (db[u] == T && ib[u] <= mid) ? 1u : 0u;
          if ((int)__reduce_add_sync(0xffffffffu, c) >= need) hi2 = mid;
          else lo2 = mid + 1;
        }
        I = lo2;
      }
    }
    if (!out) return __uint_as_float(T);
    // compact the selected keys to the front of the buffer, then place each by rank
    float dv[kPer];
#pragma unroll
    for (int u = 0; u < kPer; ++u) dv[u] = lane + 32 * u < n ? bd[wid][lane + 32 * u] : 0.f;
    __syncwarp();
    int base = 0;
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const bool sel = kk > 0 && (db[u] < T || (db[u] == T && ib[u] <= I));
      const unsigned m = __ballot_sync(0xffffffffu, sel);
      if (sel) {
        const int q = base + __popc(m & ((1u << lane) - 1u));
        bd[wid][q] = dv[u];
        bi[wid][q] = ib[u];
      }
      base += __popc(m);
    }
    __syncwarp();
    for (int e = lane; e < k; e += 32) {
      if (e < kk) {
        const float de = bd[wid][e];
        const int ie = bi[wid][e];
        int rank = 0;
        for (int j = 0; j < kk; ++j) rank += key_less(bd[wid][j], bi[wid][j], de, ie) ? 1 : 0;
        si.idx[(size_t)t * k + rank] = ie;
        si.dist[(size_t)t * k + rank] = de;
        sorted_d[wid][rank] = de;
      } else {
        si.idx[(size_t)t * k + e] = -1;
        si.dist[(size_t)t * k + e] = CUDART_INF_F;
        sorted_d[wid][e] = CUDART_INF_F;
      }
    }
    __syncwarp();
    if (lane == 0) {
      double sum = 0.0;
      for (int e = 0; e < k; ++e) sum += (double)sorted_d[wid][e];
      si.score[t] = (float)(sum / (double)k);
    }
    return __uint_as_float(T);
  };
  // with a split series only the lists of this call's strips exist
  const bool own = strip >= w.part_lo && strip < w.part_hi;
  const int s2_lo = w.part_lo, s2_hi = min(strip, w.part_hi);
  const int c_hi = own ? si.slots : c_lo;
  int n = 0;
  for (int pass = 0; pass < 64; ++pass) {
    if (lane == 0) bn[wid] = 0;
    __syncwarp();
    // lists are read four entries at a time (the list pitch ks is a multiple of 4)
    for (int c = c_lo + lane; c < c_hi; c += 32) {
      const size_t b = (size_t)(plist + c) * ks;
      if (!tk_in((long long)b + ks - 1, w.part_ints, err)) continue;
      const float4* d4 = reinterpret_cast<const float4*>(part_d + b);
      const int4* i4 = reinterpret_cast<const int4*>(part_i + b);
      bool more = true;
      for (int p = 0; more && p < k; p += 4) {
        const float4 dv = __ldg(d4 + p / 4);
        const int4 iv = __ldg(i4 + p / 4);
        const float dd[4] = {dv.x, dv.y, dv.z, dv.w};
        const int ii[4] = {iv.x, iv.y, iv.z, iv.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (!more || p + u >= k) break;
          if (ii[u] < 0 || dd[u] > thr) {
            more = false;  // sorted: nothing further qualifies
          } else {
            push(dd[u], ii[u]);
          }
        }
      }
    }
    if (w.sym) {
      // column lists (not sorted) from the strips above this row: only the non-empty
      // ones (their bit set in the row's mask) have a record. The set bits are numbered
      // across the mask words (a prefix sum over the lanes' words), each lane takes one
      // per round, and reads the first 32 bytes of its record (two loads in flight
      // together): the count and three entries
      const long long mrow = (long long)r * w.mask_words;
      const long long mlim = (long long)out_rows * w.mask_words;
      for (int wb0 = 0; wb0 < w.mask_words; wb0 += 32) {
        const int wb = wb0 + lane;
        uint32_t m = 0;
        if (wb < w.mask_words && tk_in(mrow + wb, mlim, err))
          m = __ldg(w.col_mask + mrow + wb) & bit_range32(s2_lo - 32 * wb, s2_hi - 32 * wb);
        const int pc = __popc(m);
        int incl = pc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int v = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += v;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        const int excl = incl - pc;
        for (int e0 = 0; e0 < total; e0 += 32) {
          const int e = e0 + lane;
          // the word holding set bit e: the last lane whose prefix is <= e
          int wl = 0;
#pragma unroll
          for (int step = 16; step > 0; step >>= 1) {
            const int x = __shfl_sync(0xffffffffu, excl, wl + step);
            if (x <= e) wl += step;
          }
          const uint32_t mw = __shfl_sync(0xffffffffu, m, wl);
          const int want = e - __shfl_sync(0xffffffffu, excl, wl);  // rank within the word
          if (e >= total) continue;
          int b0 = 0;  // the want-th set bit of mw: smallest b with popc(mw & bits 0..b) > want
#pragma unroll
          for (int step = 16; step > 0; step >>= 1)
            if (__popc(mw & (0xFFFFFFFFu >> (31 - (b0 + step - 1)))) <= want) b0 += step;
          const int s2 = 32 * (wb0 + wl) + b0;
          const long long ri =
              tk_in(collist(s2) * cp + cp - 1, w.col_ints, err) ? collist(s2) * cp : -1;
          if (ri < 0) continue;
          const int4* r4 = reinterpret_cast<const int4*>(w.col_rec + ri);
          const int4 h0 = __ldg(r4), h1 = __ldg(r4 + 1);
          const int nn = tk_in(h0.x, ks + 1, err) ? h0.x : 0;  // count <= k
          if (nn > 0 && __int_as_float(h0.w) <= thr) push(__int_as_float(h0.w), h0.z);
          if (nn > 1 && __int_as_float(h1.y) <= thr) push(__int_as_float(h1.y), h1.x);
          if (nn > 2 && __int_as_float(h1.w) <= thr) push(__int_as_float(h1.w), h1.z);
          for (int p = 3; p < nn; ++p) {
            const int2 en = __ldg(reinterpret_cast<const int2*>(w.col_rec + ri) + 1 + p);
            if (__int_as_float(en.y) <= thr) push(__int_as_float(en.y), en.x);
          }
        }
      }
    }
    __syncwarp();
    n = bn[wid];
    __syncwarp();
    if (n <= kMergeCap) break;
    // overflow: the k-th smallest of the buffered (valid, distinct) candidates is a
    // tighter bound; gather again under it
    thr = select_k(kMergeCap, false);
  }
  // final selection, written in (distance, index) order; if ties at the bound keep
  // the candidate set larger than the buffer, scan the lists directly each round
  const bool direct = n > kMergeCap;
  if (!direct) {
    select_k(n, true);
    return;
  }
  float last_d = -CUDART_INF_F;
  int last_i = -1;
  double sum = 0.0;
  for (int rr = 0; rr < k; ++rr) {
    float best_d = CUDART_INF_F;
    int best_i = INT_MAX;
    auto consider = [&](float d, int ii) {
      if (key_less(last_d, last_i, d, ii) && key_less(d, ii, best_d, best_i)) {
        best_d = d;
        best_i = ii;
      }
    };
    if (!direct) {
      for (int q = lane; q < n; q += 32) consider(bd[wid][q], bi[wid][q]);
    } else {
      for (int c = c_lo + lane; c < c_hi; c += 32) {
        const size_t b = (size_t)(plist + c) * ks;
        if (!tk_in((long long)b + ks - 1, w.part_ints, err)) continue;
        for (int p = 0; p < k; ++p) {
          const int ii = part_i[b + p];
          if (ii < 0 || part_d[b + p] > thr) break;
          consider(part_d[b + p], ii);
        }
      }
      if (w.sym) {
        for (int s2 = s2_lo + lane; s2 < s2_hi; s2 += 32) {
          const long long mi = (long long)r * w.mask_words + (s2 >> 5);
          if (!tk_in(mi, (long long)out_rows * w.mask_words, err) ||
              !((__ldg(w.col_mask + mi) >> (s2 & 31)) & 1u))
            continue;  // an empty list has no record
          if (!tk_in(collist(s2) * cp + cp - 1, w.col_ints, err)) continue;
          const int2* rec = reinterpret_cast<const int2*>(w.col_rec + collist(s2) * cp);
          const int nn = tk_in(rec[0].x, ks + 1, err) ? rec[0].x : 0;
          for (int p = 0; p < nn; ++p) {
            const int2 e = rec[1 + p];
            if (__int_as_float(e.y) <= thr) consider(__int_as_float(e.y), e.x);
          }
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float od2 = __shfl_xor_sync(0xffffffffu, best_d, o);
      const int oi = __shfl_xor_sync(0xffffffffu, best_i, o);
      if (key_less(od2, oi, best_d, best_i)) {
        best_d = od2;
        best_i = oi;
      }
    }
    last_d = best_d;
    last_i = best_i;
    if (lane == 0) {
      si.idx[(size_t)t * k + rr] = best_i == INT_MAX ? -1 : best_i;
      si.dist[(size_t)t * k + rr] = best_d;
      sum += (double)best_d;
    }
  }
  if (lane == 0) si.score[t] = (float)(sum / (double)k);
}

}  // namespace

cudaError_t launch_merge_tc(const TcArgs& a, const TcWork& w, const SeriesTable& sr,
                            cudaStream_t st) {
  const int blocks = (a.out_rows + kMergeWarps - 1) / kMergeWarps;
  merge_tc_kernel<<<blocks, 32 * kMergeWarps, 0, st>>>(a.part_d, a.part_i, a.out_rows, w, sr,
                                                        a.err);
  return cudaGetLastError();
}

cudaError_t launch_merge_parts(const int32_t* idx_parts, const float* dist_parts, int nparts,
                               int M, int k, int32_t* idx, float* dist, float* score,
                               cudaStream_t st) {
  if (nparts < 1 || nparts > 32) return cudaErrorInvalidValue;
  const int blocks = (M + kMergeWarps - 1) / kMergeWarps;
  merge_parts_kernel<<<blocks, 32 * kMergeWarps, 0, st>>>(idx_parts, dist_parts, nparts, M, k,
                                                          idx, dist, score);
  return cudaGetLastError();
}

cudaError_t launch_col_mean_series(const SeriesTable& sr, int D, float* partial, float* mu,
                                   bool center, cudaStream_t st) {
  if (center) {
    dim3 grid((D + 255) / 256, kMeanSlices, sr.n);
    col_partial_series_kernel<<<grid, 256, 0, st>>>(sr, D, partial);
  }
  dim3 g2((D + 255) / 256, sr.n);
  col_final_series_kernel<<<g2, 256, 0, st>>>(sr, partial, D, mu, center ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_prep_split_series(const SeriesTable& sr, int rows, int D, int emb, int groups,
                                     bool correct, const float* mu, const float* wts, void* hi,
                                     void* lo, double* norms, float* cval, cudaStream_t st,
                                     int r_lo) {
  if (rows <= r_lo) return cudaSuccess;
  __nv_bfloat16* h = static_cast<__nv_bfloat16*>(hi);
  __nv_bfloat16* l = static_cast<__nv_bfloat16*>(lo);
  if (groups <= 16) {
    // few groups per row: several rows per warp
    const int per_block = 8 * (32 / groups);
    const int nb = (rows - r_lo + per_block - 1) / per_block;
    if (correct)
      prep_split_small_kernel<true><<<nb, 256, 0, st>>>(sr, r_lo, rows, D, emb, groups, mu, wts,
                                                        h, l, norms, cval);
    else
      prep_split_small_kernel<false><<<nb, 256, 0, st>>>(sr, r_lo, rows, D, emb, groups, mu, wts,
                                                         h, l, norms, cval);
    return cudaGetLastError();
  }
  const int blocks = (rows - r_lo + 7) / 8;
  // the embedded form (values of several days per row) maps a value to its grid point
  // by a division; the plain form needs none
  if (correct && emb > 1)
    prep_split_series_kernel<true, true><<<blocks, 256, 0, st>>>(sr, r_lo, rows, D, emb, groups,
                                                                 mu, wts, h, l, norms, cval);
  else if (correct)
    prep_split_series_kernel<true, false><<<blocks, 256, 0, st>>>(sr, r_lo, rows, D, emb, groups,
                                                                  mu, wts, h, l, norms, cval);
  else if (emb > 1)
    prep_split_series_kernel<false, true><<<blocks, 256, 0, st>>>(sr, r_lo, rows, D, emb, groups,
                                                                  mu, wts, h, l, norms, cval);
  else
    prep_split_series_kernel<false, false><<<blocks, 256, 0, st>>>(sr, r_lo, rows, D, emb,
                                                                   groups, mu, wts, h, l, norms,
                                                                   cval);
  return cudaGetLastError();
}

cudaError_t launch_window_series(const SeriesTable& sr, int out_rows, const double* norms,
                                 float* W, cudaStream_t st, int r_lo) {
  if (out_rows <= r_lo) return cudaSuccess;
  window_series_kernel<<<(out_rows - r_lo + 255) / 256, 256, 0, st>>>(sr, r_lo, out_rows, norms,
                                                                     W);
  return cudaGetLastError();
}

cudaError_t launch_col_mean(const float* X, int N, int D, float* partial, float* mu, bool center,
                            cudaStream_t st) {
  dim3 grid((D + 255) / 256, kMeanSlices);
  if (center) col_partial_kernel<<<grid, 256, 0, st>>>(X, N, D, partial);
  col_final_kernel<<<(D + 255) / 256, 256, 0, st>>>(partial, N, D, mu, center ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_prep_fp32(const float* X, int N, int D, int Dp, const float* mu,
                             const float* wts, float* Xc, double* norms, cudaStream_t st) {
  prep_fp32_kernel<<<N, 256, 0, st>>>(X, D, Dp, mu, wts, Xc, norms);
  return cudaGetLastError();
}

cudaError_t launch_window(const double* norms, int M, int L, float* W, cudaStream_t st) {
  window_kernel<<<(M + 255) / 256, 256, 0, st>>>(norms, M, L, W);
  return cudaGetLastError();
}

cudaError_t launch_merge(const FusedArgs& a, int32_t* idx, float* dist, float* score,
                         cudaStream_t st) {
  const int warps_per_block = 8;
  const int blocks = (a.sch.M + warps_per_block - 1) / warps_per_block;
  merge_kernel<<<blocks, 32 * warps_per_block, 0, st>>>(a.part_d, a.part_i, a.sch.M,
                                                        a.sch.chunks, a.sch.k, idx, dist, score);
  return cudaGetLastError();
}

// ----------------------------------------------------------- kNN statistics

namespace {

// One thread per row of sorted squared distances dist[M][k]:
//   prefix[t][k'-1] = (1/k') sum_{j<k'} dist[t][j], k' = 1..k   (Eq. 3 at every k' <= k;
//                     the neighbour sets are nested in k, Sec. 6)
//   local_id[t]     = [ (1/(k_id-1)) sum_{j<k_id-1} log(T_{k_id} / T_j) ]^(-1), T = sqrt(dist)
//                     (maximum-likelihood kNN estimator of Levina and Bickel, as used in the
//                     intrinsic dimension study of Sec. 4); NaN when a distance among the
//                     first k_id is zero or all of them are equal.
// Sums are FP64 (the mean's final division and the logarithm of each distance ratio
// are FP32). A block
// stages its 128 rows through shared memory so that global loads and stores are
// coalesced (row pitch k + 1 avoids bank conflicts).
constexpr int kStatRows = 128;

__global__ void __launch_bounds__(kStatRows)
    knn_stats_kernel(const float* __restrict__ dist, int M, int k, float* __restrict__ prefix,
                     int k_id, float* __restrict__ lid) {
  extern __shared__ float tile[];  // [kStatRows][k + 1]
  const int r0 = blockIdx.x * kStatRows;
  const int rows = min(kStatRows, M - r0);
  const int pitch = k + 1;
  for (int i = threadIdx.x; i < rows * k; i += kStatRows)
    tile[(i / k) * pitch + i % k] = dist[(size_t)r0 * k + i];
  __syncthreads();
  const int r = threadIdx.x;
  float* d = tile + r * pitch;
  float out_id = CUDART_NAN_F;
  if (r < rows && lid) {
    if (d[0] > 0.f) {
      double s = 0.0;
      for (int j = 0; j < k_id - 1; ++j) s += 0.5 * (double)logf(d[k_id - 1] / d[j]);
      if (s > 0.0) out_id = (float)((double)(k_id - 1) / s);
    }
  }
  if (r < rows && prefix) {
    double s = 0.0;
    for (int j = 0; j < k; ++j) {
      s += (double)d[j];
      d[j] = (float)s / (float)(j + 1);  // in place: d[j] is not read again
    }
  }
  __syncthreads();
  if (prefix)
    for (int i = threadIdx.x; i < rows * k; i += kStatRows)
      prefix[(size_t)r0 * k + i] = tile[(i / k) * pitch + i % k];
  if (lid && r < rows) lid[r0 + r] = out_id;
}

}  // namespace

cudaError_t launch_knn_stats(const float* dist, int M, int k, float* prefix, int k_id,
                             float* local_id, cudaStream_t st) {
  if (M < 1) return cudaSuccess;
  const size_t smem = (size_t)kStatRows * (k + 1) * sizeof(float);
  knn_stats_kernel<<<(M + kStatRows - 1) / kStatRows, kStatRows, smem, st>>>(dist, M, k, prefix,
                                                                             k_id, local_id);
  return cudaGetLastError();
}

}  // namespace traknn
