// kernels_aux.cu -- the light kernels around the fused Gram/top-k kernels:
//   column means (optional centring, exact by the offset invariance of Eq. 2),
//   operand preparation with FP64 day norms (Algorithm 1, norm precomputation),
//   window sums of the norms, and the final merge of partial neighbour lists
//   into sorted neighbour sets and rarity scores (Eq. 3).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math_constants.h>

#include <climits>

#include "internal.h"

namespace traknn {
namespace {

// Column sums over fixed row slices (fixed summation order: deterministic).
__global__ void col_partial_kernel(const float* __restrict__ X, int N, int D, float* partial) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= D) return;
  const int per = (N + kMeanSlices - 1) / kMeanSlices;
  const int r0 = blockIdx.y * per, r1 = min(N, r0 + per);
  float acc = 0.f;
  for (int a = r0; a < r1; ++a) acc += X[(size_t)a * D + p];
  partial[(size_t)blockIdx.y * D + p] = acc;
}

// The centring offset only needs to be one fixed field subtracted from every
// day (any value keeps Eq. 2 exact), so FP32 sums suffice here.
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
  mu[p] = acc / (float)N;
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
                                 const float* __restrict__ mu, float* __restrict__ Xc,
                                 double* __restrict__ norms) {
  __shared__ double red[32];
  const int a = blockIdx.x;
  const float* x = X + (size_t)a * D;
  float* y = Xc + (size_t)a * Dp;
  double acc = 0.0;
  for (int p = threadIdx.x; p < Dp; p += blockDim.x) {
    const float v = p < D ? x[p] - mu[p] : 0.f;
    y[p] = v;
    acc = fma((double)v, (double)v, acc);
  }
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) norms[a] = s;
}

// One block per day: x - mu = hi + lo with hi = bf16(x - mu), lo = bf16(x - mu - hi),
// written as two BF16 copies (row pitch Dp, zero padded). The norm is taken of
// the centred FP32 value.
__global__ void prep_split_kernel(const float* __restrict__ X, int D, int Dp,
                                  const float* __restrict__ mu, __nv_bfloat16* __restrict__ hi,
                                  __nv_bfloat16* __restrict__ lo, double* __restrict__ norms) {
  __shared__ double red[32];
  const int a = blockIdx.x;
  const float* x = X + (size_t)a * D;
  double acc = 0.0;
  for (int p = threadIdx.x; p < Dp; p += blockDim.x) {
    const float v = p < D ? x[p] - mu[p] : 0.f;
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
    hi[(size_t)a * Dp + p] = h;
    lo[(size_t)a * Dp + p] = l;
    acc = fma((double)v, (double)v, acc);
  }
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) norms[a] = s;
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

}  // namespace

cudaError_t launch_col_mean(const float* X, int N, int D, float* partial, float* mu, bool center,
                            cudaStream_t st) {
  dim3 grid((D + 255) / 256, kMeanSlices);
  if (center) col_partial_kernel<<<grid, 256, 0, st>>>(X, N, D, partial);
  col_final_kernel<<<(D + 255) / 256, 256, 0, st>>>(partial, N, D, mu, center ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_prep_fp32(const float* X, int N, int D, int Dp, const float* mu, float* Xc,
                             double* norms, cudaStream_t st) {
  prep_fp32_kernel<<<N, 256, 0, st>>>(X, D, Dp, mu, Xc, norms);
  return cudaGetLastError();
}

cudaError_t launch_prep_split(const float* X, int N, int D, int Dp, const float* mu, void* hi,
                              void* lo, double* norms, cudaStream_t st) {
  prep_split_kernel<<<N, 256, 0, st>>>(X, D, Dp, mu, static_cast<__nv_bfloat16*>(hi),
                                       static_cast<__nv_bfloat16*>(lo), norms);
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

}  // namespace traknn
