// kernel_fp32.cu -- the plain FP32 path: CUDA-core FMA Gram tiles (Algorithm 1,
// "Symmetric Batched GeMM") fused with the trajectory-distance window, the
// exclusion mask and the per-row top-k (Algorithm 1, kNN step). The N x N
// snapshot matrix never leaves the chip.
//
// One persistent CTA per SM walks units (row strip x column chunk). For every
// 128 x 128 tile of G it runs a register-blocked SGEMM over the padded,
// mean-centred FP32 copy of X, stores the tile beside the L-1 Gram columns
// carried from the previous tile, and lets one thread per output row scan its
// 128 output columns.
#include <cuda_runtime.h>
#include <math_constants.h>

#include "epilogue.cuh"
#include "internal.h"

namespace traknn {
namespace {

constexpr int BM = kTileRows;  // Gram rows per tile
constexpr int BN = 128;        // Gram columns per tile
constexpr int BK = 16;         // depth of one shared-memory stage
constexpr int NT = 256;        // threads
constexpr int LDA = BM + 4;
constexpr int LDG = kHalo + BN + 1;  // odd row pitch: conflict-free diagonal reads

struct Smem {
  float As[2][BK][LDA];
  float Bs[2][BK][LDA];
  float G[BM][LDG];
};

__device__ __forceinline__ void load_stage(const float* __restrict__ Xc, int N, int Dp, int r0,
                                           int c0, int k0, int tid, float4 (&ra)[2],
                                           float4 (&rb)[2]) {
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int f = tid + q * NT;
    const int r = f >> 2, k4 = f & 3;
    const int ga = r0 + r, gb = c0 + r;
    ra[q] = ga < N ? __ldg(reinterpret_cast<const float4*>(Xc + (size_t)ga * Dp + k0) + k4)
                   : make_float4(0.f, 0.f, 0.f, 0.f);
    rb[q] = gb < N ? __ldg(reinterpret_cast<const float4*>(Xc + (size_t)gb * Dp + k0) + k4)
                   : make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

__device__ __forceinline__ void store_stage(Smem& sm, int buf, int tid, const float4 (&ra)[2],
                                            const float4 (&rb)[2]) {
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int f = tid + q * NT;
    const int r = f >> 2, k4 = f & 3;
    sm.As[buf][4 * k4 + 0][r] = ra[q].x;
    sm.As[buf][4 * k4 + 1][r] = ra[q].y;
    sm.As[buf][4 * k4 + 2][r] = ra[q].z;
    sm.As[buf][4 * k4 + 3][r] = ra[q].w;
    sm.Bs[buf][4 * k4 + 0][r] = rb[q].x;
    sm.Bs[buf][4 * k4 + 1][r] = rb[q].y;
    sm.Bs[buf][4 * k4 + 2][r] = rb[q].z;
    sm.Bs[buf][4 * k4 + 3][r] = rb[q].w;
  }
}

// G tile rows [r0, r0+128) x columns [c0, c0+128) into sm.G[.][kHalo + .].
// Products are summed in partial sums of about sqrt(Dp) terms (whole stages) that
// then join the running sum: the rounding error of the two FP32 chains grows like
// sqrt(chain length), and two chains of about sqrt(Dp) terms each keep it smallest.
__device__ __forceinline__ void gram_tile(Smem& sm, const float* __restrict__ Xc, int N, int Dp,
                                          int r0, int c0, int tid) {
  const int tx = tid & 15, ty = tid >> 4;
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

  float4 ra[2], rb[2];
  const int nk = Dp / BK;
  const int flush = max(1, (int)(sqrtf((float)Dp) / BK + 0.5f));  // stages per partial sum
  float part[8][8];
  load_stage(Xc, N, Dp, r0, c0, 0, tid, ra, rb);
  __syncthreads();  // previous users of As/Bs and G are done
  store_stage(sm, 0, tid, ra, rb);
  __syncthreads();
  for (int kt = 0; kt < nk; ++kt) {
    const int cur = kt & 1;
    if (kt + 1 < nk) load_stage(Xc, N, Dp, r0, c0, (kt + 1) * BK, tid, ra, rb);
    if (kt % flush == 0) {
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) part[i][j] = 0.f;
    }
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&sm.As[cur][kk][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&sm.As[cur][kk][64 + ty * 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&sm.Bs[cur][kk][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4*>(&sm.Bs[cur][kk][64 + tx * 4]);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) part[i][j] = fmaf(av[i], bv[j], part[i][j]);
    }
    if ((kt + 1) % flush == 0 || kt + 1 == nk) {
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] += part[i][j];
    }
    if (kt + 1 < nk) store_stage(sm, cur ^ 1, tid, ra, rb);
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int r = (i < 4) ? ty * 4 + i : 64 + ty * 4 + (i - 4);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int c = (j < 4) ? tx * 4 + j : 64 + tx * 4 + (j - 4);
      sm.G[r][kHalo + c] = acc[i][j];
    }
  }
  __syncthreads();
}

__global__ void __launch_bounds__(NT, 1)
    fused_fp32_kernel(const float* __restrict__ Xc, FusedArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem& sm = *reinterpret_cast<Smem*>(smem_raw);
  const Schedule& s = a.sch;
  SmemList list;
  list.d = reinterpret_cast<float*>(smem_raw + sizeof(Smem));
  list.i = reinterpret_cast<int32_t*>(list.d + BM * s.k);
  list.stride = BM;
  list.k = s.k;

  const int tid = threadIdx.x;
  const int L = s.L;
  for (int u = blockIdx.x; u < s.units; u += gridDim.x) {
    const UnitCoord uc = unit_coord(s, u);
    if (uc.strip >= s.strips) continue;
    RowCtx rc;
    rc.L = L;
    rc.e = s.e;
    rc.jlo = uc.chunk * s.chunk_cols;
    rc.jhi = min(s.M, rc.jlo + s.chunk_cols);
    if (rc.jlo >= rc.jhi) continue;
    const int T0 = uc.strip * s.rows_out;
    rc.lrow = tid;
    rc.t = T0 + tid;
    const bool row_ok = tid < s.rows_out && rc.t < s.M;
    rc.Wt = row_ok ? a.W[rc.t] : 0.f;
    float thr = CUDART_INF_F;
    if (tid < BM) list.reset(tid);

    const int ntiles = (rc.jhi - rc.jlo + L - 1 + BN - 1) / BN;
    for (int it = 0; it < ntiles; ++it) {
      const int c0 = rc.jlo + it * BN;  // first Gram column of the tile
      gram_tile(sm, Xc, a.N, a.Dp, T0, c0, tid);
      // output column x of this tile is j = c0 - (L-1) + x; its window starts in
      // the carried columns, which sit just left of kHalo
      if (row_ok)
        window_topk(&sm.G[0][kHalo - (L - 1)], LDG, rc, it == 0 ? L - 1 : 0, BN,
                    c0 - (L - 1), a.W, list, tid, thr);
      __syncthreads();
      for (int q = tid; q < BM * (L - 1); q += NT) {
        const int r = q / (L - 1), c = q - r * (L - 1);
        sm.G[r][kHalo - (L - 1) + c] = sm.G[r][kHalo + BN - (L - 1) + c];
      }
    }
    if (row_ok) {
      const size_t base = ((size_t)rc.t * s.chunks + uc.chunk) * s.k;
      for (int p = 0; p < s.k; ++p) {
        a.part_d[base + p] = list.d[p * BM + tid];
        a.part_i[base + p] = list.i[p * BM + tid];
      }
    }
  }
}

}  // namespace

size_t fused_fp32_smem_bytes(int k) { return sizeof(Smem) + (size_t)BM * k * 8; }

cudaError_t launch_fused_fp32(const float* Xc, const FusedArgs& a, int num_ctas,
                              cudaStream_t st) {
  const size_t smem = fused_fp32_smem_bytes(a.sch.k);
  cudaError_t err = cudaFuncSetAttribute(fused_fp32_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  fused_fp32_kernel<<<num_ctas, NT, smem, st>>>(Xc, a);
  return cudaGetLastError();
}

}  // namespace traknn
