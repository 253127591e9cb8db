// epilogue.cuh -- per-row work that turns a tile of the snapshot Gram matrix into
// trajectory distances and keeps each row's k nearest candidates, as used by the
// FP32 CUDA-core kernel (the tensor-core kernel has its own register-based scan).
//
// With day norms n_a = ||X_a||^2 and window sums W_t = sum_{m<L} n_{t+m}, the
// trajectory distance of Eq. 2 expands (Eq. 4 applied to every day pair) into
//     D(t,j) = W_t + W_j - 2 sum_{m<L} G(t+m, j+m),   G(a,b) = <X_a, X_b>.
// The sum runs down one diagonal of G. It is evaluated explicitly, L terms per
// output, from Gram values held on chip (the current tile plus the last L-1
// columns carried over from the previous tile of the same row strip), so there
// is no running add/subtract chain and no drift however long the diagonal is.
#pragma once

#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

namespace traknn {

// A sorted (ascending distance) list of k candidates per owning thread, kept in
// shared memory as [k][stride] so that consecutive threads use consecutive banks.
// Empty slots hold (+inf, -1).
struct SmemList {
  float* d;
  int32_t* i;
  int stride;
  int k;

  __device__ __forceinline__ void reset(int tid) const {
    for (int p = 0; p < k; ++p) {
      d[p * stride + tid] = CUDART_INF_F;
      i[p * stride + tid] = -1;
    }
  }

  __device__ __forceinline__ float threshold(int tid) const { return d[(k - 1) * stride + tid]; }

  // Insert (dv, jv) with dv < threshold. Candidates reach a list in increasing
  // index order, so stopping at an equal distance keeps the smaller index first:
  // the list stays sorted by (distance, index) (Algorithm 1, kNN step).
  // Returns the new threshold (the k-th distance).
  __device__ __forceinline__ float insert(int tid, float dv, int32_t jv) const {
    int p = k - 1;
    while (p > 0) {
      float q = d[(p - 1) * stride + tid];
      if (!(q > dv)) break;
      d[p * stride + tid] = q;
      i[p * stride + tid] = i[(p - 1) * stride + tid];
      --p;
    }
    d[p * stride + tid] = dv;
    i[p * stride + tid] = jv;
    return d[(k - 1) * stride + tid];
  }

  // Insert (dv, jv) in (distance, index) order when candidates arrive in any
  // index order. Requires (dv, jv) to precede the current k-th entry.
  __device__ __forceinline__ float insert_key(int tid, float dv, int32_t jv) const {
    int p = k - 1;
    while (p > 0) {
      const float q = d[(p - 1) * stride + tid];
      const int32_t qi = i[(p - 1) * stride + tid];
      if (!(q > dv || (q == dv && qi > jv))) break;
      d[p * stride + tid] = q;
      i[p * stride + tid] = qi;
      --p;
    }
    d[p * stride + tid] = dv;
    i[p * stride + tid] = jv;
    return d[(k - 1) * stride + tid];
  }
};

struct RowCtx {
  int t;        // output trajectory row
  float Wt;     // window sum of row t
  int lrow;     // row of the G buffer holding day t
  int L, e;
  int jlo, jhi; // output columns owned by the current unit
};

// Output columns x in [x0, x1) of one tile for one row. `g` points at the G
// buffer column that holds Gram column j0 (the output column of x = 0); the
// window for output x reads g[(lrow+m)*ldg + x + m], m < L.
__device__ __forceinline__ void window_topk(const float* g, int ldg, const RowCtx& rc, int x0,
                                            int x1, int j0, const float* __restrict__ W,
                                            const SmemList& list, int tid, float& thr) {
  for (int x = x0; x < x1; ++x) {
    const int j = j0 + x;
    if (j < rc.jlo || j >= rc.jhi) continue;
    const int gap = rc.t > j ? rc.t - j : j - rc.t;
    if (gap <= rc.e) continue;
    const float* gp = g + rc.lrow * ldg + x;
    float c = gp[0];
    for (int m = 1; m < rc.L; ++m) c += gp[m * (ldg + 1)];
    const float dv = fmaxf(fmaf(-2.0f, c, rc.Wt + __ldg(W + j)), 0.0f);
    if (dv < thr) thr = list.insert(tid, dv, j);
  }
}

}  // namespace traknn
