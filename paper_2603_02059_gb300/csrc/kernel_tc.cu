// kernel_tc.cu -- the tensor-core path: tcgen05 Gram tiles fed by TMA (Algorithm 1,
// "Symmetric Batched GeMM", with the norm identity of Eq. 4), fused with the
// trajectory window of Eq. 2, the exclusion mask and the per-row top-k
// (Algorithm 1, kNN step). The N x N snapshot matrix never leaves the chip.
//
// Precision forms. BF16: G = <bf16(x_a), bf16(x_b)>. Split-BF16: every centred
// value is written as x = hi + lo with hi = bf16(x), lo = bf16(x - hi), and
//     G = <hi_a, hi_b> + <hi_a, lo_b> + <lo_a, hi_b>
// (the lo.lo term, about 2^-16 of |x_a||x_b|, is dropped), accumulated in FP32
// in tensor memory. The day norms and window sums stay FP64 (kernels_aux.cu).
//
// Operands are the grouped BF16 copies of the operand preparation (kernels_aux.cu):
// per 64 K entries, 63 permuted grid points and one correction entry that makes the
// accumulator hold G - groups c_a c_b (small for close pairs); the epilogue adds
// groups c_a c_b back in FP32.
//
// One persistent CTA per SM, warp-specialised:
//   warp 0   TMA producer: A (128 strip rows) and B (256 tile columns) K-chunks of
//            32 elements into a ring of shared-memory stages (hi and lo copies);
//   warp 1   tcgen05.mma issuer into one of two 128 x 256 FP32 accumulators in
//            TMEM (512 columns). The K range of a tile is cut into segments
//            (8192 elements by default); every segment accumulates afresh into
//            the next accumulator, so segment s+1 multiplies while segment s is
//            read out. With more than one segment per tile the epilogue adds every
//            segment but the last, in FP32 on the CUDA cores, into a running total
//            of the tile in a per-CTA scratch array (L2-resident), and adds the last
//            from TMEM while scanning: the tensor cores never accumulate more than
//            one segment of products per output, which bounds the error of their
//            accumulation however large D is;
//   warps 2-5 epilogue: each thread owns one accumulator row (TMEM lane), pulls
//            32 columns at a time with tcgen05.ld, stages them beside the L-1
//            columns carried from the previous chunk, sums each output's window
//            down the diagonal, masks the exclusion zone, and keeps the row's k
//            best in registers (row side). Beyond the strip's own block the same
//            distances are offered, transposed by warp ballots, to the columns'
//            lists (column side), so each unordered pair is evaluated once.
// Work units (a strip and a range of columns, or a band unit that only seeds the
// per-row bounds) are handed out dynamically; a unit may serve several series that
// share its Gram tiles (several trajectory lengths of one record).
// Every wait is bounded (globaltimer); a wait that runs out records a timeout
// in the status word, the CTA drains its own copies and MMAs, frees TMEM and
// returns.
#include <cuda.h>
#include <cuda_runtime.h>
#include <math_constants.h>

#include "internal.h"
#include "tc_ptx.cuh"

namespace traknn {
namespace {

constexpr int BM = kTileRows;  // accumulator rows (TMEM lanes)
constexpr int BN = kTileCols;  // accumulator columns per tile (256)
constexpr int KC = 32;         // K elements per stage (64 B rows, 64-B swizzle)
constexpr int kEpiThreads = 128;  // one epilogue group: one thread per accumulator row
// Threads of a CTA: warp 0 producer, warp 1 MMA issuer, G epilogue groups of four
// warps. With G = 2 (L = 1 only: no window, no carry) group g reads the columns
// [g 128, (g+1) 128) of every tile, so that twice as many warps hide the epilogue's
// latencies when it, not the contraction, sets the pace (small grids).
__host__ __device__ constexpr int kThreadsG(int G) { return 64 + kEpiThreads * G; }
// Pitch of the Gram chunk buffer: 32 columns plus the L-1 carried ones, made odd
// so that the diagonal reads of 32 consecutive rows hit 32 different banks.
__host__ __device__ constexpr int chunk_pitch(int L) {
  return 32 + (L - 1) + (((L - 1) % 2 == 0) ? 1 : 0);
}
constexpr uint32_t kTileA = BM * KC * 2;  // bytes of one A operand tile
constexpr uint32_t kTileB = BN * KC * 2;  // bytes of one B operand tile
constexpr uint32_t kIdesc = ptx::idesc_bf16_f32(BM, BN);
constexpr int kMaxStages = 8;
constexpr size_t kSmemLimit = 232448;  // 227 KB opt-in per block

// Sorted (ascending distance) list of the K best candidates of one row, held in
// registers. Candidates arrive in increasing index order, so the strict compare
// keeps an earlier (smaller) index ahead of an equal distance: the order is
// (distance, index) (Algorithm 1, kNN step). K may exceed k; the first k entries
// are then the row's k best.
template <int K>
struct RegList {
  float d[K];
  int32_t i[K];

  __device__ __forceinline__ void reset() {
#pragma unroll
    for (int p = 0; p < K; ++p) {
      d[p] = CUDART_INF_F;
      i[p] = -1;
    }
  }
  __device__ __forceinline__ float threshold() const { return d[K - 1]; }
  // Branch-free bubble: the list stays in registers (an early-exit form makes the
  // compiler move it to local memory).
  __device__ __forceinline__ void insert(float x, int32_t xi) {
#pragma unroll
    for (int p = 0; p < K; ++p) {
      const bool sw = x < d[p];
      const float td = d[p];
      const int32_t ti = i[p];
      d[p] = sw ? x : td;
      i[p] = sw ? xi : ti;
      x = sw ? td : x;
      xi = sw ? ti : xi;
    }
  }
};

// Shared memory of one epilogue group: Gram chunk with carried columns, W, row
// bounds and correction values of a tile, column-side row masks, column lists.
__host__ __device__ constexpr size_t group_bytes(int k, int L) {
  return (size_t)BM * chunk_pitch(L) * 4 + 3 * BN * 4 + 128 * 4 + (size_t)32 * k * 8;
}

// Bits [lo, hi) of a 32-bit word (empty when hi <= lo).
__device__ __forceinline__ uint32_t bit_range(int lo, int hi) {
  lo = max(lo, 0);
  hi = min(hi, 32);
  if (hi <= lo) return 0u;
  const uint32_t w = (hi - lo >= 32) ? 0xffffffffu : ((1u << (hi - lo)) - 1u);
  return w << lo;
}

struct TcParams {
  TcArgs a;
  TcWork w;
  int nstages;
  int split;
  uint32_t stage_bytes;
  int seg_kb;  // K blocks (of KC elements) per accumulation segment
  SeriesTable sr;
};


struct Ctl {
  volatile int* abort;
  int* err;
  unsigned long long limit_ns;
};

// Bounded wait on an mbarrier phase. Records a timeout and raises the CTA's abort
// flag when the limit runs out; gives up early when another role aborted.
__device__ __forceinline__ bool wait_bounded(uint32_t bar, uint32_t parity, const Ctl& c,
                                             bool honor_abort = true) {
  if (ptx::mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = ptx::globaltimer();
  for (;;) {
    if (ptx::mbar_try_wait(bar, parity)) return true;
    if (honor_abort && *c.abort) return false;
    if (ptx::globaltimer() - t0 > c.limit_ns) {
      atomicCAS(c.err, 0, kErrTimeout);
      *c.abort = 1;
      return false;
    }
  }
}

// A unit with its series' parameters.
struct UnitSpan {
  int strip, T0, jlo, jhi, ntiles, slot, nser, step;
  int carry, adv;  // carry: the last L-1 Gram columns pass from tile to tile; adv: tile stride
  int M, L, k, e, R;      // series: trajectories, length, neighbours, exclusion, rows per strip
  int row_base, out_base, slots, strip_base;
  long long part_base, col_base;
};

// Unit u for the sj-th of the series that share its Gram tiles (sj = 0: the one
// with the most trajectories, whose tiles cover the others').
__device__ __forceinline__ bool unit_span(const TcWork& w, const SeriesInfo* sr, int u, int sj,
                                          UnitSpan& us) {
  const WorkUnit wu = w.units[u];
  const SeriesInfo& si = sr[wu.series + sj];
  us.nser = wu.pad[0] > 1 ? wu.pad[0] : 1;
  us.M = si.M;
  us.L = si.L;
  us.k = si.k;
  us.e = si.e;
  us.R = si.rows_out;
  us.row_base = si.row_base;
  us.out_base = si.out_base;
  us.slots = si.slots;
  us.strip_base = si.strip_base;
  us.part_base = si.part_base;
  us.col_base = si.col_base;
  us.strip = wu.strip;
  us.T0 = wu.strip * us.R;
  us.jlo = wu.jlo;
  us.jhi = min(wu.jhi, si.M);
  us.slot = wu.slot;
  us.step = si.step;
  if (us.jlo >= us.jhi) return false;
  // A unit of one series: Gram tiles follow each other without overlap, tile it
  // covering Gram columns [jlo + 256 it, jlo + 256 (it+1)); the epilogue carries the
  // last L-1 columns of a tile into the next, so the windows of all output columns
  // [jlo, jhi) are complete once Gram column jhi + L - 2 is in. A unit shared by
  // several series (each restages the chunk buffer with its own L) has no carry: its
  // tiles overlap by the largest L - 1 and each yields `step` output columns.
  us.carry = us.nser == 1;
  us.adv = us.carry ? BN : us.step;
  us.ntiles = us.carry ? (us.jhi - us.jlo + us.L - 1 + BN - 1) / BN
                       : (us.jhi - us.jlo + us.step - 1) / us.step;
  return true;
}

// Publish an upper bound of a row's k-th distance. The same pair distance can be
// evaluated more than once (band pre-pass and main pass; a pair and its transpose)
// with results a few ulp apart, so a bound taken from one evaluation is widened by
// a relative 2^-12 (far above those differences) before it prunes another; a wider
// bound only admits more candidates to the exact final selection.
__device__ __forceinline__ void publish_bound(unsigned int* thr, float d) {
  atomicMin(thr, __float_as_uint(__fmul_ru(d, 1.0f + 0x1p-12f)));
}

// The k-th entry of a sorted register list (k is a run-time value, K a compile-time
// bound): the minimum of entries k-1 .. K-1, written as a reduction so that the
// list stays in registers.
template <int K>
__device__ __forceinline__ float kth_of(const RegList<K>& l, int k) {
  float v = CUDART_INF_F;
#pragma unroll
  for (int p = 0; p < K; ++p) v = fminf(v, p >= k - 1 ? l.d[p] : CUDART_INF_F);
  return v;
}

constexpr int kQueue = 4;  // depth of the per-CTA unit queue
constexpr size_t kGroupBoundBytes = 2 * BM * 8;  // two groups' tagged row bounds

template <int K, int G>
__global__ void __launch_bounds__(kThreadsG(G), 1)
    fused_tc_kernel(const __grid_constant__ CUtensorMap tmA_hi,
                    const __grid_constant__ CUtensorMap tmA_lo,
                    const __grid_constant__ CUtensorMap tmB_hi,
                    const __grid_constant__ CUtensorMap tmB_lo,
                    const __grid_constant__ TcParams p) {
  extern __shared__ unsigned char smem_raw[];
  const TcArgs& a = p.a;
  const TcWork& w = p.w;
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int NS = p.nstages;

  // ---- shared memory carve-up (ring base aligned to 1 KB for the swizzle pattern)
  const uint32_t raw = ptx::smem_u32(smem_raw);
  const uint32_t ring = (raw + 1023u) & ~1023u;
  unsigned char* gptr = smem_raw + (ring - raw) + (size_t)NS * p.stage_bytes;
  // epilogue regions (one per group), sized for the largest L and k of the call
  const size_t gbytes = group_bytes(a.kmax, a.Lmax);
  // two groups: each row's current list bound in each group, tagged with the unit
  // (the other group's bound also bounds the row's k-th distance; see the scan)
  volatile unsigned long long* gbound =
      reinterpret_cast<volatile unsigned long long*>(gptr + G * gbytes);
  uint64_t* bars =
      reinterpret_cast<uint64_t*>(gptr + G * gbytes + (G == 2 ? kGroupBoundBytes : 0));
  const uint32_t full0 = ptx::smem_u32(bars);
  const uint32_t empty0 = full0 + 8u * NS;
  const uint32_t tfull0 = empty0 + 8u * NS;
  const uint32_t tempty0 = tfull0 + 16u;
  const uint32_t drain = tempty0 + 16u;
  const uint32_t qfull0 = drain + 8u;
  const uint32_t qempty0 = qfull0 + 8u * kQueue;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * NS + 5 + 2 * kQueue);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  volatile int* qval = reinterpret_cast<volatile int*>(tmem_slot + 2);  // [kQueue]

  Ctl ctl;
  ctl.abort = abort_flag;
  ctl.err = a.err;
  ctl.limit_ns = (unsigned long long)a.wait_limit_ns;

  if (threadIdx.x == 0) {
    for (int i = 0; i < NS; ++i) {
      ptx::mbar_init(full0 + 8u * i, 1);
      ptx::mbar_init(empty0 + 8u * i, 1);
    }
    for (int b = 0; b < 2; ++b) {
      ptx::mbar_init(tfull0 + 8u * b, 1);
      ptx::mbar_init(tempty0 + 8u * b, kEpiThreads * G);  // every epilogue thread
    }
    ptx::mbar_init(drain, 1);
    for (int i = 0; i < kQueue; ++i) {
      ptx::mbar_init(qfull0 + 8u * i, 1);
      ptx::mbar_init(qempty0 + 8u * i, 1 + G);  // the MMA thread and each group's leader
    }

    *abort_flag = 0;
    ptx::fence_mbar_init();
    ptx::fence_proxy_async();
  }
  if (warp == 1) {
    ptx::tmem_alloc(ptx::smem_u32(tmem_slot), 512);
    ptx::tmem_relinquish();
    ptx::tc_fence_before();
  }
  if (G == 2)  // no unit has tag 0xFFFFFFFF: every entry starts unused
    for (int i = threadIdx.x; i < 2 * BM; i += blockDim.x) gbound[i] = ~0ull;
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const int nkb = a.Dp / KC;
  const int seg_kb = p.seg_kb;                    // K blocks per accumulation segment
  // segments per tile (the two-group form runs with one segment: checked on the host)
  const int nseg = G == 2 ? 1 : (nkb + seg_kb - 1) / seg_kb;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    // Hands out units in list order (global counter) through a small queue, so the
    // units in flight across the GPU stay a contiguous window of the list.
    if (lane == 0) {
      ptx::prefetch_tensormap(&tmA_hi);
      ptx::prefetch_tensormap(&tmB_hi);
      if (p.split) {
        ptx::prefetch_tensormap(&tmA_lo);
        ptx::prefetch_tensormap(&tmB_lo);
      }
      const uint64_t pol_a = ptx::l2_policy_evict_last();
      int stage = 0, qs = 0;
      uint32_t phase = 0, qphase = 0, issued = 0, issued_par = 0;
      bool ok = true, withheld = false;
      UnitSpan us;
      while (ok) {
        if (!wait_bounded(qempty0 + 8u * qs, qphase ^ 1u, ctl)) break;
        const int u = atomicAdd(w.counter, 1);
        qval[qs] = u;
        ptx::mbar_arrive(qfull0 + 8u * qs);
        if (++qs == kQueue) {
          qs = 0;
          qphase ^= 1u;
        }
        if (u >= w.nunits) break;
        if (!unit_span(w, p.sr.s, u, 0, us)) continue;
        for (int it = 0; ok && it < us.ntiles; ++it) {
          const int c0 = us.row_base + us.jlo + it * us.adv;
          const int a0 = us.row_base + us.T0;
          for (int kb = 0; kb < nkb; ++kb) {
            if (!wait_bounded(empty0 + 8u * stage, phase ^ 1u, ctl)) {
              ok = false;
              break;
            }
            if (a.debug_withhold && u == 0 && !withheld) {
              withheld = true;  // test hook: unit 0's first stage is never filled
            } else {
              const uint32_t fb = full0 + 8u * stage;
              const uint32_t sb = ring + (uint32_t)stage * p.stage_bytes;
              ptx::mbar_arrive_expect_tx(fb, p.stage_bytes);
              // the strip operand (A) is read again for every tile of the unit: keep it
              // in L2 ahead of the column tiles when asked to
              if (a.l2_keep_a) {
                ptx::tma_load_2d_hint(sb, &tmA_hi, fb, kb * KC, a0, pol_a);
                if (p.split) ptx::tma_load_2d_hint(sb + kTileA, &tmA_lo, fb, kb * KC, a0, pol_a);
              } else {
                ptx::tma_load_2d(sb, &tmA_hi, fb, kb * KC, a0);
                if (p.split) ptx::tma_load_2d(sb + kTileA, &tmA_lo, fb, kb * KC, a0);
              }
              if (p.split) {
                ptx::tma_load_2d(sb + 2 * kTileA, &tmB_hi, fb, kb * KC, c0);
                ptx::tma_load_2d(sb + 2 * kTileA + kTileB, &tmB_lo, fb, kb * KC, c0);
              } else {
                ptx::tma_load_2d(sb + kTileA, &tmB_hi, fb, kb * KC, c0);
              }
              issued |= 1u << stage;
              issued_par = (issued_par & ~(1u << stage)) | (phase << stage);
            }
            if (++stage == NS) {
              stage = 0;
              phase ^= 1u;
            }
          }
        }
      }
      // every copy issued into this CTA's shared memory must land before exit
      for (int i = 0; i < NS; ++i)
        if ((issued >> i) & 1u) wait_bounded(full0 + 8u * i, (issued_par >> i) & 1u, ctl, false);
    }
    __syncwarp();
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      int stage = 0, qs = 0, gt = 0, gs = 0, acc = 0;  // gs: segments issued so far
      uint32_t phase = 0, qphase = 0;
      bool ok = true, issued_any = false;
      long long wait_tmem = 0, wait_full = 0;
      const long long t_start = clock64();
      UnitSpan us;
      while (ok) {
        if (!wait_bounded(qfull0 + 8u * qs, qphase, ctl)) {
          ok = false;
          break;
        }
        const int u = qval[qs];
        ptx::mbar_arrive(qempty0 + 8u * qs);
        if (++qs == kQueue) {
          qs = 0;
          qphase ^= 1u;
        }
        if (u >= w.nunits) break;
        if (!unit_span(w, p.sr.s, u, 0, us)) continue;
        for (int it = 0; ok && it < us.ntiles; ++it, ++gt) {
          for (int kb = 0; kb < nkb; ++kb) {
            if (kb % seg_kb == 0) {
              // a new segment: segment gs uses accumulator gs & 1 for the (gs >> 1)-th time
              if (kb > 0) {
                ptx::mma_commit(tfull0 + 8u * acc);  // the finished segment to the epilogue
                ++gs;
              }
              acc = gs & 1;
              const long long tw0 = w.stats ? clock64() : 0;
              if (!wait_bounded(tempty0 + 8u * acc, ((gs >> 1) & 1) ^ 1u, ctl)) {
                ok = false;
                break;
              }
              if (w.stats) wait_tmem += clock64() - tw0;
              ptx::tc_fence_after();
            }
            const uint32_t d = tmem_base + (uint32_t)(acc * BN);
            const long long tf0 = w.stats ? clock64() : 0;
            if (!wait_bounded(full0 + 8u * stage, phase, ctl)) {
              ok = false;
              break;
            }
            if (w.stats) wait_full += clock64() - tf0;
            ptx::tc_fence_after();
            const uint32_t sb = ring + (uint32_t)stage * p.stage_bytes;
            const uint32_t a_hi = sb;
            const uint32_t a_lo = sb + kTileA;
            const uint32_t b_hi = p.split ? sb + 2 * kTileA : sb + kTileA;
            const uint32_t b_lo = b_hi + kTileB;
            const uint32_t first = kb % seg_kb == 0 ? 1u : 0u;
#pragma unroll
            for (int kk = 0; kk < KC / 16; ++kk) {
              const uint64_t dah = ptx::sdesc_kmajor_sw64(a_hi + kk * 32);
              const uint64_t dbh = ptx::sdesc_kmajor_sw64(b_hi + kk * 32);
              ptx::mma_f16(d, dah, dbh, kIdesc, (first && kk == 0) ? 0u : 1u);
              if (p.split) {
                const uint64_t dal = ptx::sdesc_kmajor_sw64(a_lo + kk * 32);
                const uint64_t dbl = ptx::sdesc_kmajor_sw64(b_lo + kk * 32);
                ptx::mma_f16(d, dah, dbl, kIdesc, 1u);
                ptx::mma_f16(d, dal, dbh, kIdesc, 1u);
              }
            }
            issued_any = true;
            ptx::mma_commit(empty0 + 8u * stage);  // frees the stage once these MMAs finish
            if (++stage == NS) {
              stage = 0;
              phase ^= 1u;
            }
          }
          if (!ok) break;
          ptx::mma_commit(tfull0 + 8u * acc);  // the tile's last segment
          ++gs;
        }
      }
      if (w.stats) {
        atomicAdd(w.stats + kStatMmaWaitTmem, (unsigned long long)wait_tmem);
        atomicAdd(w.stats + kStatMmaWaitFull, (unsigned long long)wait_full);
        atomicAdd(w.stats + kStatMmaCycles, (unsigned long long)(clock64() - t_start));
      }
      if (!ok && issued_any) {
        // all MMAs of this thread must finish before TMEM is released
        ptx::mma_commit(drain);
        wait_bounded(drain, 0, ctl, false);
      }
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ epilogue
    const int gid = G == 1 ? 0 : (warp - 2) >> 2;  // epilogue group
    const int q = warp & 3;          // TMEM lane quadrant this warp may access
    const int l = q * 32 + lane;     // accumulator row owned by this thread
    const uint32_t lane_addr = (uint32_t)(q * 32) << 16;
    const int et = threadIdx.x - 64 - kEpiThreads * gid;  // 0..127 within the group
    const int bar = 1 + gid;          // the group's named barrier
    // the group's chunks of every tile
    const int ch_lo = gid * (BN / 32 / G), ch_hi = ch_lo + BN / 32 / G;
    // the group's shared memory
    float* Gbuf = reinterpret_cast<float*>(gptr + gid * gbytes);
    float* Wsh = Gbuf + BM * chunk_pitch(a.Lmax);  // window sums of the tile's output columns
    float* Tsh = Wsh + BN;         // row bounds of the tile's output columns (column side)
    float* Csh = Tsh + BN;         // correction values c of the tile's Gram columns
    uint32_t* Cmask = reinterpret_cast<uint32_t*>(Csh + BN);  // [4][32] column-side row masks
    float* Cld = reinterpret_cast<float*>(Cmask + 128);  // [kmax][32] column-side lists
    int32_t* Cli = reinterpret_cast<int32_t*>(Cld + 32 * a.kmax);
    const long long cpitch = col_pitch(w.kstride);  // ints per column-list record
    const int cx = ((warp - 2) & 3) * 8 + (lane & 7);      // column-side column of lanes 0..7
    int qs = 0, gch = 0, gt = 0;
    uint32_t qphase = 0;
    bool ok = true;
    UnitSpan us;
    // phase timing of the first epilogue thread (diagnostics)
    // (the two-group form keeps no phase timers: its registers are scarcer)
    const bool timed = G == 1 && w.stats != nullptr && et == 0 && gid == 0;
    long long ph[7] = {0, 0, 0, 0, 0, 0, 0};
    // event counts kept per thread, summed once at the end (diagnostics)
    unsigned int cnt[5] = {0, 0, 0, 0, 0};
    const long long e_start = timed ? clock64() : 0;
    long long tp = e_start;
    auto lap = [&](int i) {
      if (timed) {
        const long long now = clock64();
        ph[i] += now - tp;
        tp = now;
      }
    };
    RegList<K> list;
    // Segment folding (more than one segment per tile): segment pseg of tile pt is
    // the next to add to the tile's partial total; every segment but a tile's last
    // is folded (segment s of tile t is segment t * nseg + s overall, in accumulator
    // (t * nseg + s) & 1), the last is added while the tile is scanned. The partial
    // totals live in this CTA's scratch array, two tile slots of
    // [8 chunks][8 float4 groups][128 rows] float4; each thread folds and later
    // reads only its own row, so warps fold independently.
    int pt = 0, pseg = 0;
    long long fold_cycles = 0;
    float4* const scr = reinterpret_cast<float4*>(a.scratch) + (size_t)blockIdx.x * (2 * BM * BN / 4);
    auto fold = [&](bool block, int upto) -> bool {
      while (nseg > 1 && pt <= upto) {
        const long long gsi = (long long)pt * nseg + pseg;
        const int b = (int)(gsi & 1);
        const uint32_t par = (uint32_t)((gsi >> 1) & 1);
        if (!block) {
          const bool r = ptx::mbar_try_wait(tfull0 + 8u * b, par);
          if (!__shfl_sync(0xffffffffu, r, 0)) return true;  // not ready: try later
        }
        if (!wait_bounded(tfull0 + 8u * b, par, ctl)) return false;
        const long long f0 = timed ? clock64() : 0;
        ptx::tc_fence_after();
        const uint32_t tA = tmem_base + lane_addr + (uint32_t)(b * BN);
        float4* srow = scr + (size_t)(pt & 1) * (BM * BN / 4) + l;
        // the first segment is stored, later ones are added by FP32 reductions in L2
        // (round to nearest); every element has this thread as its only writer, so
        // the additions happen in segment order and the total is deterministic
#pragma unroll 1
        for (int c = 0; c < BN / 32; ++c) {
          uint32_t v[32];
          ptx::tmem_ld32_async(tA + c * 32, v);
          ptx::tmem_wait();
#pragma unroll
          for (int g = 0; g < 8; ++g) {
            const float4 r = make_float4(__uint_as_float(v[4 * g]), __uint_as_float(v[4 * g + 1]),
                                         __uint_as_float(v[4 * g + 2]),
                                         __uint_as_float(v[4 * g + 3]));
            if (pseg == 0)
              __stcg(srow + (c * 8 + g) * BM, r);
            else
              atomicAdd(srow + (c * 8 + g) * BM, r);
          }
        }
        ptx::tc_fence_before();
        ptx::mbar_arrive(tempty0 + 8u * b);  // the accumulator is free for the next segment
        if (timed) fold_cycles += clock64() - f0;
        if (++pseg == nseg - 1) {
          pseg = 0;
          ++pt;
        }
      }
      return true;
    };
    // 32 columns (chunk ch) of this thread's row of tile gt's total, from the scratch
    auto load_scr = [&](int tile, int ch, uint32_t (&v)[32]) {
      const float4* srow = scr + (size_t)(tile & 1) * (BM * BN / 4) + l;
#pragma unroll
      for (int g = 0; g < 8; ++g) {
        const float4 r = __ldcg(srow + (ch * 8 + g) * BM);
        v[4 * g] = __float_as_uint(r.x);
        v[4 * g + 1] = __float_as_uint(r.y);
        v[4 * g + 2] = __float_as_uint(r.z);
        v[4 * g + 3] = __float_as_uint(r.w);
      }
    };
    while (ok) {
      bool wok = wait_bounded(qfull0 + 8u * qs, qphase, ctl);
      const int u = wok ? qval[qs] : 0;
      wok = ptx::named_bar_and(bar, kEpiThreads, wok);  // everyone has read the slot
      if (!wok) {
        ok = false;
        break;
      }
      if (et == 0) ptx::mbar_arrive(qempty0 + 8u * qs);
      if (++qs == kQueue) {
        qs = 0;
        qphase ^= 1u;
      }
      if (u >= w.nunits) break;
      if (!unit_span(w, p.sr.s, u, 0, us)) continue;
      // Series that share this unit's Gram tiles (several trajectory lengths of one
      // record) are served one after another from the same accumulator; their units
      // are one tile long, so their row lists live for one tile.
      const int nser = us.nser;
      const int ntiles = us.ntiles;
      for (int it = 0; it < ntiles; ++it, ++gt) {
        lap(6);
        // the earlier segments are folded into the scratch partial total; the last
        // one is read from its accumulator while the tile is scanned
        // accumulator holding the tile's last segment (the whole tile if nseg == 1)
        const long long glast = (long long)gt * nseg + nseg - 1;
        const int acc_l = (int)(glast & 1);
        if (nseg > 1) wok = fold(true, gt);
        if (wok) wok = wait_bounded(tfull0 + 8u * acc_l, (uint32_t)((glast >> 1) & 1), ctl);
        wok = ptx::named_bar_and(bar, kEpiThreads, wok);  // all four warps agree
        if (!wok) {
          ok = false;
          break;
        }
        ptx::tc_fence_after();
        lap(0);
        bool released = false;
        for (int sj = 0; sj < nser; ++sj) {
        if (nser > 1 && !unit_span(w, p.sr.s, u, sj, us)) continue;
        const int L = G == 2 ? 1 : us.L;  // two groups run only at L = 1
        const int LDG = chunk_pitch(L);
        const int t = us.T0 + l;
        const bool row_ok = l < us.R && t < us.M;
        const float Wt = row_ok ? a.W[us.out_base + t] : 0.f;
        // the operand layout subtracts groups * c_a * c_b from every Gram entry (see the
        // operand preparation); it is added back when a chunk is staged, for every
        // accumulator row whose day exists (halo rows feed other rows' windows)
        const int N = us.M + us.L - 1;
        // (with one product on split operands the correction entries added
        // +groups c_a c_b: subtract it instead)
        const float crow =
            t < N ? (a.corr_neg ? -(float)a.groups : (float)a.groups) * a.cval[us.row_base + t]
                  : 0.f;
        const int jsym = us.T0 + us.R;  // column side from here on (sym)
        const long long cbase = w.sym ? us.col_base + w.col_off[us.strip_base + us.strip] : 0;
        if (nser > 1 || it == 0) list.reset();
        const int c0 = us.jlo + it * us.adv;
        // W and row bounds of this tile's output columns j = c0 - (L-1) + x (the
        // previous tile's readers passed its last barrier)
        for (int x = et; x < BN; x += kEpiThreads) {
          const int j = c0 - (L - 1) + x;
          const bool in = j >= 0 && j < us.M;
          Wsh[x] = in ? a.W[us.out_base + j] : 0.f;
          Tsh[x] = in ? __uint_as_float(__ldcg(w.thr + us.out_base + j)) : 0.f;
          Csh[x] = c0 + x < N ? a.cval[us.row_base + c0 + x] : 0.f;  // Gram column day c0 + x
        }
        const float thr_row = row_ok ? __uint_as_float(__ldcg(w.thr + us.out_base + t)) : 0.f;
        ptx::named_bar_sync(bar, kEpiThreads);  // Csh is read by every thread when staging
        lap(1);
        // chunk ch+1 is fetched while chunk ch is scanned: from TMEM with a single
        // segment, else the scratch partial total (the last segment's chunk is
        // added from TMEM when the chunk is staged)
        const uint32_t tlast = tmem_base + lane_addr + (uint32_t)(acc_l * BN);
        // with the largest lists, and with two epilogue groups (168 registers a thread;
        // the other group hides the latency), the chunk is fetched when it is staged
        // instead (the prefetched registers would otherwise stay live across the scan
        // and spill)
        constexpr bool kAhead = K <= 40 && G == 1;
        uint32_t vr[32];
        if (kAhead) {
          if (nseg == 1)
            ptx::tmem_ld32_async(tlast + (uint32_t)(ch_lo * 32), vr);
          else
            load_scr(gt, ch_lo, vr);
        }
#pragma unroll 1
        for (int ch = ch_lo; ch < ch_hi; ++ch) {
          if (!kAhead) {
            if (nseg == 1)
              ptx::tmem_ld32_async(tlast + (uint32_t)(ch * 32), vr);
            else
              load_scr(gt, ch, vr);
          }
          float* grow = Gbuf + l * LDG;
          // the diagonal carry: the last L-1 Gram columns of the previous chunk (of
          // the previous tile of this unit at ch = 0) start this chunk's windows
          if (ch > 0 || (it > 0 && us.carry))
            for (int c = 0; c < L - 1; ++c) grow[c] = grow[32 + c];
          const float* cs = Csh + ch * 32;
          // Gram values of the chunk (correction added back): staged in shared memory
          // for the diagonal window sums, or, with L = 1 (no window), kept in registers
          float c[32];
          if (nseg == 1) {
            ptx::tmem_wait();
#pragma unroll
            for (int x = 0; x < 32; ++x) c[x] = fmaf(crow, cs[x], __uint_as_float(vr[x]));
          } else {
            uint32_t tv[32];
            ptx::tmem_ld32_async(tlast + (uint32_t)(ch * 32), tv);
            ptx::tmem_wait();
#pragma unroll
            for (int x = 0; x < 32; ++x)
              c[x] = fmaf(crow, cs[x], __uint_as_float(vr[x]) + __uint_as_float(tv[x]));
          }
          if (L > 1) {
#pragma unroll
            for (int x = 0; x < 32; ++x) grow[(L - 1) + x] = c[x];
          }
          if (kAhead && ch + 1 < ch_hi) {
            if (nseg == 1)
              ptx::tmem_ld32_async(tlast + (uint32_t)((ch + 1) * 32), vr);
            else
              load_scr(gt, ch + 1, vr);
          }
          if (ch == ch_hi - 1 && sj == nser - 1) {
            // the accumulator has been read out: hand it back to the MMA warp
            ptx::tc_fence_before();
            ptx::mbar_arrive(tempty0 + 8u * acc_l);
            released = true;
          }
          lap(2);
          // the window sums read other rows' staged values (nothing to wait for at L = 1)
          if (L > 1) ptx::named_bar_sync(bar, kEpiThreads);
          lap(3);
          const int j0 = c0 + ch * 32 - (L - 1);
          // column side of this chunk: output columns j >= jsym inside the unit
          // the first L-1 columns of a unit's first chunk have no carried window
          const int xfirst = (ch == 0 && (it == 0 || !us.carry)) ? L - 1 : 0;
          const uint32_t colrange = w.sym ? bit_range(max(jsym, us.jlo) - j0, us.jhi - j0) &
                                                bit_range(xfirst, 32)
                                          : 0u;
          uint32_t cand = 0, ccand = 0;
          float othr = CUDART_INF_F;  // the other group's bound for this row (two groups)
          if (row_ok) {
            // output column x of this chunk is j = j0 + x; its window is the diagonal
            // Gbuf[l+m][x+m], m < L (Eq. 2 as W_t + W_j - 2 sum G)
            uint32_t valid = bit_range(xfirst, 32) & bit_range(us.jlo - j0, us.jhi - j0);
            valid &= ~bit_range(t - us.e - j0, t + us.e + 1 - j0);  // exclusion zone
            const float* g0 = Gbuf + l * LDG;
            const float* wv = Wsh + ch * 32;
            const float* tv = Tsh + ch * 32;
            if (L > 1) {
#pragma unroll
              for (int x = 0; x < 32; ++x) c[x] = g0[x];
              for (int m = 1; m < L; ++m) {
                const float* gm = g0 + m * (LDG + 1);
#pragma unroll
                for (int x = 0; x < 32; ++x) c[x] += gm[x];
              }
            }
            const float lthr = list.threshold();
            // a row candidate has D < lthr and D <= thr_row, i.e. D <= rthr (the float
            // below lthr when lthr > 0; none when lthr is 0)
            // with two groups, the other group's list for this row in this unit holds K
            // real candidates of other columns: its K-th bounds the row's k-th too
            if (G == 2) {
              const unsigned long long ob = gbound[(1 - gid) * BM + l];
              if ((unsigned)(ob >> 32) == (unsigned)u) othr = __uint_as_float((unsigned)ob);
            }
            float rthr =
                fminf(lthr > 0.f ? __uint_as_float(__float_as_uint(lthr) - 1u) : -1.f, thr_row);
            if (G == 2) rthr = fminf(rthr, othr);
            if (G == 1 && a.band_margin != 0.f) {
              // one-product band pre-pass (long operand rows only, so one epilogue
              // group): the distance raised by a bound of its error
#pragma unroll
              for (int x = 0; x < 32; ++x)
                c[x] = fmaf(a.band_margin, Wt + wv[x],
                            fmaxf(fmaf(-2.0f, c[x], Wt + wv[x]), 0.0f)) * (1.0f + 0x1p-20f);
            } else {
#pragma unroll
              for (int x = 0; x < 32; ++x)
                c[x] = fmaxf(fmaf(-2.0f, c[x], Wt + wv[x]), 0.0f);  // D(t, j0 + x)
            }
#pragma unroll
            for (int x = 0; x < 32; ++x) {
              cand |= (c[x] <= rthr ? 1u : 0u) << x;
              ccand |= (c[x] <= tv[x] ? 1u : 0u) << x;
            }
            cand &= valid;
            ccand &= valid & colrange;
          }
          // column-side candidates, transposed by ballots: lane x of warp quadrant q
          // holds the rows q*32 + b of column x that pass the column's bound
          uint32_t cm = 0;
          if (__any_sync(0xffffffffu, ccand != 0u)) {
#pragma unroll
            for (int x = 0; x < 32; ++x) {
              const uint32_t b = __ballot_sync(0xffffffffu, (ccand >> x) & 1u);
              cm = lane == x ? b : cm;
            }
            cnt[1] += __popc(ccand);
          }
          Cmask[q * 32 + lane] = cm;
          ptx::named_bar_sync(bar, kEpiThreads);
          // every window sum of the chunk is done: a row with candidates replaces the
          // first 32 entries of its Gram row by its distances (the carried columns
          // 32.. stay), so that candidates are read back instead of recomputed
          if (cand | ccand) {
            float* drow = Gbuf + l * LDG;
#pragma unroll
            for (int x = 0; x < 32; ++x) drow[x] = c[x];
          }
          if (colrange) ptx::named_bar_sync(bar, kEpiThreads);  // other rows read them
          lap(4);
          // row side: the few distances that enter the row's list
          while (cand) {
            const int x = __ffs(cand) - 1;
            cand &= cand - 1;
            const float dv = Gbuf[l * LDG + x];
            if (dv < list.threshold() && dv <= thr_row && (G == 1 || dv <= othr)) {
              list.insert(dv, j0 + x);
              ++cnt[0];
            }
          }
          if (G == 2 && row_ok)
            gbound[gid * BM + l] =
                ((unsigned long long)(unsigned)u << 32) | __float_as_uint(list.threshold());
          // column side, written by the rows themselves: column x's list holds its
          // candidate rows in row order (slot = number of candidate rows before
          // this one), unless more than k rows qualify, in which case the column's
          // own thread below keeps the k best
          while (ccand) {
            const int x = __ffs(ccand) - 1;
            ccand &= ccand - 1;
            int before = __popc(Cmask[q * 32 + x] & ((1u << lane) - 1u)), ne = 0;
#pragma unroll
            for (int wq = 0; wq < 4; ++wq) {
              const int cq = __popc(Cmask[wq * 32 + x]);
              ne += cq;
              before += wq < q ? cq : 0;
            }
            if (ne <= us.k) {
              const long long li = cbase + (j0 + x - jsym);
              const long long at = li * cpitch + 2 + 2 * before;
              if (tk_in(at + 1, w.col_ints, a.err) && tk_in(before, us.k, a.err))
                *reinterpret_cast<int2*>(w.col_rec + at) =
                    make_int2(us.T0 + l, __float_as_int(Gbuf[l * LDG + x]));
            }
          }
          if (colrange && lane < 8 && ((colrange >> cx) & 1u)) {
            const int j = j0 + cx;
            const long long li = cbase + (j - jsym);
            int ne = 0;
#pragma unroll
            for (int wq = 0; wq < 4; ++wq) ne += __popc(Cmask[wq * 32 + cx]);
            if (ne == us.k) {
              // exactly k candidates: the largest is the k-th distance
              float mx = 0.f;
              for (int wq = 0; wq < 4; ++wq) {
                uint32_t mk = Cmask[wq * 32 + cx];
                while (mk) {
                  const int r = wq * 32 + __ffs(mk) - 1;
                  mk &= mk - 1;
                  mx = fmaxf(mx, Gbuf[r * LDG + cx]);
                }
              }
              if (tk_in(us.out_base + j, a.out_rows, a.err))
                publish_bound(w.thr + us.out_base + j, mx);
            } else if (ne > us.k) {
              // more than k: keep the k best in (distance, row) order; rows arrive in
              // increasing order, so a strict compare keeps the smaller row first
              int n = 0;
              for (int wq = 0; wq < 4; ++wq) {
                uint32_t mk = Cmask[wq * 32 + cx];
                while (mk) {
                  const int r = wq * 32 + __ffs(mk) - 1;
                  mk &= mk - 1;
                  const float dv = Gbuf[r * LDG + cx];
                  int pos;
                  if (n < us.k) {
                    pos = n++;
                  } else if (dv < Cld[(us.k - 1) * 32 + cx]) {
                    pos = us.k - 1;
                  } else {
                    continue;
                  }
                  while (pos > 0 && Cld[(pos - 1) * 32 + cx] > dv) {
                    Cld[pos * 32 + cx] = Cld[(pos - 1) * 32 + cx];
                    Cli[pos * 32 + cx] = Cli[(pos - 1) * 32 + cx];
                    --pos;
                  }
                  Cld[pos * 32 + cx] = dv;
                  Cli[pos * 32 + cx] = us.T0 + r;
                }
              }
              for (int pp = 0; pp < us.k; ++pp)
                if (tk_in(li * cpitch + 3 + 2 * pp, w.col_ints, a.err))
                  *reinterpret_cast<int2*>(w.col_rec + li * cpitch + 2 + 2 * pp) =
                      make_int2(Cli[pp * 32 + cx], __float_as_int(Cld[pp * 32 + cx]));
              if (tk_in(us.out_base + j, a.out_rows, a.err))
                publish_bound(w.thr + us.out_base + j, Cld[(us.k - 1) * 32 + cx]);
            }
            if (ne > 0) {  // an empty list gets no record: its mask bit stays clear
              if (tk_in(li * cpitch, w.col_ints, a.err)) w.col_rec[li * cpitch] = min(ne, us.k);
              const long long mi = (long long)(us.out_base + j) * w.mask_words + (us.strip >> 5);
              if (tk_in(mi, (long long)a.out_rows * w.mask_words, a.err))
                atomicOr(w.col_mask + mi, 1u << (us.strip & 31));
            }
            cnt[3] += ne > 0;
            cnt[2] += ne > us.k;  // lists kept by this thread's insertion
          }
          // the column side read other rows' Gram values: keep them until it is done
          if (colrange) ptx::named_bar_sync(bar, kEpiThreads);
          cnt[4] += et == 0;
          lap(5);
          fold(false, gt + 1);  // the next tile's finished segments, if any
          lap(2);
          ++gch;
        }
        if (row_ok) {
          const float kth = kth_of(list, us.k);
          if (kth < thr_row && tk_in(us.out_base + t, a.out_rows, a.err))
            publish_bound(w.thr + us.out_base + t, kth);
        }
        if (row_ok && w.write_lists && (nser > 1 || it == ntiles - 1)) {
          const size_t base =
              (size_t)(us.part_base + (long long)t * us.slots + us.slot * G + gid) * w.kstride;
#pragma unroll
          for (int pp = 0; pp < K; ++pp) {
            if (pp < us.k) {
              if (tk_in((long long)base + pp, w.part_ints, a.err)) {
                a.part_d[base + pp] = list.d[pp];
                a.part_i[base + pp] = list.i[pp];
              }
            }
          }
        }
        // the next series restages the chunk buffer and the tile's W, bounds, masks
        if (nser > 1) ptx::named_bar_sync(bar, kEpiThreads);
        }  // series sharing the tile
        if (!released) {
          ptx::tc_fence_before();
          ptx::mbar_arrive(tempty0 + 8u * acc_l);
        }
      }
      if (!ok) break;
    }
    if (w.stats) {
#pragma unroll
      for (int i = 0; i < 5; ++i) {
        unsigned int v = cnt[i];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0 && v) atomicAdd(w.stats + kStatRowInserts + i, (unsigned long long)v);
      }
    }
    if (timed) {
      lap(6);
      for (int i = 0; i < 6; ++i) atomicAdd(w.stats + kStatEpiWaitAcc + i, (unsigned long long)ph[i]);
      atomicAdd(w.stats + kStatEpiCycles, (unsigned long long)(clock64() - e_start));
      atomicAdd(w.stats + kStatEpiStage, (unsigned long long)fold_cycles);
    }
  }

  __syncthreads();
  if (warp == 1) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem_base, 512);
  }
}

// ------------------------------------------------------------------- host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(ptr);
  }
  return fn;
}

// Row-major [N][Dp] BF16 operand copy, boxes of 32 elements x box_rows rows.
bool make_map(CUtensorMap* m, const void* base, int N, int Dp, int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)Dp, (cuuint64_t)N};
  const cuuint64_t strides[1] = {(cuuint64_t)Dp * 2};
  const cuuint32_t box[2] = {(cuuint32_t)KC, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

size_t epilogue_bytes(int k, int L, int G) {
  return G * group_bytes(k, L) + (G == 2 ? kGroupBoundBytes : 0) +
         8 * (2 * kMaxStages + 5 + 2 * kQueue) + 8 + 4 * kQueue + 16;
}

int pick_stages(bool split, int k, int L, int G) {
  const uint32_t stage = split ? 2 * kTileA + 2 * kTileB : kTileA + kTileB;
  const size_t avail = kSmemLimit - 1024 - epilogue_bytes(k, L, G);
  int ns = (int)(avail / stage);
  return ns < kMaxStages ? ns : kMaxStages;
}

template <int K, int G>
cudaError_t launch_k(const CUtensorMap& mAh, const CUtensorMap& mAl, const CUtensorMap& mBh,
                     const CUtensorMap& mBl, const TcParams& p, int num_ctas, size_t smem,
                     cudaStream_t st) {
  cudaError_t err = cudaFuncSetAttribute(fused_tc_kernel<K, G>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  fused_tc_kernel<K, G><<<num_ctas, kThreadsG(G), smem, st>>>(mAh, mAl, mBh, mBl, p);
  return cudaGetLastError();
}

}  // namespace

bool tc_available() { return encode_fn() != nullptr; }

size_t fused_tc_smem_bytes(bool split, int kmax, int Lmax, int G) {
  const uint32_t stage = split ? 2 * kTileA + 2 * kTileB : kTileA + kTileB;
  return 1024 + (size_t)pick_stages(split, kmax, Lmax, G) * stage +
         epilogue_bytes(kmax, Lmax, G);
}

cudaError_t launch_fused_tc(const void* hi, const void* lo, bool split, const TcArgs& a,
                            const TcWork& w, const SeriesTable& sr, int num_ctas, cudaStream_t st) {
  if (a.Dp % KC != 0) return cudaErrorInvalidValue;
  CUtensorMap mAh, mAl, mBh, mBl;
  if (!make_map(&mAh, hi, a.rows, a.Dp, BM) || !make_map(&mBh, hi, a.rows, a.Dp, BN))
    return cudaErrorNotSupported;
  if (split) {
    if (!make_map(&mAl, lo, a.rows, a.Dp, BM) || !make_map(&mBl, lo, a.rows, a.Dp, BN))
      return cudaErrorNotSupported;
  } else {
    mAl = mAh;
    mBl = mBh;
  }
  thread_local TcParams p;  // large (series table): kept off the stack
  p.a = a;
  p.w = w;
  p.sr = sr;
  p.split = split ? 1 : 0;
  p.stage_bytes = split ? 2 * kTileA + 2 * kTileB : kTileA + kTileB;
  const int G = a.egroups;
  // two epilogue groups: L = 1, one accumulation segment, k <= 32 (host-checked here
  // too: the kernel's two-group form has no window, carry or segment folding)
  if (G != 1 && (G != 2 || a.Lmax != 1 || a.kmax > 32 || a.Dp > a.seg_k))
    return cudaErrorInvalidValue;
  p.nstages = pick_stages(split, a.kmax, a.Lmax, G);
  if (p.nstages < 2) return cudaErrorInvalidValue;
  if (a.seg_k < KC || a.seg_k % KC != 0) return cudaErrorInvalidValue;
  p.seg_kb = a.seg_k / KC;
  const size_t smem = fused_tc_smem_bytes(split, a.kmax, a.Lmax, G);
  const int k = a.kmax;
  if (G == 2) {
    if (k <= 4) return launch_k<4, 2>(mAh, mAl, mBh, mBl, p, num_ctas, smem, st);
    if (k <= 8) return launch_k<8, 2>(mAh, mAl, mBh, mBl, p, num_ctas, smem, st);
    if (k <= 10) return launch_k<10, 2>(mAh, mAl, mBh, mBl, p, num_ctas, smem, st);
    if (k <= 16) return launch_k<16, 2>(mAh, mAl, mBh, mBl, p, num_ctas, smem, st);
    if (k <= 20) return launch_k<20, 2>(mAh, mAl, mBh, mBl, p, num_ctas, smem, st);
    return launch_k<32, 2>(mAh, mAl, mBh, mBl, p, num_ctas, smem, st);
  }
  if (k <= 4) return launch_k<4, 1>(mAh, mAl, mBh, mBl, p, num_ctas, smem, st);
  if (k <= 8) return launch_k<8, 1>(mAh, mAl, mBh, mBl, p, num_ctas, smem, st);
  if (k <= 10) return launch_k<10, 1>(mAh, mAl, mBh, mBl, p, num_ctas, smem, st);
  if (k <= 16) return launch_k<16, 1>(mAh, mAl, mBh, mBl, p, num_ctas, smem, st);
  if (k <= 20) return launch_k<20, 1>(mAh, mAl, mBh, mBl, p, num_ctas, smem, st);
  if (k <= 32) return launch_k<32, 1>(mAh, mAl, mBh, mBl, p, num_ctas, smem, st);
  if (k <= 40) return launch_k<40, 1>(mAh, mAl, mBh, mBl, p, num_ctas, smem, st);
  if (k <= 48) return launch_k<48, 1>(mAh, mAl, mBh, mBl, p, num_ctas, smem, st);
  return launch_k<64, 1>(mAh, mAl, mBh, mBl, p, num_ctas, smem, st);
}

}  // namespace traknn
