/*
 * traknn_oracle.c -- plain FP64 CPU oracle for the trajectory-kNN rarity score
 * of TRAKNN (arXiv 2603.02059).
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this code. The CUDA library never
 * calls it and shares no code, header or constant with it.
 *
 * Every quantity is computed straight from the paper's definitions, in
 * double precision, with no Gram identity, no recurrence, no blocking and no
 * pruning:
 *
 *   snapshot distance  S(a,b) = sum_p (X[a,p] - X[b,p])^2
 *                      (the inner term of Sec. 3.2, Eq. 2, by direct differences)
 *   trajectory distance D(t,j) = sum_{m=0}^{L-1} S(t+m, j+m)
 *                      (Sec. 3.2, Eq. 2, an explicit L-term sum)
 *   candidates of t    { j : |t - j| > e }            (Sec. 3.2, exclusion zone)
 *   neighbour set N_t  first k candidates after a full sort by (D(t,j), j)
 *                      (Algorithm 1, kNN step; ties go to the smaller index)
 *   rarity score       s_t = (1/k) sum_{j in N_t} D(t,j)  (Sec. 3.2, Eq. 3)
 *
 * Indices are 0-based; there are M = N - L + 1 trajectories (the paper's
 * n - d + 1, Algorithm 1 output).
 *
 * The adjoint (oracle_score_grad) is the derivative of sum_t g_t s_t with the
 * neighbour sets held fixed, written out from Eq. 2 and Eq. 3:
 *   d/dX[a] = sum_t (2 g_t / k) sum_{j in N_t} sum_m (X[t+m] - X[j+m])
 *                                   * ([a == t+m] - [a == j+m]).
 *
 * Optional grid-point weights w_p >= 0 (the *_w entry points; NULL = all ones)
 * turn the snapshot distance into sum_p w_p (X[a,p] - X[b,p])^2, e.g. area
 * weights proportional to the cosine of latitude (Sec. 5, composite analysis);
 * the adjoint then carries the same factor w_p.
 *
 * Parity pins: every function here is checked by tests against closed forms,
 * invariants and brute-force enumerations (see tests/test_oracle_pins.py).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define ORACLE_OK 0
#define ORACLE_ERR_ARGS 1
#define ORACLE_ERR_FEW_CANDIDATES 2
#define ORACLE_ERR_NOMEM 3

/* ---------------------------------------------------------------- threads */

typedef void (*row_fn)(void* ctx, int64_t row);

typedef struct {
  row_fn fn;
  void* ctx;
  int64_t nrows;
  int tid, nthreads;
} worker_arg;

static void* worker_main(void* p) {
  worker_arg* w = (worker_arg*)p;
  /* interleaved assignment keeps triangular work balanced */
  for (int64_t r = w->tid; r < w->nrows; r += w->nthreads) w->fn(w->ctx, r);
  return NULL;
}

static int resolve_threads(int nthreads) {
  if (nthreads > 0) return nthreads;
  long n = sysconf(_SC_NPROCESSORS_ONLN);
  return n > 0 ? (int)n : 1;
}

static void parallel_rows(row_fn fn, void* ctx, int64_t nrows, int nthreads) {
  nthreads = resolve_threads(nthreads);
  if (nthreads > nrows) nthreads = (int)(nrows > 0 ? nrows : 1);
  pthread_t th[256];
  worker_arg args[256];
  if (nthreads > 256) nthreads = 256;
  for (int i = 0; i < nthreads; ++i) {
    args[i].fn = fn; args[i].ctx = ctx; args[i].nrows = nrows;
    args[i].tid = i; args[i].nthreads = nthreads;
  }
  for (int i = 1; i < nthreads; ++i) pthread_create(&th[i], NULL, worker_main, &args[i]);
  worker_main(&args[0]);
  for (int i = 1; i < nthreads; ++i) pthread_join(th[i], NULL);
}

int oracle_num_threads(int nthreads) { return resolve_threads(nthreads); }

/* ------------------------------------------------ Eq. 2, snapshot term */

/* S(a,b) by direct differences of the two days' fields (weighted when w != NULL). */
static double snapshot_sqdist(const float* X, int64_t D, const double* w, int64_t a, int64_t b) {
  const float* xa = X + a * D;
  const float* xb = X + b * D;
  double s = 0.0;
  for (int64_t p = 0; p < D; ++p) {
    double d = (double)xa[p] - (double)xb[p];
    s += w ? w[p] * (d * d) : d * d;
  }
  return s;
}

typedef struct {
  const float* X;
  int64_t N, D;
  const double* w;
  double* S;
} smat_ctx;

static void smat_row(void* p, int64_t a) {
  smat_ctx* c = (smat_ctx*)p;
  c->S[a * c->N + a] = 0.0;
  for (int64_t b = a + 1; b < c->N; ++b) {
    double s = snapshot_sqdist(c->X, c->D, c->w, a, b);
    c->S[a * c->N + b] = s;
    c->S[b * c->N + a] = s;
  }
}

/* Full N x N snapshot distance matrix (row-major); w: [D] weights or NULL. */
int oracle_snapshot_matrix_w(const float* X, int64_t N, int64_t D, const double* w, double* S,
                             int nthreads) {
  if (!X || !S || N < 1 || D < 1) return ORACLE_ERR_ARGS;
  smat_ctx c = {X, N, D, w, S};
  parallel_rows(smat_row, &c, N, nthreads);
  return ORACLE_OK;
}

int oracle_snapshot_matrix(const float* X, int64_t N, int64_t D, double* S, int nthreads) {
  return oracle_snapshot_matrix_w(X, N, D, NULL, S, nthreads);
}

/* ------------------------------------------------ Eq. 2, trajectory sum */

/* D(t,j) = sum_{m<L} S(t+m, j+m) for all t, j in [0, M), from a full S. */
int oracle_traj_matrix(const double* S, int64_t N, int L, double* Dt) {
  if (!S || !Dt || L < 1 || L > N) return ORACLE_ERR_ARGS;
  int64_t M = N - L + 1;
  for (int64_t t = 0; t < M; ++t)
    for (int64_t j = 0; j < M; ++j) {
      double s = 0.0;
      for (int m = 0; m < L; ++m) s += S[(t + m) * N + (j + m)];
      Dt[t * M + j] = s;
    }
  return ORACLE_OK;
}

typedef struct {
  const float* X;
  int64_t N, D, M;
  int L;
  const double* w;
  const int64_t* rows;
  double* out;
} trows_ctx;

static void trows_row(void* p, int64_t r) {
  trows_ctx* c = (trows_ctx*)p;
  int64_t t = c->rows[r];
  double* out = c->out + r * c->M;
  for (int64_t j = 0; j < c->M; ++j) out[j] = 0.0;
  /* add the L snapshot terms of Eq. 2, one day offset m at a time */
  for (int m = 0; m < c->L; ++m)
    for (int64_t j = 0; j < c->M; ++j)
      out[j] += snapshot_sqdist(c->X, c->D, c->w, t + m, j + m);
}

/* Rows of the trajectory distance matrix, computed from X directly: for each
 * requested t, out[r*M + j] = D(t, j) for every j in [0, M). */
int oracle_traj_rows_w(const float* X, int64_t N, int64_t D, int L, const double* w,
                       const int64_t* rows, int64_t nrows, double* out, int nthreads) {
  if (!X || !rows || !out || L < 1 || L > N || D < 1) return ORACLE_ERR_ARGS;
  int64_t M = N - L + 1;
  for (int64_t r = 0; r < nrows; ++r)
    if (rows[r] < 0 || rows[r] >= M) return ORACLE_ERR_ARGS;
  trows_ctx c = {X, N, D, M, L, w, rows, out};
  parallel_rows(trows_row, &c, nrows, nthreads);
  return ORACLE_OK;
}

int oracle_traj_rows(const float* X, int64_t N, int64_t D, int L, const int64_t* rows,
                     int64_t nrows, double* out, int nthreads) {
  return oracle_traj_rows_w(X, N, D, L, NULL, rows, nrows, out, nthreads);
}

/* ------------------------------------------ kNN set and score (Eq. 3) */

typedef struct {
  double d;
  int64_t j;
} cand;

static int cand_cmp(const void* pa, const void* pb) {
  const cand* a = (const cand*)pa;
  const cand* b = (const cand*)pb;
  if (a->d < b->d) return -1;
  if (a->d > b->d) return 1;
  return (a->j < b->j) ? -1 : (a->j > b->j);
}

/* One row: full sort of all candidates |t-j| > e by (D, j), keep k.
 * kk entries (kk >= k) are written so that tests can look past the k-th. */
static int knn_one_row(const double* drow, int64_t t, int64_t M, int k, int kk, int e,
                       int32_t* idx, double* dist, double* score, cand* buf) {
  int64_t n = 0;
  for (int64_t j = 0; j < M; ++j) {
    int64_t gap = t > j ? t - j : j - t;
    if (gap > e) { buf[n].d = drow[j]; buf[n].j = j; ++n; }
  }
  if (n < k) return ORACLE_ERR_FEW_CANDIDATES;
  qsort(buf, (size_t)n, sizeof(cand), cand_cmp);
  double s = 0.0;
  for (int i = 0; i < k; ++i) s += buf[i].d;
  *score = s / (double)k;
  for (int i = 0; i < kk; ++i) {
    if (i < n) { idx[i] = (int32_t)buf[i].j; dist[i] = buf[i].d; }
    else { idx[i] = -1; dist[i] = INFINITY; }
  }
  return ORACLE_OK;
}

/* kNN + score for rows given their full distance rows (nrows x M).
 * idx/dist receive kk >= k entries per row (sorted by (D, j)). */
int oracle_knn_from_rows(const double* Drows, const int64_t* rows, int64_t nrows, int64_t M,
                         int k, int kk, int e, int32_t* idx, double* dist, double* score) {
  if (!Drows || !rows || !idx || !dist || !score || k < 1 || kk < k || e < 0) return ORACLE_ERR_ARGS;
  cand* buf = (cand*)malloc(sizeof(cand) * (size_t)M);
  if (!buf) return ORACLE_ERR_NOMEM;
  int rc = ORACLE_OK;
  for (int64_t r = 0; r < nrows && rc == ORACLE_OK; ++r)
    rc = knn_one_row(Drows + r * M, rows[r], M, k, kk, e, idx + r * kk, dist + r * kk,
                     score + r, buf);
  free(buf);
  return rc;
}

/* Whole pipeline for all M trajectories (small N only: it stores S and D). */
int oracle_knn_scores_w(const float* X, int64_t N, int64_t D, int L, const double* w, int k,
                        int kk, int e, int32_t* idx, double* dist, double* score, double* Dt_out,
                        int nthreads) {
  if (!X || L < 1 || L > N || k < 1 || kk < k || e < 0) return ORACLE_ERR_ARGS;
  int64_t M = N - L + 1;
  double* S = (double*)malloc(sizeof(double) * (size_t)(N * N));
  double* Dt = Dt_out ? Dt_out : (double*)malloc(sizeof(double) * (size_t)(M * M));
  int64_t* rows = (int64_t*)malloc(sizeof(int64_t) * (size_t)M);
  if (!S || !Dt || !rows) {
    free(S); if (!Dt_out) free(Dt); free(rows);
    return ORACLE_ERR_NOMEM;
  }
  int rc = oracle_snapshot_matrix_w(X, N, D, w, S, nthreads);
  if (rc == ORACLE_OK) rc = oracle_traj_matrix(S, N, L, Dt);
  for (int64_t t = 0; t < M; ++t) rows[t] = t;
  if (rc == ORACLE_OK) rc = oracle_knn_from_rows(Dt, rows, M, M, k, kk, e, idx, dist, score);
  free(S); free(rows);
  if (!Dt_out) free(Dt);
  return rc;
}

int oracle_knn_scores(const float* X, int64_t N, int64_t D, int L, int k, int kk, int e,
                      int32_t* idx, double* dist, double* score, double* Dt_out, int nthreads) {
  return oracle_knn_scores_w(X, N, D, L, NULL, k, kk, e, idx, dist, score, Dt_out, nthreads);
}

/* ------------------------------------- adjoint with fixed neighbour sets */

/* dX (N x D, overwritten) = d( sum_t g[t] s_t ) / dX, neighbour sets idx
 * (M x k) held fixed. Accumulated in FP64 exactly as the formula reads. */
int oracle_score_grad_w(const float* X, int64_t N, int64_t D, int L, const double* wgt, int k,
                        const int32_t* idx, const double* g, double* dX) {
  if (!X || !idx || !g || !dX || L < 1 || L > N || k < 1) return ORACLE_ERR_ARGS;
  int64_t M = N - L + 1;
  memset(dX, 0, sizeof(double) * (size_t)(N * D));
  for (int64_t t = 0; t < M; ++t) {
    double w = 2.0 * g[t] / (double)k;
    for (int i = 0; i < k; ++i) {
      int64_t j = idx[t * k + i];
      if (j < 0 || j >= M) return ORACLE_ERR_ARGS;
      for (int m = 0; m < L; ++m) {
        const float* xa = X + (t + m) * D;
        const float* xb = X + (j + m) * D;
        double* ga = dX + (t + m) * D;
        double* gb = dX + (j + m) * D;
        for (int64_t p = 0; p < D; ++p) {
          double diff = (double)xa[p] - (double)xb[p];
          if (wgt) diff *= wgt[p];
          ga[p] += w * diff;
          gb[p] -= w * diff;
        }
      }
    }
  }
  return ORACLE_OK;
}

int oracle_score_grad(const float* X, int64_t N, int64_t D, int L, int k, const int32_t* idx,
                      const double* g, double* dX) {
  return oracle_score_grad_w(X, N, D, L, NULL, k, idx, g, dX);
}
