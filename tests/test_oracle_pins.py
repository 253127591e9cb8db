"""Pins for the FP64 oracle: each check compares it with something other than itself
(hand-derived values, closed forms, library routines on special cases, exact
identities and invariants), so that a dropped term, a wrong index or sign, a
transposed operand or a wrong tie-break in the oracle fails at least one test."""
import numpy as np
import pytest
from scipy.spatial.distance import cdist

import oracle
from conftest import load_golden
from synth import make_slp_like


def _traj_vectors(X, L):
    """Trajectory tensors T_t = (X_t, ..., X_{t+L-1}) flattened (Sec. 3.2, Eq. 1)."""
    N = X.shape[0]
    M = N - L + 1
    return np.stack([X[t:t + L].reshape(-1) for t in range(M)]).astype(np.float64)


def _brute_knn(X, L, k, e):
    """Neighbours from the Frobenius form of Eq. 2 (scipy cdist on trajectory tensors)."""
    T = _traj_vectors(X, L)
    Dm = cdist(T, T, "sqeuclidean")
    M = T.shape[0]
    idx = np.empty((M, k), dtype=np.int64)
    dist = np.empty((M, k))
    for t in range(M):
        j = np.arange(M)
        keep = np.abs(j - t) > e
        order = np.lexsort((j[keep], Dm[t, keep]))[:k]
        idx[t] = j[keep][order]
        dist[t] = Dm[t, keep][order]
    return idx, dist, Dm


# ----------------------------------------------------------- hand-worked example

@pytest.mark.parametrize("case", ["A", "B"])
def test_hand_example(case):
    Xrows, cases = load_golden("hand_example_6days.txt")
    X = np.array(Xrows, dtype=np.float32)
    params, rows = cases[case]
    idx, dist, score = oracle.knn_scores(X, params["L"], params["k"], params["e"])
    assert idx.shape[0] == len(rows)
    for t, (gi, gd, gs) in rows.items():
        assert list(idx[t]) == gi
        assert list(dist[t]) == gd
        assert score[t] == gs


# ----------------------------------------------------------------- closed forms

def test_linear_days_closed_form():
    """X_t = t v: S(a,b) = (a-b)^2 |v|^2, D(t,j) = L (t-j)^2 |v|^2 exactly; the
    neighbours are the nearest allowed time gaps, earlier day first on ties."""
    N, L, e, k = 40, 4, 3, 5
    v = np.array([1.0, -2.0, 3.0, 0.0, 2.0], dtype=np.float32)
    c = float(v @ v)
    X = (np.arange(N, dtype=np.float32)[:, None] * v[None, :]).astype(np.float32)
    S = oracle.snapshot_matrix(X)
    a = np.arange(N)
    assert np.array_equal(S, ((a[:, None] - a[None, :]) ** 2) * c)
    M = N - L + 1
    idx, dist, score = oracle.knn_scores(X, L, k, e)
    for t in range(M):
        # enumerate candidates by increasing gap g > e: (t-g, t+g), smaller index first
        exp = []
        g = e + 1
        while len(exp) < k:
            for j in (t - g, t + g):
                if 0 <= j < M and len(exp) < k:
                    exp.append(j)
            g += 1
        assert list(idx[t]) == exp
        exp_d = [L * (t - j) ** 2 * c for j in exp]
        assert list(dist[t]) == exp_d
        assert score[t] == sum(exp_d) / k


def test_circular_days_closed_form():
    """X_t = r (cos(w t) u + sin(w t) q), u, q orthonormal:
    S(a,b) = 2 r^2 (1 - cos(w (a-b))), so D(t,j) = 2 L r^2 (1 - cos(w (t-j)))."""
    rng = np.random.default_rng(5)
    Dg, N, L, r, w = 24, 50, 6, 3.0, 0.37
    Q, _ = np.linalg.qr(rng.standard_normal((Dg, 2)))
    t = np.arange(N)
    X64 = r * (np.cos(w * t)[:, None] * Q[:, 0] + np.sin(w * t)[:, None] * Q[:, 1])
    X = X64.astype(np.float32)
    S = oracle.snapshot_matrix(X)
    exact = 2 * r * r * (1 - np.cos(w * (t[:, None] - t[None, :])))
    assert np.allclose(S, exact, rtol=1e-5, atol=1e-5)
    Dt = oracle.traj_matrix(S, L)
    M = N - L + 1
    tt = np.arange(M)
    assert np.allclose(Dt, L * 2 * r * r * (1 - np.cos(w * (tt[:, None] - tt[None, :]))),
                       rtol=1e-5, atol=1e-4)


# ------------------------------------------------------- library / brute force

@pytest.mark.parametrize("N,Dg,L,e,k", [(12, 3, 1, 0, 2), (12, 4, 3, 2, 3), (30, 7, 5, 4, 4),
                                         (25, 2, 2, 0, 6)])
def test_matches_cdist_bruteforce(N, Dg, L, e, k):
    rng = np.random.default_rng(N * 100 + L)
    X = rng.standard_normal((N, Dg)).astype(np.float32)
    bidx, bdist, Dm = _brute_knn(X, L, k, e)
    idx, dist, score, Dt = oracle.knn_scores(X, L, k, e, return_D=True)
    assert np.allclose(Dt, Dm, rtol=1e-12, atol=1e-12)
    assert np.array_equal(idx, bidx)
    assert np.allclose(dist, bdist, rtol=1e-12)
    assert np.allclose(score, bdist.mean(axis=1), rtol=1e-12)


def test_snapshot_matrix_vs_cdist():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((33, 17)).astype(np.float32)
    assert np.allclose(oracle.snapshot_matrix(X), cdist(X.astype(np.float64),
                                                        X.astype(np.float64), "sqeuclidean"),
                       rtol=1e-12, atol=1e-12)


def test_traj_rows_match_tensor_form():
    """Row-sampled distances (computed from X directly) equal the Frobenius form of Eq. 2."""
    rng = np.random.default_rng(11)
    X = rng.standard_normal((60, 9)).astype(np.float32)
    L = 4
    rows = np.array([0, 7, 30, 56])
    T = _traj_vectors(X, L)
    ref = cdist(T[rows], T, "sqeuclidean")
    assert np.allclose(oracle.traj_rows(X, L, rows), ref, rtol=1e-12, atol=1e-12)


def test_snapshot_case_L1_is_textbook_knn():
    """L = 1 reduces to snapshot kNN with the self match excluded (e = 0)."""
    rng = np.random.default_rng(2)
    X = rng.standard_normal((50, 6)).astype(np.float32)
    k = 5
    Dm = cdist(X.astype(np.float64), X.astype(np.float64), "sqeuclidean")
    np.fill_diagonal(Dm, np.inf)
    ref = np.argsort(Dm, axis=1, kind="stable")[:, :k]
    idx, dist, score = oracle.knn_scores(X, 1, k, 0)
    assert np.array_equal(idx, ref)
    assert np.allclose(score, np.take_along_axis(Dm, ref, 1).mean(1), rtol=1e-12)


# ------------------------------------------------------- exact identities

def test_recurrence_eq5_matches_explicit_sum():
    """The constant-time recurrence (Sec. 3.3, Eq. 5), run in FP64 from the first row
    and first column, reproduces the oracle's explicit L-term sums."""
    rng = np.random.default_rng(7)
    X = rng.standard_normal((80, 13)).astype(np.float32)
    L = 6
    S = oracle.snapshot_matrix(X)
    Dt = oracle.traj_matrix(S, L)
    M = S.shape[0] - L + 1
    R = np.empty((M, M))
    for j in range(M):
        R[0, j] = sum(S[m, j + m] for m in range(L))
        R[j, 0] = sum(S[j + m, m] for m in range(L))
    for t in range(1, M):
        for j in range(1, M):
            R[t, j] = R[t - 1, j - 1] - S[t - 1, j - 1] + S[t + L - 1, j + L - 1]
    assert np.allclose(R, Dt, rtol=1e-12, atol=1e-9)


def test_symmetry_and_zero_diagonal():
    rng = np.random.default_rng(8)
    X = rng.standard_normal((40, 11)).astype(np.float32)
    Dt = oracle.traj_matrix(oracle.snapshot_matrix(X), 3)
    assert np.array_equal(Dt, Dt.T)
    assert np.all(np.diag(Dt) == 0.0)
    assert np.all(Dt >= 0.0)


def test_constant_offset_invariance():
    """Adding one fixed field to every day changes no distance, neighbour or score.
    Values sit on a 1/64 grid so that X + F is exact in float32."""
    rng = np.random.default_rng(9)
    X = (np.round(rng.standard_normal((45, 10)) * 64) / 64).astype(np.float32)
    F = rng.integers(-1000, 1000, size=(1, 10)).astype(np.float32)
    a = oracle.knn_scores(X, 4, 3, 3)
    b = oracle.knn_scores(X + F, 4, 3, 3)
    for u, v in zip(a, b):
        assert np.array_equal(u, v)


def test_k_prefix_property():
    """The neighbour list for k' < k is the first k' entries of the list for k (Sec. 6)."""
    rng = np.random.default_rng(10)
    X = rng.standard_normal((70, 5)).astype(np.float32)
    big = oracle.knn_scores(X, 3, 12, 2)
    for kp in (1, 4, 7):
        small = oracle.knn_scores(X, 3, kp, 2)
        assert np.array_equal(small[0], big[0][:, :kp])
        assert np.allclose(small[2], big[1][:, :kp].mean(1), rtol=1e-12)


def test_k1_is_matrix_profile():
    """For k = 1 the score is the spatiotemporal matrix profile min_j D(t,j) (Sec. 6)."""
    rng = np.random.default_rng(12)
    X = rng.standard_normal((64, 6)).astype(np.float32)
    L, e = 4, 3
    _, _, Dm = _brute_knn(X, L, 1, e)
    M = Dm.shape[0]
    j = np.arange(M)
    mp = np.array([Dm[t, np.abs(j - t) > e].min() for t in range(M)])
    _, _, score = oracle.knn_scores(X, L, 1, e)
    assert np.allclose(score, mp, rtol=1e-12)


def test_kk_continues_sorted_order():
    rng = np.random.default_rng(13)
    X = rng.standard_normal((30, 4)).astype(np.float32)
    bidx, bdist, _ = _brute_knn(X, 2, 9, 1)
    idx, dist, score = oracle.knn_scores(X, 2, 5, 1, kk=9)
    assert np.array_equal(idx, bidx)
    assert np.allclose(score, bdist[:, :5].mean(1), rtol=1e-12)


def test_too_few_candidates_is_an_error():
    X = np.zeros((6, 2), dtype=np.float32)
    with pytest.raises(RuntimeError):
        oracle.knn_scores(X, 2, 3, 1)   # M=5, middle row has 5-3=2 candidates < 3


# ------------------------------------------------------- planted anomaly

def test_planted_anomaly_ranks_first():
    X, meta = make_slp_like(400, 8, 16, seed=77, n_planted=1, planted_len=3,
                            planted_sigma=6.0)
    L, k, e = 3, 5, 2
    _, _, score = oracle.knn_scores(X, L, k, e)
    s0 = meta.planted_starts[0]
    assert abs(int(np.argmax(score)) - s0) <= L - 1


# ------------------------------------------------------- adjoint

def _score_sum_numpy(X64, L, k, idx, g):
    """sum_t g_t s_t with fixed neighbour sets, via trajectory tensors (Eq. 1-3)."""
    T = _traj_vectors(X64, L)
    tot = 0.0
    for t in range(idx.shape[0]):
        d = ((T[t][None, :] - T[idx[t]]) ** 2).sum(axis=1)
        tot += g[t] * d.sum() / k
    return tot


def test_score_grad_matches_finite_differences():
    """With the neighbour sets fixed the summed score is quadratic in X, so central
    differences are exact up to rounding."""
    rng = np.random.default_rng(14)
    N, Dg, L, k, e = 30, 5, 3, 4, 2
    X = rng.standard_normal((N, Dg)).astype(np.float32)
    idx, _, _ = oracle.knn_scores(X, L, k, e)
    M = N - L + 1
    g = rng.uniform(0.5, 2.0, size=M)
    G = oracle.score_grad(X, L, k, idx, g)
    X64 = X.astype(np.float64)
    h = 1e-3
    for a, p in [(0, 0), (5, 3), (14, 1), (N - 1, 4), (N - 2, 2), (17, 0)]:
        Xp = X64.copy(); Xp[a, p] += h
        Xm = X64.copy(); Xm[a, p] -= h
        fd = (_score_sum_numpy(Xp, L, k, idx, g) - _score_sum_numpy(Xm, L, k, idx, g)) / (2 * h)
        assert abs(fd - G[a, p]) <= 1e-8 * max(1.0, abs(fd))


def test_score_grad_matches_torch_autograd():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(15)
    N, Dg, L, k, e = 36, 6, 4, 3, 3
    X = rng.standard_normal((N, Dg)).astype(np.float32)
    idx, _, _ = oracle.knn_scores(X, L, k, e)
    M = N - L + 1
    g = rng.uniform(0.1, 1.0, size=M)
    Xt = torch.tensor(X, dtype=torch.float64, requires_grad=True)
    T = torch.stack([Xt[t:t + L].reshape(-1) for t in range(M)])
    it = torch.tensor(idx, dtype=torch.long)
    D = ((T[:, None, :] - T[it]) ** 2).sum(-1)          # (M, k)
    F = (torch.tensor(g) * D.mean(1)).sum()
    F.backward()
    G = oracle.score_grad(X, L, k, idx, g)
    assert np.allclose(G, Xt.grad.numpy(), rtol=1e-10, atol=1e-10)
