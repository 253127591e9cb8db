"""Pins of the oracle's extensions against facts the definitions fix: grid-point
weights (exact scalings and reductions), scores for every k' <= k (brute force and
the nesting of neighbour sets, Sec. 6), and the Levina-Bickel local intrinsic
dimension used in the paper's intrinsic dimension study (Sec. 4)."""
import numpy as np
import pytest

import oracle
from synth import make_slp_like


@pytest.fixture(scope="module")
def small():
    X, _ = make_slp_like(160, 4, 6, seed=11)
    return X


def test_unit_weights_reproduce_unweighted_bitwise(small):
    w = np.ones(small.shape[1])
    assert np.array_equal(oracle.snapshot_matrix(small, weights=w), oracle.snapshot_matrix(small))
    a = oracle.knn_scores(small, 4, 5, 3, weights=w)
    b = oracle.knn_scores(small, 4, 5, 3)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_constant_weights_scale_every_distance_exactly(small):
    w = np.full(small.shape[1], 4.0)  # a power of two: exact in FP64
    S4 = oracle.snapshot_matrix(small, weights=w)
    assert np.array_equal(S4, 4.0 * oracle.snapshot_matrix(small))
    i4, d4, s4 = oracle.knn_scores(small, 3, 6, 2, weights=w)
    i1, d1, s1 = oracle.knn_scores(small, 3, 6, 2)
    assert np.array_equal(i4, i1) and np.array_equal(d4, 4.0 * d1) and np.array_equal(s4, 4.0 * s1)


def test_indicator_weights_equal_the_selected_grid_points(small):
    rng = np.random.default_rng(3)
    keep = rng.random(small.shape[1]) < 0.5
    w = keep.astype(np.float64)
    Sw = oracle.snapshot_matrix(small, weights=w)
    Ss = oracle.snapshot_matrix(small[:, keep])
    assert np.allclose(Sw, Ss, rtol=1e-13, atol=0)
    rows = np.array([0, 17, 80, 152])
    Dw = oracle.traj_rows(small, 5, rows, weights=w)
    Ds = oracle.traj_rows(small[:, keep], 5, rows)
    assert np.allclose(Dw, Ds, rtol=1e-13, atol=0)


def test_weighted_adjoint(small):
    L, k = 3, 4
    idx, _, _ = oracle.knn_scores(small, L, k, L - 1)
    g = np.linspace(0.5, 1.5, idx.shape[0])
    base = oracle.score_grad(small, L, k, idx, g)
    assert np.array_equal(oracle.score_grad(small, L, k, idx, g, weights=np.ones(small.shape[1])),
                          base)
    keep = np.arange(small.shape[1]) % 3 != 0
    gw = oracle.score_grad(small, L, k, idx, g, weights=keep.astype(float))
    assert np.all(gw[:, ~keep] == 0.0)
    gs = oracle.score_grad(small[:, keep], L, k, idx, g)
    assert np.allclose(gw[:, keep], gs, rtol=1e-12, atol=1e-12)


def _brute_prefix(X, L, k, e):
    """Independent numpy evaluation: D by explicit day differences, candidates sorted by
    (distance, index), mean of the first k' for every k'."""
    X = X.astype(np.float64)
    N = X.shape[0]
    M = N - L + 1
    out = np.empty((M, k))
    for t in range(M):
        cands = []
        for j in range(M):
            if abs(t - j) > e:
                d = sum(float(np.sum((X[t + m] - X[j + m]) ** 2)) for m in range(L))
                cands.append((d, j))
        cands.sort()
        ds = np.array([c[0] for c in cands[:k]])
        out[t] = np.cumsum(ds) / np.arange(1, k + 1)
    return out


def test_prefix_scores_brute_force():
    X, _ = make_slp_like(14, 2, 3, seed=4)
    got = oracle.prefix_scores(X, 3, 5, 2)
    assert np.allclose(got, _brute_prefix(X, 3, 5, 2), rtol=1e-12, atol=0)


def test_neighbour_sets_are_nested_in_k(small):
    """Sec. 6: the top-k' neighbours are the first k' of the top-k list."""
    ik, _, _ = oracle.knn_scores(small, 4, 8, 3)
    for kp in (1, 3, 5):
        ip, _, _ = oracle.knn_scores(small, 4, kp, 3)
        assert np.array_equal(ip, ik[:, :kp])
    ps = oracle.prefix_scores(small, 4, 8, 3)
    _, d8, _ = oracle.knn_scores(small, 4, 8, 3)
    assert np.allclose(ps[:, 4], d8[:, :5].mean(axis=1), rtol=1e-13, atol=0)


def test_local_id_closed_form_and_undefined_rows():
    # squared distances 1, 4, 9, 16: T = 1, 2, 3, 4
    d = np.array([[1.0, 4.0, 9.0, 16.0], [0.0, 1.0, 2.0, 3.0], [2.0, 2.0, 2.0, 2.0]])
    got = oracle.local_id(d, 4)
    want = 3.0 / (np.log(4.0) + np.log(2.0) + np.log(4.0 / 3.0))
    assert got[0] == pytest.approx(want, rel=1e-14)
    assert np.isnan(got[1]) and np.isnan(got[2])
    # k = 3 uses the first three entries only
    assert oracle.local_id(d[:1], 3)[0] == pytest.approx(2.0 / np.log(4.5), rel=1e-14)


def test_local_id_is_scale_invariant(small):
    _, d1, _ = oracle.knn_scores(small, 2, 10, 1)
    _, d2, _ = oracle.knn_scores(small * 8.0, 2, 10, 1)
    assert np.allclose(oracle.local_id(d1, 10), oracle.local_id(d2, 10), rtol=1e-9)


def test_local_id_of_a_three_dimensional_cube_in_thirty_dimensions():
    rng = np.random.default_rng(7)
    n, dim, amb = 1500, 3, 30
    Q, _ = np.linalg.qr(rng.standard_normal((amb, dim)))
    X = (rng.random((n, dim)) @ Q.T).astype(np.float32)
    _, dist, _ = oracle.knn_scores(X, 1, 20, 0)
    m = np.nanmean(oracle.local_id(dist, 20))
    assert 2.5 < m < 3.4, m
