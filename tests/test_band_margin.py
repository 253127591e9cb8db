"""The error bound behind the one-product band pre-pass, checked on the CPU.

For split-BF16 calls with long operand rows the band pre-pass (which only seeds the
rows' upper bounds) evaluates the Gram in one BF16 product, hi_a . hi_b with
hi = bf16(x), and raises every trajectory distance by m (W_t + W_j) before it may
become a bound, with

    m = 2u + u^2 + 2.1 Dp 2^-23 + 2^-19,   u = 2^-8 (BF16 unit roundoff),

so that a raised distance is never below the exact one and no true neighbour can be
pruned. The derivation: |a.b - hi_a.hi_b| <= (2u + u^2) ||a|| ||b|| by Cauchy-Schwarz;
the FP32 accumulation of the Dp products and of one correction product per group of
64 entries (magnitudes summing to about 2 ||a|| ||b||) adds at most
2.1 Dp 2^-23 ||a|| ||b||, even with every add truncated and in any order; and
2 ||a|| ||b|| <= n_a + n_b per day pair, summed over the window to W_t + W_j.

These tests emulate that arithmetic with numpy: BF16 round-to-nearest-even, the
grouped operand layout with its correction entries (c = bf16(sqrt(n / groups)),
added by the tensor cores and subtracted by the epilogue), products exact in FP32,
and FP32 sums truncated toward zero in three orders (sequential, 16-entry blocks as
the MMAs add them, reversed). They check the Gram error against the first two terms
on realistic fields and on adversarial rows whose every value sits next to a BF16
rounding midpoint (the leading term 2u is then nearly reached), and the raised
trajectory distance against the exact FP64 one."""
import numpy as np
import pytest

from synth import make_slp_like

U = 2.0 ** -8


def margin(Dp):
    """m of the band pre-pass for operand rows of Dp entries."""
    return 2 * U + U * U + 2.1 * Dp * 2.0 ** -23 + 2.0 ** -19


def gram_bound(Dp):
    """Bound of |G' - a.b| / (||a|| ||b||): the rounding and accumulation terms of m."""
    return 2 * U + U * U + 2.1 * Dp * 2.0 ** -23


def bf16(x):
    """Round float32 values to BF16 (nearest, ties to even), returned as float32."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def add_rtz(acc, t):
    """acc + t in FP32 with the result truncated toward zero (elementwise)."""
    s = acc.astype(np.float64) + t.astype(np.float64)
    r = s.astype(np.float32)
    over = np.abs(r.astype(np.float64)) > np.abs(s)
    r[over] = np.nextafter(r[over], np.float32(0))
    return r


def grouped(x, groups):
    """Operand row layout: group g holds grid points g, g + groups, ... (63 at most)
    and, as its last entry, the correction c = bf16(sqrt(n / groups)); returns the
    hi entries [rows, groups * 64] and c."""
    rows, D = x.shape
    n = (x.astype(np.float64) ** 2).sum(1)
    c = bf16(np.sqrt(n / groups).astype(np.float32))
    hi = np.zeros((rows, groups, 64), np.float32)
    h = bf16(x)
    for g in range(groups):
        pts = np.arange(g, D, groups)
        hi[:, g, :len(pts)] = h[:, pts]
        hi[:, g, 63] = c
    return hi.reshape(rows, groups * 64), c, n


def gram_one_product(a, b, groups, order):
    """G' for day pairs (a[i], b[i]): hi-only products accumulated in FP32 with
    truncated adds in the given order, then the correction groups c_a c_b subtracted
    with one FP32 rounding (the epilogue's fused multiply-add)."""
    ha, ca, na = grouped(a, groups)
    hb, cb, nb = grouped(b, groups)
    prod = ha * hb  # exact: two 8-bit significands
    Dp = prod.shape[1]
    acc = np.zeros(len(a), np.float32)
    if order == "sequential":
        for p in range(Dp):
            acc = add_rtz(acc, prod[:, p])
    elif order == "reversed":
        for p in range(Dp - 1, -1, -1):
            acc = add_rtz(acc, prod[:, p])
    else:  # blocks of 16 entries summed first, then added to the accumulator
        for p0 in range(0, Dp, 16):
            part = np.zeros(len(a), np.float32)
            for p in range(p0, p0 + 16):
                part = add_rtz(part, prod[:, p])
            acc = add_rtz(acc, part)
    crow = (-np.float32(groups) * ca).astype(np.float32)
    g = (acc.astype(np.float64) + crow.astype(np.float64) * cb.astype(np.float64))
    return g.astype(np.float32), na, nb, Dp


def adversarial_rows(D, seed):
    """Rows whose values sit just above or just below a BF16 rounding midpoint, with
    random signs shared by a and b (so that every rounding error adds up); the
    magnitudes lie just above 1, where an error of half a BF16 spacing (2^-8) is
    nearly the unit roundoff u relative to the value."""
    rng = np.random.default_rng(seed)
    mag = rng.uniform(1.0, 1.03, D).astype(np.float32)
    mid = bf16(mag) + np.float32(2.0 ** -8) * np.exp2(np.floor(np.log2(mag))).astype(np.float32)
    above = np.nextafter(mid.astype(np.float32), np.float32(2)).astype(np.float32)
    below = np.nextafter(mid.astype(np.float32), np.float32(0)).astype(np.float32)
    sign = np.where(rng.random(D) < 0.5, -1.0, 1.0).astype(np.float32)
    return (above * sign)[None, :], (below * sign)[None, :]


@pytest.mark.parametrize("order", ["sequential", "blocks16", "reversed"])
def test_gram_error_within_the_bound(order):
    D = 3726  # the 1-degree grid: 60 groups, Dp = 3,840
    groups = -(-D // 63)
    X, _ = make_slp_like(400, 46, 81, seed=5)
    X = (X - X.mean(0)).astype(np.float32)
    rng = np.random.default_rng(1)
    ia, ib = rng.integers(0, len(X), 120), rng.integers(0, len(X), 120)
    hi_above, hi_below = adversarial_rows(D, 2)
    a = np.concatenate([X[ia], X[:40], hi_above, hi_below, hi_above])
    b = np.concatenate([X[ib], X[1:41], hi_above, hi_below, -hi_above])
    g, na, nb, Dp = gram_one_product(a, b, groups, order)
    exact = (a.astype(np.float64) * b.astype(np.float64)).sum(1)
    ratio = np.abs(g.astype(np.float64) - exact) / np.sqrt(na * nb)
    assert Dp == 3840
    assert ratio.max() <= gram_bound(Dp), ratio.max()
    # the adversarial rows nearly reach the rounding term 2u (98 % of it): a bound with
    # a smaller rounding term would fail here
    assert ratio[-3:].max() >= 0.95 * 2 * U


def test_raised_window_distance_bounds_the_exact_one():
    """D' = (m (W_t + W_j) + max(W_t + W_j - 2 sum_m G'(t+m, j+m), 0)) (1 + 2^-20), with
    every epilogue operation in FP32, is at least the exact FP64 trajectory distance
    for every sampled window pair, adversarial days included."""
    D, L = 3726, 5
    groups = -(-D // 63)
    X, _ = make_slp_like(300, 46, 81, seed=9)
    X = (X - X.mean(0)).astype(np.float32)
    up, down = adversarial_rows(D, 3)
    X[100:100 + L] = up  # two windows of adversarial days
    X[200:200 + L] = down
    n = (X.astype(np.float64) ** 2).sum(1)
    W = np.convolve(n, np.ones(L), "valid").astype(np.float32)  # FP64 sums, stored FP32
    rng = np.random.default_rng(4)
    pairs = [(100, 200), (200, 100), (100, 100)] + [
        (int(t), int(j)) for t, j in rng.integers(0, len(X) - L + 1, (80, 2))]
    for t, j in pairs:
        g, _, _, Dp = gram_one_product(X[t:t + L], X[j:j + L], groups, "blocks16")
        gw = np.float32(0)
        for m in range(L):
            gw = np.float32(gw + g[m])
        s = np.float32(W[t] + W[j])
        d = np.float32(max(np.float32(s - np.float32(2) * gw), np.float32(0)))
        raised = np.float32(np.float32(np.float32(margin(Dp)) * s + d) *
                            np.float32(1 + 2.0 ** -20))
        exact = ((X[t:t + L].astype(np.float64) - X[j:j + L].astype(np.float64)) ** 2).sum()
        assert raised >= exact, (t, j, float(raised), exact)
