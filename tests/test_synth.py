"""Checks of the seeded input generator (shapes, statistics, determinism, planting)."""
import numpy as np

from synth import config_inputs, make_slp_like


def test_shape_stats_and_determinism():
    X, meta = make_slp_like(500, 8, 12, seed=1)
    assert X.shape == (500, 96) and X.dtype == np.float32
    assert abs(float(X.mean())) < 1e-3 and abs(float(X.std()) - 10.0) < 1e-3
    X2, _ = make_slp_like(500, 8, 12, seed=1)
    assert np.array_equal(X, X2)
    X3, _ = make_slp_like(500, 8, 12, seed=2)
    assert not np.array_equal(X, X3)


def test_persistence_is_ar1():
    X, _ = make_slp_like(4000, 6, 6, seed=3, phi=0.8)
    r = np.corrcoef(X[:-1].ravel(), X[1:].ravel())[0, 1]
    assert 0.75 < r < 0.85


def test_planted_sequences_and_climatology():
    X, meta = make_slp_like(3000, 6, 10, seed=4, annual_amp=5.0, n_planted=3, planted_len=5)
    assert len(meta.planted_starts) == 3
    s = sorted(meta.planted_starts)
    assert all(b - a >= 20 for a, b in zip(s, s[1:]))
    rms = np.sqrt((X ** 2).mean(axis=1))
    for st in s:
        assert rms[st:st + 5].min() > 2.5 * np.median(rms)


def test_named_small_config():
    X, meta, cfg = config_inputs("small_5y_16x32")
    assert X.shape == (1826, 512) and cfg["L"] == 3 and cfg["k"] == 10 and cfg["exclusion"] == 2
