"""Seeded synthetic inputs shaped like daily gridded sea-level-pressure anomalies.

This module only makes inputs. It holds none of the trajectory-kNN arithmetic
and is shared by the CUDA path's tests and benchmarks and by the CPU oracle's
tests, so that both sides see exactly the same arrays.

Recipe (the paper's case study runs on 75 years of daily European SLP,
Sec. 5; reanalysis data are not available here, so this generator stands in
for them with the same shapes and a comparable structure):

* ``n_modes`` random integer wavevectors (kx, ky), |kx|, |ky| <= ``kmax``, not
  both zero, drawn once per dataset, each with amplitude 1/(1+|k|^2) and a
  random phase.
* every mode carries a complex AR(1) coefficient
  c_t = phi c_{t-1} + sqrt(1-phi^2) eps_t (stationary, unit variance), so the
  day-to-day persistence is ``phi``;
* field_t(x, y) = Re sum_k A_k c_{k,t} exp(2 pi i (kx x / w + ky y / h)),
  flattened row-major to D = h*w values and rescaled to global mean 0 and
  standard deviation ``std_hpa``;
* optionally an annual cycle of amplitude ``annual_amp`` hPa with a spatially
  varying phase is added and then removed again as a daily climatology (the
  mean over all years of each day of a 365-day calendar, day = t mod 365);
* optionally ``n_planted`` anomalous sequences of ``planted_len`` days are
  added at seeded, well separated start days: each has its own random
  low-wavenumber spatial pattern scaled to an RMS of ``planted_sigma`` times
  the field's standard deviation.

Everything is drawn from ``numpy.random.default_rng(seed)`` (PCG64), so a seed
gives the same draws on every machine; the final float32 values can differ in
the last bit between BLAS builds, which is why tests always feed one array to
both the oracle and the CUDA path within a single process.
"""
from __future__ import annotations

import dataclasses

import numpy as np

__all__ = ["SynthMeta", "make_slp_like", "config_inputs", "CONFIGS"]


@dataclasses.dataclass
class SynthMeta:
    n_days: int
    h: int
    w: int
    seed: int
    planted_starts: list
    planted_len: int
    std: float


def _mode_basis(rng, h, w, n_modes, kmax):
    ks = []
    while len(ks) < n_modes:
        kx, ky = rng.integers(-kmax, kmax + 1, size=2)
        if kx == 0 and ky == 0:
            continue
        ks.append((int(kx), int(ky)))
    ks = np.array(ks, dtype=np.float64)
    amp = 1.0 / (1.0 + (ks ** 2).sum(axis=1))
    phase = rng.uniform(0.0, 2.0 * np.pi, size=n_modes)
    yy, xx = np.meshgrid(np.arange(h), np.arange(w), indexing="ij")
    arg = 2.0 * np.pi * (ks[:, 0, None] * xx.reshape(1, -1) / w
                         + ks[:, 1, None] * yy.reshape(1, -1) / h) + phase[:, None]
    # Re(A c e^{i arg}) = A (Re c cos arg - Im c sin arg)
    return amp[:, None] * np.cos(arg), -amp[:, None] * np.sin(arg)


def _ar1_coeffs(rng, n_days, n_modes, phi):
    scale = np.sqrt(0.5)
    eps = (rng.standard_normal((n_days, n_modes))
           + 1j * rng.standard_normal((n_days, n_modes))) * scale
    c = np.empty((n_days, n_modes), dtype=np.complex128)
    c[0] = eps[0]
    innov = np.sqrt(1.0 - phi * phi)
    for t in range(1, n_days):
        c[t] = phi * c[t - 1] + innov * eps[t]
    return c


def make_slp_like(n_days: int, h: int, w: int, seed: int, *, n_modes: int = 40,
                  kmax: int = 4, phi: float = 0.8, std_hpa: float = 10.0,
                  annual_amp: float = 0.0, n_planted: int = 0,
                  planted_len: int = 5, planted_sigma: float = 4.0,
                  block_cols: int = 8192):
    """Return (X, meta): X is float32 of shape (n_days, h*w), row = day.

    The field is built in blocks of ``block_cols`` grid points (FP64 inside a
    block), so that large grids need little more host memory than the output."""
    rng = np.random.default_rng(seed)
    cos_b, sin_b = _mode_basis(rng, h, w, n_modes, kmax)
    c = _ar1_coeffs(rng, n_days, n_modes, phi)
    basis = np.concatenate([cos_b, sin_b], axis=0)          # (2 n_modes, D)
    coef = np.concatenate([c.real, c.imag], axis=1)         # (n_days, 2 n_modes)
    D = h * w
    blocks = [(b, min(D, b + block_cols)) for b in range(0, D, block_cols)]

    # global mean and standard deviation of the raw mode sum (two-pass per block)
    total, count = 0.0, 0
    for b0, b1 in blocks:
        total += float((coef @ basis[:, b0:b1]).sum())
        count += n_days * (b1 - b0)
    mean = total / count
    sq = 0.0
    for b0, b1 in blocks:
        sq += float(((coef @ basis[:, b0:b1] - mean) ** 2).sum())
    scale = std_hpa / np.sqrt(sq / count)

    doy = np.arange(n_days) % 365
    if annual_amp > 0.0:
        yy, xx = np.meshgrid(np.linspace(0, 1, h), np.linspace(0, 1, w), indexing="ij")
        phase_map = (2.0 * np.pi * (0.3 * xx + 0.2 * yy)).reshape(-1)
        ang = 2.0 * np.pi * doy / 365.0
    X = np.empty((n_days, D), dtype=np.float32)
    for b0, b1 in blocks:
        blk = (coef @ basis[:, b0:b1] - mean) * scale
        if annual_amp > 0.0:
            # cos(a - p) = cos a cos p + sin a sin p
            blk += annual_amp * (np.cos(ang)[:, None] * np.cos(phase_map[b0:b1])[None, :]
                                 + np.sin(ang)[:, None] * np.sin(phase_map[b0:b1])[None, :])
            # remove the daily climatology (mean of each calendar day over the years)
            for d in range(min(365, n_days)):
                blk[d::365] -= blk[d::365].mean(axis=0)
        X[:, b0:b1] = blk

    # standard deviation of the final field, accumulated in FP64 per block
    s1 = s2 = 0.0
    for b0, b1 in blocks:
        v = X[:, b0:b1].astype(np.float64)
        s1 += float(v.sum())
        s2 += float((v * v).sum())
    n = float(n_days) * D
    std = float(np.sqrt(max(s2 / n - (s1 / n) ** 2, 0.0)))
    starts = []
    if n_planted > 0:
        gap = 4 * planted_len
        lo, hi = gap, n_days - gap - planted_len
        if hi - lo < n_planted * gap:
            raise ValueError("series too short for the requested planted anomalies")
        while len(starts) < n_planted:
            s = int(rng.integers(lo, hi))
            if all(abs(s - o) >= gap for o in starts):
                starts.append(s)
        starts.sort()
        for s in starts:
            pc, ps = _mode_basis(rng, h, w, 6, kmax)
            pat = pc.sum(axis=0) + ps.sum(axis=0)
            pat *= planted_sigma * std / np.sqrt(np.mean(pat ** 2))
            X[s:s + planted_len] += pat[None, :].astype(np.float32)

    meta = SynthMeta(n_days=n_days, h=h, w=w, seed=seed, planted_starts=starts,
                     planted_len=planted_len, std=std)
    return X, meta


# The workloads: (days, grid h, grid w, L, k, exclusion, extra generator options).
CONFIGS = {
    # 5 years of daily fields on a 16x32 grid; small enough for the full oracle.
    "small_5y_16x32": dict(n_days=1826, h=16, w=32, L=3, k=10, exclusion=2, gen={}),
    # 75 years of daily fields on the 1-degree European grid (46x81 = 3,726 points).
    "euro_75y_46x81": dict(n_days=27394, h=46, w=81, L=5, k=20, exclusion=4,
                           gen=dict(annual_amp=5.0, n_planted=10, planted_len=5)),
    # 30 years on the same grid; the adjoint workload.
    "euro_30y_46x81": dict(n_days=10957, h=46, w=81, L=5, k=10, exclusion=4, gen={}),
    # 75 years on the 0.25-degree grid (181x321 = 58,101 points).
    "euro_75y_181x321": dict(n_days=27394, h=181, w=321, L=5, k=20, exclusion=4,
                             gen=dict(annual_amp=5.0)),
    # 75 years of 32-value fields (4x8 grid): a stand-in for fields reduced to a few
    # dozen principal components (the small-grid form).
    "small_d_75y_4x8": dict(n_days=27394, h=4, w=8, L=5, k=20, exclusion=4,
                            gen=dict(annual_amp=5.0)),
}

SEED_BASE = 20260302


def config_inputs(name: str, seed_offset: int = 0):
    """Generate the input array of a named workload with its fixed seed."""
    cfg = CONFIGS[name]
    seed = SEED_BASE + list(CONFIGS).index(name) + seed_offset
    X, meta = make_slp_like(cfg["n_days"], cfg["h"], cfg["w"], seed, **cfg["gen"])
    return X, meta, cfg
