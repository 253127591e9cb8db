"""The debug build (libtraknn_bounds.so, compiled with -DTRAKNN_BOUNDS_CHECK): every
guarded device-side index (candidate-list records and slots, row bounds, the
merge's list reads, the adjoint's entry lists) is checked against its buffer, and a
bad one is reported as TRAKNN_ERR_BOUNDS instead of being used. Edge-case shapes
(one partial strip, the largest L and k, ragged units, folded K segments, batched,
several settings, split parts, the adjoint) run through its C ABI: every call must
report no failed check and give the regular build's results bit for bit."""
import ctypes

import numpy as np
import pytest

from synth import make_slp_like

pytestmark = pytest.mark.gpu

OPT = {"precision": 0, "symmetric": 6, "unit_cols": 7, "segment_k": 10, "embed": 13}
PREC = {"fp32": 0, "split_bf16": 1, "bf16": 2}


@pytest.fixture(scope="module")
def tk():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2603_02059_gb300 as m
    return m


@pytest.fixture(scope="module")
def blib(tk):
    from paper_2603_02059_gb300 import build
    return tk.bind(build.build(bounds_check=True))


@pytest.fixture(scope="module")
def bh(blib):
    h = ctypes.c_void_p()
    import torch
    assert blib.traknn_create(ctypes.byref(h), torch.cuda.current_device()) == 0
    yield h
    blib.traknn_destroy(h)


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _outs(M, k):
    import torch
    return (torch.empty((M, k), dtype=torch.int32, device="cuda"),
            torch.empty((M, k), dtype=torch.float32, device="cuda"),
            torch.empty((M,), dtype=torch.float32, device="cuda"))


def _set(blib, bh, **opts):
    for name, v in opts.items():
        v = PREC[v] if name == "precision" else v
        assert blib.traknn_set_option(bh, OPT[name], int(v)) == 0


def _ok(blib, bh):
    assert blib.traknn_sync_status(bh, _stream()) == 0


def _same(a, b):
    for x, y in zip(a, b):
        assert np.array_equal(x.cpu().numpy(), y.cpu().numpy())


CASES = [  # N, h, w, L, k, e, options
    (20, 1, 3, 2, 2, 1, dict(precision="split_bf16", embed=2)),
    (20, 1, 3, 2, 2, 1, dict(precision="split_bf16", embed=1)),
    (20, 1, 3, 2, 2, 1, dict(precision="fp32")),
    (300, 4, 5, 1, 1, 0, dict(precision="split_bf16")),
    (420, 6, 6, 17, 64, 16, dict(precision="split_bf16", embed=2)),
    (420, 6, 6, 17, 64, 16, dict(precision="split_bf16", embed=1)),
    (420, 6, 6, 17, 64, 16, dict(precision="fp32")),
    (1500, 8, 12, 5, 10, 4, dict(precision="split_bf16", unit_cols=300, embed=2)),
    (1500, 8, 12, 5, 10, 4, dict(precision="split_bf16", symmetric=0, embed=2)),
    (900, 40, 60, 5, 10, 4, dict(precision="split_bf16", segment_k=256)),
    (777, 9, 15, 10, 20, 9, dict(precision="bf16", embed=2)),
    (1500, 4, 8, 5, 20, 4, dict(precision="split_bf16", embed=1)),  # two epilogue groups
    (600, 3, 4, 1, 8, 0, dict(precision="split_bf16")),  # two epilogue groups, L = 1
]


@pytest.mark.parametrize("N,h,w,L,k,e,opts", CASES)
def test_forward_passes_index_checks(tk, blib, bh, N, h, w, L, k, e, opts):
    import torch
    X = torch.from_numpy(make_slp_like(N, h, w, seed=N + L)[0]).cuda()
    D = X.shape[1]
    M = N - L + 1
    _set(blib, bh, symmetric=1, unit_cols=0, segment_k=0, embed=0)
    _set(blib, bh, **opts)
    out = _outs(M, k)
    assert blib.traknn_knn_scores(bh, X.data_ptr(), N, D, L, k, e, *(t.data_ptr() for t in out),
                                  _stream()) == 0
    _ok(blib, bh)
    rh = tk.Handle()
    for name, v in opts.items():
        rh.set_option(name, PREC[v] if name == "precision" else v)
    ref = _outs(M, k)
    assert tk.lib().traknn_knn_scores(rh._h, X.data_ptr(), N, D, L, k, e,
                                      *(t.data_ptr() for t in ref), _stream()) == 0
    assert rh.sync_status() == 0
    _same(out, ref)
    rh.close()


def test_batched_and_several_settings_pass_index_checks(tk, blib, bh):
    import torch
    _set(blib, bh, precision="split_bf16", symmetric=1, unit_cols=0, segment_k=0, embed=0)
    shapes = [(400, 5, 8, 4), (129, 1, 3, 0), (777, 10, 20, 9)]
    Xs = [torch.from_numpy(make_slp_like(N, 9, 14, seed=5 + N)[0]).cuda() for N, *_ in shapes]
    D = Xs[0].shape[1]
    outs = [_outs(N - L + 1, k) for N, L, k, _ in shapes]
    arr = (tk.Series * 3)()
    for b, ((N, L, k, e), X, o) in enumerate(zip(shapes, Xs, outs)):
        arr[b] = tk.Series(X.data_ptr(), N, L, k, e, *(t.data_ptr() for t in o))
    assert blib.traknn_knn_scores_batched(bh, ctypes.cast(arr, ctypes.c_void_p), 3, D,
                                          _stream()) == 0
    _ok(blib, bh)
    ref = tk.knn_scores_batched([(X, L, k, e) for X, (N, L, k, e) in zip(Xs, shapes)])
    for o, r in zip(outs, ref):
        _same(o, r)
    settings = [(3, 10, 2), (5, 20, 4), (10, 5, 9)]
    X = Xs[2]
    N = X.shape[0]
    mouts = [_outs(N - L + 1, k) for L, k, _ in settings]
    marr = (tk.Series * 3)()
    for b, ((L, k, e), o) in enumerate(zip(settings, mouts)):
        marr[b] = tk.Series(X.data_ptr(), N, L, k, e, *(t.data_ptr() for t in o))
    assert blib.traknn_knn_scores_multi(bh, ctypes.cast(marr, ctypes.c_void_p), 3, D,
                                        _stream()) == 0
    _ok(blib, bh)
    mref = tk.knn_scores_multi(X, settings)
    for o, r in zip(mouts, mref):
        _same(o, r)


def test_split_parts_pass_index_checks(tk, blib, bh):
    import torch
    _set(blib, bh, precision="split_bf16", symmetric=1, unit_cols=0, segment_k=0, embed=0)
    N, L, k, e, P = 1500, 5, 10, 4, 3
    X = torch.from_numpy(make_slp_like(N, 8, 12, seed=77)[0]).cuda()
    D = X.shape[1]
    M = N - L + 1
    ip = torch.empty((P, M, k), dtype=torch.int32, device="cuda")
    dp = torch.empty((P, M, k), dtype=torch.float32, device="cuda")
    for p in range(P):
        assert blib.traknn_knn_partial(bh, X.data_ptr(), N, D, L, k, e, p, P, ip[p].data_ptr(),
                                       dp[p].data_ptr(), _stream()) == 0
        _ok(blib, bh)
    out = _outs(M, k)
    assert blib.traknn_merge_partials(bh, ip.data_ptr(), dp.data_ptr(), P, M, k,
                                      *(t.data_ptr() for t in out), _stream()) == 0
    _ok(blib, bh)
    ref = tk.knn_scores(X, L, k, e, embed="never")
    _same(out, ref)


def test_adjoint_passes_index_checks(tk, blib, bh):
    import torch
    N, L, k, e = 400, 5, 10, 4
    X = torch.from_numpy(make_slp_like(N, 6, 9, seed=13)[0]).cuda()
    D = X.shape[1]
    M = N - L + 1
    idx, _, _ = tk.knn_scores(X, L, k, e)
    g = torch.linspace(0.5, 1.5, M, device="cuda")
    dX = torch.empty_like(X)
    assert blib.traknn_score_backward(bh, X.data_ptr(), N, D, L, k, idx.data_ptr(), g.data_ptr(),
                                      dX.data_ptr(), _stream()) == 0
    _ok(blib, bh)
    ref = tk.score_backward(X, L, k, idx, g)
    torch.cuda.synchronize()
    assert torch.equal(dX, ref)
