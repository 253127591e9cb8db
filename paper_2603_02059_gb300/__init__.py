"""Python binding of libtraknn (GB300, sm_103a): exact trajectory kNN and the kNN
rarity score of TRAKNN (arXiv 2603.02059, Sec. 3.2 Eq. 2-3, Algorithm 1).

This module only marshals arguments: PyTorch provides device memory and the
current CUDA stream, and every step of the computation runs in the library's
CUDA kernels. There is no CPU fallback; calls fail loudly when the compiled
library is missing.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtraknn.so")
HEADER_PATH = os.path.join(os.path.dirname(_HERE), "include", "traknn.h")

STATUS = {0: "OK", 1: "ERR_INVALID_ARG", 2: "ERR_TOO_FEW_CANDIDATES", 3: "ERR_ALLOC",
          4: "ERR_CUDA", 5: "ERR_TIMEOUT", 6: "ERR_UNSUPPORTED_DEVICE", 7: "ERR_UNSUPPORTED",
          8: "ERR_SCRATCH_LIMIT", 9: "ERR_BOUNDS"}
PRECISION = {"fp32": 0, "split_bf16": 1, "bf16": 2}
EMBED = {"auto": 0, "always": 1, "never": 2}
OPTION = {"precision": 0, "center": 1, "col_chunks": 2, "wait_limit_ms": 3,
          "debug_withhold": 4, "profile": 5, "symmetric": 6, "unit_cols": 7, "stats": 8,
          "autotune": 9, "segment_k": 10,
          "group_strips": 11, "l2_keep_a": 12, "embed": 13, "epi_groups": 14}


class Series(ctypes.Structure):
    """traknn_series of include/traknn.h (one series of a batched call)."""
    _fields_ = [("X", ctypes.c_void_p), ("N", ctypes.c_int64), ("L", ctypes.c_int),
                ("k", ctypes.c_int), ("exclusion", ctypes.c_int), ("nbr_idx", ctypes.c_void_p),
                ("nbr_dist", ctypes.c_void_p), ("score", ctypes.c_void_p)]


class TrakNNError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {STATUS.get(status, status)}")


_lib = None
_lib_lock = threading.Lock()


def lib():
    """Load libtraknn.so (raises if it has not been built)."""
    global _lib
    with _lib_lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                                   "`python -c 'import __graft_entry__ as g; g.build()'`")
            _lib = bind(LIB_PATH)
    return _lib


def bind(path: str):
    """Load a build of the library at `path` with the C signatures of traknn.h (the
    debug variant libtraknn_bounds.so is loaded this way by its tests)."""
    L = ctypes.CDLL(path)
    P, I, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
    sig = {
        "traknn_create": [ctypes.POINTER(P), I],
        "traknn_destroy": [P],
        "traknn_set_option": [P, I, I64],
        "traknn_check_problem": [I64, I64, I, I, I],
        "traknn_knn_scores": [P, P, I64, I64, I, I, I, P, P, P, P],
        "traknn_knn_scores_host": [P, P, I64, I64, I, I, I, P, P, P, P],
        "traknn_score_backward": [P, P, I64, I64, I, I, P, P, P, P],
        "traknn_sync_status": [P, P],
        "traknn_profile_read": [P, P, I, ctypes.POINTER(I)],
        "traknn_launch_count": [P, ctypes.POINTER(I64)],
        "traknn_knn_scores_static": [P, I64, I64, I, I, I, P, P, P, P],
        "traknn_stats_read": [P, P, I],
        "traknn_knn_scores_batched": [P, P, I, I64, P],
        "traknn_set_grid_weights": [P, P, I64],
        "traknn_knn_scores_multi": [P, P, I, I64, P],
        "traknn_knn_stats": [P, P, I64, I, P, I, P, P],
        "traknn_partition": [I64, I, I, I, ctypes.POINTER(I64), ctypes.POINTER(I64)],
        "traknn_knn_partial": [P, P, I64, I64, I, I, I, I, I, P, P, P],
        "traknn_merge_partials": [P, P, P, I, I64, I, P, P, P, P],
        "traknn_work_shape": [P, ctypes.POINTER(I), ctypes.POINTER(I)],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    L.traknn_status_string.argtypes = [I]
    L.traknn_status_string.restype = ctypes.c_char_p
    return L


def header_functions(path: str = HEADER_PATH):
    """Names of the functions declared in include/traknn.h."""
    with open(path) as f:
        txt = f.read()
    return sorted(set(re.findall(r"^\s*(?:traknn_status|const char\*)\s+(traknn_\w+)\s*\(",
                                 txt, re.M)))


def _check(rc: int, what: str):
    if rc != 0:
        raise TrakNNError(rc, what)


def check_problem(N: int, D: int, L: int, k: int, exclusion: int) -> int:
    """Host-only shape check; returns the status code a compute call would give."""
    return int(lib().traknn_check_problem(N, D, L, k, exclusion))


class Handle:
    """Owns one library context (workspace cache) on one CUDA device."""

    def __init__(self, device: int | None = None):
        if device is None:
            device = torch.cuda.current_device()
        self.device = int(device)
        h = ctypes.c_void_p()
        _check(lib().traknn_create(ctypes.byref(h), self.device), "traknn_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().traknn_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_option(self, name: str, value: int):
        _check(lib().traknn_set_option(self._h, OPTION[name], int(value)), f"set_option({name})")

    def configure(self, precision=None, center=None, col_chunks=None, symmetric=None,
                  unit_cols=None, autotune=None, embed=None):
        if precision is not None:
            self.set_option("precision", PRECISION[precision])
        if center is not None:
            self.set_option("center", int(center))
        if col_chunks is not None:
            self.set_option("col_chunks", int(col_chunks))
        if symmetric is not None:
            self.set_option("symmetric", int(symmetric))
        if unit_cols is not None:
            self.set_option("unit_cols", int(unit_cols))
        if autotune is not None:
            self.set_option("autotune", int(autotune))
        if embed is not None:
            self.set_option("embed", EMBED[embed])

    def set_grid_weights(self, w):
        """Grid-point weights for later calls (a [D] float32 CUDA tensor kept alive by
        the handle), or None to clear them."""
        if w is None:
            _check(lib().traknn_set_grid_weights(self._h, None, 0), "set_grid_weights")
            self._weights = None
            return
        w = w.to(torch.float32).contiguous()
        if not w.is_cuda or w.dim() != 1:
            raise ValueError("weights must be a 1-D CUDA tensor")
        _check(lib().traknn_set_grid_weights(self._h, w.data_ptr(), w.numel()),
               "set_grid_weights")
        self._weights = w

    def profile_read(self, max_n: int = 256):
        """Durations (ms) of the fused Gram/top-k kernel of recent profiled calls."""
        buf = (ctypes.c_float * max_n)()
        n = ctypes.c_int()
        _check(lib().traknn_profile_read(self._h, buf, max_n, ctypes.byref(n)), "profile_read")
        return [buf[i] for i in range(n.value)]

    def stats_read(self):
        """Kernel event counters since the last read (TRAKNN_OPT_STATS)."""
        names = ["row_inserts", "col_emits", "col_full", "col_lists", "chunks",
                 "mma_wait_tmem", "mma_wait_full", "mma_cycles", "epi_wait_acc",
                 "epi_tile_head", "epi_stage", "epi_bar1", "epi_scan", "epi_col", "epi_cycles"]
        buf = (ctypes.c_uint64 * len(names))()
        _check(lib().traknn_stats_read(self._h, buf, len(names)), "stats_read")
        return {n: int(buf[i]) for i, n in enumerate(names)}

    def work_shape(self):
        """(Gram tiles per work unit, row strips side by side) of the last tensor-core
        forward call (the autotuner's choice when autotuning is on)."""
        t, g = ctypes.c_int(), ctypes.c_int()
        _check(lib().traknn_work_shape(self._h, ctypes.byref(t), ctypes.byref(g)), "work_shape")
        return int(t.value), int(g.value)

    def launch_count(self) -> int:
        c = ctypes.c_int64()
        _check(lib().traknn_launch_count(self._h, ctypes.byref(c)), "launch_count")
        return int(c.value)

    def sync_status(self, stream=None) -> int:
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        return int(lib().traknn_sync_status(self._h, ctypes.c_void_p(s.cuda_stream)))


_handles: dict = {}


def get_handle(device: int | None = None) -> Handle:
    if device is None:
        device = torch.cuda.current_device()
    h = _handles.get(device)
    if h is None:
        h = Handle(device)
        _handles[device] = h
    return h


def _as_input(X: torch.Tensor) -> torch.Tensor:
    if not X.is_cuda or X.dtype != torch.float32 or X.dim() != 2:
        raise ValueError("X must be a 2-D float32 CUDA tensor (days x grid points)")
    return X.contiguous()


def knn_scores(X: torch.Tensor, L: int, k: int, exclusion: int | None = None, *,
               precision: str = "split_bf16", center: bool = True, col_chunks: int = 0,
               symmetric: bool = True, unit_cols: int = 0, embed: str = "auto",
               handle: Handle | None = None, out=None):
    """Neighbour indices [M, k] int32, distances [M, k] float32 and rarity scores [M]
    float32 for every L-day trajectory of X (M = N - L + 1). `exclusion` defaults to
    L - 1 (overlapping trajectories are not candidates). `embed` ("auto", "always",
    "never") selects trajectory-embedded operands on the tensor cores
    (TRAKNN_OPT_EMBED)."""
    X = _as_input(X)
    N, D = X.shape
    e = L - 1 if exclusion is None else int(exclusion)
    M = N - L + 1
    h = handle or get_handle(X.device.index)
    h.configure(precision=precision, center=center, col_chunks=col_chunks, symmetric=symmetric,
                unit_cols=unit_cols, embed=embed)
    if out is None:
        idx = torch.empty((max(M, 0), k), dtype=torch.int32, device=X.device)
        dist = torch.empty((max(M, 0), k), dtype=torch.float32, device=X.device)
        score = torch.empty((max(M, 0),), dtype=torch.float32, device=X.device)
    else:
        idx, dist, score = out
    s = torch.cuda.current_stream(X.device)
    rc = lib().traknn_knn_scores(h._h, X.data_ptr(), N, D, L, k, e, idx.data_ptr(),
                                 dist.data_ptr(), score.data_ptr(),
                                 ctypes.c_void_p(s.cuda_stream))
    _check(rc, "traknn_knn_scores")
    return idx, dist, score


def knn_scores_batched(series, *, precision: str = "split_bf16", center: bool = True,
                       symmetric: bool = True, unit_cols: int = 0, autotune: bool = False,
                       handle: Handle | None = None, outs=None):
    """Forward pass of several series with the same grid size D in one call.
    `series` is a list of (X, L, k, exclusion) with X a [N_b, D] float32 CUDA tensor
    (exclusion None = L - 1). Returns a list of (idx, dist, score), one per series,
    each equal to knn_scores on that series alone."""
    if not series:
        return []
    Xs = [_as_input(X) for X, _, _, _ in series]
    D = Xs[0].shape[1]
    dev = Xs[0].device
    for X in Xs:
        if X.shape[1] != D or X.device != dev:
            raise ValueError("all series must share D and the device")
    h = handle or get_handle(dev.index)
    h.configure(precision=precision, center=center, symmetric=symmetric, unit_cols=unit_cols,
                autotune=autotune)
    arr = (Series * len(series))()
    results = []
    for b, ((_, L, k, exclusion), X) in enumerate(zip(series, Xs)):
        N = X.shape[0]
        e = L - 1 if exclusion is None else int(exclusion)
        M = max(N - L + 1, 0)
        if outs is None:
            idx = torch.empty((M, k), dtype=torch.int32, device=dev)
            dist = torch.empty((M, k), dtype=torch.float32, device=dev)
            score = torch.empty((M,), dtype=torch.float32, device=dev)
        else:
            idx, dist, score = outs[b]
        arr[b] = Series(X.data_ptr(), N, L, k, e, idx.data_ptr(), dist.data_ptr(),
                        score.data_ptr())
        results.append((idx, dist, score))
    s = torch.cuda.current_stream(dev)
    rc = lib().traknn_knn_scores_batched(h._h, ctypes.cast(arr, ctypes.c_void_p), len(series),
                                         D, ctypes.c_void_p(s.cuda_stream))
    _check(rc, "traknn_knn_scores_batched")
    return results


def knn_scores_multi(X: torch.Tensor, settings, *, precision: str = "split_bf16",
                     center: bool = True, symmetric: bool = True,
                     handle: Handle | None = None):
    """Several (L, k, exclusion) settings of one record X ([N, D] float32 CUDA) in one
    Gram sweep. `settings` is a list of (L, k, exclusion) (exclusion None = L - 1).
    Returns a list of (idx, dist, score), one per setting, in the given order."""
    X = _as_input(X)
    N, D = X.shape
    h = handle or get_handle(X.device.index)
    h.configure(precision=precision, center=center, symmetric=symmetric, unit_cols=0)
    arr = (Series * len(settings))()
    results = []
    for b, (L, k, exclusion) in enumerate(settings):
        e = L - 1 if exclusion is None else int(exclusion)
        M = max(N - L + 1, 0)
        idx = torch.empty((M, k), dtype=torch.int32, device=X.device)
        dist = torch.empty((M, k), dtype=torch.float32, device=X.device)
        score = torch.empty((M,), dtype=torch.float32, device=X.device)
        arr[b] = Series(X.data_ptr(), N, L, k, e, idx.data_ptr(), dist.data_ptr(),
                        score.data_ptr())
        results.append((idx, dist, score))
    s = torch.cuda.current_stream(X.device)
    rc = lib().traknn_knn_scores_multi(h._h, ctypes.cast(arr, ctypes.c_void_p), len(settings),
                                       D, ctypes.c_void_p(s.cuda_stream))
    _check(rc, "traknn_knn_scores_multi")
    return results


def knn_stats(dist: torch.Tensor, k_id: int | None = None, *, prefix: bool = True,
              handle: Handle | None = None):
    """From sorted neighbour distances [M, k] (as knn_scores returns them): the scores
    for every k' <= k ([M, k], column k'-1) and, if k_id is given, the local intrinsic
    dimension of every row with k_id neighbours ([M]). Returns (prefix or None,
    local_id or None)."""
    if not dist.is_cuda or dist.dtype != torch.float32 or dist.dim() != 2:
        raise ValueError("dist must be a 2-D float32 CUDA tensor")
    dist = dist.contiguous()
    M, k = dist.shape
    h = handle or get_handle(dist.device.index)
    pre = torch.empty((M, k), dtype=torch.float32, device=dist.device) if prefix else None
    lid = torch.empty((M,), dtype=torch.float32, device=dist.device) if k_id else None
    s = torch.cuda.current_stream(dist.device)
    rc = lib().traknn_knn_stats(h._h, dist.data_ptr(), M, k,
                                pre.data_ptr() if pre is not None else None, int(k_id or 0),
                                lid.data_ptr() if lid is not None else None,
                                ctypes.c_void_p(s.cuda_stream))
    _check(rc, "traknn_knn_stats")
    return pre, lid


def knn_scores_host(X_host: torch.Tensor, L: int, k: int, exclusion: int | None = None, *,
                    precision: str = "split_bf16", center: bool = True, col_chunks: int = 0,
                    symmetric: bool = True, unit_cols: int = 0, embed: str = "auto",
                    handle=None, out=None, device: int | None = None):
    """Host-buffer variant: X_host is a CPU float32 tensor (pinned for fast copies);
    returns CPU tensors. The call copies in, computes, copies out and synchronises."""
    if X_host.is_cuda or X_host.dtype != torch.float32 or X_host.dim() != 2:
        raise ValueError("X_host must be a 2-D float32 CPU tensor")
    X_host = X_host.contiguous()
    N, D = X_host.shape
    e = L - 1 if exclusion is None else int(exclusion)
    M = N - L + 1
    h = handle or get_handle(device)
    h.configure(precision=precision, center=center, col_chunks=col_chunks, symmetric=symmetric,
                unit_cols=unit_cols, embed=embed)
    if out is None:
        pin = X_host.is_pinned()
        idx = torch.empty((M, k), dtype=torch.int32, pin_memory=pin)
        dist = torch.empty((M, k), dtype=torch.float32, pin_memory=pin)
        score = torch.empty((M,), dtype=torch.float32, pin_memory=pin)
    else:
        idx, dist, score = out
    s = torch.cuda.current_stream(h.device)
    rc = lib().traknn_knn_scores_host(h._h, X_host.data_ptr(), N, D, L, k, e, idx.data_ptr(),
                                      dist.data_ptr(), score.data_ptr(),
                                      ctypes.c_void_p(s.cuda_stream))
    _check(rc, "traknn_knn_scores_host")
    return idx, dist, score


def knn_scores_static(X: torch.Tensor, L: int, k: int, exclusion: int | None = None):
    """FP32 forward pass that allocates no device memory inside the library: its
    scratch is a fixed 32 MiB device array (see traknn_knn_scores_static in
    include/traknn.h). The outputs are allocated here by torch."""
    X = _as_input(X)
    N, D = X.shape
    e = L - 1 if exclusion is None else int(exclusion)
    M = N - L + 1
    idx = torch.empty((M, k), dtype=torch.int32, device=X.device)
    dist = torch.empty((M, k), dtype=torch.float32, device=X.device)
    score = torch.empty((M,), dtype=torch.float32, device=X.device)
    s = torch.cuda.current_stream(X.device)
    with torch.cuda.device(X.device):
        rc = lib().traknn_knn_scores_static(X.data_ptr(), N, D, L, k, e, idx.data_ptr(),
                                            dist.data_ptr(), score.data_ptr(),
                                            ctypes.c_void_p(s.cuda_stream))
    _check(rc, "traknn_knn_scores_static")
    return idx, dist, score


def partition(M: int, L: int, nparts: int, part: int):
    """Trajectory rows [lo, hi) whose pairs part `part` of `nparts` evaluates when one
    series is split across processes (host only; see traknn_partition)."""
    lo, hi = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().traknn_partition(M, L, nparts, part, ctypes.byref(lo), ctypes.byref(hi)),
           "traknn_partition")
    return int(lo.value), int(hi.value)


def knn_partial(X: torch.Tensor, L: int, k: int, exclusion: int | None, part: int, nparts: int,
                *, precision: str = "split_bf16", center: bool = True,
                handle: Handle | None = None):
    """Candidate lists ([M, k] int32 indices, -1 = none; [M, k] float32 distances) of
    part `part` of `nparts` of one series split across processes."""
    X = _as_input(X)
    N, D = X.shape
    e = L - 1 if exclusion is None else int(exclusion)
    M = N - L + 1
    h = handle or get_handle(X.device.index)
    h.configure(precision=precision, center=center, symmetric=True, unit_cols=0)
    idx = torch.empty((M, k), dtype=torch.int32, device=X.device)
    dist = torch.empty((M, k), dtype=torch.float32, device=X.device)
    s = torch.cuda.current_stream(X.device)
    rc = lib().traknn_knn_partial(h._h, X.data_ptr(), N, D, L, k, e, part, nparts,
                                  idx.data_ptr(), dist.data_ptr(), ctypes.c_void_p(s.cuda_stream))
    _check(rc, "traknn_knn_partial")
    return idx, dist


def merge_partials(idx_parts: torch.Tensor, dist_parts: torch.Tensor, *,
                   handle: Handle | None = None):
    """Neighbour indices, distances and scores from the parts' candidate lists
    ([P, M, k] int32 and float32 CUDA tensors, part-major)."""
    if idx_parts.dim() != 3 or dist_parts.shape != idx_parts.shape or not idx_parts.is_cuda:
        raise ValueError("idx_parts and dist_parts must be [P, M, k] CUDA tensors")
    idx_parts = idx_parts.to(torch.int32).contiguous()
    dist_parts = dist_parts.to(torch.float32).contiguous()
    P, M, k = idx_parts.shape
    h = handle or get_handle(idx_parts.device.index)
    idx = torch.empty((M, k), dtype=torch.int32, device=idx_parts.device)
    dist = torch.empty((M, k), dtype=torch.float32, device=idx_parts.device)
    score = torch.empty((M,), dtype=torch.float32, device=idx_parts.device)
    s = torch.cuda.current_stream(idx_parts.device)
    rc = lib().traknn_merge_partials(h._h, idx_parts.data_ptr(), dist_parts.data_ptr(), P, M, k,
                                     idx.data_ptr(), dist.data_ptr(), score.data_ptr(),
                                     ctypes.c_void_p(s.cuda_stream))
    _check(rc, "traknn_merge_partials")
    return idx, dist, score


def gather_partials(idx: torch.Tensor, dist: torch.Tensor, group=None):
    """The exchange step of a split series: every process's [M, k] candidate lists,
    gathered from all processes of `group` (torch.distributed) into [P, M, k] tensors
    in rank order (the part index is the rank)."""
    import torch.distributed as dist_
    P = dist_.get_world_size(group)
    ilist = [torch.empty_like(idx) for _ in range(P)]
    dlist = [torch.empty_like(dist) for _ in range(P)]
    dist_.all_gather(ilist, idx.contiguous(), group=group)
    dist_.all_gather(dlist, dist.contiguous(), group=group)
    return torch.stack(ilist), torch.stack(dlist)


def knn_scores_split(X: torch.Tensor, L: int, k: int, exclusion: int | None = None, *,
                     group=None, precision: str = "split_bf16", handle: Handle | None = None):
    """traknn_knn_scores on one series shared by the processes of `group`: this
    process evaluates the pairs of its part (part = rank), the candidate lists are
    all-gathered once, and every process merges them into the full result."""
    import torch.distributed as dist_
    rank, P = dist_.get_rank(group), dist_.get_world_size(group)
    pidx, pdist = knn_partial(X, L, k, exclusion, rank, P, precision=precision, handle=handle)
    iparts, dparts = gather_partials(pidx, pdist, group)
    return merge_partials(iparts, dparts, handle=handle)


def score_backward(X: torch.Tensor, L: int, k: int, idx: torch.Tensor,
                   grad_score: torch.Tensor, *, handle: Handle | None = None) -> torch.Tensor:
    """dX = d(sum_t grad_score[t] s_t)/dX with the neighbour sets `idx` held fixed."""
    X = _as_input(X)
    N, D = X.shape
    idx = idx.to(torch.int32).contiguous()
    g = grad_score.to(torch.float32).contiguous()
    h = handle or get_handle(X.device.index)
    dX = torch.empty_like(X)
    s = torch.cuda.current_stream(X.device)
    rc = lib().traknn_score_backward(h._h, X.data_ptr(), N, D, L, k, idx.data_ptr(),
                                     g.data_ptr(), dX.data_ptr(), ctypes.c_void_p(s.cuda_stream))
    _check(rc, "traknn_score_backward")
    return dX


class TrakNNScore(torch.autograd.Function):
    """score = TrakNNScore.apply(X, L, k, exclusion, precision): the rarity scores
    (Eq. 3); backward gives d(sum g s)/dX with the forward's neighbour sets fixed."""

    @staticmethod
    def forward(ctx, X, L, k, exclusion=None, precision="split_bf16"):
        idx, dist, score = knn_scores(X, L, k, exclusion, precision=precision)
        ctx.save_for_backward(X, idx)
        ctx.L, ctx.k = L, k
        ctx.mark_non_differentiable(idx)
        return score

    @staticmethod
    def backward(ctx, grad_score):
        X, idx = ctx.saved_tensors
        dX = score_backward(X, ctx.L, ctx.k, idx, grad_score)
        return dX, None, None, None, None
