"""CPU-side checks of the C ABI: the library loads, exports every function that
include/traknn.h declares, and its host-only checks behave (no GPU needed)."""
import ctypes

import pytest

import paper_2603_02059_gb300 as tk


def test_library_exports_every_declared_function():
    lib = tk.lib()
    names = tk.header_functions()
    assert "traknn_knn_scores" in names and "traknn_score_backward" in names
    for n in names:
        assert hasattr(lib, n), f"{n} declared in traknn.h but not exported"


def test_status_strings():
    lib = tk.lib()
    for code in range(10):
        s = lib.traknn_status_string(code)
        assert isinstance(s, bytes) and len(s) > 0
    assert lib.traknn_status_string(0) == b"ok"


@pytest.mark.parametrize("args,status", [
    ((100, 10, 3, 5, 2), 0),
    ((0, 10, 3, 5, 2), 1),          # no days
    ((100, 0, 3, 5, 2), 1),         # no grid points
    ((100, 10, 0, 5, 2), 1),        # L < 1
    ((10, 10, 11, 1, 0), 1),        # L > N
    ((100, 10, 3, 0, 2), 1),        # k < 1
    ((100, 10, 3, 5, -1), 1),       # negative exclusion
    ((100, 10, 18, 5, 2), 7),       # L above the compiled limit
    ((1000, 10, 3, 65, 2), 7),      # k above the compiled limit
    ((20, 4, 3, 14, 2), 2),         # M=18, middle rows have 18-5=13 < 14 candidates
    ((20, 4, 3, 13, 2), 0),
    ((1, 1, 1, 1, 0), 2),           # a single trajectory has no candidates
])
def test_check_problem(args, status):
    assert tk.check_problem(*args) == status


def test_null_handle_is_rejected():
    lib = tk.lib()
    assert lib.traknn_knn_scores(None, None, 10, 2, 1, 1, 0, None, None, None, None) == 1
    assert lib.traknn_set_option(None, 0, 0) == 1
    assert lib.traknn_destroy(None) == 1
    assert lib.traknn_create(None, 0) == 1
