import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libtraknn.so")


def load_golden(name):
    """Parse a tests/golden/*.txt fixture: returns (X rows, {case: (params, rows)})."""
    path = os.path.join(ROOT, "tests", "golden", name)
    X, cases, cur = [], {}, None
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            tok = line.split()
            if tok[0] == "X":
                X.append([float(v) for v in tok[1:]])
            elif tok[0] == "CASE":
                params = dict(kv.split("=") for kv in tok[2:])
                cur = tok[1]
                cases[cur] = ({k: int(v) for k, v in params.items()}, {})
            elif tok[0] == "ROW":
                kv = dict(t.split("=") for t in tok[2:])
                cases[cur][1][int(tok[1])] = (
                    [int(v) for v in kv["idx"].split(",")],
                    [float(v) for v in kv["dist"].split(",")],
                    float(kv["score"]))
    return X, cases
