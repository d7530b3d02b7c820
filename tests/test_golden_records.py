"""The stored oracle solves (tests/golden/solve_*.json) against the seeded generators the GPU tests
rebuild their matrices with, on the CPU: each record is a consistent, converged run of the oracle's
restarted CB-GMRES (Fig. 1, tolerance on the explicit residual of Eq. 4), and the fingerprint of the
matrix it was computed on is that of the matrix the generator draws on this host. A GPU solve is
only comparable with a record of the same matrix."""
import glob
import json
import os
import re
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(ROOT, "tests", "golden")
sys.path.insert(0, ROOT)
sys.path.insert(0, GOLDEN)

RECORDS = sorted(glob.glob(os.path.join(GOLDEN, "solve_*.json")))


def load(path):
    with open(path) as f:
        return json.load(f)


@pytest.mark.parametrize("path", RECORDS, ids=[os.path.basename(p) for p in RECORDS])
def test_record_is_a_consistent_converged_solve(path):
    rec = load(path)
    name = os.path.basename(path)[len("solve_"):-len(".json")]
    config, fmt = name.split("_", 1)
    assert rec["config"] == config and rec["format"] == fmt
    assert rec["converged"] and rec["breakdowns"] == 0
    assert rec["iters"] >= 1 and 0 <= rec["reorths"] <= rec["iters"]
    # one restart per started cycle of `restart` steps
    assert rec["restarts"] == -(-rec["iters"] // rec["restart"])
    # converged on the explicit residual, which the writer also recomputed with the oracle's SpMV
    assert rec["true_rrn"] <= rec["tol"]
    assert rec["rrn_recomputed"] == pytest.approx(rec["true_rrn"], rel=1e-6)
    # the implicit residual of the Givens recurrence tracks the explicit one at convergence
    assert rec["implicit_rrn"] == pytest.approx(rec["true_rrn"], rel=1e-2)
    m = re.search(r"n=(\d+)", rec["matrix"])
    idx = np.asarray(rec["sample_index"])
    x = np.array([float.fromhex(v) for v in rec["sample_x"]])
    assert idx.size == x.size >= 2  # the first and last index, then up to 1024 seeded ones
    assert np.all(np.diff(idx) > 0) and idx[0] == 0
    if m:
        assert idx[-1] == int(m.group(1)) - 1
    assert np.all(np.isfinite(x)) and rec["x_norm2"] > 0


def free_bytes():
    try:
        return os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
    except (ValueError, OSError):
        return None


# peak host memory of each generator, measured: 5.6 GB (c3), 12 GB (c4)
NEEDS = {"c3": 8 << 30, "c4": 16 << 30}


@pytest.mark.parametrize("config", ["c3", "c4"])
def test_record_matrix_is_the_generators(config):
    recs = [load(p) for p in RECORDS if os.path.basename(p).startswith(f"solve_{config}_")]
    recs = [r for r in recs if "matrix_sha256" in r]
    if not recs:
        pytest.skip(f"no fingerprinted {config} record")
    free = free_bytes()
    if free is not None and free < NEEDS[config]:
        pytest.skip(f"the {config} generator needs about {NEEDS[config] >> 30} GB of free host memory")
    import make_solve_references as writer

    rp, col, vals = writer.matrix(config).numpy()
    sha = writer.matrix_sha256(rp, col, vals)
    for r in recs:
        assert r["nnz"] == col.size
        assert r["matrix_sha256"] == sha, f"{config} {r['format']}: the generator's matrix changed"
