"""Writes the oracle's reference solves of the full-size systems as text fixtures.

Each fixture records one run of the oracle's restarted CB-GMRES (Fig. 1 of arXiv 2409.15468, x0 = 0,
tolerance 1e-10 on the explicit relative residual of Eq. 4) on one of the benchmark systems:

  c3  3D 7-point convection-diffusion on a 256^3 grid (n = 16 777 216), wind (1,1,1), Peclet 50,
      b = A 1, restart 100 (the Methodology's restart length);
  c4  the power-law random matrix with n = 2^22 rows (seed 2), b = A 1, restart 100;
  c3m the 3D operator of c3 on a 48^3 grid (n = 110 592), b = A 1, restart 100: the mid-size case
      of the streamed tests;
  c1  2D 5-point convection-diffusion on a 64^2 grid (n = 4096), wind (1, 0.5), Peclet 10,
      b = A x_true with x_true uniform in [-1, 1] (seed 0), restart 50.

A fixture holds the oracle's iteration, restart, second-pass and breakdown counts, its final
explicit and implicit residuals, the norm and SHA-256 of its solution x, and x at a seeded sample
of indices (full precision, as float.hex()), so that a GPU run can be compared with it without
rerunning a solve that takes the oracle hours. Only ``oracle`` (the CPU reference) and
``workloads`` (the seeded input generators) are called here; nothing of the CUDA library.

With --band K the fixture also records the oracle's step counts for K right-hand sides that
differ from b in 8 seeded entries by one unit in the last place (the spread of the count under
rounding-level changes of the input: the short bases turn such changes into different Krylov
spaces). The oracle uses IEEE operations only, so these numbers are the same on every host.

Usage: python tests/golden/make_solve_references.py {c3,c4,c3m,c1} {fp64,fp32,fp16,bf16,frsz2_16,frsz2_21,frsz2_32} [--band K]
       python tests/golden/make_solve_references.py CONFIG FORMAT --fingerprint   (adds the matrix
       fingerprint to an existing record)
The fixture is written to tests/golden/solve_<config>_<format>.json.
"""
from __future__ import annotations

import hashlib
import json
import os
import platform
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads  # noqa: E402

CONFIGS = {
    "c3": "3D 7-point convection-diffusion 256^3 (n=16777216, nnz=117047296), wind (1,1,1)*50",
    "c4": "power-law random nonsymmetric n=4194304 (row lengths min(2000, floor(10 U^-1/1.5)), N(0,1) "
          "off-diagonals, diag 1.2 x row abs-sum, seed 2)",
    "c3m": "3D 7-point convection-diffusion 48^3 (n=110592), wind (1,1,1)*50",
    "c1": "2D 5-point convection-diffusion 64^2 (n=4096, nnz=20224), wind (1,0.5)*10",
}
RESTART = {"c3": 100, "c4": 100, "c3m": 100, "c1": 50}
SAMPLE = 1024


def matrix(config: str):
    if config == "c3":
        return workloads.convdiff(256, 3, (1.0, 1.0, 1.0), 50.0)
    if config == "c3m":
        return workloads.convdiff(48, 3, (1.0, 1.0, 1.0), 50.0)
    if config == "c4":
        return workloads.powerlaw(1 << 22, seed=2)
    if config == "c1":
        return workloads.convdiff(64, 2, (1.0, 0.5), 10.0)
    raise ValueError(config)


def rhs(config: str, rp, col, vals) -> tuple[np.ndarray, str]:
    n = rp.size - 1
    if config == "c1":
        return oracle.spmv(rp, col, vals, workloads.uniform_vector(n, 0).numpy()), \
            "b = A x_true, x_true uniform in [-1, 1] (seed 0; oracle SpMV)"
    return oracle.spmv(rp, col, vals, np.ones(n)), "b = A * ones (oracle SpMV)"


def sample_indices(n: int) -> np.ndarray:
    rng = np.random.default_rng(20240923)
    idx = np.unique(np.concatenate([[0, n - 1], rng.integers(0, n, SAMPLE)]))
    return idx


def matrix_sha256(rp, col, vals) -> str:
    """Fingerprint of the CSR arrays (int32 row pointers and columns, float64 values): a record is
    only comparable with a solve of the same matrix, and the power-law generator draws from the
    host's random number generator."""
    h = hashlib.sha256()
    for a, t in ((rp, np.int32), (col, np.int32), (vals, np.float64)):
        h.update(np.ascontiguousarray(a, dtype=t).tobytes())
    return h.hexdigest()


def fingerprint(config: str, fname: str) -> None:
    """Adds the matrix fingerprint and nnz to an existing record (regenerating the matrix)."""
    path = os.path.join(HERE, f"solve_{config}_{fname}.json")
    with open(path) as f:
        rec = json.load(f)
    rp, col, vals = matrix(config).numpy()
    rec["nnz"] = int(col.size)
    rec["matrix_sha256"] = matrix_sha256(rp, col, vals)
    with open(path, "w") as f:
        json.dump(rec, f, indent=1)
        f.write("\n")
    print(path, rec["nnz"], rec["matrix_sha256"])


def main():
    config, fname = sys.argv[1], sys.argv[2]
    if "--fingerprint" in sys.argv:
        fingerprint(config, fname)
        return
    fmt, l = (oracle.FRSZ2, int(fname.split("_")[1])) if fname.startswith("frsz2") else (oracle.FORMAT_NAMES[fname], 32)
    A = matrix(config)
    rp, col, vals = A.numpy()
    del A
    oracle.build()
    b, b_desc = rhs(config, rp, col, vals)
    restart = RESTART[config]
    t0 = time.time()
    r = oracle.gmres(rp, col, vals, b, restart=restart, tol=1e-10, max_iters=20000, fmt=fmt, l=l)
    dt = time.time() - t0
    rrn = oracle.nrm2(b - oracle.spmv(rp, col, vals, r.x)) / oracle.nrm2(b)
    idx = sample_indices(r.x.size)
    out = {
        "what": "oracle CB-GMRES (Fig. 1) reference solve, written by tests/golden/make_solve_references.py",
        "cite": "Fig. 1 (restarted CB-GMRES); Methodology (x0 = 0, Eq. 4 relative residual)",
        "config": config,
        "matrix": CONFIGS[config],
        "nnz": int(col.size),
        "matrix_sha256": matrix_sha256(rp, col, vals),
        "rhs": b_desc,
        "format": fname,
        "restart": restart,
        "tol": 1e-10,
        "max_iters": 20000,
        "iters": int(r.iters),
        "restarts": int(r.restarts),
        "reorths": int(r.reorths),
        "breakdowns": int(r.breakdowns),
        "converged": bool(r.converged),
        "true_rrn": r.true_rrn,
        "implicit_rrn": r.implicit_rrn,
        "rrn_recomputed": rrn,
        "x_norm2": oracle.nrm2(r.x),
        "x_sha256": hashlib.sha256(np.ascontiguousarray(r.x).tobytes()).hexdigest(),
        "hist_true": [float(v) for v in r.hist_true],
        "oracle_seconds": dt,
        "host": f"{platform.machine()} {platform.processor() or ''}".strip(),
        "sample_index": [int(i) for i in idx],
        "sample_x": [float(r.x[i]).hex() for i in idx],
    }
    path = os.path.join(HERE, f"solve_{config}_{fname}.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(path, r.iters, r.reorths, r.breakdowns, r.true_rrn, f"{dt:.1f} s")
    if "--band" in sys.argv:
        from concurrent.futures import ThreadPoolExecutor

        k = int(sys.argv[sys.argv.index("--band") + 1])

        def perturbed(seed):  # the oracle's C code runs outside the interpreter lock
            bb = b.copy()
            idx = np.random.default_rng(seed).integers(0, bb.size, 8)
            bb[idx] = np.nextafter(bb[idx], np.inf)
            return oracle.gmres(rp, col, vals, bb, restart=restart, tol=1e-10, max_iters=20000, fmt=fmt, l=l).iters

        with ThreadPoolExecutor(min(k, os.cpu_count() or 1)) as ex:
            band = list(ex.map(perturbed, range(1, k + 1)))
        out["iters_perturbed_b"] = band
        out["iters_perturbed_b_note"] = ("step counts for b with 8 entries (seeds 1..K) moved up by one ulp; "
                                         "the spread of the count under rounding-level changes of the input")
        with open(path, "w") as f:
            json.dump(out, f, indent=1)
            f.write("\n")
        print("band", min(band + [r.iters]), max(band + [r.iters]), band)


if __name__ == "__main__":
    main()
