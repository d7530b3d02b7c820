#!/usr/bin/env python
"""Benchmark of the CB-GMRES / FRSZ2 hot path on GB300.

Default workload (one step = one pass of the basis hot path over the standalone basis
configuration): a basis of 100 vectors x n = 2^24 values, N(0,1) * 2^k with k uniform in [-20, 20]
per 32-value block (seed 1, unit-norm vectors), stored as FRSZ2 with l = 32. A step

  1. compresses the step's vector w (n FP64 values) into the basis      (Fig. 1 steps 13-14)
  2. h := V^T w over the 100 stored vectors, decoded in registers         (step 5)
  3. w := w - V h over the 100 stored vectors, with ||w||^2              (steps 5-6)

all through the C ABI on the current stream. `value` is the algorithmic HBM traffic of a step
divided by its time (GB/s). The JSON line also carries the roofline of the dominant kernel, the
oracle timed on host cores on a bounded sample (cpu_baseline), the same step through host
buffers (e2e), the other storage formats, and the time to a 1e-10 relative residual of a full
CB-GMRES solve with the FRSZ2 and the fp64 basis.

`--impl reference` times the oracle (plain C, its rows split over the host's cores) on a bounded
sample of the same step. Under torchrun (N > 1) every rank runs its own replica of the workload (weak scaling, no
collective on the data path); rank 0 prints the line.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time to 1e-10 rel. residual, FRSZ2 vs fp64 basis; basis GB/s; p99 latency"
FMT_CODES = {"fp64": 0, "fp32": 1, "fp16": 2, "bf16": 3, "frsz2": 4}
VALUE_BYTES = {"fp64": 8, "fp32": 4, "fp16": 2, "bf16": 2}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "of measured (MEASURED_PEAKS.json hbm_gbs, torch copy)"
    return 6800.0, "of fallback (6.8 TB/s)"


def stored_bytes(fmt: str, l: int, n: int) -> int:
    """Bytes of one stored vector that a basis kernel reads: Eq. 3 for FRSZ2, n x width for casts."""
    if fmt == "frsz2":
        nb = (n + 31) // 32
        return nb * l * 4 + nb * 4
    return n * VALUE_BYTES[fmt]


def step_config(args, workload: str, world: int) -> dict:
    """The bench line's config: the same dict on the GPU arm and the reference arm (the oracle), so
    both lines name one workload."""
    per_step = sum(step_bytes(args.fmt, args.bits, args.n, args.nvec).values())
    return {"workload": workload, "n": args.n, "nvec": args.nvec, "format": args.fmt, "frsz2_bits": args.bits,
            "bytes_per_step": per_step, "l2": "inputs larger than L2 (no flush needed)",
            "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"}


def step_bytes(fmt: str, l: int, n: int, nvec: int):
    vb = stored_bytes(fmt, l, n)
    return {"store": 8 * n + vb, "dot": nvec * vb + 8 * n, "update": nvec * vb + 16 * n}


def traffic_from_profiles(kernel_tag: str):
    """Per-launch DRAM bytes of a kernel from the committed ncu summary (profiles/*.txt), if any."""
    d = os.path.join(ROOT, "profiles")
    if not os.path.isdir(d):
        return None
    for name in sorted(os.listdir(d)):
        if not name.endswith(".txt"):
            continue
        with open(os.path.join(d, name)) as f:
            for line in f:
                if line.startswith("traffic_bytes_per_full_launch") and kernel_tag in line:
                    try:
                        return float(line.split("=")[1].split()[0])
                    except (IndexError, ValueError):
                        return None
    return None


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples every 200 ms while running."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                    power.append(float(parts[3]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power)}


# ------------------------------------------------------------------------------------------------
# GPU arm
# ------------------------------------------------------------------------------------------------

def make_basis(pkg, torch, fmt, l, n, nvec, device):
    B = pkg.BasisStorage(n, nvec + 1, FMT_CODES[fmt], l, device=device)
    import workloads

    for i in range(nvec):
        B.store(i, workloads.basis_vector(i, n, seed=1, device=device))
    w = workloads.basis_vector(nvec, n, seed=1, device=device)
    torch.cuda.synchronize(device)
    return B, w


def time_steps(pkg, torch, B, w, nvec, steps, warmup, per_kernel=False):
    """Times `steps` steps on the current stream with CUDA events; returns (total_ms, per-kernel ms)."""
    stream = torch.cuda.current_stream()
    h = torch.empty(nvec, dtype=torch.float64, device=w.device)
    nrm = torch.empty(1, dtype=torch.float64, device=w.device)
    work = B.work(nvec)

    def one():
        B.store(nvec, w)
        B.dot(nvec, w, out=h, work=work)
        B.update(nvec, h, w, norm2=nrm, work=work)

    for _ in range(warmup):
        one()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    kev = []
    if per_kernel:
        kev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(steps)]
    ev[0].record(stream)
    for s in range(steps):
        if per_kernel:
            e = kev[s]
            e[0].record(stream)
            B.store(nvec, w)
            e[1].record(stream)
            B.dot(nvec, w, out=h, work=work)
            e[2].record(stream)
            B.update(nvec, h, w, norm2=nrm, work=work)
            e[3].record(stream)
        else:
            one()
    ev[1].record(stream)
    torch.cuda.synchronize()
    total = ev[0].elapsed_time(ev[1])
    kms = None
    if per_kernel:
        kms = {"store": float(np.mean([e[0].elapsed_time(e[1]) for e in kev])),
               "dot": float(np.mean([e[1].elapsed_time(e[2]) for e in kev])),
               "update": float(np.mean([e[2].elapsed_time(e[3]) for e in kev]))}
    return total, kms


def time_e2e(pkg, torch, B, w, nvec, steps, warmup):
    """The same step through host buffers: every step's w is copied in from pinned host memory and
    h, ||w||^2 go back to pinned host memory, all inside the timed region. The input copy of step
    k + 1 runs on a copy stream while step k computes (two device buffers, ordered by events), as a
    serving pipeline would do; the timed region spans the first copy to the last result read."""
    stream = torch.cuda.current_stream()
    copy_stream = torch.cuda.Stream()
    n = w.numel()
    w_host = w.cpu().pin_memory()
    h_host = torch.empty(nvec, dtype=torch.float64).pin_memory()
    nrm_host = torch.empty(1, dtype=torch.float64).pin_memory()
    wd = [torch.empty_like(w), torch.empty_like(w)]
    copied = [torch.cuda.Event(), torch.cuda.Event()]
    used = [torch.cuda.Event(), torch.cuda.Event()]
    h = torch.empty(nvec, dtype=torch.float64, device=w.device)
    nrm = torch.empty(1, dtype=torch.float64, device=w.device)
    work = B.work(nvec)

    def copy_in(k):
        i = k % 2
        with torch.cuda.stream(copy_stream):
            if k >= 2:
                copy_stream.wait_event(used[i])  # step k - 2 is done with this buffer
            wd[i].copy_(w_host, non_blocking=True)
            copied[i].record(copy_stream)

    def run(count, e0=None, e1=None):
        if e0 is not None:
            e0.record(stream)
        copy_stream.wait_stream(stream)  # no copy of this run starts before the timed region does
        copy_in(0)
        for k in range(count):
            i = k % 2
            if k + 1 < count:
                copy_in(k + 1)
            stream.wait_event(copied[i])
            B.store(nvec, wd[i])
            B.dot(nvec, wd[i], out=h, work=work)
            B.update(nvec, h, wd[i], norm2=nrm, work=work)
            used[i].record(stream)
            h_host.copy_(h, non_blocking=True)
            nrm_host.copy_(nrm, non_blocking=True)
        if e1 is not None:
            e1.record(stream)

    run(warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    run(steps, e0, e1)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), 8 * n, 8 * nvec + 8


def time_to_tol(pkg, torch, device, repeats=3):
    """Full CB-GMRES solves to a 1e-10 relative residual on the 64x64 convection-diffusion system
    (restart 50), FRSZ2-32 vs fp64 basis, through cbgmres_solve with device-resident b and x. A
    system this small runs each restart cycle as one thread-block cluster launch (the default,
    cycle="auto"); the same solves with the streamed kernels (cycle="streamed") are timed beside
    them. Per entry: median seconds of `repeats` solves after one warm-up, and us per Arnoldi step."""
    import workloads

    A = workloads.convdiff(64, 2, (1.0, 0.5), 10.0, device=device)
    xt = workloads.uniform_vector(A.n, 0, device=device)
    b = pkg.spmv(A.row_ptr, A.col, A.vals, xt).clone()
    out = {}
    for cycle in ("auto", "streamed"):
        for fmt in ("fp64", "frsz2"):
            S = pkg.Solver(A.row_ptr, A.col, A.vals, restart=50, tol=1e-10, fmt=fmt, frsz2_bits=32, cycle=cycle)
            ts, r = [], None
            for _ in range(repeats + 1):
                x = torch.zeros(A.n, dtype=torch.float64, device=device)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                r = S.solve(b, x)
                ts.append(time.perf_counter() - t0)
            sec = float(np.median(ts[1:]))
            key = fmt if cycle == "auto" else f"{fmt}_streamed"
            out[key] = {"seconds": sec, "iters": r.iters, "converged": r.converged, "true_rrn": r.true_rrn,
                        "us_per_step": sec / max(r.iters, 1) * 1e6, "cycle_cluster": S.cycle_cluster}
            S.close()
    out["speedup_frsz2_vs_fp64"] = out["fp64"]["seconds"] / out["frsz2"]["seconds"]
    out["speedup_onchip_vs_streamed_frsz2"] = out["frsz2_streamed"]["seconds"] / out["frsz2"]["seconds"]
    # every storage format on chip (one warm-up, then the median of `repeats` solves)
    fmts = {}
    for name, fmt, bits in (("fp64", "fp64", 32), ("fp32", "fp32", 32), ("fp16", "fp16", 32), ("bf16", "bf16", 32),
                            ("frsz2_16", "frsz2", 16), ("frsz2_21", "frsz2", 21), ("frsz2_32", "frsz2", 32)):
        S = pkg.Solver(A.row_ptr, A.col, A.vals, restart=50, tol=1e-10, fmt=fmt, frsz2_bits=bits)
        ts, r = [], None
        for _ in range(repeats + 1):
            x = torch.zeros(A.n, dtype=torch.float64, device=device)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = S.solve(b, x)
            ts.append(time.perf_counter() - t0)
        sec = float(np.median(ts[1:]))
        fmts[name] = {"seconds": sec, "iters": r.iters, "converged": r.converged, "true_rrn": r.true_rrn,
                      "us_per_step": sec / max(r.iters, 1) * 1e6, "cycle_cluster": S.cycle_cluster}
        S.close()
    out["formats_on_chip"] = fmts
    out["config"] = "2D 5-point convection-diffusion 64x64 (n=4096), wind (1,0.5)*10, b = A x_true, restart 50"
    return out


def stored_oracle_solve(matrix: str, fmt: str):
    """The oracle's own solve of the full-size system, as committed under tests/golden/ by
    tests/golden/make_solve_references.py (the oracle takes hours at this size), or None."""
    path = os.path.join(ROOT, "tests", "golden", f"solve_{matrix}_{fmt}.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        return json.load(f)


def solve_c3(pkg, torch, device, formats, N: int = 256, restart: int = 100, tol: float = 1e-10,
             max_iters: int = 20000, matrix: str = "c3"):
    """Full CB-GMRES(restart) solves to a relative residual of tol, one per basis format, through
    cbgmres_solve with device-resident b = A 1 and x0 = 0, on
      c3: the 3D 7-point convection-diffusion system on an N^3 grid (wind (1,1,1), Peclet 50);
      c4: the 4M-row power-law random matrix (row lengths Pareto, mean ~30, max 2000; seed 2).
    Each result is set against the oracle's solve of the same system stored in tests/golden/ when
    there is one: the step-count difference, the second passes, and the relative difference of x
    at the stored sample of indices."""
    import workloads

    if matrix == "c4":
        # generated on the host, as the oracle's stored solve is (the device generator draws other
        # random numbers), then moved to the GPU
        A = workloads.powerlaw(1 << 22, seed=2).to(device)
        desc = (f"power-law random nonsymmetric n={A.n}, nnz={A.nnz} (row lengths min(2000, floor(10 U^-1/1.5))"
                f", N(0,1) off-diagonals, diag 1.2 x row abs-sum, seed 2)")
    else:
        A = workloads.convdiff(N, 3, (1.0, 1.0, 1.0), 50.0, device=device)
        desc = f"3D 7-point convection-diffusion {N}^3 (n={A.n}, nnz={A.nnz}), wind (1,1,1)*50"
    b = pkg.spmv(A.row_ptr, A.col, A.vals, torch.ones(A.n, dtype=torch.float64, device=device)).clone()
    out = {"config": f"{desc}, b = A*1, x0 = 0, restart {restart}, tol {tol}, max_iters {max_iters}"}
    # SpMV alone (algorithmic bytes: values and column indices, row pointers, x once, y)
    y = torch.empty_like(b)
    for _ in range(3):
        pkg.spmv(A.row_ptr, A.col, A.vals, b, y=y)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(10):
        pkg.spmv(A.row_ptr, A.col, A.vals, b, y=y)
    e1.record()
    torch.cuda.synchronize()
    sp_ms = e0.elapsed_time(e1) / 10
    out["spmv"] = {"ms": sp_ms, "gbs": (12 * A.nnz + 4 * (A.n + 1) + 16 * A.n) / (sp_ms * 1e-3) / 1e9}
    for f in formats:
        fmt, bits = (f.split("_")[0], int(f.split("_")[1])) if f.startswith("frsz2") else (f, 32)
        S = pkg.Solver(A.row_ptr, A.col, A.vals, restart=restart, tol=tol, fmt=fmt, frsz2_bits=bits,
                       max_iters=max_iters)
        x = torch.zeros(A.n, dtype=torch.float64, device=device)
        torch.cuda.synchronize()
        t = time.perf_counter()
        r = S.solve(b, x)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t
        S.close()
        res = {"seconds": dt, "iters": r.iters, "restarts": r.restarts, "reorths": r.reorths,
               "breakdowns": r.breakdowns, "converged": r.converged, "true_rrn": r.true_rrn,
               "ms_per_iter": 1e3 * dt / max(r.iters, 1)}
        ref = stored_oracle_solve(matrix, f) if restart == 100 and tol == 1e-10 and (matrix == "c4" or N == 256) \
            else None
        if ref:
            idx = torch.tensor(ref["sample_index"], dtype=torch.int64, device=device)
            xo = torch.tensor([float.fromhex(v) for v in ref["sample_x"]], dtype=torch.float64, device=device)
            res["vs_oracle"] = {"oracle_iters": ref["iters"], "oracle_reorths": ref["reorths"],
                                "iters_diff_pct": 100.0 * (r.iters - ref["iters"]) / ref["iters"],
                                "x_rel_diff_at_samples": float(torch.linalg.vector_norm(x[idx] - xo) /
                                                               torch.linalg.vector_norm(xo)),
                                "oracle_true_rrn": ref["true_rrn"], "oracle_seconds_one_core": ref["oracle_seconds"]}
        out[f] = res
        del x
        torch.cuda.empty_cache()
    if "fp64" in out and "frsz2_32" in out:
        out["speedup_frsz2_32_vs_fp64"] = out["fp64"]["seconds"] / out["frsz2_32"]["seconds"]
    return out


ALL_FORMATS = ["fp64", "fp32", "fp16", "bf16", "frsz2_16", "frsz2_21", "frsz2_32"]


def exponent_spread(v: np.ndarray) -> dict:
    """Per 32-value block of a Krylov vector: the spread e_max - e_min of the IEEE exponents of its
    nonzero values (the quantity FRSZ2 truncates against), as a histogram, and the fraction of
    nonzero values each FRSZ2 width stores as zero (block-relative exponent gap >= l - 1)."""
    n = v.size
    nb = (n + 31) // 32
    pad = np.zeros(nb * 32)
    pad[:n] = v
    e = ((pad.view(np.uint64) >> np.uint64(52)) & np.uint64(0x7FF)).astype(np.int64).reshape(nb, 32)
    nz = e > 0
    emax = e.max(axis=1)
    emin = np.where(nz, e, 1 << 12).min(axis=1)
    spread = np.where(nz.any(axis=1), emax - emin, 0)
    hist = np.bincount(np.minimum(spread, 64), minlength=65)
    gap = emax[:, None] - e
    total = max(int(nz.sum()), 1)
    return {"spread_hist": {str(i): int(c) for i, c in enumerate(hist) if c},
            "spread_quantiles": {q: float(np.quantile(spread, float(q))) for q in ("0.5", "0.9", "0.99")},
            "zero_fraction": {f"frsz2_{l}": float(((gap >= l - 1) & nz).sum() / total) for l in (16, 21, 32)}}


def sweep(pkg, torch, device, matrix: str = "c3", rhs: str = "ones", formats=None, target_iters: int = 0,
          restart: int = 100, tol: float = 1e-10, max_iters: int = 20000, hist_every: int = 25):
    """The basis-format sweep (iteration ratios against the fp64 basis, implicit-RRN histories and
    per-block exponent spreads of the Krylov vectors) on c3 (256^3 convection-diffusion) or c4 (4M
    power-law). rhs "ones": b = A 1; "sin": b = A x_sol with x_sol = s / ||s||, s_i = sin(i), the
    Methodology's right-hand side. target_iters > 0 takes the Methodology's stopping protocol: the
    RRN reached by target_iters iterations of fp64-basis GMRES, times 1.1, is every format's
    tolerance."""
    import workloads

    formats = formats or ALL_FORMATS
    if matrix == "c4":
        A = workloads.powerlaw(1 << 22, seed=2, device=device)
    else:
        A = workloads.convdiff(256, 3, (1.0, 1.0, 1.0), 50.0, device=device)
    if rhs == "sin":
        s_ = workloads.sin_vector(A.n, device=device)
        xs = s_ / torch.linalg.vector_norm(s_)
    else:
        xs = torch.ones(A.n, dtype=torch.float64, device=device)
    b = pkg.spmv(A.row_ptr, A.col, A.vals, xs).clone()
    out = {"matrix": matrix, "n": A.n, "nnz": A.nnz, "rhs": rhs, "restart": restart}
    if target_iters > 0:
        S = pkg.Solver(A.row_ptr, A.col, A.vals, restart=restart, tol=1e-300, fmt="fp64", max_iters=target_iters)
        x = torch.zeros(A.n, dtype=torch.float64, device=device)
        r64 = S.solve(b, x)
        S.close()
        tol = 1.1 * r64.true_rrn
        out["target_protocol"] = {"fp64_iters": r64.iters, "fp64_rrn": r64.true_rrn, "tol": tol}
    out["tol"] = tol
    for f in formats:
        fmt, bits = (f.split("_")[0], int(f.split("_")[1])) if f.startswith("frsz2") else (f, 32)
        S = pkg.Solver(A.row_ptr, A.col, A.vals, restart=restart, tol=tol, fmt=fmt, frsz2_bits=bits,
                       max_iters=max_iters, history=1)
        x = torch.zeros(A.n, dtype=torch.float64, device=device)
        torch.cuda.synchronize()
        t = time.perf_counter()
        r = S.solve(b, x)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t
        h = S.history()
        res = {"seconds": dt, "iters": r.iters, "restarts": r.restarts, "reorths": r.reorths,
               "converged": r.converged, "true_rrn": r.true_rrn,
               "x_rel_error": float(torch.linalg.vector_norm(x - xs) / torch.linalg.vector_norm(xs)),
               "rrn_history": [[k + 1, float(h[k])] for k in range(hist_every - 1, len(h), hist_every)]}
        if f in ("fp64", "frsz2_32") and r.iters > 0:
            m_last = r.iters - (r.restarts - 1) * restart if r.restarts > 0 else r.iters
            m_last = max(1, min(restart, m_last))  # slots 0 .. m_last - 1 hold the last cycle's basis
            res["exponent_spread"] = {str(k): exponent_spread(S.basis_vector(k).cpu().numpy())
                                      for k in sorted({0, m_last // 2, m_last - 1})}
        S.close()
        out[f] = res
        del x
        torch.cuda.empty_cache()
    if "fp64" in out:
        out["iteration_ratio_vs_fp64"] = {f: out[f]["iters"] / max(out["fp64"]["iters"], 1) for f in formats}
        out["time_ratio_vs_fp64"] = {f: out[f]["seconds"] / out["fp64"]["seconds"] for f in formats}
    return out


def spmv_only(pkg, torch, device, kind: str, size: int, runs: int = 10):
    """The SpMV alone: c3 = 3D convection-diffusion on a size^3 grid, c4 = power-law matrix with
    `size` rows; the minimum of `runs` CUDA-event timings, algorithmic bytes 12 nnz + 20 n."""
    import workloads

    if kind == "c4":
        A = workloads.powerlaw(size, seed=2, device=device)
    else:
        A = workloads.convdiff(size, 3, (1.0, 1.0, 1.0), 50.0, device=device)
    x = torch.ones(A.n, dtype=torch.float64, device=device)
    y = torch.empty_like(x)
    nrm = torch.empty(1, dtype=torch.float64, device=device)
    for _ in range(2):
        pkg.spmv(A.row_ptr, A.col, A.vals, x, y=y, norm2=nrm)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best = float("inf")
    for _ in range(runs):
        e0.record()
        pkg.spmv(A.row_ptr, A.col, A.vals, x, y=y, norm2=nrm)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    byt = 12 * A.nnz + 4 * (A.n + 1) + 16 * A.n
    return {"matrix": kind, "n": A.n, "nnz": A.nnz, "ms": best, "gbs": byt / (best * 1e-3) / 1e9,
            "algorithmic_bytes": byt}


INTENSITY_R = [0, 1, 2, 3, 4, 5, 6, 7, 8, 10, 12, 14, 16, 20, 24, 28, 32, 40, 48, 56, 64, 80, 96, 112, 128, 192, 256]


def intensity_sweep(pkg, torch, device, n: int = 1 << 28, runs: int = 10, peak_gbs: float = 0.0):
    """The synthetic arithmetic-intensity benchmark (Fig. 3 protocol): 2^28 stored values per
    format, 27 settings of r fused multiply-adds per value, the minimum of 10 runs each (CUDA
    events). Per value 2r + 1 floating-point operations over the format's bytes per value."""
    import workloads

    variants = [("fp64", 32, False), ("fp32", 32, True), ("fp32", 32, False), ("fp16", 32, False),
                ("bf16", 32, False), ("frsz2", 16, False), ("frsz2", 21, False), ("frsz2", 32, False)]
    x = workloads.basis_vector(0, n, seed=1, device=device)
    out = {"n": n, "runs": runs, "r": INTENSITY_R,
           "roofs": {"hbm_gbs": peak_gbs, "fp64_gflops_probe": 2 * 599.4,
                     "fp64_note": "DFMA 599 G op/s measured on this pool's GB300 by an FMA-chain probe",
                     "fp32_gflops_probe": 2 * 37477.0}}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for fmt, l, native in variants:
        B = pkg.BasisStorage(n, 1, pkg.FORMATS[fmt], l)
        B.store(0, x)
        vb = stored_bytes(fmt, l, n)
        res = torch.empty(1, dtype=torch.float64, device=device)
        work = B.work(1)
        rows = []
        for r in INTENSITY_R:
            B.intensity(0, r, fp32_compute=native, out=res, work=work)
            best = float("inf")
            for _ in range(runs):
                e0.record()
                B.intensity(0, r, fp32_compute=native, out=res, work=work)
                e1.record()
                torch.cuda.synchronize()
                best = min(best, e0.elapsed_time(e1))
            flops = n * (2 * r + 1)
            rows.append({"r": r, "flop_per_byte": flops / vb, "gflops": flops / (best * 1e-3) / 1e9,
                         "gbs": vb / (best * 1e-3) / 1e9, "ms": best})
        name = (fmt if fmt != "frsz2" else f"frsz2_{l}") + ("_native_fp32" if native else "")
        out[name] = rows
        del B, work
        torch.cuda.empty_cache()
    return out


def serving(pkg, torch, device, count: int, n_min: float, n_max: float, budget_gb: float = 96.0,
            max_active: int = 16, steps_per_turn: int = 8, restart: int = 100, seed: int = 3):
    """The serving workload: a Poisson stream of convection-diffusion solves (n log-uniform in
    [n_min, n_max], 2D/3D, Pe in [1, 100], tol in {1e-8, 1e-10, 1e-12}, basis format uniform over
    the seven storage formats), served by the library's runtime (cbg_server_*) within an HBM
    budget. The arrival rate is 0.8 of the capacity measured with every request submitted at once.
    The baseline is sequential fp64-basis GMRES: each request's own solve time with the fp64
    basis (context creation excluded), replayed through a FIFO queue with the same arrivals."""
    import workloads

    reqs = workloads.serving_mix(count, 1.0, seed=seed, n_min=n_min, n_max=n_max)
    cases = []
    for r in reqs:
        A = workloads.convdiff(r.N, r.dim, r.wind, r.peclet, device=device)
        xt = workloads.uniform_vector(A.n, 1000 + r.rid, device=device)
        b = pkg.spmv(A.row_ptr, A.col, A.vals, xt).clone()
        o = pkg.default_opts(restart=min(restart, A.n), fmt=r.fmt, frsz2_bits=r.frsz2_bits, tol=r.tol,
                             max_iters=20000)
        cases.append((r, A, b, o))
    torch.cuda.synchronize()

    def run(arrivals):
        srv = pkg.Server(int(budget_gb * 1e9), max_active=max_active, steps_per_turn=steps_per_turn, max_bypass=8)
        xs = [torch.zeros(A.n, dtype=torch.float64, device=device) for _, A, _, _ in cases]
        done, nxt = {}, 0
        t0 = srv.clock()
        while len(done) < len(cases):
            now = srv.clock() - t0
            while nxt < len(cases) and arrivals[nxt] <= now:
                r, A, b, o = cases[nxt]
                srv.submit(nxt, A.row_ptr, A.col, A.vals, b, xs[nxt], o)
                nxt += 1
            for c in srv.poll():
                done[c.tag] = c
        srv.close()
        lat = np.array([done[i].t_done - t0 - arrivals[i] for i in range(len(cases))])
        span = max(c.t_done for c in done.values()) - t0 - arrivals[0]
        ok = sum(1 for c in done.values() if c.status == 0 and c.result.converged)
        return lat, span, ok

    # capacity: everything submitted at t = 0
    lat0, span0, _ = run(np.zeros(len(cases)))
    capacity = len(cases) / span0
    rate = 0.8 * capacity
    arrivals = np.array([r.arrival_s for r, _, _, _ in cases]) / rate
    lat, span, ok = run(arrivals)
    # sequential fp64-basis GMRES: per-request solve time, then a FIFO queue over the same arrivals
    service = []
    for r, A, b, o in cases:
        o64 = pkg.default_opts(restart=o.restart, fmt="fp64", tol=o.tol, max_iters=20000)
        S = pkg.Solver(A.row_ptr, A.col, A.vals, opts=o64)
        x = torch.zeros(A.n, dtype=torch.float64, device=device)
        torch.cuda.synchronize()
        t = time.perf_counter()
        S.solve(b, x)
        torch.cuda.synchronize()
        service.append(time.perf_counter() - t)
        S.close()
    fin, seq_lat = 0.0, []
    for a, sv in zip(arrivals, service):
        fin = max(fin, a) + sv
        seq_lat.append(fin - a)
    seq_lat = np.array(seq_lat)
    ns = [A.n for _, A, _, _ in cases]
    return {"requests": len(cases), "served_converged": ok,
            "n_range": [int(min(ns)), int(max(ns))], "n_log_uniform": [n_min, n_max],
            "capacity_solves_per_s": capacity, "arrival_rate_per_s": rate,
            "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "solves_per_s": len(cases) / span,
            "sequential_fp64": {"p50_latency_s": float(np.percentile(seq_lat, 50)),
                                "p99_latency_s": float(np.percentile(seq_lat, 99)),
                                "solves_per_s": len(cases) / (fin - arrivals[0]),
                                "capacity_solves_per_s": len(cases) / sum(service)},
            "server": {"hbm_budget_gb": budget_gb, "max_active": max_active, "steps_per_turn": steps_per_turn,
                       "restart": restart},
            "config": "Poisson arrivals at 0.8 x measured capacity; 2D/3D convection-diffusion 50/50, Pe U[1,100], "
                      "wind ones; tol {1e-8,1e-10,1e-12}; basis format uniform over fp64/fp32/fp16/bf16/frsz2_16/21/32;"
                      " b = A x, x U[-1,1]; seed 3"}


# ------------------------------------------------------------------------------------------------
# Oracle (CPU) arm
# ------------------------------------------------------------------------------------------------

def oracle_step_setup(n: int, nvec: int):
    import oracle
    import workloads

    oracle.build()
    V = [oracle.encode(workloads.basis_vector(i, n, seed=1).numpy(), oracle.FRSZ2, 32) for i in range(nvec)]
    w = workloads.basis_vector(nvec, n, seed=1).numpy().copy()
    return oracle, V, w


def oracle_step(oracle, V, w, n, nvec, pool=None, chunks=1):
    """The benchmark step on the host with the oracle as it stands: compress w, decode every stored
    vector and take the sequential dot, then decode again and subtract (sequential axpy). With a
    thread pool the rows are split into `chunks` ranges of whole 32-value blocks, each thread runs
    the same oracle calls on its range (ctypes releases the interpreter lock), and every h_i is the
    sum of the ranges' partial dots in range order, so the result does not depend on scheduling."""
    if pool is None or chunks <= 1:
        oracle.encode(w, oracle.FRSZ2, 32)
        h = np.empty(nvec)
        for i, (vals, exps) in enumerate(V):
            h[i] = oracle.dot(oracle.decode(vals, exps, n, oracle.FRSZ2, 32), w)
        for i, (vals, exps) in enumerate(V):
            oracle.axpy(-h[i], oracle.decode(vals, exps, n, oracle.FRSZ2, 32), w)
        return h, oracle.dot(w, w)
    nb = (n + 31) // 32
    bounds = [(nb * c // chunks, nb * (c + 1) // chunks) for c in range(chunks)]

    def rows(b0, b1):
        return b0 * 32, min(n, b1 * 32)

    def part_dots(rng):
        b0, b1 = rng
        k0, k1 = rows(b0, b1)
        oracle.encode(w[k0:k1], oracle.FRSZ2, 32)
        return [oracle.dot(oracle.decode(vals[b0 * 32:b1 * 32], exps[b0:b1], k1 - k0, oracle.FRSZ2, 32), w[k0:k1])
                for vals, exps in V]

    parts = list(pool.map(part_dots, bounds))
    h = np.array([sum(p[i] for p in parts) for i in range(nvec)])

    def part_update(rng):
        b0, b1 = rng
        k0, k1 = rows(b0, b1)
        wc = w[k0:k1]
        for i, (vals, exps) in enumerate(V):
            oracle.axpy(-h[i], oracle.decode(vals[b0 * 32:b1 * 32], exps[b0:b1], k1 - k0, oracle.FRSZ2, 32), wc)
        return oracle.dot(wc, wc)

    norms = list(pool.map(part_update, bounds))
    return h, sum(norms)


def oracle_rate(n: int, nvec: int, steps: int, warmup: int, threads: int = 1):
    from concurrent.futures import ThreadPoolExecutor

    oracle, V, w = oracle_step_setup(n, nvec)
    pool = ThreadPoolExecutor(threads) if threads > 1 else None
    try:
        for _ in range(warmup):
            oracle_step(oracle, V, w, n, nvec, pool, threads)
        t0 = time.perf_counter()
        for _ in range(steps):
            oracle_step(oracle, V, w, n, nvec, pool, threads)
        dt = time.perf_counter() - t0
    finally:
        if pool:
            pool.shutdown()
    byt = sum(step_bytes("frsz2", 32, n, nvec).values()) * steps
    return byt / dt / 1e9, dt


def choose_oracle_sample(nvec: int, steps_total: int, budget_s: float, n_full: int, threads: int = 1) -> int:
    """Largest sample (a multiple of 32 * threads * 4 values) whose steps_total steps fit in budget_s."""
    n0 = 4096 * max(1, threads)
    _, dt = oracle_rate(n0, nvec, 1, 0, threads)
    per_value = dt / n0
    q = 128 * max(1, threads)
    n = int(budget_s / max(steps_total, 1) / per_value)
    n = max(q, min(n_full, n // q * q))
    return n


def cpu_baseline(n_full: int, nvec: int):
    """The oracle on the host cores: on all of them (row ranges in threads, deterministic
    reduction), and on one core, each on a bounded sample of the workload's rows."""
    cores = os.cpu_count() or 1
    n = choose_oracle_sample(nvec, 3, 12.0, n_full, cores)
    gbs, dt = oracle_rate(n, nvec, 3, 0, cores)
    n1 = choose_oracle_sample(nvec, 3, 8.0, n_full)
    gbs1, dt1 = oracle_rate(n1, nvec, 3, 0)
    return {"value": gbs, "unit": "GB/s", "cores": cores, "kind": "oracle",
            "sample": f"3 steps over {nvec} x {n} values ({n / n_full:.5f} of the workload's n), plain C oracle, "
                      f"rows split over {cores} threads, {dt:.1f} s",
            "nproc": cores,
            "single_core": {"value": gbs1, "unit": "GB/s", "cores": 1,
                            "sample": f"3 steps over {nvec} x {n1} values, {dt1:.1f} s"}}


def oracle_solve_rate(config: str, fmt: str = "frsz2_32", restart: int = 100) -> dict:
    """The oracle's CB-GMRES on the host, one core, per Arnoldi step at the full size of c3 (256^3
    convection-diffusion) or c4 (the 2^22-row power-law matrix): one whole restart cycle (restart
    steps, second passes included) of the same operator at a reduced size (64^3, resp. 2^18 rows)
    is timed, and its time per step is scaled by the row count (a step's work is linear in n at a
    fixed restart length). The oracle's memory traffic grows faster than its cache share at the full
    size, so the scaled figure is a lower bound on the full-size time per step."""
    import oracle
    import workloads

    oracle.build()
    if config == "c3":
        A = workloads.convdiff(64, 3, (1.0, 1.0, 1.0), 50.0)
        scale, small = (256 / 64) ** 3, "64^3"
    else:
        A = workloads.powerlaw(1 << 18, seed=2)
        scale, small = float(1 << 4), "2^18 rows"
    rp, col, vals = A.numpy()
    b = oracle.spmv(rp, col, vals, np.ones(A.n))
    f, l = ("frsz2", int(fmt.split("_")[1])) if fmt.startswith("frsz2") else (fmt, 32)
    t = time.perf_counter()
    r = oracle.gmres(rp, col, vals, b, restart=restart, tol=1e-300, max_iters=restart,
                     fmt=oracle.FORMAT_NAMES[f], l=l)
    dt = time.perf_counter() - t
    return {"s_per_step_full_size": dt / max(r.iters, 1) * scale, "unit": "s per Arnoldi step", "cores": 1,
            "format": fmt, "sample": f"one restart cycle ({r.iters} steps, {r.reorths} second passes) on {small}, "
                                    f"{dt:.1f} s, scaled by n x{scale:g}"}


def add_oracle_solve_rates(line: dict) -> None:
    """cpu_baseline.solves: the oracle's time per Arnoldi step on c3 and c4 (oracle_solve_rate), and
    extrapolated to the step count the GPU solve of the same system took to reach 1e-10; with the
    oracle's full solve time from its stored record when one is committed (one core, on the host
    that wrote it)."""
    out = {}
    for config, key in (("c3", "time_to_tol_c3"), ("c4", "time_to_tol_c4")):
        rate = oracle_solve_rate(config)
        gpu = line.get(key, {}).get("frsz2_32")
        if gpu:
            rate["gpu_steps_to_tol"] = gpu["iters"]
            rate["time_to_tol_extrapolated_s"] = rate["s_per_step_full_size"] * gpu["iters"]
            rate["gpu_seconds"] = gpu["seconds"]
        ref = stored_oracle_solve(config, "frsz2_32")
        if ref:
            rate["stored_full_solve"] = {"seconds": ref["oracle_seconds"], "steps": ref["iters"], "cores": 1,
                                         "host": ref.get("host")}
        out[config] = rate
    line["cpu_baseline"]["solves"] = out


# ------------------------------------------------------------------------------------------------

def max_over_ranks(dist, value: float, device) -> float:
    """The maximum of a per-rank time over all ranks (the job takes as long as its slowest rank)."""
    if dist is None:
        return value
    import torch

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=1 << 24)
    ap.add_argument("--nvec", type=int, default=100)
    ap.add_argument("--fmt", default="frsz2")
    ap.add_argument("--bits", type=int, default=32)
    ap.add_argument("--no-extras", action="store_true", help="skip the format sweep, e2e, solve and CPU legs")
    ap.add_argument("--serving-requests", type=int, default=100, help="requests of the serving leg (0 skips it)")
    ap.add_argument("--serving-nmax", type=float, default=1e6, help="largest request n of the serving leg")
    ap.add_argument("--serving-only", action="store_true", help="only the serving leg (--serving-requests, "
                    "--serving-nmax)")
    ap.add_argument("--no-solve-baseline", action="store_true",
                    help="skip the oracle's per-step timing of the c3/c4 solves in cpu_baseline")
    ap.add_argument("--solve-c1", action="store_true", help="only the 64x64 solves to 1e-10 (on-chip and "
                    "streamed cycles)")
    ap.add_argument("--solve-c3", default="", help="comma-separated basis formats (fp64, fp32, fp16, bf16, "
                    "frsz2_16, frsz2_21, frsz2_32): run only the full 256^3 solves to 1e-10 and print them")
    ap.add_argument("--solve-c4", default="", help="as --solve-c3, on the 4M-row power-law matrix")
    ap.add_argument("--sweep", default="", choices=["", "c3", "c4"],
                    help="run only the basis-format sweep (iteration ratios, RRN histories, exponent spreads)")
    ap.add_argument("--rhs", default="ones", choices=["ones", "sin"], help="right-hand side of --sweep")
    ap.add_argument("--ref-budget", type=float, default=150.0,
                    help="seconds of host time the reference (oracle) arm's steps may take in total")
    ap.add_argument("--spmv", default="", choices=["", "c3", "c4"], help="run only the SpMV on a c3/c4 matrix")
    ap.add_argument("--spmv-size", type=int, default=256, help="--spmv c3: grid edge; c4: rows")
    ap.add_argument("--intensity", action="store_true",
                    help="run only the arithmetic-intensity sweep of the stored formats (Fig. 3 protocol)")
    ap.add_argument("--target-iters", type=int, default=0,
                    help="--sweep tolerance from this many fp64-basis iterations (the target-RRN protocol)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    workload = (f"basis kernels: {args.fmt}{'_' + str(args.bits) if args.fmt == 'frsz2' else ''} store + fused "
                f"decode-dot + decode-update over {args.nvec} x {args.n} values (N(0,1)*2^k per 32-block, "
                f"k in [-20,20], seed 1, unit-norm vectors)")

    if args.impl == "reference":
        if rank != 0:
            return
        cores = os.cpu_count() or 1
        n = choose_oracle_sample(args.nvec, args.steps + args.warmup, args.ref_budget, args.n, cores)
        gbs, dt = oracle_rate(n, args.nvec, args.steps, args.warmup, cores)
        line = {"impl": "reference", "metric": METRIC, "value": gbs, "unit": "GB/s", "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic",
                "config": step_config(args, workload, world),
                "cpu_baseline": {"value": gbs, "unit": "GB/s", "cores": cores, "kind": "oracle",
                                 "sample": f"each step over {args.nvec} x {n} values of the workload, rows split "
                                           f"over {cores} threads"},
                "e2e": {"value": gbs, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch

    import paper_2409_15468_gb300 as pkg

    pkg.load()
    dist = None
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    device = torch.device("cuda", local if world > 1 else torch.cuda.current_device())
    torch.cuda.set_device(device)
    peak, peak_src = load_peaks()
    if args.spmv:
        if rank == 0:
            print(json.dumps({"spmv": spmv_only(pkg, torch, device, args.spmv, args.spmv_size)}))
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return
    if args.intensity:
        if rank == 0:
            print(json.dumps({"intensity": intensity_sweep(pkg, torch, device, peak_gbs=peak)}))
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return
    if args.sweep:
        if rank == 0:
            print(json.dumps({"sweep": sweep(pkg, torch, device, args.sweep, args.rhs, target_iters=args.target_iters)}))
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return
    if args.serving_only:
        if rank == 0:
            print(json.dumps({"serving": serving(pkg, torch, device, args.serving_requests, 1e4, args.serving_nmax)}))
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return
    if args.solve_c1 or args.solve_c3 or args.solve_c4:
        if rank == 0:
            if args.solve_c1:
                print(json.dumps({"solve_c1": time_to_tol(pkg, torch, device)}))
            if args.solve_c3:
                print(json.dumps({"solve_c3": solve_c3(pkg, torch, device, args.solve_c3.split(","))}))
            if args.solve_c4:
                print(json.dumps({"solve_c4": solve_c3(pkg, torch, device, args.solve_c4.split(","), matrix="c4")}))
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return
    fmt, l = args.fmt, args.bits
    B, w = make_basis(pkg, torch, fmt, l, args.n, args.nvec, device)
    sb = step_bytes(fmt, l, args.n, args.nvec)
    per_step = sum(sb.values())

    # main timed region (with clocks sampled during it)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(device.index if device.index is not None else 0).start() if rank == 0 else None
    time.sleep(0.3)
    total_ms, _ = time_steps(pkg, torch, B, w, args.nvec, args.steps, args.warmup)
    total_ms = max_over_ranks(dist, total_ms, device)
    # per-kernel durations for the roofline (a separate pass, same launches)
    _, kms = time_steps(pkg, torch, B, w, args.nvec, max(20, min(args.steps, 100)), 2, per_kernel=True)
    clocks = sampler.stop() if sampler else None
    # end to end through host buffers, on every rank (max over ranks, like the device time)
    e_steps = max(20, args.steps // 5)
    e2e = None
    if not args.no_extras:
        e_ms, h2d, d2h = time_e2e(pkg, torch, B, w, args.nvec, e_steps, 3)
        e_ms = max_over_ranks(dist, e_ms, device)
        e2e = {"value": world * per_step * e_steps / (e_ms * 1e-3) / 1e9, "unit": "GB/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "steps": e_steps}
    if rank != 0:
        dist.barrier()
        dist.destroy_process_group()
        return

    value = world * per_step * args.steps / (total_ms * 1e-3) / 1e9
    dom = max(("dot", "update"), key=lambda k: kms[k])
    achieved = sb[dom] / (kms[dom] * 1e-3) / 1e9
    tag = f"{dom}_{fmt}{l if fmt == 'frsz2' else ''}"
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic_from_profiles(tag), "kernel": f"k_{dom}_{fmt}<{l}>" if fmt == "frsz2" else dom,
                "peak_source": peak_src,
                "per_kernel_ms": kms,
                "per_kernel_gbs": {k: sb[k] / (kms[k] * 1e-3) / 1e9 for k in kms}}
    line = {"metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": step_config(args, workload, world),
            "roofline": roofline, "gpu_launches": 3 * args.steps, "clocks": clocks}

    if e2e:
        line["e2e"] = e2e
    if not args.no_extras and world == 1:
        # the single-GPU legs (other formats, full solves, serving, the oracle on the host) run at N = 1
        del B, w
        torch.cuda.empty_cache()
        # the other storage formats on the same step
        fmts = {}
        for f2, l2 in (("fp64", 32), ("fp32", 32), ("fp16", 32), ("bf16", 32), ("frsz2", 16), ("frsz2", 21),
                       ("frsz2", 32)):
            B2, w2 = make_basis(pkg, torch, f2, l2, args.n, args.nvec, device)
            steps2 = max(10, min(args.steps, 50))
            ms2, k2 = time_steps(pkg, torch, B2, w2, args.nvec, steps2, 3, per_kernel=True)
            sb2 = step_bytes(f2, l2, args.n, args.nvec)
            name = f2 if f2 != "frsz2" else f"frsz2_{l2}"
            fmts[name] = {"gbs": sum(sb2.values()) * steps2 / (ms2 * 1e-3) / 1e9,
                          "ms_per_step": ms2 / steps2,
                          "frac_of_peak": sum(sb2.values()) * steps2 / (ms2 * 1e-3) / 1e9 / peak,
                          "dot_gbs": sb2["dot"] / (k2["dot"] * 1e-3) / 1e9,
                          "update_gbs": sb2["update"] / (k2["update"] * 1e-3) / 1e9}
            del B2, w2
            torch.cuda.empty_cache()
        fmts["speedup_frsz2_32_vs_fp64_per_step"] = fmts["fp64"]["ms_per_step"] / fmts["frsz2_32"]["ms_per_step"]
        line["formats"] = fmts
        line["time_to_tol"] = time_to_tol(pkg, torch, device)
        line["time_to_tol_c3"] = solve_c3(pkg, torch, device, ["frsz2_32", "fp64"])
        line["time_to_tol_c4"] = solve_c3(pkg, torch, device, ["frsz2_32", "fp32", "fp64"], matrix="c4")
        if args.serving_requests > 0:
            line["serving"] = serving(pkg, torch, device, args.serving_requests, 1e4, args.serving_nmax)
        line["cpu_baseline"] = cpu_baseline(args.n, args.nvec)
        if not args.no_solve_baseline:
            add_oracle_solve_rates(line)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    print(json.dumps(line))


if __name__ == "__main__":
    main()
