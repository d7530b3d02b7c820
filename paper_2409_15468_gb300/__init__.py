"""GB300-native Compressed-Basis GMRES with the FRSZ2 block compressor (arXiv 2409.15468).

A thin ctypes binding of ``libcbgmres.so`` (C ABI in ``include/cbgmres.h``). PyTorch is used only
to allocate device memory and to name the current CUDA stream; every step of the solver and of
the basis kernels runs in the library's CUDA kernels. There is no CPU fallback: without the built
library or a CUDA device every call raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

from . import build as _build

FP64, FP32, FP16, BF16, FRSZ2 = 0, 1, 2, 3, 4
FORMATS = {"fp64": FP64, "fp32": FP32, "fp16": FP16, "bf16": BF16, "frsz2": FRSZ2}
PRECOND = {"none": 0, "jacobi": 1}
CYCLE = {"auto": 0, "streamed": 1}
STATUS = {0: "CBG_OK", -1: "CBG_ERR_INVALID_ARG", -2: "CBG_ERR_CUDA", -3: "CBG_ERR_OOM", -4: "CBG_ERR_NONFINITE",
          -5: "CBG_ERR_NOT_CONVERGED", -6: "CBG_ERR_TIMEOUT", -7: "CBG_ERR_BAD_MATRIX", -8: "CBG_ERR_STATE",
          -9: "CBG_ERR_BREAKDOWN_NOT_CONVERGED", -10: "CBG_ERR_UNIMPLEMENTED"}
ERR_NOT_CONVERGED = -5
ERR_BREAKDOWN_NOT_CONVERGED = -9
# statuses with which a solve still writes x and its result
SOLVE_ENDED = (0, ERR_NOT_CONVERGED, ERR_BREAKDOWN_NOT_CONVERGED)

# Symbols declared in include/cbgmres.h (checked by the CPU tests).
EXPORTS = ["cbg_frsz2_bytes", "cbg_frsz2_compress", "cbg_frsz2_decompress", "cbg_basis_layout", "cbg_basis_store",
           "cbg_basis_append",
           "cbg_basis_load", "cbg_basis_work_bytes", "cbg_basis_dot", "cbg_basis_dot_noalloc", "cbg_basis_update", "cbg_intensity",
           "cbg_csr_validate",
           "cbg_spmv_work_bytes", "cbg_spmv", "cbg_opts_default", "cbgmres_workspace_bytes", "cbgmres_create",
           "cbgmres_solve", "cbgmres_start", "cbgmres_advance", "cbgmres_finish", "cbgmres_history",
           "cbgmres_destroy", "cbgmres_basis_vector", "cbgmres_cycle_cluster", "cbg_server_create", "cbg_server_submit", "cbg_server_poll", "cbg_server_stats",
           "cbg_server_clock", "cbg_server_destroy", "cbg_last_error", "cbg_version", "cbgmres_last_error",
           "frsz2_bytes", "frsz2_compress", "frsz2_decompress"]


class CbgError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class Opts(ctypes.Structure):
    _fields_ = [("restart", ctypes.c_int32), ("fmt", ctypes.c_int32), ("frsz2_bits", ctypes.c_int32),
                ("history", ctypes.c_int32), ("tol", ctypes.c_double), ("max_iters", ctypes.c_int64),
                ("eta", ctypes.c_double), ("precond", ctypes.c_int32), ("cycle", ctypes.c_int32)]


class Result(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int64), ("restarts", ctypes.c_int64), ("reorths", ctypes.c_int64),
                ("converged", ctypes.c_int32), ("status", ctypes.c_int32), ("true_rrn", ctypes.c_double),
                ("implicit_rrn", ctypes.c_double), ("seconds", ctypes.c_double), ("breakdowns", ctypes.c_int64)]


class Request(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_uint64), ("n", ctypes.c_int32), ("nnz", ctypes.c_int64),
                ("d_row_ptr", ctypes.c_void_p), ("d_col", ctypes.c_void_p), ("d_vals", ctypes.c_void_p),
                ("d_b", ctypes.c_void_p), ("d_x", ctypes.c_void_p), ("opts", Opts)]


class Completion(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_uint64), ("status", ctypes.c_int32), ("result", Result),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double)]


class Basis(ctypes.Structure):
    _fields_ = [("fmt", ctypes.c_int32), ("frsz2_bits", ctypes.c_int32), ("n", ctypes.c_int64),
                ("vals", ctypes.c_void_p), ("vals_stride", ctypes.c_int64), ("exps", ctypes.c_void_p),
                ("exps_stride", ctypes.c_int64)]


_lib = None


def library_path() -> str:
    return _build.LIB


def build(force: bool = False) -> str:
    return _build.build(force=force)


def load(path: str | None = None):
    """Loads libcbgmres.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2409_15468_gb300.build() (nvcc, sm_103a)")
    L = ctypes.CDLL(path)
    P, i32, i64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
    c_int = ctypes.c_int
    sig = {
        "cbg_frsz2_bytes": (i64, [i64, i32]),
        "cbg_frsz2_compress": (c_int, [P, i64, i32, P, P, P]),
        "cbg_frsz2_decompress": (c_int, [P, P, i64, i32, P, P]),
        "cbg_basis_layout": (c_int, [i64, i32, i32, ctypes.POINTER(i64), ctypes.POINTER(i64)]),
        "cbg_basis_store": (c_int, [ctypes.POINTER(Basis), i32, P, P]),
        "cbg_basis_append": (c_int, [ctypes.POINTER(Basis), i32, P, P, P, P]),
        "cbg_basis_load": (c_int, [ctypes.POINTER(Basis), i32, P, P]),
        "cbg_basis_work_bytes": (sz, [i64, i32]),
        "cbg_basis_dot": (c_int, [ctypes.POINTER(Basis), i32, P, P, P, sz, P]),
        "cbg_basis_dot_noalloc": (c_int, [ctypes.POINTER(Basis), i32, P, P, P]),
        "cbg_basis_update": (c_int, [ctypes.POINTER(Basis), i32, P, P, P, P, sz, P]),
        "cbg_intensity": (c_int, [ctypes.POINTER(Basis), i32, i32, i32, P, P, sz, P]),
        "cbg_csr_validate": (c_int, [i32, i64, P, P, P]),
        "cbg_spmv_work_bytes": (sz, [i32]),
        "cbg_spmv": (c_int, [i32, i64, P, P, P, P, P, P, P, sz, P]),
        "cbg_opts_default": (c_int, [ctypes.POINTER(Opts)]),
        "cbgmres_workspace_bytes": (sz, [i32, ctypes.POINTER(Opts)]),
        "cbgmres_create": (c_int, [ctypes.POINTER(P), i32, i64, P, P, P, ctypes.POINTER(Opts), P]),
        "cbgmres_solve": (c_int, [P, P, P, ctypes.POINTER(Result)]),
        "cbgmres_start": (c_int, [P, P, P]),
        "cbgmres_advance": (c_int, [P, i32, ctypes.POINTER(i32)]),
        "cbgmres_finish": (c_int, [P, ctypes.POINTER(Result)]),
        "cbgmres_history": (c_int, [P, P, i64, ctypes.POINTER(i64)]),
        "cbgmres_destroy": (c_int, [P]),
        "cbgmres_basis_vector": (c_int, [P, i32, P]),
        "cbgmres_cycle_cluster": (i32, [P]),
        "cbg_server_create": (c_int, [ctypes.POINTER(P), sz, i32, i32, i32]),
        "cbg_server_submit": (c_int, [P, ctypes.POINTER(Request)]),
        "cbg_server_poll": (c_int, [P, ctypes.POINTER(Completion), i32, ctypes.POINTER(i32)]),
        "cbg_server_stats": (c_int, [P, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32),
                                     ctypes.POINTER(sz)]),
        "cbg_server_clock": (ctypes.c_double, [P]),
        "cbg_server_destroy": (c_int, [P]),
        "cbg_last_error": (ctypes.c_char_p, []),
        "cbgmres_last_error": (ctypes.c_char_p, []),
        "cbg_version": (ctypes.c_char_p, []),
        "frsz2_bytes": (sz, [i64, i32]),
        "frsz2_compress": (c_int, [P, i64, i32, P, P, P]),
        "frsz2_decompress": (c_int, [P, P, i64, i32, P, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def lib():
    return load()


def last_error() -> str:
    return lib().cbg_last_error().decode()


def check(status: int, allow=(0,)) -> int:
    if status not in allow:
        raise CbgError(status, last_error())
    return status


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t: torch.Tensor | None):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _empty(nbytes: int, device=None) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device or "cuda")


# ---------------------------------------------------------------------------------------------
# FRSZ2 codec
# ---------------------------------------------------------------------------------------------

def frsz2_bytes(n: int, l: int) -> int:
    return int(lib().cbg_frsz2_bytes(n, l))


def frsz2_compress(x: torch.Tensor, l: int, exps: torch.Tensor | None = None, codes: torch.Tensor | None = None,
                   stream=None):
    """Compresses a float64 CUDA vector; returns (exps uint32[ceil(n/32)], codes uint32[ceil(n/32)*l])."""
    n = x.numel()
    nb = (n + 31) // 32
    if exps is None:
        exps = torch.empty(max(nb, 1), dtype=torch.int32, device=x.device)
    if codes is None:
        codes = torch.empty(max(nb * l, 1), dtype=torch.int32, device=x.device)
    check(lib().cbg_frsz2_compress(_ptr(x), n, l, _ptr(exps), _ptr(codes), _stream(stream)))
    return exps, codes


def frsz2_decompress(exps: torch.Tensor, codes: torch.Tensor, n: int, l: int, out: torch.Tensor | None = None,
                     stream=None) -> torch.Tensor:
    if out is None:
        out = torch.empty(max(n, 1), dtype=torch.float64, device=exps.device)
    check(lib().cbg_frsz2_decompress(_ptr(exps), _ptr(codes), n, l, _ptr(out), _stream(stream)))
    return out[:n]


# ---------------------------------------------------------------------------------------------
# Basis storage and the fused basis kernels
# ---------------------------------------------------------------------------------------------

def basis_layout(n: int, fmt: int, l: int = 32):
    vs, es = ctypes.c_int64(0), ctypes.c_int64(0)
    check(lib().cbg_basis_layout(n, fmt, l, ctypes.byref(vs), ctypes.byref(es)))
    return vs.value, es.value


class BasisStorage:
    """Device storage for nvec basis vectors of n values in one format (memory from torch)."""

    def __init__(self, n: int, nvec: int, fmt: int, l: int = 32, device=None):
        self.n, self.nvec, self.fmt, self.l = n, nvec, fmt, (l if fmt == FRSZ2 else 32)
        vs, es = basis_layout(n, fmt, self.l)
        self.vals = _empty(vs * nvec + 256, device)
        self.exps = _empty(es * nvec + 256, device) if fmt == FRSZ2 else None
        if self.vals.data_ptr() % 256 or (self.exps is not None and self.exps.data_ptr() % 256):
            raise RuntimeError("allocator returned a buffer that is not 256-byte aligned")
        self.vals_stride, self.exps_stride = vs, es
        self.struct = Basis(fmt=fmt, frsz2_bits=self.l, n=n, vals=self.vals.data_ptr(), vals_stride=vs,
                            exps=self.exps.data_ptr() if self.exps is not None else None, exps_stride=es)

    def store(self, slot: int, x: torch.Tensor, stream=None):
        check(lib().cbg_basis_store(ctypes.byref(self.struct), slot, _ptr(x), _stream(stream)))

    def append(self, slot: int, w: torch.Tensor, h: torch.Tensor, v: torch.Tensor | None = None, stream=None):
        """v := w / h (h: one positive float64 on the device) stored as vector `slot`; v, when given,
        receives the FP64 quotient (cbg_basis_append)."""
        check(lib().cbg_basis_append(ctypes.byref(self.struct), slot, _ptr(w), _ptr(h), _ptr(v), _stream(stream)))
        return v

    def load(self, slot: int, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        if out is None:
            out = torch.empty(max(self.n, 1), dtype=torch.float64, device=self.vals.device)
        check(lib().cbg_basis_load(ctypes.byref(self.struct), slot, _ptr(out), _stream(stream)))
        return out[: self.n]

    def vector_bytes(self, slot: int):
        """The stored (vals, exps) byte tensors of one vector (views, for parity checks)."""
        v = self.vals[slot * self.vals_stride:(slot + 1) * self.vals_stride]
        e = self.exps[slot * self.exps_stride:(slot + 1) * self.exps_stride] if self.exps is not None else None
        return v, e

    def work(self, nvec: int) -> torch.Tensor:
        return _empty(lib().cbg_basis_work_bytes(self.n, nvec), self.vals.device)

    def dot(self, nvec: int, w: torch.Tensor, out: torch.Tensor | None = None, work: torch.Tensor | None = None,
            stream=None) -> torch.Tensor:
        if out is None:
            out = torch.empty(max(nvec, 1), dtype=torch.float64, device=w.device)
        work = work if work is not None else self.work(nvec)
        check(lib().cbg_basis_dot(ctypes.byref(self.struct), nvec, _ptr(w), _ptr(out), _ptr(work), work.numel(),
                                  _stream(stream)))
        return out[:nvec]

    def update(self, nvec: int, h: torch.Tensor, w: torch.Tensor, norm2: torch.Tensor | None = None,
               work: torch.Tensor | None = None, stream=None):
        work = work if work is not None else self.work(nvec)
        check(lib().cbg_basis_update(ctypes.byref(self.struct), nvec, _ptr(h), _ptr(w), _ptr(norm2), _ptr(work),
                                     work.numel(), _stream(stream)))
        return w


    def intensity(self, slot: int, fma_per_value: int, fp32_compute: bool = False, out: torch.Tensor | None = None,
                  work: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """sum_k f^r(x_k) over stored vector `slot`, f(y) = 0.5 y + 0.25 (cbg_intensity)."""
        if out is None:
            out = torch.empty(1, dtype=torch.float64, device=self.vals.device)
        work = work if work is not None else self.work(1)
        check(lib().cbg_intensity(ctypes.byref(self.struct), slot, fma_per_value, int(fp32_compute), _ptr(out),
                                  _ptr(work), work.numel(), _stream(stream)))
        return out


# ---------------------------------------------------------------------------------------------
# Sparse matrix
# ---------------------------------------------------------------------------------------------

def csr_validate(row_ptr: torch.Tensor, col: torch.Tensor, stream=None) -> int:
    n = row_ptr.numel() - 1
    return lib().cbg_csr_validate(n, col.numel(), _ptr(row_ptr), _ptr(col), _stream(stream))


def spmv(row_ptr: torch.Tensor, col: torch.Tensor, vals: torch.Tensor, x: torch.Tensor,
         y: torch.Tensor | None = None, norm2: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    n = row_ptr.numel() - 1
    if y is None:
        y = torch.empty(max(n, 1), dtype=torch.float64, device=x.device)
    work = _empty(lib().cbg_spmv_work_bytes(n), x.device)
    check(lib().cbg_spmv(n, col.numel(), _ptr(row_ptr), _ptr(col), _ptr(vals), _ptr(x), _ptr(y), _ptr(norm2), _ptr(work),
                         work.numel(), _stream(stream)))
    return y[:n]


# ---------------------------------------------------------------------------------------------
# Solver
# ---------------------------------------------------------------------------------------------

def default_opts(**kw) -> Opts:
    o = Opts()
    check(lib().cbg_opts_default(ctypes.byref(o)))
    for k, v in kw.items():
        if k == "fmt" and isinstance(v, str):
            v = FORMATS[v]
        if k == "precond" and isinstance(v, str):
            v = PRECOND[v]
        if k == "cycle" and isinstance(v, str):
            v = CYCLE[v]
        setattr(o, k, v)
    return o


def workspace_bytes(n: int, opts: Opts) -> int:
    return int(lib().cbgmres_workspace_bytes(n, ctypes.byref(opts)))


@dataclass
class SolveResult:
    iters: int
    restarts: int
    reorths: int
    converged: bool
    status: int
    true_rrn: float
    implicit_rrn: float
    seconds: float
    breakdowns: int


def _result(r: Result) -> SolveResult:
    return SolveResult(r.iters, r.restarts, r.reorths, bool(r.converged), r.status, r.true_rrn, r.implicit_rrn,
                       r.seconds, r.breakdowns)


class Solver:
    """A CB-GMRES context for one CSR matrix (the matrix tensors must outlive the solver)."""

    def __init__(self, row_ptr: torch.Tensor, col: torch.Tensor, vals: torch.Tensor, opts: Opts | None = None,
                 stream: torch.cuda.Stream | None = None, **kw):
        self.opts = opts if opts is not None else default_opts(**kw)
        self.n = row_ptr.numel() - 1
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._keep = (row_ptr, col, vals)
        h = ctypes.c_void_p(None)
        check(lib().cbgmres_create(ctypes.byref(h), self.n, col.numel(), _ptr(row_ptr), _ptr(col), _ptr(vals),
                                   ctypes.byref(self.opts), ctypes.c_void_p(self.stream.cuda_stream)))
        self.handle = h

    def solve(self, b: torch.Tensor, x: torch.Tensor) -> SolveResult:
        r = Result()
        check(lib().cbgmres_solve(self.handle, _ptr(b), _ptr(x), ctypes.byref(r)), allow=SOLVE_ENDED)
        return _result(r)

    def start(self, b: torch.Tensor, x: torch.Tensor):
        self._bx = (b, x)
        check(lib().cbgmres_start(self.handle, _ptr(b), _ptr(x)))

    def advance(self, max_steps: int) -> bool:
        done = ctypes.c_int32(0)
        check(lib().cbgmres_advance(self.handle, max_steps, ctypes.byref(done)), allow=SOLVE_ENDED)
        return bool(done.value)

    def finish(self) -> SolveResult:
        r = Result()
        check(lib().cbgmres_finish(self.handle, ctypes.byref(r)), allow=SOLVE_ENDED)
        return _result(r)

    def history(self, cap: int | None = None):
        import numpy as np

        cap = cap or int(self.opts.max_iters)
        buf = np.zeros(max(cap, 1))
        cnt = ctypes.c_int64(0)
        check(lib().cbgmres_history(self.handle, ctypes.c_void_p(buf.ctypes.data), cap, ctypes.byref(cnt)))
        return buf[: cnt.value]

    @property
    def cycle_cluster(self) -> int:
        """CTAs of the cluster that runs each restart cycle on chip, or 0 (streamed cycles)."""
        return int(lib().cbgmres_cycle_cluster(self.handle))

    def basis_vector(self, slot: int, out: torch.Tensor | None = None) -> torch.Tensor:
        """Basis vector `slot` of the context's current Krylov basis, decoded (ordered on the
        solver's stream; the returned tensor is ready once that stream has run)."""
        if out is None:
            out = torch.empty(max(self.n, 1), dtype=torch.float64, device="cuda")
        check(lib().cbgmres_basis_vector(self.handle, slot, _ptr(out)))
        return out[: self.n]

    def close(self):
        if getattr(self, "handle", None):
            lib().cbgmres_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------------------------
# Serving runtime
# ---------------------------------------------------------------------------------------------

@dataclass
class ServedSolve:
    tag: int
    status: int
    result: SolveResult
    t_submit: float
    t_admit: float
    t_done: float

    @property
    def latency(self) -> float:
        return self.t_done - self.t_submit


class Server:
    """The library's serving runtime (cbg_server_*): continuous batching of solves within an HBM
    budget. Tensors of a request are kept referenced here until its completion is returned."""

    def __init__(self, hbm_budget: int, max_active: int = 16, steps_per_turn: int = 8, max_bypass: int = 8):
        h = ctypes.c_void_p(None)
        check(lib().cbg_server_create(ctypes.byref(h), int(hbm_budget), max_active, steps_per_turn, max_bypass))
        self.handle = h
        self._inflight = {}
        self._buf = (Completion * 64)()

    def clock(self) -> float:
        return float(lib().cbg_server_clock(self.handle))

    def submit(self, tag: int, row_ptr: torch.Tensor, col: torch.Tensor, vals: torch.Tensor, b: torch.Tensor,
               x: torch.Tensor, opts: Opts):
        r = Request(tag=tag, n=row_ptr.numel() - 1, nnz=col.numel(), d_row_ptr=_ptr(row_ptr).value,
                    d_col=_ptr(col).value, d_vals=_ptr(vals).value, d_b=_ptr(b).value, d_x=_ptr(x).value, opts=opts)
        check(lib().cbg_server_submit(self.handle, ctypes.byref(r)))
        self._inflight[tag] = (row_ptr, col, vals, b, x)

    def poll(self) -> list[ServedSolve]:
        out = []
        while True:
            k = ctypes.c_int32(0)
            check(lib().cbg_server_poll(self.handle, self._buf, len(self._buf), ctypes.byref(k)))
            for i in range(k.value):
                c = self._buf[i]
                self._inflight.pop(c.tag, None)
                out.append(ServedSolve(c.tag, c.status, _result(c.result), c.t_submit, c.t_admit, c.t_done))
            if k.value < len(self._buf):
                return out

    def stats(self):
        a, q, p, u = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_size_t(0)
        check(lib().cbg_server_stats(self.handle, ctypes.byref(a), ctypes.byref(q), ctypes.byref(p), ctypes.byref(u)))
        return {"active": a.value, "queued": q.value, "pending": p.value, "bytes_in_use": u.value}

    def close(self):
        if getattr(self, "handle", None):
            lib().cbg_server_destroy(self.handle)
            self.handle = None
            self._inflight.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
