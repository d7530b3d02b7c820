"""Plain FP64 CPU oracle for CB-GMRES with the FRSZ2 compressor (arXiv 2409.15468).

TEST INFRASTRUCTURE ONLY. This package wraps ``oracle.c``, the slow and obviously correct
reference that the CUDA path is checked against. Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it. It shares no
code with the CUDA library (``paper_2409_15468_gb300``), and the CUDA library never imports it.

Parity unpinned: full-solve behaviour of the compressed bases against the paper's residual
curves (Figs. 4-8), since the paper's figures and matrices are not available. Every other
function here is pinned by ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")

FP64, FP32, FP16, BF16, FRSZ2 = 0, 1, 2, 3, 4
FORMAT_NAMES = {"fp64": FP64, "fp32": FP32, "fp16": FP16, "bf16": BF16, "frsz2": FRSZ2}
BS = 32


def build(force: bool = False) -> str:
    """Compile oracle.c into a shared library next to it (plain gcc, portable flags)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "oracle.h"))
    ):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


class _Opts(ctypes.Structure):
    _fields_ = [("restart", ctypes.c_int32), ("fmt", ctypes.c_int32), ("frsz2_bits", ctypes.c_int32),
                ("precond", ctypes.c_int32), ("tol", ctypes.c_double), ("max_iters", ctypes.c_int64),
                ("eta", ctypes.c_double)]


class _Result(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int64), ("restarts", ctypes.c_int64), ("reorths", ctypes.c_int64),
                ("converged", ctypes.c_int32), ("breakdowns", ctypes.c_int32), ("true_rrn", ctypes.c_double),
                ("implicit_rrn", ctypes.c_double), ("stagnated", ctypes.c_int32)]


def lib():
    global _lib
    if _lib is None:
        # ORACLE_LIB_OVERRIDE lets the mutation tests load a deliberately broken copy of this oracle.
        path = os.environ.get("ORACLE_LIB_OVERRIDE") or build()
        L = ctypes.CDLL(path)
        P = ctypes.c_void_p
        i64, i32 = ctypes.c_int64, ctypes.c_int32
        sig = {
            "orc_frsz2_nblocks": (i64, [i64]),
            "orc_frsz2_code_words": (i64, [i64, i32]),
            "orc_frsz2_bytes": (i64, [i64, i32]),
            "orc_frsz2_compress": (ctypes.c_int, [P, i64, i32, P, P]),
            "orc_frsz2_decompress": (ctypes.c_int, [P, P, i64, i32, P]),
            "orc_frsz2_decode_one": (ctypes.c_double, [P, P, i64, i32]),
            "orc_frsz2_get_code": (ctypes.c_uint32, [P, i64, i32]),
            "orc_cast_round": (ctypes.c_double, [ctypes.c_double, i32]),
            "orc_cast_encode": (ctypes.c_int, [P, i64, i32, P]),
            "orc_cast_decode": (ctypes.c_int, [P, i64, i32, P]),
            "orc_encode": (ctypes.c_int, [P, i64, i32, i32, P, P]),
            "orc_decode": (ctypes.c_int, [P, P, i64, i32, i32, P]),
            "orc_dot": (ctypes.c_double, [P, P, i64]),
            "orc_dot2": (ctypes.c_double, [P, P, i64]),
            "orc_nrm2": (ctypes.c_double, [P, i64]),
            "orc_axpy": (None, [ctypes.c_double, P, P, i64]),
            "orc_spmv_csr": (None, [i32, P, P, P, P, P]),
            "orc_gmres": (ctypes.c_int, [i32, P, P, P, P, P, ctypes.POINTER(_Opts), ctypes.POINTER(_Result), P, P]),
            "orc_arnoldi_cycle": (ctypes.c_int, [i32, P, P, P, P, P, ctypes.POINTER(_Opts), P, P, P,
                                                 ctypes.POINTER(ctypes.c_double)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(x) -> np.ndarray:
    return np.ascontiguousarray(x, dtype=np.float64)


# ---------------------------------------------------------------------------------------------
# FRSZ2 codec
# ---------------------------------------------------------------------------------------------

def frsz2_nblocks(n: int) -> int:
    return int(lib().orc_frsz2_nblocks(n))


def frsz2_code_words(n: int, l: int) -> int:
    return int(lib().orc_frsz2_code_words(n, l))


def frsz2_bytes(n: int, l: int) -> int:
    """Eq. 3 (code words per block read as ceil(32*l/32)) plus one exponent word per block."""
    return int(lib().orc_frsz2_bytes(n, l))


def frsz2_compress(x, l: int):
    x = _f64(x)
    n = x.size
    exps = np.zeros(frsz2_nblocks(n), dtype=np.uint32)
    codes = np.zeros(frsz2_code_words(n, l), dtype=np.uint32)
    if lib().orc_frsz2_compress(_p(x), n, l, _p(exps), _p(codes)) != 0:
        raise ValueError("bad FRSZ2 arguments")
    return exps, codes


def frsz2_decompress(exps, codes, n: int, l: int) -> np.ndarray:
    exps = np.ascontiguousarray(exps, dtype=np.uint32)
    codes = np.ascontiguousarray(codes, dtype=np.uint32)
    out = np.empty(n, dtype=np.float64)
    if lib().orc_frsz2_decompress(_p(exps), _p(codes), n, l, _p(out)) != 0:
        raise ValueError("bad FRSZ2 arguments")
    return out


def frsz2_decode_one(exps, codes, i: int, l: int) -> float:
    exps = np.ascontiguousarray(exps, dtype=np.uint32)
    codes = np.ascontiguousarray(codes, dtype=np.uint32)
    return float(lib().orc_frsz2_decode_one(_p(exps), _p(codes), i, l))


def frsz2_get_code(codes, i: int, l: int) -> int:
    codes = np.ascontiguousarray(codes, dtype=np.uint32)
    return int(lib().orc_frsz2_get_code(_p(codes), i, l))


# ---------------------------------------------------------------------------------------------
# Cast formats and the generic encoded vector
# ---------------------------------------------------------------------------------------------

_BITS_DTYPE = {FP64: np.uint64, FP32: np.uint32, FP16: np.uint16, BF16: np.uint16}


def cast_round(x: float, fmt: int) -> float:
    return float(lib().orc_cast_round(float(x), fmt))


def cast_encode(x, fmt: int) -> np.ndarray:
    x = _f64(x)
    bits = np.zeros(x.size, dtype=_BITS_DTYPE[fmt])
    if lib().orc_cast_encode(_p(x), x.size, fmt, _p(bits)) != 0:
        raise ValueError("bad format")
    return bits


def cast_decode(bits, fmt: int) -> np.ndarray:
    bits = np.ascontiguousarray(bits, dtype=_BITS_DTYPE[fmt])
    out = np.empty(bits.size, dtype=np.float64)
    if lib().orc_cast_decode(_p(bits), bits.size, fmt, _p(out)) != 0:
        raise ValueError("bad format")
    return out


def encode(x, fmt: int, l: int = 32):
    """Returns (vals, exps): the stored arrays of one basis vector (exps is None for casts)."""
    if fmt == FRSZ2:
        exps, codes = frsz2_compress(x, l)
        return codes, exps
    return cast_encode(x, fmt), None


def decode(vals, exps, n: int, fmt: int, l: int = 32) -> np.ndarray:
    if fmt == FRSZ2:
        return frsz2_decompress(exps, vals, n, l)
    return cast_decode(vals, fmt)[:n]


# ---------------------------------------------------------------------------------------------
# FP64 building blocks
# ---------------------------------------------------------------------------------------------

def dot(a, b) -> float:
    a, b = _f64(a), _f64(b)
    return float(lib().orc_dot(_p(a), _p(b), a.size))


def dot2(a, b) -> float:
    a, b = _f64(a), _f64(b)
    return float(lib().orc_dot2(_p(a), _p(b), a.size))


def nrm2(a) -> float:
    a = _f64(a)
    return float(lib().orc_nrm2(_p(a), a.size))


def axpy(alpha: float, x, y: np.ndarray) -> np.ndarray:
    """y += alpha x in place (sequential FP64)."""
    x = _f64(x)
    assert y.dtype == np.float64 and y.flags.c_contiguous and y.size == x.size
    lib().orc_axpy(float(alpha), _p(x), _p(y), x.size)
    return y


def spmv(row_ptr, col, vals, x) -> np.ndarray:
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    vals, x = _f64(vals), _f64(x)
    n = row_ptr.size - 1
    y = np.empty(n, dtype=np.float64)
    lib().orc_spmv_csr(n, _p(row_ptr), _p(col), _p(vals), _p(x), _p(y))
    return y


def basis_dot(Vhat: np.ndarray, w) -> np.ndarray:
    """h_i = sum_k Vhat[i, k] w_k with the compensated dot (the decoded basis times w)."""
    w = _f64(w)
    return np.array([dot2(Vhat[i], w) for i in range(Vhat.shape[0])])


def basis_update(Vhat: np.ndarray, h, w) -> np.ndarray:
    """w_k - sum_i Vhat[i, k] h_i for every k, each element as one compensated dot of length
    nvec + 1 (the update of Fig. 1 step 5 for a given h)."""
    Vhat = np.ascontiguousarray(Vhat, dtype=np.float64)
    h = _f64(h)
    w = _f64(w)
    nvec, n = Vhat.shape
    out = np.empty(n)
    coef = np.concatenate([[1.0], -h])
    for k in range(n):
        out[k] = dot2(np.concatenate([[w[k]], Vhat[:, k]]), coef)
    return out


# ---------------------------------------------------------------------------------------------
# GMRES
# ---------------------------------------------------------------------------------------------

@dataclass
class GmresResult:
    x: np.ndarray
    iters: int
    restarts: int
    reorths: int
    converged: bool
    breakdowns: int
    true_rrn: float
    implicit_rrn: float
    hist_implicit: np.ndarray
    hist_true: np.ndarray
    stagnated: bool


PRECOND = {"none": 0, "jacobi": 1}


def _opts(restart, tol, max_iters, fmt, l, eta, precond="none"):
    return _Opts(restart=restart, fmt=fmt, frsz2_bits=l, precond=PRECOND[precond], tol=tol, max_iters=max_iters,
                 eta=eta)


DEFAULT_ETA = 1.0 / np.sqrt(2.0)


def gmres(row_ptr, col, vals, b, x0=None, *, restart=50, tol=1e-10, max_iters=20000, fmt=FP64, l=32,
          eta=DEFAULT_ETA, precond="none") -> GmresResult:
    """Restarted (CB-)GMRES of Fig. 1 with the basis stored in `fmt`; precond "jacobi" applies
    M = diag(A) on the right (steps 3 and 17), "none" is M = I."""
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    vals, b = _f64(vals), _f64(b)
    n = row_ptr.size - 1
    x = np.zeros(n) if x0 is None else _f64(x0).copy()
    o = _opts(restart, tol, max_iters, fmt, l, eta, precond)
    r = _Result()
    hi = np.zeros(max(max_iters, 1))
    ht = np.zeros(max_iters + 2)
    st = lib().orc_gmres(n, _p(row_ptr), _p(col), _p(vals), _p(b), _p(x), ctypes.byref(o), ctypes.byref(r),
                         _p(hi), _p(ht))
    if st != 0:
        raise ValueError(f"oracle gmres failed with status {st}")
    return GmresResult(x=x, iters=r.iters, restarts=r.restarts, reorths=r.reorths, converged=bool(r.converged),
                       breakdowns=r.breakdowns, true_rrn=r.true_rrn, implicit_rrn=r.implicit_rrn,
                       hist_implicit=hi[:r.iters].copy(), hist_true=ht[:r.restarts + 1].copy(),
                       stagnated=bool(r.stagnated))


def arnoldi_cycle(row_ptr, col, vals, b, x0=None, *, restart=50, tol=1e-300, fmt=FP64, l=32, eta=DEFAULT_ETA):
    """One cycle: returns (m_eff, V, Vhat, H, beta), V/Vhat of shape (m_eff+1, n) (the last row is
    only meaningful when the cycle did not end early) and H of shape (m+1, m)."""
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    vals, b = _f64(vals), _f64(b)
    n = row_ptr.size - 1
    x0 = np.zeros(n) if x0 is None else _f64(x0)
    m = restart
    V = np.zeros((m + 1, n))
    Vh = np.zeros((m + 1, n))
    H = np.zeros((m, m + 1))  # column-major (m+1) x m, stored transposed
    beta = ctypes.c_double(0.0)
    o = _opts(restart, tol, 1 << 40, fmt, l, eta)
    m_eff = lib().orc_arnoldi_cycle(n, _p(row_ptr), _p(col), _p(vals), _p(b), _p(x0), ctypes.byref(o), _p(V),
                                    _p(Vh), _p(H), ctypes.byref(beta))
    return m_eff, V, Vh, H.T.copy(), beta.value
