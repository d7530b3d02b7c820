"""The C-ABI library on a host without a GPU: it builds for sm_103a, loads, exports every function
include/cbgmres.h declares, answers the pure host calls (Eq. 3 sizes, layouts, option defaults),
rejects invalid arguments before touching a device, and has no CPU fallback: compute calls fail
with CBG_ERR_CUDA when no CUDA device is present."""
import ctypes
import os
import re

import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pkg():
    import paper_2409_15468_gb300 as p

    p.build()
    p.load()
    return p


def declared_functions():
    src = open(os.path.join(ROOT, "include", "cbgmres.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b([a-z_][a-z0-9_]*)\s*\([^;{]*\)\s*;", src)
    return sorted(set(n for n in names if n.startswith(("cbg", "frsz2_"))))


def test_exports_every_declared_symbol(pkg):
    names = declared_functions()
    assert len(names) >= 20
    assert set(names) == set(pkg.EXPORTS)
    L = ctypes.CDLL(pkg.library_path())
    for n in names:
        assert hasattr(L, n), n


def test_host_calls(pkg):
    L = pkg.lib()
    assert L.cbg_frsz2_bytes(32, 32) == 132
    assert L.cbg_frsz2_bytes(33, 21) == 2 * (21 * 4 + 4)
    assert L.cbg_frsz2_bytes(10, 17) == -1
    vs, es = pkg.basis_layout(1000, pkg.FRSZ2, 32)
    assert vs % 256 == 0 and es % 256 == 0 and vs >= 32 * 32 * 4 and es >= 32 * 4
    vs, es = pkg.basis_layout(1000, pkg.FP16)
    assert vs >= 1024 * 2 and es == 0
    o = pkg.default_opts()
    assert o.restart == 100 and o.fmt == pkg.FRSZ2 and o.frsz2_bits == 32 and o.tol == 1e-10
    assert abs(o.eta - 2 ** -0.5) < 1e-15
    assert pkg.workspace_bytes(1000, o) > 101 * vs
    assert b"sm_103a" in L.cbg_version()


def test_invalid_arguments_rejected(pkg):
    L = pkg.lib()
    h = ctypes.c_void_p()
    bad = pkg.default_opts(restart=0)
    st = L.cbgmres_create(ctypes.byref(h), 100, 0, None, None, None, ctypes.byref(bad), None)
    assert st == -1 and "invalid" in pkg.last_error()
    bad = pkg.default_opts(frsz2_bits=17)
    assert L.cbgmres_create(ctypes.byref(h), 100, 0, None, None, None, ctypes.byref(bad), None) == -10
    bad = pkg.default_opts(frsz2_bits=40)
    assert L.cbgmres_create(ctypes.byref(h), 100, 0, None, None, None, ctypes.byref(bad), None) == -1
    bad = pkg.default_opts(restart=200)
    assert L.cbgmres_create(ctypes.byref(h), 100, 0, None, None, None, ctypes.byref(bad), None) == -1
    assert L.cbg_frsz2_compress(None, 10, 21, None, None, None) == -1
    # a code width the format admits but this library does not implement, and one it does not admit
    assert L.cbg_frsz2_compress(None, 10, 20, None, None, None) == -10
    assert "not implemented" in pkg.last_error()
    assert L.cbg_frsz2_decompress(None, None, 10, 33, None, None) == -1
    assert L.cbg_frsz2_decompress(None, None, 10, 1, None, None) == -1
    b = pkg.Basis(fmt=7, frsz2_bits=32, n=10, vals=None, vals_stride=0, exps=None, exps_stride=0)
    assert L.cbg_basis_dot(ctypes.byref(b), 1, None, None, None, 0, None) == -1
    b = pkg.Basis(fmt=pkg.FRSZ2, frsz2_bits=32, n=1000, vals=256 * 3, vals_stride=100, exps=256, exps_stride=512)
    assert L.cbg_basis_dot(ctypes.byref(b), 1, None, None, None, 0, None) == -1  # stride too small
    assert L.cbgmres_advance(None, 1, None) == -1
    assert L.cbgmres_destroy(None) == 0
    # the cycle option takes CBG_CYCLE_AUTO (0) or CBG_CYCLE_STREAMED (1) only
    assert pkg.default_opts().cycle == 0
    assert pkg.workspace_bytes(1000, pkg.default_opts(cycle="streamed")) > 0
    assert pkg.workspace_bytes(1000, pkg.default_opts(cycle=2)) == 0
    bad = pkg.default_opts(cycle=-1)
    assert L.cbgmres_create(ctypes.byref(h), 100, 0, None, None, None, ctypes.byref(bad), None) == -1
    assert L.cbgmres_cycle_cluster(None) == -1


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the behaviour without a CUDA device")
def test_no_cpu_fallback(pkg):
    L = pkg.lib()
    buf = ctypes.create_string_buffer(1024)
    addr = (ctypes.addressof(buf) + 255) // 256 * 256
    st = L.cbg_frsz2_compress(ctypes.c_void_p(addr), 4, 32, ctypes.c_void_p(addr), ctypes.c_void_p(addr), None)
    assert st == -2  # CBG_ERR_CUDA: no device, and no host path to fall back to


def test_server_arguments_rejected(pkg):
    L = pkg.lib()
    h = ctypes.c_void_p()
    assert L.cbg_server_create(None, 1 << 20, 4, 4, 4) == -1
    assert L.cbg_server_create(ctypes.byref(h), 0, 4, 4, 4) == -1  # budget below one granule
    assert L.cbg_server_create(ctypes.byref(h), 1 << 20, 0, 4, 4) == -1  # no slot
    assert L.cbg_server_create(ctypes.byref(h), 1 << 20, 257, 4, 4) == -1
    assert L.cbg_server_create(ctypes.byref(h), 1 << 20, 4, 0, 4) == -1  # no step per turn
    assert L.cbg_server_create(ctypes.byref(h), 1 << 20, 4, 4, -1) == -1
    assert L.cbg_server_submit(None, None) == -1
    n = ctypes.c_int32(0)
    assert L.cbg_server_poll(None, None, 0, ctypes.byref(n)) == -1
    assert L.cbg_server_stats(None, None, None, None, None) == -1
    assert L.cbg_server_clock(None) == 0.0
    assert L.cbg_server_destroy(None) == 0


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the behaviour without a CUDA device")
def test_server_needs_a_device(pkg):
    h = ctypes.c_void_p()
    assert pkg.lib().cbg_server_create(ctypes.byref(h), 1 << 20, 4, 4, 4) == -2
    assert not h.value


def test_problem_statement_names(pkg):
    """frsz2_bytes / frsz2_compress / frsz2_decompress and cbgmres_last_error are the same functions
    as their cbg_ counterparts."""
    L = pkg.lib()
    for n, l in ((0, 32), (32, 32), (33, 21), (1000, 16)):
        assert L.frsz2_bytes(n, l) == L.cbg_frsz2_bytes(n, l)
    assert L.frsz2_bytes(10, 40) == 0 and L.cbg_frsz2_bytes(10, 40) == -1
    assert L.frsz2_compress(None, 10, 20, None, None, None) == -10
    assert L.cbgmres_last_error() == L.cbg_last_error() and b"not implemented" in L.cbgmres_last_error()
    assert L.frsz2_decompress(None, None, -1, 32, None, None) == -1


LAYOUT_PROGRAM = r"""
#include <stddef.h>
#include <stdio.h>
#include "cbgmres.h"
#define F(T, f) printf(#T " " #f " %zu %zu\n", offsetof(T, f), sizeof(((T*)0)->f))
#define S(T) printf(#T " sizeof %zu 0\n", sizeof(T))
int main(void) {
  S(cbg_opts); F(cbg_opts, restart); F(cbg_opts, fmt); F(cbg_opts, frsz2_bits); F(cbg_opts, history);
  F(cbg_opts, tol); F(cbg_opts, max_iters); F(cbg_opts, eta); F(cbg_opts, precond); F(cbg_opts, cycle);
  S(cbg_result); F(cbg_result, iters); F(cbg_result, restarts); F(cbg_result, reorths);
  F(cbg_result, converged); F(cbg_result, status); F(cbg_result, true_rrn); F(cbg_result, implicit_rrn);
  F(cbg_result, seconds); F(cbg_result, breakdowns);
  S(cbg_basis); F(cbg_basis, fmt); F(cbg_basis, frsz2_bits); F(cbg_basis, n); F(cbg_basis, vals);
  F(cbg_basis, vals_stride); F(cbg_basis, exps); F(cbg_basis, exps_stride);
  S(cbg_request); F(cbg_request, tag); F(cbg_request, n); F(cbg_request, nnz); F(cbg_request, d_row_ptr);
  F(cbg_request, d_col); F(cbg_request, d_vals); F(cbg_request, d_b); F(cbg_request, d_x); F(cbg_request, opts);
  S(cbg_completion); F(cbg_completion, tag); F(cbg_completion, status); F(cbg_completion, result);
  F(cbg_completion, t_submit); F(cbg_completion, t_admit); F(cbg_completion, t_done);
  printf("status %d %d %d %d %d %d %d %d %d %d\n", CBG_ERR_INVALID_ARG, CBG_ERR_CUDA, CBG_ERR_OOM, CBG_ERR_NONFINITE,
         CBG_ERR_NOT_CONVERGED, CBG_ERR_TIMEOUT, CBG_ERR_BAD_MATRIX, CBG_ERR_STATE, CBG_ERR_BREAKDOWN_NOT_CONVERGED,
         CBG_ERR_UNIMPLEMENTED);
  return 0;
}
"""


def test_struct_layouts_match_the_header(pkg, tmp_path):
    """A C program compiled against include/cbgmres.h prints the size and the offset of every field
    of the structs that cross the ABI; the binding's ctypes mirrors must agree field by field, and
    its status table must name every status the header defines."""
    import shutil
    import subprocess

    cc = shutil.which("cc") or shutil.which("gcc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "layout.c"
    src.write_text(LAYOUT_PROGRAM)
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    mirrors = {"cbg_opts": pkg.Opts, "cbg_result": pkg.Result, "cbg_basis": pkg.Basis, "cbg_request": pkg.Request,
               "cbg_completion": pkg.Completion}
    checked = 0
    for line in out:
        if not line:
            continue
        parts = line.split()
        if parts[0] == "status":
            assert sorted(int(v) for v in parts[1:]) == sorted(k for k in pkg.STATUS if k != 0)
            continue
        T, field, off, size = parts[0], parts[1], int(parts[2]), int(parts[3])
        M = mirrors[T]
        if field == "sizeof":
            assert ctypes.sizeof(M) == off, (T, ctypes.sizeof(M), off)
        else:
            f = getattr(M, field)
            assert (f.offset, f.size) == (off, size), (T, field, f.offset, f.size, off, size)
        checked += 1
    assert checked == 5 + 9 + 9 + 7 + 9 + 6
