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
    return sorted(set(n for n in names if n.startswith("cbg")))


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
    assert L.cbgmres_create(ctypes.byref(h), 100, 0, None, None, None, ctypes.byref(bad), None) == -1
    bad = pkg.default_opts(restart=200)
    assert L.cbgmres_create(ctypes.byref(h), 100, 0, None, None, None, ctypes.byref(bad), None) == -1
    assert L.cbg_frsz2_compress(None, 10, 21, None, None, None) == -1
    assert L.cbg_frsz2_compress(None, 10, 20, None, None, None) == -1
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
