"""cbg_basis_dot_noalloc: the basis dot product for callers that cannot allocate device memory (for
example a plugin whose host application owns all device memory, or a path that must not call
cudaMalloc because it can synchronise the device). It keeps its partial sums in a fixed array that
the library defines instead of a caller-provided work buffer.

Checked on two calls in a row (the calls share the fixed array) against the oracle's compensated
dot of the oracle-decoded basis, with the dot-product tolerance of tests/test_gpu_basis.py, and
against the regular entry point (cbg_basis_dot, which takes a work buffer); in every storage format;
on empty vectors (h must become 0 whatever it held); on a large basis of the most vectors it takes;
and for its size limit. This file is collected last so that a run stopping at its first failure
has run every other test first."""
import ctypes

import numpy as np
import pytest
import torch

from test_gpu_basis import FORMATS, dot_tolerance, make_basis

pytestmark = pytest.mark.gpu


def _noalloc(cbg, B, nvec, w, h):
    return cbg.lib().cbg_basis_dot_noalloc(ctypes.byref(B.struct), nvec, ctypes.c_void_p(w.data_ptr()),
                                           ctypes.c_void_p(h.data_ptr()),
                                           ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("fmt,l", FORMATS)
@pytest.mark.parametrize("n,nvec", [(300000 + 13, 20), (70000, 128), (4096 + 45, 7)])
def test_noalloc_matches_oracle_and_regular_entry_point(cbg, orc, fmt, l, n, nvec):
    B, Vhat, _ = make_basis(cbg, orc, n, nvec, fmt, l, seed=11 * n + nvec)
    rng = np.random.default_rng(n + fmt)
    for call in range(2):  # two calls in a row share the fixed scratch array
        w = rng.standard_normal(n) * np.exp2(rng.integers(-6, 6, n))
        wd = torch.from_numpy(w).cuda()
        regular = B.dot(nvec, wd).cpu().numpy()
        h = torch.full((nvec,), np.nan, dtype=torch.float64, device="cuda")
        assert _noalloc(cbg, B, nvec, wd, h) == 0, cbg.last_error()
        got = h.cpu().numpy()
        ref = orc.basis_dot(Vhat, w)
        tol = dot_tolerance(Vhat, w)
        assert np.all(np.abs(got - ref) <= tol), (call, (np.abs(got - ref) / tol).max())
        assert np.all(np.abs(got - regular) <= 2 * tol), (call, (np.abs(got - regular) / tol).max())


def test_noalloc_large_basis(cbg):
    """2^22 values x 128 vectors (fp32 storage, 2 GiB): the most vectors the fixed array takes, at a
    size where every CTA of the grid has work, against cbg_basis_dot on two calls in a row."""
    n, nvec = 1 << 22, 128
    B = cbg.BasisStorage(n, nvec, cbg.FP32)
    g = torch.Generator(device="cuda")
    g.manual_seed(7)
    for i in range(nvec):
        v = torch.randn(n, dtype=torch.float64, device="cuda", generator=g)
        B.store(i, v / torch.linalg.vector_norm(v))
    for call in range(2):
        w = torch.randn(n, dtype=torch.float64, device="cuda", generator=g)
        regular = B.dot(nvec, w).clone()
        h = torch.full((nvec,), np.nan, dtype=torch.float64, device="cuda")
        assert _noalloc(cbg, B, nvec, w, h) == 0, cbg.last_error()
        diff = (h - regular).abs().max().item()
        assert diff <= 1e-12 * regular.abs().max().item(), (call, diff)


@pytest.mark.parametrize("fmt,l", [(0, 32), (4, 32)])
def test_noalloc_empty_vectors_give_zero(cbg, fmt, l):
    """n = 0: every h_i is an empty sum, 0, whatever d_h held before (NaN here); nvec = 0 writes
    nothing."""
    B0 = cbg.BasisStorage(0, 3, fmt, l)
    e = torch.empty(8, dtype=torch.float64, device="cuda")[:0]
    h = torch.full((4,), np.nan, dtype=torch.float64, device="cuda")
    assert _noalloc(cbg, B0, 3, e, h) == 0, cbg.last_error()
    torch.cuda.synchronize()
    got = h.cpu().numpy()
    assert got[:3].tolist() == [0.0, 0.0, 0.0] and np.isnan(got[3])
    h.fill_(7.0)
    assert _noalloc(cbg, B0, 0, e, h) == 0
    torch.cuda.synchronize()
    assert torch.equal(h, torch.full_like(h, 7.0))


def test_noalloc_rejects_more_vectors_than_its_scratch_holds(cbg, orc):
    n = 4096
    B, _, _ = make_basis(cbg, orc, n, 2, 4, 32, seed=5)
    w = torch.zeros(n, dtype=torch.float64, device="cuda")
    h = torch.zeros(200, dtype=torch.float64, device="cuda")
    assert _noalloc(cbg, B, 129, w, h) == -1
    assert "128" in cbg.last_error()
