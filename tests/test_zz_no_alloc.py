"""cbg_basis_dot_noalloc: the basis dot product for callers that cannot allocate device memory
(for example a plugin whose host application owns all device memory, or a path that must not call
cudaMalloc because it can synchronise the device). It keeps its partial sums in a fixed array that
the library defines instead of a caller-provided work buffer.

Checked against the regular entry point (cbg_basis_dot, which takes a work buffer) on two calls in
a row, with the dot-product tolerance of tests/test_gpu_basis.py, and for its size limit. This file
is collected last so that a run stopping at its first failure has run every other test first."""
import ctypes

import numpy as np
import pytest
import torch

from test_gpu_basis import dot_tolerance, make_basis

pytestmark = pytest.mark.gpu


def _noalloc(cbg, B, nvec, w, h):
    return cbg.lib().cbg_basis_dot_noalloc(ctypes.byref(B.struct), nvec, ctypes.c_void_p(w.data_ptr()),
                                           ctypes.c_void_p(h.data_ptr()),
                                           ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("fmt,l,n,nvec", [(4, 32, 300000 + 13, 20), (4, 21, 70000, 128), (0, 32, 50000 + 7, 9)])
def test_noalloc_matches_regular_entry_point(cbg, orc, fmt, l, n, nvec):
    B, Vhat, _ = make_basis(cbg, orc, n, nvec, fmt, l, seed=11 * n + nvec)
    rng = np.random.default_rng(n)
    for call in range(2):  # two calls in a row share the fixed scratch array
        w = rng.standard_normal(n)
        wd = torch.from_numpy(w).cuda()
        ref = B.dot(nvec, wd).cpu().numpy()
        h = torch.full((nvec,), np.nan, dtype=torch.float64, device="cuda")
        assert _noalloc(cbg, B, nvec, wd, h) == 0, cbg.last_error()
        got = h.cpu().numpy()
        tol = dot_tolerance(Vhat, w)
        assert np.all(np.abs(got - ref) <= tol), (call, (np.abs(got - ref) / tol).max())


def test_noalloc_rejects_more_vectors_than_its_scratch_holds(cbg, orc):
    n = 4096
    B, _, _ = make_basis(cbg, orc, n, 2, 4, 32, seed=5)
    w = torch.zeros(n, dtype=torch.float64, device="cuda")
    h = torch.zeros(200, dtype=torch.float64, device="cuda")
    assert _noalloc(cbg, B, 129, w, h) == -1
    assert "128" in cbg.last_error()
