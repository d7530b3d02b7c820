"""Parity at the full sizes, in the launch configuration bench.py times, on outputs the oracle can
compute one by one:

* the standalone basis step: 100 FRSZ2-32 vectors x n = 2^24 values (N(0,1) 2^k per 32-value
  block, k in [-20, 20], seed 1, unit norm), compressed, then h = V^T w and w - V h with ||w||^2.
  - compressed bytes of sampled blocks: bit-exact against the oracle's codec (it is block-local);
  - h_i of sampled vectors: against the oracle's compensated dot of its own decoded vector;
  - the update at sampled elements: against the oracle over all 100 vectors;
  - the fused norm: against the oracle's compensated norm of the whole result.
  Tolerances are those of test_gpu_basis.py.
* the 256^3 convection-diffusion solve (and the 4M-row power-law solve) to 1e-10 (b = A 1 from the
  oracle's SpMV, restart 100) with
  the FRSZ2-32 and the fp64 basis: the final residual recomputed with the oracle's SpMV, and the
  solve compared with the oracle's own solve of the same system, which takes the oracle hours and
  is therefore stored as tests/golden/solve_{c3,c4}_<format>.json (written by
  tests/golden/make_solve_references.py): iterations within 2%, second-pass counts that differ by no more than the
  step counts do, equal breakdown counts, and the solution within 1e-8 (relative) at the stored sample of indices.
"""
import json
import os

import numpy as np
import pytest
import torch

import workloads

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

N, NVEC, L = 1 << 24, 100, 32


def block_words(B, slot, blocks):
    vals, exps = B.vector_bytes(slot)
    codes = vals.view(torch.int32).cpu().numpy().view(np.uint32)
    ex = exps.view(torch.int32).cpu().numpy().view(np.uint32)
    return codes, ex


def test_basis_step_full_size(cbg, orc):
    rng = np.random.default_rng(123)
    nb = N // 32
    blocks = np.unique(np.concatenate([[0, nb - 1], rng.integers(0, nb, 300)]))
    B = cbg.BasisStorage(N, NVEC + 1, cbg.FRSZ2, L)
    sampled = np.zeros((NVEC, blocks.size, 32))
    full_check = [0, 17, 63, 99]
    full_host = {}
    for i in range(NVEC):
        x = workloads.basis_vector(i, N, seed=1, device="cuda")
        B.store(i, x)
        xh = x.view(-1, 32)[torch.from_numpy(blocks).cuda()].cpu().numpy()
        sampled[i] = xh
        if i in full_check:
            full_host[i] = x.cpu().numpy()
    torch.cuda.synchronize()
    # compressed bytes of the sampled blocks, bit for bit
    for i in (0, 1, 50, 99):
        codes, ex = block_words(B, i, blocks)
        for j, b in enumerate(blocks):
            e_ref, c_ref = orc.frsz2_compress(sampled[i, j], L)
            assert ex[b] == e_ref[0], (i, b)
            assert np.array_equal(codes[b * 32:(b + 1) * 32], c_ref), (i, b)
    # the step as bench.py runs it
    w = workloads.basis_vector(NVEC, N, seed=1, device="cuda")
    wh = w.cpu().numpy()
    h = B.dot(NVEC, w).clone()
    hh = h.cpu().numpy()
    for i in full_check:
        e_i, c_i = orc.frsz2_compress(full_host[i], L)
        vhat = orc.frsz2_decompress(e_i, c_i, N, L)
        ref = orc.dot2(vhat, wh)
        wmax = np.abs(wh).reshape(-1, 32).max(axis=1)
        vabs = np.abs(vhat).reshape(-1, 32).sum(axis=1)
        tol = 4 * (2.0 ** -46 * orc.dot2(np.abs(vhat), np.abs(wh)) + 2.0 ** -54 * float(vabs @ wmax))
        assert abs(hh[i] - ref) <= tol, (i, hh[i], ref, tol)
    nrm = torch.zeros(1, dtype=torch.float64, device="cuda")
    B.update(NVEC, h, w, norm2=nrm)
    out = w.cpu().numpy()
    # the update at every element of 40 sampled blocks, over all 100 vectors
    sel = np.arange(0, blocks.size, max(1, blocks.size // 40))
    for j in sel:
        b = blocks[j]
        vh = np.stack([orc.frsz2_decompress(*orc.frsz2_compress(sampled[i, j], L), 32, L) for i in range(NVEC)])
        ref = orc.basis_update(vh, hh, wh[b * 32:(b + 1) * 32])
        exps = np.array([orc.frsz2_compress(sampled[i, j], L)[0][0] for i in range(NVEC)], dtype=np.float64)
        tmax = (np.abs(hh) * np.exp2(np.maximum(exps, 1.0) - 1023.0 + 1.0)).max()
        terms = np.abs(vh * hh[:, None]).sum(axis=0)
        tol = 4 * (2.0 ** -50 * (np.abs(wh[b * 32:(b + 1) * 32]) + terms) + NVEC * 2.0 ** -53 * tmax)
        err = np.abs(out[b * 32:(b + 1) * 32] - ref)
        assert np.all(err <= tol), (b, (err / tol).max())
    ref_n = orc.dot2(out, out)
    assert abs(nrm.item() - ref_n) <= 1e-12 * ref_n


ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def c3(orc):
    Ah = workloads.convdiff(256, 3, (1.0, 1.0, 1.0), 50.0)
    rp, col, vals = Ah.numpy()
    bh = orc.spmv(rp, col, vals, np.ones(Ah.n))
    return Ah.to("cuda"), (rp, col, vals), bh


@pytest.fixture(scope="module")
def c4(orc):
    Ah = workloads.powerlaw(1 << 22, seed=2)
    rp, col, vals = Ah.numpy()
    bh = orc.spmv(rp, col, vals, np.ones(Ah.n))
    return Ah.to("cuda"), (rp, col, vals), bh


@pytest.mark.parametrize("fmt,l,name", [("frsz2", 32, "frsz2_32"), ("fp64", 32, "fp64")])
def test_c3_solve_full_size(cbg, orc, c3, fmt, l, name):
    full_size_solve(cbg, orc, c3, fmt, l, "c3", name)


@pytest.mark.parametrize("fmt,l,name", [("frsz2", 32, "frsz2_32"), ("fp64", 32, "fp64")])
def test_c4_solve_full_size(cbg, orc, c4, fmt, l, name):
    """The 4M-row power-law system (Pareto row lengths 10-2000, seed 2), b = A 1, restart 100, to
    1e-10, against the oracle's stored solve tests/golden/solve_c4_<format>.json; its rows take the
    segment-sorted long-row SpMV."""
    full_size_solve(cbg, orc, c4, fmt, l, "c4", name)


def full_size_solve(cbg, orc, system, fmt, l, config, name):
    A, (rp, col, vals), bh = system
    S = cbg.Solver(A.row_ptr, A.col, A.vals, restart=100, tol=1e-10, fmt=fmt, frsz2_bits=l)
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    r = S.solve(torch.from_numpy(bh).cuda(), x)
    S.close()
    assert r.converged and r.true_rrn <= 1e-10
    xh = x.cpu().numpy()
    rrn = orc.nrm2(bh - orc.spmv(rp, col, vals, xh)) / orc.nrm2(bh)
    assert rrn <= 1.0001e-10
    assert abs(rrn - r.true_rrn) <= 1e-3 * rrn
    path = os.path.join(ROOT, "tests", "golden", f"solve_{config}_{name}.json")
    if not os.path.exists(path):
        pytest.skip(f"no stored oracle solve {os.path.basename(path)}")
    with open(path) as f:
        ref = json.load(f)
    if "matrix_sha256" in ref:
        import hashlib

        h = hashlib.sha256()
        for a, t in ((rp, np.int32), (col, np.int32), (vals, np.float64)):
            h.update(np.ascontiguousarray(a, dtype=t).tobytes())
        if h.hexdigest() != ref["matrix_sha256"]:
            # the stencil is deterministic; the power-law matrix is drawn from the host's generator
            assert config != "c3", "the 256^3 stencil differs from the one the record was computed on"
            pytest.skip(f"this host's generator drew another {config} matrix ({col.size} nonzeros, the record's "
                        f"{ref.get('nnz')}) than the host that wrote {os.path.basename(path)}")
    assert ref["converged"]
    assert abs(r.iters - ref["iters"]) <= max(1, 0.02 * ref["iters"]), (r.iters, ref["iters"])
    assert r.breakdowns == ref["breakdowns"]
    assert abs(r.reorths - ref["reorths"]) <= abs(r.iters - ref["iters"]), (r.reorths, ref["reorths"])
    idx = np.array(ref["sample_index"])
    xo = np.array([float.fromhex(v) for v in ref["sample_x"]])
    dx = np.linalg.norm(xh[idx] - xo) / np.linalg.norm(xo)
    print(f"{config} {name}: GPU {r.iters} steps, {r.reorths} second passes, {r.breakdowns} breakdowns; "
          f"oracle {ref['iters']}, {ref['reorths']}, {ref['breakdowns']}; x at {idx.size} indices {dx:.2e}")
    assert dx <= 1e-8
