"""GPU parity of the fused basis kernels against the oracle:

* dot    h_i = sum_k vhat_i[k] w_k          (Fig. 1 step 5, V_j^T w)
* update w_k - sum_i vhat_i[k] h_i          (Fig. 1 step 5, w - V_j h)

The reference is the oracle's compensated (twice-working-precision) dot of the oracle-decoded basis,
so the comparison measures the GPU's own error. The tolerance follows from the GPU arithmetic:
FRSZ2 blocks are summed exactly against a round-to-nearest 54-bit block fixed point of w (error at
most 2^-54 max_{k in b}|w_k| per unit of |vhat|), cross-block and cross-CTA sums are FP64 over a
tree of depth < 64 (error < 2^-46 sum |vhat w|); the update's per-block fixed point of h_i 2^{q_ib}
keeps 54 bits of the largest term, and each of its at most 2 ceil(nvec/32) integer roundings (a
group sum, a rescaling to a larger block scale) is below 2^(gb-58) of the largest possible term,
2^gb >= ceil(nvec/32). The tolerances below are those bounds with a factor-4 margin.
"""
import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu

FORMATS = [(0, 32), (1, 32), (2, 32), (3, 32), (4, 16), (4, 21), (4, 32)]


def make_basis(cbg, orc, n, nvec, fmt, l, seed):
    # Krylov vectors have unit norm, so every value lies in [-1, 1] (Problem Formulation); the
    # in-block exponent spread of N(0,1) 2^k, k in [-20, 20] per block, is kept.
    V = workloads.basis_values(nvec, n, seed=seed).numpy()
    V /= np.linalg.norm(V, axis=1, keepdims=True)
    B = cbg.BasisStorage(n, nvec, fmt, l)
    Vd = torch.from_numpy(V).cuda()
    for i in range(nvec):
        B.store(i, Vd[i].contiguous())
    enc = [orc.encode(V[i], fmt, l) for i in range(nvec)]
    Vhat = np.stack([orc.decode(v, e, n, fmt, l) for v, e in enc])
    exps = np.stack([e for _, e in enc]) if fmt == 4 else None
    return B, Vhat, exps


def fp16_update_tolerance(Vhat, h, w, idx):
    """Error bound of the binary16 update (exact integer products of the stored values, exact in
    units of 2^-24, with h_i as 54-bit fixed point against the largest |h| of its group of 32
    vectors): the coefficients' rounding adds at most 2^-53 max|h| sum_i |vhat_ik|; each group
    sum keeps 61 - gb bits of the largest of the thread's 8 sums (elements 8c .. 8c + 7), at most
    2^-55 max|h| max_{k' in the 8} sum_i |vhat_ik'| per rounding for up to 2^6 groups; the final
    conversion and subtraction add 2^-52 (|w_k| + sum_i |vhat_ik h_i|). With a factor-4 margin."""
    n = w.size
    absv = np.abs(Vhat)
    col = absv.sum(axis=0)  # sum_i |vhat_ik|
    pad = np.zeros(((n + 7) // 8) * 8)
    pad[:n] = col
    chunk = pad.reshape(-1, 8).max(axis=1)[idx // 8]
    hmax = np.abs(h).max()
    terms = (absv[:, idx] * np.abs(h)[:, None]).sum(axis=0)
    return 4 * (2.0 ** -50 * (np.abs(w[idx]) + terms) + 2.0 ** -53 * hmax * col[idx] +
                2.0 ** -52 * hmax * chunk) + 1e-300


def dot_tolerance(Vhat, w):
    n = w.size
    nb = (n + 31) // 32
    wpad = np.zeros(nb * 32)
    wpad[:n] = np.abs(w)
    wmax = wpad.reshape(nb, 32).max(axis=1)
    vpad = np.zeros((Vhat.shape[0], nb * 32))
    vpad[:, :n] = np.abs(Vhat)
    vabs_b = vpad.reshape(Vhat.shape[0], nb, 32).sum(axis=2)
    s_abs = np.abs(Vhat) @ np.abs(w)
    return 4 * (2.0 ** -46 * s_abs + 2.0 ** -54 * (vabs_b @ wmax)) + 1e-300


@pytest.mark.parametrize("fmt,l", FORMATS)
@pytest.mark.parametrize("n,nvec", [(1, 1), (77, 3), (4096, 1), (4096 + 45, 7), (70000, 20), (300000 + 13, 66),
                                    (128 * 128 * 3 + 32 * 5, 9)])
def test_dot(cbg, orc, fmt, l, n, nvec):
    B, Vhat, _ = make_basis(cbg, orc, n, nvec, fmt, l, seed=n + nvec)
    w = np.random.default_rng(n).standard_normal(n) * np.exp2(np.random.default_rng(n + 1).integers(-6, 6, n))
    h = B.dot(nvec, torch.from_numpy(w).cuda()).cpu().numpy()
    ref = orc.basis_dot(Vhat, w)
    tol = dot_tolerance(Vhat, w)
    assert np.all(np.abs(h - ref) <= tol), (np.abs(h - ref) / tol).max()


@pytest.mark.parametrize("fmt,l", FORMATS)
@pytest.mark.parametrize("n,nvec", [(1, 1), (77, 3), (4096 + 45, 7), (70000, 20), (30000 + 13, 66),
                                    (20000, 100), (300000 + 13, 66), (160000 + 7, 101)])
def test_update(cbg, orc, fmt, l, n, nvec):
    B, Vhat, exps = make_basis(cbg, orc, n, nvec, fmt, l, seed=3 * n + nvec)
    rng = np.random.default_rng(n + 5)
    w = rng.standard_normal(n)
    h = rng.standard_normal(nvec) * np.exp2(rng.integers(-30, 3, nvec))
    wd = torch.from_numpy(w).cuda()
    nrm = torch.zeros(1, dtype=torch.float64, device="cuda")
    B.update(nvec, torch.from_numpy(h).cuda(), wd, norm2=nrm)
    out = wd.cpu().numpy()
    # reference on a sample of elements (all of them for small n)
    idx = np.arange(n) if n <= 5000 else np.unique(np.concatenate([np.arange(64), n - 1 - np.arange(64),
                                                                   rng.integers(0, n, 3000)]))
    ref = orc.basis_update(Vhat[:, idx], h, w[idx])
    terms = np.abs(Vhat[:, idx] * h[:, None])
    # largest possible term of each value's block: |h_i| * 2^(block exponent + 1) for FRSZ2
    if fmt == 4:
        e = np.maximum(exps[:, idx // 32].astype(np.float64), 1.0)
        tmax = (np.abs(h)[:, None] * np.exp2(e - 1023.0 + 1.0)).max(axis=0)
    else:
        tmax = terms.max(axis=0)
    tol = 4 * (2.0 ** -50 * (np.abs(w[idx]) + terms.sum(axis=0)) + nvec * 2.0 ** -53 * tmax) + 1e-300
    if fmt == 2:
        tol = fp16_update_tolerance(Vhat, h, w, idx)
    err = np.abs(out[idx] - ref)
    assert np.all(err <= tol), (err / tol).max()
    # the fused norm is ||w||^2 of the updated vector
    assert abs(nrm.item() - orc.dot2(out, out)) <= 1e-12 * orc.dot2(out, out)


def test_dot_after_update_orthogonal(cbg, orc):
    """One classical Gram-Schmidt pass against an orthonormal FP64 basis leaves w orthogonal to it."""
    n, nvec = 50000, 12
    Q, _ = np.linalg.qr(np.random.default_rng(1).standard_normal((n, nvec)))
    B = cbg.BasisStorage(n, nvec, 0)
    Qd = torch.from_numpy(np.ascontiguousarray(Q.T)).cuda()
    for i in range(nvec):
        B.store(i, Qd[i].contiguous())
    w = torch.from_numpy(np.random.default_rng(2).standard_normal(n)).cuda()
    h = B.dot(nvec, w).clone()
    B.update(nvec, h, w)
    h2 = B.dot(nvec, w).cpu().numpy()
    assert np.abs(h2).max() <= 1e-13 * np.linalg.norm(h.cpu().numpy())


@pytest.mark.parametrize("fmt,l", FORMATS)
@pytest.mark.parametrize("r", [0, 1, 7])
def test_intensity(cbg, orc, fmt, l, r):
    """cbg_intensity (the synthetic benchmark of Fig. 3): sum_k f^r(x_k), f(y) = y/2 + 1/4, over the
    oracle-decoded stored values. Each f step is exact up to one rounding on both sides, so the
    values agree bit for bit and only the order of the final sum differs."""
    n = 4096 * 3 + 45
    B, Vhat, _ = make_basis(cbg, orc, n, 2, fmt, l, seed=11)
    y = Vhat[1].copy()
    for _ in range(r):
        y = y * 0.5 + 0.25
    ref = orc.dot2(y, np.ones(n))
    got = B.intensity(1, r).item()
    assert abs(got - ref) <= n * 2.0 ** -52 * np.abs(y).sum() + 1e-300
    if fmt == 1:  # fp32 storage computed natively in FP32
        y32 = Vhat[1].astype(np.float32)
        for _ in range(r):
            y32 = y32 * np.float32(0.5) + np.float32(0.25)
        ref32 = orc.dot2(y32.astype(np.float64), np.ones(n))
        got32 = B.intensity(1, r, fp32_compute=True).item()
        assert abs(got32 - ref32) <= 8 * 2.0 ** -24 * np.abs(y32.astype(np.float64)).sum()


@pytest.mark.parametrize("l", [16, 21, 32])
@pytest.mark.parametrize("nvec", [33, 300, 1025])
def test_update_many_groups(cbg, orc, l, nvec):
    """The FRSZ2 update combines groups of 32 vectors in integers at rescaled block scales: many
    groups (2^gb >= ceil(nvec/32) sets the rounding unit) and the largest restart the solver takes
    (1024, plus one)."""
    n = 2048 + 77
    B, Vhat, exps = make_basis(cbg, orc, n, nvec, 4, l, seed=nvec + l)
    rng = np.random.default_rng(nvec)
    w = rng.standard_normal(n)
    h = rng.standard_normal(nvec) * np.exp2(rng.integers(-30, 3, nvec))
    wd = torch.from_numpy(w).cuda()
    B.update(nvec, torch.from_numpy(h).cuda(), wd)
    out = wd.cpu().numpy()
    ref = orc.basis_update(Vhat, h, w)
    terms = np.abs(Vhat * h[:, None])
    e = np.maximum(exps[:, np.arange(n) // 32].astype(np.float64), 1.0)
    tmax = (np.abs(h)[:, None] * np.exp2(e - 1023.0 + 1.0)).max(axis=0)
    tol = 4 * (2.0 ** -50 * (np.abs(w) + terms.sum(axis=0)) + nvec * 2.0 ** -53 * tmax) + 1e-300
    err = np.abs(out - ref)
    assert np.all(err <= tol), (err / tol).max()


@pytest.mark.parametrize("fmt,l", [(0, 32), (1, 32), (4, 21), (4, 32)])
def test_empty_inputs(cbg, orc, fmt, l):
    """The degenerate sizes of the Gram-Schmidt pass: no basis vectors (nvec = 0) and empty vectors
    (n = 0). With nvec = 0 the dot writes nothing and the update leaves w as it is but still
    reports ||w||^2; with n = 0 every sum is empty: h = 0 and ||w||^2 = 0."""
    n = 4096 + 45
    B = cbg.BasisStorage(n, 3, fmt, l)
    w = torch.from_numpy(np.random.default_rng(5).standard_normal(n)).cuda()
    w0 = w.clone()
    h = torch.full((4,), 7.0, dtype=torch.float64, device="cuda")
    nrm = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    B.dot(0, w, out=h)
    B.update(0, h, w, norm2=nrm)
    torch.cuda.synchronize()
    assert torch.equal(h, torch.full_like(h, 7.0))
    assert torch.equal(w, w0)
    wh = w0.cpu().numpy()
    ref = orc.dot2(wh, wh)
    assert abs(nrm.item() - ref) <= 1e-14 * ref

    B0 = cbg.BasisStorage(0, 3, fmt, l)
    e = torch.empty(8, dtype=torch.float64, device="cuda")[:0]
    B0.store(0, e)
    B0.dot(3, e, out=h)
    nrm.fill_(-1.0)
    B0.update(3, h, e, norm2=nrm)
    torch.cuda.synchronize()
    assert h[:3].tolist() == [0.0, 0.0, 0.0] and h[3].item() == 7.0
    assert nrm.item() == 0.0


@pytest.mark.parametrize("op", ["dot", "update"])
def test_fp16_values_of_two_and_more(cbg, orc, op):
    """A binary16 basis whose vectors are not normalised (values up to ~1000): the integer path takes
    values below 2 only (exact integers in units of 2^-24); a block (dot) or a warp's range of a
    vector (update) holding a larger value goes through FP64 products instead. Mixed with unit-norm
    vectors, against the oracle."""
    n, nvec = 20000 + 13, 12
    B, Vhat, _ = make_basis(cbg, orc, n, nvec, 2, 32, seed=77)
    rng = np.random.default_rng(78)
    scale = np.where(np.arange(nvec) % 3 == 0, 300.0, 1.0)  # every third vector reaches values >= 2
    V = workloads.basis_values(nvec, n, seed=79).numpy()
    V /= np.abs(V).max(axis=1, keepdims=True)
    V *= scale[:, None]
    Vd = torch.from_numpy(V).cuda()
    for i in range(nvec):
        B.store(i, Vd[i].contiguous())
    enc = [orc.encode(V[i], 2, 32) for i in range(nvec)]
    Vhat = np.stack([orc.decode(v, e, n, 2, 32) for v, e in enc])
    assert np.abs(Vhat).max() >= 2.0 and np.abs(Vhat[1]).max() < 2.0
    if op == "dot":
        w = rng.standard_normal(n)
        got = B.dot(nvec, torch.from_numpy(w).cuda()).cpu().numpy()
        ref = orc.basis_dot(Vhat, w)
        tol = dot_tolerance(Vhat, w)
        assert np.all(np.abs(got - ref) <= tol), (np.abs(got - ref) / tol).max()
    else:
        w = rng.standard_normal(n)
        h = rng.standard_normal(nvec) * np.exp2(rng.integers(-10, 3, nvec))
        wd = torch.from_numpy(w).cuda()
        B.update(nvec, torch.from_numpy(h).cuda(), wd)
        out = wd.cpu().numpy()
        ref = orc.basis_update(Vhat, h, w)
        idx = np.arange(n)
        terms = np.abs(Vhat * h[:, None])
        # the FP64 path's bound (the cast formats') added to the integer path's
        tol = fp16_update_tolerance(Vhat, h, w, idx) + 4 * nvec * 2.0 ** -53 * terms.sum(axis=0)
        assert np.all(np.abs(out - ref) <= tol), (np.abs(out - ref) / tol).max()


@pytest.mark.parametrize("fmt", [3, 1])
def test_cast_dot_block_fixed_point_edges(cbg, orc, fmt):
    """The bfloat16 (fmt 3) and binary32 (fmt 1) dots put each 32-value block on a fixed point
    2^(148 - E), resp. 2^(188 - E), on the fly (E the block's largest exponent field). A bfloat16
    block with a nonzero value more than 14 binades below the largest, or with E below 21, takes a
    wide integer path (62-bit codes, within 54 binades); FP64 takes what neither holds: bfloat16
    subnormals beside normal values, a binary32 value more than 38 binades down or subnormal, the
    ragged last block. Blocks
    built for each branch: one value scaled down by exactly that many binades (exact unless the
    block's largest lies higher) or by more (FP64), all-zero blocks, tiny values, single nonzero
    values and subnormals; against the oracle's compensated dot of the decoded values, with the dot
    tolerance."""
    span, tiny, sub = {3: (14, 2.0 ** -120, 2.0 ** -130), 1: (38, 2.0 ** -100, 2.0 ** -140)}[fmt]
    n, nvec = 32 * 700 + 19, 9
    rng = np.random.default_rng(91 + fmt)
    V = rng.standard_normal((nvec, n)) * 2.0 ** -8
    nb = (n + 31) // 32
    for i in range(nvec):
        for b in range(nb):
            blk = V[i, 32 * b: 32 * b + 32]
            kind = (b + 3 * i) % 8
            if kind == 1:  # one value `span` binades down
                blk[rng.integers(0, blk.size)] *= 2.0 ** -span
            elif kind == 2:  # further down: FP64
                blk[rng.integers(0, blk.size)] *= 2.0 ** -rng.integers(span + 2, span + 40)
            elif kind == 3:
                blk[:] = 0.0
            elif kind == 4:  # tiny values
                blk *= tiny
            elif kind == 5:  # one nonzero value
                keep = rng.integers(0, blk.size)
                v = blk[keep]
                blk[:] = 0.0
                blk[keep] = v
            elif kind == 6:  # subnormals next to normal values: FP64
                blk[::5] = sub
    B = cbg.BasisStorage(n, nvec, fmt, 32)
    Vd = torch.from_numpy(V).cuda()
    for i in range(nvec):
        B.store(i, Vd[i].contiguous())
    Vhat = np.stack([orc.decode(*orc.encode(V[i], fmt, 32), n, fmt, 32) for i in range(nvec)])
    for seed in range(2):
        w = np.random.default_rng(100 + seed).standard_normal(n) * np.exp2(rng.integers(-30, 30, n))
        got = B.dot(nvec, torch.from_numpy(w).cuda()).cpu().numpy()
        ref = orc.basis_dot(Vhat, w)
        tol = dot_tolerance(Vhat, w)
        assert np.all(np.abs(got - ref) <= tol), (seed, (np.abs(got - ref) / tol).max())
