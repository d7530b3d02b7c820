"""GPU parity of the codec (Design section: compression steps 1-6, decompression steps 1-4) and of
the cast storage formats against the oracle: compressed bytes and cast bits must be bit-exact on
identical FP64 inputs; decoded values bit-exact. Sizes cover a single value, ragged tails, exact
block multiples and several grid-strides; inputs cover wide in-block exponent spreads, subnormals,
signed zeros and the special values of the workload generator."""
import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu

SIZES = [1, 5, 31, 32, 33, 100, 1000, 4097, 32 * 1000 + 17, 131072 + 96]
LS = [16, 21, 32]


def inputs(n, seed, kind):
    rng = np.random.default_rng(seed)
    if kind == "normal":
        return rng.standard_normal(n)
    if kind == "spread":
        return rng.standard_normal(n) * np.exp2(rng.integers(-40, 41, n))
    if kind == "blockscale":
        return workloads.basis_values(1, n, seed=seed).numpy()[0]
    if kind == "tiny":
        return rng.standard_normal(n) * np.exp2(rng.integers(-1080, -1015, n))
    if kind == "special":
        sv = workloads.special_values().numpy()
        sv = sv[np.isfinite(sv)]
        return np.resize(sv, n) * np.where(rng.random(n) < 0.5, 1.0, -1.0)
    raise ValueError(kind)


@pytest.mark.parametrize("l", LS)
@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("kind", ["normal", "spread", "blockscale", "tiny", "special"])
def test_compress_bit_exact(cbg, orc, l, n, kind):
    x = inputs(n, 1000 + n + l, kind)
    e_ref, c_ref = orc.frsz2_compress(x, l)
    xd = torch.from_numpy(x).cuda()
    exps, codes = cbg.frsz2_compress(xd, l)
    torch.cuda.synchronize()
    nb = (n + 31) // 32
    assert np.array_equal(exps[:nb].cpu().numpy().view(np.uint32), e_ref)
    assert np.array_equal(codes[: nb * l].cpu().numpy().view(np.uint32), c_ref)
    out = cbg.frsz2_decompress(exps, codes, n, l)
    ref = orc.frsz2_decompress(e_ref, c_ref, n, l)
    assert np.array_equal(out.cpu().numpy().view(np.uint64), ref.view(np.uint64))


@pytest.mark.parametrize("fmt", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("n", [1, 33, 4097, 100000])
def test_basis_store_load_bit_exact(cbg, orc, fmt, n):
    l = 32 if fmt != 4 else 21
    x = inputs(n, 7 + n + fmt, "spread" if fmt in (0, 4) else "normal")
    x[: min(n, 4)] = [0.0, -0.0, 2.0 ** -149, -(2.0 ** -24)][: min(n, 4)]  # zeros and cast subnormals
    B = cbg.BasisStorage(n, 3, fmt, l)
    xd = torch.from_numpy(x).cuda()
    B.store(1, xd)
    dec = B.load(1).cpu().numpy()
    vals_ref, exps_ref = orc.encode(x, fmt, l)
    vb, eb = B.vector_bytes(1)
    vb = vb.cpu().numpy()
    nbytes = vals_ref.nbytes
    assert np.array_equal(vb[:nbytes].view(vals_ref.dtype), vals_ref)
    if fmt == 4:
        assert np.array_equal(eb.cpu().numpy()[: exps_ref.nbytes].view(np.uint32), exps_ref)
    ref = orc.decode(vals_ref, exps_ref, n, fmt, l)
    assert np.array_equal(dec.view(np.uint64), ref.view(np.uint64))


# ---- normalise and append (Fig. 1 steps 13-14): v = w / h, correctly rounded --------------------

APPEND_H = [1.0, 3.0, 0.1, 7.0 / 16.0, 1.0 / 3.0, 2.0 ** -500 * 1.7, 2.0 ** 600 * 1.3, 0.7123456789012345,
            np.nextafter(1.0, 2.0), np.nextafter(2.0, 0.0)]


@pytest.mark.parametrize("h", APPEND_H)
@pytest.mark.parametrize("fmt,l", [(4, 32), (4, 21), (4, 16), (0, 32), (1, 32), (2, 32), (3, 32)])
def test_append_divides_exactly(cbg, orc, fmt, l, h):
    """cbg_basis_append stores v = w / h with every element the correctly rounded IEEE quotient,
    as the oracle divides (not w * (1/h)): v bit for bit against numpy's division over 300 000
    values spanning 2^-60 .. 2^60 (and signed zeros and subnormals), and the stored vector bit for
    bit against the oracle's encoding of that v."""
    n = 300000 + 7
    rng = np.random.default_rng(int(h * 1e6) % 1000 + fmt * 7 + l)
    w = rng.standard_normal(n) * np.exp2(rng.integers(-60, 61, n))
    w[::97] = 0.0
    w[::193] = -0.0
    w[5::211] = rng.standard_normal(w[5::211].size) * 2.0 ** -1060  # subnormal numerators
    if h > 1e100:
        w *= 2.0 ** 500  # keep the quotients finite and normal for the huge divisor
    ref = w / h
    B = cbg.BasisStorage(n, 3, fmt, l)
    wd = torch.from_numpy(w).cuda()
    hd = torch.tensor([h], dtype=torch.float64, device="cuda")
    v = torch.empty_like(wd)
    B.append(1, wd, hd, v)
    got = v.cpu().numpy()
    assert np.array_equal(got.view(np.uint64), ref.view(np.uint64)), int((got != ref).sum())
    vals, exps = B.vector_bytes(1)
    enc_vals, enc_exps = orc.encode(ref, fmt, l)
    vb = vals.cpu().numpy()[: enc_vals.nbytes]
    assert np.array_equal(vb, enc_vals.view(np.uint8))
    if fmt == 4:
        eb = exps.cpu().numpy()[: enc_exps.nbytes]
        assert np.array_equal(eb, enc_exps.view(np.uint8))
