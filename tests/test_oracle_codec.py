"""Pins of the oracle's FRSZ2 codec (arXiv 2409.15468, Design section) against things other than
the oracle itself: the paper's storage sizes (Eq. 3 and the 33 bits per value of frsz2_32),
hand-derived blocks (tests/golden), Eq. 2 evaluated in exact rational arithmetic, the error bound
that truncation to a per-block quantum implies, and the random-access and block-independence
properties the Decompression and Compression subsections state."""
import math
import os
import struct
from fractions import Fraction

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "frsz2_hand_blocks.txt")
LS = (16, 21, 32)
KINDS = ["normal", "spread", "blockscale", "tiny", "huge", "sparse"]


def efield(x: float) -> int:
    return (struct.unpack("<Q", struct.pack("<d", x))[0] >> 52) & 0x7FF


def signbit(x: float) -> int:
    return 1 if math.copysign(1.0, x) < 0 else 0


def eq2_block(xs, l):
    """Eq. 2 in exact arithmetic: each value becomes sign * floor(|x| / 2^q) * 2^q with
    q = max(e_max, 1) - 1023 - (l - 2); returns (e_max, codes, decoded values)."""
    xs = list(xs) + [0.0] * (32 - len(xs))
    e_max = max(efield(x) for x in xs)
    q = max(e_max, 1) - 1023 - (l - 2)
    scale = Fraction(2) ** q
    codes, dec = [], []
    for x in xs:
        S = math.floor(abs(Fraction(x)) / scale)
        assert S < 2 ** (l - 1)
        codes.append((signbit(x) << (l - 1)) | S)
        v = float(S * scale)  # exact: S has at most l-1 significant bits
        dec.append(-v if signbit(x) else v)
    return e_max, codes, dec


def pack_stream(codes, l):
    acc = 0
    for i, c in enumerate(codes):
        acc |= c << (i * l)
    return [(acc >> (32 * w)) & 0xFFFFFFFF for w in range(l)]


def bits_equal(a, b):
    return np.array_equal(np.asarray(a, dtype=np.float64).view(np.uint64), np.asarray(b, dtype=np.float64).view(np.uint64))


def test_storage_size_eq3(orc):
    # frsz2_32 stores 33 bits per value (synthetic-performance discussion): 32 values -> 132 bytes.
    assert orc.frsz2_bytes(32, 32) == 132
    assert orc.frsz2_bytes(32, 32) * 8 / 32 == 33
    assert orc.frsz2_bytes(32, 21) == 21 * 4 + 4
    assert orc.frsz2_bytes(32, 16) == 16 * 4 + 4
    assert orc.frsz2_bytes(0, 32) == 0
    assert orc.frsz2_bytes(33, 32) == 2 * 132  # ceil(n / BS) blocks
    assert orc.frsz2_bytes(2 ** 24, 32) == 2 ** 19 * 132
    assert orc.frsz2_code_words(100, 21) == 4 * 21


def test_golden_hand_blocks(orc):
    cases = 0
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            l_s, xs_s, emax_s, words_s, dec_s = line.split("|")
            l = int(l_s)
            xs = [float.fromhex(t) for t in xs_s.split(",")]
            words = [int(t, 16) for t in words_s.split(",")]
            dec = [float.fromhex(t) for t in dec_s.split(",")]
            block = np.zeros(32)
            block[: len(xs)] = xs
            exps, codes = orc.frsz2_compress(block, l)
            assert int(exps[0]) == int(emax_s)
            assert [int(c) for c in codes[: len(words)]] == words
            assert not codes[len(words):].any()
            out = orc.frsz2_decompress(exps, codes, 32, l)
            assert bits_equal(out[: len(dec)], dec)
            cases += 1
    assert cases == 8


def _random_blocks(rng, nblk, kind):
    if kind == "normal":
        return rng.standard_normal((nblk, 32))
    if kind == "spread":  # N(0,1) * 2^k, k in [-40, 40] per value
        return rng.standard_normal((nblk, 32)) * np.exp2(rng.integers(-40, 41, (nblk, 32)))
    if kind == "blockscale":
        return rng.standard_normal((nblk, 32)) * np.exp2(rng.integers(-20, 21, (nblk, 1)))
    if kind == "tiny":  # around and below the normal range
        return rng.standard_normal((nblk, 32)) * np.exp2(rng.integers(-1080, -1015, (nblk, 32)))
    if kind == "huge":
        return rng.standard_normal((nblk, 32)) * np.exp2(rng.integers(900, 1022, (nblk, 32)))
    if kind == "sparse":
        x = rng.standard_normal((nblk, 32))
        x[rng.random((nblk, 32)) < 0.7] = 0.0
        x[rng.random((nblk, 32)) < 0.1] = -0.0
        return x
    raise ValueError(kind)


@pytest.mark.parametrize("l", LS)
@pytest.mark.parametrize("kind", KINDS)
def test_eq2_exact_rational(orc, l, kind):
    rng = np.random.default_rng(1000 + 10 * l + KINDS.index(kind))
    blocks = _random_blocks(rng, 24, kind)
    x = blocks.reshape(-1)
    exps, codes = orc.frsz2_compress(x, l)
    out = orc.frsz2_decompress(exps, codes, x.size, l)
    for b in range(blocks.shape[0]):
        e_max, ecodes, edec = eq2_block(blocks[b], l)
        assert int(exps[b]) == e_max
        assert [orc.frsz2_get_code(codes, b * 32 + i, l) for i in range(32)] == ecodes
        assert pack_stream(ecodes, l) == [int(w) for w in codes[b * l:(b + 1) * l]]
        assert bits_equal(out[b * 32:(b + 1) * 32], edec)


@pytest.mark.parametrize("l", LS)
def test_error_bound_sign_and_magnitude(orc, l):
    rng = np.random.default_rng(7 + l)
    x = _random_blocks(rng, 400, "spread").reshape(-1)
    exps, codes = orc.frsz2_compress(x, l)
    xt = orc.frsz2_decompress(exps, codes, x.size, l)
    blk = x.reshape(-1, 32)
    q = np.maximum(exps.astype(np.int64), 1) - 1023 - (l - 2)
    quantum = np.exp2(q.astype(np.float64))[:, None]
    err = np.abs(blk - xt.reshape(-1, 32))
    assert np.all(err < quantum)  # truncation to the block quantum
    bmax = np.abs(blk).max(axis=1, keepdims=True)
    assert np.all(err <= 2.0 ** -(l - 2) * bmax)  # relative to the block maximum (normal blocks)
    assert np.all(np.abs(xt) <= np.abs(x))  # truncation toward zero
    assert np.array_equal(np.signbit(xt), np.signbit(x))  # sign kept, also for values cut to 0


@pytest.mark.parametrize("l", LS)
def test_idempotent(orc, l):
    rng = np.random.default_rng(11 + l)
    x = _random_blocks(rng, 200, "spread").reshape(-1)
    e1, c1 = orc.frsz2_compress(x, l)
    e2, c2 = orc.frsz2_compress(orc.frsz2_decompress(e1, c1, x.size, l), l)
    assert np.array_equal(e1, e2) and np.array_equal(c1, c2)


@pytest.mark.parametrize("l", LS)
def test_random_access_and_block_independence(orc, l):
    rng = np.random.default_rng(21 + l)
    n = 32 * 9 + 13  # ragged tail
    x = rng.standard_normal(n) * np.exp2(rng.integers(-10, 10, n))
    exps, codes = orc.frsz2_compress(x, l)
    full = orc.frsz2_decompress(exps, codes, n, l)
    for i in rng.integers(0, n, 60):
        assert struct.pack("<d", orc.frsz2_decode_one(exps, codes, int(i), l)) == struct.pack("<d", full[i])
    # the compressed bytes of a block are a function of that block alone (tail padded with +0.0)
    for b in range(exps.size):
        blk = np.zeros(32)
        seg = x[b * 32:(b + 1) * 32]
        blk[: seg.size] = seg
        eb, cb = orc.frsz2_compress(blk, l)
        assert eb[0] == exps[b] and np.array_equal(cb, codes[b * l:(b + 1) * l])


def test_l16_is_a_uint16_array(orc):
    rng = np.random.default_rng(3)
    x = rng.standard_normal(64)
    exps, codes = orc.frsz2_compress(x, 16)
    as16 = codes.view(np.uint16)
    for i in range(64):
        assert int(as16[i]) == orc.frsz2_get_code(codes, i, 16)


def test_special_values(orc):
    import workloads

    x = workloads.special_values().numpy()
    x = x[np.isfinite(x)]
    for l in LS:
        exps, codes = orc.frsz2_compress(x, l)
        out = orc.frsz2_decompress(exps, codes, x.size, l)
        for b in range(exps.size):
            seg = x[b * 32:(b + 1) * 32]
            e_max, _, dec = eq2_block(seg, l)
            assert int(exps[b]) == e_max
            assert bits_equal(out[b * 32:b * 32 + seg.size], dec[: seg.size])
