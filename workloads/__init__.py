"""Seeded synthetic inputs shaped like the paper's workloads (arXiv 2409.15468, Methodology).

This module holds only input generation: sparse matrices, vectors and request mixes. It contains
none of the method's arithmetic (no SpMV, codec, Gram-Schmidt or least squares), so that the
CUDA path and the oracle can both be fed from it without sharing any of the method's code.

The paper's matrices (11 SuiteSparse CFD matrices, Tab. 1) are not available here; these
generators stand in for them:

* ``convdiff``: the centred-difference (upwind where the mesh Peclet number exceeds 1)
  convection-diffusion operator -Laplace(u) + Pe * wind . grad(u) on the unit square or cube,
  Dirichlet boundaries eliminated, scaled by h^2 with h = 1/(N+1), unknowns ordered x-fastest.
  In 3D it is a 7-point stencil, the shape of the atmosmod* matrices (6.94 nonzeros per row).
* ``powerlaw``: a nonsymmetric random matrix with Pareto-distributed row lengths (mean ~30,
  capped at 2000), N(0,1) off-diagonals and a diagonal of 1.2 times the row's absolute sum.
* ``basis_values``: N(0,1) * 2^k values with k uniform in [-20, 20] per 32-value block, a wide
  in-block-exponent-spread stand-in for Krylov vectors (the PR02R exponent discussion).

All generators use torch only as an array library (CPU or CUDA tensors), seeded through a
``torch.Generator`` on the chosen device; the same seed on the same device gives the same input.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import torch


@dataclass
class CSR:
    """A CSR matrix: int32 row pointers and column indices, float64 values (all on one device)."""

    row_ptr: torch.Tensor
    col: torch.Tensor
    vals: torch.Tensor

    @property
    def n(self) -> int:
        return self.row_ptr.numel() - 1

    @property
    def nnz(self) -> int:
        return self.col.numel()

    def to(self, device) -> "CSR":
        return CSR(self.row_ptr.to(device), self.col.to(device), self.vals.to(device))

    def numpy(self):
        return self.row_ptr.cpu().numpy(), self.col.cpu().numpy(), self.vals.cpu().numpy()


def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    return g


def convdiff(N: int, dim: int, wind, peclet: float, device="cpu") -> CSR:
    """Convection-diffusion on an N^dim grid (see module docstring)."""
    if dim not in (2, 3):
        raise ValueError("dim must be 2 or 3")
    wind = [float(w) for w in wind]
    if len(wind) != dim:
        raise ValueError("wind needs one component per dimension")
    n = N ** dim
    h = 1.0 / (N + 1)
    idx = torch.arange(n, device=device, dtype=torch.int64)
    coord = [(idx // (N ** a)) % N for a in range(dim)]  # coord[0] is x (fastest)
    # Candidate entries in ascending column order: backward neighbours from the slowest axis,
    # the diagonal, forward neighbours from the fastest axis.
    offsets, valid, values = [], [], []
    diag = 2.0 * dim
    side = {}
    for a in range(dim):
        c = peclet * wind[a] * h  # Pe * w_a * h
        if abs(c) / 2.0 <= 1.0:  # centred differences
            back, fwd = -1.0 - c / 2.0, -1.0 + c / 2.0
        elif c > 0:  # first-order upwind, flow in +x_a
            back, fwd = -1.0 - c, -1.0
            diag += c
        else:  # first-order upwind, flow in -x_a
            back, fwd = -1.0, -1.0 + c
            diag += -c
        side[a] = (back, fwd)
    for a in reversed(range(dim)):
        offsets.append(-(N ** a))
        valid.append(coord[a] > 0)
        values.append(side[a][0])
    offsets.append(0)
    valid.append(torch.ones(n, dtype=torch.bool, device=device))
    values.append(diag)
    for a in range(dim):
        offsets.append(N ** a)
        valid.append(coord[a] < N - 1)
        values.append(side[a][1])
    off = torch.tensor(offsets, device=device, dtype=torch.int64)
    mask = torch.stack(valid, dim=1)
    cols = idx[:, None] + off[None, :]
    vals = torch.tensor(values, device=device, dtype=torch.float64).expand(n, len(values))
    counts = mask.sum(dim=1)
    row_ptr = torch.zeros(n + 1, device=device, dtype=torch.int64)
    row_ptr[1:] = torch.cumsum(counts, 0)
    col = cols[mask].to(torch.int32)
    v = vals[mask].contiguous()
    return CSR(row_ptr.to(torch.int32), col, v)


def powerlaw(n: int, seed: int = 2, device="cpu", mean_scale: float = 10.0, alpha: float = 1.5,
             max_len: int = 2000, diag_factor: float = 1.2) -> CSR:
    """Random nonsymmetric matrix with Pareto row lengths (see module docstring). Columns are
    drawn uniformly (excluding the diagonal) and duplicates within a row are dropped."""
    g = _gen(seed, device)
    u = 1.0 - torch.rand(n, generator=g, device=device, dtype=torch.float64)  # (0, 1]
    lens = torch.clamp(torch.floor(mean_scale * u.pow(-1.0 / alpha)), max=max_len).to(torch.int64)
    lens = torch.clamp(lens, max=n - 1)
    rows = torch.repeat_interleave(torch.arange(n, device=device, dtype=torch.int64), lens)
    c = torch.floor(torch.rand(rows.numel(), generator=g, device=device, dtype=torch.float64) * (n - 1))
    c = c.to(torch.int64)
    c = c + (c >= rows).to(torch.int64)  # skip the diagonal
    key = torch.unique(rows * n + c)  # sorted, duplicates dropped
    r_off, c_off = key // n, key % n
    v_off = torch.randn(key.numel(), generator=g, device=device, dtype=torch.float64)
    absrow = torch.zeros(n, device=device, dtype=torch.float64)
    absrow.index_add_(0, r_off, v_off.abs())
    diag = diag_factor * absrow
    diag = torch.where(diag == 0, torch.ones_like(diag), diag)  # an empty row keeps a unit diagonal
    dkey = torch.arange(n, device=device, dtype=torch.int64) * (n + 1)
    allkey = torch.cat([key, dkey])
    allval = torch.cat([v_off, diag])
    order = torch.argsort(allkey)
    allkey, allval = allkey[order], allval[order]
    r_all = allkey // n
    counts = torch.bincount(r_all, minlength=n)
    row_ptr = torch.zeros(n + 1, device=device, dtype=torch.int64)
    row_ptr[1:] = torch.cumsum(counts, 0)
    return CSR(row_ptr.to(torch.int32), (allkey % n).to(torch.int32), allval.contiguous())


def uniform_vector(n: int, seed: int, lo: float = -1.0, hi: float = 1.0, device="cpu") -> torch.Tensor:
    g = _gen(seed, device)
    return lo + (hi - lo) * torch.rand(n, generator=g, device=device, dtype=torch.float64)


def sin_vector(n: int, device="cpu") -> torch.Tensor:
    """s[i] = sin(i), the paper's solution vector before normalisation (Problem Selection)."""
    return torch.sin(torch.arange(n, device=device, dtype=torch.float64))


def basis_values(nvec: int, n: int, seed: int = 1, device="cpu", kmin: int = -20, kmax: int = 20) -> torch.Tensor:
    """nvec x n values N(0,1) * 2^k, k uniform in [kmin, kmax] per 32-value block."""
    g = _gen(seed, device)
    nb = (n + 31) // 32
    x = torch.randn(nvec, n, generator=g, device=device, dtype=torch.float64)
    k = torch.randint(kmin, kmax + 1, (nvec, nb), generator=g, device=device, dtype=torch.int64)
    scale = torch.pow(2.0, k.to(torch.float64)).repeat_interleave(32, dim=1)[:, :n]
    return x * scale


def basis_vector(i: int, n: int, seed: int = 1, device="cpu", kmin: int = -20, kmax: int = 20,
                 unit_norm: bool = True) -> torch.Tensor:
    """Vector i of a basis of N(0,1) * 2^k values (k uniform in [kmin, kmax] per 32-value block),
    drawn from its own stream (seed, i) so that a large basis can be generated one vector at a
    time; scaled to unit 2-norm like a Krylov vector when unit_norm is set."""
    g = _gen(seed * 1000003 + i, device)
    nb = (n + 31) // 32
    x = torch.randn(n, generator=g, device=device, dtype=torch.float64)
    k = torch.randint(kmin, kmax + 1, (nb,), generator=g, device=device, dtype=torch.int64)
    x = x * torch.pow(2.0, k.to(torch.float64)).repeat_interleave(32)[:n]
    if unit_norm:
        x = x / torch.linalg.vector_norm(x)
    return x


def special_values(device="cpu") -> torch.Tensor:
    """Hand-picked edge values: signed zeros, subnormals, the normal-range boundary, powers of
    two, values that straddle exponents, the largest finite values."""
    tiny = 2.0 ** -1022
    sub = 2.0 ** -1074
    vals = [0.0, -0.0, sub, -sub, 3 * sub, tiny, -tiny, tiny * (1 - 2 ** -52), 1.0, -1.0, 0.5, 2.0 ** -30,
            2.0 ** -31, 2.0 ** -32, 1.0 - 2 ** -53, 1.0 + 2 ** -52, math.pi, -math.e, 1e-300, -1e300,
            2.0 ** 1023, -(2.0 ** 1023) * (2 - 2 ** -52), 0.1, -0.3, 1e-5, 123456.789]
    return torch.tensor(vals, dtype=torch.float64, device=device)


@dataclass
class SolveRequest:
    """One request of the serving mix: a convection-diffusion system and its solve options."""

    rid: int
    arrival_s: float
    N: int
    dim: int
    wind: tuple
    peclet: float
    tol: float
    fmt: str
    frsz2_bits: int


def serving_mix(count: int, rate_per_s: float, seed: int = 3, n_min: float = 1e4, n_max: float = 4e6,
                formats=("fp64", "fp32", "fp16", "bf16", "frsz2_16", "frsz2_21", "frsz2_32")):
    """Poisson arrivals; n log-uniform in [n_min, n_max]; 2D or 3D with equal odds (N = round(n^(1/d)));
    Peclet uniform in [1, 100]; tol from {1e-8, 1e-10, 1e-12}; basis format uniform over ``formats``."""
    g = _gen(seed, "cpu")
    t = 0.0
    out = []
    tols = (1e-8, 1e-10, 1e-12)
    for rid in range(count):
        t += float(-math.log(1.0 - torch.rand((), generator=g, dtype=torch.float64).item()) / rate_per_s)
        logn = math.log(n_min) + (math.log(n_max) - math.log(n_min)) * torch.rand((), generator=g,
                                                                                   dtype=torch.float64).item()
        dim = 2 if torch.rand((), generator=g).item() < 0.5 else 3
        N = max(4, int(round(math.exp(logn) ** (1.0 / dim))))
        pe = 1.0 + 99.0 * torch.rand((), generator=g, dtype=torch.float64).item()
        tol = tols[int(torch.randint(0, 3, (), generator=g).item())]
        f = formats[int(torch.randint(0, len(formats), (), generator=g).item())]
        if f.startswith("frsz2_"):
            fmt, bits = "frsz2", int(f.split("_")[1])
        else:
            fmt, bits = f, 32
        wind = tuple([1.0] * dim)
        out.append(SolveRequest(rid, t, N, dim, wind, pe, tol, fmt, bits))
    return out
