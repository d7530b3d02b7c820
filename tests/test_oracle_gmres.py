"""Pins of the oracle's CB-GMRES (Fig. 1) and its FP64 building blocks against LAPACK, closed-form
special cases and textbook invariants: the exact solution after n steps on small dense systems,
one step for A = I, at most k steps for k distinct eigenvalues, the Arnoldi relation, the
orthogonality of an FP64 basis, the monotone minimal residual, and the implicit residual matching
the explicit one at each restart for the FP64 basis."""
import math
from fractions import Fraction

import numpy as np
import pytest

import workloads


def dense_to_csr(A):
    n = A.shape[0]
    row_ptr = [0]
    col, vals = [], []
    for i in range(n):
        for j in range(n):
            if A[i, j] != 0.0:
                col.append(j)
                vals.append(A[i, j])
        row_ptr.append(len(col))
    return np.array(row_ptr, np.int32), np.array(col, np.int32), np.array(vals)


def csr_to_dense(rp, col, vals):
    n = rp.size - 1
    A = np.zeros((n, n))
    for i in range(n):
        for p in range(rp[i], rp[i + 1]):
            A[i, col[p]] += vals[p]
    return A


def test_dot_and_dot2_exact(orc):
    rng = np.random.default_rng(1)
    for n in (1, 7, 100, 1000):
        a = rng.standard_normal(n) * np.exp2(rng.integers(-30, 30, n))
        b = rng.standard_normal(n)
        exact = sum(Fraction(x) * Fraction(y) for x, y in zip(a, b))
        s_abs = float(sum(abs(Fraction(x) * Fraction(y)) for x, y in zip(a, b)))
        u = 2.0 ** -53
        assert abs(Fraction(orc.dot(a, b)) - exact) <= n * u / (1 - n * u) * s_abs
        # compensated dot: as accurate as twice the working precision, then rounded
        assert abs(Fraction(orc.dot2(a, b)) - exact) <= u * abs(exact) + (n * u) ** 2 / (1 - n * u) ** 2 * s_abs * 2
    assert orc.nrm2(np.array([3.0, 4.0])) == 5.0
    a = rng.standard_normal(50)
    x = rng.standard_normal(50)
    y = rng.standard_normal(50)
    y0 = y.copy()
    orc.axpy(-0.5, x, y)
    for k in range(50):  # alpha x is exact for alpha = -1/2, so y + alpha x is rounded once
        prod = Fraction(-1, 2) * Fraction(x[k])
        exact = Fraction(y0[k]) + prod
        assert abs(Fraction(y[k]) - exact) <= 2.0 ** -53 * abs(exact)


def test_spmv_matches_dense(orc):
    A = workloads.convdiff(6, 2, (1.0, 0.5), 10.0)
    rp, col, vals = A.numpy()
    D = csr_to_dense(rp, col, vals)
    x = np.random.default_rng(2).standard_normal(A.n)
    y = orc.spmv(rp, col, vals, x)
    exact = [sum(Fraction(D[i, j]) * Fraction(x[j]) for j in range(A.n)) for i in range(A.n)]
    for i in range(A.n):
        assert abs(Fraction(y[i]) - exact[i]) <= 8 * 2.0 ** -53 * float(sum(abs(Fraction(D[i, j]) * Fraction(x[j])) for j in range(A.n)))


def test_convdiff_shape(orc):
    A2 = workloads.convdiff(64, 2, (1.0, 0.5), 10.0)
    assert A2.n == 4096 and A2.nnz == 5 * 64 ** 2 - 4 * 64 == 20224
    A3 = workloads.convdiff(8, 3, (1.0, 1.0, 1.0), 10.0)
    assert A3.nnz == 7 * 8 ** 3 - 6 * 8 ** 2
    D = csr_to_dense(*A3.numpy())
    h = 1.0 / 9
    # interior row, mesh Peclet 10 h / 2 < 1: diagonal 6, neighbours -1 -+ Pe w h / 2 (centred)
    i = 1 + 8 * (1 + 8 * 1)
    assert D[i, i] == 6.0
    assert math.isclose(D[i, i - 1], -1 - 10 * h / 2) and math.isclose(D[i, i + 1], -1 + 10 * h / 2)
    assert math.isclose(D[i, i - 64], -1 - 10 * h / 2) and math.isclose(D[i, i + 64], -1 + 10 * h / 2)
    # mesh Peclet above 1: first-order upwind (flow in +x: the backward neighbour takes Pe w h)
    Du = csr_to_dense(*workloads.convdiff(8, 3, (1.0, 1.0, 1.0), 50.0).numpy())
    assert math.isclose(Du[i, i], 6.0 + 3 * 50 * h)
    assert math.isclose(Du[i, i - 1], -1 - 50 * h) and Du[i, i + 1] == -1.0
    rp, col, _ = A3.numpy()
    for r in range(A3.n):
        assert np.all(np.diff(col[rp[r]:rp[r + 1]]) > 0)  # sorted columns


@pytest.mark.parametrize("n", [1, 2, 5, 8, 12])
def test_small_dense_vs_lapack(orc, n):
    rng = np.random.default_rng(100 + n)
    A = rng.standard_normal((n, n)) + n * np.eye(n)
    b = rng.standard_normal(n)
    rp, col, vals = dense_to_csr(A)
    r = orc.gmres(rp, col, vals, b, restart=max(n, 1), tol=1e-15, max_iters=4 * n + 4, fmt=orc.FP64)
    x_lu = np.linalg.solve(A, b)
    kappa = np.linalg.cond(A)
    # the exact solution is in the Krylov space after n steps (Background section)
    assert np.linalg.norm(r.x - x_lu) / np.linalg.norm(x_lu) <= 1e3 * kappa * 2.0 ** -53
    assert r.iters <= 2 * n + 1


def test_identity_one_step(orc):
    n = 50
    rp, col, vals = np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), np.ones(n)
    b = np.random.default_rng(3).standard_normal(n)
    r = orc.gmres(rp, col, vals, b, restart=10, tol=1e-12, fmt=orc.FP64)
    assert r.converged and r.iters == 1
    # a compressed basis reads x back through the codec: one cycle gains the code's ~30 bits
    r = orc.gmres(rp, col, vals, b, restart=10, tol=1e-12, fmt=orc.FRSZ2, l=32)
    assert r.converged and r.iters == 2 and r.hist_implicit[0] < 2.0 ** -28


@pytest.mark.parametrize("k", [1, 2, 3, 5])
def test_distinct_eigenvalues(orc, k):
    n = 60
    ev = np.arange(1, k + 1, dtype=np.float64)
    d = ev[np.arange(n) % k]
    rp, col = np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32)
    b = np.random.default_rng(4).standard_normal(n)
    r = orc.gmres(rp, col, d, b, restart=20, tol=1e-13, fmt=orc.FP64)
    assert r.converged and r.iters <= k
    assert np.allclose(r.x, b / d, rtol=1e-12, atol=0)


def _c1_small(N=16):
    A = workloads.convdiff(N, 2, (1.0, 0.5), 10.0)
    return A.numpy()


def test_arnoldi_relation_and_orthogonality_fp64(orc):
    rp, col, vals = _c1_small()
    n = rp.size - 1
    D = csr_to_dense(rp, col, vals)
    b = orc.spmv(rp, col, vals, workloads.uniform_vector(n, 0).numpy())
    m = 30
    m_eff, V, Vh, H, beta = orc.arnoldi_cycle(rp, col, vals, b, restart=m, fmt=orc.FP64)
    assert m_eff == m
    assert np.array_equal(V, Vh)  # fp64 storage is lossless
    # A V_m = V_{m+1} Hbar_m (Arnoldi relation)
    res = D @ V[:m].T - V[: m + 1].T @ H[: m + 1, :m]
    assert np.linalg.norm(res) / np.linalg.norm(D) <= 1e-13
    assert np.linalg.norm(np.eye(m + 1) - V[: m + 1] @ V[: m + 1].T) <= 1e-12
    assert np.all(np.diag(H, -1)[:m] > 0)
    assert np.allclose(np.tril(H[: m + 1, :m], -2), 0)  # upper Hessenberg


@pytest.mark.parametrize("fmt,l", [(1, 32), (2, 32), (3, 32), (4, 16), (4, 21), (4, 32)])
def test_arnoldi_relation_compressed(orc, fmt, l):
    """Compressed bases: A v_j = sum_i vhat_i h_ij + h_{j+1,j} v_{j+1} with the FP64 v on the left
    and in the last term, and the decoded basis in the Gram-Schmidt terms (Fig. 1 steps 3-13)."""
    rp, col, vals = _c1_small()
    n = rp.size - 1
    D = csr_to_dense(rp, col, vals)
    b = orc.spmv(rp, col, vals, workloads.uniform_vector(n, 0).numpy())
    m = 25
    m_eff, V, Vh, H, beta = orc.arnoldi_cycle(rp, col, vals, b, restart=m, fmt=fmt, l=l)
    assert m_eff == m
    for j in range(m):
        lhs = D @ V[j]
        rhs = Vh[: j + 1].T @ H[: j + 1, j] + H[j + 1, j] * V[j + 1]
        assert np.linalg.norm(lhs - rhs) <= 1e-13 * (np.linalg.norm(D) + np.abs(H[: j + 2, j]).sum())
    # the stored basis is the oracle codec applied to the FP64 vectors
    for j in range(m + 1):
        vals_j, exps_j = orc.encode(V[j], fmt, l)
        assert np.array_equal(orc.decode(vals_j, exps_j, n, fmt, l), Vh[j])


def test_monotone_residual_and_implicit_matches_explicit(orc):
    rp, col, vals = _c1_small(24)
    n = rp.size - 1
    b = orc.spmv(rp, col, vals, workloads.uniform_vector(n, 0).numpy())
    m = 15
    r = orc.gmres(rp, col, vals, b, restart=m, tol=1e-11, fmt=orc.FP64, max_iters=5000)
    assert r.converged
    hi, ht = r.hist_implicit, r.hist_true
    # minimal residual: non-increasing within a cycle and at the restarts
    for c in range(r.restarts):
        seg = hi[c * m:(c + 1) * m]
        assert np.all(np.diff(seg) <= 1e-15 * seg[:-1] + 1e-300)
    assert np.all(np.diff(ht) <= 1e-14)
    # implicit residual at the end of a cycle equals the explicit one at the next restart (fp64)
    for c in range(r.restarts):
        last = hi[min((c + 1) * m, r.iters) - 1]
        assert abs(last - ht[c + 1]) <= 1e-12


@pytest.mark.parametrize("fmt,l", [(0, 32), (1, 32), (2, 32), (3, 32), (4, 16), (4, 21), (4, 32)])
def test_c1_converges_all_formats(orc, fmt, l):
    """The 64x64 convection-diffusion system (wind (1,0.5), Peclet 10, b = A x_true) reaches 1e-10
    in every storage format; FRSZ2-32 and fp32 need no more iterations than fp16 (Evaluation)."""
    rp, col, vals = _c1_small(64)
    n = rp.size - 1
    xt = workloads.uniform_vector(n, 0).numpy()
    b = orc.spmv(rp, col, vals, xt)
    r = orc.gmres(rp, col, vals, b, restart=50, tol=1e-10, fmt=fmt, l=l)
    assert r.converged and r.true_rrn <= 1e-10
    assert np.linalg.norm(r.x - xt) / np.linalg.norm(xt) < 1e-6


def test_zero_rhs_and_exact_start(orc):
    rp, col, vals = _c1_small(8)
    n = rp.size - 1
    r = orc.gmres(rp, col, vals, np.zeros(n), restart=5, tol=1e-10)
    assert r.converged and r.iters == 0 and not r.x.any()
    xt = np.ones(n)
    b = orc.spmv(rp, col, vals, xt)
    r = orc.gmres(rp, col, vals, b, x0=xt, restart=5, tol=1e-10)
    assert r.converged and r.iters == 0


# ---- Jacobi preconditioner (Fig. 1 steps 3 and 17 with M = diag(A), applied on the right) -------

def test_jacobi_diagonal_matrix_one_step(orc):
    """A diagonal: A M^{-1} = I, so right-preconditioned GMRES converges in one step (without it, in
    as many steps as A has distinct eigenvalues)."""
    n = 60
    d = 1.0 + np.arange(n) % 5
    rp, col = np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32)
    b = np.random.default_rng(5).standard_normal(n)
    r = orc.gmres(rp, col, d, b, restart=20, tol=1e-13, fmt=orc.FP64, precond="jacobi")
    assert r.converged and r.iters == 1
    assert np.allclose(r.x, b / d, rtol=1e-13, atol=0)
    r0 = orc.gmres(rp, col, d, b, restart=20, tol=1e-13, fmt=orc.FP64)
    assert r0.iters == 5


@pytest.mark.parametrize("n", [3, 8, 12])
def test_jacobi_small_dense_vs_lapack(orc, n):
    rng = np.random.default_rng(200 + n)
    A = rng.standard_normal((n, n)) + np.diag(np.linspace(n, 20 * n, n))
    b = rng.standard_normal(n)
    rp, col, vals = dense_to_csr(A)
    r = orc.gmres(rp, col, vals, b, restart=n, tol=1e-15, max_iters=4 * n + 4, fmt=orc.FP64, precond="jacobi")
    x_lu = np.linalg.solve(A, b)
    assert np.linalg.norm(r.x - x_lu) / np.linalg.norm(x_lu) <= 1e3 * np.linalg.cond(A) * 2.0 ** -53


def test_jacobi_is_right_preconditioning(orc):
    """Right preconditioning: GMRES with M on A produces the iterates of plain GMRES on A M^{-1}
    mapped back by x = M^{-1} y (the residual b - A x is the same vector). So the iteration counts
    agree and the solutions agree to rounding; left preconditioning would minimise a different
    residual and fail this."""
    A = workloads.powerlaw(400, seed=7)
    rp, col, vals = A.numpy()
    D = csr_to_dense(rp, col, vals)
    d = np.diag(D).copy()
    b = np.random.default_rng(8).standard_normal(A.n)
    rj = orc.gmres(rp, col, vals, b, restart=15, tol=1e-12, fmt=orc.FP64, precond="jacobi")
    rp2, col2, vals2 = dense_to_csr(D / d[None, :])
    r2 = orc.gmres(rp2, col2, vals2, b, restart=15, tol=1e-12, fmt=orc.FP64)
    assert rj.converged and r2.converged
    assert rj.iters == r2.iters
    assert np.linalg.norm(rj.x - r2.x / d) / np.linalg.norm(rj.x) <= 1e-10
    # and the preconditioner helps here: the row sums vary over orders of magnitude
    r0 = orc.gmres(rp, col, vals, b, restart=15, tol=1e-12, fmt=orc.FP64)
    assert rj.iters < r0.iters


def test_jacobi_zero_diagonal_rejected(orc):
    rp = np.array([0, 1, 2], np.int32)
    col = np.array([1, 0], np.int32)
    with pytest.raises(ValueError):
        orc.gmres(rp, col, np.array([1.0, 1.0]), np.ones(2), restart=2, precond="jacobi")


# ---- The second Gram-Schmidt pass (Fig. 1 steps 7-11) and the breakdown exit (step 12, R10) -----
# Hand-derived cases: every quantity below is worked out by hand from Fig. 1, so the counts the
# oracle reports are fixed by the paper's algorithm, not by the oracle.

ETA = 1.0 / math.sqrt(2.0)


def dyadic_case():
    """A = diag(1, 1, 1/8, 1/8), b = (1, 1, 1, 1). All Arnoldi quantities are dyadic rationals:
      step 1: v1 = (1,1,1,1)/2; w = A v1 = (1/2, 1/2, 1/16, 1/16), omega = sqrt(65/128);
              h11 = v1.w = 9/16; w - h11 v1 = (7/32)(1, 1, -1, -1), ||w|| = 7/16 = 0.614 omega
              < eta omega (eta = 1/sqrt 2; but > eta^2 omega): the second pass runs, V^T w = 0,
              so h and ||w|| = 7/16 are unchanged and it is no breakdown (7/16 is not below
              eta * 7/16);
      step 2: v2 = w / (7/16) = (1, 1, -1, -1)/2; A v2 = (1/2, 1/2, -1/16, -1/16); h12 = 7/16,
              h22 = 9/16 and w - h12 v1 - h22 v2 = 0 exactly: ||w|| = 0 < eta omega, a second pass,
              and h_{3,2} = 0: a breakdown.
    Two distinct eigenvalues: the Krylov space is invariant after two steps and x = (1, 1, 8, 8)."""
    rp = np.arange(5, dtype=np.int32)
    col = np.arange(4, dtype=np.int32)
    vals = np.array([1.0, 1.0, 0.125, 0.125])
    return rp, col, vals, np.ones(4)


@pytest.mark.parametrize("fmt,l", [(0, 32), (4, 32), (4, 16), (1, 32)])
def test_second_pass_and_breakdown_hand_derived(orc, fmt, l):
    # every value of this case (v_1, v_2 = +-1/2) is stored exactly by each of these formats
    rp, col, vals, b = dyadic_case()
    r = orc.gmres(rp, col, vals, b, restart=4, tol=1e-14, fmt=fmt, l=l)
    assert r.converged and not r.stagnated
    assert (r.iters, r.reorths, r.breakdowns, r.restarts) == (2, 2, 1, 1)
    assert np.allclose(r.x, [1.0, 1.0, 8.0, 8.0], rtol=1e-14, atol=0)
    m_eff, V, Vh, H, beta = orc.arnoldi_cycle(rp, col, vals, b, restart=4, fmt=fmt, l=l)
    assert m_eff == 2 and beta == 2.0
    assert np.array_equal(V[0], [0.5, 0.5, 0.5, 0.5]) and np.array_equal(V[1], [0.5, 0.5, -0.5, -0.5])
    assert H[0, 0] == 9 / 16 and H[1, 0] == 7 / 16 and H[0, 1] == 7 / 16 and H[1, 1] == 9 / 16
    assert H[2, 1] == 0.0


def test_no_second_pass_when_av_is_orthogonal_to_v(orc):
    """A = [[0, 1], [-1, 0]] turns every vector by 90 degrees: A v is orthogonal to v, so the first
    pass leaves ||w|| = omega, never below eta omega: no second pass at any step. With restart 1
    (the minimal-residual iteration) the step length (r, A r) / (A r, A r) is 0: x stays 0, the
    residual stays ||b||, and no step breaks down."""
    rp = np.array([0, 1, 2], dtype=np.int32)
    col = np.array([1, 0], dtype=np.int32)
    vals = np.array([1.0, -1.0])
    r = orc.gmres(rp, col, vals, np.array([1.0, 0.0]), restart=1, tol=1e-12, max_iters=5)
    assert (r.iters, r.reorths, r.breakdowns, r.restarts) == (5, 0, 0, 5)
    assert not r.converged and not r.stagnated
    assert not r.x.any() and r.true_rrn == 1.0


def test_breakdown_without_progress_stops(orc):
    """A = [[0, 1], [0, 0]], b = (0, 1): A x = b has no solution. v1 = (0, 1), A v1 = (1, 0) is
    orthogonal to v1 (h11 = 0, ||w|| = omega = 1: no second pass); v2 = (1, 0), A v2 = 0:
    omega = 0, h_{3,2} = 0 (no second pass either: 0 < eta * 0 is false), a breakdown. The
    rotated R has a zero pivot in column 2 and the rotated g_1 = 0, so y = 0 and x = 0: the next
    restart's residual equals the one the cycle started from, and the solve stops there (R18)
    instead of repeating the cycle: 2 iterations, 1 cycle, 1 breakdown."""
    rp = np.array([0, 1, 1], dtype=np.int32)
    col = np.array([1], dtype=np.int32)
    vals = np.array([1.0])
    r = orc.gmres(rp, col, vals, np.array([0.0, 1.0]), restart=2, tol=1e-12, max_iters=100)
    assert r.stagnated and not r.converged
    assert (r.iters, r.reorths, r.breakdowns, r.restarts) == (2, 0, 1, 1)
    assert not r.x.any() and r.true_rrn == 1.0
