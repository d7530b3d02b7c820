"""GPU tests of the serving runtime (cbg_server_*): continuous batching of CB-GMRES solves.

Each request of a mix is also solved alone with cbgmres_solve on its own context; the served
result must be the same: status, iteration and restart counts, and the solution x bit for bit
(every kernel of the path reduces in a fixed order and sizes its grid from the device alone, so a
solve does not depend on what else runs on the GPU). Admission must respect the HBM budget and
the bypass limit, and a request with an invalid matrix must complete with CBG_ERR_BAD_MATRIX
without disturbing the others.
"""
import numpy as np
import pytest
import torch

import workloads
from parity import assert_same_decisions

pytestmark = pytest.mark.gpu

MIX = [  # (N, dim, Pe, fmt, bits, tol, restart)
    (40, 2, 10.0, "frsz2", 32, 1e-10, 30),
    (12, 3, 50.0, "fp64", 32, 1e-10, 20),
    (64, 2, 5.0, "frsz2", 21, 1e-8, 50),
    (20, 3, 80.0, "fp32", 32, 1e-10, 40),
    (30, 2, 100.0, "frsz2", 16, 1e-8, 25),
    (16, 3, 1.0, "bf16", 32, 1e-8, 30),
    (90, 2, 30.0, "fp16", 32, 1e-8, 60),
    (24, 3, 20.0, "frsz2", 32, 1e-12, 100),
    (50, 2, 60.0, "fp64", 32, 1e-12, 50),
    (10, 3, 5.0, "frsz2", 21, 1e-10, 10),
]


def make_case(cbg, N, dim, pe, fmt, bits, tol, restart, seed):
    A = workloads.convdiff(N, dim, tuple([1.0] * dim), pe, device="cuda")
    xt = workloads.uniform_vector(A.n, seed, device="cuda")
    b = cbg.spmv(A.row_ptr, A.col, A.vals, xt).clone()
    opts = cbg.default_opts(restart=restart, fmt=fmt, frsz2_bits=bits, tol=tol, max_iters=20000)
    return A, b, opts


def solve_alone(cbg, A, b, opts):
    S = cbg.Solver(A.row_ptr, A.col, A.vals, opts=opts)
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    r = S.solve(b, x)
    torch.cuda.synchronize()
    S.close()
    return x, r


def run_server(srv, n_expected, timeout_s=120.0):
    done = {}
    t_end = srv.clock() + timeout_s
    max_bytes = 0
    while len(done) < n_expected:
        for c in srv.poll():
            done[c.tag] = c
        max_bytes = max(max_bytes, srv.stats()["bytes_in_use"])
        assert srv.clock() < t_end, "server did not finish in time"
    return done, max_bytes


def test_mix_equals_alone(cbg):
    cases = [make_case(cbg, *m, seed=i) for i, m in enumerate(MIX)]
    alone = [solve_alone(cbg, A, b, o) for A, b, o in cases]
    sizes = [cbg.workspace_bytes(A.n, o) for A, _, o in cases]
    budget = int(sum(sorted(sizes)[-4:]) * 1.05)  # at most ~4 large solves resident at once
    srv = cbg.Server(budget, max_active=4, steps_per_turn=4, max_bypass=4)
    xs = []
    for i, (A, b, o) in enumerate(cases):
        x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
        xs.append(x)
        srv.submit(i, A.row_ptr, A.col, A.vals, b, x, o)
    done, max_bytes = run_server(srv, len(cases))
    torch.cuda.synchronize()
    assert max_bytes <= budget
    for i, (x_alone, r_alone) in enumerate(alone):
        c = done[i]
        assert c.status == r_alone.status, (i, c.status, r_alone.status)
        assert c.result.iters == r_alone.iters and c.result.restarts == r_alone.restarts, i
        assert c.result.converged == r_alone.converged
        assert c.result.true_rrn == r_alone.true_rrn
        assert torch.equal(xs[i], x_alone), f"request {i}: served x differs from the solve alone"
        assert c.t_submit <= c.t_admit <= c.t_done
    st = srv.stats()
    assert st["active"] == 0 and st["queued"] == 0 and st["bytes_in_use"] == 0
    srv.close()


def test_strict_fifo_and_budget(cbg):
    # max_bypass = 0: admission in submission order even when a later request would fit earlier
    sizes_N = [60, 20, 60, 20, 60, 20]
    cases = [make_case(cbg, N, 2, 10.0, "frsz2", 32, 1e-8, 30, seed=i) for i, N in enumerate(sizes_N)]
    big = max(cbg.workspace_bytes(A.n, o) for A, _, o in cases)
    srv = cbg.Server(int(big * 1.5), max_active=3, steps_per_turn=2, max_bypass=0)
    for i, (A, b, o) in enumerate(cases):
        srv.submit(i, A.row_ptr, A.col, A.vals, b, torch.zeros(A.n, dtype=torch.float64, device="cuda"), o)
    done, max_bytes = run_server(srv, len(cases))
    assert max_bytes <= int(big * 1.5)
    admits = [done[i].t_admit for i in range(len(cases))]
    assert admits == sorted(admits)
    assert all(done[i].status == 0 for i in range(len(cases)))
    srv.close()


def test_bad_matrix_and_oversize(cbg):
    good = [make_case(cbg, 30, 2, 10.0, "frsz2", 32, 1e-10, 30, seed=i) for i in range(3)]
    A, b, o = good[0]
    bad_col = A.col.clone()
    bad_col[5] = A.n + 7  # a column index outside [0, n): must be rejected before any SpMV
    srv = cbg.Server(4 * cbg.workspace_bytes(A.n, o), max_active=4, steps_per_turn=4, max_bypass=4)
    alone = [solve_alone(cbg, *g) for g in good]
    xs = []
    for i, (Ai, bi, oi) in enumerate(good):
        x = torch.zeros(Ai.n, dtype=torch.float64, device="cuda")
        xs.append(x)
        srv.submit(i, Ai.row_ptr, Ai.col, Ai.vals, bi, x, oi)
        if i == 0:
            srv.submit(99, A.row_ptr, bad_col, A.vals, b, torch.zeros(A.n, dtype=torch.float64, device="cuda"), o)
    with pytest.raises(cbg.CbgError) as e:  # a workspace larger than the whole budget
        Abig, bbig, obig = make_case(cbg, 200, 2, 10.0, "fp64", 32, 1e-8, 100, seed=9)
        srv.submit(7, Abig.row_ptr, Abig.col, Abig.vals, bbig, torch.zeros_like(bbig), obig)
    assert e.value.status == -3
    done, _ = run_server(srv, 4)
    assert done[99].status == -7
    for i in range(3):
        assert done[i].status == 0 and torch.equal(xs[i], alone[i][0])
    srv.close()


def test_many_small_requests_overlap(cbg):
    # 24 small requests, 8 slots: all complete, and the server's makespan is below the sum of the
    # requests' own latencies (their work overlapped on the device)
    cases = [make_case(cbg, 20 + (i % 5) * 6, 2, 5.0 + i, "frsz2", 32, 1e-10, 20, seed=i) for i in range(24)]
    srv = cbg.Server(sum(cbg.workspace_bytes(A.n, o) for A, _, o in cases), max_active=8, steps_per_turn=4,
                     max_bypass=8)
    t0 = srv.clock()
    for i, (A, b, o) in enumerate(cases):
        srv.submit(i, A.row_ptr, A.col, A.vals, b, torch.zeros(A.n, dtype=torch.float64, device="cuda"), o)
    done, _ = run_server(srv, len(cases))
    makespan = max(c.t_done for c in done.values()) - t0
    busy = sum(c.t_done - c.t_admit for c in done.values())
    assert all(c.status == 0 and c.result.converged for c in done.values())
    assert makespan < busy
    srv.close()


STREAMED_MIX = [  # (N, dim, Pe, fmt, bits, tol): 2.6e4 .. 6.4e4 rows, restart 100, all streamed cycles
    (30, 3, 30.0, "fp64", 32, 1e-10),
    (160, 2, 20.0, "frsz2", 32, 1e-10),
    (40, 3, 10.0, "frsz2", 21, 1e-10),
    (250, 2, 40.0, "fp32", 32, 1e-10),
]


def test_served_streamed_requests_match_oracle(cbg, orc):
    """Four requests of 26 000 to 64 000 rows with restart 100, too large for the on-chip cycle,
    served concurrently (four slots, two steps per turn, so their Arnoldi steps interleave on the
    device): each served solution must be the oracle's (iterations within 2%, the same second-pass
    and breakdown counts, ||x - x_oracle|| / ||x_oracle|| <= 1e-8, explicit residual <= tol) and bit
    for bit the same as the solve alone."""
    from concurrent.futures import ThreadPoolExecutor

    cases = []
    for i, (N, dim, pe, fmt, bits, tol) in enumerate(STREAMED_MIX):
        # b = A x_true from the oracle's SpMV on the host: the oracle and the GPU solve the same system
        Ah = workloads.convdiff(N, dim, tuple([1.0] * dim), pe)
        rp, col, vals = Ah.numpy()
        bh = orc.spmv(rp, col, vals, workloads.uniform_vector(Ah.n, 50 + i).numpy())
        o = cbg.default_opts(restart=100, fmt=fmt, frsz2_bits=bits, tol=tol, max_iters=20000)
        cases.append((Ah.to("cuda"), torch.from_numpy(bh).cuda(), o, fmt, bits, tol, bh))

    def oracle_solve(c):
        A, _, o, fmt, bits, tol, bh = c
        rp, col, vals = A.numpy()
        return orc.gmres(rp, col, vals, bh, restart=100, tol=tol, fmt=orc.FORMAT_NAMES[fmt], l=bits)

    with ThreadPoolExecutor(len(cases)) as ex:  # the oracle's C code runs outside the GIL
        refs = list(ex.map(oracle_solve, cases))
    alone = []
    for A, b, o, *_ in cases:
        S = cbg.Solver(A.row_ptr, A.col, A.vals, opts=o)
        assert S.cycle_cluster == 0  # streamed cycles
        S.close()
        alone.append(solve_alone(cbg, A, b, o))
    srv = cbg.Server(sum(cbg.workspace_bytes(A.n, o) for A, _, o, *_ in cases), max_active=4, steps_per_turn=2,
                     max_bypass=4)
    xs = []
    for i, (A, b, o, *_) in enumerate(cases):
        x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
        xs.append(x)
        srv.submit(i, A.row_ptr, A.col, A.vals, b, x, o)
    done, _ = run_server(srv, len(cases), timeout_s=300.0)
    torch.cuda.synchronize()
    srv.close()
    for i, ((A, b, o, fmt, bits, tol, bh), ref) in enumerate(zip(cases, refs)):
        c = done[i]
        assert ref.converged and c.status == 0 and c.result.converged, (i, c.status)
        xg = xs[i].cpu().numpy()
        rp, col, vals = A.numpy()
        assert orc.nrm2(bh - orc.spmv(rp, col, vals, xg)) / orc.nrm2(bh) <= tol * 1.0000001
        assert abs(c.result.iters - ref.iters) <= max(1, 0.02 * ref.iters), (i, c.result.iters, ref.iters)
        assert np.linalg.norm(xg - ref.x) / np.linalg.norm(ref.x) <= 1e-8, i
        assert_same_decisions(c.result, ref)
        assert torch.equal(xs[i], alone[i][0]), f"request {i}: served x differs from the solve alone"
        assert c.result.iters == alone[i][1].iters
