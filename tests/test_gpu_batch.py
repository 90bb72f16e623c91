"""Batches: independent problems concatenated into one index space (GPU).

Every problem keeps its own material, Jv step, GMRES iteration, line search and convergence
test, and a problem's internal numbering, face order and reduction chunks are the same alone
and in a batch.  So with block-Jacobi the batched solve of each problem is bitwise the solve
of that problem alone; with the multigrid preconditioner (whose coarse levels span the batch)
they agree within the displacement tolerance.
"""
import numpy as np
import pytest

import oracle as O
from paper_2502_17217_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()


def _mix():
    sizes = I.batch_sizes(6, lo=200, hi=2000, seed=4)
    cases = [I.case_batch_member(*sz, index=k) for k, sz in enumerate(sizes)]
    cases.append(I.case_nh_beam(12, 4, 4, (1.0, 0.25, 0.25), end_uy=0.1, load_steps=1))  # mixed laws
    stvk = I.case_nh_beam(10, 3, 3, (1.0, 0.3, 0.3), end_uy=0.08, load_steps=1)
    stvk.material = I.Material(I.LAW_STVK, 3.0e6, 0.35)
    cases.append(stvk)
    return cases


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_batch_residual_and_jv_match_each_problem_alone():
    from paper_2502_17217_gb300 import jfnk
    cases = _mix()
    B = jfnk.Batch(cases)
    u = np.concatenate([I.random_field(k + 1, c.mesh.n_cells, 1e-4 if c.material.law == I.LAW_LINEAR else 0.002)
                        for k, c in enumerate(cases)])
    v = np.concatenate([I.random_field(k + 50, c.mesh.n_cells, 1.0) for k, c in enumerate(cases)])
    R = B.residual(u)
    J = B.jv(u, v)
    for k, (c, Rk, Jk, uk, vk) in enumerate(zip(cases, B.split(R), B.split(J), B.split(u), B.split(v))):
        s = jfnk.Solver.from_case(c)
        assert np.array_equal(Rk, s.residual(uk)), k
        assert np.array_equal(Jk, s.jv(uk, vk)), k  # eps from this problem's norms only
        o = O.Oracle.from_case(c)
        assert _rel(Rk, o.residual(uk)) <= 1e-12


@pytest.mark.parametrize("pc_side", [0, 1])
def test_batch_solve_bitwise_equals_alone_with_block_jacobi(pc_side):
    from paper_2502_17217_gb300 import jfnk
    cases = _mix()
    B = jfnk.Batch(cases, pc=jfnk.PC_BJACOBI, newton_rtol=1e-10, pc_side=pc_side)
    u, st, rc = B.solve()
    assert rc == 0
    per = B.problem_stats()
    for k, (c, uk) in enumerate(zip(cases, B.split(u))):
        s = jfnk.Solver.from_case(c, pc=jfnk.PC_BJACOBI, newton_rtol=1e-10, pc_side=pc_side)
        ua, sta, rca = s.solve()
        assert rca == 0
        assert np.array_equal(uk, ua), (k, _rel(uk, ua))
        assert per[k].gmres_its == sta.gmres_its and per[k].newton_its == sta.newton_its


@pytest.mark.parametrize("sell", [0, 1])
def test_batch_solve_within_tolerance_with_multigrid_mixed_precision(sell, monkeypatch):
    """Batched mixed-precision multigrid solves agree with each problem solved alone and are
    the oracle's discrete solution; sell = 1 runs the coarse levels and restrictions in
    sliced-ELL form (JFNK_MG_SELL_MIN_ROWS=0), on the batch and on each problem alone."""
    from paper_2502_17217_gb300 import jfnk
    if sell:
        monkeypatch.setenv("JFNK_MG_SELL_MIN_ROWS", "0")
    cases = _mix()
    kw = dict(pc=jfnk.PC_MG, precision=jfnk.PREC_MIXED, newton_rtol=1e-11, mg_coarse_max=50)
    B = jfnk.Batch(cases, **kw)
    u, st, rc = B.solve()
    assert rc == 0
    for k, (c, uk) in enumerate(zip(cases, B.split(u))):
        ua, _, rca = jfnk.Solver.from_case(c, **kw).solve()
        assert rca == 0
        assert _rel(uk, ua) <= 1e-8, (k, _rel(uk, ua))
        # and the batched result is the discrete solution: the oracle's residual is small
        o = O.Oracle.from_case(c)
        R = o.residual(uk)
        R0 = o.residual(np.zeros_like(uk))
        assert np.linalg.norm(R) <= 1e-9 * np.linalg.norm(R0)


def test_batch_segregated_bitwise_equals_alone():
    """The segregated solver's per-component CG scalars are per problem too: a batched
    segregated solve gives each problem exactly its solve alone (block-Jacobi)."""
    from paper_2502_17217_gb300 import jfnk
    cases = _mix()
    B = jfnk.Batch(cases, pc=jfnk.PC_BJACOBI, newton_rtol=1e-9)
    u, st, rc = B.solve_segregated()
    assert rc == 0
    for k, (c, uk, ps) in enumerate(zip(cases, B.split(u), B.problem_stats())):
        ua, sta, rca = jfnk.Solver.from_case(c, pc=jfnk.PC_BJACOBI, newton_rtol=1e-9).solve_segregated()
        assert rca == 0
        assert np.array_equal(uk, ua), k
        assert ps.newton_its == sta.newton_its and ps.gmres_its == sta.gmres_its


@pytest.mark.parametrize("pc", ["mg_mixed", "mg_mixed_sell", "bjacobi_left"])
def test_skipping_problems_out_of_the_iteration_changes_no_bit(pc, monkeypatch):
    """In a batch, the problems whose Krylov cycle is done (or that left the Newton iteration)
    skip the residual passes and the V-cycle of each Arnoldi iteration: compacted launches
    over the rows of the problems that run, which get the same arithmetic.  Solves with
    skipping (the default) and without it (JFNK_SKIP_DONE=0, read when a context is created)
    are bitwise equal, with the same iteration counts, for the multigrid in mixed precision
    (coarse levels as lane-group CSR, or all in sliced-ELL form with JFNK_MG_SELL_MIN_ROWS=0)
    and for left-preconditioned block-Jacobi."""
    from paper_2502_17217_gb300 import jfnk
    cases = _mix()
    if pc == "mg_mixed_sell":
        monkeypatch.setenv("JFNK_MG_SELL_MIN_ROWS", "0")
    if pc.startswith("mg_mixed"):
        kw = dict(pc=jfnk.PC_MG, precision=jfnk.PREC_MIXED, newton_rtol=1e-10, mg_coarse_max=50)
    else:
        kw = dict(pc=jfnk.PC_BJACOBI, newton_rtol=1e-10, pc_side=jfnk.PC_LEFT)
    out = []
    for flag in ("1", "0"):
        monkeypatch.setenv("JFNK_SKIP_DONE", flag)
        B = jfnk.Batch(cases, **kw)
        u, st, rc = B.solve()
        assert rc == 0
        out.append((u, [(p.gmres_its, p.newton_its, p.jv_products) for p in B.problem_stats()]))
        B.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1]
    # the problems converge at different iteration counts, so some did sit out iterations
    assert len({its for its, _, _ in out[0][1]}) > 1
