"""GPU parity at the workloads' full sizes, in the launch configuration the benchmark times
(multigrid FP32 V-cycle, FP32 Krylov basis, autotuned launch shapes).

  * the 80,000-cell cantilever (200x20x20, +-15 % node perturbation, seed 2): residual and Jv
    element by element against the oracle, and one complete Newton-Krylov solve against the
    oracle's solve with the same multigrid options;
  * the 262,144-cell neo-Hookean beam (256x32x32) at mid-ramp (load factor 0.5, a bending field
    with the prescribed end displacement, finite strain): residual and Jv;
  * the 512-box batch (7.6 M cells in one index space): the batch's residual, Jv and solve,
    with members sampled (the largest, the smallest, seeded others) compared with the oracle
    run on each member alone.

Tolerances are those of the parity tests: residual 1e-12 relative at generic u; Jv
1e-12 (|R(u)| / (eps |Jv|) + 1), the finite-difference amplification of the residual's round-off
difference; solutions 1e-8 relative (both sides stop at |R| <= 1e-8 |R0|, where the oracle's
iterate lies within 2e-10 of the round-off floor on the cantilever).
"""
import numpy as np
import pytest

import oracle as O
from paper_2502_17217_gb300 import inputs as I

pytestmark = pytest.mark.gpu

MG_FP32 = dict(theta=0.4, coarse_max=1000, smoothed=True, sweeps=2)


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


def _bench_opts():
    from paper_2502_17217_gb300 import jfnk
    return dict(pc=jfnk.PC_MG, precision=jfnk.PREC_MIXED, newton_rtol=1e-8, gmres_restart=30, gmres_eta=1e-3)


def _jv_tol(R, Jv, u, v):
    eps = 1e-7 * (1 + np.linalg.norm(u)) / np.linalg.norm(v)
    return 1e-12 * (np.linalg.norm(R) / (eps * np.linalg.norm(Jv)) + 1.0)


def _check_residual_and_jv(s, o, u, v):
    R, Ro = s.residual(u), o.residual(u)
    assert _rel(R, Ro) <= 1e-12, _rel(R, Ro)
    J, Jo = s.jv(u, v), o.jv(u, v, R_u=Ro)
    tol = _jv_tol(Ro, Jo, u, v)
    assert _rel(J, Jo) <= tol, (_rel(J, Jo), tol)


def test_cantilever_80k_residual_and_jv():
    from paper_2502_17217_gb300 import jfnk
    case = I.case_cantilever(200, 20, 20, (1.0, 0.1, 0.1), perturb=0.15, seed=2)
    s = jfnk.Solver.from_case(case, **_bench_opts())
    s.setup()
    o = O.Oracle.from_case(case)
    n = case.mesh.n_cells
    for seed in (1, 2):
        _check_residual_and_jv(s, o, I.random_field(seed, n, 1e-4), I.random_field(seed + 10, n, 1.0))


def _mid_ramp_field(case, lam):
    """Bending of the beam toward the prescribed end displacement lam * end_uy (zero slope at
    both ends, as for a clamped x-min and a translated x-max), plus a seeded perturbation."""
    x = case.mesh.nominal_cell_centres()
    L = case.mesh.points[:, 0].max()
    xi = x[:, 0] / L
    end_uy = case.mesh.patch("xmax").values[0, 1]
    u = np.zeros((case.mesh.n_cells, 3))
    u[:, 1] = lam * end_uy * (3 * xi ** 2 - 2 * xi ** 3)
    return u + I.random_field(7, case.mesh.n_cells, 2e-4)


def test_neo_hookean_beam_262k_residual_and_jv_at_mid_ramp():
    from paper_2502_17217_gb300 import jfnk
    case = I.case_nh_beam()
    s = jfnk.Solver.from_case(case, **_bench_opts())
    s.setup()
    o = O.Oracle.from_case(case)
    s.set_load_factor(0.5)
    o.set_load_factor(0.5)
    u = _mid_ramp_field(case, 0.5)
    _check_residual_and_jv(s, o, u, I.random_field(8, case.mesh.n_cells, 1.0))


def test_cantilever_80k_solve_against_the_oracle():
    """The benchmark's solve (multigrid FP32, FP32 basis, loose GMRES(30, 2)) against the
    oracle's FP64 solve with the same hierarchy options, both to |R| <= 1e-8 |R0|."""
    from paper_2502_17217_gb300 import jfnk
    case = I.case_cantilever(200, 20, 20, (1.0, 0.1, 0.1), perturb=0.15, seed=2)
    s = jfnk.Solver.from_case(case, **_bench_opts())
    ug, st, rc = s.solve()
    assert rc == 0 and st.final_rel_res <= 1e-8
    o = O.Oracle.from_case(case)
    o.mg_setup(**MG_FP32)
    uo, rco, sto = o.newton(rtol=1e-8, pc=O.PC_MG, m=30, aug=s.options.gmres_aug)
    assert rco == 0
    assert _rel(ug, uo) <= 1e-8, _rel(ug, uo)


@pytest.fixture(scope="module")
def c4_batch():
    from paper_2502_17217_gb300 import jfnk
    members = I.batch_sizes()
    cases = [I.case_batch_member(*x, index=k) for k, x in enumerate(members)]
    b = jfnk.Batch(cases, **_bench_opts())
    b.setup()
    sizes = np.array(b.sizes)
    order = np.argsort(sizes, kind="stable")
    rng = I.splitmix64_uniform(41, 3, key=3)
    sample = sorted({int(order[-1]), int(order[0]), *(int(r * len(cases)) for r in rng)})
    return b, cases, sample


def test_batch_512_residual_and_jv_members_against_the_oracle(c4_batch):
    b, cases, sample = c4_batch
    n = b.nc
    u = I.random_field(3, n, 1e-4)
    v = I.random_field(4, n, 1.0)
    R, J = b.residual(u), b.jv(u, v)
    for p in sample:
        lo, hi = b.offsets[p], b.offsets[p + 1]
        o = O.Oracle.from_case(cases[p])
        Ro = o.residual(u[lo:hi])
        assert _rel(R[lo:hi], Ro) <= 1e-12, (p, _rel(R[lo:hi], Ro))
        Jo = o.jv(u[lo:hi], v[lo:hi], R_u=Ro)  # each member's own eps from its own u and v
        tol = _jv_tol(Ro, Jo, u[lo:hi], v[lo:hi])
        assert _rel(J[lo:hi], Jo) <= tol, (p, _rel(J[lo:hi], Jo), tol)


def test_batch_512_solve_members_against_the_oracle(c4_batch):
    b, cases, _ = c4_batch
    ug, st, rc = b.solve()
    assert rc == 0
    ps = b.problem_stats()
    assert all(q.status == 0 and q.final_rel_res <= 1e-8 for q in ps)
    sizes = np.array(b.sizes)
    order = np.argsort(sizes, kind="stable")
    # the oracle solves the two smallest members and one near 8k cells (seconds each)
    near8k = int(np.argmin(np.abs(sizes - 8000)))
    for p in sorted({int(order[0]), int(order[1]), near8k}):
        o = O.Oracle.from_case(cases[p])
        o.mg_setup(**MG_FP32)
        uo, rco, _ = o.newton(rtol=1e-8, pc=O.PC_MG, m=30, aug=b.options.gmres_aug)
        assert rco == 0
        lo, hi = b.offsets[p], b.offsets[p + 1]
        assert _rel(ug[lo:hi], uo) <= 1e-8, (p, sizes[p], _rel(ug[lo:hi], uo))
