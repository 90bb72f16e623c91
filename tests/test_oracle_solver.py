"""Oracle pins: mechanical laws (App. B), Jv (Eq. JF), J~ (Sec. 3.1), GMRES, Newton (Sec. 3.2-3.3),
multigrid (structure only: parity unpinned beyond these properties)."""
import numpy as np
import pytest

import oracle as O
from paper_2502_17217_gb300 import inputs as I


def _rot(rng):
    q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    return q * np.sign(np.linalg.det(q))


def _one_cell_oracle(law, p1, p2):
    m = I.hex_box(2, 2, 2)
    return O.Oracle(m, I.Material(law, p1, p2))


def test_neo_hookean_small_strain_limit_is_hooke():
    """App. B: for |grad u| << 1 the neo-Hookean law reduces to linear elasticity."""
    mu, kappa = 0.38e6, 8.3e6
    lam = kappa - 2 * mu / 3
    o = _one_cell_oracle(I.LAW_NEOHOOKEAN, mu, kappa)
    rng = np.random.default_rng(1)
    G0 = rng.standard_normal((3, 3))
    for t in (1e-4, 1e-5, 1e-6):
        G = t * G0
        s = o.cauchy_stress(G)
        hooke = mu * (G + G.T) + lam * np.trace(G) * np.eye(3)
        err = np.abs(s - hooke).max() / np.abs(hooke).max()
        assert err < 20 * t  # first-order agreement


def test_neo_hookean_objectivity_and_rotation():
    mu, kappa = 1.0e6, 5.0e6
    o = _one_cell_oracle(I.LAW_NEOHOOKEAN, mu, kappa)
    rng = np.random.default_rng(2)
    F = np.eye(3) + 0.3 * rng.standard_normal((3, 3))
    assert np.linalg.det(F) > 0
    Q = _rot(rng)
    s = o.cauchy_stress((F - np.eye(3)).T)
    s_rot = o.cauchy_stress((Q @ F - np.eye(3)).T)
    np.testing.assert_allclose(s_rot, Q @ s @ Q.T, atol=1e-8 * np.abs(s).max())
    np.testing.assert_allclose(s, s.T, atol=1e-9 * np.abs(s).max())
    # a pure rotation is stress free
    s0 = o.cauchy_stress((Q - np.eye(3)).T)
    assert np.abs(s0).max() < 1e-9 * mu
    # pure dilatation J: sigma = kappa/2 (J^2 - 1)/J I
    J = 1.2
    sd = o.cauchy_stress((J ** (1 / 3) - 1) * np.eye(3))
    np.testing.assert_allclose(sd, 0.5 * kappa * (J * J - 1) / J * np.eye(3), rtol=1e-12, atol=1e-6)


def test_total_lagrangian_traction_operator():
    """App. A: (J F^-T n) . sigma = n . T with T = J F^-1 sigma, checked against the first
    Piola-Kirchhoff stress P = J sigma F^-T (P^T n)."""
    o = _one_cell_oracle(I.LAW_NEOHOOKEAN, 1e6, 4e6)
    rng = np.random.default_rng(3)
    G = 0.2 * rng.standard_normal((3, 3))
    F = np.eye(3) + G.T
    grad = np.broadcast_to(G, (8, 3, 3)).copy()
    T = o.traction_operator(grad)[0]
    s = o.cauchy_stress(G)
    Pk = np.linalg.det(F) * s @ np.linalg.inv(F).T
    n = rng.standard_normal(3)
    np.testing.assert_allclose(n @ T, Pk @ n, rtol=1e-12)


def _fd_jacobian(o, u, h):
    n = u.size
    J = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n); e[j] = h
        J[:, j] = (o.residual((u.ravel() + e).reshape(u.shape)) - o.residual((u.ravel() - e).reshape(u.shape))).ravel() / (2 * h)
    return J


def test_jv_matches_bruteforce_fd_jacobian_linear():
    c = I.case_cantilever(4, 3, 3, (0.4, 0.3, 0.3), perturb=0.15, seed=2)  # 36 cells
    o = O.Oracle.from_case(c)
    u = I.random_field(1, c.mesh.n_cells, 1e-5)
    K = _fd_jacobian(o, u, 1e-6)  # exact up to round-off: R is affine
    for seed in (3, 4):
        v = I.random_field(seed, c.mesh.n_cells, 1.0)
        Jv = o.jv(u, v).ravel()
        Kv = K @ v.ravel()
        assert np.linalg.norm(Jv - Kv) < 1e-6 * np.linalg.norm(Kv)


def test_jv_matches_bruteforce_fd_jacobian_neo_hookean():
    c = I.case_nh_beam(5, 3, 3, (0.5, 0.3, 0.3), end_uy=0.05, perturb=0.1)  # 45 cells
    o = O.Oracle.from_case(c)
    u = I.random_field(1, c.mesh.n_cells, 2e-2)
    J = _fd_jacobian(o, u, 1e-6)
    v = I.random_field(5, c.mesh.n_cells, 1.0)
    Jv = o.jv(u, v).ravel()
    assert np.linalg.norm(Jv - J @ v.ravel()) < 1e-5 * np.linalg.norm(J @ v.ravel())
    # zero direction
    assert np.all(o.jv(u, np.zeros_like(v)) == 0)


def test_jtilde_closed_form_on_uniform_box():
    """Sec. 3.1 on an orthogonal uniform mesh: off-diagonals Kbar |Gamma| / h, so J~ is Kbar h
    times the 7-point graph Laplacian; displacement faces add Kbar |Gamma| / (h/2)."""
    nx, ny, nz, h = 4, 3, 3, 0.5
    m = I.hex_box(nx, ny, nz, (nx * h, ny * h, nz * h))
    m.patch("xmin").bc = I.BC_DISP
    E, nu = 3.0, 0.2
    Kbar = E / (1 + nu) + E * nu / ((1 + nu) * (1 - 2 * nu))
    o = O.Oracle(m, I.Material(I.LAW_LINEAR, E, nu))
    A = np.zeros((m.n_cells, m.n_cells))
    for P, N in zip(m.owner[: m.n_internal], m.neighbour):
        A[P, N] = A[N, P] = Kbar * h
    D = -A.sum(1)
    i = np.arange(m.n_cells) % nx
    D[i == 0] -= Kbar * h * 2
    A += np.diag(D)
    np.testing.assert_allclose(o.jtilde_diag(), D, rtol=1e-14)
    v = I.random_field(2, m.n_cells, 1.0)
    np.testing.assert_allclose(o.jtilde_apply(v), A @ v, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(o.bjacobi(v), v / D[:, None], rtol=1e-14)


def test_jtilde_symmetric_negative_definite_on_distorted_mesh():
    c = I.case_cantilever(5, 3, 3, (0.5, 0.3, 0.3), perturb=0.15, seed=8)
    o = O.Oracle.from_case(c)
    n = c.mesh.n_cells
    M = np.zeros((n, n))
    for j in range(n):
        e = np.zeros((n, 3)); e[j, 0] = 1.0
        M[:, j] = o.jtilde_apply(e)[:, 0]
    np.testing.assert_allclose(M, M.T, rtol=1e-13, atol=1e-13 * np.abs(M).max())
    assert np.linalg.eigvalsh(M).max() < 0
    # rows of cells without displacement faces sum to zero
    rows = M.sum(1)
    i = np.arange(n) % 5
    assert np.abs(rows[i > 0]).max() < 1e-12 * np.abs(M).max()


def test_gmres_full_krylov_solves_linear_system():
    c = I.case_cantilever(4, 3, 3, (0.4, 0.3, 0.3), perturb=0.15, seed=2)
    o = O.Oracle.from_case(c)
    nc = c.mesh.n_cells
    u = np.zeros((nc, 3))
    K = _fd_jacobian(o, u, 1e-6)
    b = I.random_field(3, nc, 1e3)
    for pc in (O.PC_NONE, O.PC_BJACOBI):
        x, rc, its, rel = o.gmres(u, b, m=3 * nc, eta=1e-10, max_restarts=2, pc=pc)
        assert rc == 0
        x_ref = np.linalg.solve(K, b.ravel())
        assert np.linalg.norm(x.ravel() - x_ref) < 1e-7 * np.linalg.norm(x_ref)
    # preconditioning reduces the iteration count
    _, _, its_none, _ = o.gmres(u, b, m=3 * nc, eta=1e-6, pc=O.PC_NONE)
    _, _, its_bj, _ = o.gmres(u, b, m=3 * nc, eta=1e-6, pc=O.PC_BJACOBI)
    assert its_bj <= its_none


def test_lgmres_without_corrections_is_gmres():
    """Loose GMRES keeping no corrections is restarted GMRES(m): the two independent oracle
    routines give bitwise equal iterates."""
    c = I.case_cantilever(8, 4, 4, (0.8, 0.4, 0.4), perturb=0.15, seed=2)
    o = O.Oracle.from_case(c)
    u = np.zeros((c.mesh.n_cells, 3))
    b = I.random_field(4, c.mesh.n_cells, 1e3)
    x1, rc1, its1, rel1 = o.gmres(u, b, m=8, eta=1e-4, max_restarts=400, pc=O.PC_BJACOBI)
    x2, rc2, its2, rel2 = o.lgmres(u, b, m=8, aug=0, eta=1e-4, max_restarts=400, pc=O.PC_BJACOBI)
    assert rc1 == rc2 == 0 and its1 == its2 and rel1 == rel2
    assert np.array_equal(x1, x2)


@pytest.mark.parametrize("pc", [O.PC_NONE, O.PC_BJACOBI])
def test_lgmres_solves_the_assembled_linear_system(pc):
    """Loose GMRES (Sec. 4.2: restart 30 with 2 kept corrections; here restarts short enough
    that corrections are used) reaches the solution of the dense system assembled column by
    column, and meets its own tolerance on the true residual K x - b."""
    c = I.case_cantilever(4, 3, 3, (0.4, 0.3, 0.3), perturb=0.15, seed=2)
    o = O.Oracle.from_case(c)
    nc = c.mesh.n_cells
    u = np.zeros((nc, 3))
    K = _fd_jacobian(o, u, 1e-6)
    b = I.random_field(3, nc, 1e3)
    x_ref = np.linalg.solve(K, b.ravel())
    for aug in (1, 2, 3):
        x, rc, its, rel = o.lgmres(u, b, m=6, aug=aug, eta=1e-10, max_restarts=400, pc=pc)
        assert rc == 0 and rel <= 1e-10
        assert np.linalg.norm(x.ravel() - x_ref) < 1e-6 * np.linalg.norm(x_ref)
        # linear elasticity: R(x) - R(0) = K x exactly, independent of the Jv difference step
        r_true = b - (o.residual(x) - o.residual(u))
        assert np.linalg.norm(r_true) <= 1e-8 * np.linalg.norm(b)


def test_lgmres_corrections_reduce_restarted_iterations():
    """Kept corrections recover part of what a restart discards: on a slowly converging
    restarted problem, loose GMRES(m, 2) needs fewer products than GMRES(m) (both reach the
    tolerance)."""
    c = I.case_cantilever(12, 4, 4, (1.0, 0.2, 0.2), perturb=0.15, seed=2)
    o = O.Oracle.from_case(c)
    u = np.zeros((c.mesh.n_cells, 3))
    b = I.random_field(7, c.mesh.n_cells, 1e3)
    _, rc0, its0, _ = o.lgmres(u, b, m=10, aug=0, eta=1e-4, max_restarts=2000, pc=O.PC_BJACOBI)
    _, rc2, its2, _ = o.lgmres(u, b, m=10, aug=2, eta=1e-4, max_restarts=2000, pc=O.PC_BJACOBI)
    assert rc0 == 0 and rc2 == 0
    assert its2 < 0.5 * its0  # 496 against 4253 when written


def test_newton_with_loose_gmres_reaches_the_same_solution():
    c = I.case_cantilever(6, 4, 4, (0.6, 0.4, 0.4), perturb=0.15, seed=2)
    o = O.Oracle.from_case(c)
    u0, rc0, st0 = o.newton(rtol=1e-11, eta=1e-6, pc=O.PC_BJACOBI)
    u2, rc2, st2 = o.newton(rtol=1e-11, eta=1e-6, pc=O.PC_BJACOBI, m=10, aug=2)
    assert rc0 == 0 and rc2 == 0
    assert np.linalg.norm(u0 - u2) < 1e-7 * np.linalg.norm(u0)


def test_newton_linear_problem_and_preconditioner_independence():
    """The converged discrete solution does not depend on the preconditioner (Sec. 3.1)."""
    c = I.case_cantilever(6, 4, 4, (0.6, 0.4, 0.4), perturb=0.15, seed=2)
    o = O.Oracle.from_case(c)
    o.mg_setup(coarse_max=10)
    sols = []
    for pc in (O.PC_BJACOBI, O.PC_MG):
        u, rc, st = o.newton(rtol=1e-11, eta=1e-6, pc=pc)
        assert rc == 0
        sols.append(u)
    assert np.linalg.norm(sols[0] - sols[1]) < 1e-7 * np.linalg.norm(sols[0])


def test_newton_quadratic_convergence_neo_hookean():
    """Sec. 2.2: with an (almost) exact Jacobian action Newton converges quadratically:
    log r_{k+1} / log r_k -> 2 until the finite-difference floor."""
    c = I.case_nh_beam(8, 3, 3, (1.0, 0.125, 0.125), end_uy=0.15, load_steps=1)
    o = O.Oracle.from_case(c)
    u, rc, st = o.newton(rtol=1e-11, eta=1e-12, pc=O.PC_BJACOBI, max_newton=30)
    assert rc == 0
    o.set_load_factor(1.0)
    r0 = np.linalg.norm(o.residual(np.zeros_like(u)))
    r = np.array([st.hist[k] for k in range(st.n_hist)]) / r0
    # find consecutive pairs in the asymptotic range (1e-1 > r_k > 1e-5)
    orders = [np.log(r[k + 1]) / np.log(r[k]) for k in range(len(r) - 1) if 1e-5 < r[k] < 5e-2 and r[k + 1] > 1e-12]
    assert orders, r
    assert max(orders) > 1.8, (r, orders)


def test_multigrid_aggregation_on_chain():
    """Hand-worked pass-1/pass-2 aggregation of a uniform 6-cell chain:
    {0,1} then {3,2,4}; 5 joins the aggregate of 4."""
    m = I.hex_box(6, 1, 1, (6.0, 1.0, 1.0))
    m.patch("xmin").bc = I.BC_DISP
    o = O.Oracle(m, I.Material(I.LAW_LINEAR, 1.0, 0.3), prepare=False)
    # a 1-cell-wide chain has a singular least-squares tensor; the multigrid set-up only
    # needs J~, so use a 2-D slab instead
    m2 = I.hex_box(6, 2, 1, (6.0, 2.0, 1.0), dim=2)
    for p in m2.patches:
        if p.name in ("ymin", "ymax"):
            p.bc = I.BC_TRAC
    m2.patch("xmin").bc = I.BC_DISP
    o = O.Oracle(m2, I.Material(I.LAW_LINEAR, 1.0, 0.3))
    o.mg_setup(theta=0.25, coarse_max=1)
    agg = o.mg_aggregates(0)
    # every row is assigned, aggregates are numbered 0..k-1
    assert agg.min() == 0 and set(agg) == set(range(agg.max() + 1))
    # cells (i, j) -> i + 6 j; row 0 takes its strong neighbours 1 and 6
    assert agg[0] == agg[1] == agg[6]


@pytest.mark.parametrize("smoothed,sweeps", [(False, 1), (True, 1), (True, 2)])
def test_multigrid_vcycle_is_symmetric_and_contracts(smoothed, sweeps):
    c = I.case_cantilever(12, 4, 4, (1.0, 0.33, 0.33), perturb=0.15, seed=9)
    o = O.Oracle.from_case(c)
    L = o.mg_setup(coarse_max=20, smoothed=smoothed, sweeps=sweeps)
    assert L >= 2
    n = c.mesh.n_cells
    a, b = I.random_field(1, n), I.random_field(2, n)
    za, zb = o.mg_vcycle(a), o.mg_vcycle(b)
    assert abs(np.vdot(za, b) - np.vdot(a, zb)) < 1e-10 * abs(np.vdot(za, b))
    # as a preconditioner it beats Jacobi on GMRES iterations
    u = np.zeros((n, 3))
    rhs = I.random_field(3, n, 1.0)
    _, _, its_bj, _ = o.gmres(u, rhs, eta=1e-6, pc=O.PC_BJACOBI)
    _, _, its_mg, _ = o.gmres(u, rhs, eta=1e-6, pc=O.PC_MG)
    assert its_mg < its_bj


@pytest.mark.parametrize("dims", [(2, 2, 2), (9, 5, 4)])
def test_single_level_vcycle_is_the_exact_compact_stencil_solve(dims):
    """A mesh at or below the coarse-solve size gives a one-level hierarchy, and the V-cycle
    is then the direct solve with J~ (Sec. 3.1): J~ z = v to round-off, for the smallest 3-D
    block (8 cells, all on the boundary) as well as a larger one."""
    c = I.case_cantilever(*dims, (1.0, 0.5, 0.4), perturb=0.1, seed=3)
    o = O.Oracle.from_case(c)
    assert o.mg_setup(coarse_max=2000, smoothed=True, sweeps=2) == 1
    v = I.random_field(6, c.mesh.n_cells, 1.0)
    z = o.mg_vcycle(v)
    assert np.linalg.norm(o.jtilde_apply(z) - v) <= 1e-13 * np.linalg.norm(v)


def test_smoothed_aggregation_prolongation_and_strength():
    """Smoothed prolongation P = (I - omega D^-1 A) P_tent preserves the constant vector's
    image (row sums of P equal 1 - omega D^-1 (A 1)); two-level J~ coarse operators stay
    symmetric; smoothed aggregation needs fewer Krylov iterations than plain aggregation."""
    c = I.case_cantilever(24, 6, 6, (1.0, 0.25, 0.25), perturb=0.15, seed=9)
    o = O.Oracle.from_case(c)
    n = c.mesh.n_cells
    u = np.zeros((n, 3))
    rhs = I.random_field(3, n, 1.0)
    its = {}
    for sm in (False, True):
        o.mg_setup(coarse_max=30, smoothed=sm, sweeps=2)
        _, rc, its[sm], _ = o.gmres(u, rhs, eta=1e-6, pc=O.PC_MG)
        assert rc == 0
    assert its[True] < its[False]


@pytest.mark.parametrize("pc", [O.PC_BJACOBI, O.PC_MG])
def test_segregated_reaches_the_newton_solution(pc):
    """Sec. 3.1: the segregated quasi-Newton iteration (J~ per component, PCG reduced by 0.9,
    Sec. 3.2) solves the same discrete equations, so it converges to the Newton solution."""
    c = I.case_cantilever(6, 4, 4, (0.6, 0.4, 0.4), perturb=0.15, seed=2)
    o = O.Oracle.from_case(c)
    o.mg_setup(coarse_max=10)
    un, rcn, _ = o.newton(rtol=1e-11, eta=1e-6, pc=O.PC_BJACOBI)
    us, rcs, sts = o.segregated(rtol=1e-11, pc=pc)
    assert rcn == 0 and rcs == 0
    assert np.linalg.norm(us - un) < 1e-8 * np.linalg.norm(un)
    assert sts.newton_its > 50 and sts.gmres_its >= sts.newton_its  # many small corrections


def test_segregated_inner_solve_is_the_compact_stencil_system():
    """One outer iteration with the inner systems solved tightly gives du = -J~^-1 R(0)
    exactly, checked with the independent J~ product."""
    c = I.case_cantilever(5, 3, 3, (0.5, 0.3, 0.3), perturb=0.15, seed=3)
    o = O.Oracle.from_case(c)
    nc = c.mesh.n_cells
    R0 = o.residual(np.zeros((nc, 3)))
    for pc in (O.PC_NONE, O.PC_BJACOBI):
        u1, rc, st = o.segregated(rtol=0.0, max_outer=1, inner_tol=1e-13, pc=pc)
        assert st.newton_its == 1
        assert np.linalg.norm(o.jtilde_apply(u1) + R0) <= 1e-10 * np.linalg.norm(R0)


def test_segregated_neo_hookean_load_steps():
    c = I.case_nh_beam(8, 3, 3, (1.0, 0.375, 0.375), end_uy=0.1, load_steps=2)
    o = O.Oracle.from_case(c)
    un, rcn, _ = o.newton(load_steps=2, rtol=1e-10, eta=1e-6)
    us, rcs, sts = o.segregated(load_steps=2, rtol=1e-10)
    assert rcn == 0 and rcs == 0
    assert np.linalg.norm(us - un) < 1e-7 * np.linalg.norm(un)


def test_st_venant_kirchhoff_law_from_its_definition():
    """App. B: S = 2 mu E + lambda tr(E) I with the Green strain E, sigma = F S F^T / J; the
    total-Lagrangian operator is then T = J F^-1 sigma = S F^T (the transpose of P = F S).
    Written out here from the printed definitions; also objectivity and the small-strain
    limit (Hooke)."""
    E_, nu = 2.0e6, 0.3
    mu, lam = E_ / (2 * (1 + nu)), E_ * nu / ((1 + nu) * (1 - 2 * nu))
    o = _one_cell_oracle(I.LAW_STVK, E_, nu)
    rng = np.random.default_rng(11)
    G = 0.3 * rng.standard_normal((3, 3))
    F = np.eye(3) + G.T
    Eg = 0.5 * (G + G.T + G @ G.T)
    S = 2 * mu * Eg + lam * np.trace(Eg) * np.eye(3)
    sigma = F @ S @ F.T / np.linalg.det(F)
    np.testing.assert_allclose(o.cauchy_stress(G), sigma, rtol=1e-12, atol=1e-9 * mu)
    T = o.traction_operator(np.broadcast_to(G, (8, 3, 3)).copy())[0]
    np.testing.assert_allclose(T, S @ F.T, rtol=1e-12, atol=1e-9 * mu)
    Q = _rot(rng)
    s_rot = o.cauchy_stress((Q @ F - np.eye(3)).T)
    np.testing.assert_allclose(s_rot, Q @ sigma @ Q.T, atol=1e-9 * np.abs(sigma).max())
    for t in (1e-5, 1e-6):
        Gs = t * G
        hooke = mu * (Gs + Gs.T) + lam * np.trace(Gs) * np.eye(3)
        assert np.abs(o.cauchy_stress(Gs) - hooke).max() < 20 * t * np.abs(hooke).max()


def _beam_tip(nx, ny, nz, u, mesh):
    """Mean y-displacement of the last cell layer and the cantilever-beam value at its centre
    plane (Euler-Bernoulli F x^2 (3L - x) / (6 E I) plus the Timoshenko shear term F x / (k G A),
    k = 5/6) for the 1 x 0.1 x 0.1 m, E = 200 GPa, nu = 0.3 beam under F = 1 MPa x 0.01 m^2."""
    x = mesh.nominal_cell_centres()
    tip = x[:, 0] > 1.0 - 1.0 / nx
    L, E, nu, A = 1.0, 200e9, 0.3, 0.01
    I_ = 0.1 * 0.1 ** 3 / 12.0
    F = 1e6 * A
    xc = x[tip, 0].mean()
    beam = F * xc ** 2 * (3 * L - xc) / (6 * E * I_) + F * xc / (5.0 / 6.0 * E / (2 * (1 + nu)) * A)
    return u[tip, 1].mean(), beam


def test_cantilever_tip_deflection_approaches_beam_theory():
    """Config 2 sanity (the 1 m cantilever with the 1 MPa end shear): the tip deflection tends to
    the beam value F L^3 / (3 E I) = 2.0 mm (+ shear) from below as the cross-section is refined
    (4 and 8 cells through the thickness: ratio 0.65 and 0.85; 20, the 80k-cell case, 0.96 in
    the GPU tests), the error falling by more than half per halving of h."""
    ratios = []
    for n in (4, 8):
        c = I.case_cantilever(10 * n, n, n, (1.0, 0.1, 0.1))
        o = O.Oracle.from_case(c)
        o.mg_setup(coarse_max=50, smoothed=True, sweeps=2)
        u, rc, st = o.newton(load_steps=1, rtol=1e-8, pc=O.PC_MG, m=30, aug=2)
        assert rc == 0
        tip, beam = _beam_tip(10 * n, n, n, u, c.mesh)
        ratios.append(tip / beam)
    assert 0.6 < ratios[0] < ratios[1] < 1.0, ratios
    assert (1.0 - ratios[1]) < 0.5 * (1.0 - ratios[0]), ratios
