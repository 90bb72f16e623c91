"""Oracle pins for the dynamic form (Sec. 2.3 inertia term with the BDF2 acceleration of
Eq. inertia2, the transient-continuation predictor of Eq. predictor, the J~ inertia diagonal
of Sec. 3.1)."""
import numpy as np
import pytest

import oracle as O
from paper_2502_17217_gb300 import inputs as I

RHO = 1000.0


def _bdf2_history(u_new, ut, utm1, vt, vtm1, dt):
    vn = (3 * u_new - 4 * ut + utm1) / (2 * dt)
    an = (3 * vn - 4 * vt + vtm1) / (2 * dt)
    return vn, an


def test_free_body_under_uniform_body_force_follows_the_scalar_bdf2_recurrence():
    """A body with traction-free faces under a uniform body force f moves rigidly: every cell
    follows rho a(u) = f with the BDF2 acceleration, a scalar recurrence written out here."""
    m = I.hex_box(4, 3, 3, (0.4, 0.3, 0.3), perturb=0.15, seed=3)
    f = np.array([2.0e3, -1.0e3, 0.5e3])
    case = I.Case("free", m, I.Material(I.LAW_NEOHOOKEAN, 1.0e6, 4.0e6), np.tile(f, (m.n_cells, 1)))
    o = O.Oracle.from_case(case)
    dt = 1e-3
    o.set_dynamics(RHO, dt)
    n_steps = 6
    u, rc, st, probe = o.dynamic(n_steps, rtol=1e-12, atol=1e-9, eta=1e-10, probe_cell=5)
    assert rc == 0
    k2 = 9.0 / (4 * dt * dt)
    ut = utm1 = vt = vtm1 = np.zeros(3)
    for step in range(n_steps):
        c = (3 * (-4 * ut + utm1) / (2 * dt) - 4 * vt + vtm1) / (2 * dt)
        un = (f / RHO - c) / k2  # rho (k2 u + c) = f
        vn, _ = _bdf2_history(un, ut, utm1, vt, vtm1, dt)
        utm1, ut, vtm1, vt = ut, un, vt, vn
        np.testing.assert_allclose(probe[step], un, rtol=1e-9, atol=1e-15)
    np.testing.assert_allclose(u, np.tile(ut, (m.n_cells, 1)), rtol=1e-9, atol=1e-15)


@pytest.mark.parametrize("pc", [O.PC_BJACOBI, O.PC_NONE])
def test_linear_dynamics_equal_the_assembled_bdf2_recurrence(pc):
    """Linear elasticity: R(u) = K u + b exactly, so each time step solves
    (K - 9/(4 dt^2) M) u = M c - b with M = rho diag(Omega).  K (column by column from the
    static residual), the recurrence, the history update and the predictor-independence of
    the converged step are all checked against a dense solve."""
    case, probe = I.case_dynamic_beam(2, 6, 2, traction=(2.0e3, 1.0e3, 0.0), law=I.LAW_LINEAR)
    o = O.Oracle.from_case(case)
    nc = case.mesh.n_cells
    z = np.zeros((nc, 3))
    b = o.residual(z).ravel()
    K = np.zeros((3 * nc, 3 * nc))
    for j in range(3 * nc):
        e = np.zeros(3 * nc); e[j] = 1.0
        K[:, j] = o.residual(e.reshape(nc, 3)).ravel() - b
    V = o.geometry()[2]
    dt = 2e-3
    Mdiag = np.repeat(RHO * V, 3)
    o.set_dynamics(RHO, dt)
    n_steps = 5
    u, rc, st, pr = o.dynamic(n_steps, rtol=1e-13, atol=1e-12, eta=1e-12, pc=pc, probe_cell=probe)
    assert rc == 0
    k2 = 9.0 / (4 * dt * dt)
    A = K - k2 * np.diag(Mdiag)
    ut = utm1 = vt = vtm1 = np.zeros(3 * nc)
    for step in range(n_steps):
        c = (3 * (-4 * ut + utm1) / (2 * dt) - 4 * vt + vtm1) / (2 * dt)
        un = np.linalg.solve(A, Mdiag * c - b)
        vn, _ = _bdf2_history(un, ut, utm1, vt, vtm1, dt)
        utm1, ut, vtm1, vt = ut, un, vt, vn
        np.testing.assert_allclose(pr[step], un.reshape(nc, 3)[probe], rtol=1e-7, atol=1e-14)
    assert np.linalg.norm(u.ravel() - ut) <= 1e-7 * np.linalg.norm(ut)


def test_inertia_adds_the_mass_diagonal_to_jtilde():
    """Sec. 3.1: the inertia term adds -(9/4) rho Omega / dt^2 to the diagonal of J~ and
    nothing else."""
    case, _ = I.case_dynamic_beam(2, 5, 2)
    o = O.Oracle.from_case(case)
    v = I.random_field(4, case.mesh.n_cells, 1.0)
    j0 = o.jtilde_apply(v)
    dt = 1e-3
    o.set_dynamics(RHO, dt)
    j1 = o.jtilde_apply(v)
    V = o.geometry()[2]
    np.testing.assert_allclose(j1 - j0, -2.25 * RHO * V[:, None] / dt ** 2 * v, rtol=1e-12, atol=1e-6)


def test_column_first_bending_frequency_tends_to_beam_theory():
    """Case 6 of Sec. 4 chooses E = 15.293 MPa, rho = 1000 kg/m^3 for a 1 Hz first frequency
    of the 0.2 x 2 x 0.2 m column: Euler-Bernoulli gives f1 = 1.8751^2 / (2 pi L^2)
    sqrt(E I / (rho A)) = 0.999 Hz.  The discrete frequencies come from the generalised
    eigenproblem of the linear residual's stiffness K (assembled column by column, R(u) =
    K u + b) and the lumped mass rho Omega_P (the inertia term of Sec. 2.3): the two bending
    modes of the square section coincide, and f1 falls toward the beam value from above as
    the cross-section is refined (1.53, 1.33, 1.22 Hz at 2, 3 and 4 cells across; coarse
    cross-sections are too stiff in bending, as in the static cantilever)."""
    E, L, a = 15.293e6, 2.0, 0.2
    f_eb = 1.8751 ** 2 / (2 * np.pi * L ** 2) * np.sqrt(E * a ** 4 / 12 / (RHO * a * a))
    assert abs(f_eb - 1.0) < 0.01
    f1 = []
    for dims in ((2, 20, 2), (3, 30, 3), (4, 40, 4)):
        case, _ = I.case_dynamic_beam(*dims, traction=(0.0, 0.0, 0.0), law=I.LAW_LINEAR)
        o = O.Oracle.from_case(case)
        nc = case.mesh.n_cells
        n = 3 * nc
        b = o.residual(np.zeros((nc, 3))).ravel()
        K = np.empty((n, n))
        for j in range(n):
            e = np.zeros(n)
            e[j] = 1.0
            K[:, j] = o.residual(e.reshape(nc, 3)).ravel() - b
        m = np.repeat(RHO * o.geometry()[2], 3)
        w2 = np.sort(np.linalg.eigvals(-K / m[:, None]).real)
        f = np.sqrt(w2[:2]) / (2 * np.pi)
        assert abs(f[1] - f[0]) <= 1e-8 * f[0], f  # x and z bending of the square section
        f1.append(f[0])
    assert f1[0] > f1[1] > f1[2] > f_eb, f1
    assert f1[2] < 1.25 * f_eb, f1
