"""The updated-Lagrangian form of App. A (Eq. momentum_UL) on the device, against the oracle.

  * solves of a distorted neo-Hookean beam in three load steps (each on the mesh moved by the
    last), block-Jacobi in FP64 and multigrid in mixed precision: displacements within 1e-8
    of the oracle's, both run to |R| <= 1e-11 |R0| per step;
  * the moved mesh after the solve: face and cell geometry within 1e-10 of the oracle's;
  * the homogeneous-deformation patch test over three load steps: the linear field to
    round-off;
  * at the reference configuration the residual and Jv match the oracle's updated-Lagrangian
    ones (which coincide with the total-Lagrangian ones there);
  * unsupported problems are refused.
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


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


def _beam():
    return I.case_nh_beam(16, 4, 4, (1.0, 0.25, 0.25), end_uy=0.25, load_steps=3, perturb=0.1, seed=3)


@pytest.mark.parametrize("kind", ["bjacobi_fp64", "mg_mixed"])
def test_updated_lagrangian_solve_and_moved_mesh_match_the_oracle(kind):
    from paper_2502_17217_gb300 import jfnk
    case = _beam()
    kw = dict(pc=jfnk.PC_BJACOBI) if kind == "bjacobi_fp64" else \
        dict(pc=jfnk.PC_MG, precision=jfnk.PREC_MIXED, mg_coarse_max=50)
    s = jfnk.Solver.from_case(case, newton_rtol=1e-11, **kw)
    s.set_formulation(jfnk.FORM_UPDATED_LAGRANGIAN)
    ug, st, rc = s.solve(load_steps=3)
    assert rc == 0 and st.load_steps_done == 3
    o = O.Oracle.from_case(case)
    o.set_updated_lagrangian(True)
    if kind == "mg_mixed":
        o.mg_setup(theta=s.options.mg_theta, coarse_max=50, smoothed=bool(s.options.mg_smoothed),
                   sweeps=s.options.mg_smooth_sweeps)
    uo, rco, _ = o.newton(load_steps=3, rtol=1e-11, pc=O.PC_MG if kind == "mg_mixed" else O.PC_BJACOBI,
                          m=s.options.gmres_restart, aug=s.options.gmres_aug)
    assert rco == 0
    assert _rel(ug, uo) <= 1e-8, _rel(ug, uo)
    # both leave the mesh in the final configuration
    for a, b in zip(s.geometry(), o.geometry()):
        assert _rel(a, b) <= 1e-10, _rel(a, b)
    # and the updated-Lagrangian solution differs from the total-Lagrangian one (moving mesh)
    ut, _, _ = jfnk.Solver.from_case(case, newton_rtol=1e-11, **kw).solve(load_steps=3)
    assert 1e-6 < _rel(ug, ut) < 1e-2


def test_updated_lagrangian_homogeneous_deformation_is_exact():
    from paper_2502_17217_gb300 import jfnk
    m = I.hex_box(5, 4, 4, (1.0, 0.8, 0.8), perturb=0.15, seed=24)
    rng = np.random.default_rng(5)
    A = rng.standard_normal((3, 3)) * 0.1
    b = rng.standard_normal(3) * 0.01
    mat = I.Material(I.LAW_NEOHOOKEAN, 0.38e6, 8.3e6)
    _, Cf, _, C0 = O.Oracle(m, mat).geometry()
    for p in m.patches:
        p.bc = I.BC_DISP
        p.values = Cf[p.start:p.start + p.size] @ A.T + b
    s = jfnk.Solver(m, mat, newton_rtol=1e-12, pc=jfnk.PC_BJACOBI)
    s.set_formulation(jfnk.FORM_UPDATED_LAGRANGIAN)
    u, st, rc = s.solve(load_steps=3)
    assert rc == 0
    exact = C0 @ A.T + b
    assert np.abs(u - exact).max() <= 1e-10 * np.abs(exact).max()
    _, _, _, C1 = s.geometry()
    assert np.abs(C1 - (C0 + exact)).max() <= 1e-10 * np.abs(C0).max()


def test_updated_lagrangian_residual_and_jv_at_the_reference_configuration():
    from paper_2502_17217_gb300 import jfnk
    case = _beam()
    s = jfnk.Solver.from_case(case)
    s.set_formulation(jfnk.FORM_UPDATED_LAGRANGIAN)
    o = O.Oracle.from_case(case)
    o.set_updated_lagrangian(True)
    u = I.random_field(4, case.mesh.n_cells, 0.004)
    v = I.random_field(5, case.mesh.n_cells, 1.0)
    R, Ro = s.residual(u), o.residual(u)
    assert _rel(R, Ro) <= 1e-12
    J, Jo = s.jv(u, v), o.jv(u, v, R_u=Ro)
    eps = 1e-7 * (1 + np.linalg.norm(u)) / np.linalg.norm(v)
    tol = 1e-12 * (np.linalg.norm(Ro) / (eps * np.linalg.norm(Jo)) + 1.0)
    assert _rel(J, Jo) <= tol


def test_updated_lagrangian_refuses_unsupported_problems():
    from paper_2502_17217_gb300 import jfnk
    lin = I.case_cantilever(8, 2, 2, (1.0, 0.2, 0.2))
    s = jfnk.Solver.from_case(lin)
    s.set_formulation(jfnk.FORM_UPDATED_LAGRANGIAN)
    with pytest.raises(jfnk.JfnkError, match="updated Lagrangian"):
        s.setup()
    nh = jfnk.Solver.from_case(_beam())
    nh.set_formulation(jfnk.FORM_UPDATED_LAGRANGIAN)
    with pytest.raises(jfnk.JfnkError, match="Newton-Krylov"):
        nh.solve_segregated(load_steps=1)
    with pytest.raises(jfnk.JfnkError):
        nh.set_formulation(7)
