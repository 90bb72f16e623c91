"""Oracle pins for the updated-Lagrangian form of App. A (Eq. momentum_UL).

  * homogeneous deformation (patch test): displacement data of a homogeneous deformation on
    every boundary face of a distorted mesh, reached in three load steps on meshes that move
    after each step: the solution is the linear field to round-off, every cell's total
    deformation gradient is I + A, and the moved cell centroids are the deformed reference
    centroids (the point motion is exact for linear increments);
  * a single load step starts from the reference configuration, where the updated and the
    total-Lagrangian balances coincide: the two solutions are the same bit for bit;
  * several load steps on a smooth problem: the two forms discretise the same continuous
    problem differently (moving mesh, relative deformation gradient), so their solutions
    approach each other at second order as the mesh is refined.
"""
import numpy as np
import pytest

import oracle as O
from paper_2502_17217_gb300 import inputs as I


def _all_disp(mesh, values_fn):
    for p in mesh.patches:
        p.bc = I.BC_DISP
        p.values = values_fn(p)


def test_homogeneous_deformation_is_exact_over_load_steps():
    m = I.hex_box(5, 4, 4, (1.0, 0.8, 0.8), perturb=0.15, seed=24)
    rng = np.random.default_rng(5)
    A = rng.standard_normal((3, 3)) * 0.1  # finite strain
    b = rng.standard_normal(3) * 0.01
    mat = I.Material(I.LAW_NEOHOOKEAN, 0.38e6, 8.3e6)
    probe = O.Oracle(m, mat)
    _, Cf, _, C0 = probe.geometry()
    _all_disp(m, lambda p: Cf[p.start:p.start + p.size] @ A.T + b)
    o = O.Oracle(m, mat)
    o.set_updated_lagrangian(True)
    u, rc, st = o.newton(load_steps=3, rtol=1e-12, pc=O.PC_BJACOBI)
    assert rc == 0 and st.newton_its >= 3
    exact = C0 @ A.T + b
    assert np.abs(u - exact).max() <= 1e-11 * np.abs(exact).max()
    F = o.ul_state()
    assert np.abs(F - (np.eye(3) + A)).max() <= 1e-11
    _, _, _, C1 = o.geometry()  # the mesh is left in the final configuration
    assert np.abs(C1 - (C0 + exact)).max() <= 1e-11 * np.abs(C0).max()


def test_one_load_step_equals_the_total_lagrangian_solution():
    case = I.case_nh_beam(12, 3, 3, (1.0, 0.25, 0.25), end_uy=0.2, perturb=0.1, seed=3)
    ut, rct, _ = O.Oracle.from_case(case).newton(load_steps=1, rtol=1e-11)
    o = O.Oracle.from_case(case)
    o.set_updated_lagrangian(True)
    uu, rcu, _ = o.newton(load_steps=1, rtol=1e-11)
    assert rct == 0 and rcu == 0
    assert np.array_equal(uu, ut)


def _cube(n, amp=0.1):
    """Unit cube, compressible neo-Hookean (mu = 1 MPa, kappa = 2 MPa), smooth displacement
    data on all six faces (reached in three load steps)."""
    def ustar(X):
        x, y, z = X[:, 0], X[:, 1], X[:, 2]
        return amp * np.stack([np.sin(np.pi * y) * x, 0.5 * np.sin(np.pi * z) * y + 0.3 * x * z,
                               0.4 * np.sin(np.pi * x) * z], 1)
    m = I.hex_box(n, n, n, (1.0, 1.0, 1.0))
    _all_disp(m, lambda p: ustar(m.nominal_face_centres(p)))
    return I.Case(f"cube{n}", m, I.Material(I.LAW_NEOHOOKEAN, 1.0e6, 2.0e6), None, load_steps=3)


def test_updated_and_total_lagrangian_solutions_converge_to_each_other():
    diffs = []
    for n in (8, 16, 32):
        case = _cube(n)
        sol = []
        for ul in (False, True):
            o = O.Oracle.from_case(case)
            if ul:
                o.set_updated_lagrangian(True)
            o.mg_setup(theta=0.4, coarse_max=200, smoothed=True, sweeps=2)
            u, rc, _ = o.newton(load_steps=3, rtol=1e-11, pc=O.PC_MG, m=30, aug=2)
            assert rc == 0
            sol.append(u)
        diffs.append(np.linalg.norm(sol[1] - sol[0]) / np.linalg.norm(sol[0]))
    # measured ratios 2.7 and 3.0, tending to 4 (second order)
    assert diffs[0] / diffs[1] > 2.4 and diffs[1] / diffs[2] > 2.8, diffs
    assert diffs[2] < 5e-4


def test_unsupported_problems_are_refused():
    lin = I.case_cantilever(6, 2, 2, (1.0, 0.2, 0.2))
    with pytest.raises(RuntimeError, match="neo-Hookean"):
        O.Oracle.from_case(lin).set_updated_lagrangian(True)
