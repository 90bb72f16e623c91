"""Oracle pins: the manufactured solution of Case 1 (Sec. 4.1, App. E) and the order of accuracy.

* App. E prints the body force as +div(sigma(u*)); under Eq. momentum_lingeom a static balance
  needs f_b = -div(sigma(u*)).  The golden file transcribes App. E term by term; the test
  shows it equals +div(sigma(u*)) (derived symbolically), and that the generator's f_b is
  its negative.
* Displacement converges at second order (Sec. 4.1: 'approximately second-order', average
  and maximum error alike), the cell stresses at least at the rates Sec. 4.1 reports for the
  3-D cube: average error order about 1.5 on regular hexahedra and 1 on distorted ones,
  maximum error order approaching 1.  (On this 2-D case the measured stress orders are
  1.8-2.0, above those lower bounds; a wrong gradient weight or stress term drops them to 0.)
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_2502_17217_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_params():
    vals = {}
    for line in open(os.path.join(GOLDEN, "case1_parameters.txt")):
        if line.startswith("#") or not line.strip():
            continue
        k, v = line.split()
        vals[k] = float(v)
    return vals


def _app_e(x, E, nu, a):
    mu = E / (2 * (1 + nu))
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    trig = {"sin": np.sin, "cos": np.cos}
    out = np.zeros((x.shape[0], 3))
    comp = {"x": 0, "y": 1, "z": 2}
    for line in open(os.path.join(GOLDEN, "app_e_body_force.txt")):
        if line.startswith("#") or not line.strip():
            continue
        c, mod, fac, amp, tx, ty, tz = line.split()
        m = lam if mod == "lambda" else mu
        val = m * float(fac) * a[comp[amp]] * np.pi ** 2
        val = val * trig[tx](4 * np.pi * x[:, 0]) * trig[ty](2 * np.pi * x[:, 1]) * trig[tz](np.pi * x[:, 2])
        out[:, comp[c]] += val
    return out


def test_case1_parameters_match_generator():
    p = _read_params()
    assert I.MMS_AMPLITUDES == (p["a_x"], p["a_y"], p["a_z"])


def test_app_e_is_plus_div_sigma_and_generator_is_minus():
    sp = pytest.importorskip("sympy")
    p = _read_params()
    E, nu = p["E"], p["nu"]
    a = (p["a_x"], p["a_y"], p["a_z"])
    X = sp.symbols("x y z")
    mu = E / (2 * (1 + nu))
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    phi = sp.sin(4 * sp.pi * X[0]) * sp.sin(2 * sp.pi * X[1]) * sp.sin(sp.pi * X[2])
    u = [a[k] * phi for k in range(3)]
    grad = [[sp.diff(u[j], X[i]) for j in range(3)] for i in range(3)]
    div_u = sum(grad[i][i] for i in range(3))
    sig = [[mu * (grad[i][j] + grad[j][i]) + (lam * div_u if i == j else 0) for j in range(3)] for i in range(3)]
    div_sig = [sum(sp.diff(sig[i][j], X[i]) for i in range(3)) for j in range(3)]
    f = sp.lambdify(X, div_sig, "numpy")
    rng = np.random.default_rng(0)
    x = rng.uniform(0, 0.2, (50, 3))
    ref = np.stack([np.broadcast_to(np.asarray(v, dtype=float), (50,)) for v in f(x[:, 0], x[:, 1], x[:, 2])], 1)
    np.testing.assert_allclose(_app_e(x, E, nu, a), ref, rtol=1e-10, atol=1e-10 * np.abs(ref).max())
    np.testing.assert_allclose(I.mms_body_force(x, E, nu, dim=3), -ref, rtol=1e-10, atol=1e-10 * np.abs(ref).max())
    # 2-D analogue: no z factor, a_z = 0, plane strain
    phi2 = sp.sin(4 * sp.pi * X[0]) * sp.sin(2 * sp.pi * X[1])
    u2 = [a[0] * phi2, a[1] * phi2, 0]
    g2 = [[sp.diff(u2[j], X[i]) for j in range(3)] for i in range(3)]
    d2 = sum(g2[i][i] for i in range(3))
    s2 = [[mu * (g2[i][j] + g2[j][i]) + (lam * d2 if i == j else 0) for j in range(3)] for i in range(3)]
    ds2 = [sum(sp.diff(s2[i][j], X[i]) for i in range(3)) for j in range(3)]
    f2 = sp.lambdify(X, ds2, "numpy")
    ref2 = np.stack([np.broadcast_to(np.asarray(v, dtype=float), (50,)) for v in f2(x[:, 0], x[:, 1], x[:, 2])], 1)
    np.testing.assert_allclose(I.mms_body_force(x, E, nu, dim=2), -ref2, rtol=1e-10, atol=1e-10 * np.abs(ref2).max())


def _exact_stress_2d(C, E, nu):
    """Hooke stress of the manufactured field u* = (a_x, a_y) sin(4 pi x) sin(2 pi y), plane
    strain, from its analytic gradient, (grad u)_ij = d u_j / d x_i."""
    mu = E / (2 * (1 + nu))
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    ax, ay = I.MMS_AMPLITUDES[0], I.MMS_AMPLITUDES[1]
    x, y = C[:, 0], C[:, 1]
    dx = 4 * np.pi * np.cos(4 * np.pi * x) * np.sin(2 * np.pi * y)
    dy = 2 * np.pi * np.sin(4 * np.pi * x) * np.cos(2 * np.pi * y)
    g = np.zeros((len(C), 3, 3))
    g[:, 0, 0], g[:, 0, 1] = ax * dx, ay * dx
    g[:, 1, 0], g[:, 1, 1] = ax * dy, ay * dy
    tr = np.trace(g, axis1=1, axis2=2)
    return mu * (g + np.transpose(g, (0, 2, 1))) + lam * tr[:, None, None] * np.eye(3)


def _mms_error(n, perturb):
    """(L2, Linf) of the displacement error and (L2, Linf) of the cell stress error (Frobenius
    norm per cell) after a converged Newton solve of the n x n case."""
    c = I.case_mms2d(n, perturb=perturb, seed=n)
    o = O.Oracle.from_case(c)
    _, Cf, _, C = o.geometry()
    # load at the true centroids / face centroids of this mesh
    o.set_body_force(I.mms_body_force(C, 200e9, 0.3, dim=2))
    u, rc, st = o.newton(rtol=1e-10, eta=1e-4, pc=O.PC_BJACOBI, max_newton=20)
    assert rc == 0, (rc, st.final_rel_res)
    ex = I.mms_displacement(C, dim=2)
    e = np.linalg.norm(u[:, :2] - ex[:, :2], axis=1)
    g = o.gradient(u)
    s_num = np.array([o.cauchy_stress(g[i]) for i in range(len(g))])
    es = np.linalg.norm((s_num - _exact_stress_2d(C, 200e9, 0.3)).reshape(len(g), 9), axis=1)
    return np.array([np.sqrt(np.mean(e ** 2)), e.max(), np.sqrt(np.mean(es ** 2)), es.max()])


@pytest.mark.parametrize("perturb", [0.0, 0.15])
def test_mms_second_order_displacement_and_stress_order(perturb):
    errs = np.array([_mms_error(n, perturb) for n in (16, 32, 64)])
    order = np.log2(errs[1] / errs[2])  # finest pair: displacement L2, Linf; stress L2, Linf
    assert order[0] > 1.85, (errs, order)  # measured 1.95 on both mesh types
    assert order[1] > 1.8, (errs, order)  # measured 1.99 / 1.96
    assert errs[2, 0] < 0.05 * I.MMS_AMPLITUDES[1]
    # stresses: at least the 3-D rates of Sec. 4.1 (measured 2.01 / 1.81 average, 1.88 / 1.85 max)
    assert order[2] > (1.5 if perturb == 0.0 else 1.0), (errs, order)
    assert order[3] > 1.0, (errs, order)
    assert np.all(errs[1:] < errs[:-1]), errs


def _mms3d_error(n, perturb):
    """Sec. 4.1's cube (0.2 m, n cells per side; the paper's first hexahedral meshes have 125,
    1,000 and 8,000 cells), u* = a sin(4 pi x) sin(2 pi y) sin(pi z) prescribed on all six
    sides (non-zero there) with the body force of App. E (sign as derived): (L2, Linf) of the
    displacement error at the cell centroids."""
    E, nu = 200e9, 0.3
    m = I.hex_box(n, n, n, (0.2, 0.2, 0.2), perturb=perturb, seed=n)
    mat = I.Material(I.LAW_LINEAR, E, nu)
    _, Cf, _, C = O.Oracle(m, mat).geometry()
    for p in m.patches:
        p.bc = I.BC_DISP
        p.values = I.mms_displacement(Cf[p.start:p.start + p.size], dim=3)
    o = O.Oracle(m, mat)
    o.set_body_force(I.mms_body_force(C, E, nu, dim=3))
    u, rc, st = o.newton(rtol=1e-10, eta=1e-4, pc=O.PC_BJACOBI, max_newton=20)
    assert rc == 0, (rc, st.final_rel_res)
    e = np.linalg.norm(u - I.mms_displacement(C, dim=3), axis=1)
    return np.array([np.sqrt(np.mean(e ** 2)), e.max()])


@pytest.mark.parametrize("perturb", [0.0, 0.15])
def test_mms3d_cube_second_order_displacement(perturb):
    errs = np.array([_mms3d_error(n, perturb) for n in (5, 10, 20)])
    order = np.log2(errs[1] / errs[2])
    assert order[0] > 1.8, (errs, order)  # measured 1.88 regular, 1.91 distorted
    assert order[1] > 1.5, (errs, order)  # measured 1.59 / 1.77, rising toward 2 with refinement
    assert np.all(errs[1:] < errs[:-1]), errs
