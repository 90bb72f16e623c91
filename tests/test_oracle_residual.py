"""Oracle pins for the residual R(u): Eqs. divStressDiscret, stressInterp, RhieChow, App. A-D."""
import os

import numpy as np
import pytest

import oracle as O
from paper_2502_17217_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _all_disp(mesh, values_fn):
    for p in mesh.patches:
        if p.bc == I.BC_EMPTY:
            continue
        p.bc = I.BC_DISP
        p.values = values_fn(p)


def _face_centres(o, mesh, p):
    _, Cf, _, _ = o.geometry()
    return Cf[p.start:p.start + p.size]


@pytest.mark.parametrize("dim", [2, 3])
def test_uniform_stress_patch_test_linear(dim):
    """A linear displacement field with matching Dirichlet data is reproduced exactly:
    R(u) = 0 to round-off on a distorted mesh (exact gradient, Rhie-Chow cancellation,
    closed cells)."""
    if dim == 3:
        m = I.hex_box(6, 5, 4, (1.0, 0.8, 0.6), perturb=0.15, seed=21)
    else:
        m = I.hex_box(7, 6, 1, (1.0, 0.8, 0.1), perturb=0.15, seed=22, dim=2)
    rng = np.random.default_rng(3)
    A = rng.standard_normal((3, 3)) * 1e-3
    b = rng.standard_normal(3) * 1e-3
    if dim == 2:
        A[2, :] = 0; A[:, 2] = 0; b[2] = 0
    mat = I.Material(I.LAW_LINEAR, 200e9, 0.3)
    probe = O.Oracle(m, mat)
    _all_disp(m, lambda p: _face_centres(probe, m, p) @ A.T + b)
    o = O.Oracle(m, mat)
    _, _, _, C = o.geometry()
    u = C @ A.T + b
    R = o.residual(u)
    # scale: one face force magnitude E * |A| * area
    scale = 200e9 * np.abs(A).max() * (1.0 / 6) ** 2
    assert np.abs(R).max() < 1e-12 * scale, np.abs(R).max() / scale


def test_uniform_stress_patch_test_traction_faces():
    """Same, with traction faces carrying T = n . sigma(A) on three sides."""
    m = I.hex_box(5, 5, 4, (1.0, 1.0, 0.8), perturb=0.15, seed=23)
    rng = np.random.default_rng(4)
    A = rng.standard_normal((3, 3)) * 1e-3
    b = rng.standard_normal(3) * 1e-3
    E, nu = 70e9, 0.25
    mu, lam = E / (2 * (1 + nu)), E * nu / ((1 + nu) * (1 - 2 * nu))
    G = A.T  # grad u
    sig = mu * (G + G.T) + lam * np.trace(G) * np.eye(3)
    mat = I.Material(I.LAW_LINEAR, E, nu)
    probe = O.Oracle(m, mat)
    Sf, Cf, _, _ = probe.geometry()
    for p in m.patches:
        if p.name in ("xmax", "ymax", "zmax"):
            p.bc = I.BC_TRAC
            S = Sf[p.start:p.start + p.size]
            n = S / np.linalg.norm(S, axis=1)[:, None]
            p.values = n @ sig
        else:
            p.bc = I.BC_DISP
            p.values = Cf[p.start:p.start + p.size] @ A.T + b
    o = O.Oracle(m, mat)
    _, _, _, C = o.geometry()
    R = o.residual(C @ A.T + b)
    scale = E * np.abs(A).max() * 0.04
    assert np.abs(R).max() < 1e-12 * scale


def test_uniform_stress_patch_test_neo_hookean():
    """Total-Lagrangian neo-Hookean: a homogeneous deformation gradient gives a uniform
    traction operator, so R = 0 with matching Dirichlet data."""
    m = I.hex_box(5, 4, 4, (1.0, 0.8, 0.8), perturb=0.15, seed=24)
    rng = np.random.default_rng(5)
    A = rng.standard_normal((3, 3)) * 0.1  # finite strain
    b = rng.standard_normal(3) * 0.01
    mat = I.Material(I.LAW_NEOHOOKEAN, 0.38e6, 8.3e6)
    probe = O.Oracle(m, mat)
    _all_disp(m, lambda p: _face_centres(probe, m, p) @ A.T + b)
    o = O.Oracle(m, mat)
    _, _, _, C = o.geometry()
    R = o.residual(C @ A.T + b)
    scale = 8.3e6 * 0.1 * 0.04
    assert np.abs(R).max() < 1e-12 * scale


def test_translation_invariance_without_displacement_faces():
    m = I.hex_box(5, 4, 3, (1.0, 0.8, 0.6), perturb=0.15, seed=25)
    o = O.Oracle(m, I.Material(I.LAW_LINEAR, 200e9, 0.3))
    u = I.random_field(7, m.n_cells, 1e-4)
    c = np.array([0.3, -0.2, 0.5])
    R1, R2 = o.residual(u), o.residual(u + c)
    assert np.abs(R1 - R2).max() < 1e-9 * np.abs(R1).max()


def test_conservation_internal_faces_cancel():
    """Internal-face contributions cancel pairwise, so with no displacement faces the sum of
    the residuals is the applied traction plus body force, whatever u is."""
    m = I.hex_box(6, 4, 3, (1.0, 0.6, 0.5), perturb=0.15, seed=26)
    trac = np.array([1e5, -2e5, 3e5])
    xm = m.patch("xmax")
    xm.bc = I.BC_TRAC
    xm.values = np.tile(trac, (xm.size, 1))
    fb = I.random_field(9, m.n_cells, 1e4)
    o = O.Oracle(m, I.Material(I.LAW_NEOHOOKEAN, 1e6, 10e6), body_force=fb)
    Sf, _, V, _ = o.geometry()
    area = np.linalg.norm(Sf[xm.start:xm.start + xm.size], axis=1).sum()
    expected = area * trac + (fb * V[:, None]).sum(0)
    for seed in (1, 2):
        u = I.random_field(seed, m.n_cells, 1e-2)
        R = o.residual(u)
        np.testing.assert_allclose(R.sum(0), expected, rtol=1e-10)


def _rc_only(o_rc, o_norc, u):
    return o_rc.residual(u) - o_norc.residual(u)


def _stencil():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "app_c_rhie_chow_stencil.txt")) if not l.startswith("#")]
    return {int(a): float(b) for a, b in rows}


def test_rhie_chow_1d_stencil_app_c():
    """App. C, Eq. Rhie_Chow_1D: for u depending on x only, on a uniform mesh, the
    stabilisation of a cell two or more cells from the x-ends is the 5-point stencil."""
    nx, h = 12, 0.1
    m = I.hex_box(nx, 2, 2, (nx * h, 2 * h, 2 * h))
    mat = I.Material(I.LAW_LINEAR, 1.0e3, 0.25)
    Kbar = 2 * mat.p1 / (2 * (1 + mat.p2)) + mat.p1 * mat.p2 / ((1 + mat.p2) * (1 - 2 * mat.p2))
    o1 = O.Oracle(m, mat, alpha=1.0)
    o0 = O.Oracle(m, mat, alpha=0.0)
    rng = np.random.default_rng(6)
    col = rng.standard_normal((nx, 3))
    i = np.arange(m.n_cells) % nx
    D = _rc_only(o1, o0, col[i])
    st = _stencil()
    area = h * h
    for c in range(m.n_cells):
        if 2 <= i[c] <= nx - 3:
            expect = sum(coef * col[i[c] + off] for off, coef in st.items()) * Kbar * area / (4 * h)
            np.testing.assert_allclose(D[c], expect, rtol=1e-11, atol=1e-12 * Kbar * area)
    # special cases: cubic u -> 0, u = x^4 -> -6 alpha Kbar |Gamma| dx^3
    C = o1.geometry()[3]
    x = C[:, 0]
    for p, expect in ((3, 0.0), (4, -6 * Kbar * area * h ** 3)):
        u = np.stack([x ** p, 0 * x, 0 * x], 1)
        D = _rc_only(o1, o0, u)
        for c in range(m.n_cells):
            if 2 <= i[c] <= nx - 3:
                assert abs(D[c, 0] - expect) < 1e-9 * Kbar * area * h ** 3 * 100 + 1e-12


def test_rhie_chow_jump_form_app_d():
    """App. D: on a uniform mesh each internal-face stabilisation term equals
    alpha Kbar |Gamma| / (d.n) (u_N* - u_P*), u* = u +- (d/2).grad u."""
    nx, ny, nz, h = 5, 4, 4, 0.2
    m = I.hex_box(nx, ny, nz, (nx * h, ny * h, nz * h))
    mat = I.Material(I.LAW_LINEAR, 10.0, 0.3)
    Kbar = 2 * 10.0 / 2.6 + 10.0 * 0.3 / (1.3 * 0.4)
    for p in m.patches:
        p.bc = I.BC_TRAC
    o1 = O.Oracle(m, mat, alpha=1.0)
    o0 = O.Oracle(m, mat, alpha=0.0)
    u = I.random_field(3, m.n_cells, 1.0)
    D = _rc_only(o1, o0, u)
    Sf, _, _, C = o1.geometry()
    g = o1.gradient(u)
    expect = np.zeros_like(D)
    for f in range(m.n_internal):
        P, N = m.owner[f], m.neighbour[f]
        d = C[N] - C[P]
        n = Sf[f] / np.linalg.norm(Sf[f])
        uPs = u[P] + 0.5 * d @ g[P]
        uNs = u[N] - 0.5 * d @ g[N]
        t = Kbar * np.linalg.norm(Sf[f]) / np.dot(d, n) * (uNs - uPs)
        expect[P] += t
        expect[N] -= t
    np.testing.assert_allclose(D, expect, rtol=1e-10, atol=1e-12 * np.abs(expect).max())


def test_linear_residual_is_affine():
    """For Hooke's law R(u) = K u + b: R(a u + (1-a) v) = a R(u) + (1-a) R(v)."""
    c = I.case_cantilever(6, 3, 3, (1.0, 0.5, 0.5), perturb=0.15, seed=2)
    o = O.Oracle.from_case(c)
    u, v = I.random_field(1, c.mesh.n_cells, 1e-4), I.random_field(2, c.mesh.n_cells, 1e-4)
    a = 0.3
    lhs = o.residual(a * u + (1 - a) * v)
    rhs = a * o.residual(u) + (1 - a) * o.residual(v)
    assert np.abs(lhs - rhs).max() < 1e-12 * np.abs(rhs).max() * 10


def test_uniform_stress_patch_test_st_venant_kirchhoff():
    """App. B St. Venant-Kirchhoff in the total-Lagrangian form: a homogeneous deformation
    gradient gives a uniform traction operator, so R = 0 with matching Dirichlet data."""
    m = I.hex_box(5, 4, 4, (1.0, 0.8, 0.8), perturb=0.15, seed=27)
    rng = np.random.default_rng(8)
    A = rng.standard_normal((3, 3)) * 0.1
    b = rng.standard_normal(3) * 0.01
    mat = I.Material(I.LAW_STVK, 2.0e6, 0.3)
    probe = O.Oracle(m, mat)
    _all_disp(m, lambda p: _face_centres(probe, m, p) @ A.T + b)
    o = O.Oracle(m, mat)
    _, _, _, C = o.geometry()
    R = o.residual(C @ A.T + b)
    assert np.abs(R).max() < 1e-12 * 2.0e6 * 0.1 * 0.04
