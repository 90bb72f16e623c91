"""Oracle pins for symmetry faces (Eq. symm, the symmetry terms of Eq. leastSquaresGrad and
Eq. RhieChow, Sec. 3.1).

A symmetry plane must act as a mirror: a half body with a symmetry face solves exactly the
problem of the whole, mirror-symmetric body.  With a mirror-symmetric full mesh, the face
between a cell and its mirror image has d = 2 delta n, weight 1/2 and the interpolated
stress / gradient (T_P + R T_P R) / 2, which are the readings taken for the symmetry face; so
the two residuals agree to round-off and the two solutions coincide.  (The printed
one-sided form (I - n n) . sigma_P would drop the normal traction and fails this test.)"""
import numpy as np
import pytest

import oracle as O
from paper_2502_17217_gb300 import inputs as I

L, H, W = 0.6, 0.4, 0.3


def _warp(m, a=0.12):
    """Mirror-symmetric smooth distortion (x odd, y and z even in x), vanishing on the box
    faces and the plane x = 0."""
    p = m.points
    x, y, z = p[:, 0], p[:, 1], p[:, 2]
    sx, sy, sz = np.sin(np.pi * x / L), np.sin(np.pi * y / H), np.sin(np.pi * z / W)
    h = L / 8
    p[:, 0] = x + a * h * sx * sy * sz
    p[:, 1] = y + a * h * np.cos(np.pi * x / (2 * L)) * np.sin(2 * np.pi * y / H) * sz
    p[:, 2] = z + a * h * np.cos(np.pi * x / (2 * L)) * sy * np.sin(2 * np.pi * z / W)
    return m


def _pair(law, nxh=4, ny=4, nz=3, warp=0.12):
    """Full box x in [-L, L] (2 nxh cells) and half box x in [0, L] with a symmetry face at
    x = 0; y = 0 clamped, a mirror-symmetric traction on y = H."""
    full = I.hex_box(2 * nxh, ny, nz, (2 * L, H, W))
    full.points[:, 0] -= L
    full = _warp(full, warp)
    half = _warp(I.hex_box(nxh, ny, nz, (L, H, W)), warp)
    trac = np.array([0.0, -2.0e5, 0.6e5])
    for m in (full, half):
        m.patch("ymin").bc = I.BC_DISP
        ymax = m.patch("ymax")
        ymax.bc = I.BC_TRAC
        ymax.values = np.tile(trac, (ymax.size, 1))
    half.patch("xmin").bc = I.BC_SYMM
    mat = I.Material(law, 2.0e6, 0.3) if law != I.LAW_NEOHOOKEAN else I.Material(law, 0.77e6, 1.67e6)
    return O.Oracle(full, mat), O.Oracle(half, mat), (nxh, ny, nz)


def _maps(shape):
    nxh, ny, nz = shape
    right, mirror = [], []
    for k in range(nz):
        for j in range(ny):
            for i in range(nxh):
                right.append(nxh + i + 2 * nxh * (j + ny * k))
                mirror.append(nxh - 1 - i + 2 * nxh * (j + ny * k))
    return np.array(right), np.array(mirror)


@pytest.mark.parametrize("law", [I.LAW_LINEAR, I.LAW_NEOHOOKEAN])
def test_symmetry_face_is_a_mirror_residual(law):
    of, oh, shape = _pair(law)
    right, mirror = _maps(shape)
    nh = oh.nc
    scale = 1e-3 if law == I.LAW_LINEAR else 0.02
    uh = I.random_field(3, nh, scale)
    uf = np.zeros((of.nc, 3))
    uf[right] = uh
    uf[mirror] = uh * np.array([-1.0, 1.0, 1.0])  # R u with n = e_x
    Rf, Rh = of.residual(uf), oh.residual(uh)
    np.testing.assert_allclose(Rh, Rf[right], atol=1e-11 * np.abs(Rf).max())


@pytest.mark.parametrize("pc", [O.PC_BJACOBI, O.PC_MG])
def test_symmetry_face_is_a_mirror_solution(pc):
    of, oh, shape = _pair(I.LAW_LINEAR)
    right, _ = _maps(shape)
    for o in (of, oh):
        o.mg_setup(coarse_max=10)
    uf, rcf, _ = of.newton(rtol=1e-11, eta=1e-6, pc=pc)
    uh, rch, _ = oh.newton(rtol=1e-11, eta=1e-6, pc=pc)
    assert rcf == 0 and rch == 0
    assert np.linalg.norm(uh - uf[right]) <= 1e-8 * np.linalg.norm(uh)
    assert np.abs(uh[:, 0]).max() > 0  # normal displacements vanish only on the plane itself


def test_symmetry_block_jacobi_inverts_the_block():
    """Sec. 3.1: cells on a symmetry face have the 3x3 diagonal block d I - 2 c n n; the
    block-Jacobi application times the J~ diagonal block gives back the vector."""
    _, oh, _ = _pair(I.LAW_LINEAR)
    nc = oh.nc
    v = I.random_field(5, nc, 1.0)
    z = oh.bjacobi(v)
    # block of cell P applied to z_P: J~ applied to z restricted to the cell's own terms
    # equals v only through the diagonal blocks, so check cell by cell with one-cell vectors
    for P in range(0, nc, 7):
        e = np.zeros((nc, 3))
        e[P] = z[P]
        Jz = oh.jtilde_apply(e)
        np.testing.assert_allclose(Jz[P], v[P], rtol=1e-10, atol=1e-12 * np.abs(v[P]).max())
