"""Symmetry faces on the device (Eq. symm and the symmetry terms of Eq. leastSquaresGrad,
Eq. RhieChow, Sec. 3.1) against the oracle, and the mirror property (GPU)."""
import numpy as np
import pytest

import oracle as O
from paper_2502_17217_gb300 import inputs as I

pytestmark = pytest.mark.gpu
L, H, W = 0.6, 0.4, 0.3


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


def _warp(m, a=0.12):
    p = m.points
    x, y, z = p[:, 0].copy(), p[:, 1].copy(), p[:, 2].copy()
    sx, sy, sz = np.sin(np.pi * x / L), np.sin(np.pi * y / H), np.sin(np.pi * z / W)
    h = L / 8
    p[:, 0] = x + a * h * sx * sy * sz
    p[:, 1] = y + a * h * np.cos(np.pi * x / (2 * L)) * np.sin(2 * np.pi * y / H) * sz
    p[:, 2] = z + a * h * np.cos(np.pi * x / (2 * L)) * sy * np.sin(2 * np.pi * z / W)
    return m


def _case(law, half=True, nxh=6, ny=5, nz=4):
    if half:
        m = _warp(I.hex_box(nxh, ny, nz, (L, H, W)))
        m.patch("xmin").bc = I.BC_SYMM
    else:
        m = I.hex_box(2 * nxh, ny, nz, (2 * L, H, W))
        m.points[:, 0] -= L
        m = _warp(m)
    m.patch("ymin").bc = I.BC_DISP
    ymax = m.patch("ymax")
    ymax.bc = I.BC_TRAC
    ymax.values = np.tile(np.array([0.0, -2.0e5, 0.6e5]), (ymax.size, 1))
    mat = {I.LAW_LINEAR: I.Material(I.LAW_LINEAR, 2.0e6, 0.3),
           I.LAW_NEOHOOKEAN: I.Material(I.LAW_NEOHOOKEAN, 0.77e6, 1.67e6),
           I.LAW_STVK: I.Material(I.LAW_STVK, 2.0e6, 0.3)}[law]
    return I.Case(f"sym_{law}_{half}", m, mat, None)


@pytest.mark.parametrize("law", [I.LAW_LINEAR, I.LAW_NEOHOOKEAN, I.LAW_STVK])
def test_symmetry_residual_jv_and_block_jacobi_parity(law):
    from paper_2502_17217_gb300 import jfnk
    case = _case(law)
    s = jfnk.Solver.from_case(case)
    o = O.Oracle.from_case(case)
    scale = 1e-3 if law == I.LAW_LINEAR else 0.02
    u = I.random_field(3, case.mesh.n_cells, scale)
    v = I.random_field(4, case.mesh.n_cells, 1.0)
    assert _rel(s.residual(u), o.residual(u)) <= 1e-12
    Jo = o.jv(u, v)
    eps = 1e-7 * (1 + np.linalg.norm(u)) / np.linalg.norm(v)
    tol = 1e-12 * (np.linalg.norm(o.residual(u)) / (eps * np.linalg.norm(Jo)) + 1.0)
    assert _rel(s.jv(u, v), Jo) <= tol
    assert _rel(s.precondition(v, pc=jfnk.PC_BJACOBI), o.bjacobi(v)) <= 1e-13


@pytest.mark.parametrize("pc,precision", [(1, 0), (2, 0), (2, 1)])
def test_symmetry_solve_parity_and_mirror(pc, precision):
    """Newton-Krylov solve of the half body against the oracle's, and against the whole
    mirror-symmetric body solved on the device."""
    from paper_2502_17217_gb300 import jfnk
    half, full = _case(I.LAW_LINEAR), _case(I.LAW_LINEAR, half=False)
    kw = dict(pc=pc, precision=precision, newton_rtol=1e-11, mg_coarse_max=20)
    uh, st, rc = jfnk.Solver.from_case(half, **kw).solve()
    uf, stf, rcf = jfnk.Solver.from_case(full, **kw).solve()
    assert rc == 0 and rcf == 0
    o = O.Oracle.from_case(half)
    if pc == jfnk.PC_MG:
        o.mg_setup(coarse_max=20, smoothed=True, sweeps=2)
    uo, rco, _ = o.newton(rtol=1e-11, pc=pc)
    assert rco == 0 and _rel(uh, uo) <= 1e-8
    nxh, ny, nz = 6, 5, 4
    right = np.array([nxh + i + 2 * nxh * (j + ny * k) for k in range(nz) for j in range(ny) for i in range(nxh)])
    assert _rel(uh, uf[right]) <= 1e-8


def test_symmetry_segregated_and_neo_hookean_solve():
    from paper_2502_17217_gb300 import jfnk
    half = _case(I.LAW_LINEAR)
    s = jfnk.Solver.from_case(half, pc=jfnk.PC_BJACOBI, newton_rtol=1e-10)
    us, sts, rcs = s.solve_segregated()
    uo, rco, _ = O.Oracle.from_case(half).segregated(rtol=1e-10, pc=O.PC_BJACOBI)
    assert rcs == 0 and rco == 0 and _rel(us, uo) <= 1e-8
    nh = _case(I.LAW_NEOHOOKEAN)
    un, stn, rcn = jfnk.Solver.from_case(nh, newton_rtol=1e-10).solve(load_steps=2)
    uno, rcno, _ = O.Oracle.from_case(nh).newton(load_steps=2, rtol=1e-10)
    assert rcn == 0 and rcno == 0 and _rel(un, uno) <= 1e-8
