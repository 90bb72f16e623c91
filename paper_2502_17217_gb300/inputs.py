"""Seeded synthetic inputs shared by the CUDA path's tests/bench and by the oracle's tests.

This module holds no arithmetic of the finite-volume method itself: it only builds
face-addressed hexahedral meshes (points, face-point lists, owner/neighbour, patches),
boundary-condition values, material parameters, seeded random vectors and the
manufactured-solution load of Case 1 (Sec. 4.1, App. E).  Both sides of every parity
check consume exactly the arrays produced here.

Random numbers come from a counter-based splitmix64 stream: value i of stream `seed`
is mix(seed * 2^32 + key + (i + 1) * 0x9E3779B97F4A7C15) mapped to [0, 1) with 53 bits
(Steele, Lea and Flood, "Fast splittable pseudorandom number generators", 2014).

Mesh conventions (the face-addressed polyhedral mesh of Sec. 2.3):
  * points  float64 [n_points, 3]
  * faces   CSR: face_ptr int32 [n_faces + 1], face_pts int32 [...]; the right-hand
            normal of the point loop points out of the owner cell
  * owner   int32 [n_faces];  neighbour int32 [n_internal]; internal faces come first,
            ordered by (owner, neighbour), then boundary faces grouped by patch
  * cells   index i + nx*(j + ny*k)
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Boundary-condition and material-law codes (same values as the C headers).
BC_DISP, BC_TRAC, BC_SYMM, BC_EMPTY = 0, 1, 2, 3
LAW_LINEAR, LAW_NEOHOOKEAN, LAW_STVK = 0, 1, 2

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)


def splitmix64_uniform(seed: int, n: int, key: int = 0) -> np.ndarray:
    """n uniform doubles in [0, 1) from the counter-based splitmix64 stream (seed, key)."""
    with np.errstate(over="ignore"):
        base = np.uint64((int(seed) * (1 << 32) + int(key)) & 0xFFFFFFFFFFFFFFFF)
        z = base + (np.arange(1, n + 1, dtype=np.uint64) * _GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def random_field(seed: int, n_cells: int, scale: float = 1.0, key: int = 7, dim: int = 3) -> np.ndarray:
    """Seeded per-cell vector field [n_cells, 3] with entries uniform in [-scale, scale)."""
    v = (2.0 * splitmix64_uniform(seed, 3 * n_cells, key) - 1.0).reshape(n_cells, 3) * scale
    if dim == 2:
        v[:, 2] = 0.0
    return v


@dataclass
class Patch:
    name: str
    start: int
    size: int
    bc: int = BC_TRAC
    values: np.ndarray | None = None  # [size, 3] displacement or traction; None = zero


@dataclass
class Mesh:
    dim: int
    points: np.ndarray
    face_ptr: np.ndarray
    face_pts: np.ndarray
    owner: np.ndarray
    neighbour: np.ndarray
    n_cells: int
    patches: list = field(default_factory=list)
    shape: tuple = ()
    lengths: tuple = ()

    @property
    def n_points(self) -> int:
        return self.points.shape[0]

    @property
    def n_faces(self) -> int:
        return self.owner.shape[0]

    @property
    def n_internal(self) -> int:
        return self.neighbour.shape[0]

    def patch(self, name: str) -> Patch:
        for p in self.patches:
            if p.name == name:
                return p
        raise KeyError(name)

    def nominal_face_centres(self, patch: Patch) -> np.ndarray:
        """Mean of each patch face's corner points (the face centre of an unperturbed box face)."""
        out = np.empty((patch.size, 3))
        for k in range(patch.size):
            f = patch.start + k
            out[k] = self.points[self.face_pts[self.face_ptr[f]:self.face_ptr[f + 1]]].mean(axis=0)
        return out

    def nominal_cell_centres(self) -> np.ndarray:
        """Centres of the unperturbed lattice cells (exact centroids when unperturbed)."""
        nx, ny, nz = self.shape
        lx, ly, lz = self.lengths
        k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        c = np.stack([(i.ravel() + 0.5) * lx / nx, (j.ravel() + 0.5) * ly / ny, (k.ravel() + 0.5) * lz / nz], 1)
        return c


def hex_box(nx: int, ny: int, nz: int, lengths=(1.0, 1.0, 1.0), perturb: float = 0.0,
            seed: int = 0, dim: int = 3) -> Mesh:
    """Structured nx*ny*nz hexahedral box stored as an unstructured face-addressed mesh.

    perturb: interior points are moved by independent U(-perturb*h_a, perturb*h_a) in each
    axis a (h_a = cell size along a).  dim=2 builds a one-cell-thick slab (nz must be 1):
    only x, y are perturbed, both z-layers move together, and the z-min/z-max patches are
    'empty' (front/back planes of a plane-strain model).
    """
    if dim == 2 and nz != 1:
        raise ValueError("2-D meshes are one cell thick")
    lx, ly, lz = lengths
    hx, hy, hz = lx / nx, ly / ny, lz / nz
    px, py, pz = nx + 1, ny + 1, nz + 1
    kk, jj, ii = np.meshgrid(np.arange(pz), np.arange(py), np.arange(px), indexing="ij")
    ii, jj, kk = ii.ravel(), jj.ravel(), kk.ravel()
    pts = np.stack([ii * hx, jj * hy, kk * hz], 1).astype(np.float64)
    # exact end coordinates on the far planes
    pts[ii == nx, 0] = lx
    pts[jj == ny, 1] = ly
    pts[kk == nz, 2] = lz
    if perturb > 0.0:
        if dim == 3:
            inner = (ii > 0) & (ii < nx) & (jj > 0) & (jj < ny) & (kk > 0) & (kk < nz)
            r = 2.0 * splitmix64_uniform(seed, 3 * pts.shape[0], key=1).reshape(-1, 3) - 1.0
            delta = r * perturb * np.array([hx, hy, hz])
            pts[inner] += delta[inner]
        else:
            col = ii + px * jj  # same (x, y) offset for both z-layers
            inner = (ii > 0) & (ii < nx) & (jj > 0) & (jj < ny)
            r = 2.0 * splitmix64_uniform(seed, 2 * px * py, key=1).reshape(-1, 2) - 1.0
            delta = r * perturb * np.array([hx, hy])
            pts[inner, :2] += delta[col[inner]]

    def pid(i, j, k):
        return i + px * (j + py * k)

    def cid(i, j, k):
        return i + nx * (j + ny * k)

    def grid(a, b, c):
        kk_, jj_, ii_ = np.meshgrid(np.arange(c), np.arange(b), np.arange(a), indexing="ij")
        return ii_.ravel(), jj_.ravel(), kk_.ravel()

    quads, own, nei = [], [], []
    # internal faces; the right-hand normal points from owner (lower index) to neighbour
    i, j, k = grid(nx - 1, ny, nz)  # normal +x
    quads.append(np.stack([pid(i + 1, j, k), pid(i + 1, j + 1, k), pid(i + 1, j + 1, k + 1), pid(i + 1, j, k + 1)], 1))
    own.append(cid(i, j, k)); nei.append(cid(i + 1, j, k))
    i, j, k = grid(nx, ny - 1, nz)  # normal +y
    quads.append(np.stack([pid(i, j + 1, k), pid(i, j + 1, k + 1), pid(i + 1, j + 1, k + 1), pid(i + 1, j + 1, k)], 1))
    own.append(cid(i, j, k)); nei.append(cid(i, j + 1, k))
    i, j, k = grid(nx, ny, nz - 1)  # normal +z
    quads.append(np.stack([pid(i, j, k + 1), pid(i + 1, j, k + 1), pid(i + 1, j + 1, k + 1), pid(i, j + 1, k + 1)], 1))
    own.append(cid(i, j, k)); nei.append(cid(i, j, k + 1))
    quads, own, nei = np.concatenate(quads), np.concatenate(own), np.concatenate(nei)
    order = np.lexsort((nei, own))  # by owner, then neighbour
    quads, own, nei = quads[order], own[order], nei[order]
    n_internal = own.shape[0]
    bq, bo, patches = [], [], []
    start = n_internal

    def add_patch(name, q, o):
        nonlocal start
        bq.append(q); bo.append(o)
        patches.append(Patch(name, start, o.shape[0]))
        start += o.shape[0]

    _, j, k = grid(1, ny, nz)
    add_patch("xmin", np.stack([pid(0, j, k), pid(0, j, k + 1), pid(0, j + 1, k + 1), pid(0, j + 1, k)], 1), cid(0, j, k))
    add_patch("xmax", np.stack([pid(nx, j, k), pid(nx, j + 1, k), pid(nx, j + 1, k + 1), pid(nx, j, k + 1)], 1), cid(nx - 1, j, k))
    i, _, k = grid(nx, 1, nz)
    add_patch("ymin", np.stack([pid(i, 0, k), pid(i + 1, 0, k), pid(i + 1, 0, k + 1), pid(i, 0, k + 1)], 1), cid(i, 0, k))
    add_patch("ymax", np.stack([pid(i, ny, k), pid(i, ny, k + 1), pid(i + 1, ny, k + 1), pid(i + 1, ny, k)], 1), cid(i, ny - 1, k))
    i, j, _ = grid(nx, ny, 1)
    add_patch("zmin", np.stack([pid(i, j, 0), pid(i, j + 1, 0), pid(i + 1, j + 1, 0), pid(i + 1, j, 0)], 1), cid(i, j, 0))
    add_patch("zmax", np.stack([pid(i, j, nz), pid(i + 1, j, nz), pid(i + 1, j + 1, nz), pid(i, j + 1, nz)], 1), cid(i, j, nz - 1))
    allq = np.concatenate([quads] + bq)
    face_ptr = np.arange(0, 4 * allq.shape[0] + 1, 4, dtype=np.int32)
    face_pts = np.ascontiguousarray(allq, dtype=np.int32).ravel()
    owner = np.concatenate([own] + bo).astype(np.int32)
    neigh = nei.astype(np.int32)
    m = Mesh(dim, pts, face_ptr, face_pts, owner, neigh, nx * ny * nz, patches, (nx, ny, nz), (lx, ly, lz))
    if dim == 2:
        m.patch("zmin").bc = BC_EMPTY
        m.patch("zmax").bc = BC_EMPTY
    return m


@dataclass
class Material:
    law: int
    p1: float  # E for LAW_LINEAR, mu for LAW_NEOHOOKEAN
    p2: float  # nu for LAW_LINEAR, kappa for LAW_NEOHOOKEAN


@dataclass
class Case:
    name: str
    mesh: Mesh
    material: Material
    body_force: np.ndarray | None  # force per unit volume at each cell [n_cells, 3]
    load_steps: int = 1
    alpha: float = 1.0


# --------------------------------------------------------------------------------------
# Manufactured solution of Case 1 (Sec. 4.1) and its body force (App. E, sign as derived
# from Eq. momentum_lingeom: f_b = -div(sigma(u*)) for a static balance).
# --------------------------------------------------------------------------------------
MMS_AMPLITUDES = (2e-6, 4e-6, 6e-6)


def _mms_factors(x, dim):
    X, Xp, Xpp = np.sin(4 * np.pi * x[:, 0]), 4 * np.pi * np.cos(4 * np.pi * x[:, 0]), -16 * np.pi ** 2 * np.sin(4 * np.pi * x[:, 0])
    Y, Yp, Ypp = np.sin(2 * np.pi * x[:, 1]), 2 * np.pi * np.cos(2 * np.pi * x[:, 1]), -4 * np.pi ** 2 * np.sin(2 * np.pi * x[:, 1])
    if dim == 3:
        Z, Zp, Zpp = np.sin(np.pi * x[:, 2]), np.pi * np.cos(np.pi * x[:, 2]), -np.pi ** 2 * np.sin(np.pi * x[:, 2])
    else:
        Z, Zp, Zpp = np.ones_like(X), np.zeros_like(X), np.zeros_like(X)
    return (X, Xp, Xpp), (Y, Yp, Ypp), (Z, Zp, Zpp)


def mms_displacement(x: np.ndarray, dim: int = 3, amplitudes=MMS_AMPLITUDES) -> np.ndarray:
    """u* = a * sin(4 pi x) sin(2 pi y) sin(pi z)  (dim=2: the sin(pi z) factor and a_z dropped)."""
    (X, _, _), (Y, _, _), (Z, _, _) = _mms_factors(np.atleast_2d(x), dim)
    a = np.array(amplitudes, dtype=np.float64)
    if dim == 2:
        a = a.copy(); a[2] = 0.0
    return (X * Y * Z)[:, None] * a[None, :]


def mms_body_force(x: np.ndarray, E: float, nu: float, dim: int = 3, amplitudes=MMS_AMPLITUDES) -> np.ndarray:
    """Body force per unit volume that makes u* an equilibrium field of Hooke's law.

    u_j = a_j phi(x) with separable phi; div sigma = mu lap(u) + (lam + mu) grad(div u), so
    f_b,i = -[mu a_i lap(phi) + (lam + mu) sum_k a_k d_i d_k phi].  The problem's Lame pair
    is the usual one for (E, nu).
    """
    x = np.atleast_2d(x)
    mu = E / (2.0 * (1.0 + nu))
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    (X, Xp, Xpp), (Y, Yp, Ypp), (Z, Zp, Zpp) = _mms_factors(x, dim)
    a = np.array(amplitudes, dtype=np.float64)
    if dim == 2:
        a = a.copy(); a[2] = 0.0
    H = np.empty((x.shape[0], 3, 3))
    H[:, 0, 0] = Xpp * Y * Z; H[:, 1, 1] = X * Ypp * Z; H[:, 2, 2] = X * Y * Zpp
    H[:, 0, 1] = H[:, 1, 0] = Xp * Yp * Z
    H[:, 0, 2] = H[:, 2, 0] = Xp * Y * Zp
    H[:, 1, 2] = H[:, 2, 1] = X * Yp * Zp
    lap = H[:, 0, 0] + H[:, 1, 1] + H[:, 2, 2]
    f = -(mu * lap[:, None] * a[None, :] + (lam + mu) * np.einsum("nik,k->ni", H, a))
    if dim == 2:
        f[:, 2] = 0.0
    return f


# --------------------------------------------------------------------------------------
# The workloads
# --------------------------------------------------------------------------------------
def case_mms2d(n: int = 32, perturb: float = 0.0, seed: int = 0) -> Case:
    """2-D plane-strain MMS on the unit square, n x n cells, one cell thick (thickness 1/n).

    E = 200 GPa, nu = 0.3; prescribed displacement u*(face centre) on the four sides
    (u* vanishes there); body force from the manufactured solution at nominal cell centres.
    """
    m = hex_box(n, n, 1, (1.0, 1.0, 1.0 / n), perturb=perturb, seed=seed, dim=2)
    E, nu = 200e9, 0.3
    for name in ("xmin", "xmax", "ymin", "ymax"):
        p = m.patch(name)
        p.bc = BC_DISP
        p.values = mms_displacement(m.nominal_face_centres(p), dim=2)
    fb = mms_body_force(m.nominal_cell_centres(), E, nu, dim=2)
    return Case(f"mms2d_{n}x{n}", m, Material(LAW_LINEAR, E, nu), fb)


def case_cantilever(nx: int = 200, ny: int = 20, nz: int = 20, lengths=(1.0, 0.1, 0.1),
                    perturb: float = 0.15, seed: int = 2, E: float = 200e9, nu: float = 0.3,
                    traction=(0.0, 1e6, 0.0)) -> Case:
    """3-D linear-elastic cantilever: x-min clamped, uniform traction on x-max, rest traction-free."""
    m = hex_box(nx, ny, nz, lengths, perturb=perturb, seed=seed, dim=3)
    m.patch("xmin").bc = BC_DISP
    xmax = m.patch("xmax")
    xmax.bc = BC_TRAC
    xmax.values = np.tile(np.asarray(traction, np.float64), (xmax.size, 1))
    return Case(f"cantilever_{nx}x{ny}x{nz}", m, Material(LAW_LINEAR, E, nu), None)


def case_nh_beam(nx: int = 256, ny: int = 32, nz: int = 32, lengths=(1.0, 0.125, 0.125),
                 end_uy: float = 0.5, load_steps: int = 10, mu: float = 0.38e6, kappa: float = 8.3e6,
                 perturb: float = 0.0, seed: int = 3) -> Case:
    """3-D neo-Hookean total-Lagrangian beam: x-min clamped, x-max moved by (0, end_uy, 0)
    (ramped over the load steps), other faces traction-free."""
    m = hex_box(nx, ny, nz, lengths, perturb=perturb, seed=seed, dim=3)
    m.patch("xmin").bc = BC_DISP
    xmax = m.patch("xmax")
    xmax.bc = BC_DISP
    xmax.values = np.tile(np.array([0.0, end_uy, 0.0]), (xmax.size, 1))
    return Case(f"nh_beam_{nx}x{ny}x{nz}", m, Material(LAW_NEOHOOKEAN, mu, kappa), None, load_steps=load_steps)


def case_dynamic_beam(nx: int = 3, ny: int = 30, nz: int = 3, traction=(50e3, 50e3, 0.0), E: float = 15.293e6,
                      nu: float = 0.3, law: int = LAW_NEOHOOKEAN):
    """Case 6 of Sec. 4 (vibration of a cantilevered column): 0.2 x 2 x 0.2 m with y up, the
    bottom face (y = 0) clamped, a sudden constant traction on the upper face (y = 2), the
    other faces traction-free; neo-Hookean with E = 15.293 MPa, nu = 0.3 (density 1000 kg/m^3
    and dt = 1 ms are run parameters), chosen by the paper for a 1 Hz first frequency.  The
    paper's meshes are 3x30x3 .. 24x240x24 cells.  Returns (case, probe cell): the probe is the
    cell at the centre of the upper face (one of the four central ones for even counts)."""
    m = hex_box(nx, ny, nz, (0.2, 2.0, 0.2))
    ny_ = m.shape[1]
    for pt in m.patches:
        if pt.name == "ymin":
            pt.bc = BC_DISP
            pt.values = np.zeros((pt.size, 3))
        elif pt.name == "ymax":
            pt.bc = BC_TRAC
            pt.values = np.tile(np.asarray(traction, float), (pt.size, 1))
    if law == LAW_NEOHOOKEAN:
        mu, kappa = E / (2 * (1 + nu)), E / (3 * (1 - 2 * nu))
        mat = Material(LAW_NEOHOOKEAN, mu, kappa)
    else:  # Hooke or St. Venant-Kirchhoff: E, nu
        mat = Material(law, E, nu)
    i, k = nx // 2, nz // 2
    probe = i + nx * ((ny_ - 1) + ny_ * k)
    return Case(f"dynamic_beam_{nx}x{ny}x{nz}", m, mat, None), probe


def batch_sizes(n_problems: int = 512, lo: int = 1000, hi: int = 64000, seed: int = 4):
    """Cell-count targets drawn log-uniform in [lo, hi] and box shapes nx:ny:nz ~ 4:1:1 (each >= 4)."""
    r = splitmix64_uniform(seed, 4 * n_problems, key=11).reshape(n_problems, 4)
    out = []
    for p in range(n_problems):
        n = math.exp(math.log(lo) + r[p, 0] * (math.log(hi) - math.log(lo)))
        s = (n / 4.0) ** (1.0 / 3.0)  # nx:ny:nz = 4:1:1 gives 4 s^3 cells
        nx, ny, nz = max(4, round(4 * s)), max(4, round(s)), max(4, round(s))
        E = 1e9 + r[p, 1] * (300e9 - 1e9)
        nu = 0.2 + r[p, 2] * 0.25
        out.append((nx, ny, nz, E, nu, float(r[p, 3])))
    return out


def case_batch_member(nx, ny, nz, E, nu, u01, index: int, seed: int = 4, perturb: float = 0.15) -> Case:
    """One box of the batched workload: cantilever-like, random traction direction and magnitude."""
    r = splitmix64_uniform(seed, 3, key=1000 + index)
    zc = 2.0 * r[0] - 1.0
    phi = 2.0 * math.pi * r[1]
    sxy = math.sqrt(max(0.0, 1.0 - zc * zc))
    mag = 0.1e6 + u01 * 0.9e6
    t = (mag * sxy * math.cos(phi), mag * sxy * math.sin(phi), mag * zc)
    h = 0.01
    return case_cantilever(nx, ny, nz, (nx * h, ny * h, nz * h), perturb=perturb, seed=seed * 100000 + index,
                           E=E, nu=nu, traction=t)


def serving_requests(n: int, lo: int = 2000, hi: int = 1000000, seed: int = 5, frac_nh: float = 0.3):
    """Solve requests of the serving workload: box meshes (4:1:1, +-15% interior-node
    perturbation) with cell counts log-uniform in [lo, hi]; a fraction frac_nh are neo-Hookean
    (mu = 0.38 MPa, kappa = 8.3 MPa, x-max moved transversally by 5% of the length over 2 load
    steps), the others Hooke with a random material and end traction as in the batch workload.
    Returns a list of (case, load_steps)."""
    r = splitmix64_uniform(seed, 5 * n, key=21).reshape(n, 5)
    out = []
    for k in range(n):
        cells = math.exp(math.log(lo) + r[k, 0] * (math.log(hi) - math.log(lo)))
        s = (cells / 4.0) ** (1.0 / 3.0)
        nx, ny, nz = max(4, round(4 * s)), max(4, round(s)), max(4, round(s))
        h = 0.01
        if r[k, 1] < frac_nh:
            c = case_nh_beam(nx, ny, nz, (nx * h, ny * h, nz * h), end_uy=0.05 * nx * h, load_steps=2,
                             perturb=0.15, seed=seed * 100000 + k)
            out.append((c, 2))
        else:
            E = 1e9 + r[k, 2] * (300e9 - 1e9)
            nu = 0.2 + r[k, 3] * 0.25
            out.append((case_batch_member(nx, ny, nz, E, nu, float(r[k, 4]), index=k, seed=seed), 1))
    return out
