"""ctypes wrapper of the plain-C FP64 oracle (TEST INFRASTRUCTURE ONLY).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package.  It shares no code with the CUDA path: it is built from
``oracle/jfnk_oracle.c`` with the host C compiler and consumes the same seeded inputs
(``paper_2502_17217_gb300.inputs``) as the CUDA path does.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "jfnk_oracle.c")
_LIB = os.path.join(_HERE, "libjfnk_oracle.so")
_lib = None

PC_NONE, PC_BJACOBI, PC_MG = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with plain -O2 (no fast-math, no target-specific flags)."""
    hdr = os.path.join(_HERE, "jfnk_oracle.h")
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(os.path.getmtime(_SRC), os.path.getmtime(hdr)):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fno-fast-math", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Stats(C.Structure):
    _fields_ = [("newton_its", C.c_int), ("gmres_its", C.c_int), ("residual_evals", C.c_int), ("status", C.c_int),
                ("final_rel_res", C.c_double), ("hist", C.c_double * 64), ("n_hist", C.c_int)]


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        d, i, vp = C.c_double, C.c_int, C.c_void_p
        sig = {
            "orc_create": (vp, [i, i, vp, i, vp, vp, vp, i, vp, i]),
            "orc_destroy": (None, [vp]),
            "orc_error": (C.c_char_p, [vp]),
            "orc_set_patch": (i, [vp, i, i, i, vp]),
            "orc_set_material": (i, [vp, i, d, d]),
            "orc_set_body_force": (i, [vp, vp]),
            "orc_set_alpha": (None, [vp, d, d]),
            "orc_set_load_factor": (None, [vp, d]),
            "orc_prepare": (i, [vp]),
            "orc_get_geometry": (None, [vp, vp, vp, vp, vp]),
            "orc_gradient": (None, [vp, vp, vp]),
            "orc_traction_operator": (None, [vp, vp, vp]),
            "orc_cauchy_stress": (None, [vp, vp, vp]),
            "orc_residual": (None, [vp, vp, vp]),
            "orc_jv": (None, [vp, vp, vp, vp, vp]),
            "orc_jtilde_apply": (None, [vp, vp, vp]),
            "orc_jtilde_diag": (None, [vp, vp]),
            "orc_bjacobi": (None, [vp, vp, vp]),
            "orc_mg_setup": (i, [vp, d, i, i]),
            "orc_mg_setup_ex": (i, [vp, d, i, i, i]),
            "orc_mg_set_sweeps": (None, [vp, i, i]),
            "orc_mg_levels": (i, [vp, vp]),
            "orc_mg_aggregates": (i, [vp, i, vp]),
            "orc_mg_vcycle": (None, [vp, vp, vp]),
            "orc_gmres": (i, [vp, vp, vp, vp, vp, i, d, i, i, vp, vp]),
            "orc_newton": (i, [vp, vp, i, d, d, i, i, d, i, vp]),
            "orc_lgmres": (i, [vp, vp, vp, vp, vp, i, i, d, i, i, vp, vp]),
            "orc_newton_ex": (i, [vp, vp, i, d, d, i, i, i, d, i, vp]),
            "orc_segregated": (i, [vp, vp, i, d, d, i, d, i, i, vp]),
            "orc_set_dynamics": (i, [vp, d, d]),
            "orc_dynamic": (i, [vp, vp, i, d, d, i, i, i, d, i, vp, i, vp]),
            "orc_set_updated_lagrangian": (i, [vp, i]),
            "orc_ul_state": (None, [vp, vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(_lib, name)
            f.restype = res
            f.argtypes = args
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


class Oracle:
    """One problem (mesh + boundary conditions + material) held by the C oracle."""

    def __init__(self, mesh, material=None, body_force=None, alpha=1.0, alpha_pc=1.0, prepare=True):
        L = lib()
        self.mesh = mesh
        self.nc = mesh.n_cells
        self._keep = [np.ascontiguousarray(mesh.points, np.float64), np.ascontiguousarray(mesh.face_ptr, np.int32),
                      np.ascontiguousarray(mesh.face_pts, np.int32), np.ascontiguousarray(mesh.owner, np.int32),
                      np.ascontiguousarray(mesh.neighbour, np.int32)]
        pts, fp, fq, ow, ne = self._keep
        self.h = L.orc_create(mesh.dim, mesh.n_points, _p(pts), mesh.n_faces, _p(fp), _p(fq), _p(ow),
                              mesh.n_internal, _p(ne), mesh.n_cells)
        for patch in mesh.patches:
            vals = None if patch.values is None else _f64(patch.values, (patch.size, 3))
            self._check(L.orc_set_patch(self.h, patch.start, patch.size, patch.bc, _p(vals)))
        if material is not None:
            self._check(L.orc_set_material(self.h, material.law, material.p1, material.p2))
        if body_force is not None:
            fb = _f64(body_force, (self.nc, 3))
            L.orc_set_body_force(self.h, _p(fb))
        L.orc_set_alpha(self.h, alpha, alpha_pc)
        if prepare:
            self._check(L.orc_prepare(self.h))

    @classmethod
    def from_case(cls, case, **kw):
        return cls(case.mesh, case.material, case.body_force, alpha=case.alpha, **kw)

    def _check(self, rc):
        if rc < 0:
            raise RuntimeError(lib().orc_error(self.h).decode())
        return rc

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_destroy(self.h)
            self.h = None

    def set_body_force(self, fb):
        fb = _f64(fb, (self.nc, 3))
        lib().orc_set_body_force(self.h, _p(fb))

    def set_load_factor(self, lam):
        lib().orc_set_load_factor(self.h, float(lam))

    def prepare(self):
        self._check(lib().orc_prepare(self.h))

    def geometry(self):
        nf = self.mesh.n_faces
        Sf, Cf, V, Cc = np.zeros((nf, 3)), np.zeros((nf, 3)), np.zeros(self.nc), np.zeros((self.nc, 3))
        lib().orc_get_geometry(self.h, _p(Sf), _p(Cf), _p(V), _p(Cc))
        return Sf, Cf, V, Cc

    def gradient(self, u):
        u = _f64(u, (self.nc, 3))
        g = np.zeros((self.nc, 3, 3))
        lib().orc_gradient(self.h, _p(u), _p(g))
        return g

    def traction_operator(self, grad):
        grad = _f64(grad, (self.nc, 3, 3))
        T = np.zeros((self.nc, 3, 3))
        lib().orc_traction_operator(self.h, _p(grad), _p(T))
        return T

    def cauchy_stress(self, grad_cell):
        g = _f64(grad_cell, (3, 3))
        s = np.zeros((3, 3))
        lib().orc_cauchy_stress(self.h, _p(g), _p(s))
        return s

    def residual(self, u):
        u = _f64(u, (self.nc, 3))
        R = np.zeros((self.nc, 3))
        lib().orc_residual(self.h, _p(u), _p(R))
        return R

    def jv(self, u, v, R_u=None):
        u, v = _f64(u, (self.nc, 3)), _f64(v, (self.nc, 3))
        Ru = None if R_u is None else _f64(R_u, (self.nc, 3))
        out = np.zeros((self.nc, 3))
        lib().orc_jv(self.h, _p(u), _p(v), _p(Ru), _p(out))
        return out

    def jtilde_apply(self, v):
        v = _f64(v, (self.nc, 3))
        out = np.zeros((self.nc, 3))
        lib().orc_jtilde_apply(self.h, _p(v), _p(out))
        return out

    def jtilde_diag(self):
        d = np.zeros(self.nc)
        lib().orc_jtilde_diag(self.h, _p(d))
        return d

    def bjacobi(self, v):
        v = _f64(v, (self.nc, 3))
        z = np.zeros((self.nc, 3))
        lib().orc_bjacobi(self.h, _p(v), _p(z))
        return z

    def mg_setup(self, theta=0.25, max_levels=25, coarse_max=1000, smoothed=False, sweeps=1):
        lib().orc_mg_set_sweeps(self.h, sweeps, sweeps)
        return self._check(lib().orc_mg_setup_ex(self.h, theta, max_levels, coarse_max, 1 if smoothed else 0))

    def mg_levels(self):
        n = lib().orc_mg_levels(self.h, None)
        s = np.zeros(max(n, 1), np.int32)
        lib().orc_mg_levels(self.h, _p(s))
        return list(s[:n])

    def mg_aggregates(self, level):
        sizes = self.mg_levels()
        a = np.zeros(sizes[level], np.int32)
        self._check(lib().orc_mg_aggregates(self.h, level, _p(a)))
        return a

    def mg_vcycle(self, v):
        v = _f64(v, (self.nc, 3))
        z = np.zeros((self.nc, 3))
        lib().orc_mg_vcycle(self.h, _p(v), _p(z))
        return z

    def gmres(self, u, b, m=30, eta=1e-3, max_restarts=100, pc=PC_BJACOBI, R_u=None):
        u, b = _f64(u, (self.nc, 3)), _f64(b, (self.nc, 3))
        Ru = self.residual(u) if R_u is None else _f64(R_u, (self.nc, 3))
        x = np.zeros((self.nc, 3))
        its, rel = C.c_int(0), C.c_double(0)
        rc = lib().orc_gmres(self.h, _p(u), _p(Ru), _p(b), _p(x), m, eta, max_restarts, pc, C.byref(its), C.byref(rel))
        return x, rc, its.value, rel.value

    def lgmres(self, u, b, m=30, aug=2, eta=1e-3, max_restarts=100, pc=PC_BJACOBI, R_u=None):
        """Loose GMRES (Sec. 4.2): m columns per cycle, of which up to `aug` are corrections
        kept from earlier cycles; aug = 0 is GMRES(m)."""
        u, b = _f64(u, (self.nc, 3)), _f64(b, (self.nc, 3))
        Ru = self.residual(u) if R_u is None else _f64(R_u, (self.nc, 3))
        x = np.zeros((self.nc, 3))
        its, rel = C.c_int(0), C.c_double(0)
        rc = lib().orc_lgmres(self.h, _p(u), _p(Ru), _p(b), _p(x), m, aug, eta, max_restarts, pc, C.byref(its),
                              C.byref(rel))
        return x, rc, its.value, rel.value

    def set_updated_lagrangian(self, on=True):
        """App. A updated-Lagrangian form (neo-Hookean, 3-D): newton() then solves each load
        step for the increment on the last converged configuration and returns the total
        displacement; the mesh is left in the final configuration (geometry() shows it)."""
        self._check(lib().orc_set_updated_lagrangian(self.h, 1 if on else 0))

    def ul_state(self):
        """Total deformation gradient of the last converged step, [n_cells, 3, 3]."""
        F = np.zeros((self.nc, 3, 3))
        lib().orc_ul_state(self.h, _p(F))
        return F

    def set_dynamics(self, rho, dt):
        """Inertia with density rho and time step dt (BDF2, from rest); before mg_setup."""
        self._check(lib().orc_set_dynamics(self.h, float(rho), float(dt)))

    def dynamic(self, n_steps, rtol=1e-8, atol=1e-50, max_newton=50, m=30, aug=0, eta=1e-3, pc=PC_BJACOBI,
                probe_cell=-1):
        """n_steps time steps from the stored state (predictor + Newton-Krylov per step);
        returns (u, status, stats, probe [n_steps, 3] displacement of probe_cell)."""
        u = np.zeros((self.nc, 3))
        probe = np.zeros((max(1, n_steps), 3))
        st = Stats()
        rc = lib().orc_dynamic(self.h, _p(u), n_steps, rtol, atol, max_newton, m, aug, eta, pc, C.byref(st),
                               int(probe_cell), _p(probe))
        return u, rc, st, probe[:n_steps]

    def segregated(self, u0=None, load_steps=1, rtol=1e-8, atol=1e-50, max_outer=100000, inner_tol=0.9,
                   max_inner=1000, pc=PC_BJACOBI):
        """The segregated quasi-Newton method of Sec. 3.1 (J~ per component, PCG to inner_tol);
        stats.newton_its = outer iterations, stats.gmres_its = CG iterations."""
        u = np.zeros((self.nc, 3)) if u0 is None else _f64(u0, (self.nc, 3)).copy()
        st = Stats()
        rc = lib().orc_segregated(self.h, _p(u), load_steps, rtol, atol, max_outer, inner_tol, max_inner, pc,
                                  C.byref(st))
        return u, rc, st

    def newton(self, u0=None, load_steps=1, rtol=1e-8, atol=1e-50, max_newton=50, m=30, eta=1e-3, pc=PC_BJACOBI,
               aug=0):
        u = np.zeros((self.nc, 3)) if u0 is None else _f64(u0, (self.nc, 3)).copy()
        st = Stats()
        rc = lib().orc_newton_ex(self.h, _p(u), load_steps, rtol, atol, max_newton, m, aug, eta, pc, C.byref(st))
        return u, rc, st
