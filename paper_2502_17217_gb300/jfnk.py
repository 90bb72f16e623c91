"""Thin ctypes binding of the C ABI in include/jfnk_gb300.h (argument marshalling only).

Every call goes to libjfnk_gb300.so; there is no Python or CPU fallback: importing the
binding without the built library raises.  Host arrays are numpy float64 [n_cells, 3];
device arrays are torch CUDA float64 tensors of the same shape (PyTorch supplies device
memory and streams only).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import inputs as _inputs

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libjfnk_gb300.so")

OK, EINVAL, ENOMEM, ECUDA, ESTATE, DIVERGED, MAXIT, LS_FAILED, GMRES_STAGNATED = 0, -1, -2, -3, -4, -5, -6, -7, -8
BC_DISP, BC_TRAC, BC_SYMM, BC_EMPTY = 0, 1, 2, 3
LAW_LINEAR, LAW_NEOHOOKEAN, LAW_STVK = 0, 1, 2
PC_NONE, PC_BJACOBI, PC_MG = 0, 1, 2
MEM_HOST, MEM_DEVICE = 0, 1
PREC_FP64, PREC_MIXED = 0, 1
PC_RIGHT, PC_LEFT = 0, 1
FORM_TOTAL_LAGRANGIAN, FORM_UPDATED_LAGRANGIAN = 0, 1

# every function declared in include/jfnk_gb300.h
EXPORTS = [
    "jfnk_default_options", "jfnk_create", "jfnk_destroy", "jfnk_last_error", "jfnk_set_options",
    "jfnk_set_mesh", "jfnk_set_patch", "jfnk_set_material", "jfnk_set_body_force", "jfnk_set_load_factor",
    "jfnk_setup", "jfnk_residual", "jfnk_residual_noalloc", "jfnk_jv", "jfnk_precondition", "jfnk_solve", "jfnk_get_geometry",
    "jfnk_get_gradient", "jfnk_get_permutation", "jfnk_profile_enable", "jfnk_profile_get", "jfnk_profile_reset",
    "jfnk_launch_count", "jfnk_device_bytes", "jfnk_convert_f32_to_f64", "jfnk_batch_add", "jfnk_batch_size",
    "jfnk_batch_problem_cells", "jfnk_batch_stats", "jfnk_measure_fp64_rate", "jfnk_get_tuning", "jfnk_set_tuning",
    "jfnk_solve_segregated", "jfnk_solve_dynamic", "jfnk_dynamic_reset", "jfnk_synchronize",
    "jfnk_set_mesh_hex", "jfnk_hex_patch", "jfnk_dynamic_get_state", "jfnk_dynamic_set_state",
    "jfnk_mg_hierarchy", "jfnk_set_formulation",
]


class Options(C.Structure):
    _fields_ = [("device", C.c_int), ("gmres_restart", C.c_int), ("gmres_eta", C.c_double),
                ("gmres_max_restarts", C.c_int), ("newton_rtol", C.c_double), ("newton_atol", C.c_double),
                ("newton_max_its", C.c_int), ("line_search_max", C.c_int), ("alpha_residual", C.c_double),
                ("alpha_pc", C.c_double), ("jv_eps_scale", C.c_double), ("pc", C.c_int), ("precision", C.c_int),
                ("reorth", C.c_int), ("renumber", C.c_int), ("mg_max_levels", C.c_int), ("mg_coarse_max", C.c_int),
                ("mg_theta", C.c_double), ("mg_smooth_sweeps", C.c_int), ("mg_smoothed", C.c_int),
                ("autotune", C.c_int), ("gmres_aug", C.c_int), ("seg_inner_tol", C.c_double),
                ("seg_max_outer", C.c_int), ("seg_max_inner", C.c_int), ("density", C.c_double), ("dt", C.c_double),
                ("pc_side", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("newton_its", C.c_int), ("gmres_its", C.c_int), ("residual_evals", C.c_int),
                ("load_steps_done", C.c_int), ("status", C.c_int), ("final_rel_res", C.c_double),
                ("final_abs_res", C.c_double), ("solve_ms", C.c_double), ("hist", C.c_double * 64), ("n_hist", C.c_int),
                ("reorth_its", C.c_int), ("jv_products", C.c_int), ("arnoldi_cols", C.c_double),
                ("reorth_cols", C.c_double)]


_lib = None


def load():
    """Loads libjfnk_gb300.so (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() (no CPU fallback exists)")
    L = C.CDLL(LIB_PATH)
    vp, i, d, i32p, dp = C.c_void_p, C.c_int, C.c_double, C.c_void_p, C.c_void_p
    sig = {
        "jfnk_default_options": (None, [C.POINTER(Options)]),
        "jfnk_create": (i, [C.POINTER(vp), C.POINTER(Options)]),
        "jfnk_destroy": (i, [vp]),
        "jfnk_last_error": (C.c_char_p, [vp]),
        "jfnk_set_options": (i, [vp, C.POINTER(Options)]),
        "jfnk_set_mesh": (i, [vp, i, C.c_int32, dp, C.c_int32, i32p, i32p, i32p, C.c_int32, i32p, C.c_int32]),
        "jfnk_set_patch": (i, [vp, C.c_int32, C.c_int32, i, dp]),
        "jfnk_set_material": (i, [vp, i, d, d]),
        "jfnk_set_body_force": (i, [vp, dp]),
        "jfnk_set_load_factor": (i, [vp, d]),
        "jfnk_setup": (i, [vp]),
        "jfnk_residual": (i, [vp, dp, dp, i, vp]),
        "jfnk_residual_noalloc": (i, [vp, dp, dp, vp]),
        "jfnk_jv": (i, [vp, dp, dp, dp, i, vp]),
        "jfnk_precondition": (i, [vp, dp, dp, i, i, vp]),
        "jfnk_solve": (i, [vp, dp, i, i, C.POINTER(Stats), vp]),
        "jfnk_solve_segregated": (i, [vp, dp, i, i, C.POINTER(Stats), vp]),
        "jfnk_solve_dynamic": (i, [vp, dp, i, i, C.c_int32, dp, i, C.POINTER(Stats), vp]),
        "jfnk_dynamic_reset": (i, [vp]),
        "jfnk_dynamic_get_state": (i, [vp, dp]),
        "jfnk_dynamic_set_state": (i, [vp, dp]),
        "jfnk_synchronize": (i, [vp]),
        "jfnk_set_mesh_hex": (i, [vp, i, i, i, dp, i]),
        "jfnk_hex_patch": (i, [i, i, i, i, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
        "jfnk_get_geometry": (i, [vp, dp, dp, dp, dp]),
        "jfnk_get_gradient": (i, [vp, dp]),
        "jfnk_get_permutation": (i, [vp, i32p]),
        "jfnk_profile_enable": (i, [vp, i]),
        "jfnk_profile_get": (i, [vp, C.c_char_p, C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
        "jfnk_profile_reset": (i, [vp]),
        "jfnk_launch_count": (C.c_int64, [vp]),
        "jfnk_device_bytes": (C.c_int64, [vp]),
        "jfnk_convert_f32_to_f64": (i, [vp, vp, C.c_int64, vp]),
        "jfnk_batch_add": (i, [vp, vp, C.POINTER(C.c_int32)]),
        "jfnk_batch_size": (i, [vp]),
        "jfnk_batch_problem_cells": (i, [vp, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
        "jfnk_batch_stats": (i, [vp, C.POINTER(Stats)]),
        "jfnk_measure_fp64_rate": (i, [i, C.POINTER(C.c_double)]),
        "jfnk_get_tuning": (i, [vp, i32p, i]),
        "jfnk_set_tuning": (i, [vp, i32p, i]),
        "jfnk_mg_hierarchy": (i, [vp, i, vp, vp, vp]),
        "jfnk_set_formulation": (i, [vp, i]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


class JfnkError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"[{code}] {msg}")
        self.code = code


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return a.ctypes.data_as(C.c_void_p)


def default_options(**kw) -> Options:
    o = Options()
    load().jfnk_default_options(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def _is_device(a):
    return hasattr(a, "is_cuda") and a.is_cuda


def _stream(a):
    """The caller's current torch stream for device arrays; torch's default stream (handle 0)
    is passed as cudaStreamLegacy, so that the library's work is ordered with the torch work
    around it (a NULL stream would select the context's own, unordered, stream)."""
    if _is_device(a):
        import torch
        h = torch.cuda.current_stream(a.device).cuda_stream
        return C.c_void_p(h if h else 1)  # 1 = cudaStreamLegacy
    return None


class Solver:
    """One problem on one GPU: mesh, boundary conditions, material, then the hot-path calls."""

    def __init__(self, mesh, material, body_force=None, options: Options | None = None, **opt_kw):
        self.L = load()
        self.options = options if options is not None else default_options(**opt_kw)
        h = C.c_void_p()
        rc = self.L.jfnk_create(C.byref(h), C.byref(self.options))
        if rc != OK:
            raise JfnkError(rc, "jfnk_create failed (no usable CUDA device?)")
        self.h = h
        self.mesh = mesh
        self.nc = mesh.n_cells
        self._keep = [np.ascontiguousarray(mesh.points, np.float64), np.ascontiguousarray(mesh.face_ptr, np.int32),
                      np.ascontiguousarray(mesh.face_pts, np.int32), np.ascontiguousarray(mesh.owner, np.int32),
                      np.ascontiguousarray(mesh.neighbour, np.int32)]
        pts, fp, fq, ow, ne = self._keep
        self._check(self.L.jfnk_set_mesh(h, mesh.dim, mesh.n_points, _ptr(pts), mesh.n_faces, _ptr(fp), _ptr(fq),
                                         _ptr(ow), mesh.n_internal, _ptr(ne), mesh.n_cells))
        for p in mesh.patches:
            vals = None if p.values is None else np.ascontiguousarray(p.values, np.float64).reshape(p.size, 3)
            self._check(self.L.jfnk_set_patch(h, p.start, p.size, p.bc, _ptr(vals)))
        self._check(self.L.jfnk_set_material(h, material.law, material.p1, material.p2))
        if body_force is not None:
            self.set_body_force(body_force)

    @classmethod
    def from_case(cls, case, **kw):
        kw.setdefault("alpha_residual", case.alpha)
        return cls(case.mesh, case.material, case.body_force, **kw)

    def _check(self, rc):
        if rc != OK:
            raise JfnkError(rc, self.L.jfnk_last_error(self.h).decode())
        return rc

    def close(self):
        if getattr(self, "h", None):
            self.L.jfnk_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_body_force(self, fb):
        fb = np.ascontiguousarray(fb, np.float64).reshape(self.nc, 3)
        self._check(self.L.jfnk_set_body_force(self.h, _ptr(fb)))

    def set_load_factor(self, lam):
        self._check(self.L.jfnk_set_load_factor(self.h, float(lam)))

    def set_formulation(self, form):
        """FORM_TOTAL_LAGRANGIAN (default) or FORM_UPDATED_LAGRANGIAN (App. A); next set-up."""
        self._check(self.L.jfnk_set_formulation(self.h, int(form)))

    def set_options(self, **kw):
        for k, v in kw.items():
            setattr(self.options, k, v)
        self._check(self.L.jfnk_set_options(self.h, C.byref(self.options)))

    def setup(self):
        self._check(self.L.jfnk_setup(self.h))

    # -------- hot path: host numpy arrays or torch CUDA tensors (float64, [n_cells, 3])
    def _io(self, *arrs):
        dev = _is_device(arrs[0])
        return (MEM_DEVICE if dev else MEM_HOST), _stream(arrs[0])

    def _out_like(self, a):
        if _is_device(a):
            import torch
            return torch.empty((self.nc, 3), dtype=torch.float64, device=a.device)
        return np.zeros((self.nc, 3))

    def _in(self, a):
        if _is_device(a):
            return a.contiguous()
        return np.ascontiguousarray(a, np.float64).reshape(self.nc, 3)

    def residual(self, u, out=None):
        u = self._in(u)
        R = self._out_like(u) if out is None else out
        mem, s = self._io(u)
        self._check(self.L.jfnk_residual(self.h, _ptr(u), _ptr(R), mem, s))
        return R

    def residual_noalloc(self, u, out=None):
        """R(u) through the entry point that allocates nothing (jfnk_residual_noalloc).

        u and out must be contiguous float64 torch CUDA tensors of shape (n_cells, 3) on the
        context's device; anything else raises TypeError before the library is called.  With
        out=None the result tensor is allocated here, by torch, before the call."""
        dev = self.options.device
        for name, a in (("u", u), ("out", out)):
            if a is None and name == "out":
                continue
            if not (_is_device(a) and a.dtype.is_floating_point and a.element_size() == 8 and a.is_contiguous()
                    and tuple(a.shape) == (self.nc, 3) and a.device.index == dev):
                raise TypeError(f"residual_noalloc: {name} must be a contiguous float64 CUDA tensor of shape "
                                f"({self.nc}, 3) on cuda:{dev}")
        R = self._out_like(u) if out is None else out
        self._check(self.L.jfnk_residual_noalloc(self.h, _ptr(u), _ptr(R), _stream(u)))
        return R

    def jv(self, u, v, out=None):
        u, v = self._in(u), self._in(v)
        J = self._out_like(u) if out is None else out
        mem, s = self._io(u)
        self._check(self.L.jfnk_jv(self.h, _ptr(u), _ptr(v), _ptr(J), mem, s))
        return J

    def precondition(self, v, pc=PC_BJACOBI, out=None):
        v = self._in(v)
        z = self._out_like(v) if out is None else out
        mem, s = self._io(v)
        self._check(self.L.jfnk_precondition(self.h, _ptr(v), _ptr(z), pc, mem, s))
        return z

    def solve_dynamic(self, n_steps, probe_cell=-1, raise_on_fail=True, segregated=False):
        """n_steps time steps (options.density, options.dt) from the context's state, each
        solved by the Newton-Krylov method (or the segregated one); returns
        (u, stats, status, probe [steps, 3] displacement of probe_cell)."""
        u = np.zeros((self.nc, 3))
        probe = np.zeros((max(1, n_steps), 3))
        st = Stats()
        rc = self.L.jfnk_solve_dynamic(self.h, _ptr(u), MEM_HOST, int(n_steps), int(probe_cell),
                                       probe.ctypes.data if probe_cell >= 0 else None, 1 if segregated else 0,
                                       C.byref(st), None)
        if rc != OK and raise_on_fail and rc not in (MAXIT, LS_FAILED, DIVERGED):
            self._check(rc)
        return u, st, rc, probe[:st.load_steps_done]

    def dynamic_reset(self):
        self._check(self.L.jfnk_dynamic_reset(self.h))

    def dynamic_state(self):
        """Checkpoint of the time integration: [5, n_cells, 3] (u_t, u_t-1, v_t, v_t-1, a_t)."""
        st = np.zeros((5, self.nc, 3))
        self._check(self.L.jfnk_dynamic_get_state(self.h, _ptr(st)))
        return st

    def set_dynamic_state(self, state):
        """Restart the time integration from a checkpoint of dynamic_state()."""
        st = np.ascontiguousarray(state, np.float64).reshape(5, self.nc, 3)
        self._check(self.L.jfnk_dynamic_set_state(self.h, _ptr(st)))

    def solve_segregated(self, u0=None, load_steps=1, raise_on_fail=True):
        """The segregated quasi-Newton solve of Sec. 3.1 (the paper's comparison method);
        returns (u, stats, status) as solve(); stats.newton_its = outer iterations,
        stats.gmres_its = conjugate-gradient iterations."""
        return self._solve_with(self.L.jfnk_solve_segregated, u0, load_steps, raise_on_fail)

    def solve(self, u0=None, load_steps=1, raise_on_fail=True):
        """Newton solve; returns (u, stats, status).  u0: numpy or torch CUDA tensor (copied)."""
        return self._solve_with(self.L.jfnk_solve, u0, load_steps, raise_on_fail)

    def _solve_with(self, fn, u0, load_steps, raise_on_fail):
        if u0 is None:
            u = np.zeros((self.nc, 3))
        elif _is_device(u0):
            u = u0.clone().contiguous()
        else:
            u = np.array(u0, dtype=np.float64).reshape(self.nc, 3)
        st = Stats()
        mem, s = self._io(u)
        rc = fn(self.h, _ptr(u), mem, int(load_steps), C.byref(st), s)
        if rc != OK and raise_on_fail and rc not in (MAXIT, LS_FAILED, DIVERGED):
            self._check(rc)
        return u, st, rc

    # -------- inspection
    def geometry(self):
        nf = self.mesh.n_faces
        Sf, Cf, V, Cc = np.zeros((nf, 3)), np.zeros((nf, 3)), np.zeros(self.nc), np.zeros((self.nc, 3))
        self._check(self.L.jfnk_get_geometry(self.h, _ptr(Sf), _ptr(Cf), _ptr(V), _ptr(Cc)))
        return Sf, Cf, V, Cc

    def gradient(self):
        g = np.zeros((self.nc, 3, 3))
        self._check(self.L.jfnk_get_gradient(self.h, _ptr(g)))
        return g

    def permutation(self):
        p = np.zeros(self.nc, np.int32)
        self._check(self.L.jfnk_get_permutation(self.h, _ptr(p)))
        return p

    def profile(self, enable=True, detail=False):
        """Per-kernel CUDA-event timing; detail=True also times the steps inside each V-cycle."""
        self._check(self.L.jfnk_profile_enable(self.h, (2 if detail else 1) if enable else 0))

    def profile_get(self, name):
        ms, n = C.c_double(0), C.c_int64(0)
        rc = self.L.jfnk_profile_get(self.h, name.encode(), C.byref(ms), C.byref(n))
        if rc != OK:
            return 0.0, 0
        return ms.value, n.value

    def profile_reset(self):
        self._check(self.L.jfnk_profile_reset(self.h))

    def synchronize(self):
        """Waits for the work of the last call (its stream, or the context's own)."""
        self._check(self.L.jfnk_synchronize(self.h))

    def launch_count(self):
        return int(self.L.jfnk_launch_count(self.h))

    def device_bytes(self):
        return int(self.L.jfnk_device_bytes(self.h))

    def mg_hierarchy(self):
        """Levels of the multigrid hierarchy: list of dicts rows / nnz_a / nnz_p (empty when
        the context was set up without the multigrid preconditioner)."""
        n = 32
        rows, na, npv = (np.zeros(n, np.int64) for _ in range(3))
        nl = self.L.jfnk_mg_hierarchy(self.h, n, _ptr(rows), _ptr(na), _ptr(npv))
        if nl < 0:
            self._check(nl)
        return [{"rows": int(rows[l]), "nnz_a": int(na[l]), "nnz_p": int(npv[l])} for l in range(min(nl, n))]

    TUNING_KEYS = ("grad_bs", "flux_bs", "flux_stage", "finish_bs", "mg_bs", "tuned")

    def tuning(self):
        """Launch shapes of the hot-path kernels (dict; `tuned` = chosen by the autotuner)."""
        out = np.zeros(6, np.int32)
        self._check(self.L.jfnk_get_tuning(self.h, out.ctypes.data_as(C.POINTER(C.c_int32)), 6))
        return dict(zip(self.TUNING_KEYS, (int(v) for v in out)))

    def set_tuning(self, grad_bs, flux_bs, flux_stage, finish_bs, mg_bs):
        v = np.array([grad_bs, flux_bs, flux_stage, finish_bs, mg_bs], np.int32)
        self._check(self.L.jfnk_set_tuning(self.h, v.ctypes.data_as(C.POINTER(C.c_int32)), 5))


class Batch(Solver):
    """Independent problems solved together in one concatenated index space.

    Vectors are [sum of n_cells, 3] in the order the problems were added."""

    def __init__(self, cases, options: Options | None = None, **opt_kw):
        self.L = load()
        if cases and "alpha_residual" not in opt_kw and options is None:
            opt_kw["alpha_residual"] = cases[0].alpha
        self.options = options if options is not None else default_options(**opt_kw)
        h = C.c_void_p()
        rc = self.L.jfnk_create(C.byref(h), C.byref(self.options))
        if rc != OK:
            raise JfnkError(rc, "jfnk_create failed (no usable CUDA device?)")
        self.h = h
        self.cases = list(cases)
        self.sizes = [c.mesh.n_cells for c in self.cases]
        self.offsets = np.concatenate([[0], np.cumsum(self.sizes)]).astype(int)
        self.nc = int(self.offsets[-1])
        self.mesh = None
        for case in self.cases:
            prob = Solver(case.mesh, case.material, case.body_force, options=self.options)
            idx = C.c_int32(0)
            self._check(self.L.jfnk_batch_add(self.h, prob.h, C.byref(idx)))
            prob.close()

    def problem_stats(self):
        n = self.L.jfnk_batch_size(self.h)
        arr = (Stats * n)()
        self._check(self.L.jfnk_batch_stats(self.h, arr))
        return list(arr)

    def split(self, u):
        """Per-problem views of a concatenated vector."""
        return [u[self.offsets[p]:self.offsets[p + 1]] for p in range(len(self.sizes))]


def measure_fp64_rate(device: int = 0) -> float:
    """Measured FP64 FMA throughput of the device in TFLOP/s."""
    v = C.c_double(0.0)
    rc = load().jfnk_measure_fp64_rate(device, C.byref(v))
    if rc != OK:
        raise JfnkError(rc, "jfnk_measure_fp64_rate failed")
    return v.value


def solver_for_case(case, **kw) -> Solver:
    return Solver.from_case(case, **kw)


__all__ = ["Solver", "Batch", "Options", "Stats", "default_options", "load", "EXPORTS", "JfnkError", "solver_for_case", "_inputs"]
