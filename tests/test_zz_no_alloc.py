"""The allocation-free residual entry point (jfnk_residual_noalloc).

Some callers cannot allocate device memory at the time they need a residual: code running
inside a CUDA stream capture (cudaMalloc is not allowed there), code under a framework that
owns the device's memory, and loops that must not synchronise on cudaMalloc.  This entry point
serves them from a fixed 16 MiB device array.  These tests check that it gives the same R(u)
as the regular entry point (jfnk_residual with device pointers), bit for bit, on two calls in
a row, and the oracle's R(u) within the residual tolerance (1e-12 relative); that a graph
captured from it after a load-factor change replays correctly without allocating; and that
meshes beyond the array and inputs that are not device tensors are refused.

This file is collected last so that a run stopping at the first failure has run every other
test first.
"""
import dataclasses

import numpy as np
import pytest

from paper_2502_17217_gb300 import inputs as I


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


def _symmetry_case():
    """A block with one symmetry plane (x-min), clamped y-min and a traction on y-max."""
    m = I.hex_box(8, 5, 4, (0.6, 0.4, 0.3), perturb=0.12, seed=11)
    m.patch("xmin").bc = I.BC_SYMM
    m.patch("ymin").bc = I.BC_DISP
    ymax = m.patch("ymax")
    ymax.bc = I.BC_TRAC
    ymax.values = np.tile(np.array([0.0, -2.0e5, 0.6e5]), (ymax.size, 1))
    return I.Case("sym_block_8x5x4", m, I.Material(I.LAW_LINEAR, 2.0e6, 0.3), None)


CASES = {
    "cantilever_40x8x8": (lambda: I.case_cantilever(40, 8, 8, (1.0, 0.2, 0.2), perturb=0.15, seed=2), 1e-4),
    "nh_beam_24x6x6": (lambda: I.case_nh_beam(24, 6, 6, (1.0, 0.25, 0.25), end_uy=0.2, perturb=0.1, seed=3), 0.004),
    "stvk_beam_20x5x5": (lambda: dataclasses.replace(
        I.case_nh_beam(20, 5, 5, (1.0, 0.25, 0.25), end_uy=0.2, perturb=0.1, seed=5),
        material=I.Material(I.LAW_STVK, 2.0e6, 0.3)), 0.004),
    "symmetry_block_8x5x4": (_symmetry_case, 1e-3),
}


def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    return torch


@pytest.mark.gpu
@pytest.mark.parametrize("name", list(CASES))
def test_noalloc_residual_matches_regular_entry_point_and_oracle(name):
    torch = _gpu()
    import oracle as O
    from paper_2502_17217_gb300 import jfnk
    case_fn, scale = CASES[name]
    case = case_fn()
    s = jfnk.Solver.from_case(case)
    s.setup()
    o = O.Oracle.from_case(case)
    for seed in (1, 2):  # two calls in a row share (and overwrite) the fixed scratch array
        u_h = I.random_field(seed, case.mesh.n_cells, scale)
        u = torch.from_numpy(u_h).cuda()
        R_ref = s.residual(u)
        R_na = s.residual_noalloc(u)
        torch.cuda.synchronize()
        a, b = R_na.cpu().numpy(), R_ref.cpu().numpy()
        assert np.array_equal(a, b), _rel(a, b)  # same kernels, same order: bitwise equal
        assert _rel(a, o.residual(u_h)) <= 1e-12


@pytest.mark.gpu
def test_noalloc_residual_in_a_captured_graph_after_a_load_change():
    """A graph captured from the call replays it without allocating and keeps the load factor
    of the captured call (the call never waits on the host, so capture stays valid)."""
    torch = _gpu()
    from paper_2502_17217_gb300 import jfnk
    case = I.case_cantilever(40, 8, 8, (1.0, 0.2, 0.2), perturb=0.15, seed=2)
    s = jfnk.Solver.from_case(case)
    s.setup()
    nc = case.mesh.n_cells
    u = torch.from_numpy(I.random_field(3, nc, 1e-4)).cuda()
    R = torch.empty_like(u)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):  # first call on the device: looks up the array's address
        s.residual_noalloc(u, out=R)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    s.residual_noalloc(u, out=R)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0  # the call allocated no device memory

    s.set_load_factor(0.61)  # the context's load factor changes before the capture
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        s.residual_noalloc(u, out=R)
    for seed in (4, 5):
        u.copy_(torch.from_numpy(I.random_field(seed, nc, 1e-4)))
        g.replay()
        torch.cuda.synchronize()
        ref = s.residual(u).cpu().numpy()
        assert np.array_equal(R.cpu().numpy(), ref), _rel(R.cpu().numpy(), ref)


@pytest.mark.gpu
def test_noalloc_rejects_meshes_beyond_the_scratch_size_and_host_pointers():
    torch = _gpu()
    from paper_2502_17217_gb300 import jfnk
    case = I.case_cantilever(200, 20, 20)  # 80k cells: more scratch than the fixed 16 MiB array
    s = jfnk.Solver.from_case(case)
    s.setup()
    u = torch.zeros((case.mesh.n_cells, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(jfnk.JfnkError, match="scratch"):
        s.residual_noalloc(u)
    small = I.case_cantilever(8, 4, 4, (1.0, 0.2, 0.2))
    s2 = jfnk.Solver.from_case(small)
    s2.setup()
    u_host = np.zeros((small.mesh.n_cells, 3))
    R_dev = torch.empty((small.mesh.n_cells, 3), dtype=torch.float64, device="cuda")
    # a host pointer passed straight to the C ABI is refused, not dereferenced on the GPU
    rc = s2.L.jfnk_residual_noalloc(s2.h, jfnk._ptr(u_host), jfnk._ptr(R_dev), None)
    assert rc == jfnk.EINVAL


def test_noalloc_wrapper_refuses_non_device_inputs():
    """The binding checks dtype, shape, layout and device before calling the library (CPU)."""
    from paper_2502_17217_gb300 import jfnk
    s = jfnk.Solver.__new__(jfnk.Solver)  # no context: the check happens before any call
    s.nc = 12
    s.options = jfnk.Options()
    s.options.device = 0
    with pytest.raises(TypeError, match="float64 CUDA tensor"):
        s.residual_noalloc(np.zeros((12, 3)))
    torch = pytest.importorskip("torch")
    with pytest.raises(TypeError, match="float64 CUDA tensor"):
        s.residual_noalloc(torch.zeros((12, 3), dtype=torch.float64))
