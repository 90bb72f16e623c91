"""The allocation-free residual entry point (jfnk_residual_noalloc) gives the same R(u) as the
regular entry point (jfnk_residual, device pointers), on two calls in a row.

It exists for callers that cannot allocate device memory at the time they need a residual
(inside a stream capture, under a framework that owns the device's memory, or in loops that
must not synchronise on cudaMalloc); its scratch is a fixed 16 MiB device array.  This file is
collected last so that a run stopping at the first failure has run every other test first.
"""
import numpy as np
import pytest

from paper_2502_17217_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()


@pytest.mark.parametrize("case_fn,scale", [
    (lambda: I.case_cantilever(40, 8, 8, (1.0, 0.2, 0.2), perturb=0.15, seed=2), 1e-4),
    (lambda: I.case_nh_beam(24, 6, 6, (1.0, 0.25, 0.25), end_uy=0.2, perturb=0.1, seed=3), 0.004),
])
def test_noalloc_residual_matches_regular_entry_point(case_fn, scale):
    import torch
    from paper_2502_17217_gb300 import jfnk
    case = case_fn()
    s = jfnk.Solver.from_case(case)
    s.setup()
    for seed in (1, 2):  # two calls in a row share (and overwrite) the fixed scratch array
        u = torch.from_numpy(I.random_field(seed, case.mesh.n_cells, scale)).cuda()
        R_ref = s.residual(u)
        R_na = s.residual_noalloc(u)
        torch.cuda.synchronize()
        a, b = R_na.cpu().numpy(), R_ref.cpu().numpy()
        assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(b)


def test_noalloc_rejects_meshes_beyond_the_scratch_size():
    import torch
    from paper_2502_17217_gb300 import jfnk
    case = I.case_cantilever(200, 20, 20)  # 80k cells: more scratch than the fixed 16 MiB array
    s = jfnk.Solver.from_case(case)
    s.setup()
    u = torch.zeros((case.mesh.n_cells, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(jfnk.JfnkError, match="scratch"):
        s.residual_noalloc(u)
