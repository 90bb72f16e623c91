"""Dynamics on the device (Sec. 2.3 inertia, BDF2 of Eq. inertia2, predictor of Eq. predictor)
against the oracle (GPU)."""
import numpy as np
import pytest

import oracle as O
from paper_2502_17217_gb300 import inputs as I

pytestmark = pytest.mark.gpu
RHO, DT = 1000.0, 1e-3


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


@pytest.mark.parametrize("pc,precision", [(1, 0), (2, 1)])
def test_dynamic_column_parity_with_the_oracle(pc, precision):
    """Case 6 column (3x30x3, neo-Hookean, sudden traction on the upper face), 25 steps of
    1 ms: displacement history of the upper-face centre and the final field."""
    from paper_2502_17217_gb300 import jfnk
    case, probe = I.case_dynamic_beam(3, 30, 3)
    s = jfnk.Solver.from_case(case, pc=pc, precision=precision, density=RHO, dt=DT, newton_rtol=1e-10,
                              mg_coarse_max=20)
    u, st, rc, pr = s.solve_dynamic(25, probe_cell=probe)
    assert rc == 0 and st.load_steps_done == 25
    o = O.Oracle.from_case(case)
    o.set_dynamics(RHO, DT)
    if pc == jfnk.PC_MG:
        o.mg_setup(coarse_max=20, smoothed=bool(s.options.mg_smoothed), sweeps=s.options.mg_smooth_sweeps)
    uo, rco, sto, pro = o.dynamic(25, rtol=1e-10, pc=pc, probe_cell=probe, m=s.options.gmres_restart,
                                  aug=s.options.gmres_aug)
    assert rco == 0
    assert _rel(u, uo) <= 1e-8
    assert _rel(pr, pro) <= 1e-8
    assert pr[-1, 0] > 0.02  # the column is moving in the load direction


def test_free_body_follows_the_scalar_bdf2_recurrence():
    from paper_2502_17217_gb300 import jfnk
    m = I.hex_box(6, 4, 4, (0.6, 0.4, 0.4), perturb=0.15, seed=3)
    f = np.array([2.0e3, -1.0e3, 0.5e3])
    case = I.Case("free", m, I.Material(I.LAW_NEOHOOKEAN, 1.0e6, 4.0e6), np.tile(f, (m.n_cells, 1)))
    s = jfnk.Solver.from_case(case, density=RHO, dt=DT, newton_rtol=1e-12, newton_atol=1e-9, gmres_eta=1e-10)
    u, st, rc, pr = s.solve_dynamic(6, probe_cell=7)
    assert rc == 0
    k2 = 9.0 / (4 * DT * DT)
    ut = utm1 = vt = vtm1 = np.zeros(3)
    for step in range(6):
        c = (3 * (-4 * ut + utm1) / (2 * DT) - 4 * vt + vtm1) / (2 * DT)
        un = (f / RHO - c) / k2
        vn = (3 * un - 4 * ut + utm1) / (2 * DT)
        utm1, ut, vtm1, vt = ut, un, vt, vn
        np.testing.assert_allclose(pr[step], un, rtol=1e-9, atol=1e-15)


def test_calls_continue_the_motion_and_reset_restarts_it():
    from paper_2502_17217_gb300 import jfnk
    case, probe = I.case_dynamic_beam(3, 12, 3)
    s = jfnk.Solver.from_case(case, density=RHO, dt=DT)
    u20, _, rc, p20 = s.solve_dynamic(20, probe_cell=probe)
    assert rc == 0
    s.dynamic_reset()
    u10a, _, _, pa = s.solve_dynamic(10, probe_cell=probe)
    u10b, _, _, pb = s.solve_dynamic(10, probe_cell=probe)
    assert np.array_equal(u10b, u20)
    assert np.array_equal(np.concatenate([pa, pb]), p20)


def test_batch_dynamics_bitwise_equal_alone():
    from paper_2502_17217_gb300 import jfnk
    cases = [I.case_dynamic_beam(3, 10, 3)[0], I.case_dynamic_beam(2, 14, 3, traction=(20e3, 0.0, 10e3))[0],
             I.case_dynamic_beam(3, 9, 2, law=I.LAW_LINEAR)[0]]
    B = jfnk.Batch(cases, pc=jfnk.PC_BJACOBI, density=RHO, dt=DT)
    u, st, rc, _ = B.solve_dynamic(8)
    assert rc == 0
    for k, (c, uk) in enumerate(zip(cases, B.split(u))):
        ua, sta, rca, _ = jfnk.Solver.from_case(c, pc=jfnk.PC_BJACOBI, density=RHO, dt=DT).solve_dynamic(8)
        assert rca == 0 and np.array_equal(uk, ua), k


def test_static_context_rejects_time_integration():
    from paper_2502_17217_gb300 import jfnk
    case, _ = I.case_dynamic_beam(2, 6, 2)
    s = jfnk.Solver.from_case(case)
    with pytest.raises(jfnk.JfnkError):
        s.solve_dynamic(2)


def test_dynamic_steps_by_the_segregated_method_reach_the_same_motion():
    """The paper's dynamic comparison: each time step solved by the segregated method of
    Sec. 3.1 instead gives the same motion (same equations, tight tolerances)."""
    from paper_2502_17217_gb300 import jfnk
    case, probe = I.case_dynamic_beam(3, 12, 3)
    opts = dict(pc=jfnk.PC_BJACOBI, density=RHO, dt=DT, newton_rtol=1e-10)
    u1, st1, rc1, p1 = jfnk.Solver.from_case(case, **opts).solve_dynamic(10, probe_cell=probe)
    u2, st2, rc2, p2 = jfnk.Solver.from_case(case, **opts).solve_dynamic(10, probe_cell=probe, segregated=True)
    assert rc1 == 0 and rc2 == 0
    assert _rel(u2, u1) <= 1e-7 and _rel(p2, p1) <= 1e-7
    assert st2.newton_its > st1.newton_its  # outer iterations against Newton iterations


def test_checkpoint_restart_continues_the_motion_bitwise():
    """A checkpoint of the time-integration state (jfnk_dynamic_get_state) restarted in a fresh
    context (jfnk_dynamic_set_state) continues the motion exactly: 10 + 10 steps across two
    contexts equal 20 steps in one, and the state reads back as written."""
    from paper_2502_17217_gb300 import jfnk
    case, probe = I.case_dynamic_beam(3, 12, 3)
    kw = dict(density=RHO, dt=DT, pc=jfnk.PC_MG, precision=jfnk.PREC_MIXED, mg_coarse_max=20)
    a = jfnk.Solver.from_case(case, **kw)
    u20, _, rc, p20 = a.solve_dynamic(20, probe_cell=probe)
    assert rc == 0
    b = jfnk.Solver.from_case(case, **kw)
    _, _, rc, pb = b.solve_dynamic(10, probe_cell=probe)
    assert rc == 0
    state = b.dynamic_state()
    assert state.shape == (5, case.mesh.n_cells, 3) and np.any(state != 0)
    c = jfnk.Solver.from_case(case, **kw)
    c.setup()
    c.set_dynamic_state(state)
    assert np.array_equal(c.dynamic_state(), state)
    u, _, rc, pc_ = c.solve_dynamic(10, probe_cell=probe)
    assert rc == 0
    assert np.array_equal(u, u20)
    assert np.array_equal(np.concatenate([pb, pc_]), p20)
    static = jfnk.Solver.from_case(case)
    static.setup()
    with pytest.raises(jfnk.JfnkError):
        static.dynamic_state()
