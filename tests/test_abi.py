"""The C-ABI library loads and exports every function include/jfnk_gb300.h declares (no GPU
needed: nothing here launches a kernel)."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "jfnk_gb300.h")


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_2502_17217_gb300 import jfnk
    return jfnk.load()


def _declared():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"\b(jfnk_[a-z0-9_]+)\s*\(", txt)))


def test_header_and_binding_agree():
    from paper_2502_17217_gb300 import jfnk
    assert sorted(jfnk.EXPORTS) == _declared()


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib._name], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (jfnk_[a-z0-9_]+)\b", out))
    missing = [f for f in _declared() if f not in exported]
    assert not missing, missing
    for f in _declared():
        assert hasattr(lib, f)


def test_default_options_match_header_defaults(lib):
    from paper_2502_17217_gb300 import jfnk
    o = jfnk.default_options()
    assert o.gmres_restart == 30 and o.gmres_eta == 1e-3 and o.newton_rtol == 1e-8 and o.newton_atol == 1e-50
    assert o.pc == jfnk.PC_BJACOBI and o.precision == jfnk.PREC_FP64 and o.jv_eps_scale == 1e-7
    assert o.alpha_residual == 1.0 and o.alpha_pc == 1.0 and o.mg_smooth_sweeps == 2 and o.mg_smoothed == 1


def test_null_arguments_are_rejected_without_a_device(lib):
    # argument validation happens before any device work
    assert lib.jfnk_create(None, None) == -1
    assert lib.jfnk_destroy(None) == 0
    assert lib.jfnk_residual(None, None, None, 0, None) == -1
    assert lib.jfnk_last_error(None) == b"null context"
    assert lib.jfnk_launch_count(None) == 0


def test_no_cpu_fallback_in_the_binding():
    # the product binding never imports the oracle
    src = open(os.path.join(ROOT, "paper_2502_17217_gb300", "jfnk.py")).read()
    assert "oracle" not in src
    for name in os.listdir(os.path.join(ROOT, "paper_2502_17217_gb300", "csrc")):
        assert "oracle" not in open(os.path.join(ROOT, "paper_2502_17217_gb300", "csrc", name)).read().lower()


def test_hex_patch_ranges_match_the_python_block_builder(lib):
    """jfnk_hex_patch (pure arithmetic, no device) gives the face ranges of the six sides of the
    structured block, in the order and sizes of the face-addressed builder in inputs.py."""
    from paper_2502_17217_gb300 import inputs as I
    for nx, ny, nz in [(3, 4, 5), (1, 1, 1), (7, 2, 1), (200, 20, 20)]:
        m = I.hex_box(nx, ny, nz)
        for side, name in enumerate(["xmin", "xmax", "ymin", "ymax", "zmin", "zmax"]):
            f0, nf = C.c_int32(-1), C.c_int32(-1)
            assert lib.jfnk_hex_patch(nx, ny, nz, side, C.byref(f0), C.byref(nf)) == 0
            p = m.patch(name)
            assert (f0.value, nf.value) == (p.start, p.size), (nx, ny, nz, name)
    assert lib.jfnk_hex_patch(0, 1, 1, 0, None, None) == -1
    assert lib.jfnk_hex_patch(2, 2, 2, 6, None, None) == -1
