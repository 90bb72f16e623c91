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
