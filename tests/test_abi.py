"""The C ABI library builds, loads and exports every entry point ``include/ot.h`` declares.

CPU-only: no compute call is made (there may be no GPU).
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for mt in re.finditer(r"\b(?:ot_status|void|const char\s*\*)\s+(ot_[a-z0-9_]+)\s*\(", text):
            names.add(mt.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    path = __graft_entry__._builder().build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ["ot_solve", "ot_step", "ot_certificate", "ot_state_create", "ot_state_get",
                     "ot_state_set", "ot_context_create"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_and_defaults(lib):
    lib.ot_status_str.restype = ctypes.c_char_p
    assert lib.ot_status_str(0) == b"OT_OK"
    assert b"invalid" in lib.ot_status_str(1)
    import paper_2609_33814_b300 as P
    prm = P.make_params()
    assert prm.eps0 == 1.0 and prm.lam == 1.0 and prm.cert_every == 100
    assert ctypes.sizeof(P.OtProblem) == 8 * 2 + 4 * 2 + 8 * 4 + 8 * 3
    assert ctypes.sizeof(P.OtResult) == 8 * 3 + 8 * 10 + 4 * 2 + 8 * 2


def test_python_package_fails_loudly_without_library(tmp_path):
    """The binding, loaded from a package directory that holds no libot.so, refuses to import (there
    is no CPU fallback to use instead)."""
    import importlib.util
    pkg = tmp_path / "paper_2609_33814_b300"
    pkg.mkdir()
    (pkg / "__init__.py").write_text(open(os.path.join(ROOT, "paper_2609_33814_b300", "__init__.py")).read())
    spec = importlib.util.spec_from_file_location("ot_binding_without_library", str(pkg / "__init__.py"))
    mod = importlib.util.module_from_spec(spec)
    with pytest.raises(ImportError) as ei:
        spec.loader.exec_module(mod)
    assert "libot.so" in str(ei.value)


def test_without_a_gpu_no_context_is_created(lib):
    """With no visible GPU the library refuses to create a context and says why: there is no CPU
    path to fall back to."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is visible")
    import paper_2609_33814_b300 as P
    with pytest.raises(P.OTError) as ei:
        P.Context(0)
    assert "ot_context_create" in str(ei.value)
