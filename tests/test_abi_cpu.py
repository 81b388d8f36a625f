"""Host-side checks of the C ABI library (no GPU compute).

The library must load, export every function include/lbm.h declares, and
refuse to run without a GPU instead of falling back to the CPU.  The product
package must not reach the oracle.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1107_4543_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def declared_functions():
    src = open(os.path.join(ROOT, "include", "lbm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(lbm_[a-z_0-9]+)\s*\(", src))
    # typedefs of function pointers are not entry points
    names -= set(re.findall(r"\(\*\s*(lbm_[a-z_0-9]+)\)", src))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("lbm_create", "lbm_init_field", "lbm_step", "lbm_moments", "lbm_destroy",
                 "lbm_submit", "lbm_poll", "lbm_get_populations", "lbm_set_populations",
                 "lbm_set_stream", "lbm_set_allocator", "lbm_drift", "lbm_strerror"):
        assert must in names


def test_library_exports_every_declared_function(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_wraps_every_declared_function():
    from paper_1107_4543_gb300 import lbm

    missing = [n for n in declared_functions() if not callable(getattr(lbm, n, None))]
    assert not missing, missing


def test_error_strings(lib):
    lib.lbm_strerror.restype = ctypes.c_char_p
    for code in (0, 1, -1, -2, -3, -4, -5, -6, -7):
        assert lib.lbm_strerror(code)
    assert lib.lbm_strerror(-99) == b"unknown error"


def test_no_cpu_fallback_without_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1107_4543_gb300 import lbm

    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_create(8, 8, [0, 1.64, 1.54, 0, 1.9, 0, 1.9, 1.9, 1.9])
    assert e.value.code == lbm.LBM_ECUDA


def test_product_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_1107_4543_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "lbm_oracle" not in text and "liboracle" not in text, f
