"""The C-ABI library builds, loads and exports every symbol include/cheb.h declares.

No GPU needed: only loading, symbol lookup and argument checks that fail before
any CUDA call.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "cheb.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(cheb_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_1704_00512_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary_calls():
    names = _declared()
    for want in ("cheb_pattern_build", "cheb_bounds", "cheb_coeffs", "cheb_expand", "cheb_trace",
                 "cheb_mu_search", "cheb_newton_schulz", "cheb_masked_product", "cheb_plan_create"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    from paper_1704_00512_gb300 import _lib
    assert sorted(_lib.EXPORTS) == _declared()


def test_invalid_arguments_fail_before_any_cuda_call():
    from paper_1704_00512_gb300 import _lib as L
    lib = L.load()
    nnzb = ctypes.c_int64(0)
    assert lib.cheb_pattern_build(None, 0, 1.0, 1.0, None, None, ctypes.byref(nnzb), None) == L.ERR_INVALID
    assert "bad arguments" in lib.cheb_last_error().decode()
    h = ctypes.c_void_p()
    nb = ctypes.c_size_t()
    assert lib.cheb_plan_create(None, L.F64, -1, ctypes.byref(h), ctypes.byref(nb), None) == L.ERR_INVALID
    assert lib.cheb_bounds_workspace_size(10, 0, ctypes.byref(nb)) == L.ERR_INVALID
    assert lib.cheb_bounds_workspace_size(10, 40, ctypes.byref(nb)) == L.OK and nb.value > 0
    assert lib.cheb_coeffs_workspace_size(1, 8, ctypes.byref(nb)) == L.ERR_INVALID
    assert lib.cheb_coeffs_workspace_size(2, 1024, ctypes.byref(nb)) == L.OK
    assert lib.cheb_mu_search(None, 10, 0.0, 1.0, L.FERMI, 0.1, 1.0, 1e-9, 50, None, None, None, 0, None) \
        == L.ERR_INVALID
    assert lib.cheb_expand(None, None, 10, None, 10, 0, None, None, None, None, L.F64, None, 0, None) \
        == L.ERR_INVALID


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1704_00512_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.sub(r"#.*|//.*", "", src).replace("the oracle", ""), f
