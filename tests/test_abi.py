"""The C-ABI library builds, loads without a GPU, and exports every symbol include/fe.h declares
(no compute calls here)."""
import os
import re

import pytest

from paper_2603_09038_gb300 import fe

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "fe.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fe_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(fe.LIB_PATH):
        from paper_2603_09038_gb300 import build
        build.build()
    return fe.load()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("fe_mesh_setup", "fe_pa_setup", "fe_apply_diffusion", "fe_apply_mass",
                     "fe_pcg", "fe_assemble_diagonal", "fe_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header(lib):
    for n in _declared():
        assert hasattr(fe, n), n


def test_version_and_error_without_gpu(lib):
    assert "sm_103a" in fe.fe_version()
    assert fe.fe_last_error() == ""


def test_argument_errors_need_no_gpu(lib):
    import ctypes
    out = ctypes.c_void_p()
    st = lib.fe_mesh_setup(2, 2, 2, 9, ctypes.c_void_p(1), ctypes.byref(out))
    assert st == fe.FE_ERR_UNSUPPORTED and out.value is None
    assert "order" in fe.fe_last_error()
    st = lib.fe_mesh_setup(0, 2, 2, 2, ctypes.c_void_p(1), ctypes.byref(out))
    assert st == fe.FE_ERR_ARG
    st = lib.fe_pa_setup(None, 0, None, 1, None, ctypes.byref(out))
    assert st == fe.FE_ERR_ARG
    assert lib.fe_apply_diffusion(None, None, None, None) == fe.FE_ERR_ARG
    assert lib.fe_pcg(None, 1, 1, None, None, 1e-8, 10, None, None) == fe.FE_ERR_ARG
