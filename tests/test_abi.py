"""The C-ABI library loads without a GPU and exports every function declared in include/tetmf.h."""
import ctypes

import pytest

from paper_2509_10226_gb300 import _lib


def test_header_declares_the_boundary():
    names = _lib.header_functions()
    for required in ["fem_create", "fem_destroy", "fem_apply", "fem_apply_adjoint", "fem_coeff_grad",
                     "fem_solve", "fem_csr_apply", "fem_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    L = _lib.lib()
    missing = [n for n in _lib.header_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_every_declared_function_has_a_binding_signature():
    declared = set(_lib.header_functions()) - {"fem_last_error"}
    assert declared <= set(_lib._SIGNATURES), declared - set(_lib._SIGNATURES)


def test_null_arguments_rejected():
    L = _lib.lib()
    assert L.fem_create(None, None, None) == _lib.FEM_EINVAL
    assert b"null" in L.fem_last_error()
    assert L.fem_apply(None, 0, None, None, None, None) == _lib.FEM_EINVAL
    assert L.fem_destroy(None) == _lib.FEM_OK
