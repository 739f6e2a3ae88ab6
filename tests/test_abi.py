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


def test_device_calls_refused_on_a_host_only_context():
    """A host-only context (device = -1) refuses every device call with FEM_EINVAL before any CUDA
    call is made (this runs without a GPU)."""
    import numpy as np

    import synth
    from paper_2509_10226_gb300.fem import FemSpace

    xyz, cells = synth.kuhn_cube(2)
    sp = FemSpace(xyz, cells, degree=1, device=-1)
    L = _lib.lib()
    assert L.fem_apply(sp._h, _lib.FEM_FP32, None, None, None, None) == _lib.FEM_EINVAL
    assert b"host-only" in L.fem_last_error()
    st = _lib.SolveStats()
    opts = _lib.SolveOpts(_lib.FEM_SOLVE_FP64_PCG, _lib.FEM_FP32, 1e-10, 1e-3, 5, 5)
    assert L.fem_solve_noalloc(sp._h, ctypes.byref(opts), None, None, ctypes.byref(st), None) == _lib.FEM_EINVAL
    assert b"host-only" in L.fem_last_error()
    assert np.isfinite(sp.n_dofs)


@pytest.mark.gpu
def test_device_mismatch_refused_before_launch():
    """Device calls need the calling thread's current device to be the context's device; with another
    device current they return FEM_EINVAL and launch nothing.  Needs two visible GPUs."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available() or torch.cuda.device_count() < 2:
        pytest.skip("needs two CUDA devices")
    import synth
    from paper_2509_10226_gb300.fem import FemSpace

    xyz, cells = synth.kuhn_cube(2)
    sp = FemSpace(xyz, cells, degree=1, device=0)
    u = torch.zeros(sp.n_dofs, device="cuda:0")
    y = torch.full((sp.n_dofs,), 7.0, device="cuda:0")
    L = _lib.lib()
    with torch.cuda.device(1):
        s = L.fem_apply(sp._h, _lib.FEM_FP32, ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(y.data_ptr()), None,
                        None)
        assert s == _lib.FEM_EINVAL and b"current device 1" in L.fem_last_error()
    torch.cuda.synchronize(0)
    assert bool((y == 7.0).all())
