"""fem_solve_noalloc: the solver for callers whose device memory must not be allocated by this
library (their memory manager owns the device, or their path cannot afford the synchronisation
an allocation may cause).  Its work space is a fixed device array inside the library instead of a
buffer the context allocates.  Checked through the C ABI against fem_solve on two calls in a row;
this file is collected last and needs nothing from the other test files."""
import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# the tolerances of the other solve tests: relative residual 1e-10, and two solutions of the same
# system agree to 1e-7 relative (the residual bound times the condition number; the scatter's
# atomics make repeated solves differ in the last bits)
RTOL = 1e-10
XTOL = 1e-7


@pytest.fixture(scope="module")
def space():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_10226_gb300.fem import FemSpace

    xyz, cells = synth.kuhn_cube(6, jitter=0.2, seed=0)
    return FemSpace(xyz, cells, degree=3, dirichlet=True, device=0)  # 19^3 = 6859 DoFs


def _solve(sp, fn_name, b, mode, inner):
    from paper_2509_10226_gb300 import _lib

    x = torch.zeros_like(b)
    opts = _lib.SolveOpts(_lib.FEM_SOLVE_IR_MIXED if mode == "ir" else _lib.FEM_SOLVE_FP64_PCG,
                          {"fp32": _lib.FEM_FP32, "tf32": _lib.FEM_TF32}[inner], 1e-10, 1e-3, 50, 20000)
    st = _lib.SolveStats()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    status = getattr(_lib.lib(), fn_name)(sp._h, ctypes.byref(opts), ctypes.c_void_p(b.data_ptr()),
                                          ctypes.c_void_p(x.data_ptr()), ctypes.byref(st), stream)
    _lib.check(status, fn_name)
    torch.cuda.synchronize()
    return x.cpu().numpy(), (st.outer_iterations, st.inner_iterations, st.rel_residual)


@pytest.mark.parametrize("mode,inner", [("pcg", "fp32"), ("ir", "fp32"), ("ir", "tf32")])
def test_noalloc_matches_fem_solve_twice(space, mode, inner):
    b = space.rhs_const(1.0)
    x_ref, st_ref = _solve(space, "fem_solve", b, mode, inner)
    assert st_ref[2] <= RTOL
    for _ in range(2):
        x, st = _solve(space, "fem_solve_noalloc", b, mode, inner)
        assert st[2] <= RTOL
        assert np.linalg.norm(x - x_ref) <= XTOL * np.linalg.norm(x_ref)
        # the inner iteration counts may differ (the scatter's atomics change the last bits, which can
        # move an outer refinement step across the tolerance), but not by more than an outer step
        assert st[1] <= 2 * st_ref[1] + 16 and st_ref[1] <= 2 * st[1] + 16


def test_noalloc_allocates_no_device_memory():
    """A fresh context of 185,193 DoFs (fem_solve would allocate about 12 MB of work vectors for
    it): after a first call (which loads the library's device code and looks the work array up),
    two more fem_solve_noalloc calls leave the device's free memory unchanged, while one fem_solve
    call on the same context visibly takes its work space."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_10226_gb300 import _lib
    from paper_2509_10226_gb300.fem import FemSpace

    xyz, cells = synth.kuhn_cube(28, jitter=0.2, seed=0)
    sp = FemSpace(xyz, cells, degree=2, dirichlet=True, device=0)  # 57^3 = 185,193 DoFs
    assert 150_000 < sp.n_dofs <= _lib.FEM_SOLVE_NOALLOC_MAX_DOFS
    b = sp.rhs_const(1.0)
    x = torch.zeros_like(b)
    opts = _lib.SolveOpts(_lib.FEM_SOLVE_IR_MIXED, _lib.FEM_TF32, 1e-10, 1e-3, 50, 20000)
    st = _lib.SolveStats()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    def call(name):
        x.zero_()
        status = getattr(_lib.lib(), name)(sp._h, ctypes.byref(opts), ctypes.c_void_p(b.data_ptr()),
                                           ctypes.c_void_p(x.data_ptr()), ctypes.byref(st), stream)
        _lib.check(status, name)
        torch.cuda.synchronize()
        assert st.rel_residual <= RTOL

    call("fem_solve_noalloc")
    free0 = torch.cuda.mem_get_info()[0]
    call("fem_solve_noalloc")
    call("fem_solve_noalloc")
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0, f"fem_solve_noalloc changed free device memory by {free0 - free1} bytes"
    call("fem_solve")
    free2 = torch.cuda.mem_get_info()[0]
    assert free1 - free2 >= 8 << 20, "fem_solve's work space should be visible to this check"


def test_noalloc_rejects_oversize():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_10226_gb300 import FemError, _lib
    from paper_2509_10226_gb300.fem import FemSpace

    xyz, cells = synth.kuhn_cube(64)
    sp = FemSpace(xyz, cells, degree=1, dirichlet=True, device=0)  # 65^3 = 274,625 DoFs
    assert sp.n_dofs > _lib.FEM_SOLVE_NOALLOC_MAX_DOFS
    b = sp.rhs_const(1.0)
    with pytest.raises(FemError) as e:
        sp.solve(b, mode="pcg", no_alloc=True)
    assert e.value.status == _lib.FEM_EINVAL and "static work space" in str(e.value)
