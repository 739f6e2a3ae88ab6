"""GPU parity of the host-buffer apply (fem_apply_host): a stream of host vectors through the
device gives the FP64 oracle's operator within the precision's tolerance and the device apply's
result up to the order of its atomic sums, including slot reuse (more vectors than the two
device slots), a repeated output buffer, a precision switch on one context and DG."""
import numpy as np
import pytest

import synth
from oracle import cg, topology
from tests.gpu_util import assert_close, require_gpu, to_dev, to_host

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    require_gpu()


def _host(x, prec, pinned=True):
    t = torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64 if prec == "fp64" else torch.float32)
    return t.pin_memory() if pinned else t


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32", "bf16", "tf32x3"])
@pytest.mark.parametrize("nvec", [1, 2, 5])
def test_cg_host_stream_matches_oracle_and_device_apply(prec, nvec):
    from paper_2509_10226_gb300.fem import FemSpace

    p = 3
    xyz, cells = synth.kuhn_cube(5, jitter=0.2, seed=11)
    sp = FemSpace(xyz, cells, kind="cg", degree=p, dirichlet=True, device=0)
    dofs, keys = topology.cg_numbering(cells, p)
    mask = topology.dirichlet_mask(cells, p, keys)
    perm = sp.dof_permutation()
    U = [synth.uniform_vector(sp.n_dofs, 100 + b) for b in range(nvec)]
    us = [_host(u[perm], prec) for u in U]
    ys = [_host(np.zeros(sp.n_dofs), prec) for _ in range(nvec)]
    sp.apply_host(us, ys, prec=prec)
    for b in range(nvec):
        y = ys[b].double().numpy()
        y_ref = cg.apply(xyz, cells, U[b], p, dirichlet_mask=mask, dofs=dofs)[perm]
        assert_close(y, y_ref, prec, f"vector {b}")
        y_dev = to_host(sp.apply(to_dev(U[b][perm], prec), prec=prec))
        # same kernel and inputs: only the order of the atomic sums may differ
        np.testing.assert_allclose(y, y_dev, rtol=0, atol=1e-5 * np.abs(y_dev).max() if prec != "fp64"
                                   else 1e-13 * np.abs(y_dev).max())


def test_repeated_buffers_pageable_and_precision_switch():
    from paper_2509_10226_gb300.fem import FemSpace

    p = 2
    xyz, cells = synth.kuhn_cube(6, jitter=0.2, seed=3)
    sp = FemSpace(xyz, cells, kind="cg", degree=p, device=0)
    dofs, _ = topology.cg_numbering(cells, p)
    perm = sp.dof_permutation()
    U = [synth.uniform_vector(sp.n_dofs, 7 + b) for b in range(4)]
    # FP32 first (4-byte slots), then FP64 on the same context (the slots grow)
    for prec in ("fp32", "fp64"):
        us = [_host(u[perm], prec, pinned=(prec == "fp32")) for u in U]
        y_shared = _host(np.zeros(sp.n_dofs), prec)
        sp.apply_host(us, [y_shared] * len(us), prec=prec)  # the last vector's result remains
        y_ref = cg.apply(xyz, cells, U[-1], p, dofs=dofs)[perm]
        assert_close(y_shared.double().numpy(), y_ref, prec, prec)


@pytest.mark.parametrize("prec", ["fp64", "tf32"])
def test_dg_host_stream(prec):
    """DG through host buffers equals the device apply (itself pinned to the oracle by the DG tests)
    up to the order of its atomic sums."""
    from paper_2509_10226_gb300.fem import FemSpace

    xyz, cells = synth.kuhn_cube(4, jitter=0.2, seed=5)
    sp = FemSpace(xyz, cells, kind="dg", degree=2, device=0)
    U = [synth.uniform_vector(sp.n_dofs, 40 + b) for b in range(3)]
    us = [_host(u, prec) for u in U]
    ys = [_host(np.zeros(sp.n_dofs), prec) for _ in U]
    sp.apply_host(us, ys, prec=prec)
    for b in range(3):
        y_dev = to_host(sp.apply(to_dev(U[b], prec), prec=prec))
        tol = 1e-13 if prec == "fp64" else 1e-5
        np.testing.assert_allclose(ys[b].double().numpy(), y_dev, rtol=0, atol=tol * np.abs(y_dev).max())


def test_host_apply_rejects_bad_arguments():
    from paper_2509_10226_gb300._lib import FemError
    from paper_2509_10226_gb300.fem import FemSpace

    xyz, cells = synth.kuhn_cube(2, jitter=0.0, seed=0)
    sp = FemSpace(xyz, cells, kind="cg", degree=1, device=0)
    u = _host(np.zeros(sp.n_dofs), "fp32")
    with pytest.raises(ValueError):
        sp.apply_host([u], [], prec="fp32")
    with pytest.raises(ValueError):
        sp.apply_host([u.cuda()], [u], prec="fp32")
    with pytest.raises(ValueError):
        sp.apply_host([u], [u.double()], prec="fp32")
    from paper_2509_10226_gb300 import _lib
    import ctypes
    with pytest.raises(FemError):
        arr = (ctypes.c_void_p * 1)(u.data_ptr())
        _lib.call("fem_apply_host", sp._h, _lib.FEM_FP32, 0, arr, arr)
