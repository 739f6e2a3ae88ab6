"""Helpers for the GPU parity tests: build a device space, move vectors between
library and canonical orders, compare against the oracle with stated tolerances."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

# Tolerances, normwise: max_i |y_i - y_ref_i| <= tol * max_i |y_ref_i| and
# ||y - y_ref||_2 <= tol * ||y_ref||_2.
#   fp64: 1e-12 (stated for FP64 paths)
#   fp32: 1e-5  (stated for FP32)
#   tf32: 5e-3  TF32 keeps 10 mantissa bits: operands round with relative error
#         <= 2^-11 = 4.9e-4; two chained products (E u, then E^T t) and the
#         FP32 metric give a few units of that, cancellation in y = A u (rows sum
#         to zero) amplifies it by the ratio of term size to result size (~3-5)
#   bf16: 4e-2  BF16 keeps 7 mantissa bits: unit roundoff 2^-8 = 3.9e-3, same chain
#   tf32x3: 1e-5  each operand is split into a TF32 high part and a TF32 low part and three
#         products (hi hi + hi lo + lo hi) are accumulated in FP32: the dropped lo*lo term and
#         the truncation of the low parts are below 2^-20 relative, so the result is as accurate
#         as the FP32 path (same bound)
TOL = {"fp64": 1e-12, "fp32": 1e-5, "tf32": 5e-3, "bf16": 4e-2, "tf32x3": 1e-5}


def require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def dtype(prec):
    return torch.float64 if prec == "fp64" else torch.float32


def to_dev(x, prec):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype(prec), device="cuda")


def to_host(t):
    torch.cuda.synchronize()
    return t.detach().double().cpu().numpy()


def assert_close(y, y_ref, prec, what=""):
    tol = TOL[prec]
    y = np.asarray(y, dtype=np.float64)
    y_ref = np.asarray(y_ref, dtype=np.float64)
    assert y.shape == y_ref.shape, (y.shape, y_ref.shape)
    scale = np.abs(y_ref).max()
    err_inf = np.abs(y - y_ref).max()
    rel_l2 = np.linalg.norm(y - y_ref) / max(np.linalg.norm(y_ref), 1e-300)
    assert err_inf <= tol * scale, f"{what} {prec}: max err {err_inf:.3e} > {tol} * {scale:.3e}"
    assert rel_l2 <= tol, f"{what} {prec}: rel-l2 {rel_l2:.3e} > {tol}"
    return rel_l2


def encode_keys(keys, nv):
    """Pack sorted vertex tuples into one int64 (valid while nv ** p < 2 ** 63)."""
    keys = np.asarray(keys, dtype=np.int64)
    code = np.zeros(keys.shape[0], dtype=np.int64)
    for r in range(keys.shape[1]):
        code = code * np.int64(nv) + keys[:, r]
    return code


def sampled_rows(sp, xyz, cells, p, u_lib, sample, k_user=None, mask_lib=None):
    """Oracle values of (A u)_i at sampled library DoFs i: the oracle's element products of every cell
    touching a sampled DoF, gathered from and scattered to library positions found through the DoF keys.
    With a Dirichlet mask the operator is P A P + (I - P)."""
    from oracle import cg, topology

    lib_keys = sp.dof_keys()
    nv = xyz.shape[0]
    lib_code = encode_keys(lib_keys, nv)
    order = np.argsort(lib_code)
    want = np.unique(lib_keys[sample])
    touch = np.where(np.isin(cells, want).any(axis=1))[0]
    keys_t = topology.dof_keys(cells[touch], p)
    code_t = encode_keys(keys_t.reshape(-1, p), nv)
    lib_of = order[np.searchsorted(lib_code, code_t, sorter=order)].reshape(keys_t.shape[:2])
    ue = u_lib[lib_of]
    if mask_lib is not None:
        ue = np.where(mask_lib[lib_of], 0.0, ue)
    ye = cg.element_apply(xyz, cells[touch], ue, p, None if k_user is None else k_user[touch])
    y = np.zeros(sp.n_dofs)
    np.add.at(y, lib_of.ravel(), ye.ravel())
    if mask_lib is not None:
        y[mask_lib] = u_lib[mask_lib]
    return y[sample]


def sampled_rhs(sp, xyz, cells, p, sample, mask_lib=None):
    """Oracle load vector b_i = int phi_i (f = 1) at sampled library DoFs."""
    from oracle import cg, topology

    lib_keys = sp.dof_keys()
    nv = xyz.shape[0]
    lib_code = encode_keys(lib_keys, nv)
    order = np.argsort(lib_code)
    touch = np.where(np.isin(cells, np.unique(lib_keys[sample])).any(axis=1))[0]
    keys_t = topology.dof_keys(cells[touch], p)
    lib_of = order[np.searchsorted(lib_code, encode_keys(keys_t.reshape(-1, p), nv), sorter=order)]
    lib_of = lib_of.reshape(keys_t.shape[:2])
    local = np.arange(lib_of.size).reshape(lib_of.shape)
    be = cg.rhs_const(xyz, cells[touch], p, lib_of.size, dofs=local)
    b = np.zeros(sp.n_dofs)
    np.add.at(b, lib_of.ravel(), be)
    if mask_lib is not None:
        b[mask_lib] = 0.0
    return b[sample]
