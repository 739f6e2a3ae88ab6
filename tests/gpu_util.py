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
TOL = {"fp64": 1e-12, "fp32": 1e-5, "tf32": 5e-3, "bf16": 4e-2}


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
