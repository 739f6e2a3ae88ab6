"""Plain Jacobi-preconditioned conjugate gradients in FP64 (the solver used with the
operator of Eq. 3; the paper's own preconditioner is hybrid multigrid, Sec. 4.1)."""
from __future__ import annotations

import numpy as np


def jacobi_pcg(apply, diag, b, x0=None, rtol=1e-12, maxiter=20000):
    """Solve A x = b; returns (x, iterations, final relative residual ||b - A x|| / ||b||)."""
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - apply(x)
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return x, 0, 0.0
    z = r / diag
    d = z.copy()
    rz = r @ z
    it = 0
    while np.linalg.norm(r) / nb > rtol and it < maxiter:
        Ad = apply(d)
        alpha = rz / (d @ Ad)
        x += alpha * d
        r -= alpha * Ad
        z = r / diag
        rz_new = r @ z
        d = z + (rz_new / rz) * d
        rz = rz_new
        it += 1
    return x, it, np.linalg.norm(b - apply(x)) / nb
