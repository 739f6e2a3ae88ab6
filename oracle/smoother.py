"""Chebyshev iteration preconditioned by the operator's diagonal (the Chebyshev-Jacobi smoother of
the paper's multigrid, Sec. 4.1), and a power iteration for the largest eigenvalue of D^-1 A.

Plain FP64 numpy, test infrastructure only.  The recurrence is the classical three-term form of
Chebyshev acceleration for a spectrum in [lam_min, lam_max] (theta = centre, delta = half width,
sigma = theta / delta):
    x_1 = x_0 + D^-1 r_0 / theta,
    rho_0 = 1 / sigma,  rho_k = 1 / (2 sigma - rho_{k-1}),
    d_k = rho_k rho_{k-1} d_{k-1} + (2 rho_k / delta) D^-1 r_k,  x_{k+1} = x_k + d_k,
with r_k = b - A x_k.  After m steps the error is P_m(D^-1 A) e_0 with
P_m(lambda) = T_m((theta - lambda) / delta) / T_m(theta / delta), T_m the Chebyshev polynomial.
"""
from __future__ import annotations

import numpy as np


def step_coefficients(degree, lam_max, lam_min):
    """(c_d, c_r) of each step: d_k = c_d d_{k-1} + c_r D^-1 r_k (c_d = 0 for the first step)."""
    theta = 0.5 * (lam_max + lam_min)
    delta = 0.5 * (lam_max - lam_min)
    sigma = theta / delta
    out = [(0.0, 1.0 / theta)]
    rho = 1.0 / sigma
    for _ in range(degree - 1):
        rho_new = 1.0 / (2.0 * sigma - rho)
        out.append((rho_new * rho, 2.0 * rho_new / delta))
        rho = rho_new
    return out


def chebyshev(apply, diag, b, x0, degree, lam_max, lam_min):
    """degree >= 1 steps; returns x_degree."""
    x = np.array(x0, dtype=np.float64)
    d = np.zeros_like(x)
    for c_d, c_r in step_coefficients(degree, lam_max, lam_min):
        r = b - apply(x)
        d = c_d * d + c_r * (r / diag)
        x = x + d
    return x


def lambda_max(apply, diag, v0, iterations):
    """Largest eigenvalue of A v = lambda D v by power iteration on D^-1 A: v <- D^-1 A v / ||.||_2;
    returns the generalised Rayleigh quotient (v, A v) / (v, D v) of the last iterate."""
    v = np.array(v0, dtype=np.float64)
    v = v / np.linalg.norm(v)
    lam = 0.0
    for _ in range(iterations):
        av = apply(v)
        lam = (v @ av) / (v @ (diag * v))
        w = av / diag
        v = w / np.linalg.norm(w)
    return lam
