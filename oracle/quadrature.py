"""Grundmann-Moeller quadrature on the unit n-simplex, computed in exact rationals.

The paper (Sec. 2.3, text after Eq. 7) integrates with symmetric simplex rules;
the workloads fix the Grundmann-Moeller family with s = p, which is exact for
polynomials of total degree 2s+1 >= 2p.

Rule (Grundmann & Moeller 1978), d = 2s+1, unit simplex {x >= 0, sum x <= 1}:

  Q[f] = sum_{i=0..s} (-1)^i 2^{-2s} (d+n-2i)^d / (i! (d+n-i)!)
         * sum_{beta in N^{n+1}, |beta| = s-i} f(lambda),
  lambda_j = (2 beta_j + 1) / (d + n - 2i),  j = 0..n.

The weights already include the simplex volume 1/n!.  Point order: i ascending,
then beta in lexicographic ascending order.  Reference coordinates are
x_hat = (lambda_1, ..., lambda_n) (vertex 0 at the origin, vertex k at e_k).
"""
from __future__ import annotations

from fractions import Fraction
from functools import lru_cache
from math import factorial

import numpy as np


def compositions(total: int, parts: int):
    """All beta in N^parts with sum == total, in lexicographic ascending order."""
    if parts == 1:
        return [(total,)]
    out = []
    for first in range(total + 1):
        for rest in compositions(total - first, parts - 1):
            out.append((first,) + rest)
    return out


@lru_cache(maxsize=None)
def gm_rule_exact(s: int, n: int):
    """Exact (barycentric points, weights) as tuples of Fractions."""
    if s < 0 or n < 1:
        raise ValueError("need s >= 0 and n >= 1")
    d = 2 * s + 1
    pts, wts = [], []
    for i in range(s + 1):
        w = Fraction((-1) ** i, 2 ** (2 * s)) * Fraction((d + n - 2 * i) ** d, factorial(i) * factorial(d + n - i))
        den = d + n - 2 * i
        for beta in compositions(s - i, n + 1):
            pts.append(tuple(Fraction(2 * b + 1, den) for b in beta))
            wts.append(w)
    return tuple(pts), tuple(wts)


def gm_rule(s: int, n: int):
    """(x_hat [nq, n] float64, w [nq] float64) of the GM rule with parameter s on the unit n-simplex."""
    pts, wts = gm_rule_exact(s, n)
    lam = np.array([[float(c) for c in p] for p in pts], dtype=np.float64)
    return lam[:, 1:].copy(), np.array([float(w) for w in wts], dtype=np.float64)


def tet_rule(p: int, modified: bool = False):
    """Cell rule for degree p: GM with s = p (exact to degree 2p+1); with modified=True the rule of
    Sec. 3.3, exact to degree 2p-2, taken as GM with s = p-1 (exact to degree 2p-1)."""
    return gm_rule(p - 1 if modified else p, 3)


def tri_rule(p: int):
    """Face rule for degree p: GM with s = p on the triangle."""
    return gm_rule(p, 2)
