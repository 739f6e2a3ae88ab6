"""Brute-force references used to pin the oracle (independent of oracle/ and of the library).

Shape functions are built in barycentric coordinates with Silvester's product
formula, polynomials are multiplied symbolically (exponent dictionaries with
exact Fraction coefficients) and integrated exactly with

    int_K lambda^alpha dx = 3! |K| alpha! / (|alpha| + 3)!         (tetrahedron)
    int_F lambda^alpha ds = 2! |F| alpha! / (|alpha| + 2)!         (triangle)

so no quadrature rule and no reference-to-physical Jacobian convention is shared
with the oracle.
"""
from __future__ import annotations

from fractions import Fraction
from functools import lru_cache
from itertools import product
from math import factorial

import numpy as np


def compositions(total, parts):
    out = []
    for c in product(range(total + 1), repeat=parts):
        if sum(c) == total:
            out.append(c)
    return sorted(out)


def poly_mul(a, b):
    out = {}
    for ea, ca in a.items():
        for eb, cb in b.items():
            e = tuple(x + y for x, y in zip(ea, eb))
            out[e] = out.get(e, 0) + ca * cb
    return {e: c for e, c in out.items() if c != 0}


def poly_diff(a, i):
    out = {}
    for e, c in a.items():
        if e[i] > 0:
            e2 = list(e)
            e2[i] -= 1
            out[tuple(e2)] = out.get(tuple(e2), 0) + c * e[i]
    return out


@lru_cache(maxsize=None)
def silvester_basis(p):
    """Shape functions phi_beta (beta lexicographic, |beta| = p) as polynomials in (l0, l1, l2, l3)."""
    basis = []
    for beta in compositions(p, 4):
        poly = {(0, 0, 0, 0): Fraction(1)}
        for i in range(4):
            for m in range(beta[i]):
                e = [0, 0, 0, 0]
                e[i] = 1
                factor = {tuple(e): Fraction(p, m + 1), (0, 0, 0, 0): Fraction(-m, m + 1)}
                poly = poly_mul(poly, factor)
        basis.append(poly)
    return basis


def int_bary(poly, n):
    """Integral over an n-simplex of volume 1 (barycentric monomials)."""
    tot = Fraction(0)
    for e, c in poly.items():
        num = factorial(n)
        for x in e:
            num *= factorial(x)
        tot += c * Fraction(num, factorial(sum(e) + n))
    return tot


@lru_cache(maxsize=None)
def _grad_pair_integrals(p):
    """I[a, b, i, j] = int_K (d phi_a / d l_i)(d phi_b / d l_j) dx / |K|."""
    B = silvester_basis(p)
    nd = len(B)
    I = np.zeros((nd, nd, 4, 4))
    d = [[poly_diff(B[a], i) for i in range(4)] for a in range(nd)]
    for a in range(nd):
        for b in range(nd):
            for i in range(4):
                for j in range(4):
                    I[a, b, i, j] = float(int_bary(poly_mul(d[a][i], d[b][j]), 3))
    return I


def barycentric_gradients(X):
    """Rows: grad lambda_i for the tet with vertices X [4,3]; and its volume."""
    T = np.vstack([np.ones(4), X.T])  # 4x4: [1; x]
    Tinv = np.linalg.inv(T)
    return Tinv[:, 1:], abs(np.linalg.det(T)) / 6.0


def stiffness(X, p):
    """Exact element stiffness matrix int_K grad phi_a . grad phi_b for vertices X [4,3]."""
    gl, vol = barycentric_gradients(np.asarray(X, dtype=np.float64))
    G = gl @ gl.T
    return vol * np.einsum("abij,ij->ab", _grad_pair_integrals(p), G)


def node_coordinates(X, p):
    """Physical node positions of the element (beta lexicographic)."""
    X = np.asarray(X, dtype=np.float64)
    return np.array([sum(b[i] * X[i] for i in range(4)) / p for b in compositions(p, 4)])


def assemble_cg(xyz, cells, p):
    """Dense global stiffness matrix with DoFs identified by rounded node coordinates.

    Returns (A [N,N], node_xyz [N,3]).  Only for tiny meshes.
    """
    index = {}
    coords = []
    local = []
    for c in cells:
        ids = []
        for x in node_coordinates(xyz[c], p):
            key = tuple(np.round(x, 10))
            if key not in index:
                index[key] = len(coords)
                coords.append(x)
            ids.append(index[key])
        local.append(ids)
    N = len(coords)
    A = np.zeros((N, N))
    for c, ids in zip(cells, local):
        K = stiffness(xyz[c], p)
        A[np.ix_(ids, ids)] += K
    return A, np.array(coords)


def five_tet_cube(n):
    """Unit cube split into n^3 subcubes x 5 tets with the alternating (conforming) pattern."""
    def vid(i, j, k):
        return i + (n + 1) * (j + (n + 1) * k)

    g = np.arange(n + 1) / n
    xyz = np.array([[g[i], g[j], g[k]] for k in range(n + 1) for j in range(n + 1) for i in range(n + 1)])
    cells = []
    even = [(0, 0, 0), (1, 1, 0), (1, 0, 1), (0, 1, 1)]
    odd = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 1)]
    for k in range(n):
        for j in range(n):
            for i in range(n):
                centre, corners = (even, odd) if (i + j + k) % 2 == 0 else (odd, even)
                cells.append([vid(i + a, j + b, k + c) for a, b, c in centre])
                for a, b, c in corners:
                    nb = [(a ^ 1, b, c), (a, b ^ 1, c), (a, b, c ^ 1)]
                    cells.append([vid(i + a, j + b, k + c)] + [vid(i + x, j + y, k + z) for x, y, z in nb])
    return xyz, np.array(cells, dtype=np.int64)
