"""Jacobi polynomials and 1D Gauss rules (float64).

Used by every basis of Sec. 2.1: Legendre (alpha=beta=0) for the hexahedron,
Jacobi P^{(2i+1,0)} for the wedge (Sec. 2.1.3), P^{(2k+3,0)} for the pyramid
(Sec. 2.1.4), Gauss-Jacobi (1,0) / (2,0) weights for collapsed cubatures.
"""
from __future__ import annotations

from math import gamma

import numpy as np


def jacobi_p(n, alpha, beta, x):
    """Standard Jacobi polynomial P_n^{(alpha,beta)}(x), P_n(1) = binom(n+alpha, n)."""
    x = np.asarray(x, dtype=np.float64)
    p0 = np.ones_like(x)
    if n == 0:
        return p0
    a, b = alpha, beta
    p1 = 0.5 * ((a + b + 2.0) * x + (a - b))
    for m in range(2, n + 1):
        c = 2.0 * m + a + b
        A = 2.0 * m * (m + a + b) * (c - 2.0)
        B = (c - 1.0) * (c * (c - 2.0) * x + a * a - b * b)
        C = 2.0 * (m + a - 1.0) * (m + b - 1.0) * c
        p0, p1 = p1, (B * p1 - C * p0) / A
    return p1


def jacobi_dp(n, alpha, beta, x):
    """d/dx P_n^{(alpha,beta)}(x) = (n+alpha+beta+1)/2 P_{n-1}^{(alpha+1,beta+1)}(x)."""
    x = np.asarray(x, dtype=np.float64)
    if n == 0:
        return np.zeros_like(x)
    return 0.5 * (n + alpha + beta + 1.0) * jacobi_p(n - 1, alpha + 1, beta + 1, x)


def gauss_jacobi(n, alpha=0.0, beta=0.0):
    """n-point Gauss-Jacobi rule for weight (1-x)^alpha (1+x)^beta (Golub-Welsch).

    Exact for polynomials of degree 2n-1.  Nodes ascending.
    """
    if n < 1:
        raise ValueError("n >= 1")
    a, b = float(alpha), float(beta)
    k = np.arange(n, dtype=np.float64)
    s = 2.0 * k + a + b
    with np.errstate(divide="ignore", invalid="ignore"):
        diag = (b * b - a * a) / (s * (s + 2.0))
    if abs(a + b) < 1e-14:
        diag[0] = (b - a) / (a + b + 2.0)
    kk = np.arange(1, n, dtype=np.float64)
    s = 2.0 * kk + a + b
    off = np.sqrt(4.0 * kk * (kk + a) * (kk + b) * (kk + a + b) / (s * s * (s + 1.0) * (s - 1.0)))
    T = np.diag(diag) + np.diag(off, 1) + np.diag(off, -1)
    x, V = np.linalg.eigh(T)
    mu0 = 2.0 ** (a + b + 1.0) * gamma(a + 1.0) * gamma(b + 1.0) / gamma(a + b + 2.0)
    w = mu0 * V[0, :] ** 2
    return x, w


def gauss_legendre(n):
    """n-point Gauss-Legendre rule on [-1,1]."""
    return gauss_jacobi(n, 0.0, 0.0)


def gauss_lobatto(n):
    """n-point Gauss-Legendre-Lobatto rule on [-1,1] (n >= 2), exact to degree 2n-3."""
    if n < 2:
        raise ValueError("n >= 2")
    if n == 2:
        return np.array([-1.0, 1.0]), np.array([1.0, 1.0])
    xi, _ = gauss_jacobi(n - 2, 1.0, 1.0)
    x = np.concatenate([[-1.0], xi, [1.0]])
    P = jacobi_p(n - 1, 0.0, 0.0, x)
    w = 2.0 / ((n - 1) * n * P * P)
    return x, w


def lagrange_1d(nodes, x):
    """Values ell_i(x) of the Lagrange polynomials at ``nodes`` -> (len(x), len(nodes))."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    L = np.ones((x.size, nodes.size))
    for i, xi in enumerate(nodes):
        for j, xj in enumerate(nodes):
            if j != i:
                L[:, i] *= (x - xj) / (xi - xj)
    return L


def lagrange_1d_deriv(nodes, x):
    """Derivatives ell_i'(x) -> (len(x), len(nodes)), by the product rule."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = nodes.size
    D = np.zeros((x.size, n))
    for i in range(n):
        for m in range(n):
            if m == i:
                continue
            term = np.full(x.size, 1.0 / (nodes[i] - nodes[m]))
            for j in range(n):
                if j != i and j != m:
                    term *= (x - nodes[j]) / (nodes[i] - nodes[j])
            D[:, i] += term
    return D
