"""Trace and Markov constants on the reference elements (Appendix B, Sec. 3.2-3.3).

C_T(N) is the largest eigenvalue of M_s v = lambda M v, with M the reference
mass matrix and M_s the surface mass matrix (the sum over all faces of the
face integrals of phi_i phi_j); C_M(N) is the largest eigenvalue of
K v = lambda M v with K the stiffness matrix.  ``measure="euclid"`` integrates
each reference face with its Euclidean area element in (r,s,t); the
alternative ``"unit"`` scales every triangle to area 2 and every quadrilateral
to area 4 (Sec. 3.2 states the face constants for those areas).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from .elements import make_element
from .mesh import face_reference_points


def reference_mass(el, lobatto=False):
    if lobatto:                                # SEM hexahedron: GLL collocation (lumped)
        return np.diag(el.wnodes)
    P, W = el.exact_rule(el.N + 2)
    B = el.basis(P)
    return B.T @ (W[:, None] * B)


def reference_surface_mass(el, measure="euclid", lobatto=False):
    Ms = np.zeros((el.Np, el.Np))
    for f, corners in enumerate(el.faces):
        key = tuple(range(len(corners)))
        rst, w, d1, d2 = face_reference_points(el, f, key, el.N, lobatto)
        if measure == "euclid":
            w = w * np.linalg.norm(np.cross(d1, d2), axis=1)
        B = el.basis(rst)
        Ms += B.T @ (w[:, None] * B)
    return Ms


def trace_constant(t, N, measure="euclid", lobatto=False):
    """C_T(N) of Table computedTrace (or C_SEM(N) of Table computedTraceSEM if lobatto)."""
    el = make_element(t, N, lobatto)
    M = reference_mass(el, lobatto and t == 0)
    Ms = reference_surface_mass(el, measure, lobatto)
    return float(scipy.linalg.eigh(Ms, M, eigvals_only=True)[-1])


def markov_constant(t, N, lobatto=False):
    """C_M(N) of Table markovConsts: largest eigenvalue of K v = lambda M v.

    lobatto (hexahedron only): the SEM hexahedron of Sec. 2.1.1, whose inner product is the GLL
    quadrature at its (N+1)^3 nodes, for the mass and the stiffness alike (M = diag(w),
    K = D^T diag(w) D with D the nodal gradients at the nodes).  The table's hexahedron row is
    this constant (it is not the one of Q_N in the exact L2 inner product)."""
    if lobatto:
        if t != 0:
            raise ValueError("lobatto applies to the hexahedron only")
        el = make_element(t, N, True)
        G = el.grad(el.nodes)                     # (3, Np, Np): d l_j / d r_a at node q
        W = el.wnodes
        M = np.diag(W)
        K = np.einsum("q,aqi,aqj->ij", W, G, G)
        return float(scipy.linalg.eigh(K, M, eigvals_only=True)[-1])
    el = make_element(t, N)
    P, W = el.exact_rule(N + 2)
    B = el.basis(P)
    G = el.grad(P)
    M = B.T @ (W[:, None] * B)
    K = np.einsum("q,aqi,aqj->ij", W, G, G)
    return float(scipy.linalg.eigh(K, M, eigvals_only=True)[-1])
