"""Geometry and connectivity of a vertex-mapped hybrid mesh (float64).

Faces are matched by their sorted global vertex ids.  Surface integrals are
evaluated at face points defined in a *canonical frame* of each face, which
both neighbouring elements see identically (reading of the face-matching step
the paper leaves implicit, Sec. 2.2):

* triangle: the corners ordered by increasing global vertex id G0 < G1 < G2;
  a point of the reference triangle {xi,eta >= -1, xi+eta <= 0} has
  barycentric weights (-(xi+eta)/2, (1+xi)/2, (1+eta)/2) on (G0, G1, G2);
* quadrilateral: C00 = the corner with the smallest id, C10 = its edge
  neighbour with the smaller id, C01 = its other edge neighbour, C11 the
  opposite corner; a point (alpha,beta) of [-1,1]^2 is the bilinear blend.

The surface Jacobian J^s is the area ratio between the physical face and this
canonical reference face (area 2 for triangles, 4 for quadrilaterals).
"""
from __future__ import annotations

import numpy as np

from .elements import make_element, quad_face_rule, tri_face_rule


def canonical_corners(gids):
    """Canonical ordering of a face's corners (see module docstring).

    ``gids`` are the global ids of the local corners (triangle order c0,c1,c2 or
    quad lexicographic c00,c10,c01,c11).  Returns the local corner positions
    (indices into ``gids``) of (G0,G1,G2) or (C00,C10,C01,C11).
    """
    gids = list(gids)
    if len(gids) == 3:
        return tuple(int(i) for i in np.argsort(gids))
    cyc = [0, 1, 3, 2]                      # c00 -> c10 -> c11 -> c01 around the quad
    p = min(range(4), key=lambda m: gids[cyc[m]])
    n1, n2 = cyc[(p + 1) % 4], cyc[(p + 3) % 4]
    c10, c01 = (n1, n2) if gids[n1] < gids[n2] else (n2, n1)
    return (cyc[p], c10, c01, cyc[(p + 2) % 4])


def face_reference_points(el, f, key, N, lobatto=False):
    """Canonical face points in the element's reference coordinates.

    Returns (rst (nq,3), weights (nq,), d rst/d(canonical 1st coord), d rst/d(2nd)).
    """
    corners = np.array(el.faces[f])
    R = el.verts[corners][list(key)]
    if len(key) == 3:
        pts, w = tri_face_rule(N)
        xi, eta = pts[:, 0], pts[:, 1]
        mu = np.stack([-(xi + eta) / 2, (1 + xi) / 2, (1 + eta) / 2], axis=1)
        rst = mu @ R
        d1 = np.broadcast_to((R[1] - R[0]) / 2, rst.shape)
        d2 = np.broadcast_to((R[2] - R[0]) / 2, rst.shape)
    else:
        pts, w = quad_face_rule(N, lobatto)
        a, b = pts[:, 0], pts[:, 1]
        Nb = np.stack([(1 - a) * (1 - b), (1 + a) * (1 - b), (1 - a) * (1 + b), (1 + a) * (1 + b)], 1) / 4
        rst = Nb @ R
        d1 = np.stack([-(1 - b), (1 - b), -(1 + b), (1 + b)], 1) / 4 @ R
        d2 = np.stack([-(1 - a), -(1 + a), (1 - a), (1 + a)], 1) / 4 @ R
    return rst, w, np.array(d1), np.array(d2)


class Side:
    """One element's view of one face: canonical points, geometry, neighbour."""

    __slots__ = ("t", "e", "f", "key", "rst", "w", "n", "Js", "Js_ref", "J", "nbr", "tau_p")


class MeshGeometry:
    """Per-face-side canonical points, normals and surface Jacobians; face matching."""

    def __init__(self, mesh, N, lobatto=False):
        self.mesh = mesh
        self.N = N
        self.els = [make_element(t, N, lobatto) for t in range(4)]
        self.lobatto = lobatto
        xyz = mesh.xyz
        sides = []
        by_key = {}
        for t in range(4):
            el = self.els[t]
            for e in range(mesh.conn[t].shape[0]):
                vid = mesh.conn[t][e]
                xv = xyz[vid]
                for f, corners in enumerate(el.faces):
                    gids = vid[corners]
                    key = canonical_corners(gids)
                    rst, w, d1, d2 = face_reference_points(el, f, key, N, lobatto)
                    _, F = el.vmap(xv, rst)
                    x1 = np.einsum("qab,qb->qa", F, d1)
                    x2 = np.einsum("qab,qb->qa", F, d2)
                    G = np.linalg.inv(F)                          # G[q, a, d] = d r_a / d x_d
                    nvec = np.einsum("qad,a->qd", G, el.face_grad[f])
                    s = Side()
                    s.t, s.e, s.f, s.key, s.rst, s.w = t, e, f, key, rst, w
                    s.n = nvec / np.linalg.norm(nvec, axis=1, keepdims=True)
                    s.Js = np.linalg.norm(np.cross(x1, x2), axis=1)
                    # area element of the reference face itself (Euclidean, in r,s,t)
                    s.Js_ref = np.linalg.norm(np.cross(d1, d2), axis=1)
                    s.J = np.linalg.det(F)
                    s.nbr = -1
                    s.tau_p = 0.0
                    sk = tuple(sorted(int(g) for g in gids))
                    by_key.setdefault(sk, []).append(len(sides))
                    sides.append(s)
        for sk, lst in by_key.items():
            if len(lst) > 2:
                raise ValueError(f"face {sk} shared by {len(lst)} elements")
            if len(lst) == 2:
                a, b = lst
                sides[a].nbr, sides[b].nbr = b, a
        # penalties tau_p = 1/{rho c}, rho c = 1/c for kappa = 1, rho = 1/c^2 (Sec. 2.2)
        for s in sides:
            c_m = np.sqrt(mesh.c2[s.t][s.e])
            if s.nbr >= 0:
                o = sides[s.nbr]
                c_p = np.sqrt(mesh.c2[o.t][o.e])
            else:
                c_p = c_m
            s.tau_p = 1.0 / (0.5 * (1.0 / c_m + 1.0 / c_p))
        self.sides = sides
        self.side_of = {}
        for i, s in enumerate(sides):
            self.side_of[(s.t, s.e, s.f)] = i

    def boundary_sides(self):
        return [i for i, s in enumerate(self.sides) if s.nbr < 0]
