"""Seeded synthetic inputs shared by the CUDA path and by the oracle tests.

This module produces *inputs only*: vertex coordinates, element-to-vertex
connectivity, per-element wave speed, and random state vectors.  It holds no
step of the discontinuous Galerkin method (no basis, no quadrature, no flux).

Layered hybrid mesh
-------------------
The unit of construction is a grid of ``nx*ny*nz`` cells on ``[-1,1]^3``.
Each z-layer of cells has one of five codes:

``H``  one hexahedron per cell.
``W``  two wedges per cell: the cell is cut by the plane through its
       ``(y0,z0)``-``(y1,z1)`` diagonal and extruded along ``x``.
``T``  transition cell: five pyramids whose bases are the bottom and the four
       side faces and whose apex is the cell centre, plus two tetrahedra on the
       top face, which is split along the ``(x0,y0,z1)``-``(x1,y1,z1)`` diagonal
       so that it conforms with a Kuhn cell above.
``U``  inverted transition cell: pyramids on the top and four side faces, two
       tetrahedra on the bottom face split along ``(x0,y0,z0)``-``(x1,y1,z0)``,
       which conforms with a Kuhn cell below.
``K``  Kuhn (Freudenthal) cell: six tetrahedra around the ``v000-v111``
       diagonal.

Interior grid vertices are displaced by a smooth seeded field of amplitude
``amp*h`` per axis; vertices on the boundary of the cube are left in place, so
the domain stays ``[-1,1]^3`` exactly.  Cell centres of transition cells are
the mean of the eight displaced cell vertices.

Local vertex orders (the reference coordinates of each local vertex):

* hex      v0..v7 at ``(r,s,t) = (+-1,+-1,+-1)``, lexicographic with r fastest.
* wedge    v0,v1,v2 = triangle corners ``(r,t) = (-1,-1),(1,-1),(-1,1)`` at
           ``s=-1``; v3,v4,v5 the same corners at ``s=+1``.
* pyramid  v0..v3 = base corners ``(r,s) = (-1,-1),(1,-1),(-1,1),(1,1)`` at
           ``t=-1``, lexicographic; v4 = apex ``(-1,-1,1)``.
* tet      v0 ``(-1,-1,-1)``, v1 ``(1,-1,-1)``, v2 ``(-1,1,-1)``, v3 ``(-1,-1,1)``.

Every element is emitted with positive orientation (the vertex map has a
positive Jacobian on the undisplaced grid).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

HEX, WEDGE, PYR, TET = 0, 1, 2, 3
TYPE_NAMES = ("hex", "wedge", "pyramid", "tet")
NVERT = (8, 6, 5, 4)


@dataclass
class HybridMesh:
    """Vertex-mapped hybrid mesh: coordinates, connectivity and wave speed."""

    xyz: np.ndarray                      # (nv, 3) float64
    conn: list                           # per type: (K_t, NVERT[t]) int32
    c2: list                             # per type: (K_t,) float64, squared wave speed
    layer: list = field(default_factory=list)   # per type: (K_t,) int32 z-layer index
    dims: tuple = (0, 0, 0)
    layers: str = ""

    @property
    def nelem(self):
        return [int(c.shape[0]) for c in self.conn]

    def ndof(self, N):
        return sum(k * npn for k, npn in zip(self.nelem, nodes_per_element(N)))


def nodes_per_element(N):
    """Number of degrees of freedom per element for order N: hex, wedge, pyramid, tet."""
    return ((N + 1) ** 3,
            (N + 1) ** 2 * (N + 2) // 2,
            (N + 1) * (N + 2) * (2 * N + 3) // 6,
            (N + 1) * (N + 2) * (N + 3) // 6)


def _displacement(pts, h, amp, rng):
    """Smooth field d(x) with d_a = amp*h_a*sin(2*pi*k_a.x + phi_a), |k_a| = 2."""
    d = np.zeros_like(pts)
    for a in range(3):
        k = rng.normal(size=3)
        k *= 2.0 / np.linalg.norm(k)
        phi = rng.uniform(0.0, 2.0 * np.pi)
        d[:, a] = amp * h[a] * np.sin(2.0 * np.pi * (pts @ k) + phi)
    return d


def _orient_tet(xyz, tet):
    """Swap two vertices if the tet is negatively oriented (on the given coordinates)."""
    p = xyz[tet]
    vol = np.linalg.det(np.stack([p[1] - p[0], p[2] - p[0], p[3] - p[0]]))
    if vol < 0:
        tet = [tet[0], tet[2], tet[1], tet[3]]
    return tet


def layered_mesh(nx, ny, nz, layers, seed=0, amp=0.1, c_of_layer=None):
    """Build the layered hybrid mesh.

    ``layers`` is a string of ``nz`` layer codes from bottom to top, e.g.
    ``"HWHTK"``.  ``c_of_layer(k)`` returns the wave speed of layer ``k``
    (default 1).  Returns a :class:`HybridMesh`.
    """
    if len(layers) != nz:
        raise ValueError("need one layer code per z-layer")
    for a, b in zip(layers[:-1], layers[1:]):
        top_tri = a in "TK"          # triangulated top face
        bot_tri = b in "UK"          # triangulated bottom face
        if top_tri != bot_tri:
            raise ValueError(f"layers {a}{b} do not conform")
    rng = np.random.default_rng(seed)
    xs = np.linspace(-1.0, 1.0, nx + 1)
    ys = np.linspace(-1.0, 1.0, ny + 1)
    zs = np.linspace(-1.0, 1.0, nz + 1)
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    grid = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)   # vid = i + (nx+1)(j + (ny+1)k)
    h = np.array([2.0 / nx, 2.0 / ny, 2.0 / nz])
    d = _displacement(grid, h, amp, rng)
    ii = np.tile(np.arange(nx + 1), (nz + 1) * (ny + 1))
    jj = np.tile(np.repeat(np.arange(ny + 1), nx + 1), nz + 1)
    kk = np.repeat(np.arange(nz + 1), (nx + 1) * (ny + 1))
    interior = (ii > 0) & (ii < nx) & (jj > 0) & (jj < ny) & (kk > 0) & (kk < nz)
    grid[interior] += d[interior]

    def vid(i, j, k):
        return i + (nx + 1) * (j + (ny + 1) * k)

    verts = [grid]
    nv = grid.shape[0]
    conn = [[], [], [], []]
    lay = [[], [], [], []]
    centres = []
    c_of_layer = c_of_layer or (lambda k: 1.0)
    c2 = [[], [], [], []]

    for k in range(nz):
        code = layers[k]
        ck = float(c_of_layer(k)) ** 2
        for j in range(ny):
            for i in range(nx):
                v = {(a, b, c): vid(i + a, j + b, k + c)
                     for a in (0, 1) for b in (0, 1) for c in (0, 1)}
                out = []
                if code == "H":
                    out.append((HEX, [v[(a, b, c)] for c in (0, 1) for b in (0, 1) for a in (0, 1)]))
                elif code == "W":
                    # (y,z) corners; clockwise triangles in the (y,z) plane give J > 0
                    for tri in (((0, 0), (1, 1), (1, 0)), ((0, 0), (0, 1), (1, 1))):
                        bot = [v[(0, b, c)] for b, c in tri]
                        top = [v[(1, b, c)] for b, c in tri]
                        out.append((WEDGE, bot + top))
                elif code in "TU":
                    cid = nv + len(centres)
                    centres.append(np.mean([grid[x] for x in v.values()], axis=0))
                    # pyramid bases, ordered so that (x_r x x_s) points to the apex
                    bases = {
                        "zlo": [v[(0, 0, 0)], v[(1, 0, 0)], v[(0, 1, 0)], v[(1, 1, 0)]],
                        "zhi": [v[(0, 0, 1)], v[(0, 1, 1)], v[(1, 0, 1)], v[(1, 1, 1)]],
                        "xlo": [v[(0, 0, 0)], v[(0, 1, 0)], v[(0, 0, 1)], v[(0, 1, 1)]],
                        "xhi": [v[(1, 0, 0)], v[(1, 0, 1)], v[(1, 1, 0)], v[(1, 1, 1)]],
                        "ylo": [v[(0, 0, 0)], v[(0, 0, 1)], v[(1, 0, 0)], v[(1, 0, 1)]],
                        "yhi": [v[(0, 1, 0)], v[(1, 1, 0)], v[(0, 1, 1)], v[(1, 1, 1)]],
                    }
                    pyr_faces = ["xlo", "xhi", "ylo", "yhi", "zlo" if code == "T" else "zhi"]
                    for f in pyr_faces:
                        out.append((PYR, bases[f] + [cid]))
                    cz = 1 if code == "T" else 0
                    for mid in ((1, 0), (0, 1)):
                        tet = [v[(0, 0, cz)], v[(mid[0], mid[1], cz)], v[(1, 1, cz)], cid]
                        out.append((TET, tet))
                elif code == "K":
                    import itertools
                    for perm in itertools.permutations(range(3)):
                        p = [0, 0, 0]
                        path = [v[(0, 0, 0)]]
                        for ax in perm:
                            p[ax] = 1
                            path.append(v[tuple(p)])
                        out.append((TET, path))
                else:
                    raise ValueError(f"unknown layer code {code!r}")
                for t, vl in out:
                    conn[t].append(vl)
                    lay[t].append(k)
                    c2[t].append(ck)
    if centres:
        verts.append(np.array(centres))
    xyz = np.concatenate(verts, axis=0)
    # orientation of tets is fixed on the final coordinates (all other types are
    # positively oriented by construction)
    conn[TET] = [_orient_tet(xyz, t) for t in conn[TET]]
    conn = [np.array(c, dtype=np.int32).reshape(-1, NVERT[t]) for t, c in enumerate(conn)]
    c2 = [np.array(c, dtype=np.float64) for c in c2]
    lay = [np.array(x, dtype=np.int32) for x in lay]
    return HybridMesh(xyz=xyz, conn=conn, c2=c2, layer=lay, dims=(nx, ny, nz), layers=layers)


def small_hybrid_mesh(seed=0):
    """4x4x5 cells, layers hex | wedge | hex | transition | Kuhn, c = 1."""
    return layered_mesh(4, 4, 5, "HWHTK", seed=seed)


def scale_layers():
    """Layer codes of the 80-layer throughput mesh (72 hex, 2 wedge, 2 transition, 4 Kuhn)."""
    return "H" * 34 + "W" * 2 + "H" * 36 + "T" + "K" * 4 + "U" + "H" * 2


def scale_mesh(nx=64, ny=64, seed=0):
    """64x64x80-cell throughput mesh, c alternating 1.0 / 1.5 by layer parity."""
    L = scale_layers()
    return layered_mesh(nx, ny, len(L), L, seed=seed,
                        c_of_layer=lambda k: 1.0 if k % 2 == 0 else 1.5)


def random_state(ndof, seed=0):
    """(4, ndof) float64 standard-normal state: p, u, v, w."""
    return np.random.default_rng(seed).standard_normal((4, ndof))


def batch_specs(count=256, seed=0, nmin=6, nmax=40):
    """Seeded recipe of the many-mesh workload, one (n, N, layers, c per layer) per mesh:
    n log-uniform in [nmin, nmax] (an n x n x n cell grid), N uniform in {2..6}, layer codes
    H*a | W | H*b | T | K*k with k = max(1, round(0.05 n)), a = (n - 2 - k) // 2,
    b = n - 2 - k - a, and c uniform in [1, 3] per layer."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(round(float(np.exp(rng.uniform(np.log(nmin), np.log(nmax))))))
        N = int(rng.integers(2, 7))
        k = max(1, int(round(0.05 * n)))
        a = (n - 2 - k) // 2
        b = n - 2 - k - a
        layers = "H" * a + "W" + "H" * b + "T" + "K" * k
        c = rng.uniform(1.0, 3.0, size=len(layers))
        out.append((n, N, layers, c))
    return out


def batch_mesh(spec, seed=0):
    """The layered mesh of one batch_specs entry (c^2 from its per-layer wave speeds)."""
    n, _, layers, c = spec
    return layered_mesh(n, n, n, layers, seed=seed, c_of_layer=lambda k: float(c[k]))
