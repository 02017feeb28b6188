"""Sampled oracle checks on meshes too large for the oracle.

The rhs of an element depends on its own state and on the traces of its face neighbours only
(Sec. 2.2: the numerical flux couples the two sides of a face, nothing else).  So the rhs at a
set S of elements is computed exactly by the oracle on the sub-mesh made of S and its face
neighbours: the neighbours' own rhs are wrong there (their other neighbours are missing and
become walls), but S's are those of the whole mesh.  One LSRK step has five stages, each of
which widens the region whose values are exact by one ring less, so S after a step needs the
sub-mesh of S and five rings of neighbours.

submesh() builds that sub-mesh (same vertex array, the kept elements in their original order per
type) and dof_index() maps its DOFs to the DOFs of the whole mesh (the [4][ndof] layout: types
one after the other, elements in order, nodes of an element contiguous), so that a state of the
whole mesh can be gathered into the sub-mesh's layout and results compared at S.
"""
import numpy as np
import scipy.sparse as sp

from paper_1507_02557_b300.inputs import HybridMesh, nodes_per_element


def _incidence(mesh):
    """(elements x vertices) 0/1 matrix over all elements, types one after the other."""
    rows, cols = [], []
    base = 0
    for c in mesh.conn:
        k, nv = c.shape
        rows.append(np.repeat(np.arange(base, base + k), nv))
        cols.append(c.reshape(-1).astype(np.int64))
        base += k
    rows, cols = np.concatenate(rows), np.concatenate(cols)
    return sp.csr_matrix((np.ones(rows.size, np.int32), (rows, cols)), shape=(base, mesh.xyz.shape[0]))


def submesh(mesh, samples, rings):
    """samples: per type, element indices.  Returns (sub-mesh, keep) with keep[t] the sorted
    element indices of type t in the sub-mesh: the samples and every element within `rings`
    face-neighbour steps of them (two elements are face neighbours when they share at least three
    vertices; in a conforming mesh that is exactly a shared face)."""
    A = _incidence(mesh)
    AT = A.T.tocsr()
    start = np.concatenate([[0], np.cumsum(mesh.nelem)])
    cur = np.unique(np.concatenate([np.asarray(s, np.int64) + start[t] for t, s in enumerate(samples)]))
    for _ in range(rings):
        shared = (A[cur] @ AT).tocoo()
        cur = np.union1d(cur, shared.col[shared.data >= 3])
    keep = [cur[(cur >= start[t]) & (cur < start[t + 1])] - start[t] for t in range(4)]
    sub = HybridMesh(xyz=mesh.xyz, conn=[mesh.conn[t][keep[t]] for t in range(4)],
                     c2=[np.asarray(mesh.c2[t])[keep[t]] for t in range(4)],
                     layer=[np.asarray(mesh.layer[t])[keep[t]] for t in range(4)] if mesh.layer else [],
                     dims=mesh.dims, layers=mesh.layers)
    return sub, keep


def dof_index(mesh, keep, N):
    """Indices into one field of the whole mesh's state for the sub-mesh's DOFs, in the
    sub-mesh's layout."""
    npn = nodes_per_element(N)
    off = np.concatenate([[0], np.cumsum([k * n for k, n in zip(mesh.nelem, npn)])])
    parts = [off[t] + (np.asarray(keep[t], np.int64)[:, None] * npn[t] + np.arange(npn[t])[None, :]).reshape(-1)
             for t in range(4)]
    return np.concatenate(parts)


def sample_positions(keep, samples, N):
    """For each type, the sub-mesh DOF indices (one field) of the sampled elements, in sample order."""
    npn = nodes_per_element(N)
    ksub = [len(k) for k in keep]
    off = np.concatenate([[0], np.cumsum([k * n for k, n in zip(ksub, npn)])])
    out = []
    for t in range(4):
        pos = np.searchsorted(keep[t], np.asarray(samples[t], np.int64))
        out.append((off[t] + (pos[:, None] * npn[t] + np.arange(npn[t])[None, :])).reshape(-1))
    return out


def pick_samples(mesh, per_type, seed=0):
    """Per type: `per_type` random elements, plus the first and last element of the type (at the
    mesh's walls) and one element of the type's lowest and highest layer (next to the layers of
    other types)."""
    rng = np.random.default_rng(seed)
    out = []
    for t in range(4):
        k = mesh.nelem[t]
        if k == 0:
            out.append(np.zeros(0, np.int64))
            continue
        s = set(rng.choice(k, size=min(per_type, k), replace=False).tolist()) | {0, k - 1}
        if mesh.layer:
            lay = np.asarray(mesh.layer[t])
            for L in (lay.min(), lay.max()):
                idx = np.nonzero(lay == L)[0]
                s.add(int(idx[rng.integers(idx.size)]))
        out.append(np.array(sorted(s), np.int64))
    return out
