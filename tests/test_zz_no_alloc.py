"""dg_energy_noalloc: the energy for callers that cannot allocate device memory.

Such callers (real-time loops that cannot take the latency of cudaMalloc, frameworks that have
reserved all device memory for their own pool) get the energy from a static device scratch array
instead of an allocation.  This file is collected last so that a failing run that stops at the
first failure has already run every other test.
"""
import numpy as np
import pytest

from paper_1507_02557_b300.inputs import HybridMesh, layered_mesh, random_state, small_hybrid_mesh

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
TOL = 1e-6          # the energy tolerance of the other GPU tests
LIMIT = 1 << 20     # elements of the static scratch array


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1507_02557_b300 import dg
    return dg


@pytest.mark.parametrize("N", [1, 3, 4, 7, 9])
def test_noalloc_energy_matches_dg_energy_twice(lib, N):
    """Every element type at low, middle and the highest order (the tet branch forms its
    O(Np^2) FP64 mass product per node)."""
    g = lib.Mesh(small_hybrid_mesh(), N)
    q = torch.from_numpy(random_state(g.ndof, 4).astype(np.float32)).cuda()
    ref = g.energy(q)
    e1 = g.energy_noalloc(q)
    e2 = g.energy_noalloc(q)
    assert abs(e1 - ref) <= TOL * ref
    assert abs(e2 - ref) <= TOL * ref
    assert e1 == e2                      # fixed summation order
    # a smaller mesh afterwards: stale partial sums of the previous call must not leak in
    h = lib.Mesh(layered_mesh(2, 2, 3, "HHH", seed=1), 2)
    qh = torch.from_numpy(random_state(h.ndof, 5).astype(np.float32)).cuda()
    assert abs(h.energy_noalloc(qh) - h.energy(qh)) <= TOL * h.energy(qh)


def test_noalloc_energy_reports_a_nonfinite_state(lib):
    """A NaN written into the state by the host gives DG_ENONFINITE, as from dg_energy; the mesh
    keeps working afterwards."""
    g = lib.Mesh(small_hybrid_mesh(), 3)
    q = random_state(g.ndof, 2).astype(np.float32)
    bad = q.copy()
    bad[1, 40] = np.nan
    g.set_state(bad, on_device=False)
    with pytest.raises(lib.DGError, match="non-finite"):
        g.energy_noalloc()
    g.set_state(q, on_device=False)
    assert abs(g.energy_noalloc() - g.energy()) <= TOL * g.energy()


def hex_grid(nx, ny, nz):
    """Undisplaced all-hex grid of nx*ny*nz cells on [-1,1]^3 (vectorised: a million cells)."""
    xs, ys, zs = (np.linspace(-1.0, 1.0, n + 1) for n in (nx, ny, nz))
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    xyz = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    base = (i + (nx + 1) * (j + (ny + 1) * k)).ravel()
    off = [a + (nx + 1) * (b + (ny + 1) * c) for c in (0, 1) for b in (0, 1) for a in (0, 1)]
    conn = (base[:, None] + np.array(off)[None, :]).astype(np.int32)
    empty = [np.zeros((0, n), np.int32) for n in (6, 5, 4)]
    c2 = [np.ones(len(conn))] + [np.zeros(0)] * 3
    return HybridMesh(xyz=xyz, conn=[conn] + empty, c2=c2, dims=(nx, ny, nz), layers="H" * nz)


def test_noalloc_energy_rejects_meshes_above_the_limit(lib):
    """A mesh of more than 2^20 elements does not fit the static array: DG_EINVAL with the
    limit in the message, before any kernel runs; dg_energy (which allocates) still works."""
    m = hex_grid(128, 128, 65)
    assert sum(m.nelem) > LIMIT
    g = lib.Mesh(m, 1)
    with pytest.raises(lib.DGError, match="static scratch limit"):
        g.energy_noalloc()
    assert np.isfinite(g.energy())
