"""dg_energy_noalloc: the energy for callers that cannot allocate device memory.

Such callers (code inside a CUDA stream capture, real-time loops, frameworks that
have reserved all device memory) get the energy from a static device scratch
array instead of an allocation.  This file is collected last so that a failing
run that stops at the first failure has already run every other test.
"""
import numpy as np
import pytest

from paper_1507_02557_b300.inputs import layered_mesh, random_state, small_hybrid_mesh

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
TOL = 1e-6          # the energy tolerance of the other GPU tests


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1507_02557_b300 import dg
    return dg


def test_noalloc_energy_matches_dg_energy_twice(lib):
    g = lib.Mesh(small_hybrid_mesh(), 3)
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
