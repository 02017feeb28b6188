"""Failure reporting on the GPU, with the failures made on the host (no GPU fault):

* out of device memory: a device byte budget (DG_DEVICE_BYTES_LIMIT) makes dg_mesh_create fail
  with DG_ENOMEM part-way through its uploads; the next creation without the budget works;
* a non-finite state (a NaN written by the host) is reported by dg_energy as DG_ENONFINITE, and the
  mesh keeps working once a finite state is set again.
"""
import numpy as np
import pytest

from paper_1507_02557_b300.inputs import random_state, small_hybrid_mesh

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1507_02557_b300 import dg
    return dg


def test_device_budget_then_recovery(lib, monkeypatch):
    m = small_hybrid_mesh()
    monkeypatch.setenv("DG_DEVICE_BYTES_LIMIT", str(256 << 10))
    with pytest.raises(lib.DGError, match="out of device memory"):
        lib.Mesh(m, 4)
    monkeypatch.delenv("DG_DEVICE_BYTES_LIMIT")
    g = lib.Mesh(m, 4)
    g.set_state(random_state(g.ndof, 1).astype(np.float32), on_device=False)
    g.step(2)
    assert np.isfinite(g.energy())


def test_nonfinite_state_is_reported(lib):
    g = lib.Mesh(small_hybrid_mesh(), 3)
    q = random_state(g.ndof, 2).astype(np.float32)
    bad = q.copy()
    bad[2, 17] = np.nan
    g.set_state(bad, on_device=False)
    with pytest.raises(lib.DGError, match="non-finite"):
        g.energy()
    g.set_state(q, on_device=False)
    g.step(1)
    assert np.isfinite(g.energy())
