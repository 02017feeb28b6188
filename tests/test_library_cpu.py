"""libdg on the CPU: exported symbols and the host setup against the oracle (no GPU calls)."""
import os
import re

import numpy as np
import pytest

from oracle.constants import trace_constant
from oracle.dg import DGOracle
from paper_1507_02557_b300.inputs import layered_mesh, small_hybrid_mesh

dg = pytest.importorskip("paper_1507_02557_b300.dg")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_every_declared_symbol_is_exported():
    hdr = open(os.path.join(ROOT, "include", "dg.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    declared = set(re.findall(r"\b(dg_[a-z_]+)\s*\(", hdr))
    assert {"dg_mesh_create", "dg_rhs", "dg_step", "dg_energy", "dg_set_state"} <= declared
    for name in declared:
        assert hasattr(dg._lib, name), name
    assert declared == set(dg.EXPORTS)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 9])
def test_host_setup_time_step_matches_oracle(N):
    """Eq. dtK computed by the library's own host setup vs the oracle."""
    m = small_hybrid_mesh()
    dt, ct = dg.host_check(m, N)
    o = DGOracle(m, N)
    cto = [trace_constant(t, N) for t in range(4)]
    assert np.allclose(ct, cto, rtol=1e-12)
    assert abs(dt - o.global_dt(cto)) < 1e-12 * dt


def test_host_setup_wave_speed_jump():
    m = layered_mesh(3, 3, 5, "HWHTK", seed=3, c_of_layer=lambda k: 1.0 if k % 2 == 0 else 1.5)
    dt, _ = dg.host_check(m, 3)
    o = DGOracle(m, 3)
    assert abs(dt - o.global_dt([trace_constant(t, 3) for t in range(4)])) < 1e-12 * dt


def test_host_trace_constants_against_paper_table():
    """Library C_T(N) vs the printed Table computedTrace (independent of the oracle)."""
    tab = {1: [9, 9.93, 11.68, 12.22], 4: [45, 42.99, 47.59, 41.65], 8: [135, 123.76, 135.07, 109.04],
           9: [165, 150.48, 164.11, 130.67]}
    for N, row in tab.items():
        _, ct = dg.host_check(small_hybrid_mesh(), N)
        assert np.allclose(ct, row, atol=0.006)


@pytest.mark.parametrize("N", [1, 2, 4])
def test_host_setup_sem_matches_oracle_and_table(N):
    """SEM hexahedra (hex_basis 1): C_SEM(N) of the printed Table computedTraceSEM for hex, wedge
    and pyramid, and dt equal to the oracle's with the same rules."""
    m = small_hybrid_mesh()
    dt, ct = dg.host_check(m, N, hex_basis=1)
    tab = {1: [3, 46.46, 31.58], 2: [9, 51.70, 37.12], 4: [30, 83.32, 60.95]}[N]
    assert np.allclose(ct[:3], tab, atol=0.006)
    o = DGOracle(m, N, hex_basis="gll")
    cto = [trace_constant(t, N, lobatto=True) for t in range(4)]
    assert np.allclose(ct, cto, rtol=1e-12)
    assert abs(dt - o.global_dt(cto)) < 1e-12 * dt


def test_host_setup_rejects_bad_meshes():
    m = small_hybrid_mesh()
    with pytest.raises(dg.DGError, match="not supported"):
        dg.host_check(m, 10)          # orders 1..9 are built
    bad = small_hybrid_mesh()
    c = bad.conn[0].copy()
    c[0] = c[0][[1, 0, 3, 2, 5, 4, 7, 6]]          # mirrored hexahedron: J < 0
    bad.conn[0] = c
    with pytest.raises(dg.DGError, match="invalid mesh"):
        dg.host_check(bad, 2)
    dup = small_hybrid_mesh()
    dup.conn[0] = np.concatenate([dup.conn[0], dup.conn[0][:1]])   # a face shared three times
    dup.c2[0] = np.concatenate([dup.c2[0], dup.c2[0][:1]])
    with pytest.raises(dg.DGError, match="invalid mesh"):
        dg.host_check(dup, 2)
    neg = small_hybrid_mesh()
    neg.c2[3] = -neg.c2[3]
    with pytest.raises(dg.DGError, match="invalid argument"):
        dg.host_check(neg, 2)


@pytest.mark.parametrize("kw", [dict(precision=3), dict(precision=-1), dict(hex_basis=2), dict(nlevels=3),
                                dict(integrator=2)])
def test_mesh_create_rejects_unbuilt_options_before_touching_a_device(kw):
    """dg_mesh_create checks the descriptor's options first: an option value that is not built
    returns DG_ENOTSUP with a message naming the built ones, also on a machine without a GPU."""
    with pytest.raises(dg.DGError, match="not supported"):
        dg.Mesh(small_hybrid_mesh(), 2, **kw)


def test_host_setup_multirate_levels_match_oracle():
    """Sec. 2.4 level binning and neighbour smoothing: library vs oracle element counts."""
    from oracle.dg import mr_levels
    m = layered_mesh(3, 3, 5, "HWHTK", seed=3, c_of_layer=lambda k: 1.0 if k % 2 == 0 else 1.5)
    N = 2
    _, _, lc = dg.host_check(m, N, nlevels=2, levels=True)
    o = DGOracle(m, N)
    lev, _ = mr_levels(o, [trace_constant(t, N) for t in range(4)], 2)
    want = [sum(int(np.sum(l == L)) for l in lev) for L in (1, 2)]
    assert lc == want and lc[1] > 0


def test_batch_calls_reject_bad_arguments_without_a_device():
    """dg_batch_* argument checks come before any CUDA call."""
    import ctypes as C
    h = C.c_void_p()
    assert dg._lib.dg_batch_create(None, 0, None, C.byref(h)) == -1 and not h.value
    arr = (C.c_void_p * 2)(None, None)
    assert dg._lib.dg_batch_create(arr, 2, None, C.byref(h)) == -1
    assert dg._lib.dg_batch_step(None, 3, None, None) == -1
    assert dg._lib.dg_batch_stats(None, None, None) == -1
    dg._lib.dg_batch_destroy(None)


def test_device_byte_budget_fails_cleanly_before_allocating(monkeypatch):
    """Host-side out-of-memory injection: with a device byte budget the setup stops with
    DG_ENOMEM before its first cudaMalloc (and frees what it holds)."""
    monkeypatch.setenv("DG_DEVICE_BYTES_LIMIT", "1")
    with pytest.raises(dg.DGError, match="out of device memory.*DG_DEVICE_BYTES_LIMIT"):
        dg.Mesh(small_hybrid_mesh(), 2)
