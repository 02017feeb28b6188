"""Tensor-core volume products of tets and pyramids, and the first volume contraction of the wedges,
in split 16-bit precision (precision 1 = BF16 x 3, 2 = FP16 x 3) against the FP64 oracle.

Tolerances from the arithmetic of the split (x = x_hi + x_lo, product x_hi b_hi + x_hi b_lo +
x_lo b_hi accumulated in FP32):
* FP16 (11 significant bits per part): each operand is held to 2^-24 relative and the dropped
  x_lo b_lo term is below 2^-22 |x b|, so products are FP32-class; the tolerance is the FP32 one,
  relative L2 1e-5.
* BF16 (8 bits per part): each operand to 2^-18, the dropped term below 2^-18 |x b|, i.e. about
  3 * 2^-18 = 1.1e-5 relative per product; the tolerance allows a cancellation factor of 3 in the
  operator sums, relative L2 3e-5 (measured: 3e-6 - 4e-6 on pyramids, below 1e-6 on tets).
"""
import numpy as np
import pytest

from oracle.dg import DGOracle
from paper_1507_02557_b300.inputs import layered_mesh, random_state, small_hybrid_mesh

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
TOL = {1: 3e-5, 2: 1e-5}


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1507_02557_b300 import dg
    return dg


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def per_type(o, a, b):
    return [rel(o.split(a)[t], o.split(b)[t]) for t in range(4) if o.K[t]]


@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6, 7, 8, 9])
def test_rhs_matches_oracle(lib, N, precision):
    """N = 8, 9: the pyramids (285 and 385 nodes, more than one MMA's N of 256) compute each
    output block of the GEMM in two halves."""
    meshes = [small_hybrid_mesh()]
    if N in (2, 5):   # wave-speed jumps and both transition layers
        meshes.append(layered_mesh(3, 2, 6, "HTKKUH", seed=2, c_of_layer=lambda k: 1.0 + 0.4 * (k % 2)))
    for m in meshes:
        o = DGOracle(m, N)
        q32 = random_state(o.ndof, 17).astype(np.float32)
        want = o.rhs(q32.astype(np.float64))
        g = lib.Mesh(m, N, precision=precision)
        qd = torch.from_numpy(q32).cuda()
        rd = torch.zeros_like(qd)
        g.rhs(qd, rd)
        got = rd.cpu().numpy().astype(np.float64)
        errs = per_type(o, got, want)
        assert rel(got, want) < TOL[precision] and max(errs) < TOL[precision], errs


@pytest.mark.parametrize("precision", [1, 2])
def test_lsrk_steps_match_oracle(lib, precision):
    """Ten LSRK(5,4) steps at N = 4 from the projected standing mode."""
    from oracle.dg import standing_mode
    m, N = small_hybrid_mesh(), 4
    o = DGOracle(m, N)
    q0 = o.project(standing_mode, 0.0).astype(np.float32)
    g = lib.Mesh(m, N, precision=precision)
    dt = g.timestep()
    g.set_state(q0, on_device=False)
    g.step(10, dt)
    got = g.get_state(np.zeros_like(q0), on_device=False).astype(np.float64)
    q = q0.astype(np.float64)
    for _ in range(10):
        q = o.lsrk_step(q, dt)
    assert rel(got, q) < TOL[precision], per_type(o, got, q)


@pytest.mark.parametrize("precision", [1, 2])
def test_multirate_matches_oracle(lib, precision):
    """Start-up + 3 coarse MRAB3 steps at N = 4: the fused coarse / fine kernels of tets and
    pyramids take their volume products from the tensor-core pass of their level's elements."""
    from oracle.constants import trace_constant
    from oracle.dg import MRAB3, mr_levels, standing_mode
    m, N = layered_mesh(3, 3, 5, "HWHTK", seed=3, c_of_layer=lambda k: 1.0 if k % 2 == 0 else 1.5), 4
    o = DGOracle(m, N)
    lev, _ = mr_levels(o, [trace_constant(t, N) for t in range(4)], 2)
    g = lib.Mesh(m, N, nlevels=2, precision=precision)
    h = g.timestep()
    q0 = o.project(standing_mode, 0.0).astype(np.float32)
    g.set_state(q0, on_device=False)
    g.step(3, h)
    got = g.get_state(np.zeros_like(q0), on_device=False).astype(np.float64)
    mr = MRAB3(o, lev)
    q, hist = mr.start(q0.astype(np.float64), h)
    for _ in range(3):
        q, hist = mr.step(q, hist, h)
    assert rel(got, q) < TOL[precision], per_type(o, got, q)


@pytest.mark.parametrize("N", [7, 9])
def test_single_wedge_against_a_tet(lib, N):
    """One wedge and one tet sharing a triangle face (the quadrature-point face exchange; the tet
    keeps its FP32 kernel there): the wedge's tensor-core pass on a single element, 8 or 10 rows
    of one 128-row tile."""
    from paper_1507_02557_b300.inputs import HybridMesh
    xyz = np.array([[0, 0, 0], [1, 0, 0], [0, 0, 1], [0, 1, 0], [1, 1, 0], [0, 1, 1], [0, -1, 0]], float)
    conn = [np.zeros((0, 8), np.int32), np.array([[0, 1, 2, 3, 4, 5]], np.int32),
            np.zeros((0, 5), np.int32), np.array([[0, 1, 2, 6]], np.int32)]
    m = HybridMesh(xyz=xyz, conn=conn, c2=[np.zeros(0), np.array([1.0]), np.zeros(0), np.array([2.25])])
    o = DGOracle(m, N)
    q32 = random_state(o.ndof, 23).astype(np.float32)
    want = o.rhs(q32.astype(np.float64))
    g = lib.Mesh(m, N, precision=2)
    qd = torch.from_numpy(q32).cuda()
    rd = torch.zeros_like(qd)
    g.rhs(qd, rd)
    got = rd.cpu().numpy().astype(np.float64)
    assert rel(got, want) < TOL[2], per_type(o, got, want)


@pytest.mark.parametrize("N", [6, 7])
def test_sem_rhs_matches_oracle(lib, N):
    """SEM hexahedra (GLL nodes; GLL points on the quadrilateral faces of wedges and pyramids too)
    with FP16 x 3 products at N = 6, 7 (the column hex kernel; at N = 7 the wedges' tensor-core
    pass with the SEM face rules around it)."""
    m = small_hybrid_mesh()
    o = DGOracle(m, N, hex_basis="gll")
    q32 = random_state(o.ndof, 19).astype(np.float32)
    want = o.rhs(q32.astype(np.float64))
    g = lib.Mesh(m, N, hex_basis=1, precision=2)
    qd = torch.from_numpy(q32).cuda()
    rd = torch.zeros_like(qd)
    g.rhs(qd, rd)
    got = rd.cpu().numpy().astype(np.float64)
    errs = per_type(o, got, want)
    assert rel(got, want) < TOL[2] and max(errs) < TOL[2], errs


@pytest.mark.parametrize("N", [5, 7])
def test_multirate_unfused_matches_oracle(lib, N):
    """Start-up + 3 coarse MRAB3 steps at N = 5, 7 (FP16 x 3): the unfused schedule evaluates the
    rhs on each level's element lists, so the tensor-core pass packs and multiplies only the
    listed elements (at N = 7 the wedges' too; this mesh has no fine wedges, an empty list)."""
    from oracle.constants import trace_constant
    from oracle.dg import MRAB3, mr_levels, standing_mode
    m = layered_mesh(3, 3, 5, "HWHTK", seed=3, c_of_layer=lambda k: 1.0 if k % 2 == 0 else 1.5)
    o = DGOracle(m, N)
    lev, _ = mr_levels(o, [trace_constant(t, N) for t in range(4)], 2)
    g = lib.Mesh(m, N, nlevels=2, precision=2)
    h = g.timestep()
    q0 = o.project(standing_mode, 0.0).astype(np.float32)
    g.set_state(q0, on_device=False)
    g.step(3, h)
    got = g.get_state(np.zeros_like(q0), on_device=False).astype(np.float64)
    mr = MRAB3(o, lev)
    q, hist = mr.start(q0.astype(np.float64), h)
    for _ in range(3):
        q, hist = mr.step(q, hist, h)
    assert rel(got, q) < TOL[2], per_type(o, got, q)


@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("N", [3, 5])
def test_error_against_exact_mode(lib, N, precision):
    """FP16 x 3 (FP32-class products) leaves the L2 error against the exact standing mode where the
    FP64 oracle has it (within 5 %: equal error).  BF16 x 3 does at N = 3; at N = 5, where the
    discretisation error of this mesh after these steps (2e-6) approaches the split's rounding
    (2^-17 per product times the operators' cancellation), its error is up to 1.5 times the
    oracle's (measured 1.22): BF16 x 3 is not an equal-error replacement at high order here."""
    from oracle.dg import standing_mode
    m = small_hybrid_mesh()
    o = DGOracle(m, N)
    q0 = o.project(standing_mode, 0.0)
    g = lib.Mesh(m, N, precision=precision)
    T = 0.02 if N <= 4 else 0.01
    n = int(np.ceil(T / g.timestep()))
    dt = T / n
    g.set_state(q0.astype(np.float32), on_device=False)
    g.step(n, dt)
    got = g.get_state(np.zeros(q0.shape, np.float32), on_device=False).astype(np.float64)
    q = q0.copy()
    for _ in range(n):
        q = o.lsrk_step(q, dt)
    e_gpu, e_orc = o.l2_error(got, standing_mode, T), o.l2_error(q, standing_mode, T)
    bound = 0.5 if (precision == 1 and N >= 5) else 0.05
    assert abs(e_gpu - e_orc) <= bound * e_orc, (e_gpu, e_orc)


def test_adjoint_refuses_split_precision(lib):
    g = lib.Mesh(small_hybrid_mesh(), 2, precision=2)
    lam = torch.zeros((4, g.ndof), dtype=torch.float32, device="cuda")
    with pytest.raises(lib.DGError, match="not supported"):
        g.adjoint_step(1, lam)
