"""CUDA path (libdg through its C ABI) against the FP64 oracle, element by element.

Tolerance: relative L2 difference <= 1e-5 over all four fields (the FP32
tolerance of the method's GPU/oracle comparison), also checked per element type.
"""
import numpy as np
import pytest

from oracle.dg import DGOracle
from paper_1507_02557_b300.inputs import layered_mesh, random_state, small_hybrid_mesh

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1507_02557_b300 import dg
    return dg


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def per_type_rel(o, a, b):
    out = []
    for t in range(4):
        if o.K[t]:
            out.append(rel(o.split(a)[t], o.split(b)[t]))
    return out


def gpu_rhs(lib, m, N, q32, **kw):
    g = lib.Mesh(m, N, **kw)
    qd = torch.from_numpy(q32).cuda()
    rd = torch.zeros_like(qd)
    g.rhs(qd, rd)
    torch.cuda.synchronize()
    return rd.cpu().numpy().astype(np.float64), g


MESHES = {
    "hybrid": lambda: small_hybrid_mesh(),
    "cjump": lambda: layered_mesh(3, 3, 5, "HWHTK", seed=3, c_of_layer=lambda k: 1.0 if k % 2 == 0 else 1.5),
    "ragged": lambda: layered_mesh(5, 3, 6, "HHWHTK", seed=5),         # odd counts, tail blocks
    "inverted": lambda: layered_mesh(3, 2, 6, "HTKKUH", seed=2),       # both transition layers
}


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6, 7, 8, 9])
@pytest.mark.parametrize("name", ["hybrid", "cjump", "ragged", "inverted"])
def test_rhs_matches_oracle(lib, name, N):
    """Every mesh at every order N = 1..9: the c-jump and both-transition meshes reach the N >= 5
    kernel instantiations with wave-speed jumps and the inverted transition layer."""
    m = MESHES[name]()
    for ts in (1.0, 0.0):
        o = DGOracle(m, N, tau_scale=ts)
        q32 = random_state(o.ndof, 11).astype(np.float32)
        want = o.rhs(q32.astype(np.float64))
        got, _ = gpu_rhs(lib, m, N, q32, tau_scale=ts)
        errs = per_type_rel(o, got, want)
        assert rel(got, want) < TOL and max(errs) < TOL, (ts, errs)


def test_rhs_single_type_meshes(lib):
    for L in ("HHH", "KKK", "WWW"):
        m = layered_mesh(2, 3, 3, L, seed=4)
        o = DGOracle(m, 3)
        q32 = random_state(o.ndof, 5).astype(np.float32)
        got, _ = gpu_rhs(lib, m, 3, q32)
        assert rel(got, o.rhs(q32.astype(np.float64))) < TOL, L


@pytest.mark.parametrize("N", [2, 3, 4, 6, 8])
def test_lsrk_steps_match_oracle(lib, N):
    """Ten LSRK(5,4) steps at the paper's dt from the projected standing mode (N = 4: the
    hexahedra run the TMA-staged stage kernel; N = 6: the pyramids read their operators from
    global memory, the tets and wedges keep them in shared memory with fewer warps; N = 8: every
    operator from global memory, hexahedra in blocks of 736 threads)."""
    from oracle.dg import standing_mode
    m = small_hybrid_mesh()
    o = DGOracle(m, N)
    q0 = o.project(standing_mode, 0.0).astype(np.float32)
    g = lib.Mesh(m, N)
    dt = g.timestep()
    g.set_state(q0, on_device=False)
    g.step(10, dt)
    got = g.get_state(np.zeros_like(q0), on_device=False).astype(np.float64)
    q = q0.astype(np.float64)
    for _ in range(10):
        q = o.lsrk_step(q, dt)
    assert rel(got, q) < TOL, per_type_rel(o, got, q)


def test_energy_matches_oracle(lib):
    m = small_hybrid_mesh(seed=1)
    o = DGOracle(m, 3)
    q32 = random_state(o.ndof, 2).astype(np.float32)
    g = lib.Mesh(m, 3)
    qd = torch.from_numpy(q32).cuda()
    E = g.energy(qd)
    Eo = o.energy(q32.astype(np.float64))
    assert abs(E - Eo) < 1e-6 * Eo


def test_energy_nonincreasing_under_upwind_steps(lib):
    m = small_hybrid_mesh()
    o = DGOracle(m, 3)
    q0 = o.project(lambda x, t: np.stack([np.exp(-8 * np.sum(x ** 2, 1)), 0 * x[:, 0], 0 * x[:, 0], 0 * x[:, 0]]))
    g = lib.Mesh(m, 3)
    g.set_state(q0.astype(np.float32), on_device=False)
    E = [g.energy()]
    for _ in range(5):
        g.step(4)
        E.append(g.energy())
    assert all(b <= a * (1 + 1e-6) for a, b in zip(E, E[1:])), E


def test_state_roundtrip_and_layout(lib):
    m = small_hybrid_mesh()
    g = lib.Mesh(m, 2)
    o = DGOracle(m, 2)
    assert g.ndof == o.ndof
    for t in range(4):
        off, K, npn = g.layout(t)
        assert (off, K, npn) == (o.off[t], o.K[t], o.Np[t])
    q = random_state(g.ndof, 9).astype(np.float32)
    g.set_state(q, on_device=False)
    back = g.get_state(np.zeros_like(q), on_device=False)
    assert np.array_equal(back, q)


@pytest.mark.parametrize("N", [2, 3, 4, 5, 9])
def test_multirate_ab3_matches_oracle(lib, N):
    """Two-level MRAB3 (Sec. 2.4 reading): start-up + 5 coarse steps vs the oracle
    (fused kernels for N <= 4, separate rhs / AB3 kernels for N = 5)."""
    from oracle.constants import trace_constant
    from oracle.dg import MRAB3, mr_levels, standing_mode
    m = MESHES["cjump"]()
    o = DGOracle(m, N)
    lev, dmin = mr_levels(o, [trace_constant(t, N) for t in range(4)], 2)
    g = lib.Mesh(m, N, nlevels=2)
    assert g.level_counts() == [sum(int(np.sum(l == L)) for l in lev) for L in (1, 2)]
    for L in (1, 2):
        assert g.level_type_counts(L) == [int(np.sum(l == L)) for l in lev]
    # coarse elements with a fine face neighbour (the writers of the half-step traces)
    iface = [set() for _ in range(4)]
    for sd in o.geo.sides:
        if sd.nbr >= 0:
            nb = o.geo.sides[sd.nbr]
            if lev[sd.t][sd.e] == 1 and lev[nb.t][nb.e] == 2:
                iface[sd.t].add(sd.e)
    assert g.level_type_counts(-1) == [len(x) for x in iface]
    h = g.timestep()
    assert abs(h - dmin) < 1e-12 * dmin
    q0 = o.project(standing_mode, 0.0).astype(np.float32)
    g.set_state(q0, on_device=False)
    t = g.step(5, h)
    got = g.get_state(np.zeros_like(q0), on_device=False).astype(np.float64)
    mr = MRAB3(o, lev)
    q, hist = mr.start(q0.astype(np.float64), h)
    for _ in range(5):
        q, hist = mr.step(q, hist, h)
    assert abs(t - 14 * h) < 1e-12
    assert rel(got, q) < TOL, per_type_rel(o, got, q)


def wedge_tet_mesh():
    """One wedge and one tet sharing a triangle face, c^2 = 1 and 2.25: a wedge triangle face
    against a tet selects the quadrature-point face exchange for tets and pyramids."""
    from paper_1507_02557_b300.inputs import HybridMesh
    xyz = np.array([[0, 0, 0], [1, 0, 0], [0, 0, 1], [0, 1, 0], [1, 1, 0], [0, 1, 1], [0, -1, 0]], float)
    conn = [np.zeros((0, 8), np.int32), np.array([[0, 1, 2, 3, 4, 5]], np.int32),
            np.zeros((0, 5), np.int32), np.array([[0, 1, 2, 6]], np.int32)]
    c2 = [np.zeros(0), np.array([1.0]), np.zeros(0), np.array([2.25])]
    return HybridMesh(xyz=xyz, conn=conn, c2=c2)


@pytest.mark.parametrize("N", [2, 4, 8, 9])
def test_wedge_tet_triangle_face_rhs(lib, N):
    m = wedge_tet_mesh()
    o = DGOracle(m, N)
    q32 = random_state(o.ndof, 3).astype(np.float32)
    got, _ = gpu_rhs(lib, m, N, q32)
    assert rel(got, o.rhs(q32.astype(np.float64))) < TOL


def test_wedge_tet_triangle_face_multirate(lib):
    """Start-up + 3 coarse MRAB3 steps through the unfused schedule of this mesh."""
    from oracle.constants import trace_constant
    from oracle.dg import MRAB3, mr_levels, standing_mode
    m, N = wedge_tet_mesh(), 3
    o = DGOracle(m, N)
    lev, dmin = mr_levels(o, [trace_constant(t, N) for t in range(4)], 2)
    g = lib.Mesh(m, N, nlevels=2)
    h = g.timestep()
    q0 = o.project(standing_mode, 0.0).astype(np.float32)
    g.set_state(q0, on_device=False)
    g.step(3, h)
    got = g.get_state(np.zeros_like(q0), on_device=False).astype(np.float64)
    mr = MRAB3(o, lev)
    q, hist = mr.start(q0.astype(np.float64), h)
    for _ in range(3):
        q, hist = mr.step(q, hist, h)
    assert rel(got, q) < TOL


def test_watchdog_reports_timeout(lib):
    """A bounded device wait that runs out (on an mbarrier nothing arrives on) is reported as
    DG_ETIMEOUT by the synchronizing call; the word is cleared and the mesh stays usable."""
    m = small_hybrid_mesh()
    g = lib.Mesh(m, 2)
    assert g.watchdog_selftest(1 << 20) == -5
    g.set_state(random_state(g.ndof, 1).astype(np.float32), on_device=False)
    g.step(1)
    assert np.isfinite(g.energy())


@pytest.mark.parametrize("N", [2, 3, 4, 5])
def test_error_against_exact_mode_matches_oracle(lib, N):
    """FP32 state with the tensor-core (TF32x3) tets and FP32 SIMT kernels elsewhere: the L2
    error against the exact standing mode after LSRK steps to t = 0.02 equals the FP64 oracle's
    (the discretisation error dominates; rounding stays far below it)."""
    from oracle.dg import standing_mode
    m = small_hybrid_mesh()
    o = DGOracle(m, N)
    q0 = o.project(standing_mode, 0.0)
    g = lib.Mesh(m, N)
    T = 0.02 if N <= 4 else 0.01        # fewer oracle steps at N = 5
    n = int(np.ceil(T / g.timestep()))
    dt = T / n
    g.set_state(q0.astype(np.float32), on_device=False)
    g.step(n, dt)
    got = g.get_state(np.zeros(q0.shape, np.float32), on_device=False).astype(np.float64)
    q = q0.copy()
    for _ in range(n):
        q = o.lsrk_step(q, dt)
    e_gpu, e_orc = o.l2_error(got, standing_mode, T), o.l2_error(q, standing_mode, T)
    assert abs(e_gpu - e_orc) <= 0.01 * e_orc + 1e-6, (e_gpu, e_orc)


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_sem_rhs_matches_oracle(lib, N):
    """SEM hexahedra (GLL nodes, GLL points on every quadrilateral face, also those of wedges and
    pyramids): rhs against the oracle with the same rules."""
    for name in ("hybrid", "cjump"):
        m = MESHES[name]()
        o = DGOracle(m, N, hex_basis="gll")
        q32 = random_state(o.ndof, 13).astype(np.float32)
        got, _ = gpu_rhs(lib, m, N, q32, hex_basis=1)
        want = o.rhs(q32.astype(np.float64))
        errs = per_type_rel(o, got, want)
        assert rel(got, want) < TOL and max(errs) < TOL, (name, errs)


@pytest.mark.parametrize("N", [3, 4])
def test_sem_steps_match_oracle(lib, N):
    """SEM: ten LSRK(5,4) steps, and the multi-rate start-up + 3 coarse steps, against the oracle
    (N = 4: TMA-staged hex stage and fused multi-rate kernels with the GLL tables)."""
    from oracle.constants import trace_constant
    from oracle.dg import MRAB3, mr_levels, standing_mode
    m = MESHES["cjump"]()
    o = DGOracle(m, N, hex_basis="gll")
    q0 = o.project(standing_mode, 0.0).astype(np.float32)
    g = lib.Mesh(m, N, hex_basis=1)
    dt = g.timestep()
    g.set_state(q0, on_device=False)
    g.step(10, dt)
    got = g.get_state(np.zeros_like(q0), on_device=False).astype(np.float64)
    q = q0.astype(np.float64)
    for _ in range(10):
        q = o.lsrk_step(q, dt)
    assert rel(got, q) < TOL, per_type_rel(o, got, q)
    lev, dmin = mr_levels(o, [trace_constant(t, N, lobatto=True) for t in range(4)], 2)
    gm = lib.Mesh(m, N, nlevels=2, hex_basis=1)
    h = gm.timestep()
    assert abs(h - dmin) < 1e-12 * dmin
    gm.set_state(q0, on_device=False)
    gm.step(3, h)
    got = gm.get_state(np.zeros_like(q0), on_device=False).astype(np.float64)
    mr = MRAB3(o, lev)
    q, hist = mr.start(q0.astype(np.float64), h)
    for _ in range(3):
        q, hist = mr.step(q, hist, h)
    assert rel(got, q) < TOL, per_type_rel(o, got, q)


def bench_slab(ncol=4):
    """The elements of the 64x64x80 throughput mesh (layers H34 W2 H36 T K4 U H2, c = 1.0 / 1.5 by
    layer parity, seed 0) whose cells lie in the first ncol x ncol columns: the same element shapes,
    wave speeds and time-step levels as the timed workload; the cut faces become walls."""
    from paper_1507_02557_b300.inputs import HybridMesh, scale_mesh
    full = scale_mesh()
    lim = -1.0 + ncol * 2.0 / 64
    keep, conn = [], []
    for t in range(4):
        cen = full.xyz[full.conn[t]].mean(axis=1)
        k = (cen[:, 0] < lim) & (cen[:, 1] < lim)
        keep.append(k)
        conn.append(full.conn[t][k])
    used = np.unique(np.concatenate([c.ravel() for c in conn]))
    remap = np.full(len(full.xyz), -1, np.int64)
    remap[used] = np.arange(len(used))
    return HybridMesh(xyz=full.xyz[used], conn=[remap[c].astype(np.int32) for c in conn],
                      c2=[full.c2[t][keep[t]] for t in range(4)],
                      layer=[full.layer[t][keep[t]] for t in range(4)], layers=full.layers)


def test_multirate_on_the_throughput_workload_slab(lib):
    """The configuration the throughput benchmark times (N = 4, two levels, fused coarse / fine
    kernels, TMA-staged hexahedra, tensor-core tets, element types on their own streams) on a
    4x4-column slab of its mesh: start-up + 3 coarse MRAB3 steps against the oracle, overall and
    per element type (Sec. 2.4 reading)."""
    from oracle.constants import trace_constant
    from oracle.dg import MRAB3, mr_levels
    m, N = bench_slab(), 4
    o = DGOracle(m, N)
    lev, dmin = mr_levels(o, [trace_constant(t, N) for t in range(4)], 2)
    g = lib.Mesh(m, N, nlevels=2)
    assert g.level_type_counts(2) == [int(np.sum(l == 2)) for l in lev]
    fine = g.level_type_counts(2)
    assert fine[2] > 0 and fine[3] > 0          # fine pyramids and tets, as at scale
    h = g.timestep()
    assert abs(h - dmin) < 1e-12 * dmin
    q0 = random_state(o.ndof, 21).astype(np.float32)
    g.set_state(q0, on_device=False)
    g.step(3, h)
    got = g.get_state(np.zeros_like(q0), on_device=False).astype(np.float64)
    mr = MRAB3(o, lev)
    q, hist = mr.start(q0.astype(np.float64), h)
    for _ in range(3):
        q, hist = mr.step(q, hist, h)
    errs = per_type_rel(o, got, q)
    assert rel(got, q) < TOL and max(errs) < TOL, errs


@pytest.mark.parametrize("N", [2, 4, 5])
def test_multirate_lsrk_matches_oracle(lib, N):
    """Two-level multi-rate LSRK(5,4) (integrator 1): 3 coarse steps against the oracle's scheme on
    the c-jump mesh (fine pyramids, tets and wedges next to coarse hexahedra)."""
    from oracle.constants import trace_constant
    from oracle.dg import MRLSRK, mr_levels, standing_mode
    m = MESHES["cjump"]()
    o = DGOracle(m, N)
    lev, dmin = mr_levels(o, [trace_constant(t, N) for t in range(4)], 2)
    g = lib.Mesh(m, N, nlevels=2, integrator=1)
    h = g.timestep()
    q0 = o.project(standing_mode, 0.0).astype(np.float32)
    g.set_state(q0, on_device=False)
    t = g.step(3, h)
    got = g.get_state(np.zeros_like(q0), on_device=False).astype(np.float64)
    mr = MRLSRK(o, lev)
    q = q0.astype(np.float64)
    for _ in range(3):
        q = mr.step(q, h)
    assert abs(t - 6 * h) < 1e-12
    assert rel(got, q) < TOL, per_type_rel(o, got, q)


def test_multirate_lsrk_on_the_throughput_workload_slab(lib):
    """Multi-rate LSRK on the 4x4-column slab of the throughput mesh at N = 4 (default kernel
    choices: TMA hexahedra, tensor-core tets, type streams): 2 coarse steps against the oracle."""
    from oracle.constants import trace_constant
    from oracle.dg import MRLSRK, mr_levels
    m, N = bench_slab(), 4
    o = DGOracle(m, N)
    lev, _ = mr_levels(o, [trace_constant(t, N) for t in range(4)], 2)
    g = lib.Mesh(m, N, nlevels=2, integrator=1)
    h = g.timestep()
    q0 = random_state(o.ndof, 23).astype(np.float32)
    g.set_state(q0, on_device=False)
    g.step(2, h)
    got = g.get_state(np.zeros_like(q0), on_device=False).astype(np.float64)
    mr = MRLSRK(o, lev)
    q = q0.astype(np.float64)
    for _ in range(2):
        q = mr.step(q, h)
    errs = per_type_rel(o, got, q)
    assert rel(got, q) < TOL and max(errs) < TOL, errs
