"""dg_batch: several meshes stepped through one captured CUDA graph.

* Bit-for-bit equality with the same meshes stepped one by one through dg_step in the
  chunking the batch documents (nsteps mod 3 steps, then chunks of 3), for a mix of N,
  element types, time-step levels, hex node sets (GL and SEM hexahedra of the same N
  in one batch) and precision modes (two N = 7 FP16 x 3 meshes packed together).
* The batched result of one small mesh against the FP64 oracle (relative L2 <= 1e-5).
* Graph reuse: a second call with the same step sizes and history phases replays the
  cached graph; a call that shifts the multi-rate phase causes one new capture.
"""
import numpy as np
import pytest

from oracle.dg import DGOracle, standing_mode
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


# (mesh factory, N, nlevels, hex_basis, precision): N = 2..5, LSRK and multi-rate, fused and
# unfused multi-rate schedules, GL and SEM hexahedra at N = 4 side by side; two N = 7 meshes
# with FP16 x 3 tensor-core products (tets, pyramids, wedges) that the batch packs together
CASES = [
    (lambda: small_hybrid_mesh(), 3, 1, 0, 0),
    (lambda: layered_mesh(3, 3, 5, "HWHTK", seed=3, c_of_layer=lambda k: 1.0 if k % 2 == 0 else 1.5), 4, 2, 0, 0),
    (lambda: layered_mesh(3, 3, 5, "HWHTK", seed=3, c_of_layer=lambda k: 1.0 if k % 2 == 0 else 1.5), 4, 2, 1, 0),
    (lambda: layered_mesh(5, 3, 6, "HHWHTK", seed=5), 2, 1, 0, 0),
    (lambda: layered_mesh(3, 2, 6, "HTKKUH", seed=2), 4, 1, 1, 0),
    (lambda: layered_mesh(3, 3, 5, "HWHTK", seed=3, c_of_layer=lambda k: 1.0 if k % 2 == 0 else 1.5), 5, 2, 0, 0),
    (lambda: small_hybrid_mesh(), 7, 1, 0, 2),
    (lambda: layered_mesh(3, 3, 5, "HWHTK", seed=4), 7, 1, 0, 2),
]


def make(lib, i):
    fac, N, nl, hb, prec = CASES[i]
    m = fac()
    g = lib.Mesh(m, N, nlevels=nl, hex_basis=hb, precision=prec)
    q0 = random_state(g.ndof, 40 + i).astype(np.float32)
    g.set_state(q0, on_device=False)
    return g, m, q0


def state(g):
    return g.get_state(np.zeros((4, g.ndof), np.float32), on_device=False)


def test_batch_equals_separate_steps_bitwise(lib):
    ref, t_ref = [], []
    for i in range(len(CASES)):
        g, _, _ = make(lib, i)
        t = 0.0
        t = g.step(7 % 3, t=t)
        for _ in range(7 // 3):
            t = g.step(3, t=t)
        t = g.step(3, t=t)                   # second batch call: 3 more steps
        ref.append(state(g))
        t_ref.append(t)
        g.close()
    meshes = [make(lib, i)[0] for i in range(len(CASES))]
    b = lib.Batch(meshes)
    t = b.step(7)
    t = b.step(3, t=t)
    assert b.stats() == (3, 1)               # 2 + 1 replays of one captured graph
    for i, g in enumerate(meshes):
        got = state(g)
        assert np.array_equal(got, ref[i]), (i, float(np.abs(got - ref[i]).max()))
        assert abs(t[i] - t_ref[i]) <= 1e-12 * t_ref[i]
    b.close()


def test_batch_graph_cache_and_phase_change(lib):
    meshes = [make(lib, i)[0] for i in (0, 1)]   # one LSRK mesh, one multi-rate mesh
    b = lib.Batch(meshes)
    b.step(3)
    b.step(6)
    assert b.stats() == (3, 1)
    b.step(1)                                     # multi-rate phase moves by one coarse step
    b.step(3)
    assert b.stats() == (4, 2)
    dts = [g.timestep() * 0.5 for g in meshes]   # other step sizes: another graph
    b.step(3, dt=dts)
    assert b.stats() == (5, 3)
    b.close()


def test_batched_mesh_matches_oracle(lib):
    """The LSRK mesh of a mixed batch after 5 steps against the oracle's 5 LSRK steps."""
    m = small_hybrid_mesh()
    N = 3
    o = DGOracle(m, N)
    q0 = o.project(standing_mode, 0.0).astype(np.float32)
    g = lib.Mesh(m, N)
    g.set_state(q0, on_device=False)
    other = make(lib, 1)[0]
    b = lib.Batch([other, g])
    dt = g.timestep()
    b.step(5, dt=[0.0, dt])
    got = state(g).astype(np.float64)
    q = q0.astype(np.float64)
    for _ in range(5):
        q = o.lsrk_step(q, dt)
    assert float(np.linalg.norm(got - q) / np.linalg.norm(q)) < TOL
    b.close()


def test_batch_rejects_repeated_mesh(lib):
    g = make(lib, 0)[0]
    with pytest.raises(lib.DGError, match="invalid argument"):
        lib.Batch([g, g])


def test_gl_and_sem_meshes_of_one_order_coexist(lib):
    """Hex constants are kept per node set: an SEM mesh created after a GL mesh of the same N
    leaves the GL mesh's right-hand side unchanged."""
    m = small_hybrid_mesh()
    g = lib.Mesh(m, 4)
    q = torch.from_numpy(random_state(g.ndof, 5).astype(np.float32)).cuda()
    r0 = torch.zeros_like(q)
    g.rhs(q, r0)
    s = lib.Mesh(m, 4, hex_basis=1)
    rs = torch.zeros((4, s.ndof), dtype=torch.float32, device="cuda")
    s.rhs(torch.from_numpy(random_state(s.ndof, 6).astype(np.float32)).cuda(), rs)
    r1 = torch.zeros_like(q)
    g.rhs(q, r1)
    torch.cuda.synchronize()
    assert torch.equal(r0, r1)


def test_autotune_choices_all_match_the_oracle(lib):
    """Every combination of the run-time kernel choices (TMA / cp.async hex staging, tensor-core /
    SIMT tets, element types on their own streams or one) gives the oracle's LSRK steps; the
    autotuner leaves the mesh's state as it found it and picks one of them."""
    from oracle.dg import standing_mode
    import itertools
    m = small_hybrid_mesh()
    N = 4
    o = DGOracle(m, N)
    q0 = o.project(standing_mode, 0.0).astype(np.float32)
    g = lib.Mesh(m, N)
    dt = g.timestep()
    q = q0.astype(np.float64)
    for _ in range(3):
        q = o.lsrk_step(q, dt)
    for combo in itertools.product((True, False), repeat=3):
        g.set_choices(*combo)
        g.set_state(q0, on_device=False)
        g.step(3, dt)
        got = g.get_state(np.zeros_like(q0), on_device=False).astype(np.float64)
        assert float(np.linalg.norm(got - q) / np.linalg.norm(q)) < TOL, combo
    g.set_state(q0, on_device=False)
    ch = g.autotune(2)
    assert set(ch) == set(g.CHOICES)
    assert np.array_equal(g.get_state(np.zeros_like(q0), on_device=False), q0)


PACK_CASES = [   # four single-rate N = 3 meshes (one combined mesh, four different dt_min), and
    (lambda: small_hybrid_mesh(), 3, 1, 0),                                  # meshes that stay alone
    (lambda: layered_mesh(3, 3, 5, "HWHTK", seed=3, c_of_layer=lambda k: 1.0 if k % 2 == 0 else 1.5), 3, 1, 0),
    (lambda: layered_mesh(5, 3, 6, "HHWHTK", seed=5), 3, 1, 0),
    (lambda: layered_mesh(3, 2, 6, "HTKKUH", seed=2), 3, 1, 0),
    (lambda: layered_mesh(3, 3, 5, "HWHTK", seed=3, c_of_layer=lambda k: 1.0 if k % 2 == 0 else 1.5), 3, 2, 0),
    (lambda: layered_mesh(5, 3, 6, "HHWHTK", seed=5), 2, 1, 0),
    (lambda: small_hybrid_mesh(), 3, 1, 1),
]


def make_pack(lib, i):
    fac, N, nl, hb = PACK_CASES[i]
    g = lib.Mesh(fac(), N, nlevels=nl, hex_basis=hb)
    g.set_state(random_state(g.ndof, 70 + i).astype(np.float32), on_device=False)
    return g


def test_packed_batch_equals_separate_steps_bitwise(lib):
    """Same-kind single-rate meshes stepped through one combined mesh (each element with its own
    mesh's dt) give bit for bit the results of stepping each mesh alone; so does the unpacked
    schedule, and the batch autotuner leaves every state as it found it."""
    ref = []
    for i in range(len(PACK_CASES)):
        g = make_pack(lib, i)
        g.step(7 % 3)
        for _ in range(7 // 3 + 1):
            g.step(3)
        ref.append(state(g))
        g.close()
    meshes = [make_pack(lib, i) for i in range(len(PACK_CASES))]
    b = lib.Batch(meshes)
    b.step(7)
    b.step(3)
    assert b.stats() == (3, 1)
    for i, g in enumerate(meshes):
        got = state(g)
        assert np.array_equal(got, ref[i]), (i, float(np.abs(got - ref[i]).max()))
    # three more steps packed, and the same three steps unpacked from the same states
    single = [i for i, c in enumerate(PACK_CASES) if c[2] == 1]   # (set_state restarts multi-rate)
    before = [state(g) for g in meshes]
    b.step(3)
    packed = [state(g) for g in meshes]
    for i in single:
        meshes[i].set_state(before[i], on_device=False)
    b.set_packing(0)
    b.step(3)
    for i in single:
        assert np.array_equal(state(meshes[i]), packed[i]), i
    now = [state(g) for g in meshes]
    assert b.autotune(3) in (0, 1)
    for i, g in enumerate(meshes):
        assert np.array_equal(state(g), now[i]), i
    b.close()
