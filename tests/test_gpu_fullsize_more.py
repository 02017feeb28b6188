"""Full-size checks of the bench's other workloads, in the launch configurations it times.  The
oracle cannot run these sizes, so the checks are properties that hold at any size:

* the 64x64x80 mesh at N = 5 and N = 7: a linear pressure field (nodal in the hexahedra, zero
  elsewhere, u = 0) has rhs_u = -c^2 grad p and rhs_p = 0 at every hexahedron away from walls and
  from non-hex layers; at N = 7 the discrete energy does not increase under upwind LSRK steps;
* the many-mesh workload (the 104 meshes with n <= 12): one dg_batch graph gives the per-mesh
  dg_step results bit for bit;
* the differentiation mesh (32x32x40, N = 4) with its point source and receivers: for
  L = w . d (d the receiver samples after each step), the adjoint's dL/dq_0 satisfies
  L(q_0) - L(0) = dL/dq_0 . q_0, and its dL/damp equals (L(amp) - L(0)) / amp (L is affine in
  q_0 and in amp), to FP32 rounding.
"""
import numpy as np
import pytest

from paper_1507_02557_b300.inputs import HEX, batch_mesh, batch_specs, layered_mesh, random_state, scale_layers, scale_mesh

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1507_02557_b300 import dg as lib
    return lib


@pytest.fixture(scope="module")
def mesh64():
    return scale_mesh(64, 64)


def hex_nodes(m, N):
    """Physical coordinates of the GL nodes of every hexahedron, (K, (N+1)^3, 3) float64 on the
    GPU; node i + n1 (j + n1 k) at (r_i, s_j, t_k) of the trilinear vertex map."""
    n1 = N + 1
    x, _ = np.polynomial.legendre.leggauss(n1)
    n = np.arange(n1 ** 3)
    rst = np.stack([x[n % n1], x[(n // n1) % n1], x[n // n1 ** 2]], 1)
    corner = np.array([[(-1) ** (1 + (v & 1)), (-1) ** (1 + ((v >> 1) & 1)), (-1) ** (1 + ((v >> 2) & 1))]
                       for v in range(8)], float)
    shape = np.prod(1 + rst[:, None, :] * corner[None, :, :], axis=2) / 8
    xv = torch.from_numpy(m.xyz[m.conn[HEX]]).cuda()
    return torch.einsum("nv,kvd->knd", torch.from_numpy(shape).cuda(), xv)


@pytest.mark.parametrize("N", [5, 7])
def test_high_order_linear_pressure_rhs(dg, mesh64, N):
    m = mesh64
    g = dg.Mesh(m, N)
    K = m.nelem[HEX]
    off, Kh, npn = g.layout(HEX)
    assert (off, Kh, npn) == (0, K, (N + 1) ** 3)
    a = torch.tensor([0.3, -0.2, 0.5], dtype=torch.float64, device="cuda")
    q = torch.zeros(4, g.ndof, dtype=torch.float32, device="cuda")
    q[0, :K * npn] = (hex_nodes(m, N) @ a).reshape(-1).float()
    r = torch.zeros_like(q)
    g.rhs(q, r)
    torch.cuda.synchronize()
    L = scale_layers()
    okl = np.array([all(0 <= k + d < len(L) and L[k + d] == "H" for d in (-1, 0, 1)) for k in range(len(L))])
    inner = np.all(np.abs(m.xyz[m.conn[HEX]]) < 1 - 1e-9, axis=(1, 2)) & okl[m.layer[HEX]]
    sel = torch.from_numpy(np.nonzero(inner)[0]).cuda()
    c2 = torch.from_numpy(m.c2[HEX]).cuda()[sel][:, None]
    scale = float((c2 * a.abs().max()).max())
    assert float(r[0, :K * npn].reshape(K, npn)[sel].double().abs().max()) < 2e-3 * scale
    for d in range(3):
        rd = r[1 + d, :K * npn].reshape(K, npn)[sel].double()
        assert float((rd + c2 * a[d]).abs().max()) < 2e-3 * scale, d


def test_high_order_energy_nonincreasing(dg, mesh64):
    g = dg.Mesh(mesh64, 7)
    g.set_state((1e-3 * random_state(g.ndof, 3)).astype(np.float32), on_device=False)
    dt = g.timestep()
    E = [g.energy()]
    for _ in range(3):
        g.step(1, dt)
        E.append(g.energy())
    assert all(np.isfinite(E)) and E[0] > 0
    assert all(b <= a * (1 + 1e-6) for a, b in zip(E, E[1:])), E


def test_batch_of_small_meshes_equals_separate_steps(dg):
    specs = [sp for sp in batch_specs() if sp[0] <= 12]
    assert len(specs) > 50
    hm = [batch_mesh(sp) for sp in specs]
    states = [random_state(sum(h.nelem[t] * n for t, n in enumerate(dg_np(sp[1]))), 200 + i).astype(np.float32)
              for i, (h, sp) in enumerate(zip(hm, specs))]
    ref = []
    for h, sp, q0 in zip(hm, specs, states):
        g = dg.Mesh(h, sp[1])
        g.set_state(q0, on_device=False)
        g.step(1)
        g.step(3)
        ref.append(g.get_state(np.zeros_like(q0), on_device=False))
        g.close()
    meshes = []
    for h, sp, q0 in zip(hm, specs, states):
        g = dg.Mesh(h, sp[1])
        g.set_state(q0, on_device=False)
        meshes.append(g)
    b = dg.Batch(meshes)
    b.step(4)
    assert b.stats() == (1, 1)
    for g, want in zip(meshes, ref):
        assert np.array_equal(g.get_state(np.zeros_like(want), on_device=False), want)
    b.close()


def dg_np(N):
    """Nodes per element of order N: hex, wedge, pyramid, tet."""
    return [(N + 1) ** 3, (N + 1) ** 2 * (N + 2) // 2, (N + 1) * (N + 2) * (2 * N + 3) // 6,
            (N + 1) * (N + 2) * (N + 3) // 6]


def test_differentiation_mesh_adjoint_is_exact_for_affine_losses(dg):
    layers = "H" * 17 + "W" + "H" * 19 + "T" + "K" * 2
    m = layered_mesh(32, 32, 40, layers, seed=0)
    g = dg.Mesh(m, 4)
    # receivers near the source, so that the source reaches them within the window
    recs = [[x, y, -0.45] for y in (-0.05, 0.05) for x in (-0.05, 0.0, 0.05)]
    g.set_receivers(recs)
    amp = 1.0
    g.set_source([0.0, 0.0, -0.5], amp, 3.0, 0.0)
    dt = g.timestep()
    n = 20
    w = torch.from_numpy(np.random.default_rng(4).standard_normal((n, len(recs))).astype(np.float32)).cuda()

    def loss(q0, a):
        g.set_source([0.0, 0.0, -0.5], a, 3.0, 0.0)
        g.set_state(q0, on_device=True)
        d = torch.empty((n, len(recs)), dtype=torch.float32, device="cuda")
        t = 0.0
        for k in range(n):
            t = g.step(1, dt, t)
            g.sample_receivers(d[k])
        return float((d.double() * w.double()).sum())

    q0 = torch.from_numpy((1e-2 * random_state(g.ndof, 5)).astype(np.float32)).cuda()
    zero = torch.zeros_like(q0)
    L1, L0 = loss(q0, amp), loss(zero, amp)
    La0 = loss(zero, 0.0)
    g.set_source([0.0, 0.0, -0.5], amp, 3.0, 0.0)
    g.set_state(q0, on_device=True)
    lam = torch.zeros_like(q0)
    ga = torch.zeros(1, dtype=torch.float64, device="cuda")
    g.adjoint_step(n, lam, None, dt, 0.0, w.contiguous(), ga)
    torch.cuda.synchronize()
    lin = float((lam.double() * q0.double()).sum())
    # differences of FP32 forward runs: the rounding of each run is ~1e-7 of |L|
    assert abs((L1 - L0) - lin) < 1e-5 * (abs(L1) + abs(L0)), (L1 - L0, lin)
    assert abs(L0 - La0) > 1e-3 * abs(L0), "the source must reach the receivers"
    assert abs((L0 - La0) / amp - float(ga.item())) < 1e-5 * (abs(L0) + abs(La0)), ((L0 - La0), float(ga.item()))
