"""Full-size checks on the 64x64x80-cell, N = 4 throughput mesh in the launch configuration the
bench times (TMA-staged hex kernels, tensor-core tets, fused multi-rate schedule).  The oracle
cannot run this mesh, so these are properties that hold at any size:

* a linear pressure field (nodal in the hexahedra, zero elsewhere) with u = 0 has
  rhs_u = -c^2 grad p and rhs_p = 0 at every hexahedron away from the walls and from the
  non-hex layers (there the traces from both sides agree, so every flux term vanishes);
* the upwind scheme does not increase the discrete energy (multi-rate steps);
* multi-rate and single-rate runs of a smooth pulse agree at equal times: both are high-order
  consistent and the steps are ~3e-5, so they differ by rounding only.
"""
import numpy as np
import pytest

from paper_1507_02557_b300.inputs import HEX, scale_layers, scale_mesh

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
N = 4


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1507_02557_b300 import dg
    return dg, scale_mesh(64, 64)


def hex_nodes(m):
    """Physical coordinates of the GL nodes of every hexahedron, (K, 125, 3) float64 on the GPU;
    node index i + 5 (j + 5 k) at (r_i, s_j, t_k), trilinear vertex map (vertex a + 2b + 4c at
    r = +-1 (a), s = +-1 (b), t = +-1 (c))."""
    x, _ = np.polynomial.legendre.leggauss(N + 1)
    n = np.arange((N + 1) ** 3)
    rst = np.stack([x[n % (N + 1)], x[(n // (N + 1)) % (N + 1)], x[n // (N + 1) ** 2]], 1)
    corner = np.array([[(-1) ** (1 + (v & 1)), (-1) ** (1 + ((v >> 1) & 1)), (-1) ** (1 + ((v >> 2) & 1))]
                       for v in range(8)], float)
    shape = np.prod(1 + rst[:, None, :] * corner[None, :, :], axis=2) / 8          # (125, 8)
    dev = torch.device("cuda")
    xv = torch.from_numpy(m.xyz[m.conn[HEX]]).to(dev)                              # (K, 8, 3)
    return torch.einsum("nv,kvd->knd", torch.from_numpy(shape).to(dev), xv)


def test_full_size_linear_pressure_rhs(ctx):
    dg, m = ctx
    g = dg.Mesh(m, N)
    K = m.nelem[HEX]
    X = hex_nodes(m)
    a = torch.tensor([0.3, -0.2, 0.5], dtype=torch.float64, device="cuda")
    q = torch.zeros(4, g.ndof, dtype=torch.float32, device="cuda")
    off, Kh, npn = g.layout(HEX)
    assert (off, Kh, npn) == (0, K, (N + 1) ** 3)
    q[0, :K * npn] = (X @ a).reshape(-1).float()
    r = torch.zeros_like(q)
    g.rhs(q, r)
    torch.cuda.synchronize()
    # hexahedra with no wall face and whose layer and both neighbouring layers are hex layers
    L = scale_layers()
    lay = m.layer[HEX]
    okl = np.array([all(0 <= k + d < len(L) and L[k + d] == "H" for d in (-1, 0, 1)) for k in range(len(L))])
    xv = m.xyz[m.conn[HEX]]
    inner = np.all(np.abs(xv) < 1 - 1e-9, axis=(1, 2)) & okl[lay]
    assert inner.sum() > 0.8 * K
    sel = torch.from_numpy(np.nonzero(inner)[0]).cuda()
    c2 = torch.from_numpy(m.c2[HEX]).cuda()[sel][:, None]
    rp = r[0, :K * npn].reshape(K, npn)[sel].double()
    scale = float((c2 * a.abs().max()).max())
    assert float(rp.abs().max()) < 2e-3 * scale
    for d in range(3):
        rd = r[1 + d, :K * npn].reshape(K, npn)[sel].double()
        err = float((rd + c2 * a[d]).abs().max())
        assert err < 2e-3 * scale, (d, err, scale)


def pulse_state(g, m):
    """p = exp(-|x - x0|^2 / 0.12^2) at the hexahedra's nodes, centred in the lower hex block
    (x0 = (0, 0, -0.6)); it is below 1e-6 at the wedge layers and the walls; zero elsewhere."""
    X = hex_nodes(m)
    x0 = torch.tensor([0.0, 0.0, -0.6], dtype=torch.float64, device="cuda")
    q = torch.zeros(4, g.ndof, dtype=torch.float32, device="cuda")
    K, npn = m.nelem[HEX], (N + 1) ** 3
    q[0, :K * npn] = torch.exp(-((X - x0) ** 2).sum(-1) / 0.12 ** 2).reshape(-1).float()
    return q


def test_full_size_energy_and_multirate_vs_single_rate(ctx):
    dg, m = ctx
    gm = dg.Mesh(m, N, nlevels=2)
    q0 = pulse_state(gm, m)
    h = gm.timestep()
    gm.set_state(q0, on_device=True)
    E = [gm.energy()]
    for _ in range(2):
        gm.step(2, h)                      # first call: start-up (4 LSRK steps of h) + 2 coarse steps
        E.append(gm.energy())
    assert all(np.isfinite(E)) and E[0] > 0
    assert all(b <= a_ * (1 + 1e-6) for a_, b in zip(E, E[1:])), E
    qm = torch.empty_like(q0)
    gm.get_state(qm, on_device=True)
    del gm
    torch.cuda.synchronize()
    gs = dg.Mesh(m, N)
    assert abs(gs.timestep() - h) < 1e-12 * h
    gs.set_state(q0, on_device=True)
    gs.step(4 + 2 * 2 * 2, h)              # t = 4h + 4 coarse steps of 2h
    qs = torch.empty_like(q0)
    gs.get_state(qs, on_device=True)
    torch.cuda.synchronize()
    rel = float(torch.linalg.norm((qm - qs).double()) / torch.linalg.norm(qs.double()))
    assert rel < 1e-4, rel
