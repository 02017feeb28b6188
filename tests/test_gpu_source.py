"""Point source, receivers and the receiver-misfit gradient on the GPU against the FP64 oracle.

* Receiver traces of LSRK(5,4) steps with a Ricker point source (oracle/sources.py): relative
  to the largest sample <= 1e-5.
* dL/dq_0, dL/dc^2 and dL/damp of L = 1/2 sum (d - d_obs)^2 through dg_adjoint_step with
  receiver forcing, against the oracle's reverse sweep (N = 2, 4).
* The autograd bridge (checkpoint windows) against one adjoint call, and dL/dc^2 along random
  directions against central differences of GPU forward runs (h = 1e-3).
"""
import dataclasses

import numpy as np
import pytest

from oracle.adjoint import adjoint_steps
from oracle.dg import DGOracle
from oracle.sources import PointSources, record
from paper_1507_02557_b300.inputs import layered_mesh, random_state

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
XS = [0.1, -0.2, -0.7]
RECS = [[0.3, 0.2, -0.1], [-0.4, 0.5, 0.05], [0.0, 0.0, -0.15], [0.55, -0.6, 0.1]]
AMP, F0, T0 = 1.3, 3.0, 0.05


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1507_02557_b300 import dg
    return dg


def tiny(c=(1.0, 1.6, 0.8, 1.3, 1.1)):
    return layered_mesh(2, 2, 5, "HWHTK", seed=4, c_of_layer=lambda k: c[k])


def gpu_mesh(lib, m, N):
    g = lib.Mesh(m, N)
    g.set_source(XS, AMP, F0, T0)
    g.set_receivers(RECS)
    return g


def gpu_record(g, q0, dt, n):
    g.set_state(q0, on_device=False)
    out = torch.empty((n, len(RECS)), dtype=torch.float32, device="cuda")
    t = 0.0
    for k in range(n):
        t = g.step(1, dt, t)
        g.sample_receivers(out[k])
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("N", [2, 4, 6])
def test_receiver_traces_match_oracle(lib, N):
    m = tiny()
    o = DGOracle(m, N)
    src = PointSources(o, XS, AMP, F0, T0, RECS)
    g = gpu_mesh(lib, m, N)
    dt = g.timestep()
    q0 = (0.1 * random_state(o.ndof, 1)).astype(np.float32)
    want, _ = record(o, q0.astype(np.float64), dt, 8, src)
    got = gpu_record(g, q0, dt, 8)
    assert np.abs(got - want).max() < 1e-5 * np.abs(want).max()
    # a zero initial state: the traces come from the source alone
    z = np.zeros_like(q0)
    want0, _ = record(o, z.astype(np.float64), dt, 8, src)
    got0 = gpu_record(g, z, dt, 8)
    assert np.abs(want0).max() > 0
    assert np.abs(got0 - want0).max() < 1e-5 * np.abs(want0).max()


@pytest.mark.parametrize("N", [2, 4])
def test_misfit_gradient_matches_oracle(lib, N):
    m = tiny()
    o = DGOracle(m, N)
    src = PointSources(o, XS, AMP, F0, T0, RECS)
    g = gpu_mesh(lib, m, N)
    dt = g.timestep()
    n = 5
    q0 = (0.1 * random_state(o.ndof, 1)).astype(np.float32)
    d = gpu_record(g, q0, dt, n)
    obs = d + 0.05 * np.random.default_rng(3).standard_normal(d.shape)
    resid = (d - obs).astype(np.float32)
    l0_o, gc_o, ga_o = adjoint_steps(o, q0.astype(np.float64), np.zeros((4, o.ndof)), dt, n,
                                     Rm=None if N <= 2 else "similarity", src=src, resid=resid.astype(np.float64))
    gc_o = np.concatenate(gc_o)
    g.set_state(q0, on_device=False)
    lam = torch.zeros((4, g.ndof), dtype=torch.float32, device="cuda")
    gc = torch.zeros(sum(m.nelem), dtype=torch.float64, device="cuda")
    ga = torch.zeros(1, dtype=torch.float64, device="cuda")
    g.adjoint_step(n, lam, gc, dt, 0.0, torch.from_numpy(resid).cuda(), ga)
    torch.cuda.synchronize()
    l0 = lam.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(l0 - l0_o) < 1e-5 * np.linalg.norm(l0_o)
    gc = gc.cpu().numpy()
    assert np.abs(gc - gc_o).max() < 1e-4 * np.abs(gc_o).max()
    assert abs(float(ga.item()) - ga_o) < 1e-4 * abs(ga_o)


def test_seismogram_autograd_and_finite_differences(lib):
    from paper_1507_02557_b300.autograd import seismogram
    m = tiny()
    N = 3
    g = gpu_mesh(lib, m, N)
    dt = g.timestep()
    n = 30
    q0 = torch.zeros((4, g.ndof), dtype=torch.float32, device="cuda")
    nel = sum(m.nelem)
    with torch.no_grad():
        obs = seismogram(g, q0, torch.zeros(nel, dtype=torch.float64, device="cuda"),
                         torch.zeros(1, dtype=torch.float64, device="cuda"), n, dt, 0.0, 7) * 1.05

    def loss_of(mesh_c2=None):
        gg = g if mesh_c2 is None else gpu_mesh(lib, dataclasses.replace(m, c2=mesh_c2), N)
        c2 = torch.zeros(nel, dtype=torch.float64, device="cuda", requires_grad=True)
        amp = torch.zeros(1, dtype=torch.float64, device="cuda", requires_grad=True)
        d = seismogram(gg, q0, c2, amp, n, dt, 0.0, 7)
        L = 0.5 * ((d.double() - obs.double()) ** 2).sum()
        return L, c2, amp

    L, c2, amp = loss_of()
    L.backward()
    # one adjoint call over all steps gives the same gradients
    d = seismogram(g, q0, torch.zeros(nel, dtype=torch.float64, device="cuda"),
                   torch.zeros(1, dtype=torch.float64, device="cuda"), n, dt, 0.0, n)
    lam = torch.zeros_like(q0)
    gc = torch.zeros(nel, dtype=torch.float64, device="cuda")
    ga = torch.zeros(1, dtype=torch.float64, device="cuda")
    g.set_state(q0, on_device=True)
    g.adjoint_step(n, lam, gc, dt, 0.0, (d - obs).contiguous(), ga)
    torch.cuda.synchronize()
    assert float((c2.grad - gc).abs().max()) <= 1e-5 * float(gc.abs().max())
    assert abs(float(amp.grad.item()) - float(ga.item())) <= 1e-5 * abs(float(ga.item()))
    # central differences of GPU forward runs along random c^2 directions (relative step 1e-3)
    rng = np.random.default_rng(11)
    gcd = c2.grad.cpu().numpy()
    for _ in range(3):
        dirs = [rng.standard_normal(k) for k in m.nelem]
        cp = [c * (1 + 1e-3 * dd) for c, dd in zip(m.c2, dirs)]
        cm = [c * (1 - 1e-3 * dd) for c, dd in zip(m.c2, dirs)]
        fd = (float(loss_of(cp)[0].detach()) - float(loss_of(cm)[0].detach())) / 2e-3
        ad = float(np.sum(gcd * np.concatenate([c * dd for c, dd in zip(m.c2, dirs)])))
        assert abs(fd - ad) < 2e-3 * abs(ad) + 1e-6, (fd, ad)
