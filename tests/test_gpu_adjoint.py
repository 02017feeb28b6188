"""dg_adjoint_step (discrete adjoint of LSRK(5,4) steps) against the FP64 oracle.

* dL/dq_0 and dL/dc^2 after 3 steps on a hybrid mesh with wave-speed jumps, against the oracle's
  reverse sweep (dense transpose at N = 1, 2; the pinned similarity form at N = 3, 4, where the
  hexahedra run the TMA kernel and the tets the tensor-core kernel): relative L2 <= 1e-5 for
  dL/dq_0, <= 1e-4 of the largest entry for dL/dc^2 (a sum of products of FP32 traces).
* The dot-product identity of the CUDA path alone on a larger mesh: lambda . q_n (dg_step) equals
  dL/dq_0 . q_0 (dg_adjoint_step) to FP32 rounding.
* Formulations the transpose identity does not cover are refused.
"""
import numpy as np
import pytest

from oracle.adjoint import adjoint_steps
from oracle.dg import DGOracle
from paper_1507_02557_b300.inputs import layered_mesh, random_state

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1507_02557_b300 import dg
    return dg


def tiny():
    return layered_mesh(2, 2, 5, "HWHTK", seed=4, c_of_layer=lambda k: [1.0, 1.6, 0.8, 1.3, 1.1][k])


@pytest.mark.parametrize("N", [1, 2, 3, 4, 6])
def test_adjoint_matches_oracle(lib, N):
    """N = 6: the hexahedra run the column kernel (several warps per element)."""
    m = tiny()
    o = DGOracle(m, N)
    g = lib.Mesh(m, N)
    dt = g.timestep()
    q0 = random_state(o.ndof, 1).astype(np.float32)
    lam = random_state(o.ndof, 2).astype(np.float32)
    steps = 3
    l0_o, g_o = adjoint_steps(o, q0.astype(np.float64), lam.astype(np.float64), dt, steps,
                              Rm=None if N <= 2 else "similarity")
    g_o = np.concatenate(g_o)
    g.set_state(q0, on_device=False)
    lam_d = torch.from_numpy(lam).cuda()
    grad = torch.zeros(sum(m.nelem), dtype=torch.float64, device="cuda")
    g.adjoint_step(steps, lam_d, grad, dt)
    torch.cuda.synchronize()
    l0 = lam_d.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(l0 - l0_o) < 1e-5 * np.linalg.norm(l0_o)
    gg = grad.cpu().numpy()
    assert np.abs(gg - g_o).max() < 1e-4 * np.abs(g_o).max(), float(np.abs(gg - g_o).max() / np.abs(g_o).max())
    # the state is left at the checkpoint
    back = g.get_state(np.zeros_like(q0), on_device=False)
    assert np.array_equal(back, q0)


def test_adjoint_dot_product_on_the_gpu(lib):
    m = layered_mesh(4, 3, 6, "HHWHTK", seed=5, c_of_layer=lambda k: 1.0 + 0.3 * (k % 2))
    N = 4
    g = lib.Mesh(m, N)
    q0 = random_state(g.ndof, 3).astype(np.float32)
    lam = random_state(g.ndof, 4).astype(np.float32)
    g.set_state(q0, on_device=False)
    g.step(5)
    qn = g.get_state(np.zeros_like(q0), on_device=False).astype(np.float64)
    g.set_state(q0, on_device=False)
    lam_d = torch.from_numpy(lam).cuda()
    g.adjoint_step(5, lam_d)
    l0 = lam_d.cpu().numpy().astype(np.float64)
    lhs, rhs = float(np.sum(lam * qn)), float(np.sum(l0 * q0))
    scale = np.linalg.norm(lam) * np.linalg.norm(qn)
    assert abs(lhs - rhs) < 1e-5 * scale, (lhs, rhs, scale)


def test_adjoint_refuses_uncovered_formulations(lib):
    m = tiny()
    for kw in ({"nlevels": 2}, {"hex_basis": 1}, {"pyr_form": 1}):
        g = lib.Mesh(m, 2, **kw)
        lam = torch.zeros((4, g.ndof), dtype=torch.float32, device="cuda")
        with pytest.raises(lib.DGError, match="not supported"):
            g.adjoint_step(1, lam)


def test_autograd_checkpointed_windows(lib):
    """torch.autograd through Propagate (checkpoints every 7 of 20 steps) against one
    dg_adjoint_step over the 20 steps (dL/dq_0 bit for bit: it does not depend on the states);
    dL/dq_0 against central differences of the forward."""
    from paper_1507_02557_b300.autograd import propagate
    m = tiny()
    N = 3
    g = lib.Mesh(m, N)
    q0 = torch.from_numpy(random_state(g.ndof, 5).astype(np.float32)).cuda()
    w = torch.from_numpy(random_state(g.ndof, 6).astype(np.float32)).cuda()
    c2 = torch.zeros(sum(m.nelem), dtype=torch.float64, device="cuda", requires_grad=True)
    qa = q0.clone().requires_grad_(True)
    loss = (propagate(g, qa, c2, 20, every=7) * w).sum()
    loss.backward()
    lam = w.clone()
    grad = torch.zeros(sum(m.nelem), dtype=torch.float64, device="cuda")
    g.set_state(q0, on_device=True)
    g.adjoint_step(20, lam, grad)
    torch.cuda.synchronize()
    assert torch.equal(qa.grad, lam)
    # the stage states of the two runs agree to FP32 rounding: the windows restart from dg_step's
    # states, whose traces between steps come from the fused stage kernels (one trace launch per
    # window instead of per step)
    assert float((c2.grad - grad).abs().max()) <= 1e-6 * float(grad.abs().max())
    # the loss is linear in q0: a central difference along a random direction is exact up to FP32
    d = torch.from_numpy(random_state(g.ndof, 7).astype(np.float32)).cuda()

    def L(q):
        g.set_state(q, on_device=True)
        g.step(20)
        out = torch.empty_like(q)
        g.get_state(out, on_device=True)
        return float((out.double() * w.double()).sum())

    fd = (L(q0 + 0.5 * d) - L(q0 - 0.5 * d)) / 1.0
    ad = float((lam.double() * d.double()).sum())
    assert abs(fd - ad) < 1e-5 * float(lam.norm()) * float(d.norm()), (fd, ad)
