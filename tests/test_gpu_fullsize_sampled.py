"""Oracle parity at full size, on sampled elements (the sampling of tests/sampled.py, checked on
the CPU by tests/test_oracle_sampling.py): the CUDA path runs the whole 64x64x80-cell throughput
mesh in the launch configuration the bench times; the FP64 oracle computes the sampled elements
from the sub-mesh of the samples and their neighbours (one ring for an rhs, five for an LSRK(5,4)
step).  Samples: random elements of every type, the first and last element of each type (at the
walls) and elements of each type's lowest and highest layer (next to other types).

* N = 4, the rhs (every type's kernel in its rhs mode);
* N = 4, one LSRK(5,4) step (the stage kernels of the bench's single-rate line): the new state,
  and the step's increment on its own;
* N = 7 with precision 2 (FP16 x 3 tensor-core products of tets, pyramids and the wedges' first
  contraction: the bench's high-order line), the rhs.

Tolerance: relative L2 1e-5 per type over the sampled elements, as the small-mesh parity tests
(FP32 arithmetic against FP64; the measured errors there are 1e-7 - 1e-6).
"""
import numpy as np
import pytest

from oracle.dg import DGOracle
from paper_1507_02557_b300.inputs import scale_mesh
from sampled import dof_index, pick_samples, sample_positions, submesh

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1507_02557_b300 import dg
    return dg, scale_mesh(64, 64)


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def device_state(ndof, seed):
    g = torch.Generator(device="cuda").manual_seed(seed)
    return torch.randn(4, ndof, generator=g, device="cuda", dtype=torch.float32)


def compare(m, N, q_dev, out_dev, samples, rings, oracle_fn):
    """Gather the sub-mesh's state from the device, run the oracle there and compare the sampled
    elements' values with the device result."""
    sub, keep = submesh(m, samples, rings)
    idx = dof_index(m, keep, N)
    it = torch.from_numpy(idx).cuda()
    qs = q_dev[:, it].double().cpu().numpy()
    got_sub = out_dev[:, it].double().cpu().numpy()
    o = DGOracle(sub, N)
    assert o.ndof == idx.size
    want_sub = oracle_fn(o, qs)
    errs = []
    for t, p in enumerate(sample_positions(keep, samples, N)):
        if p.size:
            errs.append(rel(got_sub[:, p], want_sub[:, p]))
    return errs, [len(k) for k in keep]


def test_full_size_rhs_sampled(ctx):
    dg, m = ctx
    N = 4
    g = dg.Mesh(m, N)
    q = device_state(g.ndof, 11)
    r = torch.zeros_like(q)
    g.rhs(q, r)
    torch.cuda.synchronize()
    samples = pick_samples(m, 48, seed=4)
    errs, sizes = compare(m, N, q, r, samples, 1, lambda o, qs: o.rhs(qs))
    assert len(errs) == 4 and max(errs) < TOL, (errs, sizes)


def test_full_size_lsrk_step_sampled(ctx):
    dg, m = ctx
    N = 4
    g = dg.Mesh(m, N)
    q0 = device_state(g.ndof, 12)
    dt = g.timestep()
    g.set_state(q0, on_device=True)
    g.step(1, dt)
    q1 = torch.empty_like(q0)
    g.get_state(q1, on_device=True)
    torch.cuda.synchronize()
    samples = pick_samples(m, 2, seed=5)
    errs, sizes = compare(m, N, q0, q1, samples, 5, lambda o, qs: o.lsrk_step(qs, dt))
    assert len(errs) == 4 and max(errs) < TOL, (errs, sizes)
    # the step's increment q1 - q0 on its own (about 1 % of q at this dt): FP32 storage of q at
    # each of the five stages bounds its relative error near 5 x 2^-24 / 0.01 = 3e-5
    dq = q1 - q0
    errs, sizes = compare(m, N, q0, dq, samples, 5, lambda o, qs: o.lsrk_step(qs, dt) - qs)
    assert len(errs) == 4 and max(errs) < 1e-3, (errs, sizes)


def test_full_size_high_order_precision_rhs_sampled(ctx):
    dg, m = ctx
    N = 7
    g = dg.Mesh(m, N, precision=2)
    q = device_state(g.ndof, 13)
    r = torch.zeros_like(q)
    g.rhs(q, r)
    torch.cuda.synchronize()
    samples = pick_samples(m, 12, seed=6)
    errs, sizes = compare(m, N, q, r, samples, 1, lambda o, qs: o.rhs(qs))
    assert len(errs) == 4 and max(errs) < TOL, (errs, sizes)
