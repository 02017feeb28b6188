"""The sampling behind the full-size oracle checks (tests/sampled.py), on meshes the oracle runs
whole: the rhs at sampled elements from the sub-mesh of the samples and their face neighbours
equals the whole mesh's rhs there, and one LSRK step equals it with five rings of neighbours.
Controls: without the neighbours (rhs), or with one ring too few (LSRK step), the sampled values
differ, so the checks see the coupling they claim to capture."""
import numpy as np
import pytest

from oracle.dg import DGOracle
from paper_1507_02557_b300.inputs import layered_mesh, random_state
from sampled import dof_index, pick_samples, sample_positions, submesh

N = 2


@pytest.fixture(scope="module")
def case():
    # every element type, both transition layers, a wave-speed jump between layers
    m = layered_mesh(5, 4, 9, "HWHTKKUHH", seed=3, c_of_layer=lambda k: 1.0 + 0.5 * (k % 2))
    o = DGOracle(m, N)
    q = random_state(o.ndof, 5)
    return m, o, q


def sampled_values(m, o, q, samples, rings, fn):
    sub, keep = submesh(m, samples, rings)
    os_ = DGOracle(sub, N)
    idx = dof_index(m, keep, N)
    assert idx.size == os_.ndof
    out = fn(os_, q[:, idx])
    return [out[:, p] for p in sample_positions(keep, samples, N)]


def full_values(m, o, samples, full):
    pos = sample_positions([np.arange(k) for k in m.nelem], samples, N)
    return [full[:, p] for p in pos]


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_rhs_from_one_ring(case):
    m, o, q = case
    samples = pick_samples(m, 6, seed=1)
    assert all(len(s) > 0 for s in samples)
    want = full_values(m, o, samples, o.rhs(q))
    got = sampled_values(m, o, q, samples, 1, lambda os_, qs: os_.rhs(qs))
    for t in range(4):
        assert rel(got[t], want[t]) < 1e-12, t
    bare = sampled_values(m, o, q, samples, 0, lambda os_, qs: os_.rhs(qs))
    assert min(rel(bare[t], want[t]) for t in range(4)) > 1e-3


def test_lsrk_step_from_five_rings(case):
    m, o, q = case
    samples = pick_samples(m, 1, seed=2)
    dt = 5e-3   # about the stable step of this mesh at N = 2
    want = full_values(m, o, samples, o.lsrk_step(q, dt))
    got = sampled_values(m, o, q, samples, 5, lambda os_, qs: os_.lsrk_step(qs, dt))
    for t in range(4):
        assert rel(got[t], want[t]) < 1e-12, t
    short = sampled_values(m, o, q, samples, 4, lambda os_, qs: os_.lsrk_step(qs, dt))
    assert max(rel(short[t], want[t]) for t in range(4)) > 1e-9   # measured 3e-8 - 5e-6
