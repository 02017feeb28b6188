"""Oracle pins of the discrete adjoint (oracle/adjoint.py), CPU only.

* R^T = W F R F W^{-1} on the dense matrices (upwind and central flux): the structure the CUDA
  adjoint relies on.
* Dot-product identity of the reverse sweep: lambda . S(q0) = (S^T lambda) . q0 for the map S of
  two LSRK(5,4) steps (linear in q0), so the sweep is the transpose of the forward stages.
* dL/dc^2 of the reverse sweep (explicit 1/rho term + penalty terms through tau_p = 1/{rho c},
  walls included) against central differences of the forward map in FP64, on elements of every
  type, on walls and at wave-speed jumps.
"""
import numpy as np
import pytest

from oracle.adjoint import adjoint_steps, dense_rhs, forward, grad_c2_fd, similarity_defect
from oracle.dg import DGOracle
from paper_1507_02557_b300.inputs import layered_mesh, random_state


def mesh():
    return layered_mesh(2, 2, 5, "HWHTK", seed=4, c_of_layer=lambda k: [1.0, 1.6, 0.8, 1.3, 1.1][k])


@pytest.mark.parametrize("tau_scale", [1.0, 0.0])
def test_transpose_is_similar_to_the_operator(tau_scale):
    o = DGOracle(mesh(), 1, tau_scale=tau_scale)
    assert similarity_defect(o) < 1e-13


def test_transpose_similarity_fails_without_the_velocity_flip():
    """A plausible slip (dropping F) is caught: R^T differs from W R W^{-1} at O(1)."""
    from oracle.adjoint import apply_w, apply_winv
    o = DGOracle(mesh(), 1)
    Rm = dense_rhs(o)
    x = random_state(o.ndof, 3)
    wrong = apply_w(o, o.rhs(apply_winv(o, x)))
    right = (Rm.T @ x.ravel()).reshape(4, o.ndof)
    assert np.abs(wrong - right).max() > 0.1 * np.abs(right).max()


@pytest.mark.parametrize("N", [1, 2])
def test_adjoint_sweep_and_c2_gradient(N):
    m = mesh()
    o = DGOracle(m, N)
    dt = 0.015
    q0, lam = random_state(o.ndof, 1), random_state(o.ndof, 2)
    l0, g = adjoint_steps(o, q0, lam, dt, 2)
    lhs = float(np.sum(lam * forward(o, q0, dt, 2)))
    assert abs(lhs - float(np.sum(l0 * q0))) < 1e-12 * abs(lhs)
    # a wall hexahedron, an interior hexahedron, a wedge, a pyramid and tets (both layers)
    elems = [(0, 0), (0, 5), (1, 3), (2, 7), (3, 0), (3, 20)]
    fd = grad_c2_fd(m, N, q0, lam, dt, 2, elems)
    ad = np.array([g[t][e] for t, e in elems])
    assert np.abs(ad - fd).max() < 1e-8 * np.abs(fd).max(), (ad, fd)
