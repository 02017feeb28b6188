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


def test_point_source_and_receivers_are_exact_on_linear_fields():
    """Receivers read a nodal linear field exactly at their points, and the source vector is the
    weak delta: sum_n (M g)_n u_n = u(x_s) for u linear (GL collocation is exact for it)."""
    from oracle.sources import PointSources
    m = mesh()
    o = DGOracle(m, 2)
    xs = [0.1, -0.2, -0.7]
    recs = [[0.3, 0.2, -0.1], [-0.4, 0.5, 0.05], [0.0, 0.0, -0.15]]
    src = PointSources(o, xs, 1.0, 3.0, 0.0, recs)
    a = np.array([0.3, -0.7, 0.45])
    hx = o.els[0]
    X = m.xyz[m.conn[0]]
    q = np.zeros((4, o.ndof))
    for e in range(o.K[0]):
        x, _ = hx.vmap(X[e], hx.nodes)
        q[0, o.off[0] + e * hx.Np:o.off[0] + (e + 1) * hx.Np] = x @ a + 0.2
    assert np.allclose(src.sample(q), np.array(recs) @ a + 0.2, atol=1e-12)
    u = q[0, o.off[0] + src.e_s * hx.Np:o.off[0] + (src.e_s + 1) * hx.Np]
    Mg = src.g * hx.wnodes * o.hex_J[src.e_s]
    assert abs(float(Mg @ u) - (float(np.dot(xs, a)) + 0.2)) < 1e-12


def test_receiver_misfit_gradient_against_finite_differences():
    """L = 1/2 sum (d - d_obs)^2 over 4 steps with a Ricker point source: dL/damp, dL/dc^2 (source
    and receiver hexahedra, a wedge, a pyramid, a tet) and dL/dq_0 along a random direction from
    the reverse sweep with receiver forcing, against FP64 central differences."""
    import dataclasses
    from oracle.adjoint import misfit
    from oracle.sources import PointSources, record
    m = mesh()
    N = 2
    o = DGOracle(m, N)
    xs = [0.1, -0.2, -0.7]
    recs = [[0.3, 0.2, -0.1], [-0.4, 0.5, 0.05], [0.0, 0.0, -0.15]]
    amp, f0, t0 = 1.3, 3.0, 0.05
    src = PointSources(o, xs, amp, f0, t0, recs)
    dt, n = 0.01, 4
    q0 = 0.1 * random_state(o.ndof, 1)
    d, _ = record(o, q0, dt, n, src)
    obs = d + 0.05 * np.random.default_rng(3).standard_normal(d.shape)
    lam0, g, gamp = adjoint_steps(o, q0, np.zeros((4, o.ndof)), dt, n, src=src, resid=d - obs)
    L = lambda mm, a: misfit(mm, N, q0, dt, n, xs, a, f0, t0, recs, obs)
    h = 1e-5
    fd_amp = (L(m, amp * (1 + h)) - L(m, amp * (1 - h))) / (2 * h * amp)
    assert abs(gamp - fd_amp) < 1e-6 * abs(fd_amp)
    elems = [(0, src.e_s), (0, src.e_r[0]), (1, 2), (2, 5), (3, 10)]
    ad, fd = [], []
    for t, e in elems:
        c2p = [c.copy() for c in m.c2]
        c2m = [c.copy() for c in m.c2]
        c2p[t][e] *= 1 + h
        c2m[t][e] *= 1 - h
        fd.append((L(dataclasses.replace(m, c2=c2p), amp) - L(dataclasses.replace(m, c2=c2m), amp))
                  / (2 * h * m.c2[t][e]))
        ad.append(g[t][e])
    assert np.abs(np.array(ad) - fd).max() < 1e-6 * np.abs(fd).max(), (ad, fd)
    dq = random_state(o.ndof, 9)

    def Lq(q):
        dd, _ = record(o, q, dt, n, src)
        return 0.5 * float(np.sum((dd - obs) ** 2))

    fdq = (Lq(q0 + 1e-4 * dq) - Lq(q0 - 1e-4 * dq)) / 2e-4
    assert abs(float(np.sum(lam0 * dq)) - fdq) < 1e-8 * abs(fdq)
