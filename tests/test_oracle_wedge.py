"""Pins of the oracle's LSC-DG wedge (Sec. 2.1.3, Alg. wedge_vol1/2) on warped wedges (CPU only).

The LSC test and trial functions are phi_i / sqrt(J).  Their physical gradients carry the term
-phi_i grad_x J / (2 J^{3/2}); the energy identity cancels it by construction and affine meshes
have grad J = 0, so these tests pin it on warped (non-affine) wedges by routes that do not use the
oracle's analytic derivatives:

* ``Wedge.jac_grad`` against central differences of det(dx/drst) of the vertex map;
* the assembled volume terms against their definitions, with every derivative of phi_i / sqrt(J)
  taken by central differences of basis values in reference coordinates;
* the L2 convergence rate to the standing mode on wedge-only meshes deformed by a smooth map
  (the LSC experiment of Sec. 4.1), which drops below N + 1/2 without the term.
"""
import dataclasses

import numpy as np
import pytest

from oracle.constants import trace_constant
from oracle.dg import DGOracle, standing_mode
from oracle.elements import Wedge
from paper_1507_02557_b300.inputs import layered_mesh, random_state


def warped_wedge(rng, amp=0.25):
    """Reference wedge vertices moved by up to amp per coordinate (J stays positive)."""
    return Wedge.verts + amp * rng.uniform(-1.0, 1.0, size=(6, 3))


def reference_points(rng, n):
    """Random points inside the reference wedge {r, t >= -1, r + t <= 0, |s| <= 1}."""
    r = rng.uniform(-1.0, 1.0, size=(n, 2))
    r = np.where((r[:, 0] + r[:, 1] > 0)[:, None], -r, r)
    return np.stack([r[:, 0], rng.uniform(-1.0, 1.0, n), r[:, 1]], axis=1) * 0.95


def test_wedge_jacobian_gradient_matches_finite_differences():
    rng = np.random.default_rng(11)
    eps = 1e-6
    for _ in range(5):
        xv = warped_wedge(rng)
        P = reference_points(rng, 40)
        g = Wedge.jac_grad(xv, P)
        fd = np.zeros_like(g)
        for d in range(3):
            step = np.zeros(3)
            step[d] = eps
            Jp = np.linalg.det(Wedge.vmap(xv, P + step)[1])
            Jm = np.linalg.det(Wedge.vmap(xv, P - step)[1])
            fd[:, d] = (Jp - Jm) / (2 * eps)
        assert np.all(np.linalg.det(Wedge.vmap(xv, P)[1]) > 0)
        assert np.abs(fd).max() > 1e-2            # the wedge is genuinely warped
        assert np.abs(g - fd).max() < 1e-8 * np.abs(fd).max()


def _lsc_gradients(el, xv, P, eps=1e-6):
    """Physical gradients of psi_i = phi_i / sqrt(J) at points P by central differences of basis
    values in reference coordinates: (nq, 3, Np); also psi (nq, Np) and J (nq,)."""
    def psi(rst):
        J = np.linalg.det(el.vmap(xv, rst)[1])
        return el.basis(rst) / np.sqrt(J)[:, None]
    dref = np.zeros((len(P), 3, el.Np))
    for a in range(3):
        step = np.zeros(3)
        step[a] = eps
        dref[:, a] = (psi(P + step) - psi(P - step)) / (2 * eps)
    F = el.vmap(xv, P)[1]
    G = np.linalg.inv(F)                                  # G[q, a, d] = d r_a / d x_d
    grad = np.einsum("qad,qai->qdi", G, dref)
    return grad, psi(P), np.linalg.det(F)


@pytest.mark.parametrize("N", [1, 2, 3])
def test_wedge_volume_terms_match_their_definition(N):
    """Volume terms of the LSC wedge, written from their definitions with the wedge cubature
    (M = I for the orthonormal LSC basis):
        p-equation:  int u_h . grad psi_i dx,
        u-equation: -c^2 int psi_i grad p_h dx,
    with u_h = sum_j u_j psi_j, p_h = sum_j p_j psi_j."""
    m = layered_mesh(2, 2, 2, "WW", seed=4, amp=0.3, c_of_layer=lambda k: 1.0 + 0.5 * k)
    o = DGOracle(m, N)
    q = random_state(o.ndof, 5)
    got = o.split(o.volume(q))[1]
    qw = o.split(q)[1]
    el = o.els[1]
    P, W = el.cubature()
    warped = 0.0
    for e in range(m.nelem[1]):
        xv = m.xyz[m.conn[1][e]]
        grad, psi, J = _lsc_gradients(el, xv, P)
        warped = max(warped, J.max() / J.min() - 1)
        wJ = W * J
        uh = np.einsum("qi,di->qd", psi, qw[1:, e])            # (nq, 3)
        gp = np.einsum("qdi,i->qd", grad, qw[0, e])            # (nq, 3)
        want_p = np.einsum("q,qd,qdi->i", wJ, uh, grad)
        want_u = -m.c2[1][e] * np.einsum("q,qi,qd->di", wJ, psi, gp)
        scale = np.abs(want_p).max() + np.abs(want_u).max()
        assert np.abs(got[0, e] - want_p).max() < 1e-7 * scale
        assert np.abs(got[1:, e] - want_u).max() < 1e-7 * scale
    assert warped > 0.2                                     # J varies inside the wedges


def smooth_map(x, A=0.15):
    """A fixed smooth deformation of [-1,1]^3 that leaves its boundary in place."""
    b = (1 - x[:, 0] ** 2) * (1 - x[:, 1] ** 2) * (1 - x[:, 2] ** 2)
    d = np.stack([np.sin(np.pi * x[:, 1]) + 0.5, np.cos(np.pi * x[:, 2]) - 0.3,
                  np.sin(np.pi * x[:, 0] + 1.0)], axis=1)
    return x + A * b[:, None] * d


@pytest.mark.parametrize("N", [1, 2])
def test_lsc_wedge_converges_on_warped_meshes(N):
    """Sec. 4.1: the LSC-DG wedge keeps the optimal rate on non-affine wedges.  Wedge-only meshes
    of 2, 4, 8 cells per side whose vertices are moved by one fixed smooth map of the cube (the
    wedges stay vertex-mapped, so their quad faces are bilinear and J varies inside them);
    standing mode to t = 0.05 by LSRK(5,4) at the Eq. (dtK) step.  Rate >= N + 1/2 over both
    refinements.  Without the grad J / (2J) terms of the LSC gradients the N = 2 rate of the last
    refinement falls below 1."""
    errs = []
    for n in (2, 4, 8):
        m = layered_mesh(n, n, n, "W" * n, seed=2, amp=0.0)
        m = dataclasses.replace(m, xyz=smooth_map(m.xyz))
        o = DGOracle(m, N)
        CT = [trace_constant(t, N) for t in range(4)]
        T = 0.05
        nst = int(np.ceil(T / o.global_dt(CT)))
        q = o.project(standing_mode, 0.0)
        for _ in range(nst):
            q = o.lsrk_step(q, T / nst)
        errs.append(o.l2_error(q, standing_mode, T))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > N + 0.5), (errs, rates)
