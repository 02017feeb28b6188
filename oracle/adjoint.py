"""Discrete adjoint of the LSRK(5,4) time stepping of the DG operator (float64, test oracle).

Test infrastructure only: imported by tests/, never by the library.

The paper has no adjoint; what is fixed here is the derivative of its discrete map.  For a
loss L(q_n) of the state after n steps of LSRK(5,4) (Sec. 2.4 time stepping of
dq/dt = R(c^2) q, R = M^{-1} A of Sec. 2.2-2.3), with lambda = dL/dq_n given:

* ``adjoint_steps``   dL/dq_0 and dL/dc^2 (per element) by the reverse sweep of the 2N-storage
  stages (res^{k+1} = a_k res^k + dt R q^k, q^{k+1} = q^k + b_k res^{k+1}):
      rho += b_k lambda;  lambda += dt R^T rho;  g += dt (d(R q^k)/dc^2)^T rho;  rho *= a_k
  for k = 4..0, with R^T the transpose of the dense matrix of R (small meshes only) and the
  c^2 term from ``c2_term`` below;
* ``grad_c2_fd``      the same gradient as central differences of the forward map
  (the definition, for pinning ``c2_term``);
* ``similarity``      the identity R^T = W F R F W^{-1} with W = blockdiag(M, M / c^2) (the
  energy weight of Sec. 3) and F = diag(1, -1, -1, -1): the central part of W R is skew
  (the energy identity of Sec. 3), the upwind penalty part symmetric, and flipping the sign
  of u negates the central part and keeps the penalty.  The CUDA adjoint applies R^T this way.

d(R q)/dc^2_K (c^2 enters through 1/rho = c^2 of the u-equation and through
tau_p = 1/{rho c} = 2 / (1/c^- + 1/c^+), tau_u = 1/tau_p on every face of K):
  rho^T d(Rq)/dc^2_K = sum_{nodes of K} rho_u . (R q)_u / c^2_K
                     + sum_{faces of K} -1/2 tau_scale (d tau_p/dc^2_K I_p + d tau_u/dc^2_K I_u),
  I_p = int_f [q_p][v_p],  I_u = int_f [q.n][v.n],  v = W^{-1} rho,
and on a wall face (mirror state) the p term with [q_p][v_p] replaced by 2 q_p v_p (one side).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from .dg import LSRK_A, LSRK_B, LSRK_C, DGOracle
from .sources import PointSources, lsrk_step_src, record, ricker


def dense_rhs(o: DGOracle):
    """The matrix of q -> o.rhs(q) on the flattened state (4*ndof); small meshes only."""
    n = 4 * o.ndof
    Rm = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        Rm[:, j] = o.rhs(e.reshape(4, o.ndof)).ravel()
    return Rm


def apply_w(o: DGOracle, x):
    """W x: the per-type mass matrices with the material weights (1 for p, 1/c^2 for u)."""
    return o.mass_apply(x) * o.material_weights()


def apply_winv(o: DGOracle, x):
    """W^{-1} x: M^{-1}, times c^2 on the velocity (the oracle's apply_minv)."""
    return o.apply_minv(x)


def flip(x):
    """F x: the velocity negated."""
    y = x.copy()
    y[1:] *= -1.0
    return y


def c2_term(o: DGOracle, q, rho):
    """Per element (type order, element order): rho^T d(R q)/dc^2_K."""
    g = [np.zeros(k) for k in o.K]
    Rq = o.rhs(q)
    Rv, rv = o.split(Rq), o.split(rho)
    for t in range(4):
        if o.K[t]:
            g[t] += np.einsum("fen,fen->e", rv[t][1:], Rv[t][1:]) / o.c2[t]
    v = apply_winv(o, rho)
    tq, tv = o.traces(q), o.traces(v)
    eq, ev = o.neighbour_traces(tq), o.neighbour_traces(tv)
    n = o.s_n
    jq_p, jv_p = eq[:, 0] - tq[:, 0], ev[:, 0] - tv[:, 0]
    jq_n = np.sum((np.moveaxis(eq[:, 1:], 1, 2) - np.moveaxis(tq[:, 1:], 1, 2)) * n, axis=2)
    jv_n = np.sum((np.moveaxis(ev[:, 1:], 1, 2) - np.moveaxis(tv[:, 1:], 1, 2)) * n, axis=2)
    sides = o.geo.sides
    for s, sd in enumerate(sides):
        cK = np.sqrt(o.c2[sd.t][sd.e])
        if sd.nbr >= 0:
            if sd.nbr < s:
                continue                      # each interior face once
            od = sides[sd.nbr]
            cO = np.sqrt(o.c2[od.t][od.e])
            Ip = float(np.sum(o.s_wJ[s] * jq_p[s] * jv_p[s]))
            Iu = float(np.sum(o.s_wJ[s] * jq_n[s] * jv_n[s]))
            sig = 1.0 / cK + 1.0 / cO
            for (t, e, c) in ((sd.t, sd.e, cK), (od.t, od.e, cO)):
                dtp = 1.0 / (sig * sig * c ** 3)          # d tau_p / d c^2 of this side's element
                dtu = -1.0 / (4.0 * c ** 3)               # d (1/tau_p) / d c^2
                g[t][e] += -0.5 * o.tau_scale * (dtp * Ip + dtu * Iu)
        else:
            # wall: tau_p = c_K, mirror p+ = -p-, u+ = u- (no u jump); [q_p][v_p] = 4 q_p v_p
            # seen from the one existing side, whose flux term is tau_p/2 [q_p] against v_p
            Ip = float(np.sum(o.s_wJ[s] * tq[s, 0] * tv[s, 0]))
            g[sd.t][sd.e] += -0.5 * o.tau_scale * (0.5 / cK) * 2.0 * Ip
    return g


def adjoint_steps(o: DGOracle, q0, lam, dt, nsteps, Rm=None, t0=0.0, src: PointSources | None = None,
                  resid=None):
    """(dL/dq_0, dL/dc^2 per type[, dL/damp]) for lambda = dL/dq_n after nsteps LSRK(5,4) steps
    from q0 at time t0.  R^T from the dense matrix Rm (computed when None), or, with
    Rm = "similarity", as W F R F W^{-1} (for meshes too large for the dense matrix; the identity
    is pinned on the dense matrices).  With a source, the steps include it and dL/damp is
    returned as a third value; with receiver residuals resid[n, r] (of the state after step n+1),
    lambda += the receivers' transpose of resid[n] before step n is reversed (the gradient of
    L = 1/2 sum |d - d_obs|^2 when resid = d - d_obs)."""
    shape = (4, o.ndof)
    if isinstance(Rm, str):
        rt = lambda x: apply_w(o, flip(o.rhs(flip(apply_winv(o, x)))))
    else:
        if Rm is None:
            Rm = dense_rhs(o)
        rt = lambda x: (Rm.T @ x.ravel()).reshape(shape)
    states = [q0.copy()]
    for j in range(nsteps - 1):
        states.append(lsrk_step_src(o, states[-1], dt, t0 + j * dt, src))
    lam = lam.copy()
    g = [np.zeros(k) for k in o.K]
    g_amp = 0.0
    for j in range(nsteps - 1, -1, -1):
        if resid is not None:
            lam = lam + src.inject(resid[j])
        tj = t0 + j * dt
        # stage inputs q^0..q^4 of step j
        Q = [states[j].copy()]
        res = np.zeros(shape)
        for k in range(4):
            r = o.rhs(Q[-1]) + (src.field(tj + LSRK_C[k] * dt) if src is not None else 0.0)
            res = LSRK_A[k] * res + dt * r
            Q.append(Q[-1] + LSRK_B[k] * res)
        rho = np.zeros(shape)
        for k in range(4, -1, -1):
            rho = rho + LSRK_B[k] * lam
            lam = lam + dt * rt(rho)
            for t, gt in enumerate(c2_term(o, Q[k], rho)):
                g[t] += dt * gt
            if src is not None:
                g_amp += dt * float(np.sum(rho * src.unit_field(tj + LSRK_C[k] * dt)))
            rho = LSRK_A[k] * rho
    if src is not None:
        return lam, g, g_amp
    return lam, g


def forward(o: DGOracle, q0, dt, nsteps):
    q = q0.copy()
    for _ in range(nsteps):
        q = o.lsrk_step(q, dt)
    return q


def grad_c2_fd(mesh, N, q0, lam, dt, nsteps, elems, h=1e-5, **kw):
    """Central differences of lambda . q_n with respect to c^2 of the listed (type, element)s,
    relative step h."""
    out = []
    for (t, e) in elems:
        vals = []
        for s in (1.0, -1.0):
            c2 = [c.copy() for c in mesh.c2]
            c2[t][e] *= 1.0 + s * h
            m2 = dataclasses.replace(mesh, c2=c2)
            vals.append(float(np.sum(lam * forward(DGOracle(m2, N, **kw), q0, dt, nsteps))))
        out.append((vals[0] - vals[1]) / (2.0 * h * mesh.c2[t][e]))
    return np.array(out)


def similarity_defect(o: DGOracle, Rm=None):
    """max |R^T - W F R F W^{-1}| / max |R| on the dense matrices."""
    if Rm is None:
        Rm = dense_rhs(o)
    n = 4 * o.ndof
    rhs_of = lambda x: (Rm @ x.ravel()).reshape(4, o.ndof)
    T = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        x = e.reshape(4, o.ndof)
        T[:, j] = apply_w(o, flip(rhs_of(flip(apply_winv(o, x))))).ravel()
    return float(np.abs(Rm.T - T).max() / np.abs(Rm).max())


def misfit(mesh, N, q0, dt, nsteps, xs, amp, f0, t0, receivers, obs, **kw):
    """L = 1/2 sum_n sum_r (d[n, r] - obs[n, r])^2 of a forward run (the definition)."""
    o = DGOracle(mesh, N, **kw)
    src = PointSources(o, xs, amp, f0, t0, receivers)
    d, _ = record(o, q0, dt, nsteps, src)
    return 0.5 * float(np.sum((d - obs) ** 2))
