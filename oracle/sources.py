"""Point source and receivers in hexahedra, and LSRK(5,4) steps with the source (float64, test
oracle).  Test infrastructure only: imported by tests/, never by the library.

The paper's acoustic system carries a source f on the pressure equation, (1/kappa) p_t + div u = f
(Sec. 2.2), which its experiments set to zero.  Here f(x, t) = amp ricker(t) delta(x - x_s):
* ricker(t) = (1 - 2 pi^2 f0^2 (t - t0)^2) exp(-pi^2 f0^2 (t - t0)^2);
* the weak form of the delta gives the p-equation rhs term amp ricker(t) g with
  g = M_K^{-1} phi(x_s) in the hexahedron K that contains x_s (GL-collocated mass w_n J_n);
* a receiver reads p(x_r) = sum_n phi_n(x_r) p_n in the hexahedron that contains x_r.
A point on a face shared by two hexahedra belongs to the one of lower index.  Stage k of the step
from t adds the source at t + c_k dt (the LSRK(5,4) stage times).
"""
from __future__ import annotations

import numpy as np

from .dg import LSRK_A, LSRK_B, LSRK_C, DGOracle


def ricker(t, f0, t0):
    a = (np.pi * f0 * (t - t0)) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


def locate_hex(o: DGOracle, x, tol=1e-10):
    """(element, reference point) of the lowest-index hexahedron containing x, or None."""
    hx = o.els[0]
    X = o.mesh.xyz[o.mesh.conn[0]]                     # (K, 8, 3)
    lo, hi = X.min(axis=1) - 1e-9, X.max(axis=1) + 1e-9
    for e in np.nonzero(np.all((x >= lo) & (x <= hi), axis=1))[0]:
        r = np.zeros(3)
        for _ in range(50):                            # Newton on the trilinear map
            xr, F = hx.vmap(X[e], r)
            dr = np.linalg.solve(F[0], x - xr[0])
            r = r + dr
            if np.abs(dr).max() < 1e-14:
                break
        if np.all(np.abs(r) <= 1.0 + tol):
            return int(e), r
    return None


class PointSources:
    """Source vector and receiver rows of one mesh (all points in hexahedra)."""

    def __init__(self, o: DGOracle, xs, amp, f0, t0, receivers):
        self.o = o
        self.amp, self.f0, self.t0 = float(amp), float(f0), float(t0)
        hx = o.els[0]
        loc = locate_hex(o, np.asarray(xs, float))
        if loc is None:
            raise ValueError("source not inside a hexahedron")
        self.e_s = loc[0]
        phi = hx.basis(loc[1])[0]
        self.g = phi / (hx.wnodes * o.hex_J[self.e_s])
        self.e_r, self.rows = [], []
        for x in np.atleast_2d(receivers):
            loc = locate_hex(o, np.asarray(x, float))
            if loc is None:
                raise ValueError("receiver not inside a hexahedron")
            self.e_r.append(loc[0])
            self.rows.append(hx.basis(loc[1])[0])
        self.rows = np.array(self.rows)

    def field(self, t):
        """(4, ndof): the source term amp ricker(t) g on p."""
        f = np.zeros((4, self.o.ndof))
        n = len(self.g)
        f[0, self.o.off[0] + self.e_s * n:self.o.off[0] + (self.e_s + 1) * n] = self.amp * ricker(t, self.f0, self.t0) * self.g
        return f

    def unit_field(self, t):
        """d field / d amp."""
        return self.field(t) / self.amp if self.amp != 0 else self.field(t)

    def sample(self, q):
        """p at the receivers."""
        n = self.rows.shape[1]
        return np.array([self.rows[r] @ q[0, self.o.off[0] + e * n:self.o.off[0] + (e + 1) * n]
                         for r, e in enumerate(self.e_r)])

    def inject(self, resid):
        """(4, ndof): sum_r resid_r d p(x_r)/dq, the transpose of sample."""
        f = np.zeros((4, self.o.ndof))
        n = self.rows.shape[1]
        for r, e in enumerate(self.e_r):
            f[0, self.o.off[0] + e * n:self.o.off[0] + (e + 1) * n] += resid[r] * self.rows[r]
        return f


def lsrk_step_src(o: DGOracle, q, dt, t, src: PointSources | None):
    """One LSRK(5,4) step from time t with the source at the stage times t + c_k dt."""
    q = q.copy()
    res = np.zeros_like(q)
    for a, b, c in zip(LSRK_A, LSRK_B, LSRK_C):
        r = o.rhs(q)
        if src is not None:
            r = r + src.field(t + c * dt)
        res = a * res + dt * r
        q = q + b * res
    return q


def record(o: DGOracle, q0, dt, nsteps, src: PointSources, t0=0.0):
    """Receiver traces d[n, r] after steps n = 1..nsteps, and the final state."""
    q, out = q0.copy(), []
    for n in range(nsteps):
        q = lsrk_step_src(o, q, dt, t0 + n * dt, src)
        out.append(src.sample(q))
    return np.array(out), q
