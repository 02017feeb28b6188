"""Right-hand side, time stepping and energy of the hybrid DG method (float64).

Follows Sec. 2.2 - 2.3 of the paper with kappa = 1, rho = 1/c^2:

* volume terms per element type (Alg. hex_vol, tet_vol, wedge_vol1/2, pyr_vol),
* upwind flux with tau_p = 1/{rho c}, tau_u = {rho c} (Eq. skewform and the
  strong form), free-surface wall p = 0 by the mirror state p+ = -p-, u+ = u-,
* the per-type inverse mass matrices of Sec. 2.1,
* LSRK(5,4) (Carpenter-Kennedy 2N-storage) stages,
* local time steps of Eq. (dtK) and the multi-rate levels of Sec. 2.4.

State layout: ``q[4, ndof]`` with fields (p, u, v, w); DOFs of all hexes, then
wedges, pyramids, tets; within a type, element-major.
"""
from __future__ import annotations

import numpy as np

from .mesh import MeshGeometry

# Carpenter & Kennedy (1994) five-stage fourth-order 2N-storage Runge-Kutta.
LSRK_A = np.array([0.0,
                   -567301805773.0 / 1357537059087.0,
                   -2404267990393.0 / 2016746695238.0,
                   -3550918686646.0 / 2091501179385.0,
                   -1275806237668.0 / 842570457699.0])
LSRK_B = np.array([1432997174477.0 / 9575080441904.0,
                   5161836677717.0 / 13612068292357.0,
                   1720146321549.0 / 2090206949498.0,
                   3134564353537.0 / 4481467310338.0,
                   2277821191437.0 / 14882151754819.0])
LSRK_C = np.array([0.0,
                   1432997174477.0 / 9575080441904.0,
                   2526269341429.0 / 6820363962896.0,
                   2006345519317.0 / 3224310063776.0,
                   2802321613138.0 / 2924317926251.0])


class DGOracle:
    """The discrete operator dq/dt = M^{-1} A q of the paper on a hybrid mesh.

    ``tau_scale`` multiplies both penalties (1 = upwind, 0 = central flux).
    ``pyr_form`` is ``"skew"`` (Alg. pyr_vol, default) or ``"strong"``.
    ``hex_basis`` is ``"gl"`` (default) or ``"gll"``: the SEM hexahedron of Sec. 2.1.1 (nodes
    and collocated mass at the GLL points), with GLL points on every quadrilateral face.
    """

    def __init__(self, mesh, N, tau_scale=1.0, pyr_form="skew", hex_basis="gl"):
        self.mesh = mesh
        self.N = N
        self.tau_scale = float(tau_scale)
        self.pyr_form = pyr_form
        self.hex_basis = hex_basis
        self.geo = MeshGeometry(mesh, N, lobatto=hex_basis == "gll")
        self.els = self.geo.els
        self.K = mesh.nelem
        self.Np = [el.Np for el in self.els]
        self.off = np.concatenate([[0], np.cumsum([k * n for k, n in zip(self.K, self.Np)])]).astype(int)
        self.ndof = int(self.off[-1])
        xyz = mesh.xyz
        self.c2 = mesh.c2
        X = [xyz[mesh.conn[t]] for t in range(4)]       # (K, nv, 3)

        # ---- hexahedron: geometric factors at the GL nodes (Alg. hex_vol)
        hx = self.els[0]
        self.hex_G, self.hex_J = self._factors(hx, X[0], hx.nodes)
        # ---- tetrahedron: constant factors; nodal derivative matrices D^r,D^s,D^t (Sec. 2.3.2)
        tt = self.els[3]
        self.tet_G, self.tet_J = self._factors(tt, X[3], tt.nodes[:1])
        self.tet_D = tt.grad(tt.nodes)                      # (3, Np, Np): D^a[n,m] = d l_m/d r_a (x_n)
        P, W = tt.exact_rule(tt.N + 2)
        B = tt.basis(P)
        self.tet_Mhat = B.T @ (W[:, None] * B)
        self.tet_Mhat_inv = np.linalg.inv(self.tet_Mhat)
        # ---- wedge: cubature of Sec. 2.1.3 and LSC factors (Alg. wedge_vol1/2)
        wd = self.els[1]
        self.wq_pts, self.wq_w = wd.cubature()
        self.wq_V = wd.basis(self.wq_pts)
        self.wq_Vg = wd.grad(self.wq_pts)
        self.wedge_G, self.wedge_J = self._factors(wd, X[1], self.wq_pts)
        gJ = np.array([wd.jac_grad(xv, self.wq_pts) for xv in X[1]]).reshape(len(X[1]), len(self.wq_w), 3)
        # physical gradient of J: grad_x J = G^T grad_rst J
        self.wedge_gradJ = np.einsum("kqad,kqa->kqd", self.wedge_G, gJ) if len(X[1]) else gJ
        # ---- pyramid: weak derivative operators and factors at the semi-nodal points
        py = self.els[2]
        self.pyr_D = self.pyramid_operators(py)
        ab = py.ab
        rst_ab = np.stack([(ab[:, 0] - 1) / 2, (ab[:, 1] - 1) / 2, np.zeros(len(ab))], axis=1)
        self.pyr_G, self.pyr_J = self._factors(py, X[2], rst_ab)

        # ---- face traces: basis values at the canonical points of every side.
        # Sides sharing (type, local face, canonical corner order) share one matrix.
        sides = self.geo.sides
        self.groups = {}
        for i, s in enumerate(sides):
            self.groups.setdefault((s.t, s.f, s.key), []).append(i)
        self.group_T = {g: self.els[g[0]].basis(sides[idx[0]].rst) for g, idx in self.groups.items()}
        self.group_e = {g: np.array([sides[i].e for i in idx]) for g, idx in self.groups.items()}
        nq = len(sides[0].w) if sides else 0
        self.nq = nq
        self.s_n = np.array([s.n for s in sides]).reshape(-1, nq, 3)
        self.s_wJ = np.array([s.w * s.Js for s in sides]).reshape(-1, nq)
        self.s_sqrtJ = np.array([np.sqrt(s.J) if s.t == 1 else np.ones(nq) for s in sides]).reshape(-1, nq)
        self.s_taup = np.array([s.tau_p for s in sides])
        self.s_nbr = np.array([s.nbr for s in sides], dtype=int)
        skew = lambda s: s.t == 1 or (s.t == 2 and pyr_form == "skew")
        self.s_skew = np.array([skew(s) for s in sides], dtype=bool)

    # ------------------------------------------------------------------ setup helpers
    @staticmethod
    def _factors(el, X, rst):
        """G[k, q, a, d] = d r_a / d x_d and J[k, q] at reference points rst for all elements."""
        if len(X) == 0:
            return np.zeros((0, len(rst), 3, 3)), np.zeros((0, len(rst)))
        F = np.array([el.vmap(xv, rst)[1] for xv in X])
        return np.linalg.inv(F), np.linalg.det(F)

    @staticmethod
    def pyramid_operators(py):
        """D^a_{lmn,ijk} = integral over the reference pyramid of phi_lmn d phi_ijk / d r_a.

        The weak derivative operators of Sec. 2.3.4 built from their definition
        with an over-integrated rule (GL x GL x GJ(2,0), N+3 points).
        """
        P, W = py.exact_rule(py.N + 3)
        B = py.basis(P)
        G = py.grad(P)
        return np.einsum("q,ql,aqm->alm", W, B, G)

    # ------------------------------------------------------------------ views
    def split(self, q):
        """Per-type views (4, K_t, Np_t) of a global state (4, ndof)."""
        return [q[:, self.off[t]:self.off[t + 1]].reshape(4, self.K[t], self.Np[t]) for t in range(4)]

    def traces(self, q):
        """(nsides, 4, nq) traces p, u, v, w at the canonical points of every side.

        For the LSC wedge the trace is (sum_j q_j phi_j) / sqrt(J) (Sec. 2.1.3).
        """
        qv = self.split(q)
        tr = np.zeros((len(self.geo.sides), 4, self.nq))
        for g, idx in self.groups.items():
            tr[idx] = np.einsum("qi,fei->efq", self.group_T[g], qv[g[0]][:, self.group_e[g]])
        return tr / self.s_sqrtJ[:, None, :]

    def neighbour_traces(self, tr):
        """Exterior traces: the neighbour's, or the p = 0 wall mirror state p+ = -p-, u+ = u-."""
        ext = tr[np.maximum(self.s_nbr, 0)].copy()
        wall = self.s_nbr < 0
        ext[wall] = tr[wall]
        ext[wall, 0] *= -1.0
        return ext

    # ------------------------------------------------------------------ rhs
    def volume(self, q):
        """Volume contributions, already multiplied by M^{-1} and by kappa or 1/rho."""
        out = np.zeros_like(q)
        qv = self.split(q)
        ov = self.split(out)
        c2 = self.c2
        # hexahedron, collocated strong form (Alg. hex_vol): M^{-1} cancels w J
        if self.K[0]:
            hx = self.els[0]
            n1 = hx.N + 1
            Q = qv[0].reshape(4, self.K[0], n1, n1, n1)              # [..., k, j, i]
            D = hx.D1
            dr = np.einsum("il,fekjl->fekji", D, Q).reshape(4, self.K[0], -1)
            ds = np.einsum("jl,fekli->fekji", D, Q).reshape(4, self.K[0], -1)
            dt = np.einsum("kl,felji->fekji", D, Q).reshape(4, self.K[0], -1)
            dref = np.stack([dr, ds, dt])                             # (3, 4, K, Np)
            self._collocated(ov[0], dref, self.hex_G, c2[0])
        # tetrahedron, strong form with nodal D^r, D^s, D^t (Alg. tet_vol)
        if self.K[3]:
            dref = np.einsum("anm,fem->afen", self.tet_D, qv[3])
            G = np.broadcast_to(self.tet_G, (self.K[3], self.Np[3], 3, 3))
            self._collocated(ov[3], dref, G, c2[3])
        # wedge, LSC-DG skew-symmetric form (Alg. wedge_vol1/2), M = I
        if self.K[1]:
            V, Vg, w = self.wq_V, self.wq_Vg, self.wq_w
            G, J, gJ = self.wedge_G, self.wedge_J, self.wedge_gradJ
            Pq = np.einsum("qm,em->eq", V, qv[1][0])
            Pg = np.einsum("aqm,em->aeq", Vg, qv[1][0])
            Uq = np.einsum("qm,dem->deq", V, qv[1][1:])
            half = gJ / (2.0 * J[:, :, None])                        # grad_x J / (2J)
            # u-equation: -int phi_i (sqrt(J) grad p)_d, (sqrt J grad p)_d = sum_a G_ad P_a - P J_d/(2J)
            A = np.einsum("eqad,aeq->deq", G, Pg) - Pq[None] * np.moveaxis(half, 2, 0)
            ov[1][1:] = -np.einsum("q,qi,deq->dei", w, V, A) * c2[1][None, :, None]
            # p-equation: int [grad_rst phi_i . (G U)] - phi_i (U . grad J)/(2J)
            GU = np.einsum("eqad,deq->aeq", G, Uq)
            UJ = np.einsum("deq,eqd->eq", Uq, half)
            ov[1][0] = np.einsum("q,aqi,aeq->ei", w, Vg, GU) - np.einsum("q,qi,eq->ei", w, V, UJ)
        # pyramid (Alg. pyr_vol): skew form with transposed operators, or strong form
        if self.K[2]:
            D = self.pyr_D
            G, J = self.pyr_G, self.pyr_J
            p, U = qv[2][0], qv[2][1:]
            Dp = np.einsum("alm,em->ael", D, p)
            ov[2][1:] = -np.einsum("elad,ael->del", G, Dp) * c2[2][None, :, None]   # (1/J) * J * ...
            if self.pyr_form == "skew":
                Ua = J[None] * np.einsum("emad,dem->aem", G, U)              # u^r_j = J r_x u ...
                ov[2][0] = np.einsum("aml,aem->el", D, Ua) / J               # (D^a)^T
            else:
                DU = np.einsum("alm,dem->adel", D, U)
                ov[2][0] = -np.einsum("elad,adel->el", G, DU)
        return out

    @staticmethod
    def _collocated(ov, dref, G, c2):
        """-div u and -c^2 grad p at nodes from reference derivatives (3, 4, K, Np)."""
        grad = np.einsum("enad,afen->dfen", G, dref)                  # grad[d, f] = d q_f / d x_d
        ov[0] = -(grad[0, 1] + grad[1, 2] + grad[2, 3])
        for d in range(3):
            ov[1 + d] = -c2[:, None] * grad[d, 0]

    def surface_integrals(self, q):
        """S[f, dof] = sum over faces of int flux_f phi~_i J^s (before M^{-1}).

        Flux of Eq. (skewform) for skew-form elements (wedge, skew pyramid),
        of the strong form otherwise; u-equation flux 1/2 (tau_u [u].n - [p]) n.
        """
        tr = self.traces(q)
        ext = self.neighbour_traces(tr)
        n = self.s_n                                             # (S, nq, 3)
        um, up = np.moveaxis(tr[:, 1:], 1, 2), np.moveaxis(ext[:, 1:], 1, 2)
        jp = ext[:, 0] - tr[:, 0]
        ju_n = np.sum((up - um) * n, axis=2)
        avg_u_n = np.sum(0.5 * (up + um) * n, axis=2)
        tau_p = (self.tau_scale * self.s_taup)[:, None]
        tau_u = (self.tau_scale / self.s_taup)[:, None]
        fp = np.where(self.s_skew[:, None], 0.5 * tau_p * jp - avg_u_n, 0.5 * (tau_p * jp - ju_n))
        fu = 0.5 * (tau_u * ju_n - jp)
        wJ = self.s_wJ / self.s_sqrtJ                            # LSC test function phi/sqrt(J)
        flux = np.concatenate([(wJ * fp)[:, None], (wJ * fu)[:, None] * np.moveaxis(n, 2, 1)], axis=1)
        S = np.zeros_like(q)
        Sv = self.split(S)
        for g, idx in self.groups.items():
            Sv[g[0]][:, self.group_e[g]] += np.einsum("qi,efq->fei", self.group_T[g], flux[idx])
        return S

    def apply_minv(self, S):
        """Per-type inverse mass matrices of Sec. 2.1 (times kappa = 1 or 1/rho = c^2)."""
        out = np.zeros_like(S)
        Sv, ov = self.split(S), self.split(out)
        hx = self.els[0]
        if self.K[0]:
            ov[0][:] = Sv[0] / (hx.wnodes[None, None, :] * self.hex_J[None])
        if self.K[1]:
            ov[1][:] = Sv[1]
        if self.K[2]:
            ov[2][:] = Sv[2] / self.pyr_J[None]
        if self.K[3]:
            ov[3][:] = np.einsum("nm,fem->fen", self.tet_Mhat_inv, Sv[3]) / self.tet_J[None, :, :1]
        for t in range(4):
            if self.K[t]:
                ov[t][1:] *= self.c2[t][None, :, None]
        return out

    def rhs(self, q):
        """dq/dt = M^{-1} A q."""
        return self.volume(q) + self.apply_minv(self.surface_integrals(q))

    # ------------------------------------------------------------------ mass / energy
    def mass_apply(self, q):
        """M q with the per-type mass matrices of the method (no material weights)."""
        out = np.zeros_like(q)
        qv, ov = self.split(q), self.split(out)
        if self.K[0]:
            ov[0][:] = qv[0] * self.els[0].wnodes[None, None, :] * self.hex_J[None]
        if self.K[1]:
            ov[1][:] = qv[1]
        if self.K[2]:
            ov[2][:] = qv[2] * self.pyr_J[None]
        if self.K[3]:
            ov[3][:] = np.einsum("nm,fem->fen", self.tet_Mhat, qv[3]) * self.tet_J[None, :, :1]
        return out

    def material_weights(self):
        """(4, ndof): 1/kappa = 1 for p, rho = 1/c^2 for u."""
        wts = np.ones((4, self.ndof))
        for t in range(4):
            wts[1:, self.off[t]:self.off[t + 1]] = np.repeat(1.0 / self.c2[t], self.Np[t])[None]
        return wts

    def energy(self, q):
        """E = 1/2 sum_K (p^T M_K p / kappa + rho u^T M_K u) (Sec. 3 energy norm)."""
        return 0.5 * float(np.sum(q * self.mass_apply(q) * self.material_weights()))

    def jump_dissipation(self, q):
        """-1/2 sum over faces of int (tau_p [p]^2 + tau_u [u_n]^2) (Eq. sym).

        Each interior face counted once; a wall face with the mirror state counts
        half of its jump energy (the mirror element does not exist).
        """
        tr = self.traces(q)
        ext = self.neighbour_traces(tr)
        jp = ext[:, 0] - tr[:, 0]
        jun = np.sum((np.moveaxis(ext[:, 1:], 1, 2) - np.moveaxis(tr[:, 1:], 1, 2)) * self.s_n, axis=2)
        # every interior face is seen from both sides (factor 1/2 each); wall faces once, halved
        fac = 0.5
        dens = self.s_taup[:, None] * jp ** 2 + jun ** 2 / self.s_taup[:, None]
        return -0.5 * fac * self.tau_scale * float(np.sum(self.s_wJ * dens))

    # ------------------------------------------------------------------ time stepping
    def lsrk_step(self, q, dt):
        """One LSRK(5,4) step: res = a_k res + dt rhs(q); q = q + b_k res."""
        q = q.copy()
        res = np.zeros_like(q)
        for a, b in zip(LSRK_A, LSRK_B):
            res = a * res + dt * self.rhs(q)
            q = q + b * res
        return q

    # ------------------------------------------------------------------ time step (Eq. dtK)
    def local_dt(self, CT, cfl=0.5):
        """dtau_K = C / (C^K_{rho,kappa} C_T(N) C_J^K) for every element (Eq. dtK).

        ``CT[t]`` is the reference trace constant C_T(N) of type t, computed with
        the Euclidean face measure of the reference element (Table computedTrace);
        J^s is therefore taken relative to that same reference face measure.
        C_J^K = max J^s * max 1/J over quadrature points (hex: GL nodes, pyramid:
        semi-nodal points, tet: constant) or max J^s/J over face points (LSC wedge).
        C^K_{rho,kappa} = max(tau_p,K kappa, tau_u,K / rho) with tau_p,K, tau_u,K
        the largest penalties over the faces of K.
        """
        out = [np.zeros(k) for k in self.K]
        jsmax = [np.zeros(k) for k in self.K]
        jsj = [np.zeros(k) for k in self.K]
        taup = [np.zeros(k) for k in self.K]
        tauu = [np.zeros(k) for k in self.K]
        for s in self.geo.sides:
            js = s.Js / s.Js_ref
            jsmax[s.t][s.e] = max(jsmax[s.t][s.e], float(np.max(js)))
            jsj[s.t][s.e] = max(jsj[s.t][s.e], float(np.max(js / s.J)))
            taup[s.t][s.e] = max(taup[s.t][s.e], s.tau_p)
            tauu[s.t][s.e] = max(tauu[s.t][s.e], 1.0 / s.tau_p)
        Jinv = {0: np.max(1.0 / self.hex_J, axis=1) if self.K[0] else None,
                2: np.max(1.0 / self.pyr_J, axis=1) if self.K[2] else None,
                3: (1.0 / self.tet_J[:, 0]) if self.K[3] else None}
        for t in range(4):
            if not self.K[t]:
                continue
            crk = np.maximum(taup[t] * 1.0, tauu[t] * self.c2[t])
            cj = jsj[t] if t == 1 else jsmax[t] * Jinv[t]
            out[t] = cfl / (crk * CT[t] * cj)
        return out

    def global_dt(self, CT, cfl=0.5):
        """dtau_min = min_K dtau_K."""
        return min(float(np.min(d)) for d in self.local_dt(CT, cfl) if len(d))

    # ------------------------------------------------------------------ projection / error
    def _element_rule(self, t, e, q=None):
        el = self.els[t]
        P, W = el.exact_rule(q or self.N + 3)
        xv = self.mesh.xyz[self.mesh.conn[t][e]]
        x, F = el.vmap(xv, P)
        J = np.linalg.det(F)
        return el, P, W, x, J

    def project(self, fun, time=0.0):
        """L2 projection onto the discrete space, (4, ndof): c = M_K^{-1} int f phi~ (over-integrated).

        For the LSC wedge, int f phi/sqrt(J) J = int f phi sqrt(J) and M = I.
        """
        q = np.zeros((4, self.ndof))
        qv = self.split(q)
        for t in range(4):
            for e in range(self.K[t]):
                el, P, W, x, J = self._element_rule(t, e)
                B = el.basis(P)
                vals = fun(x, time)                                   # (4, nq)
                if t == 1:
                    rhs = np.einsum("q,qi,fq->fi", W * np.sqrt(J), B, vals)
                    qv[t][:, e] = rhs
                    continue
                rhs = np.einsum("q,qi,fq->fi", W * J, B, vals)
                if t == 0:
                    Mk = self.els[0].wnodes * self.hex_J[e]
                    qv[t][:, e] = rhs / Mk
                elif t == 2:
                    qv[t][:, e] = rhs / self.pyr_J[e]
                else:
                    qv[t][:, e] = rhs @ self.tet_Mhat_inv.T / self.tet_J[e, 0]
        return q

    def l2_error(self, q, fun, time):
        """sqrt( sum_K int |q_h - q_exact|^2 dx ) over all four fields (over-integrated)."""
        qv = self.split(q)
        err = 0.0
        for t in range(4):
            for e in range(self.K[t]):
                el, P, W, x, J = self._element_rule(t, e)
                uh = el.basis(P) @ qv[t][:, e].T                      # (nq, 4)
                if t == 1:
                    uh = uh / np.sqrt(J)[:, None]
                err += float(np.sum(W * J * np.sum((uh.T - fun(x, time)) ** 2, axis=0)))
        return np.sqrt(err)


def standing_mode(x, time):
    """Exact standing mode on [-1,1]^3 with c = 1 and p = 0 walls.

    p = cos(pi x/2) cos(pi y/2) cos(pi z/2) cos(sqrt(3) pi t/2),
    u = (1/sqrt(3)) (sin cos cos, cos sin cos, cos cos sin)(pi x/2, ...) sin(sqrt(3) pi t/2).
    """
    x = np.atleast_2d(x)
    h = np.pi / 2 * x
    c, s = np.cos(h), np.sin(h)
    w = np.sqrt(3.0) * np.pi / 2 * time
    p = c[:, 0] * c[:, 1] * c[:, 2] * np.cos(w)
    a = np.sin(w) / np.sqrt(3.0)
    return np.stack([p, a * s[:, 0] * c[:, 1] * c[:, 2], a * c[:, 0] * s[:, 1] * c[:, 2],
                     a * c[:, 0] * c[:, 1] * s[:, 2]])


# ---------------------------------------------------------------------- multi-rate AB3
AB3 = np.array([23.0, -16.0, 5.0]) / 12.0          # int_0^1 of the quadratic through r^n, r^{n-1}, r^{n-2}
AB3_HALF = np.array([17.0, -7.0, 2.0]) / 24.0      # int_0^{1/2} of the same quadratic


def mr_levels(dg, CT, nlevels, cfl=0.5):
    """Multi-rate levels of Sec. 2.4 (level 1 = coarsest, nlevels = finest).

    dtau_lev = 2^(nlevels - lev) dtau_min.  Reading of the binning (the printed
    inequality is reversed): element K gets the coarsest level whose step does
    not exceed dtau_K.  A second sweep moves elements to finer levels until
    face neighbours differ by at most one level.  Returns per-type int arrays.
    """
    dts = dg.local_dt(CT, cfl)
    dmin = min(float(np.min(d)) for d in dts if len(d))
    lev = []
    for d in dts:
        lv = np.full(len(d), nlevels, dtype=int)
        for idx in range(len(d)):
            for L in range(1, nlevels + 1):
                if (2.0 ** (nlevels - L)) * dmin <= d[idx] * (1 + 1e-12):
                    lv[idx] = L
                    break
        lev.append(lv)
    sides = dg.geo.sides
    changed = True
    while changed:
        changed = False
        for s in sides:
            if s.nbr < 0:
                continue
            o = sides[s.nbr]
            a, b = lev[s.t][s.e], lev[o.t][o.e]
            if a < b - 1:
                lev[s.t][s.e] = b - 1
                changed = True
    return lev, dmin


class MRAB3:
    """Two-level multi-rate Adams-Bashforth 3 (reading of Sec. 2.4; details of the
    scheme are deferred by the paper to other work).

    Fine step h, coarse step 2h.  Per coarse step from t_n:
      r = rhs(q) for all elements;
      fine:    q_f <- q_f + h sum AB3 * (r_f^n, r_f^{n-1}, r_f^{n-2});
      coarse:  predicted q_c(t_n + h) = q_c + 2h sum AB3_HALF * (r_c^n, r_c^{n-1}, r_c^{n-2});
      r' = rhs(q_f, predicted q_c), fine part only;
      fine:    q_f <- q_f + h sum AB3 * (r'_f, r_f^n, r_f^{n-1});
      coarse:  q_c <- q_c + 2h sum AB3 * (r_c^n, r_c^{n-1}, r_c^{n-2}).
    Start-up: four LSRK(5,4) steps of size h, recording rhs at t = 0, 2h (coarse
    history) and 2h, 3h (fine history).
    """

    def __init__(self, dg, level):
        self.dg = dg
        mask = np.zeros((4, dg.ndof), dtype=bool)
        mv = dg.split(mask)
        for t in range(4):
            mv[t][:] = (level[t] == 2)[None, :, None]
        self.fine = mask
        self.coarse = ~mask

    def start(self, q, h):
        """Returns (q(4h), history) with history = (coarse [r(2h), r(0)], fine [r(3h), r(2h)])."""
        dg = self.dg
        r0 = dg.rhs(q)
        q = dg.lsrk_step(q, h)
        q = dg.lsrk_step(q, h)
        r2 = dg.rhs(q)
        q = dg.lsrk_step(q, h)
        r3 = dg.rhs(q)
        q = dg.lsrk_step(q, h)
        return q, ([r2, r0], [r3, r2])

    def step(self, q, hist, h):
        dg = self.dg
        F, Cm = self.fine, self.coarse
        (c1, c2), (f1, f2) = hist
        r = dg.rhs(q)
        qn = q.copy()
        qn[F] = q[F] + h * (AB3[0] * r[F] + AB3[1] * f1[F] + AB3[2] * f2[F])
        pred = qn.copy()
        pred[Cm] = q[Cm] + 2 * h * (AB3_HALF[0] * r[Cm] + AB3_HALF[1] * c1[Cm] + AB3_HALF[2] * c2[Cm])
        rh = dg.rhs(pred)
        out = qn.copy()
        out[F] = qn[F] + h * (AB3[0] * rh[F] + AB3[1] * r[F] + AB3[2] * f1[F])
        out[Cm] = q[Cm] + 2 * h * (AB3[0] * r[Cm] + AB3[1] * c1[Cm] + AB3[2] * c2[Cm])
        return out, ([r, c1], [rh, r])


# ---------------------------------------------------------------------- multi-rate LSRK
def lsrk_stability_coefficients():
    """rho_0..rho_5 of R(z) = sum rho_i z^i, the amplification of LSRK(5,4) on y' = lambda y
    (the 2N-storage recursion applied to polynomials in z)."""
    poly = np.polynomial.polynomial
    y, res = np.array([1.0]), np.array([0.0])
    for a, b in zip(LSRK_A, LSRK_B):
        res = poly.polyadd(a * res, poly.polymul([0.0, 1.0], y))
        y = poly.polyadd(y, b * res)
    return np.concatenate([y, np.zeros(6 - len(y))])[:6]


class MRLSRK:
    """Two-level multi-rate LSRK(5,4) (reading of Sec. 2.4 for a Runge-Kutta integrator), a local
    time-stepping scheme in the manner of the LTS-RK methods of Grote, Mehlin & Mitkova (2015):
    the coarse region's influence over a coarse step is a polynomial in time built from operator
    powers at t_n, and the fine region is integrated by LSRK(5,4) substeps against it.

    Fine step h, coarse step H = 2h, P = restriction to the fine elements' DOFs, B = M^{-1} A.
    Per coarse step from y_n:
      z_0 = y_n, z_j = B z_{j-1} (j = 1..4);   u_j = B (I - P) z_j (j = 0..4);
      W(tau) = sum_j rho_{j+1} tau^{j+1} u_j, with R(z) = sum rho_i z^i the LSRK(5,4) amplification;
      v(0) = 0, v' = B P (y_n + W(tau) + v), integrated by two LSRK(5,4) steps of h;
      y_{n+1} = y_n + W(H) + v(H).
    W' = sum_j (j+1) rho_{j+1} tau^j u_j agrees with the Taylor expansion of B (I - P) y(t_n + tau)
    through tau^3, so the scheme is fourth order.  With no fine element (P = 0), v = 0 and
    y_{n+1} = R(H B) y_n, one LSRK(5,4) step of H; with only fine elements (P = I), u_j = 0 and
    the scheme is two LSRK(5,4) steps of h.  B P v and u_j vanish outside the fine elements and
    the coarse elements that share a face with one.
    """

    def __init__(self, dg, level):
        self.dg = dg
        mask = np.zeros((4, dg.ndof), dtype=bool)
        mv = dg.split(mask)
        for t in range(4):
            mv[t][:] = (level[t] == 2)[None, :, None]
        self.fine = mask
        self.rho = lsrk_stability_coefficients()

    def step(self, y, h):
        dg, F, rho = self.dg, self.fine, self.rho
        H = 2.0 * h
        z = [y]
        for _ in range(4):
            z.append(dg.rhs(z[-1]))
        u = []
        for zj in z:
            zc = zj.copy()
            zc[F] = 0.0
            u.append(dg.rhs(zc))
        W = lambda tau: sum(rho[j + 1] * tau ** (j + 1) * u[j] for j in range(5))

        def fine_rhs(v, tau):
            x = y + W(tau) + v
            x[~F] = 0.0
            return dg.rhs(x)

        v = np.zeros_like(y)
        for s in range(2):
            res = np.zeros_like(y)
            for a, b, c in zip(LSRK_A, LSRK_B, LSRK_C):
                res = a * res + h * fine_rhs(v, (s + c) * h)
                v = v + b * res
        return y + W(H) + v
