"""Reference elements of Sec. 2.1 (float64, plain loops / numpy).

Each class gives, for order N:

* ``basis(rst)`` / ``grad(rst)``: values and reference gradients of the
  polynomial basis phi_i (for the LSC wedge this is the *numerator* of
  phi_i / sqrt(J), Sec. 2.1.3);
* ``faces``: local vertex lists of the faces (triangles ``[c0,c1,c2]``, quads
  lexicographic ``[c00,c10,c01,c11]``) and ``face_grad``: the reference gradient
  of a function that increases out of the element through that face;
* ``vmap(xv, rst)``: physical points and the Jacobian matrix dx/d(rst) of the
  vertex map;
* ``exact_rule(q)``: a tensor cubature exact for reference-polynomial degree
  about 2q-1 (used to build operators from their definitions).

Reference coordinates and local vertex orders are the ones documented in
``paper_1507_02557_b300.inputs``.
"""
from __future__ import annotations

import numpy as np

from .jacobi import (gauss_jacobi, gauss_legendre, gauss_lobatto, jacobi_dp,
                     jacobi_p, lagrange_1d, lagrange_1d_deriv)


# ---------------------------------------------------------------- helpers
def _collapsed_tri(n):
    """Collapsed (Stroud) rule on the triangle {xi,eta >= -1, xi+eta <= 0}.

    GL(n) in a times Gauss-Jacobi(1,0)(n) in b, xi = (1+a)(1-b)/2 - 1, eta = b.
    Exact for total degree 2n-1; weights sum to 2.  Point index ia + n*ib.
    """
    a, wa = gauss_legendre(n)
    b, wb = gauss_jacobi(n, 1.0, 0.0)
    A, B = np.meshgrid(a, b, indexing="xy")
    WA, WB = np.meshgrid(wa, wb, indexing="xy")
    xi = (1.0 + A) * (1.0 - B) / 2.0 - 1.0
    eta = B
    return np.stack([xi.ravel(), eta.ravel()], axis=1), (WA * WB).ravel() / 2.0


def tri_face_rule(N):
    """Triangle face rule of Sec. 2.3 (reading: collapsed rule with N+1 points per direction)."""
    return _collapsed_tri(N + 1)


def quad_face_rule(N, lobatto=False):
    """Quadrilateral face rule: (N+1)^2 tensor GL (or GLL for SEM), index i + (N+1) j."""
    x, w = gauss_lobatto(N + 1) if lobatto else gauss_legendre(N + 1)
    X, Y = np.meshgrid(x, x, indexing="xy")
    W1, W2 = np.meshgrid(w, w, indexing="xy")
    return np.stack([X.ravel(), Y.ravel()], axis=1), (W1 * W2).ravel()


# ---------------------------------------------------------------- hexahedron
class Hex:
    """Nodal Q_N basis at tensor GL (or GLL = SEM) nodes, Sec. 2.1.1."""

    nverts = 8
    verts = np.array([[-1, -1, -1], [1, -1, -1], [-1, 1, -1], [1, 1, -1],
                      [-1, -1, 1], [1, -1, 1], [-1, 1, 1], [1, 1, 1]], dtype=float)
    faces = [[0, 2, 4, 6], [1, 3, 5, 7], [0, 1, 4, 5], [2, 3, 6, 7], [0, 1, 2, 3], [4, 5, 6, 7]]
    face_grad = np.array([[-1, 0, 0], [1, 0, 0], [0, -1, 0], [0, 1, 0], [0, 0, -1], [0, 0, 1]], float)

    def __init__(self, N, lobatto=False):
        self.N = N
        self.Np = (N + 1) ** 3
        self.lobatto = lobatto
        self.r1, self.w1 = gauss_lobatto(N + 1) if lobatto else gauss_legendre(N + 1)
        n1 = N + 1
        idx = np.arange(self.Np)
        self.ijk = np.stack([idx % n1, (idx // n1) % n1, idx // (n1 * n1)], axis=1)
        self.nodes = self.r1[self.ijk]
        self.wnodes = np.prod(self.w1[self.ijk], axis=1)
        # D_il = ell_l'(r_i), the 1D derivative matrix of Alg. hex_vol
        self.D1 = lagrange_1d_deriv(self.r1, self.r1)

    def basis(self, rst):
        rst = np.atleast_2d(rst)
        L = [lagrange_1d(self.r1, rst[:, a]) for a in range(3)]
        return L[0][:, self.ijk[:, 0]] * L[1][:, self.ijk[:, 1]] * L[2][:, self.ijk[:, 2]]

    def grad(self, rst):
        rst = np.atleast_2d(rst)
        L = [lagrange_1d(self.r1, rst[:, a]) for a in range(3)]
        dL = [lagrange_1d_deriv(self.r1, rst[:, a]) for a in range(3)]
        i, j, k = self.ijk.T
        return np.stack([dL[0][:, i] * L[1][:, j] * L[2][:, k],
                         L[0][:, i] * dL[1][:, j] * L[2][:, k],
                         L[0][:, i] * L[1][:, j] * dL[2][:, k]])

    @staticmethod
    def vmap(xv, rst):
        """Trilinear vertex map; xv (8,3).  Returns x (n,3), F (n,3,3) with F[:, a, b] = dx_a/dr_b."""
        rst = np.atleast_2d(rst)
        r, s, t = rst.T
        x = np.zeros((rst.shape[0], 3))
        F = np.zeros((rst.shape[0], 3, 3))
        for v in range(8):
            sr, ss, st = Hex.verts[v]
            fr, fs, ft = (1 + sr * r) / 2, (1 + ss * s) / 2, (1 + st * t) / 2
            x += np.outer(fr * fs * ft, xv[v])
            F[:, :, 0] += np.outer(sr / 2 * fs * ft, xv[v])
            F[:, :, 1] += np.outer(fr * ss / 2 * ft, xv[v])
            F[:, :, 2] += np.outer(fr * fs * st / 2, xv[v])
        return x, F

    @staticmethod
    def exact_rule(q):
        x, w = gauss_legendre(q)
        P = np.array(np.meshgrid(x, x, x, indexing="ij")).reshape(3, -1).T
        W = np.einsum("i,j,k->ijk", w, w, w).ravel()
        return P, W


# ---------------------------------------------------------------- tetrahedron
class Tet:
    """Nodal P_N basis on the bi-unit right tetrahedron, Sec. 2.1.2.

    Reading (the optimised node set of the paper is not tabulated in it): nodes on
    the equispaced lattice r,s,t = -1 + 2(i,j,k)/N, ordered k, then j, then i.
    The nodal basis is built from the Legendre-tensor monomials P_a(r)P_b(s)P_c(t),
    a+b+c <= N, which span P_N.
    """

    nverts = 4
    verts = np.array([[-1, -1, -1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], dtype=float)
    faces = [[0, 1, 2], [0, 1, 3], [1, 2, 3], [0, 2, 3]]
    face_grad = np.array([[0, 0, -1], [0, -1, 0], [1, 1, 1], [-1, 0, 0]], float)

    def __init__(self, N):
        self.N = N
        self.Np = (N + 1) * (N + 2) * (N + 3) // 6
        nodes = []
        for k in range(N + 1):
            for j in range(N + 1 - k):
                for i in range(N + 1 - j - k):
                    nodes.append([-1 + 2 * i / N, -1 + 2 * j / N, -1 + 2 * k / N])
        self.nodes = np.array(nodes)
        self.modes = [(a, b, c) for a in range(N + 1) for b in range(N + 1) for c in range(N + 1)
                      if a + b + c <= N]
        self.Vinv = np.linalg.inv(self._modal(self.nodes))

    def _modal(self, rst):
        rst = np.atleast_2d(rst)
        return np.stack([jacobi_p(a, 0, 0, rst[:, 0]) * jacobi_p(b, 0, 0, rst[:, 1])
                         * jacobi_p(c, 0, 0, rst[:, 2]) for a, b, c in self.modes], axis=1)

    def _modal_grad(self, rst):
        rst = np.atleast_2d(rst)
        r, s, t = rst.T
        g = np.zeros((3, rst.shape[0], len(self.modes)))
        for m, (a, b, c) in enumerate(self.modes):
            Pa, Pb, Pc = jacobi_p(a, 0, 0, r), jacobi_p(b, 0, 0, s), jacobi_p(c, 0, 0, t)
            g[0, :, m] = jacobi_dp(a, 0, 0, r) * Pb * Pc
            g[1, :, m] = Pa * jacobi_dp(b, 0, 0, s) * Pc
            g[2, :, m] = Pa * Pb * jacobi_dp(c, 0, 0, t)
        return g

    def basis(self, rst):
        return self._modal(rst) @ self.Vinv

    def grad(self, rst):
        return self._modal_grad(rst) @ self.Vinv

    @staticmethod
    def vmap(xv, rst):
        rst = np.atleast_2d(rst)
        lam = np.stack([-(1 + rst[:, 0] + rst[:, 1] + rst[:, 2]) / 2,
                        (1 + rst[:, 0]) / 2, (1 + rst[:, 1]) / 2, (1 + rst[:, 2]) / 2], axis=1)
        x = lam @ xv
        Fm = np.stack([(xv[1] - xv[0]) / 2, (xv[2] - xv[0]) / 2, (xv[3] - xv[0]) / 2], axis=1)
        return x, np.broadcast_to(Fm, (rst.shape[0], 3, 3)).copy()

    @staticmethod
    def exact_rule(q):
        """Duffy-collapsed rule: GL(a) x GJ(1,0)(b) x GJ(2,0)(c), weight /8."""
        a, wa = gauss_legendre(q)
        b, wb = gauss_jacobi(q, 1.0, 0.0)
        c, wc = gauss_jacobi(q, 2.0, 0.0)
        A, B, C = np.meshgrid(a, b, c, indexing="ij")
        W = np.einsum("i,j,k->ijk", wa, wb, wc).ravel() / 8.0
        A, B, C = A.ravel(), B.ravel(), C.ravel()
        r = (1 + A) * (1 - B) / 2 * (1 - C) / 2 - 1
        s = (1 + B) * (1 - C) / 2 - 1
        return np.stack([r, s, C], axis=1), W


# ---------------------------------------------------------------- wedge
class Wedge:
    """Orthonormal modal basis of Sec. 2.1.3 (LSC-DG numerator).

    phi_ijk = P_i(a) P_j(b) ((1-c)/2)^i P_k^{(2i+1,0)}(c) / norm, with
    r = (1+a)(1-c)/2 - 1, s = b, t = c; 0<=i,j<=N, 0<=k<=N-i.  DOF index
    m + Ntri*j, where m enumerates (i,k) with i outer and k inner.
    The LSC basis function is phi/sqrt(J).
    """

    nverts = 6
    verts = np.array([[-1, -1, -1], [1, -1, -1], [-1, -1, 1],
                      [-1, 1, -1], [1, 1, -1], [-1, 1, 1]], dtype=float)
    faces = [[0, 1, 2], [3, 4, 5], [0, 1, 3, 4], [1, 2, 4, 5], [0, 2, 3, 5]]
    face_grad = np.array([[0, -1, 0], [0, 1, 0], [0, 0, -1], [1, 0, 1], [-1, 0, 0]], float)

    def __init__(self, N):
        self.N = N
        self.tri = [(i, k) for i in range(N + 1) for k in range(N + 1 - i)]
        self.Ntri = len(self.tri)
        self.modes = [(i, j, k) for j in range(N + 1) for (i, k) in self.tri]
        self.Np = len(self.modes)
        # normalisation by quadrature on the reference wedge
        P, W = self.exact_rule(N + 2)
        raw = self._raw(P)
        self.norm = np.sqrt(np.einsum("q,qm,qm->m", W, raw, raw))

    @staticmethod
    def _abc(rst):
        # collapsed coordinate of the triangle (r, t); at its collapsed vertex t = 1 every mode
        # with i >= 1 carries ((1 - t)/2)^i, so the limit is taken at a = 0 there (values only)
        r, s, t = rst.T
        h = 1 - t
        a = np.where(h > 1e-14, 2 * (1 + r) / np.where(h > 1e-14, h, 1.0) - 1, 0.0)
        return a, s, t

    def _raw(self, rst):
        rst = np.atleast_2d(rst)
        a, b, c = self._abc(rst)
        return np.stack([jacobi_p(i, 0, 0, a) * jacobi_p(j, 0, 0, b) * ((1 - c) / 2) ** i
                         * jacobi_p(k, 2 * i + 1, 0, c) for i, j, k in self.modes], axis=1)

    def basis(self, rst):
        return self._raw(rst) / self.norm

    def grad(self, rst):
        rst = np.atleast_2d(rst)
        a, b, c = self._abc(rst)
        g = np.zeros((3, rst.shape[0], self.Np))
        for m, (i, j, k) in enumerate(self.modes):
            Pi, dPi = jacobi_p(i, 0, 0, a), jacobi_dp(i, 0, 0, a)
            Pj, dPj = jacobi_p(j, 0, 0, b), jacobi_dp(j, 0, 0, b)
            Pk, dPk = jacobi_p(k, 2 * i + 1, 0, c), jacobi_dp(k, 2 * i + 1, 0, c)
            h = ((1 - c) / 2)
            # d/da term carries a factor ((1-c)/2)^(i-1) after the chain rule d a/d r = 2/(1-c)
            hi1 = h ** (i - 1) if i > 0 else np.zeros_like(c)
            d_a = dPi * Pj * Pk * hi1            # (d phi/d a) * 2/(1-c)
            g[0, :, m] = d_a
            g[1, :, m] = Pi * dPj * h ** i * Pk
            dc = Pi * Pj * (h ** i * dPk - (i / 2.0) * hi1 * Pk)
            g[2, :, m] = d_a * (1 + a) / 2 + dc
        return g / self.norm

    @staticmethod
    def vmap(xv, rst):
        rst = np.atleast_2d(rst)
        r, s, t = rst.T
        lam = np.stack([-(r + t) / 2, (1 + r) / 2, (1 + t) / 2], axis=1)
        dlam_dr = np.array([-0.5, 0.5, 0.0])
        dlam_dt = np.array([-0.5, 0.0, 0.5])
        lo, hi = xv[:3], xv[3:]
        fs0, fs1 = (1 - s) / 2, (1 + s) / 2
        x = (lam @ lo) * fs0[:, None] + (lam @ hi) * fs1[:, None]
        F = np.zeros((rst.shape[0], 3, 3))
        F[:, :, 0] = np.outer(fs0, dlam_dr @ lo) + np.outer(fs1, dlam_dr @ hi)
        F[:, :, 1] = (lam @ hi - lam @ lo) / 2
        F[:, :, 2] = np.outer(fs0, dlam_dt @ lo) + np.outer(fs1, dlam_dt @ hi)
        return x, F

    @staticmethod
    def jac_grad(xv, rst):
        """Reference gradient of J = det(dx/drst) for the wedge map (analytic)."""
        rst = np.atleast_2d(rst)
        s = rst[:, 1]
        lo, hi = xv[:3], xv[3:]
        dlam_dr = np.array([-0.5, 0.5, 0.0])
        dlam_dt = np.array([-0.5, 0.0, 0.5])
        _, F = Wedge.vmap(xv, rst)
        # second derivatives of the map: only x_rs, x_ts, x_sr, x_st are nonzero
        x_rs = (dlam_dr @ hi - dlam_dr @ lo) / 2
        x_ts = (dlam_dt @ hi - dlam_dt @ lo) / 2
        dF = np.zeros((3, rst.shape[0], 3, 3))   # dF[d] = dF/d rst_d
        dF[0, :, :, 1] = x_rs                   # d x_s / d r
        dF[2, :, :, 1] = x_ts                   # d x_s / d t
        dF[1, :, :, 0] = x_rs                   # d x_r / d s
        dF[1, :, :, 2] = x_ts                   # d x_t / d s
        g = np.zeros((rst.shape[0], 3))
        for d in range(3):
            for col in range(3):
                M = F.copy()
                M[:, :, col] = dF[d, :, :, col]
                g[:, d] += np.linalg.det(M)
        return g

    def cubature(self):
        """Wedge volume rule of Sec. 2.1.3: triangle rule (degree 2N+1) in (r,t) x GL(N+1) in s.

        Reading: the triangle rule is the collapsed rule with N+1 points per
        direction (the Xiao-Gimbutas tables are not in the paper).  Index
        q_tri + Ntq * l.
        """
        tp, tw = _collapsed_tri(self.N + 1)
        sx, sw = gauss_legendre(self.N + 1)
        P = np.array([[tp[q, 0], sx[l], tp[q, 1]] for l in range(len(sx)) for q in range(len(tw))])
        W = np.array([tw[q] * sw[l] for l in range(len(sx)) for q in range(len(tw))])
        return P, W

    @staticmethod
    def exact_rule(q):
        tp, tw = _collapsed_tri(q)
        sx, sw = gauss_legendre(q)
        P = np.array([[tp[i, 0], sx[l], tp[i, 1]] for l in range(q) for i in range(len(tw))])
        W = np.array([tw[i] * sw[l] for l in range(q) for i in range(len(tw))])
        return P, W


# ---------------------------------------------------------------- pyramid
class Pyramid:
    """Semi-nodal orthogonal basis of Sec. 2.1.4 on the rational space B_N.

    phi_ijk = l^k_i(a) l^k_j(b) ((1-c)/2)^k P^{(2k+3,0)}_{N-k}(c) / sqrt(w^k_i w^k_j gamma_k),
    0 <= i,j <= k <= N, with l^k the Lagrange polynomials at the (k+1)-point GL
    nodes, w^k their weights, r = (1+a)(1-c)/2 - 1, s = (1+b)(1-c)/2 - 1, t = c.

    Reading of the normalisation (the printed constant C^N_{N-k} is not
    consistent with the integral it normalises): gamma_k is the integral of
    ((1-c)/2)^{2k+2} (P^{(2k+3,0)}_{N-k})^2 over [-1,1], so that the reference
    mass matrix is the identity and the mapped one is diag(J(a^k_i, b^k_j)).
    DOF order: k outer, then j, then i.
    """

    nverts = 5
    verts = np.array([[-1, -1, -1], [1, -1, -1], [-1, 1, -1], [1, 1, -1], [-1, -1, 1]], dtype=float)
    faces = [[0, 1, 2, 3], [0, 1, 4], [1, 3, 4], [2, 3, 4], [0, 2, 4]]
    face_grad = np.array([[0, 0, -1], [0, -1, 0], [1, 0, 1], [0, 1, 1], [-1, 0, 0]], float)

    def __init__(self, N):
        self.N = N
        self.levels = []
        for k in range(N + 1):
            x, w = gauss_legendre(k + 1)
            self.levels.append((x, w))
        self.modes = [(i, j, k) for k in range(N + 1) for j in range(k + 1) for i in range(k + 1)]
        self.Np = len(self.modes)
        c, wc = gauss_jacobi(N + 4, 0.0, 0.0)
        self.gamma = np.array([np.sum(wc * ((1 - c) / 2) ** (2 * k + 2)
                                      * jacobi_p(N - k, 2 * k + 3, 0, c) ** 2) for k in range(N + 1)])
        # semi-nodal points (a^k_i, b^k_j) of each DOF
        self.ab = np.array([[self.levels[k][0][i], self.levels[k][0][j]] for i, j, k in self.modes])
        self.wab = np.array([self.levels[k][1][i] * self.levels[k][1][j] for i, j, k in self.modes])

    @staticmethod
    def abc(rst):
        r, s, t = np.atleast_2d(rst).T
        return 2 * (1 + r) / (1 - t) - 1, 2 * (1 + s) / (1 - t) - 1, t

    def basis_abc(self, a, b, c):
        out = np.zeros((np.size(a), self.Np))
        for m, (i, j, k) in enumerate(self.modes):
            x, w = self.levels[k]
            la = lagrange_1d(x, a)[:, i]
            lb = lagrange_1d(x, b)[:, j]
            out[:, m] = (la * lb * ((1 - c) / 2) ** k * jacobi_p(self.N - k, 2 * k + 3, 0, c)
                         / np.sqrt(w[i] * w[j] * self.gamma[k]))
        return out

    def basis(self, rst):
        return self.basis_abc(*self.abc(rst))

    def grad(self, rst):
        a, b, c = self.abc(rst)
        g = np.zeros((3, np.size(a), self.Np))
        h = (1 - c) / 2
        for m, (i, j, k) in enumerate(self.modes):
            x, w = self.levels[k]
            la, dla = lagrange_1d(x, a)[:, i], lagrange_1d_deriv(x, a)[:, i]
            lb, dlb = lagrange_1d(x, b)[:, j], lagrange_1d_deriv(x, b)[:, j]
            P = jacobi_p(self.N - k, 2 * k + 3, 0, c)
            dP = jacobi_dp(self.N - k, 2 * k + 3, 0, c)
            nrm = np.sqrt(w[i] * w[j] * self.gamma[k])
            hk1 = h ** (k - 1) if k > 0 else np.zeros_like(c)
            # d/dr = (2/(1-c)) d/da ; d/ds = (2/(1-c)) d/db
            g_r = dla * lb * hk1 * P
            g_s = la * dlb * hk1 * P
            g_c = la * lb * (h ** k * dP - (k / 2.0) * hk1 * P)
            g[0, :, m] = g_r / nrm
            g[1, :, m] = g_s / nrm
            # d/dt = (1+a)/(1-c) d/da + (1+b)/(1-c) d/db + d/dc
            g[2, :, m] = ((1 + a) / 2 * g_r + (1 + b) / 2 * g_s + g_c) / nrm
        return g

    @staticmethod
    def vmap(xv, rst):
        """Rational (Bedrosian) vertex map x = (1-c)/2 B(a,b) + (1+c)/2 x_apex."""
        a, b, c = Pyramid.abc(rst)
        base = xv[:4]
        Nab = np.stack([(1 - a) * (1 - b), (1 + a) * (1 - b), (1 - a) * (1 + b), (1 + a) * (1 + b)], 1) / 4
        dNa = np.stack([-(1 - b), (1 - b), -(1 + b), (1 + b)], 1) / 4
        dNb = np.stack([-(1 - a), -(1 + a), (1 - a), (1 + a)], 1) / 4
        B, Ba, Bb = Nab @ base, dNa @ base, dNb @ base
        x = B * ((1 - c) / 2)[:, None] + np.outer((1 + c) / 2, xv[4])
        F = np.zeros((np.size(a), 3, 3))
        F[:, :, 0] = Ba
        F[:, :, 1] = Bb
        F[:, :, 2] = Ba * ((1 + a) / 2)[:, None] + Bb * ((1 + b) / 2)[:, None] + (xv[4][None, :] - B) / 2
        return x, F

    @staticmethod
    def exact_rule(q):
        """GL(a) x GL(b) x GJ(2,0)(c) with dr ds dt = ((1-c)/2)^2 da db dc (Sec. 2.1.4)."""
        a, wa = gauss_legendre(q)
        c, wc = gauss_jacobi(q, 2.0, 0.0)
        A, B, C = np.meshgrid(a, a, c, indexing="ij")
        W = np.einsum("i,j,k->ijk", wa, wa, wc).ravel() / 4.0
        A, B, C = A.ravel(), B.ravel(), C.ravel()
        r = (1 + A) * (1 - C) / 2 - 1
        s = (1 + B) * (1 - C) / 2 - 1
        return np.stack([r, s, C], axis=1), W


def make_element(t, N, lobatto=False):
    """Reference element of type t (0 hex, 1 wedge, 2 pyramid, 3 tet)."""
    if t == 0:
        return Hex(N, lobatto)
    if t == 1:
        return Wedge(N)
    if t == 2:
        return Pyramid(N)
    return Tet(N)
