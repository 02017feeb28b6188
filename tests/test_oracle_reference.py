"""Pins of the oracle's rules, bases and reference operators (CPU only).

Each test checks the oracle against something it does not compute itself:
closed-form integrals, the paper's printed tables (tests/golden), closed-form
trace constants (Appendix A), or brute-force integration of the definition.
"""
import math
import os

import numpy as np
import pytest

from oracle.constants import markov_constant, trace_constant
from oracle.elements import Hex, Pyramid, Tet, Wedge, quad_face_rule, tri_face_rule
from oracle.jacobi import (gauss_jacobi, gauss_lobatto, jacobi_p, lagrange_1d,
                           lagrange_1d_deriv)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
TYPES = {"hex": 0, "wedge": 1, "pyramid": 2, "tet": 3}


def read_table(name):
    rows = {}
    for line in open(os.path.join(GOLDEN, name)):
        if line.startswith("#") or not line.strip():
            continue
        parts = line.split()
        rows[parts[0]] = [float(v) for v in parts[1:]]
    return rows


# ------------------------------------------------------------------ 1D rules
def beta_moment(k, a, b):
    """int_{-1}^{1} x^k (1-x)^a (1+x)^b dx, exactly in rationals (integer a, b).

    Expands x^k = sum_j C(k,j) (1+x)^j (-1)^(k-j) and uses
    int (1-x)^a (1+x)^(b+j) = 2^(a+b+j+1) a! (b+j)! / (a+b+j+1)!.
    """
    from fractions import Fraction
    tot = Fraction(0)
    for j in range(k + 1):
        c = math.comb(k, j) * (-1) ** (k - j)
        tot += c * Fraction(2 ** (a + b + j + 1) * math.factorial(a) * math.factorial(b + j),
                            math.factorial(a + b + j + 1))
    return float(tot)


@pytest.mark.parametrize("ab", [(0, 0), (1, 0), (2, 0), (1, 1), (3, 0)])
@pytest.mark.parametrize("n", [1, 2, 5, 9])
def test_gauss_jacobi_exactness(n, ab):
    x, w = gauss_jacobi(n, *ab)
    for k in range(2 * n):
        assert abs(np.sum(w * x ** k) - beta_moment(k, *ab)) < 1e-12 * max(1.0, abs(beta_moment(k, *ab)))
    # degree 2n is not integrated exactly (rules the wrong point count out)
    assert abs(np.sum(w * x ** (2 * n)) - beta_moment(2 * n, *ab)) > 1e-10


@pytest.mark.parametrize("n", [2, 3, 5, 8])
def test_gauss_lobatto(n):
    x, w = gauss_lobatto(n)
    assert x[0] == -1.0 and x[-1] == 1.0
    for k in range(2 * n - 2):
        assert abs(np.sum(w * x ** k) - beta_moment(k, 0, 0)) < 1e-12
    # endpoint weights 2/(N(N+1)) for N+1 points (Appendix A, SEM lemma)
    N = n - 1
    assert abs(w[0] - 2.0 / (N * (N + 1))) < 1e-13


@pytest.mark.parametrize("N", [1, 3, 5])
def test_triangle_and_quad_face_rules(N):
    pts, w = tri_face_rule(N)
    l1, l2 = (1 + pts[:, 0]) / 2, (1 + pts[:, 1]) / 2
    for a in range(2 * N + 2):
        for b in range(2 * N + 2 - a):
            exact = 4.0 * math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
            assert abs(np.sum(w * l1 ** a * l2 ** b) - exact) < 1e-13
    qp, qw = quad_face_rule(N)
    assert abs(qw.sum() - 4.0) < 1e-13
    assert abs(np.sum(qw * qp[:, 0] ** (2 * N) * qp[:, 1] ** (2 * N)) - (2 / (2 * N + 1)) ** 2) < 1e-13


def test_jacobi_endpoint_and_orthogonality():
    for n, a in [(3, 5.0), (4, 7.0), (2, 3.0)]:
        assert abs(jacobi_p(n, a, 0, 1.0) - math.comb(int(n + a), n)) < 1e-10
        x, w = gauss_jacobi(n + 2, a, 0)
        for m in range(n):
            assert abs(np.sum(w * jacobi_p(n, a, 0, x) * jacobi_p(m, a, 0, x))) < 1e-10


# ------------------------------------------------------------------ trace / Markov constants
@pytest.mark.parametrize("N", range(1, 10))
def test_hex_trace_constants_closed_form(N):
    """C_T = 3(N+1)(N+2)/2 (GL) and C_SEM = 3N(N+1)/2 (Sec. 3.2, Appendix A)."""
    assert abs(trace_constant(0, N) - 3 * (N + 1) * (N + 2) / 2) < 1e-9
    assert abs(trace_constant(0, N, lobatto=True) - 3 * N * (N + 1) / 2) < 1e-9


@pytest.mark.parametrize("name", ["hex", "wedge", "pyramid", "tet"])
def test_trace_constants_table(name):
    """Table computedTrace: pins the hex (its printed row is 3(N+1)(N+2)/2), wedge, pyramid
    (rational B_N) and tet spaces."""
    tab = read_table("trace_constants.txt")[name]
    for N in range(1, 10):
        assert abs(trace_constant(TYPES[name], N) - tab[N - 1]) < 0.006, (name, N)


@pytest.mark.parametrize("name", ["hex", "wedge", "pyramid"])
def test_sem_trace_constants_table(name):
    """Table computedTraceSEM: GLL nodes for the hexahedron and GLL points on every quadrilateral
    face (also those of wedges and pyramids) reproduce the printed SEM constants."""
    tab = read_table("trace_constants_sem.txt")[name]
    for N in range(1, 10):
        assert abs(trace_constant(TYPES[name], N, lobatto=True) - tab[N - 1]) < 0.006 * max(1, tab[N - 1] / 100), (name, N)


@pytest.mark.parametrize("name", ["wedge", "pyramid", "tet"])
def test_markov_constants_table(name):
    """Table markovConsts: pins the reference gradients of each basis."""
    tab = read_table("markov_constants.txt")[name]
    for N in range(1, 10):
        assert abs(markov_constant(TYPES[name], N) - tab[N - 1]) < 0.006 * max(1, tab[N - 1] / 100), (name, N)


def test_markov_constants_table_hex_sem():
    """Table markovConsts, hexahedron row (N = 1..9): the SEM hexahedron's constant, its mass and
    stiffness both in the GLL quadrature of its nodes.  The same Q_N space in the exact L2 inner
    product gives other values (9, 45, 127.6 at N = 1..3), so the row pins that reading."""
    tab = read_table("markov_constants.txt")["hex"]
    for N in range(1, 10):
        assert abs(markov_constant(0, N, lobatto=True) - tab[N - 1]) < 0.006 * max(1, tab[N - 1] / 100), N
    assert abs(markov_constant(0, 1) - 9.0) < 1e-9 and abs(markov_constant(0, 2) - 45.0) < 1e-9


def test_trace_constant_needs_euclidean_face_measure():
    """With unit-area faces the tet value would differ from the table (documents the reading)."""
    assert abs(trace_constant(3, 1, measure="unit") - 12.22) > 1.0


# ------------------------------------------------------------------ mass matrices (Sec. 2.1)
def perturbed(el, seed, amp=0.15):
    rng = np.random.default_rng(seed)
    return el.verts * 0.4 + amp * 0.4 * rng.uniform(-1, 1, el.verts.shape) + 0.1


@pytest.mark.parametrize("N", [1, 3, 4])
def test_hex_gl_mass_is_diagonal(N):
    """Sec. 2.1.1: with J in Q_1 the GL-collocated mass diag(w J) is the exact mass.

    Holds on affine hexes; on a general trilinear hex J is quadratic per direction
    and diag(w J) is the (N+1)-point GL quadrature of the mass (still used, as in
    the paper's kernels), so there the off-diagonal entries are small but not zero.
    """
    hx = Hex(N)
    rng = np.random.default_rng(1)
    A = 0.4 * np.eye(3) + 0.05 * rng.uniform(-1, 1, (3, 3))
    for xv, exact in ((hx.verts @ A.T + 0.1, True), (perturbed(hx, 1), False)):
        P, W = hx.exact_rule(N + 3)
        _, F = hx.vmap(xv, P)
        B = hx.basis(P)
        M = B.T @ ((W * np.linalg.det(F))[:, None] * B)
        _, Fn = hx.vmap(xv, hx.nodes)
        err = np.abs(M - np.diag(hx.wnodes * np.linalg.det(Fn))).max() / np.abs(M).max()
        assert (err < 1e-13) if exact else (1e-9 < err < 1e-2)


@pytest.mark.parametrize("N", [1, 3, 4])
def test_pyramid_mass_is_diagonal_J_at_seminodal_points(N):
    """Sec. 2.1.4: the mapped mass matrix is diag(J(a^k_i, b^k_j))."""
    py = Pyramid(N)
    xv = perturbed(py, 2)
    P, W = py.exact_rule(N + 3)
    _, F = py.vmap(xv, P)
    B = py.basis(P)
    M = B.T @ ((W * np.linalg.det(F))[:, None] * B)
    rst = np.stack([(py.ab[:, 0] - 1) / 2, (py.ab[:, 1] - 1) / 2, np.zeros(py.Np)], axis=1)
    _, Fn = py.vmap(xv, rst)
    assert np.allclose(M, np.diag(np.linalg.det(Fn)), atol=1e-12 * np.abs(M).max())


@pytest.mark.parametrize("N", [1, 3])
def test_wedge_lsc_mass_is_identity(N):
    """Sec. 2.1.3: int (phi_i/sqrt J)(phi_j/sqrt J) J = delta_ij for every vertex-mapped wedge."""
    wd = Wedge(N)
    xv = perturbed(wd, 3)
    P, W = wd.exact_rule(N + 3)
    B = wd.basis(P)
    M = B.T @ (W[:, None] * B)
    assert np.allclose(M, np.eye(wd.Np), atol=1e-12)


@pytest.mark.parametrize("N", [1, 2, 4])
def test_tet_nodal_derivatives_exact(N):
    tt = Tet(N)
    D = tt.grad(tt.nodes)
    r, s, t = tt.nodes.T
    for a in range(N + 1):
        for b in range(N + 1 - a):
            for c in range(N + 1 - a - b):
                f = r ** a * s ** b * t ** c
                fr = a * r ** max(a - 1, 0) * s ** b * t ** c
                ft = c * r ** a * s ** b * t ** max(c - 1, 0)
                assert np.allclose(D[0] @ f, fr, atol=1e-11)
                assert np.allclose(D[2] @ f, ft, atol=1e-11)


def test_hex_face_interpolation_symmetry():
    """GL symmetry used by Alg. hex_upd: ell_k(1) = ell_{N-k}(-1)."""
    for N in range(1, 10):
        hx = Hex(N)
        vm = lagrange_1d(hx.r1, -1.0)[0]
        vp = lagrange_1d(hx.r1, 1.0)[0]
        assert np.allclose(vp, vm[::-1], atol=1e-13)


# ------------------------------------------------------------------ pyramid operators (Sec. 2.3.4)
def pyramid_operators_quadrature_free(py, test_node=True):
    """D^r, D^s, D^t assembled from the paper's quadrature-free formulas.

    D^r_{lmn,ijk} = sqrt(w^n_l w^n_m / (w^k_i w^k_j)) l^k_i'(a^n_l) l^k_j(b^n_m) M^c_{nk},
    M^c_{nk} = int P^{(2k+3)}_{N-k} P^{(2n+3)}_{N-n} ((1-c)/2)^{1+k+n} / sqrt(g_n g_k),
    D^c with the c-derivative integral, D^t = diag((1+a)/2) D^r + diag((1+b)/2) D^s + D^c,
    the factor (1+a)/2 taken at the test node (test_node=True) or the trial node.
    """
    N = py.N
    c, wc = gauss_jacobi(2 * N + 4, 0, 0)
    h = (1 - c) / 2
    Pk = [jacobi_p(N - k, 2 * k + 3, 0, c) for k in range(N + 1)]
    dPk = [0.5 * (N - k + 2 * k + 4) * jacobi_p(N - k - 1, 2 * k + 4, 1, c) if N > k else 0 * c
           for k in range(N + 1)]
    g = py.gamma
    Mc = np.array([[np.sum(wc * Pk[k] * Pk[n] * h ** (1 + k + n)) / np.sqrt(g[n] * g[k])
                    for k in range(N + 1)] for n in range(N + 1)])
    Cc = np.zeros((N + 1, N + 1))
    for n in range(N + 1):
        for k in range(N + 1):
            dk = dPk[k] * h ** k - (k / 2.0) * (h ** (k - 1) if k > 0 else 0 * c) * Pk[k]
            Cc[n, k] = np.sum(wc * dk * Pk[n] * h ** (2 + n)) / np.sqrt(g[n] * g[k])
    Dr = np.zeros((py.Np, py.Np))
    Ds, Dc = np.zeros_like(Dr), np.zeros_like(Dr)
    for row, (l, m, n) in enumerate(py.modes):
        an, wn = py.levels[n]
        for col, (i, j, k) in enumerate(py.modes):
            ak, wk = py.levels[k]
            fac = np.sqrt(wn[l] * wn[m] / (wk[i] * wk[j]))
            la = lagrange_1d(ak, an[l])[0, i]
            lb = lagrange_1d(ak, an[m])[0, j]
            dla = lagrange_1d_deriv(ak, an[l])[0, i]
            dlb = lagrange_1d_deriv(ak, an[m])[0, j]
            Dr[row, col] = fac * dla * lb * Mc[n, k]
            Ds[row, col] = fac * la * dlb * Mc[n, k]
            Dc[row, col] = fac * la * lb * Cc[n, k]
    if test_node:
        A = (1 + py.ab[:, 0]) / 2
        B = (1 + py.ab[:, 1]) / 2
        Dt = A[:, None] * Dr + B[:, None] * Ds + Dc
    else:
        A = (1 + py.ab[:, 0]) / 2
        B = (1 + py.ab[:, 1]) / 2
        Dt = Dr * A[None, :] + Ds * B[None, :] + Dc
    return np.stack([Dr, Ds, Dt])


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_pyramid_operators_match_quadrature_free_formula(N):
    from oracle.dg import DGOracle
    py = Pyramid(N)
    D = DGOracle.pyramid_operators(py)
    Dq = pyramid_operators_quadrature_free(py, test_node=True)
    assert np.allclose(D, Dq, atol=1e-12), np.abs(D - Dq).max()
    if N >= 2:   # the trial-node reading of the (1+a)/2 factor is not the weak derivative
        assert np.abs(D[2] - pyramid_operators_quadrature_free(py, test_node=False)[2]).max() > 1e-6


@pytest.mark.parametrize("N", [1, 2, 4])
def test_pyramid_weak_derivative_of_polynomials(N):
    """For u in P_N(r,s,t): D^a c(u) = c(d u/d r_a), with c(.) = coefficients (M = I)."""
    from oracle.dg import DGOracle
    py = Pyramid(N)
    D = DGOracle.pyramid_operators(py)
    P, W = py.exact_rule(N + 3)
    B = py.basis(P)
    r, s, t = P.T
    for (a, b, cc) in [(1, 0, 0), (0, 1, 0), (0, 0, 1), (N, 0, 0), (1, 1, N - 2 if N >= 2 else 0)]:
        if a + b + cc > N:
            continue
        u = r ** a * s ** b * t ** cc
        du = [a * r ** max(a - 1, 0) * s ** b * t ** cc,
              b * r ** a * s ** max(b - 1, 0) * t ** cc,
              cc * r ** a * s ** b * t ** max(cc - 1, 0)]
        coef = B.T @ (W * u)
        for d in range(3):
            assert np.allclose(D[d] @ coef, B.T @ (W * du[d]), atol=1e-11)
