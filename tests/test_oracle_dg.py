"""Pins of the oracle's discrete operator, time stepper and time step (CPU only)."""
import numpy as np
import pytest

from oracle.constants import trace_constant
from oracle.dg import LSRK_A, LSRK_B, LSRK_C, DGOracle, standing_mode
from paper_1507_02557_b300.inputs import layered_mesh, random_state, small_hybrid_mesh


@pytest.fixture(scope="module")
def mesh():
    return small_hybrid_mesh()


@pytest.fixture(scope="module")
def mesh_c():
    """Small hybrid mesh with a wave-speed jump between layers (c = 1, 1.5 by parity)."""
    return layered_mesh(3, 3, 5, "HWHTK", seed=3, c_of_layer=lambda k: 1.0 if k % 2 == 0 else 1.5)


def energy_rate(dg, q):
    return float(np.sum(q * dg.mass_apply(dg.rhs(q)) * dg.material_weights()))


@pytest.fixture(scope="module")
def mesh_affine_c():
    """Undisplaced (affine) hybrid mesh with a wave-speed jump: the SEM hexahedron's GLL
    collocation integrates its (constant) metric terms exactly there."""
    return layered_mesh(3, 3, 5, "HWHTK", seed=3, amp=0.0, c_of_layer=lambda k: 1.0 if k % 2 == 0 else 1.5)


@pytest.mark.parametrize("N", [1, 2, 3])
@pytest.mark.parametrize("which,hex_basis", [("mesh", "gl"), ("mesh_c", "gl"), ("mesh_affine_c", "gll")])
def test_energy_identity(N, which, hex_basis, request):
    """Eq. (sym): U^T A U = 0 for central flux and = -1/2 sum int (tau_p[p]^2 + tau_u[u_n]^2) for
    upwind.  SEM hexahedra (GLL collocation, GLL points on every quad face) satisfy it exactly on
    affine hexahedra; on trilinear ones the GLL rule (exact to 2N-1) misses the metric terms."""
    m = request.getfixturevalue(which)
    for ts in (0.0, 1.0):
        dg = DGOracle(m, N, tau_scale=ts, hex_basis=hex_basis)
        q = random_state(dg.ndof, 7)
        rate = energy_rate(dg, q)
        diss = dg.jump_dissipation(q)
        scale = float(np.sum(q * dg.mass_apply(q)))
        assert abs(rate - diss) < 1e-12 * scale, (ts, rate, diss)
        if ts == 0.0:
            assert abs(rate) < 1e-12 * scale
        else:
            assert diss < 0


@pytest.mark.parametrize("N", [1, 3])
def test_pyramid_strong_and_skew_forms_agree(mesh, N):
    """Sec. 2.2: with GL quadrature on the quadrilateral face the strong and skew-symmetric
    pyramid forms are equivalent.  The cofactors J dr/dx are bilinear in (a,b) for a
    vertex-mapped pyramid, so collocating them at the semi-nodal points keeps it exact."""
    a = DGOracle(mesh, N, pyr_form="skew")
    b = DGOracle(mesh, N, pyr_form="strong")
    q = random_state(a.ndof, 3)
    ra, rb = a.split(a.rhs(q))[2], b.split(b.rhs(q))[2]
    assert np.abs(ra - rb).max() < 1e-12 * np.abs(ra).max()


def test_lsrk_order_conditions():
    """LSRK(5,4) applied to y' = z y gives R(z) with Taylor coefficients 1, 1, 1/2, 1/6, 1/24."""
    poly = np.polynomial.polynomial
    y = np.array([1.0])
    res = np.array([0.0])
    for a, b in zip(LSRK_A, LSRK_B):
        res = poly.polyadd(a * res, poly.polymul([0.0, 1.0], y))
        y = poly.polyadd(y, b * res)
    assert np.allclose(y[:5], [1, 1, 1 / 2, 1 / 6, 1 / 24], atol=1e-10)
    # stage times: y' = t^m integrates exactly for m <= 3
    for m in range(4):
        yy, rr = 0.0, 0.0
        for a, b, c in zip(LSRK_A, LSRK_B, LSRK_C):
            rr = a * rr + c ** m
            yy += b * rr
        assert abs(yy - 1.0 / (m + 1)) < 1e-10   # published rationals hold to ~1e-12


def test_faces_conform_and_walls_on_cube(mesh):
    dg = DGOracle(mesh, 3)
    sides = dg.geo.sides
    nb = 0
    for s in sides:
        xv = mesh.xyz[mesh.conn[s.t][s.e]]
        x, F = dg.els[s.t].vmap(xv, s.rst)
        assert np.all(np.linalg.det(F) > 0)
        if s.nbr >= 0:
            o = sides[s.nbr]
            xo, _ = dg.els[o.t].vmap(mesh.xyz[mesh.conn[o.t][o.e]], o.rst)
            assert np.abs(x - xo).max() < 1e-13
            assert np.abs(s.n + o.n).max() < 1e-12
            assert np.abs(s.Js - o.Js).max() < 1e-13
        else:
            nb += 1
            assert np.all(np.min(np.abs(np.abs(x) - 1.0), axis=1) < 1e-13)
    # 4x4x5 cells: 2*16 + 4*20 wall quads/triangle pairs
    assert nb > 0


@pytest.mark.parametrize("N,hex_basis", [(1, "gl"), (3, "gl"), (2, "gll"), (3, "gll")])
def test_linear_fields_are_reproduced(N, hex_basis):
    """Continuous linear fields: zero jumps, and -div u, -grad p exact at interior elements.

    Affine mesh (amp = 0), so that the LSC wedge space contains the linear fields.  SEM: from
    N = 2 on, the GLL-lumped projection of a linear field is its interpolant.
    """
    m = layered_mesh(3, 3, 5, "HWHTK", seed=0, amp=0.0)
    dg = DGOracle(m, N, hex_basis=hex_basis)
    f = lambda x, t: np.stack([1 + 2 * x[:, 0] - x[:, 1] + 0.5 * x[:, 2],
                               0.3 * x[:, 0], -0.7 * x[:, 1] + 0.1, 0.2 * x[:, 2] + 0.4 * x[:, 0]])
    q = dg.project(f)
    r = dg.rhs(q)
    exact = lambda x, t: np.stack([np.full(len(x), -(0.3 - 0.7 + 0.2)),
                                   np.full(len(x), -2.0), np.full(len(x), 1.0), np.full(len(x), -0.5)])
    want = dg.project(exact)
    inner = np.ones((4, dg.ndof), bool)
    rv = dg.split(inner)
    for s in dg.geo.sides:
        if s.nbr < 0:
            rv[s.t][:, s.e] = False
    assert np.abs(r - want)[inner].max() < 1e-10


def assemble(dg):
    n = 4 * dg.ndof
    A = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        A[:, j] = dg.rhs(e.reshape(4, -1)).ravel()
    return A


@pytest.mark.parametrize("N", [1, 2])
def test_spectral_radius_below_trace_bound(N):
    """Eq. (bnd_re), (dtK): rho(M^{-1}A) <= max_K C^K C_T(N) C_J^K, and LSRK(5,4) is stable at
    the paper's dt (C = 0.5) for every eigenvalue of the assembled operator."""
    m = layered_mesh(2, 2, 5, "HWHTK", seed=1)
    dg = DGOracle(m, N)
    lam = np.linalg.eigvals(assemble(dg))
    CT = [trace_constant(t, N) for t in range(4)]
    bound = 1.0 / dg.global_dt(CT, cfl=1.0)
    rho = np.abs(lam).max()
    assert rho <= bound
    assert np.max(lam.real) < 1e-9
    dt = dg.global_dt(CT, cfl=0.5)
    z = lam * dt
    R = np.ones_like(z)
    res = np.zeros_like(z)
    y = np.ones_like(z)
    for a, b in zip(LSRK_A, LSRK_B):
        res = a * res + z * y
        y = y + b * res
    assert np.abs(y).max() <= 1.0 + 1e-12


def test_convergence_to_standing_mode():
    """GL formulation on refined hybrid meshes: L2 error rate >= N + 1/2 (Sec. 4.1-4.2)."""
    N = 1
    errs = []
    for mlev in (1, 2):
        L = "H" * mlev + "W" * mlev + "H" * mlev + "T" + "K" * mlev
        m = layered_mesh(2 * mlev, 2 * mlev, len(L), L, seed=0)
        dg = DGOracle(m, N)
        CT = [trace_constant(t, N) for t in range(4)]
        T = 0.1
        nst = int(np.ceil(T / dg.global_dt(CT)))
        q = dg.project(standing_mode, 0.0)
        for _ in range(nst):
            q = dg.lsrk_step(q, T / nst)
        errs.append(dg.l2_error(q, standing_mode, T))
    assert np.log2(errs[0] / errs[1]) > N + 0.5


def test_mrab3_is_third_order():
    """Two-level MRAB3 (Sec. 2.4 reading): halving the fine step divides the error by ~8."""
    from oracle.dg import MRAB3, mr_levels
    m = layered_mesh(3, 3, 5, "HWHTK", seed=3, c_of_layer=lambda k: 1.0 if k % 2 == 0 else 1.5)
    N = 2
    o = DGOracle(m, N)
    lev, dmin = mr_levels(o, [trace_constant(t, N) for t in range(4)], 2)
    assert sum(int(np.sum(l == 2)) for l in lev) > 0 and sum(int(np.sum(l == 1)) for l in lev) > 0
    q0 = o.project(standing_mode, 0.0)
    errs = []
    for h in (dmin, dmin / 2):
        mr = MRAB3(o, lev)
        q, hist = mr.start(q0, h)
        nsteps = int(round((0.06 - 4 * h) / (2 * h)))
        for _ in range(nsteps):
            q, hist = mr.step(q, hist, h)
        T = 4 * h + 2 * h * nsteps
        nref = int(np.ceil(T / (dmin / 4)))
        qr = q0.copy()
        for _ in range(nref):
            qr = o.lsrk_step(qr, T / nref)
        errs.append(np.linalg.norm(q - qr) / np.linalg.norm(qr))
    assert 6.0 < errs[0] / errs[1] < 11.0, errs


@pytest.mark.parametrize("level", [1, 2])
def test_mrab3_on_one_level_is_single_rate_ab3(mesh, level):
    """Sec. 2.4 reading: with every element on one level the multi-rate scheme is plain
    Adams-Bashforth 3 (coefficients 23/12, -16/12, 5/12 from integrating the quadratic through the
    last three rhs values): all coarse, one AB3 step of 2h per coarse step; all fine, two AB3 steps
    of h.  The start-up history (LSRK steps, rhs at 0, 2h, 3h) is the one AB3 needs at 4h."""
    from oracle.dg import MRAB3
    N = 2
    o = DGOracle(mesh, N)
    lev = [np.full(k, level, dtype=int) for k in o.K]
    q0 = random_state(o.ndof, 9)
    h = 1e-3
    mr = MRAB3(o, lev)
    q, hist = mr.start(q0, h)
    for _ in range(3):
        q, hist = mr.step(q, hist, h)
    # plain AB3 from the same start-up
    qa = q0.copy()
    rs = {}
    for k in range(4):
        if k in (0, 2, 3):
            rs[k] = o.rhs(qa)
        qa = o.lsrk_step(qa, h)
    H = 2 * h if level == 1 else h
    hist_a = [rs[2], rs[0]] if level == 1 else [rs[3], rs[2]]
    for _ in range(3 if level == 1 else 6):
        r = o.rhs(qa)
        qa = qa + H * (23 * r - 16 * hist_a[0] + 5 * hist_a[1]) / 12
        hist_a = [r, hist_a[0]]
    assert np.abs(q - qa).max() < 1e-13 * np.abs(qa).max()


def _two_level(N=2):
    from oracle.dg import mr_levels
    m = layered_mesh(3, 3, 5, "HWHTK", seed=3, c_of_layer=lambda k: 1.0 if k % 2 == 0 else 1.5)
    o = DGOracle(m, N)
    lev, dmin = mr_levels(o, [trace_constant(t, N) for t in range(4)], 2)
    return o, lev, dmin


@pytest.mark.parametrize("level", [1, 2])
def test_mrlsrk_on_one_level_is_lsrk(level):
    """Multi-rate LSRK with every element coarse is one LSRK(5,4) step of 2h (the coarse
    polynomial integrates to R(2h B) y); with every element fine it is two LSRK(5,4) steps of h."""
    from oracle.dg import MRLSRK
    o, _, dmin = _two_level()
    lev = [np.full(k, level, dtype=int) for k in o.K]
    y = random_state(o.ndof, 12)
    got = MRLSRK(o, lev).step(y, dmin)
    want = o.lsrk_step(y, 2 * dmin) if level == 1 else o.lsrk_step(o.lsrk_step(y, dmin), dmin)
    assert np.abs(got - want).max() < 1e-12 * np.abs(want).max()


def test_mrlsrk_is_fourth_order():
    """Two levels (fine pyramids, tets and wedges next to coarse hexahedra): halving h divides the
    error against a small-step LSRK(5,4) reference by about 16."""
    from oracle.dg import MRLSRK
    o, lev, dmin = _two_level()
    q0 = o.project(standing_mode, 0.0)
    T = 16 * dmin
    errs = []
    for h in (dmin, dmin / 2):
        mr = MRLSRK(o, lev)
        q = q0.copy()
        for _ in range(int(round(T / (2 * h)))):
            q = mr.step(q, h)
        errs.append(q)
    ref = q0.copy()
    for _ in range(64):
        ref = o.lsrk_step(ref, T / 64)
    e = [np.linalg.norm(x - ref) / np.linalg.norm(ref) for x in errs]
    assert 12.0 < e[0] / e[1] < 22.0, e


def test_mrlsrk_energy_nonincreasing_under_upwind():
    """Upwind flux, two levels at the multi-rate step: the discrete energy does not grow."""
    from oracle.dg import MRLSRK
    o, lev, dmin = _two_level()
    mr = MRLSRK(o, lev)
    q = random_state(o.ndof, 3)
    E = [o.energy(q)]
    for _ in range(6):
        q = mr.step(q, dmin)
        E.append(o.energy(q))
    assert all(b <= a * (1 + 1e-12) for a, b in zip(E, E[1:])), E


@pytest.mark.parametrize("N", [3, 4])
def test_tet_results_do_not_depend_on_the_node_set(monkeypatch, N):
    """Reading of Sec. 2.1.2 (the paper's optimised tet nodes are not tabulated): the tet volume
    term is the exact derivative of the nodal interpolant and the faces are integrated exactly, so
    the rhs as a polynomial does not depend on where the nodes sit.  Moving every non-vertex node
    of the equispaced lattice (a different unisolvent set) and interpolating the same state gives
    the same rhs polynomial to rounding; the other element types are untouched.  (The oracle takes
    tet traces by evaluating the basis at the face points, so face nodes may move off the face.)"""
    import oracle.elements as E
    m = small_hybrid_mesh()
    oa = DGOracle(m, N)
    tet_a = oa.els[3]
    orig_init = E.Tet.__init__

    def moved_init(self, n):
        orig_init(self, n)
        rng = np.random.default_rng(n)
        vert = np.array([any(np.allclose(x, v) for v in self.verts) for x in self.nodes])
        shift = 0.1 * rng.uniform(-1, 1, self.nodes.shape) / n
        self.nodes = np.where(vert[:, None], self.nodes, self.nodes + shift)
        self.Vinv = np.linalg.inv(self._modal(self.nodes))

    monkeypatch.setattr(E.Tet, "__init__", moved_init)
    ob = DGOracle(m, N)
    tet_b = ob.els[3]
    assert np.abs(tet_b.nodes - tet_a.nodes).max() > 1e-3
    T = tet_a.basis(tet_b.nodes)                     # nodal values in set A -> values at set B's nodes
    qa = random_state(oa.ndof, 4)
    qb = qa.copy()
    lo, K, npn = oa.off[3], oa.K[3], oa.Np[3]
    sl = slice(lo, lo + K * npn)
    qb[:, sl] = np.einsum("bn,fkn->fkb", T, qa[:, sl].reshape(4, K, npn)).reshape(4, -1)
    ra, rb = oa.rhs(qa), ob.rhs(qb)
    ra_at_b = ra.copy()
    ra_at_b[:, sl] = np.einsum("bn,fkn->fkb", T, ra[:, sl].reshape(4, K, npn)).reshape(4, -1)
    assert np.abs(rb - ra_at_b).max() < 1e-11 * np.abs(ra).max()   # measured 3e-15, 3e-14
    # control: the moved set read as if it were the lattice gives another rhs
    assert np.abs(ob.rhs(qa) - ra).max() > 1e-3 * np.abs(ra).max()
