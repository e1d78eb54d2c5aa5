"""Pins of the CPU oracle against what the mathematics fixes (no GPU needed).

Each test checks the oracle against something other than itself: closed forms,
structural facts the paper states (D square, D diagonal for dual LMs, Sec. 2.2),
exact special cases, brute force, or finite differences.
"""
import math

import numpy as np
import pytest

from paper_2202_03933_gb300 import inputs


# ---------------------------------------------------------------- helpers
def mass1d(n, h):
    """Consistent 1D linear mass matrix on a uniform grid: (h/6) tridiag(1,4,1), ends 2."""
    M = np.zeros((n + 1, n + 1))
    for e in range(n):
        M[e:e + 2, e:e + 2] += (h / 6.0) * np.array([[2.0, 1.0], [1.0, 2.0]])
    return M


def mortar1d(xs_nodes, xm_nodes, dual=False):
    """Exact 1D mortar matrix int Phi_i N_k between two 1D grids.

    On every sub-interval of the merged grid the integrand is a product of two
    linear functions; Simpson's rule integrates it exactly.
    """
    ns, nm = len(xs_nodes), len(xm_nodes)
    M = np.zeros((ns, nm))
    cuts = np.unique(np.concatenate([xs_nodes, xm_nodes]))
    lo = max(xs_nodes[0], xm_nodes[0])
    hi = min(xs_nodes[-1], xm_nodes[-1])
    cuts = cuts[(cuts >= lo) & (cuts <= hi)]

    def hats(nodes, x):
        e = min(np.searchsorted(nodes, x, side="right") - 1, len(nodes) - 2)
        t = (x - nodes[e]) / (nodes[e + 1] - nodes[e])
        return e, np.array([1.0 - t, t])

    for a, b in zip(cuts[:-1], cuts[1:]):
        mid = 0.5 * (a + b)
        es, _ = hats(xs_nodes, mid)
        em, _ = hats(xm_nodes, mid)
        for x, w in ((a, 1.0), (mid, 4.0), (b, 1.0)):
            ts = (x - xs_nodes[es]) / (xs_nodes[es + 1] - xs_nodes[es])
            tm = (x - xm_nodes[em]) / (xm_nodes[em + 1] - xm_nodes[em])
            Ns = np.array([1.0 - ts, ts])
            Nm = np.array([1.0 - tm, tm])
            Phi = np.array([2 * Ns[0] - Ns[1], 2 * Ns[1] - Ns[0]]) if dual else Ns
            M[es:es + 2, em:em + 2] += (b - a) / 6.0 * w * np.outer(Phi, Nm)
    return M


def rel(a, b):
    a = np.asarray(a.todense() if hasattr(a, "todense") else a)
    b = np.asarray(b.todense() if hasattr(b, "todense") else b)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def dense(A):
    return np.asarray(A.todense())


# ---------------------------------------------------------------- inputs
def test_golden_paper_interface_sizes():
    """The structured generator reproduces the paper's slave interface sizes."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_interface_sizes.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 5
    for r in rows:
        n, nodes, elems = int(r[0]), int(r[1]), int(r[2])
        assert inputs.grid_nodes(n, n).shape[0] == nodes
        assert inputs.grid_quad4(n, n).shape[0] == elems


def test_generator_is_counter_based_and_seeded():
    a = inputs.uniform01(123, 0, 1000)
    b = inputs.uniform01(123, 0, 2000)[:1000]
    assert np.array_equal(a, b)
    assert not np.array_equal(a, inputs.uniform01(124, 0, 1000))
    assert a.min() >= 0 and a.max() < 1 and abs(a.mean() - 0.5) < 0.05
    # SplitMix64 reference value: state 0 advanced once gives 0xE220A8397B1DCDAF
    z = inputs._mix64(np.array([0x9E3779B97F4A7C15], dtype=np.uint64))
    assert int(z[0]) == 0xE220A8397B1DCDAF


# ---------------------------------------------------------------- rules
def test_tri7_rule_degree5_exact(orc):
    r = orc.tri_rule(7)
    assert r.shape == (7, 4)
    assert abs(r[:, 3].sum() - 1.0) < 1e-15
    for i in range(7):
        for j in range(7 - i):
            exact = math.factorial(i) * math.factorial(j) / math.factorial(i + j + 2)
            q = 0.5 * np.sum(r[:, 3] * r[:, 1] ** i * r[:, 2] ** j)
            if i + j <= 5:
                assert abs(q - exact) < 1e-15, (i, j)
    # not exact at degree 6 (it is a degree-5 rule)
    q6 = 0.5 * np.sum(r[:, 3] * r[:, 1] ** 6)
    assert abs(q6 - math.factorial(6) / math.factorial(8)) > 1e-8


def test_duffy_rule_degree8_exact(orc):
    r = orc.tri_rule(25)
    assert r.shape == (25, 4)
    for i in range(9):
        for j in range(9 - i):
            exact = math.factorial(i) * math.factorial(j) / math.factorial(i + j + 2)
            q = 0.5 * np.sum(r[:, 3] * r[:, 1] ** i * r[:, 2] ** j)
            assert abs(q - exact) < 1e-15 * max(1, 1 / exact) ** 0.5 + 1e-16, (i, j)


# ---------------------------------------------------------------- dual basis
def _single_element(X, nen):
    conn = np.arange(nen, dtype=np.int32)[None, :]
    return inputs.Interface("one", np.asarray(X, float), conn, nen, np.asarray(X, float), conn, nen)


def test_dual_closed_form_parallelogram(orc):
    X = [[0, 0, 0], [2.0, 0.3, 0], [2.5, 1.3, 0], [0.5, 1.0, 0]]
    A, De = orc.element_blocks(_single_element(X, 4), lm=1)
    expect = np.array([[4, -2, 1, -2], [-2, 4, -2, 1], [1, -2, 4, -2], [-2, 1, -2, 4]], float)
    assert np.abs(A[0] - expect).max() < 1e-13
    area = abs(np.cross(np.subtract(X[1], X[0]), np.subtract(X[3], X[0]))[2])
    assert np.abs(De[0] - np.diag([area / 4] * 4)).max() < 1e-14 * area


def test_dual_closed_form_triangle(orc):
    X = [[0, 0, 0], [1.5, 0.2, 0.1], [0.3, 0.9, -0.2]]
    A, De = orc.element_blocks(_single_element(X, 3), lm=1)
    expect = np.array([[3, -1, -1], [-1, 3, -1], [-1, -1, 3]], float)
    assert np.abs(A[0][:3, :3] - expect).max() < 1e-13
    area = 0.5 * np.linalg.norm(np.cross(np.subtract(X[1], X[0]), np.subtract(X[2], X[0])))
    assert np.abs(De[0][:3, :3] - np.diag([area / 3] * 3)).max() < 1e-14 * area


def _bilinear_moments(X, ng=12):
    """int N_a N_b |x_xi x x_eta| and int N_a |.| by an independent product rule."""
    g, w = np.polynomial.legendre.leggauss(ng)
    X = np.asarray(X, float)
    corners = np.array([[-1, -1], [1, -1], [1, 1], [-1, 1]], float)
    Me = np.zeros((4, 4))
    dh = np.zeros(4)
    for xi, wx in zip(g, w):
        for eta, wy in zip(g, w):
            N = 0.25 * (1 + corners[:, 0] * xi) * (1 + corners[:, 1] * eta)
            dxi = 0.25 * corners[:, 0] * (1 + corners[:, 1] * eta)
            deta = 0.25 * corners[:, 1] * (1 + corners[:, 0] * xi)
            J = np.linalg.norm(np.cross(dxi @ X, deta @ X))
            Me += wx * wy * J * np.outer(N, N)
            dh += wx * wy * J * N
    return Me, dh


def test_dual_biorthogonal_general_quad(orc):
    """int Phi_a N_b = delta_ab int N_b on a warped, non-parallelogram quad."""
    X = [[0, 0, 0], [1.7, -0.2, 0.1], [2.1, 1.4, -0.15], [-0.3, 0.9, 0.05]]
    A, _ = orc.element_blocks(_single_element(X, 4), lm=1)
    Me, dh = _bilinear_moments(X)
    # the 3x3 rule in the oracle is not exact for a warped element's J, so
    # compare against the same biorthogonality up to that rule's error
    B = A[0] @ Me
    assert np.abs(B - np.diag(dh)).max() < 1e-4 * dh.max()
    # for a planar general quad J is bilinear -> 3x3 Gauss is exact
    Xp = [[0, 0, 0], [1.7, -0.2, 0], [2.1, 1.4, 0], [-0.3, 0.9, 0]]
    A, _ = orc.element_blocks(_single_element(Xp, 4), lm=1)
    Me, dh = _bilinear_moments(Xp)
    assert np.abs(A[0] @ Me - np.diag(dh)).max() < 1e-14 * dh.max()
    assert np.abs(A[0] - A[0].T).max() > 1e-3   # genuinely non-symmetric here


# ---------------------------------------------------------------- Newton
def test_newton_backprojection_reproduces_points(orc):
    rng = np.random.default_rng(7)
    corners = np.array([[-1, -1], [1, -1], [1, 1], [-1, 1]], float)
    for _ in range(200):
        p = corners * 0.5 + rng.uniform(-0.12, 0.12, size=(4, 2)) + rng.uniform(-3, 3, 2)
        xi_true = rng.uniform(-1, 1, 2)
        N = 0.25 * (1 + corners[:, 0] * xi_true[0]) * (1 + corners[:, 1] * xi_true[1])
        x = N @ p
        xi, ok = orc.invert_map(p, x)
        assert ok
        Nr = 0.25 * (1 + corners[:, 0] * xi[0]) * (1 + corners[:, 1] * xi[1])
        assert np.abs(Nr @ p - x).max() < 1e-13
        assert np.abs(xi - xi_true).max() < 1e-12
    # triangle: direct solve
    p = np.array([[0.1, 0.2], [1.3, 0.1], [0.4, 1.1]])
    lam = np.array([0.2, 0.5, 0.3])
    xi, ok = orc.invert_map(p, lam @ p)
    assert ok and np.abs(xi - lam[1:]).max() < 1e-14


# ---------------------------------------------------------------- search
@pytest.mark.parametrize("make", [
    inputs.planar_8x7,
    lambda: inputs.cylinder_patch(14, 11, name="cyl_small"),
    lambda: inputs.mixed_tri(12, 17, name="mixed_small"),
    lambda: inputs.planar_noisy(9, 9, 0, 5, "equal_noisy"),
])
def test_binned_search_equals_bruteforce(orc, make):
    itf = make()
    s1, m1 = orc.search_bruteforce(itf)
    s2, m2 = orc.search_binned(itf)
    assert s1.size > 0
    assert np.array_equal(s1, s2) and np.array_equal(m1, m2)
    key = s1.astype(np.int64) * 10**7 + m1
    assert np.all(np.diff(key) > 0)   # sorted by (s, m), unique


def test_binned_search_equals_bruteforce_batched(orc):
    for itf in inputs.batched_512()[:24]:
        s1, m1 = orc.search_bruteforce(itf)
        s2, m2 = orc.search_binned(itf)
        assert np.array_equal(s1, s2) and np.array_equal(m1, m2)


def test_search_inflation_touching_boxes(orc):
    """Closed comparison: boxes that only touch count, separated ones do not."""
    xs = inputs.grid_nodes(1, 1)
    cs = inputs.grid_quad4(1, 1)
    for gap, want in ((0.0, 1), (1e-12, 1), (3e-9, 0)):
        xm = inputs.grid_nodes(1, 1, 1.0 + gap, 0.0, 2.0 + gap, 1.0)
        itf = inputs.Interface("t", xs, cs, 4, xm, cs.copy(), 4, delta=1e-9)
        s, _ = orc.search_bruteforce(itf)
        assert s.size == want, gap


# ---------------------------------------------------------------- D, M
def test_sumD_equals_slave_area(orc):
    itf = inputs.planar_8x7()
    r = orc.evaluate(itf)
    assert abs(r.D.sum() - 1.0) < 1e-13
    cyl = inputs.cylinder_patch()
    A, De = orc.element_blocks(cyl, lm=1)
    assert abs(De.sum() / (800 * math.sin(math.pi / 800)) - 1) < 1e-13


def test_sumM_equals_overlap_area_full_and_offset(orc):
    r = orc.evaluate(inputs.planar_8x7())
    assert abs(r.M.sum() - 1.0) < 1e-13
    for itf in inputs.batched_512()[:6]:
        r = orc.evaluate(itf)
        dx, dy = itf.info["dx"], itf.info["dy"]
        assert abs(r.M.sum() - (1 - abs(dx)) * (1 - abs(dy))) < 1e-13


def test_sumM_rotated_overlap(orc):
    from scipy.spatial import ConvexHull, HalfspaceIntersection
    itf = inputs.mixed_tri(12, 17, name="mixed_small")
    r = orc.evaluate(itf)
    # intersection area of the unit square and the rotated, offset unit square
    a = math.radians(7.0)
    c, s = math.cos(a), math.sin(a)
    sq = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], float)
    rot = np.array([[0.5 + c * (x - .5) - s * (y - .5) + 0.013,
                     0.5 + s * (x - .5) + c * (y - .5) + 0.029] for x, y in sq])

    def halfspaces(P):
        hs = []
        for i in range(4):
            p, q = P[i], P[(i + 1) % 4]
            nrm = np.array([q[1] - p[1], -(q[0] - p[0])])  # outward for CCW
            hs.append([nrm[0], nrm[1], -nrm @ p])
        return hs
    H = np.array(halfspaces(sq) + halfspaces(rot))
    inter = HalfspaceIntersection(H, np.array([0.5, 0.5]))
    area = ConvexHull(inter.intersections).volume
    assert abs(r.M.sum() - area) < 1e-13
    # D (element mode) covers the whole slave square regardless of coverage
    assert abs(r.D.sum() - 1.0) < 1e-13


def test_row_sums_fully_covered(orc):
    for itf in (inputs.planar_8x7(), inputs.planar_noisy(11, 13, 1, 77, "p11")):
        r = orc.evaluate(itf)
        rd = np.asarray(r.D.sum(1)).ravel()
        rm = np.asarray(r.M.sum(1)).ravel()
        assert np.abs(rd - rm).max() < 1e-13 * rd.max()
    # partially covered: only rows whose whole support lies inside the master
    itf = inputs.mixed_tri(12, 17, name="mixed_small")
    r = orc.evaluate(itf)
    rd = np.asarray(r.D.sum(1)).ravel()
    rm = np.asarray(r.M.sum(1)).ravel()
    a = math.radians(7.0)
    c, s = math.cos(a), math.sin(a)

    def inside_master(p):
        # inverse of the rotation/offset applied to the master square
        u = p[0] - 0.5 - 0.013
        v = p[1] - 0.5 - 0.029
        x = c * u + s * v + 0.5
        y = -s * u + c * v + 0.5
        return -1e-12 <= x <= 1 + 1e-12 and -1e-12 <= y <= 1 + 1e-12
    n = itf.info["ns"]
    covered = 0
    for j in range(itf.n_slave_nodes):
        i, k = j % (n + 1), j // (n + 1)
        sup = [(i + di, k + dk) for di in (-1, 0, 1) for dk in (-1, 0, 1)]
        pts = [(x / n, y / n) for x, y in sup if 0 <= x <= n and 0 <= y <= n]
        if all(inside_master(p) for p in pts):
            covered += 1
            assert abs(rd[j] - rm[j]) < 1e-13 * rd.max(), j
    assert covered > 50


@pytest.mark.parametrize("lm", [0, 1])
@pytest.mark.parametrize("d_domain", [0, 1])
@pytest.mark.parametrize("noise", [0.0, 0.15])
def test_matching_meshes_M_equals_D_permuted(orc, lm, d_domain, noise):
    itf, perm = inputs.matching(6, lm, noise=noise)
    o = orc.make_opts(lm=lm, d_domain=d_domain, delta=itf.delta)
    r = orc.evaluate(itf, o)
    Ns = itf.n_slave_nodes
    Pt = np.zeros((Ns, Ns))
    Pt[np.arange(Ns), perm] = 1.0   # slave node i -> master node perm[i]
    if noise == 0.0 or d_domain == 1:
        # same integration domain and rule on both sides -> equal to rounding
        assert rel(dense(r.M), dense(r.D) @ Pt) < 1e-14
    else:
        # non-parallelogram elements: element-domain D uses the exact 3x3
        # Gauss rule, M the 7-point cell rule on a non-polynomial integrand
        assert 1e-12 < rel(dense(r.M), dense(r.D) @ Pt) < 1e-4


def test_dual_D_diagonal_uniform(orc):
    n = 9
    h = 1.0 / n
    itf = inputs.planar_noisy(n, 7, 1, 3, "dual_uniform")
    r = orc.evaluate(itf)
    D = dense(r.D)
    off = D - np.diag(np.diag(D))
    assert np.abs(off).max() < 1e-14 * np.abs(np.diag(D)).max()
    want = np.full((n + 1, n + 1), h * h)
    want[0, :] /= 2; want[-1, :] /= 2; want[:, 0] /= 2; want[:, -1] /= 2
    assert np.abs(np.diag(D) - want.ravel()).max() < 1e-14


def test_dual_D_diagonal_segment_mode(orc):
    itf = inputs.planar_noisy(8, 7, 1, 3, "dual_seg")
    o = orc.make_opts(lm=1, d_domain=1, delta=itf.delta)
    r = orc.evaluate(itf, o)
    D = dense(r.D)
    off = D - np.diag(np.diag(D))
    # fully covered -> segment D equals element D up to rounding
    assert np.abs(off).max() < 1e-14 * np.abs(np.diag(D)).max()
    assert abs(D.sum() - 1.0) < 1e-13 and abs(r.M.sum() - D.sum()) < 1e-13


def test_standard_D_is_q1_mass(orc):
    n = 8
    r = orc.evaluate(inputs.planar_8x7())
    M1 = mass1d(n, 1.0 / n)
    assert rel(r.D, np.kron(M1, M1)) < 1e-14


@pytest.mark.parametrize("lm", [0, 1])
def test_tensor_grid_M_is_kronecker(orc, lm):
    ns, nm = 8, 7
    itf = inputs.planar_noisy(ns, nm, lm, 0, "tensor", noise=0.0)
    r = orc.evaluate(itf)
    x1s = np.arange(ns + 1) / ns
    x1m = np.arange(nm + 1) / nm
    M1 = mortar1d(x1s, x1m, dual=bool(lm))
    assert rel(r.M, np.kron(M1, M1)) < 1e-13


def test_tensor_grid_offset_M_is_kronecker(orc):
    itf = inputs.batched_512()[3]
    r = orc.evaluate(itf)
    n, nm, dx, dy = itf.info["n"], itf.info["nm"], itf.info["dx"], itf.info["dy"]
    xs1 = np.arange(n + 1) / n
    Mx = mortar1d(xs1, dx + np.arange(nm + 1) / nm)
    My = mortar1d(xs1, dy + np.arange(nm + 1) / nm)
    assert rel(r.M, np.kron(My, Mx)) < 1e-13


def test_affine_master_rule_and_triangulation_independent(orc):
    itf = inputs.mixed_tri(10, 13, name="mixed_small")
    base = orc.evaluate(itf)
    ear = orc.evaluate(itf, orc.make_opts(lm=0, delta=itf.delta, fan=1))
    duffy = orc.evaluate(itf, orc.make_opts(lm=0, delta=itf.delta, tri_rule=25))
    assert rel(ear.M, base.M) < 1e-13
    assert rel(duffy.M, base.M) < 1e-13
    dual = orc.evaluate(itf, orc.make_opts(lm=1, delta=itf.delta))
    dual25 = orc.evaluate(itf, orc.make_opts(lm=1, delta=itf.delta, tri_rule=25, fan=1))
    assert rel(dual25.M, dual.M) < 1e-13


def test_nonaffine_master_rule_dependence_is_small(orc):
    """Noisy bilinear masters: integrands are not polynomial, so the result
    depends on the rule at quadrature-error level only."""
    itf = inputs.planar_8x7()
    a = orc.evaluate(itf)
    b = orc.evaluate(itf, orc.make_opts(lm=0, delta=itf.delta, tri_rule=25))
    assert 1e-16 < rel(a.M, b.M) < 1e-5


@pytest.mark.parametrize("lm", [0, 1])
def test_linear_field_reproduction(orc, lm):
    itf = inputs.planar_noisy(12, 10, lm, 99, "lin")
    r = orc.evaluate(itf)
    for c in (0, 1):
        assert np.abs(r.M @ itf.xm[:, c] - r.D @ itf.xs[:, c]).max() < 1e-14
    lam = np.random.default_rng(1).uniform(-1, 1, itf.xs.shape)
    J, _, _ = orc.weighted_gap_grad(itf, lam, r.s, r.m, orc.make_opts(lm=lm, delta=itf.delta))
    assert abs(J) < 1e-14


# ---------------------------------------------------------------- gradient
def _J(orc, itf, o, s, m, lam):
    J, _, _ = orc.weighted_gap_grad(itf, lam, s, m, o)
    return J


@pytest.mark.parametrize("case", ["mixed", "noisy_dual_segment", "cylinder"])
def test_gradient_matches_central_differences(orc, case):
    if case == "mixed":
        itf = inputs.mixed_tri(6, 8, name="mixed_tiny")
        o = orc.make_opts(lm=0, delta=itf.delta)
    elif case == "noisy_dual_segment":
        itf = inputs.planar_noisy(5, 4, 1, 21, "nds")
        # master larger than the slave (no coincident boundary edges, where J
        # is only one-sided differentiable) and slightly non-planar
        itf.xm[:, :2] = 0.5 + 1.1 * (itf.xm[:, :2] - 0.5)
        itf.xm[:, 2] = 1e-3 * inputs.uniform(5, 9, itf.xm.shape[0], -1, 1)
        o = orc.make_opts(lm=1, d_domain=1, delta=2e-3)
    else:
        itf = inputs.cylinder_patch(6, 5, name="cyl_tiny")
        # stretch the master beyond the slave patch in angle and length
        th = np.arctan2(itf.xm[:, 1], itf.xm[:, 0])
        r = np.hypot(itf.xm[:, 0], itf.xm[:, 1])
        th = 1.06 * th - 0.03 * (0.5 * np.pi)
        itf.xm = np.stack([r * np.cos(th), r * np.sin(th), 1.1 * itf.xm[:, 2] - 0.1], axis=1)
        o = orc.make_opts(lm=1, delta=itf.delta)
    s, m = orc.search_bruteforce(itf, o.delta)
    rng = np.random.default_rng(3)
    lam = rng.uniform(-1, 1, itf.xs.shape)
    J, gs, gm = orc.weighted_gap_grad(itf, lam, s, m, o)
    h = 1e-6
    scale = max(np.abs(gs).max(), np.abs(gm).max())
    picks = [("s", i, c) for i, c in zip(rng.integers(0, itf.xs.shape[0], 32), rng.integers(0, 3, 32))]
    picks += [("m", i, c) for i, c in zip(rng.integers(0, itf.xm.shape[0], 32), rng.integers(0, 3, 32))]
    for side, i, c in picks:
        X = itf.xs if side == "s" else itf.xm
        x0 = X[i, c]
        X[i, c] = x0 + h
        jp = _J(orc, itf, o, s, m, lam)
        X[i, c] = x0 - h
        jm = _J(orc, itf, o, s, m, lam)
        X[i, c] = x0
        fd = (jp - jm) / (2 * h)
        g = (gs if side == "s" else gm)[i, c]
        assert abs(fd - g) <= 1e-6 * scale + 1e-9, (side, i, c, fd, g)


@pytest.mark.parametrize("lm", [0, 1])
def test_gradient_euler_and_translation(orc, lm):
    itf = inputs.planar_noisy(7, 6, lm, 31, "eul")
    rng = np.random.default_rng(5)
    lam = rng.uniform(-1, 1, itf.xs.shape)
    o = orc.make_opts(lm=lm, delta=itf.delta)
    s, m = orc.search_binned(itf)
    J, gs, gm = orc.weighted_gap_grad(itf, lam, s, m, o)
    # translate the whole problem away from the origin so J != 0 is possible:
    # Euler: J(t X) = t^3 J(X) -> sum X.g = 3 J
    scale = np.abs(gs).max() * np.abs(itf.xs).max()
    assert abs(np.sum(itf.xs * gs) + np.sum(itf.xm * gm) - 3 * J) < 1e-11 * scale
    # translation invariance on full coverage: sum of all gradients is zero
    tot = gs.sum(0) + gm.sum(0)
    assert np.abs(tot).max() < 1e-11 * np.abs(gs).max()


def test_gradient_euler_nonzero_J(orc):
    itf = inputs.cylinder_patch(8, 7, name="cyl_eu")
    o = orc.make_opts(lm=1, delta=itf.delta)
    lam = np.random.default_rng(2).uniform(-1, 1, itf.xs.shape)
    s, m = orc.search_binned(itf)
    J, gs, gm = orc.weighted_gap_grad(itf, lam, s, m, o)
    assert abs(J) > 1e-8
    scale = np.abs(gs).max() * np.abs(itf.xs).max()
    assert abs(np.sum(itf.xs * gs) + np.sum(itf.xm * gm) - 3 * J) < 1e-11 * scale
