"""Pins of the oracle's linearisation of the mortar terms (no GPU needed).

K(y) = d/dX [(D (x) I3) ys - (M (x) I3) ym] with y held fixed is checked against
what does not depend on the oracle's derivative code: central differences of
the oracle's plain FP64 D and M, Euler's theorem (D and M are homogeneous of
degree 2 in the coordinates), invariance of D and M under rigid translations
and rotations, a closed-form derivative of an overlap area, and the
scalar-functional gradient.
"""
import numpy as np
import pytest

from paper_2202_03933_gb300 import inputs


def _case(orc, name):
    if name == "mixed_std_elem":
        itf = inputs.mixed_tri(4, 5, name="mixed_tiny")
        o = orc.make_opts(lm=0, d_domain=0, delta=itf.delta)
    elif name == "noisy_dual_seg":
        itf = inputs.planar_noisy(4, 3, 1, 21, "nds")
        # master larger than the slave (no coincident boundary edges, where the
        # terms are only one-sided differentiable) and slightly non-planar
        itf.xm[:, :2] = 0.5 + 1.1 * (itf.xm[:, :2] - 0.5)
        itf.xm[:, 2] = 1e-3 * inputs.uniform(5, 9, itf.xm.shape[0], -1, 1)
        o = orc.make_opts(lm=1, d_domain=1, delta=2e-3)
    elif name == "noisy_std_seg_warped":
        itf = inputs.planar_noisy(3, 4, 0, 23, "nss")
        itf.xm[:, :2] = 0.5 + 1.08 * (itf.xm[:, :2] - 0.5)
        itf.xs[:, 2] = 2e-3 * inputs.uniform(7, 1, itf.xs.shape[0], -1, 1)   # warped slave quads
        o = orc.make_opts(lm=0, d_domain=1, delta=4e-3)
    elif name == "tri_slave_dual_seg":
        base = inputs.mixed_tri(4, 3, lm=1, name="tsd")
        itf = inputs.Interface("swap", base.xm, base.conn_m, base.type_m, base.xs, base.conn_s, base.type_s,
                               lm=1, delta=1e-9)
        # master (now the quad grid) stretched beyond the slave: no coincident boundary edges
        itf.xm = itf.xm.copy()
        itf.xm[:, :2] = 0.5 + 1.2 * (itf.xm[:, :2] - 0.5)
        o = orc.make_opts(lm=1, d_domain=1, delta=1e-9)
    else:
        itf = inputs.cylinder_patch(4, 3, name="cyl_tiny")
        th = np.arctan2(itf.xm[:, 1], itf.xm[:, 0])
        r = np.hypot(itf.xm[:, 0], itf.xm[:, 1])
        th = 1.06 * th - 0.03 * (0.5 * np.pi)
        itf.xm = np.stack([r * np.cos(th), r * np.sin(th), 1.1 * itf.xm[:, 2] - 0.1], axis=1)
        o = orc.make_opts(lm=1, d_domain=0, delta=itf.delta)
    s, m = orc.search_bruteforce(itf, o.delta)
    return itf, o, s, m


CASES = ["mixed_std_elem", "noisy_dual_seg", "noisy_std_seg_warped", "cylinder_dual_elem", "tri_slave_dual_seg"]


def _G(orc, itf, o, s, m, ys, ym):
    """(D (x) I3) ys - (M (x) I3) ym from the oracle's FP64 matrices."""
    r = orc.evaluate(itf, o, pairs=(s, m))
    return r.D @ ys - r.M @ ym


def _K(orc, itf, o, s, m, ys, ym, add_direct=False):
    rp, ci, v = orc.tangent(itf, s, m, ys, ym, o, add_direct=add_direct)
    Ns, Nm = itf.xs.shape[0], itf.xm.shape[0]
    return orc.bsr_dense(rp, ci, v, Ns, Ns + Nm)


def _fields(itf, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(-1, 1, itf.xs.shape), rng.uniform(-1, 1, itf.xm.shape)


@pytest.mark.parametrize("case", CASES)
def test_tangent_matches_central_differences(orc, case):
    itf, o, s, m = _case(orc, case)
    ys, ym = _fields(itf, 1)
    K = _K(orc, itf, o, s, m, ys, ym)
    rng = np.random.default_rng(2)
    h = 1e-6
    X0s, X0m = itf.xs.copy(), itf.xm.copy()
    for trial in range(4):
        vs = rng.uniform(-1, 1, itf.xs.shape)
        vm = rng.uniform(-1, 1, itf.xm.shape)
        itf.xs, itf.xm = X0s + h * vs, X0m + h * vm
        gp = _G(orc, itf, o, s, m, ys, ym)
        itf.xs, itf.xm = X0s - h * vs, X0m - h * vm
        gn = _G(orc, itf, o, s, m, ys, ym)
        itf.xs, itf.xm = X0s, X0m
        fd = (gp - gn) / (2 * h)
        kv = (K @ np.concatenate([vs.ravel(), vm.ravel()])).reshape(-1, 3)
        scale = np.abs(K).max() * 3 * (itf.xs.shape[0] + itf.xm.shape[0])
        assert np.abs(fd - kv).max() <= 1e-7 * scale, (case, trial, np.abs(fd - kv).max(), scale)
        assert np.abs(kv).max() > 1e-3 * np.abs(K).max()


@pytest.mark.parametrize("case", CASES)
def test_tangent_euler_translation_rotation(orc, case):
    itf, o, s, m = _case(orc, case)
    ys, ym = _fields(itf, 3)
    K = _K(orc, itf, o, s, m, ys, ym)
    G = _G(orc, itf, o, s, m, ys, ym)
    X = np.concatenate([itf.xs, itf.xm])
    scale = np.abs(K).max() * np.abs(X).max() * 24
    # Euler: D(tX) = t^2 D(X), M(tX) = t^2 M(X)  ->  K X = 2 G
    assert np.abs((K @ X.ravel()).reshape(-1, 3) - 2 * G).max() < 1e-12 * scale
    assert np.abs(G).max() > 1e-6
    # rigid translation of every node leaves D and M unchanged
    for d in range(3):
        T = np.zeros_like(X)
        T[:, d] = 1.0
        assert np.abs(K @ T.ravel()).max() < 1e-12 * scale
    # infinitesimal rigid rotation (omega x X) leaves them unchanged too
    for w in np.eye(3):
        R = np.cross(w, X)
        assert np.abs(K @ R.ravel()).max() < 1e-12 * scale


@pytest.mark.parametrize("case", CASES)
def test_tangent_consistent_with_gradient(orc, case):
    """lambda^T (K(X) + [D (x) I | -M (x) I]) = dJ/dX of J = lambda . g."""
    itf, o, s, m = _case(orc, case)
    lam = np.random.default_rng(4).uniform(-1, 1, itf.xs.shape)
    K = _K(orc, itf, o, s, m, itf.xs, itf.xm, add_direct=True)
    J, gs, gm = orc.weighted_gap_grad(itf, lam, s, m, o)
    g = lam.ravel() @ K
    ref = np.concatenate([gs.ravel(), gm.ravel()])
    assert np.abs(g - ref).max() < 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("lm", [0, 1])
@pytest.mark.parametrize("d_domain", [0, 1])
def test_tangent_overlap_area_closed_form(orc, lm, d_domain):
    """One unit slave square vs one unit master square offset by (a, b).

    With ys = 0 and ym = e_x at every master node, sum_j g_j.x = -sum(M) =
    -overlap area (sum of the LM and master shape functions is 1).  The overlap
    [a,1] x [b,1] becomes a trapezoid when one corner moves, so
      d area / d x(master corner (a, b)) = -(1 - b)(1 + b) / 2,
      d area / d y(master corner (a, b)) = -(1 - a)(1 + a) / 2,
      d area / d x(slave corner (1, 1))  =  (1 - b)(1 + b) / 2.
    """
    a, b = 0.3, 0.45
    xs = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0]], float)
    xm = np.array([[a, b, 0], [a + 1, b, 0], [a + 1, b + 1, 0], [a, b + 1, 0]], float)
    c4 = np.array([[0, 1, 2, 3]], np.int32)
    itf = inputs.Interface("two_squares", xs, c4, inputs.QUAD4, xm, c4.copy(), inputs.QUAD4,
                           lm=lm, delta=1e-9)
    o = orc.make_opts(lm=lm, d_domain=d_domain, delta=1e-9)
    s, m = orc.search_bruteforce(itf)
    ys = np.zeros_like(xs)
    ym = np.zeros_like(xm)
    ym[:, 0] = 1.0
    K = _K(orc, itf, o, s, m, ys, ym)
    G = _G(orc, itf, o, s, m, ys, ym)
    assert abs(G[:, 0].sum() + (1 - a) * (1 - b)) < 1e-15
    dA = -K[0::3].sum(axis=0)            # d area / d (all coordinates)
    assert abs(dA[3 * (4 + 0) + 0] + 0.5 * (1 - b) * (1 + b)) < 1e-14
    assert abs(dA[3 * (4 + 0) + 1] + 0.5 * (1 - a) * (1 + a)) < 1e-14
    assert abs(dA[3 * 2 + 0] - 0.5 * (1 - b) * (1 + b)) < 1e-14
    assert abs(dA[3 * (4 + 0) + 2]) < 1e-14            # out-of-plane: flat overlap unchanged


def test_tangent_pattern_rule(orc):
    """Structural blocks: every non-empty pair's (slave row, pair node) and, in
    element-domain mode, every element's (slave row, slave node)."""
    itf, o, s, m = _case(orc, "mixed_std_elem")
    ys, ym = _fields(itf, 5)
    rp, ci, v = orc.tangent(itf, s, m, ys, ym, o)
    _, _, fl = orc.tangent_blocks(itf, s, m, ys, ym, o)
    Ns = itf.xs.shape[0]
    want = set()
    for p in np.flatnonzero(fl):
        for j in itf.conn_s[s[p]]:
            for k in itf.conn_s[s[p]]:
                want.add((int(j), int(k)))
            for k in itf.conn_m[m[p]]:
                want.add((int(j), Ns + int(k)))
    for e in range(itf.conn_s.shape[0]):
        for j in itf.conn_s[e]:
            for k in itf.conn_s[e]:
                want.add((int(j), int(k)))
    got = {(j, int(ci[q])) for j in range(Ns) for q in range(rp[j], rp[j + 1])}
    assert got == want
    assert all(np.all(np.diff(ci[rp[j]:rp[j + 1]]) > 0) for j in range(Ns))
