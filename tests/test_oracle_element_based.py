"""Pins of the oracle's element-based integration (no GPU needed).

Element-based integration (Sec. 1, Sec. 2.3) puts an n x n rule on each slave
element and back-projects every point onto the master element that covers it,
with no clipping.  What fixes its result independently of the oracle: on full
coverage the LM and master shape functions sum to one at every point, so
sum(M) is the slave area and M reproduces linear fields exactly; on matching
meshes the integrand is polynomial on each element, so M = D P^T; a brute-force
point location over all master elements written here in numpy gives the same
blocks; and the result converges to the segment-based one as n grows.
"""
import numpy as np
import pytest

from paper_2202_03933_gb300 import inputs


def _swap(itf):
    """Noisy quad mesh as the slave side (non-parallelogram slave elements)."""
    return inputs.Interface("swap", itf.xm, itf.conn_m, itf.type_m, itf.xs, itf.conn_s, itf.type_s,
                            lm=itf.lm, delta=itf.delta)


@pytest.mark.parametrize("lm", [0, 1])
@pytest.mark.parametrize("n", [2, 5, 8])
@pytest.mark.parametrize("noisy_slave", [False, True])
def test_full_coverage_area_and_linear_fields(orc, lm, n, noisy_slave):
    itf = inputs.planar_noisy(8, 7, lm, 5, "ebfull")
    if noisy_slave:
        itf = _swap(itf)
    o = orc.make_opts(lm=lm, delta=itf.delta)
    D, M, _, _ = orc.evaluate_element_based(itf, n, o)
    assert abs(M.sum() - 1.0) < 1e-14
    for c in (0, 1):
        assert np.abs(M @ itf.xm[:, c] - D @ itf.xs[:, c]).max() < 1e-15


@pytest.mark.parametrize("lm", [0, 1])
@pytest.mark.parametrize("d_domain", [0, 1])
def test_matching_meshes_exact(orc, lm, d_domain):
    itf, perm = inputs.matching(5, lm)
    o = orc.make_opts(lm=lm, d_domain=d_domain, delta=itf.delta)
    D, M, _, _ = orc.evaluate_element_based(itf, 2, o)
    Dd = np.asarray(D.todense())
    P = np.zeros((itf.xs.shape[0], itf.xm.shape[0]))
    P[np.arange(itf.xs.shape[0]), perm] = 1.0
    assert np.abs(np.asarray(M.todense()) - Dd @ P).max() < 1e-15


def _bilinear_inverse(p, x):
    """(xi, eta) with sum_a N_a(xi, eta) p_a = x for a quad (Newton from the
    centre, plain numpy), or barycentric coordinates for a triangle."""
    if len(p) == 3:
        A = np.array([p[1] - p[0], p[2] - p[0]]).T
        return np.linalg.solve(A, x - p[0])
    xi = np.zeros(2)
    for _ in range(60):
        a, b, c, d = 1 - xi[0], 1 + xi[0], 1 - xi[1], 1 + xi[1]
        N = 0.25 * np.array([a * c, b * c, b * d, a * d])
        dxi = 0.25 * np.array([-c, c, d, -d])
        deta = 0.25 * np.array([-a, -b, b, a])
        r = N @ p - x
        J = np.array([dxi @ p, deta @ p]).T
        step = np.linalg.solve(J, r)
        xi = xi - step
        if np.abs(step).max() < 1e-15:
            break
    return xi


def _shape(nen, xi):
    if nen == 3:
        return np.array([1 - xi[0] - xi[1], xi[0], xi[1]])
    a, b, c, d = 1 - xi[0], 1 + xi[0], 1 - xi[1], 1 + xi[1]
    return 0.25 * np.array([a * c, b * c, b * d, a * d])


@pytest.mark.parametrize("case", ["quad", "tri", "noisy_slave"])
def test_brute_force_point_location(orc, case):
    """Flat z = 0 interfaces: every slave quadrature point located among ALL
    master elements by the numpy inverse above; blocks summed per (slave
    element, master element).  In-plane rigid motions leave the blocks
    unchanged, so raw (x, y) serve as plane coordinates."""
    if case == "quad":
        itf = inputs.planar_noisy(4, 3, 1, 17, "bf")
    elif case == "tri":
        itf = inputs.mixed_tri(4, 3, lm=1, name="bft")
    else:
        itf = _swap(inputs.planar_noisy(4, 3, 1, 19, "bfn", noise=0.2))
    n = 4
    o = orc.make_opts(lm=itf.lm, delta=itf.delta)
    s, m = orc.search_bruteforce(itf)
    Mb, _, fl = orc.element_based_blocks(itf, s, m, n, o)
    A, _ = orc.element_blocks(itf)
    g, w = np.polynomial.legendre.leggauss(n)
    ref = {}
    nm = itf.conn_m.shape[1]
    for e, conn in enumerate(itf.conn_s):
        ps = itf.xs[conn, :2]
        for i in range(n):
            for j in range(n):
                xi = np.array([g[i], g[j]])
                N = _shape(4, xi)
                a, b, c, d = 1 - xi[0], 1 + xi[0], 1 - xi[1], 1 + xi[1]
                J = np.array([0.25 * np.array([-c, c, d, -d]) @ ps, 0.25 * np.array([-a, -b, b, a]) @ ps]).T
                W = w[i] * w[j] * abs(np.linalg.det(J))
                x = N @ ps
                Phi = A[e, :4, :4] @ N
                owners = []
                for f, cm in enumerate(itf.conn_m):
                    xim = _bilinear_inverse(itf.xm[cm, :2], x)
                    inside = (np.all(np.abs(xim) <= 1 + 1e-10) if nm == 4 else
                              (xim.min() >= -1e-10 and xim.sum() <= 1 + 1e-10))
                    if inside:
                        owners.append((f, xim))
                if not owners:
                    continue
                f, xim = owners[0]
                blk = ref.setdefault((e, f), np.zeros((4, 4)))
                blk[:, :nm] += W * np.outer(Phi, _shape(nm, xim))
    got = {(int(s[p]), int(m[p])): Mb[p] for p in np.flatnonzero(fl)}
    assert set(got) == set(ref)
    for k in ref:
        assert np.abs(got[k] - ref[k]).max() < 1e-15 * 4, k


@pytest.mark.parametrize("case", ["planar", "mixed", "cylinder"])
def test_converges_to_segment_based(orc, case):
    if case == "planar":
        itf = inputs.planar_noisy(8, 7, 1, 3, "cv")
    elif case == "mixed":
        itf = inputs.mixed_tri(8, 11, name="cvm")
    else:
        # master stretched beyond the slave patch: the slave is fully covered
        # (where coverage ends inside a slave element the integrand jumps and
        # element-based quadrature converges only as the points resolve the
        # uncovered strip)
        itf = inputs.cylinder_patch(8, 7, name="cvc")
        th = np.arctan2(itf.xm[:, 1], itf.xm[:, 0])
        r = np.hypot(itf.xm[:, 0], itf.xm[:, 1])
        th = 1.06 * th - 0.03 * (0.5 * np.pi)
        itf.xm = np.stack([r * np.cos(th), r * np.sin(th), 1.1 * itf.xm[:, 2] - 0.1], axis=1)
    o = orc.make_opts(lm=itf.lm, delta=itf.delta)
    seg = orc.evaluate(itf, o)
    errs = []
    for n in (2, 4, 8, 16):
        _, M, _, _ = orc.evaluate_element_based(itf, n, o, pairs=(seg.s, seg.m))
        errs.append(np.abs(np.asarray((M - seg.M).todense())).max() / np.abs(seg.M.data).max())
    assert all(b < 0.6 * a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 5e-3, errs
