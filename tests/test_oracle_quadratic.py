"""Pins of the oracle's quadratic slave elements (tri6, quad8) -- no GPU.

The quadratic shape functions are fixed by properties that determine them
uniquely: each lies in the element's polynomial space (quad8: the serendipity
space 1, xi, eta, xi^2, xi eta, eta^2, xi^2 eta, xi eta^2; tri6: the complete
quadratics), they interpolate (N_a(node_b) = delta_ab), and their derivatives
are the derivatives of those polynomials.  The element D is checked against
exact integrals of the fitted polynomials over the parameter domain.  The
assembled D and M are checked against what the mathematics fixes on planar
straight-sided meshes: sum D = slave area, sum M = overlap area, equal row
sums on covered rows, exact reproduction of linear fields (M X_m = D X_s)
against a noisy non-matching quad4 master, and the brute-force pair set.
A planted mistake in any of these parts (a wrong mid-side function, a
transposed parent map, a dropped Jacobian) fails one of them.
"""
import itertools

import numpy as np
import pytest

from paper_2202_03933_gb300 import inputs

QUAD8_NODES = np.array([(-1, -1), (1, -1), (1, 1), (-1, 1), (0, -1), (1, 0), (0, 1), (-1, 0)], float)
TRI6_NODES = np.array([(0, 0), (1, 0), (0, 1), (0.5, 0), (0.5, 0.5), (0, 0.5)], float)
QUAD8_SPACE = [(0, 0), (1, 0), (0, 1), (2, 0), (1, 1), (0, 2), (2, 1), (1, 2)]
TRI6_SPACE = [(0, 0), (1, 0), (0, 1), (2, 0), (1, 1), (0, 2)]


def _cases():
    return [(8, QUAD8_NODES, QUAD8_SPACE), (6, TRI6_NODES, TRI6_SPACE)]


def _sample(nen, k, rng):
    if nen == 8:
        return rng.uniform(-1, 1, (k, 2))
    p = rng.uniform(0, 1, (k, 2))
    flip = p.sum(1) > 1
    p[flip] = 1 - p[flip]
    return p


def _fit(orc, nen, space, rng):
    """Polynomial coefficients (nen x len(space)) of the oracle's shape
    functions, least squares over random points; also the max residual."""
    pts = _sample(nen, 60, rng)
    V = np.array([[x ** i * y ** j for (i, j) in space] for x, y in pts])
    N = np.array([orc.shape_quadratic(nen, x, y)[0] for x, y in pts])
    C, *_ = np.linalg.lstsq(V, N, rcond=None)
    return C.T, np.abs(V @ C - N).max()


@pytest.mark.parametrize("nen,nodes,space", _cases(), ids=["quad8", "tri6"])
def test_shape_functions_are_the_quadratic_interpolants(orc, nen, nodes, space):
    rng = np.random.default_rng(1)
    C, res = _fit(orc, nen, space, rng)
    assert res < 1e-14                       # each N_a lies in the element's polynomial space
    for b, (x, y) in enumerate(nodes):       # interpolation: N_a(node_b) = delta_ab
        N, _ = orc.shape_quadratic(nen, x, y)
        assert np.allclose(N, np.eye(nen)[b], atol=1e-15, rtol=0)
    for x, y in _sample(nen, 10, rng):       # derivatives of the same polynomials
        _, dN = orc.shape_quadratic(nen, x, y)
        dx = np.array([[i * x ** (i - 1) * y ** j if i else 0.0 for (i, j) in space]])
        dy = np.array([[j * x ** i * y ** (j - 1) if j else 0.0 for (i, j) in space]])
        assert np.allclose(dN[:, 0], (dx @ C.T).ravel(), atol=1e-13, rtol=0)
        assert np.allclose(dN[:, 1], (dy @ C.T).ravel(), atol=1e-13, rtol=0)


def _monomial_integral(nen, i, j):
    """Exact integral of x^i y^j over the parameter domain."""
    if nen == 8:
        return (0.0 if i % 2 else 2.0 / (i + 1)) * (0.0 if j % 2 else 2.0 / (j + 1))
    from math import factorial
    return factorial(i) * factorial(j) / factorial(i + j + 2)


@pytest.mark.parametrize("nen,nodes,space", _cases(), ids=["quad8", "tri6"])
def test_element_D_of_an_affine_element_is_the_exact_mass_matrix(orc, nen, nodes, space):
    """Affine (straight-sided) element with a constant Jacobian J0: D_ab =
    J0 int N_a N_b, integrated exactly from the polynomial coefficients."""
    rng = np.random.default_rng(2)
    C, _ = _fit(orc, nen, space, rng)
    Aff = np.array([[0.7, 0.2], [-0.1, 0.5]])
    off = np.array([0.3, -0.4])
    X = np.zeros((nen, 3))
    X[:, :2] = nodes @ Aff.T + off
    J0 = abs(np.linalg.det(Aff))
    itf = inputs.Interface("one", X, np.arange(nen, dtype=np.int32)[None, :], nen, X[:1], np.zeros((0, 4), np.int32),
                           4)
    De = orc.quadratic_element_D(itf)[0][:nen, :nen]
    exact = np.zeros((nen, nen))
    for a, b in itertools.product(range(nen), range(nen)):
        for (p, cp), (q, cq) in itertools.product(zip(space, C[a]), zip(space, C[b])):
            exact[a, b] += cp * cq * _monomial_integral(nen, p[0] + q[0], p[1] + q[1])
    assert np.abs(De - J0 * exact).max() <= 1e-14 * np.abs(exact).max() * J0
    assert abs(De.sum() - J0 * (4.0 if nen == 8 else 0.5)) < 1e-14


@pytest.mark.parametrize("kind", ["quad8", "tri6"])
@pytest.mark.parametrize("warp", [0.0, 0.3])
def test_slave_area_and_pair_set(orc, kind, warp):
    """sum D = slave area (1): curved interior edges (warp) keep the boundary,
    and the rule integrates the polynomial Jacobian exactly; binned search =
    brute force on quadratic boxes."""
    itf = inputs.quadratic_planar(7, 6, kind, warp=warp)
    s1, m1 = orc.search_bruteforce(itf)
    s2, m2 = orc.search_binned(itf)
    assert np.array_equal(s1, s2) and np.array_equal(m1, m2) and s1.size > 0
    r = orc.evaluate(itf)
    assert abs(r.D.sum() - 1.0) < 1e-13
    assert r.stats["newton_fail"] == 0


@pytest.mark.parametrize("kind", ["quad8", "tri6"])
def test_planar_invariants(orc, kind):
    """Straight-sided slave elements on a fully covered square, noisy quad4
    master: sum M = 1, equal row sums of D and M, and linear fields
    reproduced exactly (the master interpolates x exactly; N_a(xi_parent) x is
    a cubic on every cell, inside the 7-point rule's degree)."""
    itf = inputs.quadratic_planar(8, 7, kind, noise=0.1)
    r = orc.evaluate(itf)
    assert abs(r.M.sum() - 1.0) < 1e-13
    assert np.abs(np.asarray(r.D.sum(1)).ravel() - np.asarray(r.M.sum(1)).ravel()).max() < 1e-15
    for c in (0, 1):
        assert np.abs(r.M @ itf.xm[:, c] - r.D @ itf.xs[:, c]).max() < 1e-15
    assert r.stats["xi_out_of_range"] == 0 and r.stats["clip_overflow"] == 0


def test_curved_cylinder_patch(orc):
    """Quad8 on the cylinder (every node on r = 1): sum D is the area of the
    quadratic isoparametric surface, within its geometric error of the exact
    quarter cylinder (pi) and far closer than the chord approximation of the
    same nodes; sum M is bounded by the area of the piecewise flat
    sub-elements (the chord master covers their projections up to the
    curvature gaps)."""
    itf = inputs.quadratic_cylinder(8, 7, "quad8")
    r = orc.evaluate(itf)
    assert abs(r.D.sum() - np.pi) < 1e-4
    chord = 32 * np.sin(np.pi / 64) * 2.0     # 16 flat sub-element columns x length 2
    assert chord - 1e-3 < r.M.sum() <= chord + 1e-13
    assert abs(r.D.sum() - np.pi) < 0.05 * abs(chord - np.pi)
