"""GPU parity of quadratic slave elements (tri6, quad8) against the oracle.

A quadratic slave element is integrated on its piecewise flat approximation:
its four linear sub-elements are each clipped against the master element, and
the quadratic shape functions are evaluated at the parent parameters of every
quadrature point.  The CUDA path and the oracle share no code; the oracle's
quadratic functions are pinned by tests/test_oracle_quadratic.py.  Checks:
identical pair sets and nonempty flags, per-pair 8 x 4 M blocks and the
element D within 1e-12 of the largest reference value, assembled D and M
through the same entrywise checks as the linear elements, and the counters.
"""
import numpy as np
import pytest

from paper_2202_03933_gb300 import inputs
from gpu_util import blocks_parity, forward_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2202_03933_gb300 import build, mortar
    build()
    return mortar


def tri3_master(kind, ns, nm, name):
    """Quadratic slave mesh on the unit square against the rotated, offset
    tri3 master of mixed_tri (partial coverage, non-matching, affine master)."""
    q = inputs.quadratic_planar(ns, 2, kind, noise=0.0, warp=0.2)
    m = inputs.mixed_tri(2, nm, name=name)
    return inputs.Interface(name, q.xs, q.conn_s, q.type_s, m.xm, m.conn_m, m.type_m, lm=0, delta=1e-9)


def cases():
    return [
        ("quad8_planar", inputs.quadratic_planar(9, 8, "quad8", name="q8p")),
        ("quad8_warped", inputs.quadratic_planar(9, 8, "quad8", warp=0.3, name="q8w")),
        ("tri6_planar", inputs.quadratic_planar(9, 8, "tri6", name="t6p")),
        ("tri6_warped", inputs.quadratic_planar(9, 8, "tri6", warp=0.3, name="t6w")),
        ("quad8_cylinder", inputs.quadratic_cylinder(12, 11, "quad8", name="q8c")),
        ("tri6_cylinder", inputs.quadratic_cylinder(12, 11, "tri6", name="t6c")),
        ("quad8_tri3", tri3_master("quad8", 10, 13, "q8t")),
        ("tri6_tri3", tri3_master("tri6", 10, 13, "t6t")),
        ("quad8_ragged_37x31", inputs.quadratic_planar(37, 31, "quad8", warp=0.2, name="q8r")),
    ]


def run_gpu(mt, itf, graph=False):
    m = mt.Mortar(lm=0, d_domain=0, delta=itf.delta)
    m.set_interface(itf.xs, itf.conn_s, itf.xm, itf.conn_m)
    if graph:
        m.run_graph()
        m.run_graph()
    else:
        m.evaluate()
    return m


@pytest.mark.parametrize("name,itf", cases(), ids=[c[0] for c in cases()])
def test_quadratic_forward_parity(mt, orc, name, itf):
    o = orc.make_opts(lm=0, d_domain=0, delta=itf.delta)
    ref = orc.evaluate(itf, o, search="bruteforce")
    m = run_gpu(mt, itf)
    s, mm = m.pairs()
    assert np.array_equal(s, ref.s) and np.array_equal(mm, ref.m) and s.size > 0
    Mb, _, ne = m.pair_blocks()
    assert Mb.shape == (s.size, 8, 4)
    assert np.array_equal(ne, ref.nonempty)
    blocks_parity(Mb, ref.Mb)
    forward_parity(m.scipy(mt.MATRIX_D), m.scipy(mt.MATRIX_M), ref.D, ref.M,
                   lambda x: (lambda r: (r.D, r.M))(orc.evaluate(x, o, pairs=(ref.s, ref.m))), itf)
    st = m.stats()
    assert st["n_nonempty"] == ref.stats["nonempty"]
    assert st["n_gauss_points"] == ref.stats["gauss_points"]
    assert st["n_newton_fail"] == 0 and st["n_clip_overflow"] == 0


def test_quadratic_element_D_blocks(mt, orc):
    """The assembled element-domain D of a small curved mesh is the plain
    scatter-sum of the oracle's 8 x 8 (6 x 6) element blocks."""
    for kind in ("quad8", "tri6"):
        itf = inputs.quadratic_cylinder(3, 2, kind, name="elemD")
        nen = itf.conn_s.shape[1]
        De = orc.quadratic_element_D(itf)
        ref = np.zeros((itf.xs.shape[0],) * 2)
        for e, c in enumerate(itf.conn_s):
            ref[np.ix_(c, c)] += De[e][:nen, :nen]
        m = run_gpu(mt, itf)
        blocks_parity(m.scipy(mt.MATRIX_D).toarray(), ref)


def test_quadratic_graph_replay_bitwise(mt):
    itf = inputs.quadratic_planar(20, 17, "quad8", warp=0.2, name="q8g")
    a = run_gpu(mt, itf)
    b = run_gpu(mt, itf, graph=True)
    for w in (mt.MATRIX_D, mt.MATRIX_M):
        A, B = a.scipy(w), b.scipy(w)
        assert np.array_equal(A.indptr, B.indptr) and np.array_equal(A.indices, B.indices)
        assert np.array_equal(A.data, B.data)


def test_quadratic_batch(mt, orc):
    """Three quadratic interfaces in one batch: D and M are block diagonal,
    each block the oracle's result of its interface."""
    itfs = [inputs.quadratic_planar(6, 5, "quad8", name="b0"),
            inputs.quadratic_planar(9, 11, "quad8", warp=0.3, name="b1"),
            inputs.quadratic_planar(4, 3, "quad8", noise=0.05, name="b2")]
    m = mt.Mortar(lm=0, d_domain=0, delta=1e-9)
    m.set_batch(itfs)
    m.run_graph()
    m.run_graph()
    D, M = m.scipy(mt.MATRIX_D), m.scipy(mt.MATRIX_M)
    off = m.offsets
    for k, itf in enumerate(itfs):
        ref = orc.evaluate(itf, orc.make_opts(lm=0, d_domain=0, delta=itf.delta))
        s0, s1 = off["slave_nodes"][k], off["slave_nodes"][k + 1]
        m0, m1 = off["master_nodes"][k], off["master_nodes"][k + 1]
        forward_parity(D[s0:s1, s0:s1].tocsr(), M[s0:s1, m0:m1].tocsr(), ref.D, ref.M,
                       lambda x: (lambda r: (r.D, r.M))(orc.evaluate(x, orc.make_opts(lm=0, d_domain=0,
                                                                                       delta=x.delta))), itf)
    assert D.nnz == sum(orc.evaluate(i).D.nnz for i in itfs)


def test_quadratic_full_coverage_invariants(mt):
    """100 x 100 quad8 (and tri6) slave against a noisy 87 x 87 quad4 master on
    the unit square: sum D = sum M = 1, equal row sums, and linear fields
    reproduced (M x_m = D x_s) -- the properties that hold at any size."""
    for kind in ("quad8", "tri6"):
        itf = inputs.quadratic_planar(100, 87, kind, name=f"{kind}_100")
        m = run_gpu(mt, itf, graph=True)
        D, M = m.scipy(mt.MATRIX_D), m.scipy(mt.MATRIX_M)
        assert abs(D.sum() - 1.0) < 1e-12 and abs(M.sum() - 1.0) < 1e-12
        rows = np.abs(np.asarray(D.sum(1)).ravel() - np.asarray(M.sum(1)).ravel()).max()
        assert rows < 1e-15
        for c in (0, 1):
            assert np.abs(M @ itf.xm[:, c] - D @ itf.xs[:, c]).max() < 1e-15
        st = m.stats()
        assert st["n_newton_fail"] == 0 and st["n_clip_overflow"] == 0


def test_quadratic_refusals(mt):
    """Options and calls the quadratic path does not support are refused with
    MORTAR_ERR_INVALID_ARG; the context stays usable."""
    itf = inputs.quadratic_planar(4, 3, "quad8", name="ref")
    Err = mt._native.MortarError
    for kw in (dict(lm=1), dict(d_domain=1), dict(integration=1), dict(facing_test=1)):
        m = mt.Mortar(delta=1e-9, **kw)
        with pytest.raises(Err, match="INVALID_ARG"):
            m.set_interface(itf.xs, itf.conn_s, itf.xm, itf.conn_m)
    m = run_gpu(mt, itf)
    lam = np.ones_like(itf.xs)
    with pytest.raises(Err, match="INVALID_ARG"):
        m.weighted_gap_grad(lam)
    with pytest.raises(Err, match="INVALID_ARG"):
        m.tangent(itf.xs, itf.xm)
    with pytest.raises(Err, match="INVALID_ARG"):
        m.contact_terms()
    with pytest.raises(Err, match="INVALID_ARG"):
        m.autotune()
    with pytest.raises(Err, match="INVALID_ARG"):
        m.run_graph(lam)
    with pytest.raises(Err, match="INVALID_ARG"):   # quadratic master elements
        mt.Mortar(delta=1e-9).set_interface(itf.xm, itf.conn_m, itf.xs, itf.conn_s)
    m.evaluate()
    assert abs(m.scipy(mt.MATRIX_D).sum() - 1.0) < 1e-13
    # the same context takes a linear interface afterwards
    lin = inputs.planar_8x7()
    m.set_interface(lin.xs, lin.conn_s, lin.xm, lin.conn_m)
    m.evaluate()
    assert m.pair_blocks()[0].shape[1:] == (4, 4)
    assert abs(m.scipy(mt.MATRIX_D).sum() - 1.0) < 1e-13


def test_quadratic_nonfinite_and_folded(mt, orc):
    """A non-finite slave coordinate gives MORTAR_ERR_INVALID_ARG and the same
    context gives the oracle's result once it is finite again; a quad8 element
    with two corners swapped (folded sub-elements) gives MORTAR_ERR_DEGENERATE,
    its pairs come out empty and every other pair equals the oracle."""
    itf = inputs.quadratic_planar(8, 7, "quad8", name="q8nf")
    o = orc.make_opts(lm=0, d_domain=0, delta=itf.delta)
    m = mt.Mortar(lm=0, d_domain=0, delta=itf.delta)
    m.set_interface(itf.xs, itf.conn_s, itf.xm, itf.conn_m)
    xs = itf.xs.copy()
    xs[int(itf.conn_s[20, 5]), 0] = np.nan
    m.set_coordinates(xs, itf.xm)
    with pytest.raises(mt._native.MortarError, match="INVALID_ARG"):
        m.evaluate()
    m.set_coordinates(itf.xs, itf.xm)
    m.evaluate()
    ref = orc.evaluate(itf, o)
    forward_parity(m.scipy(mt.MATRIX_D), m.scipy(mt.MATRIX_M), ref.D, ref.M,
                   lambda x: (lambda r: (r.D, r.M))(orc.evaluate(x, o, pairs=(ref.s, ref.m))), itf)
    cs = itf.conn_s.copy()
    e = 27
    cs[e, [0, 2]] = cs[e, [2, 0]]   # corners 0 and 2 swapped: the sub-elements fold
    bad = inputs.Interface("q8fold", itf.xs, cs, itf.type_s, itf.xm, itf.conn_m, itf.type_m, lm=0,
                           delta=itf.delta)
    mb = mt.Mortar(lm=0, d_domain=0, delta=itf.delta)
    mb.set_interface(bad.xs, bad.conn_s, bad.xm, bad.conn_m)
    assert mb.evaluate() == -2   # MORTAR_ERR_DEGENERATE
    s, mm = mb.pairs()
    Mb, _, ne = mb.pair_blocks()
    assert (s == e).any() and not ne[s == e].any()
    keep = s != e
    rMb, rne, _ = orc.quadratic_pair_blocks(bad, s[keep], mm[keep], o)
    assert np.array_equal(ne[keep], rne)
    blocks_parity(Mb[keep], rMb)
