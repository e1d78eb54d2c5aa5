"""Failure paths of the library on the GPU, all made on the host side (bad
inputs, a time budget that runs out); nothing here faults or hangs the GPU.

* non-finite node coordinates (NaN, +-Inf, either side): the run returns
  MORTAR_ERR_INVALID_ARG, and the same context gives the oracle's D and M once
  the coordinates are finite again (eager and graph paths);
* slave elements with reversed node order (clockwise about the normal): D and
  M do not depend on the orientation, so they equal those of the original
  mesh and the oracle's;
* a folded (self-intersecting) slave quad: MORTAR_ERR_DEGENERATE, its pairs
  integrate to nothing, every other pair equals the oracle;
* empty members of a batch (no slave elements, no master elements): the other
  members are unaffected;
* the watchdog of the persistent pair kernels: a budget far below the kernel
  time returns MORTAR_ERR_TIMEOUT; the context then runs normally once the
  budget is lifted.
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


def _dm(res):
    return res.D, res.M


def _check(mt, m, orc, itf, o):
    ref = orc.evaluate(itf, o)
    s, mm = m.pairs()
    assert np.array_equal(s, ref.s) and np.array_equal(mm, ref.m)
    forward_parity(m.scipy(mt.MATRIX_D), m.scipy(mt.MATRIX_M), ref.D, ref.M,
                   lambda x: _dm(orc.evaluate(x, o, pairs=(ref.s, ref.m))), itf)


@pytest.mark.parametrize("side,value", [("s", np.nan), ("s", np.inf), ("m", np.nan), ("m", -np.inf)])
@pytest.mark.parametrize("graph", [False, True])
def test_nonfinite_coordinates(mt, orc, side, value, graph):
    itf = inputs.planar_noisy(14, 12, 1, 81, "nf")
    o = orc.make_opts(lm=1, delta=itf.delta)
    lam = np.random.default_rng(3).uniform(-1, 1, itf.xs.shape)
    m = mt.Mortar(lm=1, delta=itf.delta)
    m.set_interface(itf.xs, itf.conn_s, itf.xm, itf.conn_m)
    if graph:   # capture the graph on good coordinates first
        m.run_graph(lam)
        m.run_graph(lam)
    xs, xm = itf.xs.copy(), itf.xm.copy()
    (xs if side == "s" else xm)[37, 1] = value
    m.set_coordinates(xs, xm)
    with pytest.raises(mt._native.MortarError, match="INVALID_ARG"):
        if graph:
            m.run_graph(lam)
        else:
            m.evaluate()
    m.set_coordinates(itf.xs, itf.xm)   # finite again: same context, correct results
    if graph:
        m.run_graph(lam)
    else:
        m.evaluate()
    _check(mt, m, orc, itf, o)


def test_reversed_slave_elements(mt, orc):
    itf = inputs.planar_noisy(16, 13, 1, 82, "rev")
    o = orc.make_opts(lm=1, delta=itf.delta)
    a = mt.Mortar(lm=1, delta=itf.delta)
    a.set_interface(itf.xs, itf.conn_s, itf.xm, itf.conn_m)
    a.evaluate()
    rev = inputs.Interface("rev2", itf.xs, itf.conn_s.copy(), 4, itf.xm, itf.conn_m, 4, lm=1, delta=itf.delta)
    flip = [0, 17, 100, 255]
    rev.conn_s[flip] = rev.conn_s[flip][:, ::-1]
    b = mt.Mortar(lm=1, delta=itf.delta)
    b.set_interface(rev.xs, rev.conn_s, rev.xm, rev.conn_m)
    assert b.evaluate() == 0
    for w in (mt.MATRIX_D, mt.MATRIX_M):
        A, B = a.scipy(w), b.scipy(w)
        assert np.array_equal(A.indptr, B.indptr) and np.array_equal(A.indices, B.indices)
        assert np.abs(A.data - B.data).max() <= 1e-12 * np.abs(A.data).max()
    _check(mt, b, orc, rev, o)


def test_folded_slave_element(mt, orc):
    itf = inputs.planar_noisy(10, 9, 0, 83, "fold")
    cs = itf.conn_s.copy()
    e = 44
    cs[e] = cs[e][[0, 1, 3, 2]]   # self-intersecting (bow-tie) node order
    bad = inputs.Interface("fold2", itf.xs, cs, 4, itf.xm, itf.conn_m, 4, lm=0, delta=itf.delta)
    m = mt.Mortar(lm=0, d_domain=1, delta=itf.delta)
    m.set_interface(bad.xs, bad.conn_s, bad.xm, bad.conn_m)
    assert m.evaluate() == -2   # MORTAR_ERR_DEGENERATE; results of the other elements still written
    s, mm = m.pairs()
    Mb, Db, ne = m.pair_blocks(with_D=True)
    assert not ne[s == e].any()
    keep = s != e
    rMb, rDb, rne, _ = orc.pair_blocks(bad, s[keep], mm[keep], orc.make_opts(lm=0, d_domain=1, delta=itf.delta))
    assert np.array_equal(ne[keep], rne)
    blocks_parity(Mb[keep], rMb)
    blocks_parity(Db[keep], rDb)


def test_batch_with_empty_members(mt, orc):
    a = inputs.planar_noisy(9, 7, 0, 84, "a")
    b = inputs.planar_noisy(6, 8, 0, 85, "b")
    no_slave = inputs.Interface("no_slave", np.zeros((0, 3)), np.zeros((0, 4), np.int32), 4,
                                a.xm.copy(), a.conn_m.copy(), 4, lm=0, delta=1e-9)
    no_master = inputs.Interface("no_master", b.xs.copy(), b.conn_s.copy(), 4,
                                 np.zeros((0, 3)), np.zeros((0, 4), np.int32), 4, lm=0, delta=1e-9)
    batch = [a, no_slave, b, no_master]
    lam = np.random.default_rng(5).uniform(-1, 1, (sum(i.xs.shape[0] for i in batch), 3))
    m = mt.Mortar(lm=0, delta=1e-9)
    m.set_batch(batch)
    m.run_graph(lam)
    m.run_graph(lam)
    J, gs, gm = m.gradient()
    D, M = m.scipy(mt.MATRIX_D), m.scipy(mt.MATRIX_M)
    sn, mn = m.offsets["slave_nodes"], m.offsets["master_nodes"]
    o = orc.make_opts(lm=0, delta=1e-9)
    J_ref = 0.0
    for k, itf in enumerate(batch):
        Dk, Mk = D[sn[k]:sn[k + 1], sn[k]:sn[k + 1]], M[sn[k]:sn[k + 1], mn[k]:mn[k + 1]]
        if itf.conn_s.shape[0] == 0 or itf.conn_m.shape[0] == 0:
            assert Mk.nnz == 0
            assert np.all(gm[mn[k]:mn[k + 1]] == 0.0)
            continue
        ref = orc.evaluate(itf, o)
        forward_parity(Dk, Mk, ref.D, ref.M, lambda x: _dm(orc.evaluate(x, o, pairs=(ref.s, ref.m))), itf)
        Jk, rs, rm = orc.weighted_gap_grad(itf, lam[sn[k]:sn[k + 1]], ref.s, ref.m, o)
        scale = max(np.abs(rs).max(), np.abs(rm).max())
        assert max(np.abs(gs[sn[k]:sn[k + 1]] - rs).max(), np.abs(gm[mn[k]:mn[k + 1]] - rm).max()) <= 1e-12 * scale
        J_ref += Jk
    # the slave-only member still has its element-domain D: the term lam.D Xs
    # of J and its gradient
    k = 3
    e0 = np.zeros(0, np.int32)
    Jk, rs, _ = orc.weighted_gap_grad(no_master, lam[sn[k]:sn[k + 1]], e0, e0, o)
    assert np.abs(gs[sn[k]:sn[k + 1]] - rs).max() <= 1e-12 * np.abs(rs).max()
    J_ref += Jk
    assert abs(J - J_ref) <= 1e-12 * max(1.0, abs(J_ref))


@pytest.mark.parametrize("graph", [False, True])
def test_watchdog_timeout(mt, orc, graph):
    itf = inputs.planar_noisy(300, 260, 1, 86, "wd")
    o = orc.make_opts(lm=1, delta=itf.delta)
    lam = np.random.default_rng(7).uniform(-1, 1, itf.xs.shape)
    m = mt.Mortar(lm=1, delta=itf.delta, watchdog_us=1)
    m.set_interface(itf.xs, itf.conn_s, itf.xm, itf.conn_m)
    for _ in range(2):
        with pytest.raises(mt._native.MortarError, match="TIMEOUT"):
            if graph:
                m.run_graph(lam)
            else:
                m.evaluate()
    m.set_watchdog(0)
    if graph:
        m.run_graph(lam)
        m.run_graph(lam)
    else:
        m.evaluate()
    _check(mt, m, orc, itf, o)
