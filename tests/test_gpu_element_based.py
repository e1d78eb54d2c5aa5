"""GPU parity of element-based integration (Sec. 1, Sec. 2.3) against the oracle.

Same candidate pairs, same point ownership (first covering master in pair
order), identical CSR patterns, values within 1e-12 (forward_parity), per-pair
blocks within 1e-12; determinism and graph replay; sampled rows at the
profiling size; the gradient and linearisation refuse element-based contexts.
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


def _swap(itf):
    return inputs.Interface("swap", itf.xm, itf.conn_m, itf.type_m, itf.xs, itf.conn_s, itf.type_s,
                            lm=itf.lm, delta=itf.delta)


def cases():
    return [
        ("planar_8x7", inputs.planar_8x7(), 0, 8),
        ("planar_8x7_seg_n3", inputs.planar_8x7(), 1, 3),
        ("planar_dual_n16", inputs.planar_noisy(9, 8, 1, 41, "pd"), 0, 16),
        ("mixed_small", inputs.mixed_tri(14, 19, name="mixed_small"), 0, 8),
        ("mixed_dual_seg", inputs.mixed_tri(14, 19, lm=1, name="mds"), 1, 5),
        ("cyl_dual", inputs.cylinder_patch(12, 10, name="cyl"), 0, 8),
        ("cyl_dual_seg", inputs.cylinder_patch(12, 10, name="cyl"), 1, 8),
        ("tri_slave", _swap(inputs.mixed_tri(9, 7, name="ts")), 0, 8),
        ("tri_slave_seg_dual", _swap(inputs.mixed_tri(9, 7, lm=1, name="tsd")), 1, 6),
        ("noisy_slave_dual", _swap(inputs.planar_noisy(7, 9, 1, 43, "ns", noise=0.2)), 0, 8),
        ("kite_master", inputs.kite_master(9, 7, 0.45), 0, 8),
    ]


@pytest.mark.parametrize("name,itf,d_domain,n", cases(), ids=[c[0] for c in cases()])
def test_element_based_matches_oracle(mt, orc, name, itf, d_domain, n):
    m = mt.Mortar(lm=itf.lm, d_domain=d_domain, delta=itf.delta, integration=mt.INTEGRATE_ELEMENT,
                  element_rule_n=n)
    m.set_interface(itf.xs, itf.conn_s, itf.xm, itf.conn_m)
    m.evaluate()
    s, mm = m.pairs()
    o = orc.make_opts(lm=itf.lm, d_domain=d_domain, delta=itf.delta, n_threads=8)
    D, M, _, fl = orc.evaluate_element_based(itf, n, o, pairs=(s, mm))
    Mb, Db, gfl = m.pair_blocks(with_D=d_domain == 1)
    rMb, rDb, _ = orc.element_based_blocks(itf, s, mm, n, o)
    assert np.array_equal(gfl, fl)
    blocks_parity(Mb, rMb)
    if d_domain == 1:
        blocks_parity(Db, rDb)
    forward_parity(m.scipy(mt.MATRIX_D), m.scipy(mt.MATRIX_M), D, M,
                   lambda x: orc.evaluate_element_based(x, n, o, pairs=(s, mm))[:2], itf)
    st = m.stats()
    assert st["n_nonempty"] == int(fl.sum()) and st["n_cells"] == 0


def test_element_based_determinism_graph_and_refusals(mt):
    itf = inputs.planar_noisy(20, 17, 1, 7, "ebd")
    m = mt.Mortar(lm=1, delta=itf.delta, integration=mt.INTEGRATE_ELEMENT, element_rule_n=8)
    m.set_interface(itf.xs, itf.conn_s, itf.xm, itf.conn_m)
    m.evaluate()
    a = m.csr(mt.MATRIX_M)
    m.run_graph()
    m.run_graph()
    b = m.csr(mt.MATRIX_M)
    for x, y in zip(a[:3], b[:3]):
        assert np.array_equal(x, y)
    assert abs(a[2].sum() - 1.0) < 1e-13          # full coverage: slave area
    lam = np.zeros_like(itf.xs)
    with pytest.raises(mt.MortarError):
        m.weighted_gap_grad(lam)
    with pytest.raises(mt.MortarError):
        m.tangent(itf.xs, itf.xm)
    with pytest.raises(mt.MortarError):
        mt.Mortar(integration=mt.INTEGRATE_ELEMENT, element_rule_n=17)


def test_element_based_sampled_rows_planar_600x520(mt, orc):
    """Rows of slave nodes inside a strip of element rows: the GPU on the whole
    interface against the oracle on the strip's elements and pairs."""
    itf = inputs.by_name("planar_600x520")
    n = itf.info["ns"]
    m = mt.Mortar(lm=itf.lm, delta=itf.delta, integration=mt.INTEGRATE_ELEMENT, element_rule_n=8)
    m.set_interface(itf.xs, itf.conn_s, itf.xm, itf.conn_m)
    m.evaluate()
    G = m.scipy(mt.MATRIX_M)
    s, mm = m.pairs()
    r0, r1 = 300, 306
    elems = np.arange(r0 * n, r1 * n)
    sel = (s >= elems[0]) & (s <= elems[-1])
    sub = inputs.Interface("strip", itf.xs, itf.conn_s[elems], itf.type_s, itf.xm, itf.conn_m,
                           itf.type_m, lm=itf.lm, delta=itf.delta)
    o = orc.make_opts(lm=itf.lm, delta=itf.delta, n_threads=16)
    _, R, _, _ = orc.evaluate_element_based(sub, 8, o, pairs=(s[sel] - elems[0], mm[sel]))
    nodes = np.concatenate([np.arange(j * (n + 1), (j + 1) * (n + 1)) for j in range(r0 + 1, r1)])
    scale = np.abs(R.data).max()
    for j in nodes:
        g, rr = G.getrow(j), R.getrow(j)
        assert np.array_equal(g.indices, rr.indices), j
        assert np.abs(g.data - rr.data).max() <= 1e-12 * max(np.abs(rr.data).max(), 1e-2 * scale), j


def test_element_based_batched(mt, orc):
    """A batch of independent interfaces: M equals the oracle's element-based M
    on the concatenated meshes (no pair crosses interfaces)."""
    itfs = inputs.batched_512(n_interfaces=6, n_hi=10.0)
    m = mt.Mortar(lm=0, d_domain=0, delta=1e-9, integration=mt.INTEGRATE_ELEMENT, element_rule_n=5)
    m.set_batch(itfs)
    m.evaluate()
    xs = np.concatenate([i.xs for i in itfs])
    xm = np.concatenate([i.xm for i in itfs])
    cs, cm, ns, nm = [], [], 0, 0
    for i in itfs:
        cs.append(i.conn_s + ns)
        cm.append(i.conn_m + nm)
        ns += i.xs.shape[0]
        nm += i.xm.shape[0]
    big = inputs.Interface("cat", xs, np.concatenate(cs).astype(np.int32), inputs.QUAD4, xm,
                           np.concatenate(cm).astype(np.int32), inputs.QUAD4, lm=0, delta=1e-9)
    s, mm = m.pairs()
    o = orc.make_opts(lm=0, delta=1e-9)
    D, M, _, _ = orc.evaluate_element_based(big, 5, o, pairs=(s, mm))
    forward_parity(m.scipy(mt.MATRIX_D), m.scipy(mt.MATRIX_M), D, M,
                   lambda x: orc.evaluate_element_based(x, 5, o, pairs=(s, mm))[:2], big)
