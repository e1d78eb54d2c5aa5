"""GPU parity of the forward path (search, integration, assembly) against the oracle.

Everything goes through the C ABI via the Python binding.  Pair sets must be
identical; CSR patterns identical; values within 1e-12 relative (max abs
difference over max abs reference value).
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


def swap_sides(itf, name):
    return inputs.Interface(name, itf.xm, itf.conn_m, itf.type_m, itf.xs, itf.conn_s, itf.type_s,
                            lm=itf.lm, delta=itf.delta)


def small_cases():
    dual_seg = inputs.planar_noisy(9, 8, 1, 41, "dual_seg")
    tri_slave = swap_sides(inputs.mixed_tri(14, 11, name="m"), "tri_slave")
    cyl = inputs.cylinder_patch(24, 21, name="cyl_small")
    return [
        ("planar_8x7", inputs.planar_8x7(), 0),
        ("planar_8x7_seg", inputs.planar_8x7(), 1),
        ("cyl_small_dual", cyl, 0),
        ("cyl_small_dual_seg", cyl, 1),
        ("mixed_small", inputs.mixed_tri(30, 40, name="mixed_small"), 0),
        ("mixed_small_dual", inputs.mixed_tri(30, 40, lm=1, name="mixed_small_dual"), 0),
        ("tri_slave", tri_slave, 0),
        ("tri_slave_seg", tri_slave, 1),
        ("dual_seg", dual_seg, 1),
        ("matching_std", inputs.matching(7, 0, noise=0.15)[0], 1),
        ("matching_dual", inputs.matching(7, 1, noise=0.15)[0], 0),
        ("ragged_33x29", inputs.planar_noisy(33, 29, 0, 43, "ragged"), 0),
    ]


def _dm(res):
    return res.D, res.M


def check_dm(mt, m, orc, itf, o, ref):
    """D and M of context m against the oracle result ref (computed with
    options o on ref's pair list)."""
    return forward_parity(m.scipy(mt.MATRIX_D), m.scipy(mt.MATRIX_M), ref.D, ref.M,
                          lambda x: _dm(orc.evaluate(x, o, pairs=(ref.s, ref.m))), itf)


def run_gpu(mt, itf, d_domain, graph=False):
    m = mt.Mortar(lm=itf.lm, d_domain=d_domain, delta=itf.delta)
    m.set_interface(itf.xs, itf.conn_s, itf.xm, itf.conn_m)
    if graph:
        m.run_graph()
        m.run_graph()
    else:
        m.evaluate()
    return m


@pytest.mark.parametrize("name,itf,d_domain", small_cases(), ids=[c[0] for c in small_cases()])
def test_forward_parity_small(mt, orc, name, itf, d_domain):
    o = orc.make_opts(lm=itf.lm, d_domain=d_domain, delta=itf.delta)
    ref = orc.evaluate(itf, o, search="bruteforce")
    m = run_gpu(mt, itf, d_domain)
    s, mm = m.pairs()
    assert np.array_equal(s, ref.s) and np.array_equal(mm, ref.m)
    Mb, Db, ne = m.pair_blocks(with_D=d_domain == 1)
    assert np.array_equal(ne, ref.nonempty)
    blocks_parity(Mb, ref.Mb)
    if d_domain == 1:
        blocks_parity(Db, ref.Db)
    check_dm(mt, m, orc, itf, o, ref)
    st = m.stats()
    assert st["n_nonempty"] == ref.stats["nonempty"]
    assert st["n_gauss_points"] == ref.stats["gauss_points"]
    assert st["n_newton_fail"] == 0 and st["n_clip_overflow"] == 0


def test_deterministic_and_graph_replay(mt):
    itf = inputs.mixed_tri(40, 55, name="det")
    a = run_gpu(mt, itf, 0)
    b = run_gpu(mt, itf, 0, graph=True)
    for w in (mt.MATRIX_D, mt.MATRIX_M):
        A, B = a.scipy(w), b.scipy(w)
        assert np.array_equal(A.indptr, B.indptr) and np.array_equal(A.indices, B.indices)
        assert np.array_equal(A.data, B.data)   # bitwise
    Ma, _, _ = a.pair_blocks()
    Mb, _, _ = b.pair_blocks()
    assert np.array_equal(Ma, Mb)


def test_coordinate_update_reuses_context(mt, orc):
    itf = inputs.planar_noisy(12, 10, 0, 51, "upd")
    m = run_gpu(mt, itf, 0)
    itf2 = inputs.planar_noisy(12, 10, 0, 52, "upd2")
    m.set_coordinates(itf2.xs, itf2.xm)
    m.evaluate()
    o = orc.make_opts(lm=itf2.lm, delta=itf2.delta)
    check_dm(mt, m, orc, itf2, o, orc.evaluate(itf2, o))


# ---------------------------------------------------------------- edge cases
def test_no_overlap_gives_empty_M(mt):
    itf = inputs.planar_noisy(4, 3, 0, 1, "far")
    itf.xm = itf.xm + np.array([5.0, 0.0, 0.0])
    m = run_gpu(mt, itf, 0)
    assert m.stats()["n_pairs"] == 0
    M = m.scipy(mt.MATRIX_M)
    assert M.nnz == 0 and M.shape == (25, 16)
    assert abs(m.scipy(mt.MATRIX_D).sum() - 1.0) < 1e-13


def test_empty_slave_mesh(mt):
    xs = np.zeros((0, 3))
    cs = np.zeros((0, 4), np.int32)
    itf = inputs.planar_8x7()
    m = mt.Mortar()
    m.set_interface(xs, cs, itf.xm, itf.conn_m)
    m.evaluate()
    assert m.stats()["n_pairs"] == 0
    assert m.csr_size(mt.MATRIX_M) == (0, itf.xm.shape[0], 0)


def test_single_element_each(mt, orc):
    xs = inputs.grid_nodes(1, 1)
    cs = inputs.grid_quad4(1, 1)
    xm = inputs.grid_nodes(1, 1, 0.3, -0.2, 1.3, 0.8)
    itf = inputs.Interface("one", xs, cs, 4, xm, cs.copy(), 4)
    m = run_gpu(mt, itf, 1)
    o = orc.make_opts(d_domain=1)
    check_dm(mt, m, orc, itf, o, orc.evaluate(itf, o))
    assert abs(m.scipy(mt.MATRIX_M).sum() - 0.7 * 0.8) < 1e-15


def test_touching_only_pairs_are_empty(mt, orc):
    """Neighbouring elements that share only an edge: candidate pair, empty clip."""
    itf = inputs.matching(3, 0)[0]
    m = run_gpu(mt, itf, 0)
    o = orc.make_opts(lm=itf.lm, delta=itf.delta)
    ref = orc.evaluate(itf, o)
    _, _, ne = m.pair_blocks()
    assert np.array_equal(ne, ref.nonempty) and (~ne).sum() > 0
    check_dm(mt, m, orc, itf, o, ref)


def test_bad_connectivity_rejected(mt):
    itf = inputs.planar_8x7()
    cs = itf.conn_s.copy()
    cs[3, 2] = 10_000
    m = mt.Mortar()
    with pytest.raises(mt._native.MortarError, match="INVALID_ARG"):
        m.set_interface(itf.xs, cs, itf.xm, itf.conn_m)


def test_degenerate_slave_element_flagged(mt):
    itf = inputs.planar_noisy(3, 3, 0, 2, "deg")
    xs = itf.xs.copy()
    cs = itf.conn_s.copy()
    cs[4] = [cs[4][0], cs[4][0], cs[4][0], cs[4][0]]   # zero-area element
    m = mt.Mortar()
    m.set_interface(xs, cs, itf.xm, itf.conn_m)
    assert m.evaluate() == -2   # MORTAR_ERR_DEGENERATE, results still written
    Mb, _, ne = m.pair_blocks()
    s, _ = m.pairs()
    assert not ne[s == 4].any()


def test_capacity_error_on_small_buffer(mt):
    import ctypes
    itf = inputs.planar_8x7()
    m = run_gpu(mt, itf, 0)
    nr, nc, nnz = m.csr_size(mt.MATRIX_M)
    rp = np.empty(nr + 1, np.int64)
    ci = np.empty(nnz, np.int32)
    va = np.empty(nnz)
    r = mt.lib().mortar_csr_copy(m.h, 1, rp.ctypes.data_as(ctypes.c_void_p), ci.ctypes.data_as(ctypes.c_void_p),
                                 va.ctypes.data_as(ctypes.c_void_p), nnz - 1, 0)
    assert r == -4


# ---------------------------------------------------------------- full sizes
def _sampled_rows(orc, itf, s, m, rows, o):
    """Oracle CSR rows for the given slave nodes, from only the pairs whose
    slave element touches one of them."""
    cs = np.asarray(itf.conn_s)
    touch = np.isin(cs, rows).any(axis=1)
    keep = touch[s]
    Mb, Db, ne, _ = orc.pair_blocks(itf, s[keep], m[keep], o)
    _, De = orc.element_blocks(itf, o.lm)
    D, M = orc.assemble(itf, s[keep], m[keep], Mb, Db, ne, De, o.d_domain, o.lm)
    return D[rows], M[rows]


@pytest.mark.parametrize("cfg", ["cylinder_200x173", "mixed_300x400"])
def test_full_size_parity(mt, orc, cfg):
    itf = inputs.by_name(cfg)
    o = orc.make_opts(lm=itf.lm, delta=itf.delta, n_threads=16)
    ref = orc.evaluate(itf, o)
    m = run_gpu(mt, itf, 0, graph=True)
    s, mm = m.pairs()
    assert np.array_equal(s, ref.s) and np.array_equal(mm, ref.m)
    check_dm(mt, m, orc, itf, o, ref)
    if itf.lm == 1:
        D = m.scipy(mt.MATRIX_D)
        off = D - __import__("scipy.sparse", fromlist=["diags"]).diags(D.diagonal())
        assert abs(off).max() <= 1e-14 * D.diagonal().max()


def test_full_size_planar_2000(mt, orc):
    """The benchmark workload in its benchmark launch (graph replay): exact
    pair set against the oracle's binned search, sampled pair blocks and
    sampled CSR rows against the oracle, and closed-form invariants."""
    itf = inputs.planar_2000x1733()
    m = run_gpu(mt, itf, 0, graph=True)
    s, mm = m.pairs()
    rs, rm = orc.search_binned(itf)
    assert np.array_equal(s, rs) and np.array_equal(mm, rm)
    rng = np.random.default_rng(11)
    idx = np.sort(rng.choice(s.size, 20000, replace=False))
    idx = np.unique(np.concatenate([idx, [0, s.size - 1]]))
    o = orc.make_opts(lm=itf.lm, delta=itf.delta, n_threads=16)
    Mb_ref, _, ne_ref, _ = orc.pair_blocks(itf, s[idx], mm[idx], o)
    Mb, _, ne = m.pair_blocks()
    assert np.array_equal(ne[idx], ne_ref)
    blocks_parity(Mb[idx], Mb_ref)
    rows = np.unique(np.concatenate([rng.choice(itf.xs.shape[0], 300, replace=False), [0, itf.xs.shape[0] - 1]]))
    Dr, Mr = _sampled_rows(orc, itf, s, mm, rows, o)
    D = m.scipy(mt.MATRIX_D)
    M = m.scipy(mt.MATRIX_M)
    forward_parity(D[rows], M[rows], Dr, Mr, lambda x: _sampled_rows(orc, x, s, mm, rows, o), itf)
    # invariants at full size: unit square fully covered
    assert abs(D.sum() - 1.0) < 1e-12 and abs(M.sum() - 1.0) < 1e-12
    for c in (0, 1):
        assert np.abs(M @ itf.xm[:, c] - D @ itf.xs[:, c]).max() < 1e-15
    off = D - __import__("scipy.sparse", fromlist=["diags"]).diags(D.diagonal())
    assert abs(off).max() <= 1e-14 * D.diagonal().max()


@pytest.mark.parametrize("variant,rounds,block", [(1, 0, 64), (1, 0, 256), (0, 1, 64), (0, 2, 256), (0, 4, 128),
                                                  (0, 16, 64)])
def test_launch_variants_agree(mt, orc, variant, rounds, block):
    """Every integration schedule gives the oracle's blocks (bilinear masters,
    tri3 masters, a non-affine warped slave, segment mode)."""
    cases = [(inputs.planar_noisy(41, 37, 1, 44, "v"), 1), (inputs.mixed_tri(33, 41, name="vt"), 0)]
    warped = inputs.planar_noisy(21, 17, 0, 45, "w")
    warped.xs = warped.xs.copy()
    warped.xs[:, 0] += 0.2 / 21 * np.sin(7 * warped.xs[:, 1]) * (warped.xs[:, 0] * (1 - warped.xs[:, 0]))
    cases.append((warped, 0))
    for itf, d_domain in cases:
        o = orc.make_opts(lm=itf.lm, d_domain=d_domain, delta=itf.delta)
        ref = orc.evaluate(itf, o)
        m = mt.Mortar(lm=itf.lm, d_domain=d_domain, delta=itf.delta)
        m.set_interface(itf.xs, itf.conn_s, itf.xm, itf.conn_m)
        m.set_launch(variant=variant, block_size=block, rounds=rounds)
        m.evaluate()
        Mb, Db, ne = m.pair_blocks(with_D=d_domain == 1)
        assert np.array_equal(ne, ref.nonempty)
        blocks_parity(Mb, ref.Mb)
        if d_domain == 1:
            blocks_parity(Db, ref.Db)
        check_dm(mt, m, orc, itf, o, ref)
        assert m.stats()["n_newton_fail"] == 0


def test_launch_shape_validation(mt, orc):
    """Shapes outside the documented set are refused (blocks above 256 threads,
    blocks that are not whole warps, round counts other than 1, 2, 4, 8, 16, 32);
    the largest accepted shape evaluates correctly."""
    m = mt.Mortar()
    for args in ((0, 512, 0, 2), (1, 96 + 16, 0, 0), (0, 128, 0, 64), (0, 128, 0, 3), (0, 128, 0, 12)):
        with pytest.raises(mt._native.MortarError, match="INVALID_ARG"):
            m.set_launch(*args)
    m.set_launch(0, 256, 0, 2)
    m.set_launch(0, 256, 0, 32)
    m.set_launch(1, 256, 128, 0)
    itf = inputs.planar_noisy(20, 17, 1, 49, "shape")
    m = mt.Mortar(lm=1, delta=itf.delta)
    m.set_interface(itf.xs, itf.conn_s, itf.xm, itf.conn_m)
    m.set_launch(0, 256, 0, 32)
    m.evaluate()
    o = orc.make_opts(lm=1, delta=itf.delta)
    check_dm(mt, m, orc, itf, o, orc.evaluate(itf, o))


@pytest.mark.parametrize("lm,d_domain", [(0, 0), (1, 1)])
def test_distorted_master_quads(mt, orc, lm, d_domain):
    """Strongly distorted but valid bilinear master quads (kite mesh, a corner
    angle near 180 degrees): the FP32-seeded back-projection does not settle at
    a fraction of the points there and continues with FP64 Newton.  Pair blocks
    and D, M against the oracle in both schedules, and no Newton failure."""
    itf = inputs.kite_master(20, 17, 0.45, lm=lm)
    o = orc.make_opts(lm=lm, d_domain=d_domain, delta=itf.delta)
    ref = orc.evaluate(itf, o)
    assert ref.stats["newton_fail"] == 0
    for variant, rounds in ((0, 2), (1, 0)):
        m = mt.Mortar(lm=lm, d_domain=d_domain, delta=itf.delta)
        m.set_interface(itf.xs, itf.conn_s, itf.xm, itf.conn_m)
        m.set_launch(variant=variant, rounds=rounds)
        m.evaluate()
        Mb, Db, ne = m.pair_blocks(with_D=d_domain == 1)
        assert np.array_equal(ne, ref.nonempty)
        blocks_parity(Mb, ref.Mb)
        if d_domain == 1:
            blocks_parity(Db, ref.Db)
        check_dm(mt, m, orc, itf, o, ref)
        assert m.stats()["n_newton_fail"] == 0


def test_autotune_keeps_results(mt, orc):
    itf = inputs.mixed_tri(36, 45, name="at")
    m = mt.Mortar(lm=0, delta=itf.delta)
    m.set_interface(itf.xs, itf.conn_s, itf.xm, itf.conn_m)
    lam = np.random.default_rng(3).uniform(-1, 1, itf.xs.shape)
    pick = m.autotune(lam)
    assert pick["variant"] in (0, 1) and pick["rounds"] in (0, 1, 2, 4, 8, 16, 32) and pick["ms"] > 0
    assert pick["block"] in (64, 128, 256)
    m.run_graph(lam)
    m.run_graph(lam)
    o = orc.make_opts(lm=itf.lm, delta=itf.delta)
    check_dm(mt, m, orc, itf, o, orc.evaluate(itf, o))


def test_moving_interface_reevaluation(mt, orc):
    """Repeated evaluation of one context while the master slides and turns
    (coordinates updated on the device between graph replays, bins rebuilt
    every step, bin size with the velocity margin of Sec. 3.5)."""
    import math
    import torch
    base = inputs.planar_noisy(24, 21, 1, 48, "mov")
    xm0 = base.xm.copy()
    m = mt.Mortar(lm=1, delta=1e-9, bin_margin=2 * 0.01)
    m.set_interface(torch.from_numpy(base.xs).cuda(), torch.from_numpy(base.conn_s).cuda(),
                    torch.from_numpy(xm0).cuda(), torch.from_numpy(base.conn_m).cuda())
    lam = np.random.default_rng(6).uniform(-1, 1, base.xs.shape)
    for step in range(4):
        a = 0.02 * step
        xm = xm0.copy()
        u, v = xm[:, 0] - 0.5, xm[:, 1] - 0.5
        xm[:, 0] = 0.5 + math.cos(a) * u - math.sin(a) * v + 0.01 * step
        xm[:, 1] = 0.5 + math.sin(a) * u + math.cos(a) * v
        m.set_coordinates(None, torch.from_numpy(xm).cuda())
        m.run_graph(torch.from_numpy(lam).cuda())
        itf = inputs.Interface("mov", base.xs, base.conn_s, 4, xm, base.conn_m, 4, lm=1, delta=1e-9)
        o = orc.make_opts(lm=1, delta=1e-9)
        ref = orc.evaluate(itf, o)
        s, mm = m.pairs()
        assert np.array_equal(s, ref.s) and np.array_equal(mm, ref.m), step
        check_dm(mt, m, orc, itf, o, ref)
