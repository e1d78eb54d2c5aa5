"""GPU parity of the linearisation K = d/dX[(D (x) I3) ys - (M (x) I3) ym].

Against the oracle's forward-mode (dual number) blocks: identical block
pattern, every block row within 1e-12 of its largest entry, or within 4x the
oracle's own change under 1-ulp input perturbations where that is larger
(curved interfaces whose projected master edges run nearly parallel to slave
edges: the derivative of a shallow-angle intersection is ill-conditioned; the
oracle's own sensitivity there is ~2e-12 and must stay below 2.5e-12).  Also: the scalar
gradient of the GPU adjoint (lambda^T K with the direct terms), Euler
homogeneity and rigid-motion invariance of the GPU's own K, determinism, the
direct terms, batched interfaces, and sampled rows at full size.
"""
import numpy as np
import pytest

from paper_2202_03933_gb300 import inputs
from gpu_util import bsr_parity, grad_term_scale, oracle_ulp_sensitivity

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


def _nonplanar(itf, amp=1e-3, seed=9):
    itf.xm = itf.xm.copy()
    itf.xm[:, 2] += amp * inputs.uniform(seed, 0, itf.xm.shape[0], -1, 1)
    return itf


def cases():
    return [
        ("planar_8x7", inputs.planar_8x7(), 0),
        ("planar_8x7_seg", inputs.planar_8x7(), 1),
        ("planar_dual", inputs.planar_noisy(9, 8, 1, 41, "pd"), 0),
        ("mixed_small", inputs.mixed_tri(14, 19, name="mixed_small"), 0),
        ("mixed_small_dual_seg", inputs.mixed_tri(14, 19, lm=1, name="mds"), 1),
        ("cyl_dual", inputs.cylinder_patch(12, 10, name="cyl"), 0),
        ("cyl_dual_seg", inputs.cylinder_patch(12, 10, name="cyl"), 1),
        ("nonplanar_dual", _nonplanar(inputs.planar_noisy(8, 7, 1, 61, "np")), 0),
        ("tri_slave", _swap(inputs.mixed_tri(9, 7, name="ts")), 0),
        ("tri_slave_seg_dual", _swap(inputs.mixed_tri(9, 7, lm=1, name="tsd")), 1),
    ]


def _fields(itf, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(-1, 1, itf.xs.shape), rng.uniform(-1, 1, itf.xm.shape)


def _dense(orc, K, itf):
    Ns, Nm = itf.xs.shape[0], itf.xm.shape[0]
    return orc.bsr_dense(*K, Ns, Ns + Nm)


@pytest.mark.parametrize("name,itf,d_domain", cases(), ids=[c[0] for c in cases()])
def test_tangent_matches_oracle(mt, orc, name, itf, d_domain):
    ys, ym = _fields(itf, 11)
    m = mt.Mortar(lm=itf.lm, d_domain=d_domain, delta=itf.delta)
    m.set_interface(itf.xs, itf.conn_s, itf.xm, itf.conn_m)
    G = m.tangent(ys, ym)
    s, mm = m.pairs()
    o = orc.make_opts(lm=itf.lm, d_domain=d_domain, delta=itf.delta, n_threads=8)
    R = orc.tangent(itf, s, mm, ys, ym, o)
    assert G[0][-1] > 0
    sens = oracle_ulp_sensitivity(orc, itf, s, mm, ys, ym, o)
    assert sens < 2.5e-12, f"oracle ill-conditioned here: {sens:.2e}"
    tol = max(1e-12, 4 * sens)
    bsr_parity(G, R, tol)
    # direct terms: pattern unchanged, blocks differ by D (x) I3 and -M (x) I3
    Gd = m.tangent(ys, ym, add_direct=True)
    Rd = orc.tangent(itf, s, mm, ys, ym, o, add_direct=True)
    bsr_parity(Gd, Rd, tol)


CONSIST = [cases()[i] for i in (0, 2, 4, 7, 9)]


@pytest.mark.parametrize("name,itf,d_domain", CONSIST, ids=[c[0] for c in CONSIST])
def test_tangent_consistent_with_adjoint(mt, orc, name, itf, d_domain):
    """lambda^T (K(X) + [D (x) I3 | -M (x) I3]) equals the adjoint kernel's gradient."""
    m = mt.Mortar(lm=itf.lm, d_domain=d_domain, delta=itf.delta)
    m.set_interface(itf.xs, itf.conn_s, itf.xm, itf.conn_m)
    lam = np.random.default_rng(5).uniform(-1, 1, itf.xs.shape)
    K = _dense(orc, m.tangent(itf.xs, itf.xm, add_direct=True), itf)
    _, gs, gm = m.weighted_gap_grad(lam)
    s, mm = m.pairs()
    o = orc.make_opts(lm=itf.lm, d_domain=d_domain, delta=itf.delta, n_threads=8)
    scale = grad_term_scale(orc, itf, lam, s, mm, o)
    g = lam.ravel() @ K
    ref = np.concatenate([gs.ravel(), gm.ravel()])
    assert np.abs(g - ref).max() <= 1e-12 * scale


def test_tangent_invariants_and_determinism(mt, orc):
    """Euler (K X = 2 G), translation and rotation invariance on the GPU's own
    K and D, M; two runs bitwise equal."""
    itf = _nonplanar(inputs.cylinder_patch(10, 9, name="cinv"), amp=2e-3)
    ys, ym = _fields(itf, 3)
    m = mt.Mortar(lm=1, d_domain=0, delta=itf.delta)
    m.set_interface(itf.xs, itf.conn_s, itf.xm, itf.conn_m)
    K1 = m.tangent(ys, ym)
    K2 = m.tangent(ys, ym)
    for a, b in zip(K1, K2):
        assert np.array_equal(a, b)
    K = _dense(orc, K1, itf)
    Gv = m.scipy(0) @ ys - m.scipy(1) @ ym
    X = np.concatenate([itf.xs, itf.xm])
    scale = np.abs(K).max() * np.abs(X).max() * 24
    assert np.abs((K @ X.ravel()).reshape(-1, 3) - 2 * Gv).max() < 1e-12 * scale
    for w in np.eye(3):
        assert np.abs(K @ np.tile(w, X.shape[0])).max() < 1e-12 * scale
        assert np.abs(K @ np.cross(w, X).ravel()).max() < 1e-12 * scale


def test_tangent_edge_cases(mt):
    """No overlap at all: segment mode with standard LMs has no blocks, element
    mode keeps the element blocks; an interface without elements is empty."""
    itf = inputs.planar_noisy(4, 3, 0, 5, "far")
    itf.xm = itf.xm + np.array([5.0, 0.0, 0.0])
    ys, ym = _fields(itf, 1)
    m = mt.Mortar(lm=0, d_domain=1, delta=itf.delta)
    m.set_interface(itf.xs, itf.conn_s, itf.xm, itf.conn_m)
    rp, ci, va = m.tangent(ys, ym)
    assert rp[-1] == 0 and np.all(rp == 0)
    m = mt.Mortar(lm=0, d_domain=0, delta=itf.delta)
    m.set_interface(itf.xs, itf.conn_s, itf.xm, itf.conn_m)
    rp, ci, va = m.tangent(ys, ym)
    assert rp[-1] == sum(len({int(k) for e in range(16) if j in itf.conn_s[e] for k in itf.conn_s[e]})
                         for j in range(itf.xs.shape[0]))
    m = mt.Mortar(lm=1, d_domain=0, delta=1e-9)
    m.set_interface(np.zeros((0, 3)), np.zeros((0, 4), np.int32), itf.xm, itf.conn_m)
    rp, ci, va = m.tangent(np.zeros((0, 3)), ym)
    assert rp.shape == (1,) and len(ci) == 0


def test_tangent_batched(mt, orc):
    """A batch of independent interfaces: block rows of every interface equal
    the oracle's on the concatenated meshes (no pair crosses interfaces)."""
    itfs = inputs.batched_512(n_interfaces=6, n_hi=10.0)
    m = mt.Mortar(lm=0, d_domain=0, delta=1e-9)
    m.set_batch(itfs)
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
    ys, ym = _fields(big, 2)
    G = m.tangent(ys, ym)
    s, mm = m.pairs()
    R = orc.tangent(big, s, mm, ys, ym, orc.make_opts(lm=0, d_domain=0, delta=1e-9, n_threads=8))
    bsr_parity(G, R)


def _strip_parity(mt, orc, itf, d_domain, rows=(3, 7)):
    """Rows of slave nodes inside a strip of slave element rows: the GPU's K
    on the whole interface against the oracle on the strip's elements and pairs."""
    n = itf.info["ns"]
    ys, ym = _fields(itf, 9)
    m = mt.Mortar(lm=itf.lm, d_domain=d_domain, delta=itf.delta)
    m.set_interface(itf.xs, itf.conn_s, itf.xm, itf.conn_m)
    grp, gci, gva = m.tangent(ys, ym)
    s, mm = m.pairs()
    r0, r1 = rows
    elems = np.arange(r0 * n, r1 * n)                       # element rows r0 .. r1-1
    sel = (s >= elems[0]) & (s <= elems[-1])
    sub = inputs.Interface("strip", itf.xs, itf.conn_s[elems], itf.type_s, itf.xm, itf.conn_m,
                           itf.type_m, lm=itf.lm, delta=itf.delta)
    o = orc.make_opts(lm=itf.lm, d_domain=d_domain, delta=itf.delta, n_threads=16)
    rrp, rci, rva = orc.tangent(sub, s[sel] - elems[0], mm[sel], ys, ym, o)
    # slave nodes all of whose elements lie in the strip: node rows r0+1 .. r1-1
    nodes = np.concatenate([np.arange(j * (n + 1) + 1, j * (n + 1) + n) for j in range(r0 + 1, r1)])
    scale = np.abs(rva).max()
    for j in nodes:
        g = slice(grp[j], grp[j + 1])
        r = slice(rrp[j], rrp[j + 1])
        assert np.array_equal(gci[g], rci[r]), j
        rmax = max(np.abs(rva[r]).max(), 1e-2 * scale)
        assert np.abs(gva[g] - rva[r]).max() <= 1e-12 * rmax, j
    return len(nodes)


def test_tangent_sampled_rows_planar_600x520(mt, orc):
    assert _strip_parity(mt, orc, inputs.by_name("planar_600x520"), 0) > 1000


@pytest.mark.slow
def test_tangent_sampled_rows_planar_2000x1733(mt, orc):
    """Full size (14.9 M candidate pairs, 2.3 KB per pair of linearisation
    blocks on the device): rows of a strip of 4 element rows."""
    assert _strip_parity(mt, orc, inputs.planar_2000x1733(), 0, rows=(997, 1001)) > 5000
