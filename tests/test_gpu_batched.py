"""Batched uneven interfaces against the oracle, interface by interface.

The workload: 512 independent planar quad4/quad4 interfaces with n x n slave
elements, n log-uniform in [4, 128], master resolution ratio U(0.7, 1.3) and a
random in-plane offset per interface (inputs.batched_512).  One context holds
all of them: one search, one persistent pair kernel over all pairs, one CUDA
graph, with the launch shape picked by the library's autotuner.  Pairs never
cross interfaces, so D and M are block diagonal and the gradient of the
weighted gap splits into independent per-interface gradients.

Every one of the 512 interfaces is compared with the oracle: the pair set
exactly, the D and M blocks at the CSR parity tolerance, and the gradient of
lambda.(D Xs - M Xm) (lambda ~ U(-1, 1) per component of every slave node) at
1e-12 of the interface's largest reference gradient entry.  This is the
load-imbalance setting of the paper's dynamic rebalancing (Sec. 4.4, the
imbalance measure eta_t), run on one GPU.
"""
import os

import numpy as np
import pytest

from paper_2202_03933_gb300 import inputs
from gpu_util import forward_parity

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def mt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2202_03933_gb300 import build, mortar
    build()
    return mortar


@pytest.fixture(scope="module")
def batch():
    itfs = inputs.batched_512()
    n_s = sum(i.xs.shape[0] for i in itfs)
    lam = np.random.default_rng(2202).uniform(-1.0, 1.0, (n_s, 3))
    return itfs, lam


def _dm(res):
    return res.D, res.M


def _interface_pairs(s, m, se, me, k):
    lo, hi = np.searchsorted(s, [se[k], se[k + 1]])
    return s[lo:hi] - se[k], m[lo:hi] - me[k]


def _off_block_free(M, row_off, col_off):
    """No entry of M lies outside the diagonal interface blocks."""
    rows = np.repeat(np.arange(M.shape[0]), np.diff(M.indptr))
    blk_r = np.searchsorted(row_off, rows, side="right") - 1
    blk_c = np.searchsorted(col_off, M.indices, side="right") - 1
    return np.array_equal(blk_r, blk_c)


def test_batched_512_forward_and_adjoint_parity(mt, orc, batch):
    itfs, lam = batch
    m = mt.Mortar(lm=0, delta=1e-9)
    m.set_batch(itfs)
    pick = m.autotune(lam)
    assert pick["variant"] in (0, 1) and pick["ms"] > 0
    m.run_graph(lam)   # eager run, then capture
    m.run_graph(lam)   # graph replay
    J, gs, gm = m.gradient()
    s, mm = m.pairs()
    D = m.scipy(mt.MATRIX_D)
    M = m.scipy(mt.MATRIX_M)
    sn, se = m.offsets["slave_nodes"], m.offsets["slave_elems"]
    mn, me = m.offsets["master_nodes"], m.offsets["master_elems"]
    assert _off_block_free(M, sn, mn) and _off_block_free(D, sn, sn)
    o = orc.make_opts(lm=0, delta=1e-9, n_threads=os.cpu_count() or 1)
    J_ref = 0.0
    J_scale = 0.0
    for k, itf in enumerate(itfs):
        ks, km = _interface_pairs(s, mm, se, me, k)
        rs, rm = orc.search_binned(itf)
        assert np.array_equal(ks, rs) and np.array_equal(km, rm), k
        ref = orc.evaluate(itf, o, pairs=(rs, rm))
        forward_parity(D[sn[k]:sn[k + 1], sn[k]:sn[k + 1]], M[sn[k]:sn[k + 1], mn[k]:mn[k + 1]], ref.D, ref.M,
                       lambda x: _dm(orc.evaluate(x, o, pairs=(rs, rm))), itf)
        Jk, gsk, gmk = orc.weighted_gap_grad(itf, lam[sn[k]:sn[k + 1]], rs, rm, o)
        scale = max(np.abs(gsk).max(), np.abs(gmk).max())
        err = max(np.abs(gs[sn[k]:sn[k + 1]] - gsk).max(), np.abs(gm[mn[k]:mn[k + 1]] - gmk).max()) / scale
        assert err <= 1e-12, f"interface {k}: gradient rel err {err:.3e}"
        J_ref += Jk
        # Euler homogeneity (J is of degree 3 in the coordinates: sum X.g = 3 J)
        # puts J's rounding on the scale of sum |X| |g|
        J_scale += np.sum(np.abs(itf.xs * gsk)) + np.sum(np.abs(itf.xm * gmk))
    assert abs(J - J_ref) <= 1e-12 * J_scale
    st = m.stats()
    assert st["n_interfaces"] == 512 and st["n_newton_fail"] == 0 and st["n_clip_overflow"] == 0


def test_batched_512_forward_graph_parity(mt, orc, batch):
    """The forward-only graph of the same batch (the integration kernel, not the
    fused adjoint) with its own autotuned launch shape."""
    itfs, _ = batch
    m = mt.Mortar(lm=0, delta=1e-9)
    m.set_batch(itfs)
    m.autotune()
    m.run_graph()
    m.run_graph()
    D = m.scipy(mt.MATRIX_D)
    M = m.scipy(mt.MATRIX_M)
    sn, mn = m.offsets["slave_nodes"], m.offsets["master_nodes"]
    o = orc.make_opts(lm=0, delta=1e-9, n_threads=os.cpu_count() or 1)
    for k, itf in enumerate(itfs):
        ref = orc.evaluate(itf, o)
        forward_parity(D[sn[k]:sn[k + 1], sn[k]:sn[k + 1]], M[sn[k]:sn[k + 1], mn[k]:mn[k + 1]], ref.D, ref.M,
                       lambda x: _dm(orc.evaluate(x, o, pairs=(ref.s, ref.m))), itf)
    assert _off_block_free(M, sn, mn)
