"""The no-allocation entry point (mortar_integrate_pairs_static) against the
regular context path, through the C ABI, on two calls in a row.

Some callers of this library cannot call cudaMalloc (code running during a
host framework's graph capture or inside an allocator callback, processes with
a device-memory budget fixed up front); this entry point keeps its scratch in a
static device array instead.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_2202_03933_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2202_03933_gb300 import build, mortar
    build()
    return mortar


def _cases():
    return [
        ("planar_dual", inputs.planar_noisy(60, 52, 1, 91, "p"), 0),
        ("planar_dual_segment", inputs.planar_noisy(40, 35, 1, 92, "ps"), 1),
        ("mixed_tri3_master", inputs.mixed_tri(50, 64, name="mx"), 0),
    ]


@pytest.mark.parametrize("name,itf,d_domain", _cases(), ids=[c[0] for c in _cases()])
def test_static_entry_point_matches_context_path(mt, name, itf, d_domain):
    import torch
    ref = mt.Mortar(lm=itf.lm, d_domain=d_domain, delta=itf.delta)
    ref.set_interface(itf.xs, itf.conn_s, itf.xm, itf.conn_m)
    ref.evaluate()
    s, m = ref.pairs()
    Mr, Dr, ner = ref.pair_blocks(with_D=d_domain == 1)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    args = (dev(itf.xs), dev(itf.conn_s), dev(itf.xm), dev(itf.conn_m), dev(s), dev(m))
    scale = np.abs(Mr).max()
    for call in range(2):   # two calls in a row share the static scratch
        Mb, Db, ne = mt.integrate_pairs_static(*args, lm=itf.lm, d_domain=d_domain, delta=itf.delta)
        torch.cuda.synchronize()
        assert np.array_equal(ne.cpu().numpy().astype(bool), ner), call
        assert np.abs(Mb.cpu().numpy() - Mr).max() <= 1e-12 * scale, call
        if d_domain == 1:
            assert np.abs(Db.cpu().numpy() - Dr).max() <= 1e-12 * np.abs(Dr).max(), call


def test_static_entry_point_rejects_oversize_and_bad_ids(mt):
    import torch
    L = mt.lib()
    o = mt.default_options()
    # more slave elements than the static scratch holds: refused before any launch
    r = L.mortar_integrate_pairs_static(ctypes.byref(o), None, None, 0, None, 8193, 4, None, 0, None, 0, 4,
                                        None, None, 0, None, None, None)
    assert r == -4
    itf = inputs.planar_noisy(6, 5, 0, 93, "bad")
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    s = np.array([0, 1, 99], np.int32)   # slave id 99 is out of range
    m = np.array([0, 0, 0], np.int32)
    with pytest.raises(mt._native.MortarError, match="INVALID_ARG"):
        mt.integrate_pairs_static(dev(itf.xs), dev(itf.conn_s), dev(itf.xm), dev(itf.conn_m), dev(s), dev(m))
