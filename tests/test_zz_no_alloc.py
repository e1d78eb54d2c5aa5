"""The no-allocation entry point (mortar_integrate_pairs_static) through the
C ABI, on two calls in a row: against the regular context path (the existing
entry point) and against the oracle's per-pair blocks.

Some callers of this library cannot call cudaMalloc: code inside a
device-memory allocator's own callback, where an allocation re-enters the
allocator, and processes whose device memory is reserved up front by a pool or
a fixed budget.  This entry point keeps its scratch in a static device array
instead.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_2202_03933_gb300 import inputs
from gpu_util import blocks_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2202_03933_gb300 import build, mortar
    build()
    return mortar


def _swap(itf, name):
    return inputs.Interface(name, itf.xm, itf.conn_m, itf.type_m, itf.xs, itf.conn_s, itf.type_s,
                            lm=itf.lm, delta=itf.delta)


def _cases():
    return [
        ("planar_dual", inputs.planar_noisy(60, 52, 1, 91, "p"), 0),
        ("planar_dual_segment", inputs.planar_noisy(40, 35, 1, 92, "ps"), 1),
        ("mixed_tri3_master", inputs.mixed_tri(50, 64, name="mx"), 0),
        ("tri3_slave_quad4_master", _swap(inputs.mixed_tri(24, 19, name="ts"), "ts"), 1),
        ("tri3_both", _tri_both(), 0),
    ]


def _tri_both():
    a = inputs.mixed_tri(18, 15, name="a")   # tri3 master of a 15x15 grid
    b = inputs.mixed_tri(13, 11, name="b")   # tri3 master of an 11x11 grid
    return inputs.Interface("tri3_both", a.xm, a.conn_m, 3, b.xm, b.conn_m, 3, lm=0, delta=1e-9)


@pytest.mark.parametrize("name,itf,d_domain", _cases(), ids=[c[0] for c in _cases()])
def test_static_entry_point_matches_context_path_and_oracle(mt, orc, name, itf, d_domain):
    import torch
    ref = mt.Mortar(lm=itf.lm, d_domain=d_domain, delta=itf.delta)
    ref.set_interface(itf.xs, itf.conn_s, itf.xm, itf.conn_m)
    ref.evaluate()
    s, m = ref.pairs()
    Mr, Dr, ner = ref.pair_blocks(with_D=d_domain == 1)
    Mo, Do, neo, _ = orc.pair_blocks(itf, s, m, orc.make_opts(lm=itf.lm, d_domain=d_domain, delta=itf.delta))
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    args = (dev(itf.xs), dev(itf.conn_s), dev(itf.xm), dev(itf.conn_m), dev(s), dev(m))
    for call in range(2):   # two calls in a row share the static scratch
        Mb, Db, ne = mt.integrate_pairs_static(*args, lm=itf.lm, d_domain=d_domain, delta=itf.delta)
        torch.cuda.synchronize()
        ne = ne.cpu().numpy().astype(bool)
        Mb = Mb.cpu().numpy()
        assert np.array_equal(ne, ner) and np.array_equal(ne, neo), call
        blocks_parity(Mb, Mr)    # the existing entry point
        blocks_parity(Mb, Mo)    # the oracle
        if d_domain == 1:
            Db = Db.cpu().numpy()
            blocks_parity(Db, Dr)
            blocks_parity(Db, Do)


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
    with pytest.raises(TypeError):   # int64 pair ids are refused by the binding, not misread
        mt.integrate_pairs_static(dev(itf.xs), dev(itf.conn_s), dev(itf.xm), dev(itf.conn_m),
                                  dev(s.astype(np.int64)), dev(m.astype(np.int64)))
