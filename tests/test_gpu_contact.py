"""GPU contact-specific terms against the oracle: averaged nodal normals,
weighted normal gap, active set / complementarity residual, and the facing
test on candidate pairs (Sec. 2.1)."""
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


def _contact_pair(seed=9):
    """Flat slave at z = 0 (normal +z); above it a noisy, slightly wavy master
    whose first half of elements is reversed (normal -z, facing the slave)
    and whose second half keeps the slave's orientation."""
    base = inputs.planar_noisy(12, 10, 1, seed, "contact", noise=0.2)
    xm = base.xm.copy()
    xm[:, 2] = 0.004 + 0.002 * inputs.uniform(seed, 3, xm.shape[0], -1, 1)
    half = base.conn_m.shape[0] // 2
    cm = np.concatenate([base.conn_m[:half, ::-1], base.conn_m[half:]]).astype(np.int32)
    return inputs.Interface("contact", base.xs, base.conn_s, 4, xm, cm, 4, lm=1, delta=0.02)


def test_facing_test_pairs(mt, orc):
    itf = _contact_pair()
    m = mt.Mortar(lm=1, delta=itf.delta, facing_test=1)
    m.set_interface(itf.xs, itf.conn_s, itf.xm, itf.conn_m)
    n = m.search()
    s, mm = m.pairs()
    rs, rm = orc.facing_pairs(itf, *orc.search_bruteforce(itf))
    assert np.array_equal(s, rs) and np.array_equal(mm, rm)
    all_s, _ = orc.search_bruteforce(itf)
    assert 0 < n < len(all_s)


@pytest.mark.parametrize("case", ["planar_dual", "cylinder", "mixed", "tri_slave"])
def test_contact_terms_match_oracle(mt, orc, case):
    if case == "planar_dual":
        itf = inputs.planar_noisy(10, 9, 1, 7, "cp")
        itf.xm = itf.xm.copy()
        itf.xm[:, 2] = 0.01 + 0.003 * itf.xm[:, 0]
        itf.delta = 0.05
    elif case == "cylinder":
        itf = inputs.cylinder_patch(12, 10, name="cyl")
    elif case == "mixed":
        itf = inputs.mixed_tri(10, 13, name="mx")
    else:
        base = inputs.mixed_tri(9, 7, name="ts")
        itf = inputs.Interface("swap", base.xm, base.conn_m, base.type_m, base.xs, base.conn_s, base.type_s,
                               lm=0, delta=1e-9)
    m = mt.Mortar(lm=itf.lm, delta=itf.delta)
    m.set_interface(itf.xs, itf.conn_s, itf.xm, itf.conn_m)
    lam = np.random.default_rng(3).uniform(-1, 0.2, itf.xs.shape[0]) * 1e-2
    out = m.contact_terms(lam, c=50.0)
    nrm = orc.nodal_normals(itf)
    assert np.abs(out["normals"] - nrm).max() < 1e-14
    o = orc.make_opts(lm=itf.lm, delta=itf.delta)
    r = orc.evaluate(itf, o)
    g = orc.weighted_normal_gap(itf, r.D, r.M)
    scale = abs(r.D).max() * np.abs(itf.xs).max() + abs(r.M).max() * np.abs(itf.xm).max()
    assert np.abs(out["gap"] - g).max() <= 1e-13 * scale
    # the active-set decision taken in the same precision on the GPU's gap
    act, C = orc.ncp(lam, out["gap"], 50.0)
    assert np.array_equal(out["active"], act)
    assert np.array_equal(out["ncp"], C)
    # without multipliers: normals and gap only
    out2 = m.contact_terms()
    assert np.array_equal(out2["gap"], out["gap"])
