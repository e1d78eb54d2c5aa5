"""GPU parity of the adjoint kernel: gradient of J = sum_j lam_j.((D Xs)_j - (M Xm)_j).

Compared against the oracle's forward-mode (dual number) gradient to 1e-12
relative (max abs difference over the max abs reference gradient), against
central finite differences of the GPU's own J, and against exact invariants
(Euler homogeneity of degree 3, translation invariance on full coverage).
"""
import numpy as np
import pytest

from paper_2202_03933_gb300 import inputs
from gpu_util import grad_parity, grad_sensitivity, grad_term_scale

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
        ("mixed_small", inputs.mixed_tri(20, 27, name="mixed_small"), 0),
        ("mixed_small_dual_seg", inputs.mixed_tri(20, 27, lm=1, name="mds"), 1),
        ("cyl_dual", inputs.cylinder_patch(16, 13, name="cyl"), 0),
        ("cyl_dual_seg", inputs.cylinder_patch(16, 13, name="cyl"), 1),
        ("nonplanar_dual", _nonplanar(inputs.planar_noisy(10, 9, 1, 61, "np")), 0),
        ("tri_slave", _swap(inputs.mixed_tri(12, 9, name="ts")), 0),
        ("tri_slave_seg_dual", _swap(inputs.mixed_tri(12, 9, lm=1, name="tsd")), 1),
        ("kite_master_dual_seg", inputs.kite_master(16, 13, 0.45, lm=1), 1),
    ]


def _grad_parity(gs, gm, rs, rm, tol=1e-12, scale=None):
    scale = max(np.abs(rs).max(), np.abs(rm).max(), scale or 0.0)
    err = max(np.abs(gs - rs).max(), np.abs(gm - rm).max()) / scale
    assert err <= tol, f"gradient rel err {err:.3e}"
    return err


@pytest.mark.parametrize("name,itf,d_domain", cases(), ids=[c[0] for c in cases()])
def test_adjoint_matches_oracle(mt, orc, name, itf, d_domain):
    lam = np.random.default_rng(7).uniform(-1, 1, itf.xs.shape)
    m = mt.Mortar(lm=itf.lm, d_domain=d_domain, delta=itf.delta)
    m.set_interface(itf.xs, itf.conn_s, itf.xm, itf.conn_m)
    J, gs, gm = m.weighted_gap_grad(lam)
    o = orc.make_opts(lm=itf.lm, d_domain=d_domain, delta=itf.delta, n_threads=8)
    s, mm = m.pairs()
    Jr, rs, rm = orc.weighted_gap_grad(itf, lam, s, mm, o)
    scale = grad_term_scale(orc, itf, lam, s, mm, o)
    assert abs(J - Jr) <= 1e-12 * scale * np.abs(itf.xs).max()
    _grad_parity(gs, gm, rs, rm, scale=scale)


def test_adjoint_central_differences(mt):
    """GPU gradient against central differences of the GPU's own J (step 1e-6,
    64 coordinates) on a rotated tri3 master with a slightly non-planar master."""
    itf = _nonplanar(inputs.mixed_tri(24, 32, name="fd"), amp=2e-4)
    itf.delta = 1e-3
    lam = np.random.default_rng(3).uniform(-1, 1, itf.xs.shape)
    m = mt.Mortar(lm=0, delta=itf.delta)
    m.set_interface(itf.xs, itf.conn_s, itf.xm, itf.conn_m)
    J, gs, gm = m.weighted_gap_grad(lam)
    rng = np.random.default_rng(5)
    h = 1e-6
    scale = max(np.abs(gs).max(), np.abs(gm).max())
    for k in range(64):
        side = "s" if k % 2 == 0 else "m"
        X = itf.xs if side == "s" else itf.xm
        i = int(rng.integers(0, X.shape[0]))
        c = int(rng.integers(0, 3))
        x0 = X[i, c]
        vals = []
        for sgn in (1, -1):
            X[i, c] = x0 + sgn * h
            m.set_coordinates(itf.xs, itf.xm)
            vals.append(m.weighted_gap_grad(lam)[0])
        X[i, c] = x0
        fd = (vals[0] - vals[1]) / (2 * h)
        g = (gs if side == "s" else gm)[i, c]
        assert abs(fd - g) <= 1e-6 * scale, (side, i, c, fd, g)


@pytest.mark.parametrize("lm", [0, 1])
def test_adjoint_invariants(mt, lm):
    """Euler (J(sX) = s^3 J(X)) on a curved, fully covered interface, and
    translation invariance, which needs equal row sums of D and M: true in
    segment mode, where both integrate over the same auxiliary planes (with
    element-domain D on warped slave elements D integrates the curved
    element, M its flat projection)."""
    itf = inputs.planar_noisy(40, 35, lm, 71, "inv")
    itf.xm = itf.xm.copy()
    itf.xm[:, :2] = 0.5 + 1.08 * (itf.xm[:, :2] - 0.5)   # full coverage of the curved slave
    itf.xs = itf.xs.copy()
    itf.xs[:, 2] = 0.01 * np.sin(3 * itf.xs[:, 0]) * np.cos(2 * itf.xs[:, 1])   # curved slave
    itf.xm = itf.xm.copy()
    itf.xm[:, 2] = 0.01 * np.sin(3 * itf.xm[:, 0]) * np.cos(2 * itf.xm[:, 1]) + 1e-3
    itf.delta = 5e-3
    lam = np.random.default_rng(1).uniform(-1, 1, itf.xs.shape)
    m = mt.Mortar(lm=lm, d_domain=1, delta=itf.delta)
    m.set_interface(itf.xs, itf.conn_s, itf.xm, itf.conn_m)
    J, gs, gm = m.weighted_gap_grad(lam)
    scale = np.abs(gs).max() * np.abs(itf.xs).max()
    assert abs(J) > 1e-8
    assert abs(np.sum(itf.xs * gs) + np.sum(itf.xm * gm) - 3 * J) <= 1e-11 * scale   # Euler
    assert np.abs(gs.sum(0) + gm.sum(0)).max() <= 1e-11 * np.abs(gs).max()           # translation


def test_adjoint_deterministic_and_graph(mt):
    itf = inputs.mixed_tri(30, 40, lm=1, name="det")
    lam = np.random.default_rng(2).uniform(-1, 1, itf.xs.shape)
    a = mt.Mortar(lm=1, delta=itf.delta)
    a.set_interface(itf.xs, itf.conn_s, itf.xm, itf.conn_m)
    Ja, gsa, gma = a.weighted_gap_grad(lam)
    b = mt.Mortar(lm=1, delta=itf.delta)
    b.set_interface(itf.xs, itf.conn_s, itf.xm, itf.conn_m)
    b.run_graph(lam)
    b.run_graph(lam)
    Jb, gsb, gmb = b.gradient()
    assert Ja == Jb and np.array_equal(gsa, gsb) and np.array_equal(gma, gmb)


def test_autograd_function(mt, orc):
    import torch
    itf = inputs.mixed_tri(14, 18, name="ag")
    m = mt.Mortar(lm=0, delta=itf.delta)
    m.set_interface(itf.xs, itf.conn_s, itf.xm, itf.conn_m)
    xs = torch.tensor(itf.xs, device="cuda", requires_grad=True)
    xm = torch.tensor(itf.xm, device="cuda", requires_grad=True)
    lam = torch.tensor(np.random.default_rng(4).uniform(-1, 1, itf.xs.shape), device="cuda")
    J = mt.WeightedGap.apply(xs, xm, lam, m)
    (2.0 * J).backward()
    s, mm = m.pairs()
    Jr, rs, rm = orc.weighted_gap_grad(itf, lam.cpu().numpy(), s, mm)
    _grad_parity(xs.grad.cpu().numpy() / 2, xm.grad.cpu().numpy() / 2, rs, rm)


def test_full_size_mixed_adjoint(mt, orc):
    """mixed_300x400 with the adjoint: full gradient against the oracle."""
    itf = inputs.mixed_tri()
    lam = np.random.default_rng(8).uniform(-1, 1, itf.xs.shape)
    m = mt.Mortar(lm=0, delta=itf.delta)
    m.set_interface(itf.xs, itf.conn_s, itf.xm, itf.conn_m)
    m.run_graph(lam)
    m.run_graph(lam)
    J, gs, gm = m.gradient()
    s, mm = m.pairs()
    Jr, rs, rm = orc.weighted_gap_grad(itf, lam, s, mm, orc.make_opts(lm=0, delta=itf.delta, n_threads=16))
    _grad_parity(gs, gm, rs, rm)


def test_full_size_cylinder_adjoint(mt, orc):
    """cylinder_200x173 (curved, dual LMs) with the adjoint in its graph: the
    full gradient (lambda on every slave node) against the oracle's, at the
    two-term scale of R16 (the slave and master terms nearly cancel on the
    curved surface)."""
    import os
    itf = inputs.cylinder_patch()
    lam = np.random.default_rng(13).uniform(-1, 1, itf.xs.shape)
    m = mt.Mortar(lm=itf.lm, delta=itf.delta)
    m.set_interface(itf.xs, itf.conn_s, itf.xm, itf.conn_m)
    m.run_graph(lam)
    m.run_graph(lam)
    J, gs, gm = m.gradient()
    s, mm = m.pairs()
    o = orc.make_opts(lm=itf.lm, delta=itf.delta, n_threads=os.cpu_count() or 1)
    Jr, rs, rm = orc.weighted_gap_grad(itf, lam, s, mm, o)
    scale = grad_term_scale(orc, itf, lam, s, mm, o)
    grad_parity(gs, gm, rs, rm, scale, lambda: grad_sensitivity(orc, itf, lam, s, mm, o))
    assert abs(J - Jr) <= 1e-12 * (np.sum(np.abs(itf.xs * rs)) + np.sum(np.abs(itf.xm * rm)))


def test_full_size_mixed_central_differences(mt):
    """mixed_300x400 itself: the GPU gradient against central differences of
    the GPU's J at step 1e-6 on 64 random coordinates (half slave, half master).

    J = sum_j lam_j . r_j(X) and r_j depends on a coordinate X_i only through
    the pairs that contain node i, so the difference quotient of J equals that
    of J restricted to lam_j of the slave nodes within 3 slave element widths
    of node i (in the plane); the restriction keeps the rounding of the
    ~90,000 unaffected terms out of the quotient.  The gradient compared is
    the one of the full J."""
    itf = inputs.mixed_tri()
    lam = np.random.default_rng(17).uniform(-1, 1, itf.xs.shape)
    m = mt.Mortar(lm=0, delta=itf.delta)
    m.set_interface(itf.xs, itf.conn_s, itf.xm, itf.conn_m)
    J, gs, gm = m.weighted_gap_grad(lam)
    scale = max(np.abs(gs).max(), np.abs(gm).max())
    hs = 1.0 / itf.info["ns"]
    rng = np.random.default_rng(19)
    h = 1e-6
    xs0, xm0 = itf.xs.copy(), itf.xm.copy()
    worst = 0.0
    for k in range(64):
        side = "s" if k % 2 == 0 else "m"
        X = xs0 if side == "s" else xm0
        i = int(rng.integers(0, X.shape[0]))
        c = int(rng.integers(0, 3))
        near = np.hypot(xs0[:, 0] - X[i, 0], xs0[:, 1] - X[i, 1]) <= 3.0 * hs
        lam_loc = np.where(near[:, None], lam, 0.0)
        vals = []
        for sgn in (1, -1):
            xs, xm = xs0.copy(), xm0.copy()
            (xs if side == "s" else xm)[i, c] += sgn * h
            m.set_coordinates(xs, xm)
            vals.append(m.weighted_gap_grad(lam_loc)[0])
        fd = (vals[0] - vals[1]) / (2 * h)
        g = (gs if side == "s" else gm)[i, c]
        worst = max(worst, abs(fd - g) / scale)
        assert abs(fd - g) <= 1e-6 * scale, (side, i, c, fd, g)
    m.set_coordinates(xs0, xm0)


def test_full_size_planar_2000_adjoint_sampled(mt, orc):
    """The benchmark workload with lambda nonzero on a scattered 0.5 % of slave
    nodes: the oracle then needs only the pairs of slave elements touching
    them, and the full GPU gradient must equal the oracle's everywhere."""
    itf = inputs.planar_2000x1733()
    rng = np.random.default_rng(12)
    lam = np.zeros_like(itf.xs)
    pick = rng.choice(itf.xs.shape[0], itf.xs.shape[0] // 200, replace=False)
    lam[pick] = rng.uniform(-1, 1, (pick.size, 3))
    m = mt.Mortar(lm=itf.lm, delta=itf.delta)
    m.set_interface(itf.xs, itf.conn_s, itf.xm, itf.conn_m)
    m.run_graph(lam)
    m.run_graph(lam)
    J, gs, gm = m.gradient()
    s, mm = m.pairs()
    active = (lam != 0).any(axis=1)
    keep = active[np.asarray(itf.conn_s)[s]].any(axis=1)
    o = orc.make_opts(lm=itf.lm, delta=itf.delta, n_threads=16)
    Jr, rs, rm = orc.weighted_gap_grad(itf, lam, s[keep], mm[keep], o)
    _grad_parity(gs, gm, rs, rm)
    assert abs(J - Jr) <= 1e-12 * np.abs(rs).max()


@pytest.mark.parametrize("variant,rounds,block", [(1, 0, 64), (1, 0, 256), (0, 1, 256), (0, 4, 64), (0, 8, 128),
                                                  (0, 16, 256), (0, 32, 64), (0, 32, 256)])
def test_adjoint_launch_variants(mt, orc, variant, rounds, block):
    """Both adjoint schedules give the oracle's gradient (bilinear and tri3
    masters, dual segment mode, warped slave)."""
    warped = inputs.planar_noisy(13, 11, 1, 46, "w")
    warped.xs = warped.xs.copy()
    warped.xs[:, 2] = 0.02 * np.sin(5 * warped.xs[:, 0]) * np.cos(3 * warped.xs[:, 1])
    warped.xm = warped.xm.copy()
    warped.xm[:, 2] = 0.02 * np.sin(5 * warped.xm[:, 0]) * np.cos(3 * warped.xm[:, 1]) + 1e-3
    warped.delta = 5e-3
    for itf, d_domain in ((inputs.planar_noisy(15, 13, 1, 47, "v"), 1), (inputs.mixed_tri(16, 21, name="t"), 0),
                          (warped, 0)):
        lam = np.random.default_rng(9).uniform(-1, 1, itf.xs.shape)
        m = mt.Mortar(lm=itf.lm, d_domain=d_domain, delta=itf.delta)
        m.set_interface(itf.xs, itf.conn_s, itf.xm, itf.conn_m)
        m.set_launch(variant=variant, block_size=block, rounds=rounds)
        J, gs, gm = m.weighted_gap_grad(lam)
        s, mm = m.pairs()
        o = orc.make_opts(lm=itf.lm, d_domain=d_domain, delta=itf.delta, n_threads=8)
        Jr, rs, rm = orc.weighted_gap_grad(itf, lam, s, mm, o)
        _grad_parity(gs, gm, rs, rm, scale=grad_term_scale(orc, itf, lam, s, mm, o))
