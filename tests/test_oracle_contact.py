"""Pins of the oracle's contact-specific terms (no GPU needed).

Averaged nodal normals, the facing test on candidate pairs, the weighted
normal gap g_j = -n_j . ((D Xs)_j - (M Xm)_j) and the active set / residual of
the Hertz-Signorini-Moreau conditions (Sec. 2.1), each against a closed form
or a definition written here in numpy.
"""
import math

import numpy as np
import pytest

from paper_2202_03933_gb300 import inputs


def test_nodal_normals_flat_and_cylinder(orc):
    itf = inputs.planar_noisy(6, 5, 0, 3, "nf")
    n = orc.nodal_normals(itf)
    assert np.abs(n - np.array([0.0, 0.0, 1.0])).max() < 1e-15
    # chord quads of a cylinder: at interior nodes the two adjacent chords'
    # normals are mirror images about the radial direction, so their
    # average is radial; boundary columns see one chord (normal tilted by
    # half the chord angle)
    k = 8
    itf = inputs.cylinder_patch(k, 7)
    n = orc.nodal_normals(itf)
    r = itf.xs.copy()
    r[:, 2] = 0.0
    r /= np.linalg.norm(r, axis=1)[:, None]
    col = np.arange(itf.xs.shape[0]) % (k + 1)
    inner = (col > 0) & (col < k)
    assert np.abs(n[inner] - r[inner]).max() < 1e-15
    tilt = np.arccos(np.clip(np.einsum("ij,ij->i", n[~inner], r[~inner]), -1, 1))
    assert np.allclose(tilt, 0.25 * math.pi / k, atol=1e-12)


def _element_normal_numpy(X):
    """Unit normal at the centre of a quad (diagonal cross product) or triangle."""
    if len(X) == 4:
        n = np.cross(X[2] - X[0], X[3] - X[1])
    else:
        n = np.cross(X[1] - X[0], X[2] - X[0])
    return n / np.linalg.norm(n)


def test_facing_pairs_definition(orc):
    """Slave at z = 0 (normal +z); a master sheet above it with reversed node
    order (normal -z: facing) and one with the slave's orientation."""
    base = inputs.planar_noisy(5, 4, 0, 9, "fc", noise=0.2)
    xm = base.xm.copy()
    xm[:, 2] = 0.01 + 0.002 * inputs.uniform(9, 3, xm.shape[0], -1, 1)
    cm_face = base.conn_m[:, ::-1].copy()
    cm = np.concatenate([cm_face[::2], base.conn_m[1::2]]).astype(np.int32)
    itf = inputs.Interface("facing", base.xs, base.conn_s, 4, xm, cm, 4, lm=0, delta=0.05)
    s, m = orc.search_bruteforce(itf)
    fs, fm = orc.facing_pairs(itf, s, m)
    keep = [p for p in range(len(s))
            if _element_normal_numpy(itf.xs[itf.conn_s[s[p]]]) @ _element_normal_numpy(itf.xm[cm[m[p]]]) < 0]
    assert np.array_equal(fs, s[keep]) and np.array_equal(fm, m[keep])
    assert 0 < len(fs) < len(s)
    assert np.all(fm < cm_face[::2].shape[0])          # exactly the reversed (facing) half


@pytest.mark.parametrize("lm", [0, 1])
def test_weighted_gap_parallel_and_tilted_planes(orc, lm):
    """Master at z = a + b x + c y over a flat slave at z = 0 (full coverage):
    M reproduces the linear field, so g = D (a + b xs + c ys) exactly; for a
    parallel plane g_j = a sum_k D_jk."""
    for a, b, c in ((0.02, 0.0, 0.0), (0.02, 0.01, -0.015)):
        itf = inputs.planar_noisy(7, 6, lm, 13, "gap")
        itf.xm = itf.xm.copy()
        itf.xm[:, 2] = a + b * itf.xm[:, 0] + c * itf.xm[:, 1]
        o = orc.make_opts(lm=lm, delta=0.05)
        r = orc.evaluate(itf, o)
        g = orc.weighted_normal_gap(itf, r.D, r.M)
        ref = r.D @ (a + b * itf.xs[:, 0] + c * itf.xs[:, 1])
        assert np.abs(g - ref).max() < 1e-15
        if b == 0.0:
            assert np.abs(g - a * np.asarray(r.D.sum(axis=1)).ravel()).max() < 1e-16


def test_ncp_cases(orc):
    """Active where lam + c g < 0; the residual vanishes exactly on points that
    satisfy the conditions (g >= 0, lam <= 0, g lam = 0)."""
    lam = np.array([0.0, 0.0, -2.0, -1.0, 0.5, -0.5, 0.0])
    gap = np.array([0.3, 0.0, 0.0, 0.2, 0.0, -0.1, -0.4])
    active, C = orc.ncp(lam, gap, 10.0)
    assert active.tolist() == [False, False, True, False, False, True, True]
    ok = (gap >= 0) & (lam <= 0) & (gap * lam == 0)
    assert np.all(C[ok] == 0.0)
    assert np.all(C[~ok] != 0.0)
    assert C[3] == -1.0 and C[4] == 0.5 and C[5] == 1.0 and C[6] == 4.0
