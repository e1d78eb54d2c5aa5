"""Helpers shared by the GPU parity tests (comparison only; no method arithmetic)."""
import numpy as np


def csr_parity(G, R, tol=1e-12):
    """Identical CSR pattern; max|G - R| / max|R| <= tol, and the same bound
    row by row against each row's largest entry (floored at 1 % of max|R|).
    Returns the max relative error."""
    assert G.shape == R.shape
    assert np.array_equal(G.indptr, R.indptr), "row pointers differ"
    assert np.array_equal(G.indices, R.indices), "column indices differ"
    if R.nnz == 0:
        assert G.nnz == 0
        return 0.0
    scale = np.abs(R.data).max()
    err = np.abs(G.data - R.data).max() / scale
    assert err <= tol, f"max rel err {err:.3e} > {tol}"
    # row-relative: every row within tol of its own largest reference entry,
    # floored at 1 % of the global scale.  This catches errors confined to
    # rows of small values; the floor keeps sliver rows (a node barely
    # covered at a boundary: entries built from polygons much smaller than
    # the element, whose rounding is relative to the element size) from being
    # held to a bound below their own rounding.  A per-entry relative bound
    # would likewise flag entries that are sums with heavy cancellation.
    rows = np.repeat(np.arange(R.shape[0]), np.diff(R.indptr))
    rmax = np.zeros(R.shape[0])
    np.maximum.at(rmax, rows, np.abs(R.data))
    dif = np.abs(G.data - R.data)
    rel_row = dif / np.maximum(rmax[rows], 1e-2 * scale)
    assert rel_row.max() <= tol, f"row-relative err {rel_row.max():.3e}"
    return err


def blocks_parity(Gb, Rb, tol=1e-12):
    scale = max(np.abs(Rb).max(), 1e-300)
    err = np.abs(Gb - Rb).max() / scale
    assert err <= tol, f"pair blocks rel err {err:.3e}"
    return err


def grad_term_scale(orc, itf, lam, s, m, o):
    """Scale of the weighted-gap gradient: the larger max-abs gradient of its
    two terms lam.D Xs and lam.M Xm, each computed alone by the oracle.

    J is their difference; where the two nearly cancel (x_s and x_m are the
    two surfaces at the same projected point) the rounding of the result is
    relative to the terms, not to their difference."""
    scale = 0.0
    for terms in (1, 2):
        o.terms = terms
        _, gs, gm = orc.weighted_gap_grad(itf, lam, s, m, o)
        scale = max(scale, np.abs(gs).max(), np.abs(gm).max())
    o.terms = 3
    return scale


def oracle_ulp_sensitivity(orc, itf, s, m, ys, ym, o, trials=4, seed=0):
    """Largest block-row-relative change of the oracle's own K when every input
    coordinate is perturbed by one unit in the last place (random signs): the
    rounding-level conditioning of K at this configuration."""
    R = orc.tangent(itf, s, m, ys, ym, o)
    rng = np.random.default_rng(seed)
    xs0, xm0 = itf.xs.copy(), itf.xm.copy()
    worst = 0.0
    try:
        for _ in range(trials):
            itf.xs = xs0 * (1 + 2.2e-16 * rng.choice([-1.0, 1.0], xs0.shape))
            itf.xm = xm0 * (1 + 2.2e-16 * rng.choice([-1.0, 1.0], xm0.shape))
            worst = max(worst, bsr_parity(orc.tangent(itf, s, m, ys, ym, o), R, tol=np.inf))
    finally:
        itf.xs, itf.xm = xs0, xm0
    return worst


def bsr_parity(G, R, tol=1e-12):
    """Identical block pattern (rowptr, colidx) of two 3x3-block BSR triples;
    every block row within tol of its own largest reference entry, floored at
    1 % of the global largest (as csr_parity).  Returns the max row-relative
    error."""
    grp, gci, gva = G
    rrp, rci, rva = R
    assert np.array_equal(grp, rrp), "block row pointers differ"
    assert np.array_equal(gci, rci), "block column indices differ"
    if rva.shape[0] == 0:
        return 0.0
    scale = np.abs(rva).max()
    rows = np.repeat(np.arange(len(rrp) - 1), np.diff(rrp))
    rmax = np.zeros(len(rrp) - 1)
    np.maximum.at(rmax, rows, np.abs(rva).reshape(-1, 9).max(axis=1))
    dif = np.abs(gva - rva).reshape(-1, 9).max(axis=1)
    rel = dif / np.maximum(rmax[rows], 1e-2 * scale)
    assert rel.max() <= tol, f"block-row-relative err {rel.max():.3e} (row {rows[rel.argmax()]})"
    return float(rel.max())
