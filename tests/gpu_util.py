"""Helpers shared by the GPU parity tests (comparison only; no method arithmetic)."""
import numpy as np


ENTRY_FLOOR = 1e-8     # entries checked one by one: |ref| >= ENTRY_FLOOR * max|ref|
# Multiple of the oracle's own per-entry rounding sensitivity allowed where an
# entry is ill-conditioned.  A one-ulp perturbation of the inputs emulates one
# layer of rounding; each entry is the result of 10^2 - 10^3 rounded
# operations (back-projections, shape functions, 7-point sums over the cells,
# the product with the dual coefficients), and the measured GPU-vs-oracle
# deviation of the ill-conditioned entries is up to 20x the one-ulp figure.
SENS_FACTOR = 64.0


class EntrywiseError(AssertionError):
    """The entrywise relative check failed (and no sensitivity was supplied)."""


def csr_parity(G, R, tol=1e-12, sens=None):
    """GPU-vs-oracle parity of one CSR matrix.

    * identical pattern;
    * max|G - R| / max|R| <= tol;
    * every entry with |R_e| >= ENTRY_FLOOR max|R| within tol of itself:
      |G_e - R_e| <= tol |R_e| -- or, where ``sens`` (the oracle's own change of
      each entry under random 1-ulp perturbations of all input coordinates,
      aligned with R's pattern) is given, within max(tol |R_e|, SENS_FACTOR
      sens_e): entries whose value the input rounding alone already moves by
      more than tol relative (dual-basis cancellations, sliver polygons at
      near-parallel edges) are held to their own conditioning;
    * every row within tol of its own largest reference entry, floored at 1 %
      of max|R| (catches errors confined to rows of small values).
    Returns the max relative error."""
    assert G.shape == R.shape
    assert np.array_equal(G.indptr, R.indptr), "row pointers differ"
    assert np.array_equal(G.indices, R.indices), "column indices differ"
    if R.nnz == 0:
        assert G.nnz == 0
        return 0.0
    scale = np.abs(R.data).max()
    dif = np.abs(G.data - R.data)
    err = dif.max() / scale
    assert err <= tol, f"max rel err {err:.3e} > {tol}"
    rows = np.repeat(np.arange(R.shape[0]), np.diff(R.indptr))
    rmax = np.zeros(R.shape[0])
    np.maximum.at(rmax, rows, np.abs(R.data))
    rel_row = dif / np.maximum(rmax[rows], 1e-2 * scale)
    assert rel_row.max() <= tol, f"row-relative err {rel_row.max():.3e}"
    big = np.abs(R.data) >= ENTRY_FLOOR * scale
    bound = tol * np.abs(R.data)
    if sens is not None:
        bound = np.maximum(bound, SENS_FACTOR * np.asarray(sens))
    bad = big & (dif > bound)
    if bad.any():
        i = np.flatnonzero(bad)[np.argmax(dif[bad] / np.abs(R.data[bad]))]
        msg = (f"entrywise: {int(bad.sum())} entries; worst row {rows[i]} col {R.indices[i]}: "
               f"ref {R.data[i]:.6e}, rel err {dif[i] / abs(R.data[i]):.3e}"
               + ("" if sens is None else f", oracle sensitivity {sens[i] / abs(R.data[i]):.3e} rel"))
        raise EntrywiseError(msg)
    return err


def oracle_sensitivity(ref_fn, itf, refs, trials=3, seed=0):
    """Per-entry rounding sensitivity of oracle matrices: the largest change of
    each entry of ``refs`` (CSR matrices from ``ref_fn(itf)``) when every input
    coordinate is perturbed by one unit in the last place (random signs),
    over ``trials`` perturbations; aligned with each matrix's pattern."""
    rng = np.random.default_rng(seed)
    xs0, xm0 = itf.xs.copy(), itf.xm.copy()
    out = [np.zeros(R.nnz) for R in refs]
    keys = []
    for R in refs:
        r = np.repeat(np.arange(R.shape[0]), np.diff(R.indptr))
        keys.append((r, R.indices))
    try:
        for _ in range(trials):
            itf.xs = xs0 * (1 + 2.2e-16 * rng.choice([-1.0, 1.0], xs0.shape))
            itf.xm = xm0 * (1 + 2.2e-16 * rng.choice([-1.0, 1.0], xm0.shape))
            for k, P in enumerate(ref_fn(itf)):
                d = (P - refs[k]).tocsr()
                if d.nnz:
                    v = np.abs(np.asarray(d[keys[k][0], keys[k][1]]).ravel())
                    out[k] = np.maximum(out[k], v)
    finally:
        itf.xs, itf.xm = xs0, xm0
    return out


def forward_parity(GD, GM, RD, RM, ref_fn, itf, tol=1e-12):
    """csr_parity of D and M.  The strict entrywise check is tried first; where
    it fails, the oracle's own per-entry sensitivity is measured (``ref_fn(itf)``
    recomputes the reference (D, M) at itf's current coordinates) and the
    check is repeated against it.  Returns the number of entries that needed
    their measured sensitivity."""
    try:
        csr_parity(GD, RD, tol)
        csr_parity(GM, RM, tol)
        return 0
    except EntrywiseError:
        pass
    sD, sM = oracle_sensitivity(ref_fn, itf, (RD, RM))
    csr_parity(GD, RD, tol, sens=sD)
    csr_parity(GM, RM, tol, sens=sM)
    n = 0
    for G, R in ((GD, RD), (GM, RM)):
        if R.nnz:
            big = np.abs(R.data) >= ENTRY_FLOOR * np.abs(R.data).max()
            n += int((big & (np.abs(G.data - R.data) > tol * np.abs(R.data))).sum())
    return n


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


def grad_sensitivity(orc, itf, lam, s, m, o, trials=4, seed=0):
    """Per-entry rounding sensitivity of the oracle's weighted-gap gradient:
    the largest change of each entry when every input coordinate is perturbed
    by one unit in the last place (random signs), over ``trials``."""
    rng = np.random.default_rng(seed)
    _, gs0, gm0 = orc.weighted_gap_grad(itf, lam, s, m, o)
    xs0, xm0 = itf.xs.copy(), itf.xm.copy()
    ss, sm = np.zeros_like(gs0), np.zeros_like(gm0)
    try:
        for _ in range(trials):
            itf.xs = xs0 * (1 + 2.2e-16 * rng.choice([-1.0, 1.0], xs0.shape))
            itf.xm = xm0 * (1 + 2.2e-16 * rng.choice([-1.0, 1.0], xm0.shape))
            _, gs, gm = orc.weighted_gap_grad(itf, lam, s, m, o)
            ss = np.maximum(ss, np.abs(gs - gs0))
            sm = np.maximum(sm, np.abs(gm - gm0))
    finally:
        itf.xs, itf.xm = xs0, xm0
    return ss, sm


def grad_parity(gs, gm, rs, rm, scale, sens_fn=None, tol=1e-12):
    """Gradient parity: every entry within tol * scale of the oracle's
    gradient; where that fails and ``sens_fn()`` gives the oracle's own
    per-entry one-ulp sensitivity (ss, sm), within max(tol * scale,
    SENS_FACTOR * sensitivity).  Returns the max error relative to scale."""
    dif_s, dif_m = np.abs(gs - rs), np.abs(gm - rm)
    err = max(dif_s.max(initial=0.0), dif_m.max(initial=0.0)) / scale
    if err <= tol:
        return err
    assert sens_fn is not None, f"gradient rel err {err:.3e}"
    ss, sm = sens_fn()
    ok_s = dif_s <= np.maximum(tol * scale, SENS_FACTOR * ss)
    ok_m = dif_m <= np.maximum(tol * scale, SENS_FACTOR * sm)
    big_s, big_m = dif_s > tol * scale, dif_m > tol * scale
    ratio = max((dif_s[big_s] / np.maximum(ss[big_s], 1e-300)).max(initial=0.0),
                (dif_m[big_m] / np.maximum(sm[big_m], 1e-300)).max(initial=0.0))
    assert ok_s.all() and ok_m.all(), (
        f"gradient rel err {err:.3e}; beyond the oracle's sensitivity at "
        f"{int((~ok_s).sum()) + int((~ok_m).sum())} entries (largest deviation / sensitivity {ratio:.1f}, "
        f"deviations {np.concatenate([dif_s[~ok_s], dif_m[~ok_m]]) / scale} of the scale)")
    return err
