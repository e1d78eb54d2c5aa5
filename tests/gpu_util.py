"""Helpers shared by the GPU parity tests (comparison only; no method arithmetic)."""
import numpy as np


def csr_parity(G, R, tol=1e-12):
    """Identical CSR pattern; max|G - R| / max|R| <= tol, and the same bound
    row by row against each row's largest entry.  Returns the max relative error."""
    assert G.shape == R.shape
    assert np.array_equal(G.indptr, R.indptr), "row pointers differ"
    assert np.array_equal(G.indices, R.indices), "column indices differ"
    if R.nnz == 0:
        assert G.nnz == 0
        return 0.0
    scale = np.abs(R.data).max()
    err = np.abs(G.data - R.data).max() / scale
    assert err <= tol, f"max rel err {err:.3e} > {tol}"
    # row-relative: every row within tol of its own largest reference entry
    # (catches errors in rows of small values, e.g. partially covered rows;
    # a per-entry relative bound would flag entries that are sums with heavy
    # cancellation, which carry rounding of the size of their terms)
    rows = np.repeat(np.arange(R.shape[0]), np.diff(R.indptr))
    rmax = np.zeros(R.shape[0])
    np.maximum.at(rmax, rows, np.abs(R.data))
    dif = np.abs(G.data - R.data)
    rel_row = dif / np.where(rmax[rows] > 0, rmax[rows], scale)
    assert rel_row.max() <= tol, f"row-relative err {rel_row.max():.3e}"
    return err


def blocks_parity(Gb, Rb, tol=1e-12):
    scale = max(np.abs(Rb).max(), 1e-300)
    err = np.abs(Gb - Rb).max() / scale
    assert err <= tol, f"pair blocks rel err {err:.3e}"
    return err
