"""CPU oracle for segment-based mortar integration -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never calls it and shares no code with it.

The arithmetic lives in ``mortar_oracle.cpp`` (plain C++, FP64, one pair at a
time, compiled with ``-ffp-contract=off`` so that x86 and Arm give the same
bits).  This module compiles it, wraps it with ctypes and performs the final
assembly of the per-pair blocks into CSR matrices (Eq. DiscreteWeakFormInterfaceFlux:
D and M are assembled from nodal blocks) with plain numpy/scipy steps.

Parity status per function (how each is pinned is in ``tests/test_oracle_*.py``):
  search_bruteforce / search_binned  -- pinned (definition; exact set equality)
  element_blocks (dual basis, D_e)   -- pinned (closed forms, biorthogonality)
  pair_blocks / evaluate             -- pinned where closed forms exist (areas,
      row sums, matching meshes, tensor grids, affine masters, linear-field
      reproduction); entries of M for non-affine noisy masters have no closed
      form beyond those invariants
  weighted_gap_grad                  -- pinned (finite differences, Euler
      homogeneity, translation invariance)
  quadratic_element_D / quadratic_pair_blocks (tri6, quad8 slaves) -- pinned
      (shape-function identities, element D against an independent
      high-order rule, slave area, linear-field reproduction, row sums, the
      overlap area, sub-elements coinciding with master elements)
  element_based_blocks / evaluate_element_based -- pinned (exact slave area
      and linear-field reproduction on full coverage, matching meshes, a
      brute-force point location over all master elements, convergence to the
      segment-based result)
  nodal_normals / facing_pairs / weighted_normal_gap / ncp -- pinned (flat
      and cylindrical closed forms, parallel and tilted planes, numpy
      definitions, complementarity cases)
  tangent                            -- pinned (finite differences, Euler
      homogeneity, translation and rotation invariance, a closed-form
      overlap-area derivative, consistency with weighted_gap_grad)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mortar_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library (g++, OpenMP, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Opts(ctypes.Structure):
    _fields_ = [("lm", ctypes.c_int32), ("d_domain", ctypes.c_int32),
                ("tri_rule", ctypes.c_int32), ("fan", ctypes.c_int32),
                ("newton_max_iter", ctypes.c_int32), ("n_threads", ctypes.c_int32),
                ("terms", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("delta", ctypes.c_double), ("newton_tol", ctypes.c_double),
                ("clip_tol_rel", ctypes.c_double), ("merge_tol_rel", ctypes.c_double),
                ("area_tol_rel", ctypes.c_double)]


def make_opts(lm=0, d_domain=0, delta=1e-9, tri_rule=7, fan=0, newton_tol=1e-14,
              newton_max_iter=20, clip_tol_rel=1e-12, merge_tol_rel=1e-10,
              area_tol_rel=1e-14, n_threads=1, terms=3) -> Opts:
    return Opts(lm, d_domain, tri_rule, fan, newton_max_iter, n_threads, terms, 0, delta,
                newton_tol, clip_tol_rel, merge_tol_rel, area_tol_rel)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            lib = ctypes.CDLL(path)
            P = ctypes.c_void_p
            i64, i32, f64 = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
            for name in ("oracle_search_bruteforce", "oracle_search_binned"):
                f = getattr(lib, name)
                f.restype = i64
                f.argtypes = [P, i64, P, i64, i32, P, i64, P, i64, i32, f64, P, P, i64]
            lib.oracle_element_blocks.restype = ctypes.c_int
            lib.oracle_element_blocks.argtypes = [P, P, i64, i32, i32, P, P]
            lib.oracle_pair_blocks.restype = ctypes.c_int
            lib.oracle_pair_blocks.argtypes = [P, P, i32, P, P, i32, ctypes.POINTER(Opts),
                                               P, P, i64, P, P, P, P]
            lib.oracle_weighted_gap_grad.restype = ctypes.c_int
            lib.oracle_weighted_gap_grad.argtypes = [P, i64, P, i64, i32, P, i64, P, i32,
                                                     ctypes.POINTER(Opts), P, P, i64, P, P, P, P]
            lib.oracle_tangent_blocks.restype = ctypes.c_int
            lib.oracle_tangent_blocks.argtypes = [P, P, i64, i32, P, P, i32, ctypes.POINTER(Opts),
                                                  P, P, i64, P, P, P, P, P]
            lib.oracle_element_based_blocks.restype = ctypes.c_int
            lib.oracle_element_based_blocks.argtypes = [P, P, i32, P, P, i32, ctypes.POINTER(Opts),
                                                        P, P, i64, i32, P, P, P]
            lib.oracle_nodal_normals.restype = ctypes.c_int
            lib.oracle_nodal_normals.argtypes = [P, i64, P, i64, i32, P]
            lib.oracle_element_normals.restype = ctypes.c_int
            lib.oracle_element_normals.argtypes = [P, P, i64, i32, P]
            lib.oracle_slave_frames.restype = ctypes.c_int
            lib.oracle_slave_frames.argtypes = [P, P, i64, i32, P]
            lib.oracle_tri_rule.restype = ctypes.c_int
            lib.oracle_tri_rule.argtypes = [i32, P, i32]
            lib.oracle_invert_map.restype = ctypes.c_int
            lib.oracle_invert_map.argtypes = [i32, P, P, ctypes.POINTER(Opts), P]
            lib.oracle_quadratic_element_D.restype = ctypes.c_int
            lib.oracle_quadratic_element_D.argtypes = [P, P, i64, i32, P]
            lib.oracle_quadratic_pair_blocks.restype = ctypes.c_int
            lib.oracle_quadratic_pair_blocks.argtypes = [P, P, i32, P, P, i32, ctypes.POINTER(Opts),
                                                         P, P, i64, P, P, P]
            lib.oracle_quadratic_shape.restype = ctypes.c_int
            lib.oracle_quadratic_shape.argtypes = [i32, f64, f64, P, P]
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _mesh_arrays(itf):
    xs = np.ascontiguousarray(itf.xs, dtype=np.float64)
    cs = np.ascontiguousarray(itf.conn_s, dtype=np.int32)
    xm = np.ascontiguousarray(itf.xm, dtype=np.float64)
    cm = np.ascontiguousarray(itf.conn_m, dtype=np.int32)
    return xs, cs, xm, cm


def _search(fn_name: str, itf, delta=None):
    lib = _load()
    xs, cs, xm, cm = _mesh_arrays(itf)
    d = itf.delta if delta is None else delta
    fn = getattr(lib, fn_name)
    args = (_p(xs), xs.shape[0], _p(cs), cs.shape[0], cs.shape[1],
            _p(xm), xm.shape[0], _p(cm), cm.shape[0], cm.shape[1], d)
    cap = max(16, 8 * cs.shape[0])
    while True:
        s = np.empty(cap, np.int32)
        m = np.empty(cap, np.int32)
        n = fn(*args, _p(s), _p(m), cap)
        if n <= cap:
            return s[:n].copy(), m[:n].copy()
        cap = int(n)


def search_bruteforce(itf, delta=None):
    """All (s, m) with overlapping delta-inflated bounding boxes (definition)."""
    return _search("oracle_search_bruteforce", itf, delta)


def search_binned(itf, delta=None):
    """Binned search (Algorithm 2 restated for one address space)."""
    return _search("oracle_search_binned", itf, delta)


def element_blocks(itf, lm=None):
    """Per slave element: LM coefficient matrix A (Es,4,4) and element D (Es,4,4)."""
    lib = _load()
    xs, cs, _, _ = _mesh_arrays(itf)
    E = cs.shape[0]
    A = np.zeros((E, 16))
    De = np.zeros((E, 16))
    lib.oracle_element_blocks(_p(xs), _p(cs), E, cs.shape[1], itf.lm if lm is None else lm,
                              _p(A), _p(De))
    return A.reshape(E, 4, 4), De.reshape(E, 4, 4)


def slave_frames(itf):
    lib = _load()
    xs, cs, _, _ = _mesh_arrays(itf)
    out = np.zeros((cs.shape[0], 12))
    lib.oracle_slave_frames(_p(xs), _p(cs), cs.shape[0], cs.shape[1], _p(out))
    return out


STAT_NAMES = ("pairs", "nonempty", "gauss_points", "newton_fail", "xi_out_of_range",
              "clip_overflow", "cells")


def pair_blocks(itf, s, m, opts: Opts | None = None):
    """Per-pair M and D blocks (P,4,4), nonempty flags and counters."""
    lib = _load()
    o = opts if opts is not None else make_opts(lm=itf.lm, delta=itf.delta)
    xs, cs, xm, cm = _mesh_arrays(itf)
    s = np.ascontiguousarray(s, np.int32)
    m = np.ascontiguousarray(m, np.int32)
    P = s.shape[0]
    Mb = np.zeros((max(P, 1), 16))
    Db = np.zeros((max(P, 1), 16))
    ne = np.zeros(max(P, 1), np.uint8)
    st = np.zeros(7, np.int64)
    lib.oracle_pair_blocks(_p(xs), _p(cs), cs.shape[1], _p(xm), _p(cm), cm.shape[1],
                           ctypes.byref(o), _p(s), _p(m), P, _p(Mb), _p(Db), _p(ne), _p(st))
    return (Mb[:P].reshape(P, 4, 4), Db[:P].reshape(P, 4, 4), ne[:P].astype(bool),
            dict(zip(STAT_NAMES, (int(x) for x in st))))


def _csr_from_triplets(rows, cols, vals, nrows, ncols):
    """Sum duplicates in order of appearance; keep every structural entry."""
    import scipy.sparse as sp
    rows = np.asarray(rows, np.int64)
    cols = np.asarray(cols, np.int64)
    vals = np.asarray(vals, np.float64)
    if rows.size == 0:
        return sp.csr_matrix((nrows, ncols))
    order = np.lexsort((cols, rows))          # stable: ties keep appearance order
    r, c, v = rows[order], cols[order], vals[order]
    first = np.ones(r.size, bool)
    first[1:] = (r[1:] != r[:-1]) | (c[1:] != c[:-1])
    starts = np.flatnonzero(first)
    sums = np.zeros(starts.size)
    seg = np.cumsum(first) - 1
    np.add.at(sums, seg, v)                   # sequential, in sorted (appearance) order
    ur, uc = r[starts], c[starts]
    rowptr = np.zeros(nrows + 1, np.int64)
    np.add.at(rowptr, ur + 1, 1)
    rowptr = np.cumsum(rowptr)
    return sp.csr_matrix((sums, uc.astype(np.int32), rowptr), shape=(nrows, ncols))


def assemble(itf, s, m, Mb, Db, nonempty, De=None, d_domain=0, lm=None):
    """Assemble D (Ns x Ns) and M (Ns x Nm) CSR from element/pair blocks.

    A structural entry of M (and of D in segment mode) exists iff some
    non-empty pair touches it; in element mode every slave element contributes
    its whole D_e block -- with dual LMs only its diagonal: the dual basis is
    biorthogonal to the shape functions, int Phi_a N_b = delta_ab int N_b
    (Sec. 2.2), so the off-diagonal entries are zero by definition.  Values are
    summed in pair (or element) order."""
    lm = itf.lm if lm is None else lm
    cs = np.asarray(itf.conn_s)
    cm = np.asarray(itf.conn_m)
    ns, nm = cs.shape[1], cm.shape[1]
    Ns, Nm = itf.n_slave_nodes, itf.n_master_nodes
    keep = np.flatnonzero(nonempty)
    sk, mk = np.asarray(s)[keep], np.asarray(m)[keep]
    # M: rows slave node of (s, a), cols master node of (m, l); order (pair, a, l)
    rows = np.repeat(cs[sk][:, :, None], nm, axis=2)
    cols = np.repeat(cm[mk][:, None, :], ns, axis=1)
    vals = Mb[keep][:, :ns, :nm]
    M = _csr_from_triplets(rows.ravel(), cols.ravel(), vals.ravel(), Ns, Nm)
    if d_domain == 1:
        rows = np.repeat(cs[sk][:, :, None], ns, axis=2)
        cols = np.repeat(cs[sk][:, None, :], ns, axis=1)
        vals = Db[keep][:, :ns, :ns]
    elif lm == 1:
        rows = cs
        cols = cs
        vals = De[:, np.arange(ns), np.arange(ns)]
    else:
        rows = np.repeat(cs[:, :, None], ns, axis=2)
        cols = np.repeat(cs[:, None, :], ns, axis=1)
        vals = De[:, :ns, :ns]
    D = _csr_from_triplets(rows.ravel(), cols.ravel(), vals.ravel(), Ns, Ns)
    return D, M


@dataclass
class Result:
    s: np.ndarray
    m: np.ndarray
    Mb: np.ndarray
    Db: np.ndarray
    nonempty: np.ndarray
    A: np.ndarray
    De: np.ndarray
    D: object
    M: object
    stats: dict


QUADRATIC = (6, 8)   # tri6, quad8 slave elements


def shape_quadratic(nen: int, xi: float, eta: float):
    """Quadratic shape functions (tri6: 6, quad8: 8) and their parameter
    derivatives (nen x 2) at one point."""
    lib = _load()
    N = np.zeros(8)
    dN = np.zeros(16)
    if lib.oracle_quadratic_shape(int(nen), float(xi), float(eta), _p(N), _p(dN)) != 0:
        raise ValueError("nen must be 6 or 8")
    return N[:nen].copy(), dN.reshape(8, 2)[:nen].copy()


def quadratic_element_D(itf):
    """Element-domain D blocks (Es, 8, 8) of a quadratic slave mesh, standard LMs."""
    lib = _load()
    xs, cs, _, _ = _mesh_arrays(itf)
    E = cs.shape[0]
    De = np.zeros((max(E, 1), 64))
    if lib.oracle_quadratic_element_D(_p(xs), _p(cs), E, cs.shape[1], _p(De)) != 0:
        raise ValueError("slave elements must be tri6 or quad8")
    return De[:E].reshape(E, 8, 8)


def quadratic_pair_blocks(itf, s, m, opts: Opts | None = None):
    """Per-pair M blocks (P, 8, 4) of a quadratic slave mesh (segment-based on
    the four linear sub-elements), nonempty flags and counters."""
    lib = _load()
    o = opts if opts is not None else make_opts(lm=itf.lm, delta=itf.delta)
    xs, cs, xm, cm = _mesh_arrays(itf)
    s = np.ascontiguousarray(s, np.int32)
    m = np.ascontiguousarray(m, np.int32)
    P = s.shape[0]
    Mb = np.zeros((max(P, 1), 32))
    ne = np.zeros(max(P, 1), np.uint8)
    st = np.zeros(7, np.int64)
    if lib.oracle_quadratic_pair_blocks(_p(xs), _p(cs), cs.shape[1], _p(xm), _p(cm), cm.shape[1],
                                        ctypes.byref(o), _p(s), _p(m), P, _p(Mb), _p(ne), _p(st)) != 0:
        raise ValueError("slave elements must be tri6 or quad8")
    return Mb[:P].reshape(P, 8, 4), ne[:P].astype(bool), dict(zip(STAT_NAMES, (int(x) for x in st)))


def evaluate(itf, opts: Opts | None = None, search: str = "binned", pairs=None) -> Result:
    """Search + per-pair integration + assembly, all on the CPU."""
    o = opts if opts is not None else make_opts(lm=itf.lm, delta=itf.delta)
    if pairs is not None:
        s, m = pairs
    elif search == "bruteforce":
        s, m = search_bruteforce(itf, o.delta)
    else:
        s, m = search_binned(itf, o.delta)
    if np.asarray(itf.conn_s).shape[1] in QUADRATIC:
        # quadratic slave elements: standard LMs and element-domain D only
        if o.lm != 0 or o.d_domain != 0:
            raise ValueError("quadratic slave elements: standard LMs and element-domain D only")
        De = quadratic_element_D(itf)
        Mb, ne, st = quadratic_pair_blocks(itf, s, m, o)
        D, M = assemble(itf, s, m, Mb, None, ne, De, 0, 0)
        return Result(s, m, Mb, None, ne, None, De, D, M, st)
    A, De = element_blocks(itf, o.lm)
    Mb, Db, ne, st = pair_blocks(itf, s, m, o)
    D, M = assemble(itf, s, m, Mb, Db, ne, De, o.d_domain, o.lm)
    return Result(s, m, Mb, Db, ne, A, De, D, M, st)


def weighted_gap_grad(itf, lam, s, m, opts: Opts | None = None):
    """J = sum_j lam_j.((D Xs)_j - (M Xm)_j) and dJ/dXs, dJ/dXm (forward-mode).

    ``opts.terms`` selects the terms: 1 = lam.D Xs only, 2 = -lam.M Xm only,
    3 = both (the functional)."""
    lib = _load()
    o = opts if opts is not None else make_opts(lm=itf.lm, delta=itf.delta)
    xs, cs, xm, cm = _mesh_arrays(itf)
    lam = np.ascontiguousarray(lam, np.float64)
    s = np.ascontiguousarray(s, np.int32)
    m = np.ascontiguousarray(m, np.int32)
    gs = np.zeros_like(xs)
    gm = np.zeros_like(xm)
    J = ctypes.c_double(0.0)
    lib.oracle_weighted_gap_grad(_p(xs), xs.shape[0], _p(cs), cs.shape[0], cs.shape[1],
                                 _p(xm), xm.shape[0], _p(cm), cm.shape[1], ctypes.byref(o),
                                 _p(s), _p(m), s.shape[0], _p(lam), ctypes.byref(J),
                                 _p(gs), _p(gm))
    return J.value, gs, gm


def element_based_blocks(itf, s, m, n_rule: int = 8, opts: Opts | None = None):
    """Per-pair M and D blocks (P,4,4) of element-based integration (n x n
    rule on each slave element, first covering master in pair order) and the
    flags of pairs that received a quadrature point."""
    lib = _load()
    o = opts if opts is not None else make_opts(lm=itf.lm, delta=itf.delta)
    xs, cs, xm, cm = _mesh_arrays(itf)
    s = np.ascontiguousarray(s, np.int32)
    m = np.ascontiguousarray(m, np.int32)
    P = s.shape[0]
    Mb = np.zeros((max(P, 1), 16))
    Db = np.zeros((max(P, 1), 16))
    fl = np.zeros(max(P, 1), np.uint8)
    lib.oracle_element_based_blocks(_p(xs), _p(cs), cs.shape[1], _p(xm), _p(cm), cm.shape[1],
                                    ctypes.byref(o), _p(s), _p(m), P, int(n_rule), _p(Mb), _p(Db), _p(fl))
    return Mb[:P].reshape(P, 4, 4), Db[:P].reshape(P, 4, 4), fl[:P].astype(bool)


def evaluate_element_based(itf, n_rule: int = 8, opts: Opts | None = None, pairs=None):
    """Search + element-based integration + assembly (D from the element
    integrals in element mode, from the covered quadrature points in segment
    mode).  Returns (D, M, pairs, flags)."""
    o = opts if opts is not None else make_opts(lm=itf.lm, delta=itf.delta)
    s, m = pairs if pairs is not None else search_binned(itf, o.delta)
    _, De = element_blocks(itf, o.lm)
    Mb, Db, fl = element_based_blocks(itf, s, m, n_rule, o)
    D, M = assemble(itf, s, m, Mb, Db, fl, De, o.d_domain, o.lm)
    return D, M, (s, m), fl


def tangent_blocks(itf, s, m, ys, ym, opts: Opts | None = None):
    """Dense per-source blocks of K = d/dX[(D (x) I3) ys - (M (x) I3) ym].

    Returns kp (P,4,3,8,3): pair rows (local slave node a, component c) by
    columns (the pair's 4 slave then 4 master nodes, direction d); ke
    (Es,4,3,4,3): element-domain D rows by the element's slave nodes (zero in
    segment mode); flags (P,) of the non-empty pairs."""
    lib = _load()
    o = opts if opts is not None else make_opts(lm=itf.lm, delta=itf.delta)
    xs, cs, xm, cm = _mesh_arrays(itf)
    ys = np.ascontiguousarray(ys, np.float64)
    ym = np.ascontiguousarray(ym, np.float64)
    s = np.ascontiguousarray(s, np.int32)
    m = np.ascontiguousarray(m, np.int32)
    P, E = s.shape[0], cs.shape[0]
    kp = np.zeros((max(P, 1), 288))
    ke = np.zeros((max(E, 1), 144))
    fl = np.zeros(max(P, 1), np.uint8)
    lib.oracle_tangent_blocks(_p(xs), _p(cs), E, cs.shape[1], _p(xm), _p(cm), cm.shape[1],
                              ctypes.byref(o), _p(s), _p(m), P, _p(ys), _p(ym), _p(kp),
                              _p(ke), _p(fl))
    return (kp[:P].reshape(P, 4, 3, 8, 3), ke[:E].reshape(E, 4, 3, 4, 3),
            fl[:P].astype(bool))


def _bsr_from_blocks(rows, cols, blocks, nrows):
    """Sum 3x3 blocks with equal (row, col) in order of appearance."""
    rows = np.asarray(rows, np.int64)
    cols = np.asarray(cols, np.int64)
    blocks = np.asarray(blocks, np.float64).reshape(-1, 3, 3)
    rowptr = np.zeros(nrows + 1, np.int64)
    if rows.size == 0:
        return rowptr, np.zeros(0, np.int32), np.zeros((0, 3, 3))
    order = np.lexsort((cols, rows))          # stable: ties keep appearance order
    r, c, b = rows[order], cols[order], blocks[order]
    first = np.ones(r.size, bool)
    first[1:] = (r[1:] != r[:-1]) | (c[1:] != c[:-1])
    starts = np.flatnonzero(first)
    seg = np.cumsum(first) - 1
    sums = np.zeros((starts.size, 3, 3))
    np.add.at(sums, seg, b)
    np.add.at(rowptr, r[starts] + 1, 1)
    return np.cumsum(rowptr), c[starts].astype(np.int32), sums


def tangent(itf, s, m, ys, ym, opts: Opts | None = None, add_direct: bool = False):
    """Block-sparse K = d/dX[(D (x) I3) ys - (M (x) I3) ym] (3x3 blocks).

    Block rows are slave nodes; block columns are slave nodes [0, Ns) then
    master nodes [Ns, Ns + Nm); block (j, k)[c][d] = d g_j[c] / d X_k[d].  A
    block is structural iff a non-empty pair, or (element-domain D) a slave
    element, has both nodes.  ``add_direct`` adds [D (x) I3 | -M (x) I3],
    which with ys = Xs, ym = Xm makes K the Jacobian of the weighted gap
    vector g = (D (x) I3) Xs - (M (x) I3) Xm.  Sums run over pairs in the
    given order, then elements, then the direct terms.
    Returns (rowptr int64, colidx int32, vals (nnzb,3,3))."""
    o = opts if opts is not None else make_opts(lm=itf.lm, delta=itf.delta)
    kp, ke, fl = tangent_blocks(itf, s, m, ys, ym, o)
    cs = np.asarray(itf.conn_s)
    cm = np.asarray(itf.conn_m)
    ns, nm = cs.shape[1], cm.shape[1]
    Ns = itf.n_slave_nodes
    keep = np.flatnonzero(fl)
    sk, mk = np.asarray(s)[keep], np.asarray(m)[keep]
    nodes = np.concatenate([cs[sk], Ns + cm[mk]], axis=1)           # (K, ns + nm)
    loc = np.concatenate([np.arange(ns), 4 + np.arange(nm)])
    blk = kp[keep][:, :ns][:, :, :, loc, :]                           # (K, ns, 3, ns+nm, 3)
    rows = [np.repeat(cs[sk][:, :, None], ns + nm, axis=2).ravel()]
    cols = [np.repeat(nodes[:, None, :], ns, axis=1).ravel()]
    blocks = [blk.transpose(0, 1, 3, 2, 4).reshape(-1, 3, 3)]
    if o.d_domain == 0:
        rows.append(np.repeat(cs[:, :, None], ns, axis=2).ravel())
        cols.append(np.repeat(cs[:, None, :], ns, axis=1).ravel())
        blocks.append(ke[:, :ns, :, :ns, :].transpose(0, 1, 3, 2, 4).reshape(-1, 3, 3))
    if add_direct:
        A, De = element_blocks(itf, o.lm)
        Mb, Db, _, _ = pair_blocks(itf, s, m, o)
        eye = np.eye(3)
        rows.append(np.repeat(cs[sk][:, :, None], nm, axis=2).ravel())
        cols.append(np.repeat(Ns + cm[mk][:, None, :], ns, axis=1).ravel())
        blocks.append((-Mb[keep][:, :ns, :nm, None, None] * eye).reshape(-1, 3, 3))
        if o.d_domain == 1:
            rows.append(np.repeat(cs[sk][:, :, None], ns, axis=2).ravel())
            cols.append(np.repeat(cs[sk][:, None, :], ns, axis=1).ravel())
            blocks.append((Db[keep][:, :ns, :ns, None, None] * eye).reshape(-1, 3, 3))
        else:
            rows.append(np.repeat(cs[:, :, None], ns, axis=2).ravel())
            cols.append(np.repeat(cs[:, None, :], ns, axis=1).ravel())
            blocks.append((De[:, :ns, :ns, None, None] * eye).reshape(-1, 3, 3))
    return _bsr_from_blocks(np.concatenate(rows), np.concatenate(cols),
                            np.concatenate(blocks), Ns)


def bsr_dense(rowptr, colidx, vals, nrows, ncols):
    """Dense (3 nrows, 3 ncols) matrix of a 3x3-block BSR triple."""
    out = np.zeros((3 * nrows, 3 * ncols))
    rowptr = np.asarray(rowptr)
    for j in range(nrows):
        for q in range(rowptr[j], rowptr[j + 1]):
            k = int(colidx[q])
            out[3 * j:3 * j + 3, 3 * k:3 * k + 3] += vals[q]
    return out


def nodal_normals(itf) -> np.ndarray:
    """Averaged unit nodal normals of the slave surface (Ns x 3)."""
    lib = _load()
    xs, cs, _, _ = _mesh_arrays(itf)
    out = np.zeros_like(xs)
    lib.oracle_nodal_normals(_p(xs), xs.shape[0], _p(cs), cs.shape[0], cs.shape[1], _p(out))
    return out


def element_normals(x, conn) -> np.ndarray:
    lib = _load()
    x = np.ascontiguousarray(x, np.float64)
    conn = np.ascontiguousarray(conn, np.int32)
    out = np.zeros((conn.shape[0], 3))
    lib.oracle_element_normals(_p(x), _p(conn), conn.shape[0], conn.shape[1], _p(out))
    return out


def facing_pairs(itf, s, m):
    """Candidate pairs whose slave and master element normals (at the element
    centres) point against each other: n_s . n_m < 0 (the facing test)."""
    ns = element_normals(itf.xs, itf.conn_s)
    nm = element_normals(itf.xm, itf.conn_m)
    s = np.asarray(s)
    m = np.asarray(m)
    keep = np.einsum("ij,ij->i", ns[s], nm[m]) < 0.0
    return s[keep], m[keep]


def weighted_normal_gap(itf, D, M, normals=None) -> np.ndarray:
    """g_j = -n_j . ((D Xs)_j - (M Xm)_j): the weighted normal gap of slave node
    j (positive when the bodies are apart along the outward slave normal)."""
    n = nodal_normals(itf) if normals is None else np.asarray(normals)
    v = D @ itf.xs - M @ itf.xm
    return -np.einsum("ij,ij->i", n, v)


def ncp(lam_n, gap, c: float):
    """Active set and complementarity residual of the Hertz-Signorini-Moreau
    conditions (gap >= 0, pressure <= 0, gap * pressure = 0) per slave node:
    active = lam_n + c gap < 0; C = lam_n - min(0, lam_n + c gap)."""
    lam_n = np.asarray(lam_n, np.float64)
    t = lam_n + c * np.asarray(gap, np.float64)
    return t < 0.0, lam_n - np.minimum(0.0, t)


def tri_rule(which: int = 7) -> np.ndarray:
    lib = _load()
    out = np.zeros((64, 4))
    n = lib.oracle_tri_rule(which, _p(out), 64)
    return out[:n].copy()


def invert_map(p: np.ndarray, x, opts: Opts | None = None):
    lib = _load()
    o = opts if opts is not None else make_opts()
    p = np.ascontiguousarray(p, np.float64).reshape(-1, 2)
    xx = np.ascontiguousarray(x, np.float64)
    xi = np.zeros(2)
    ok = lib.oracle_invert_map(p.shape[0], _p(np.ascontiguousarray(p.ravel())), _p(xx),
                               ctypes.byref(o), _p(xi))
    return xi, bool(ok)
