"""Python binding of the GB300 mortar library (argument marshalling only).

Every step of the path -- search, integration, assembly, adjoint -- runs in
the CUDA library behind ``include/mortar.h``.  This module converts numpy
arrays / torch tensors into pointers and sizes, calls the C ABI with the same
names, and wraps results.  Host arrays (numpy, CPU tensors) are passed with
``on_device=0``; CUDA tensors with ``on_device=1``.

PyTorch provides device memory and streams only.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _native
from ._native import MortarError, Options, Stats, call, lib  # noqa: F401

QUAD4 = 4
TRI3 = 3
QUAD8 = 8   # quadratic slave elements (forward path only)
TRI6 = 6
LM_STANDARD = 0
LM_DUAL = 1
D_ELEMENT = 0
D_SEGMENT = 1
MATRIX_D = 0
MATRIX_M = 1

_OK_OR_NEWTON = (0, -3)


INTEGRATE_SEGMENT, INTEGRATE_ELEMENT = 0, 1


def _torch():
    import torch
    return torch


def _is_cuda_tensor(a) -> bool:
    try:
        torch = _torch()
    except ImportError:
        return False
    return isinstance(a, torch.Tensor) and a.is_cuda


def _ptr_in(a, dtype):
    """(pointer, keepalive, on_device) for an input array."""
    if _is_cuda_tensor(a):
        torch = _torch()
        t = a.to(dtype={np.float64: torch.float64, np.int32: torch.int32, np.int64: torch.int64}[dtype])
        t = t.contiguous()
        return ctypes.c_void_p(t.data_ptr()), t, 1
    if hasattr(a, "detach"):   # CPU tensor
        a = a.detach().numpy()
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr.ctypes.data_as(ctypes.c_void_p), arr, 0


def default_options() -> Options:
    o = Options()
    call("mortar_default_options", ctypes.byref(o))
    return o


class Mortar:
    """One context of the C library (one interface or one batch)."""

    def __init__(self, lm: int = LM_STANDARD, d_domain: int = D_ELEMENT, delta: float = 1e-9,
                 stream=None, **kw):
        self.opt = default_options()
        self.opt.lm = lm
        self.opt.d_domain = d_domain
        self.opt.search_inflation = delta
        names = {f[0] for f in Options._fields_}
        for k, v in kw.items():
            if k not in names:
                raise TypeError(f"unknown option {k!r}")
            setattr(self.opt, k, v)
        h = ctypes.c_void_p()
        if stream is None:
            try:
                torch = _torch()
                if torch.cuda.is_available():
                    stream = torch.cuda.current_stream().cuda_stream
            except ImportError:
                pass
        call("mortar_create", ctypes.byref(h), ctypes.byref(self.opt),
             ctypes.c_void_p(stream or 0))
        self.h = h
        self.Ns = self.Nm = self.Es = self.Em = 0
        self.type_s = QUAD4

    def close(self):
        if getattr(self, "h", None):
            lib().mortar_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------- inputs
    def set_interface(self, xs, conn_s, xm, conn_m, type_s: int | None = None, type_m: int | None = None):
        px, kx, dx = _ptr_in(xs, np.float64)
        pcs, kcs, _ = _ptr_in(conn_s, np.int32)
        pm, km, _ = _ptr_in(xm, np.float64)
        pcm, kcm, _ = _ptr_in(conn_m, np.int32)
        self.Ns, self.Nm = int(kx.shape[0]), int(km.shape[0])
        self.Es, self.Em = int(kcs.shape[0]), int(kcm.shape[0])
        ts = type_s or int(kcs.shape[1])
        tm = type_m or int(kcm.shape[1])
        self.type_s = ts
        call("mortar_set_interface", self.h, px, self.Ns, pcs, self.Es, ts, pm, self.Nm, pcm, self.Em, tm, dx)
        return self

    def set_batch(self, interfaces):
        """Concatenate interfaces (inputs.Interface objects) into one batch."""
        xs, cs, xm, cm = [], [], [], []
        sn, se, mn, me = [0], [0], [0], [0]
        for itf in interfaces:
            cs.append(np.asarray(itf.conn_s, np.int64) + sn[-1])
            cm.append(np.asarray(itf.conn_m, np.int64) + mn[-1])
            xs.append(np.asarray(itf.xs, np.float64))
            xm.append(np.asarray(itf.xm, np.float64))
            sn.append(sn[-1] + itf.xs.shape[0])
            se.append(se[-1] + itf.conn_s.shape[0])
            mn.append(mn[-1] + itf.xm.shape[0])
            me.append(me[-1] + itf.conn_m.shape[0])
        ts, tm = interfaces[0].type_s, interfaces[0].type_m
        self.type_s = ts
        arrs = [np.ascontiguousarray(np.concatenate(xs)), np.ascontiguousarray(np.concatenate(cs), np.int32),
                np.ascontiguousarray(np.concatenate(xm)), np.ascontiguousarray(np.concatenate(cm), np.int32)]
        offs = [np.asarray(o, np.int64) for o in (sn, se, mn, me)]
        self._batch_keep = arrs + offs
        p = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
        call("mortar_set_batch", self.h, len(interfaces), p(offs[0]), p(offs[1]), p(offs[2]), p(offs[3]),
             p(arrs[0]), p(arrs[1]), ts, p(arrs[2]), p(arrs[3]), tm, 0)
        self.Ns, self.Es, self.Nm, self.Em = int(sn[-1]), int(se[-1]), int(mn[-1]), int(me[-1])
        self.offsets = {"slave_nodes": offs[0], "slave_elems": offs[1],
                        "master_nodes": offs[2], "master_elems": offs[3]}
        return self

    def set_coordinates(self, xs=None, xm=None):
        ps, ks, ds = _ptr_in(xs, np.float64) if xs is not None else (None, None, 0)
        pm, km, dm = _ptr_in(xm, np.float64) if xm is not None else (None, None, 0)
        if xs is not None and xm is not None and ds != dm:
            raise ValueError("xs and xm must both be host or both be device arrays")
        call("mortar_set_coordinates", self.h, ps, pm, ds or dm)

    # ------------------------------------------------------------- compute
    def search(self) -> int:
        n = ctypes.c_int64()
        call("mortar_search", self.h, ctypes.byref(n), ok=(0, -2))
        return int(n.value)

    def evaluate(self) -> int:
        return call("mortar_evaluate", self.h, ok=(0, -2, -3))

    def run_graph(self, lam=None) -> int:
        if lam is None:
            return call("mortar_run_graph", self.h, None, 0, ok=(0, -2, -3))
        p, k, d = _ptr_in(lam, np.float64)
        self._lam_keep = k
        return call("mortar_run_graph", self.h, p, d, ok=(0, -2, -3))

    def weighted_gap_grad(self, lam, out_device: bool = False):
        """J and dJ/dXs, dJ/dXm (numpy, or CUDA tensors if out_device)."""
        p, k, d = _ptr_in(lam, np.float64)
        J = ctypes.c_double()
        if out_device:
            torch = _torch()
            gs = torch.empty((self.Ns, 3), dtype=torch.float64, device="cuda")
            gm = torch.empty((self.Nm, 3), dtype=torch.float64, device="cuda")
            call("mortar_weighted_gap_grad", self.h, p, ctypes.byref(J), ctypes.c_void_p(gs.data_ptr()),
                 ctypes.c_void_p(gm.data_ptr()), 1, ok=(0, -2, -3))
        else:
            gs = np.empty((self.Ns, 3))
            gm = np.empty((self.Nm, 3))
            call("mortar_weighted_gap_grad", self.h, p, ctypes.byref(J), gs.ctypes.data_as(ctypes.c_void_p),
                 gm.ctypes.data_as(ctypes.c_void_p), 0, ok=(0, -2, -3))
        return J.value, gs, gm

    def tangent(self, ys, ym, add_direct: bool = False, out_device: bool = False):
        """Linearisation K = d/dX[(D (x) I3) ys - (M (x) I3) ym] (ys, ym fixed), plus
        [D (x) I3 | -M (x) I3] if add_direct, as a BSR triple (rowptr int64,
        colidx int32, vals (nnzb, 3, 3)): numpy arrays, or CUDA tensors if out_device.
        Block rows are slave nodes, block columns slave nodes then Ns + master nodes."""
        ps, ks, ds = _ptr_in(ys, np.float64)
        pm, km, dm = _ptr_in(ym, np.float64)
        if ds != dm:
            raise ValueError("ys and ym must both be CUDA tensors or both host arrays")
        nb = ctypes.c_int64()
        call("mortar_tangent", self.h, ps, pm, int(bool(add_direct)), ds, ctypes.byref(nb), ok=(0, -2, -3))
        n = int(nb.value)
        if out_device:
            torch = _torch()
            rp = torch.empty(self.Ns + 1, dtype=torch.int64, device="cuda")
            ci = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
            va = torch.empty((max(n, 1), 3, 3), dtype=torch.float64, device="cuda")
            call("mortar_tangent_copy", self.h, ctypes.c_void_p(rp.data_ptr()), ctypes.c_void_p(ci.data_ptr()),
                 ctypes.c_void_p(va.data_ptr()), max(n, 1), 1)
        else:
            rp = np.empty(self.Ns + 1, np.int64)
            ci = np.empty(max(n, 1), np.int32)
            va = np.empty((max(n, 1), 3, 3))
            call("mortar_tangent_copy", self.h, rp.ctypes.data_as(ctypes.c_void_p),
                 ci.ctypes.data_as(ctypes.c_void_p), va.ctypes.data_as(ctypes.c_void_p), max(n, 1), 0)
        return rp, ci[:n], va[:n]

    def torch_bsr_tangent(self, ys, ym, add_direct: bool = False):
        """The linearisation as a torch sparse BSR tensor (3x3 blocks) on the CUDA device."""
        torch = _torch()
        rp, ci, va = self.tangent(ys, ym, add_direct, out_device=True)
        return torch.sparse_bsr_tensor(rp, ci.to(torch.int64), va,
                                       size=(3 * self.Ns, 3 * (self.Ns + self.Nm)))

    def contact_terms(self, lambda_n=None, c: float = 1.0):
        """Averaged nodal normals (Ns x 3), weighted normal gap (Ns) and, with
        normal multipliers lambda_n (Ns), the active set and complementarity
        residual of the Hertz-Signorini-Moreau conditions (numpy arrays)."""
        normals = np.empty((self.Ns, 3))
        gap = np.empty(self.Ns)
        P = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
        if lambda_n is None:
            call("mortar_contact_terms", self.h, None, float(c), P(normals), P(gap), None, None, 0, ok=(0, -2, -3))
            return {"normals": normals, "gap": gap}
        lam = np.ascontiguousarray(lambda_n, np.float64)
        active = np.empty(self.Ns, np.uint8)
        ncp = np.empty(self.Ns)
        call("mortar_contact_terms", self.h, P(lam), float(c), P(normals), P(gap), P(active), P(ncp), 0,
             ok=(0, -2, -3))
        return {"normals": normals, "gap": gap, "active": active.astype(bool), "ncp": ncp}

    def gradient(self):
        J = ctypes.c_double()
        gs = np.empty((self.Ns, 3))
        gm = np.empty((self.Nm, 3))
        call("mortar_get_gradient", self.h, ctypes.byref(J), gs.ctypes.data_as(ctypes.c_void_p),
             gm.ctypes.data_as(ctypes.c_void_p), 0)
        return J.value, gs, gm

    # ------------------------------------------------------------- outputs
    def pairs(self):
        n = self.stats()["n_pairs"]
        s = np.empty(n, np.int32)
        m = np.empty(n, np.int32)
        call("mortar_get_pairs", self.h, s.ctypes.data_as(ctypes.c_void_p), m.ctypes.data_as(ctypes.c_void_p), n, 0)
        return s, m

    def csr_size(self, which: int):
        r, c, n = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        call("mortar_csr_size", self.h, which, ctypes.byref(r), ctypes.byref(c), ctypes.byref(n))
        return int(r.value), int(c.value), int(n.value)

    def csr(self, which: int):
        """(rowptr int64, colidx int32, vals f64, shape) as numpy arrays."""
        nr, nc, nnz = self.csr_size(which)
        rp = np.empty(nr + 1, np.int64)
        ci = np.empty(max(nnz, 1), np.int32)
        va = np.empty(max(nnz, 1), np.float64)
        call("mortar_csr_copy", self.h, which, rp.ctypes.data_as(ctypes.c_void_p),
             ci.ctypes.data_as(ctypes.c_void_p), va.ctypes.data_as(ctypes.c_void_p), max(nnz, 1), 0)
        return rp, ci[:nnz], va[:nnz], (nr, nc)

    def scipy(self, which: int):
        import scipy.sparse as sp
        rp, ci, va, shape = self.csr(which)
        return sp.csr_matrix((va, ci, rp), shape=shape)

    def torch_csr(self, which: int):
        """The matrix as a torch sparse CSR tensor on the current CUDA device."""
        torch = _torch()
        nr, nc, nnz = self.csr_size(which)
        rp = torch.empty(nr + 1, dtype=torch.int64, device="cuda")
        ci = torch.empty(max(nnz, 1), dtype=torch.int32, device="cuda")
        va = torch.empty(max(nnz, 1), dtype=torch.float64, device="cuda")
        call("mortar_csr_copy", self.h, which, ctypes.c_void_p(rp.data_ptr()), ctypes.c_void_p(ci.data_ptr()),
             ctypes.c_void_p(va.data_ptr()), max(nnz, 1), 1)
        return torch.sparse_csr_tensor(rp, ci[:nnz].to(torch.int64), va[:nnz], size=(nr, nc))

    def pair_blocks(self, with_D: bool = False):
        """Per-pair blocks (n_pairs, 4, 4) -- (n_pairs, 8, 4) for quadratic slave
        elements -- the segment-mode D blocks if with_D, and the nonempty flags."""
        n = self.stats()["n_pairs"]
        rows = 8 if getattr(self, "type_s", QUAD4) in (TRI6, QUAD8) else 4
        M = np.empty((max(n, 1), rows, 4))
        D = np.empty((max(n, 1), 4, 4)) if with_D else None
        f = np.empty(max(n, 1), np.uint8)
        call("mortar_get_pair_blocks", self.h, M.ctypes.data_as(ctypes.c_void_p),
             D.ctypes.data_as(ctypes.c_void_p) if with_D else None, f.ctypes.data_as(ctypes.c_void_p), max(n, 1), 0)
        return M[:n], (D[:n] if with_D else None), f[:n].astype(bool)

    def stats(self) -> dict:
        s = Stats()
        call("mortar_get_stats", self.h, ctypes.byref(s))
        return s.as_dict()

    def set_timing(self, on: bool = True):
        call("mortar_set_timing", self.h, 1 if on else 0)

    def set_watchdog(self, us: int = 0):
        """Time budget of the persistent pair kernels in microseconds (0 = none)."""
        call("mortar_set_watchdog", self.h, int(us))

    def set_launch(self, variant: int = 0, block_size: int = 0, chunk_pairs: int = 0, rounds: int = 0):
        call("mortar_set_launch", self.h, variant, block_size, chunk_pairs, rounds)

    def autotune(self, lam=None) -> dict:
        """Pick the fastest launch shape for this workload (see mortar_autotune)."""
        v, r, b, t = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_float()
        if lam is None:
            call("mortar_autotune", self.h, None, 0, ctypes.byref(v), ctypes.byref(r), ctypes.byref(b),
                 ctypes.byref(t))
        else:
            p, k, d = _ptr_in(lam, np.float64)
            call("mortar_autotune", self.h, p, d, ctypes.byref(v), ctypes.byref(r), ctypes.byref(b),
                 ctypes.byref(t))
        return {"variant": v.value, "rounds": r.value, "block": b.value, "ms": t.value}


def evaluate(xs, conn_s, xm, conn_m, lm: int = LM_STANDARD, d_domain: int = D_ELEMENT, delta: float = 1e-9):
    """(D, M) as torch sparse CSR tensors on the GPU."""
    m = Mortar(lm=lm, d_domain=d_domain, delta=delta)
    m.set_interface(xs, conn_s, xm, conn_m)
    m.evaluate()
    return m.torch_csr(MATRIX_D), m.torch_csr(MATRIX_M)


def probe_dfma(blocks: int, threads: int, iters: int, active_lanes: int = 32, stream=None, sink=None):
    """Launch the FP64 FMA throughput probe (measurement utility)."""
    torch = _torch()
    if sink is None:
        sink = torch.empty(blocks * threads, dtype=torch.float64, device="cuda")
    st = stream if stream is not None else torch.cuda.current_stream().cuda_stream
    call("mortar_probe_dfma", ctypes.c_void_p(st), blocks, threads, iters, active_lanes,
         ctypes.c_void_p(sink.data_ptr()))
    return sink


def integrate_pairs_static(xs, conn_s, xm, conn_m, pair_s, pair_m, lm: int = LM_STANDARD,
                           d_domain: int = D_ELEMENT, delta: float = 1e-9, stream=None):
    """Per-pair M (and segment D) blocks through the no-allocation entry point.

    All arguments are CUDA tensors; returns (M_blocks, D_blocks or None,
    nonempty) as CUDA tensors.  The output tensors are allocated here, by
    torch -- a caller that cannot allocate passes its own buffers to the C ABI
    directly."""
    torch = _torch()
    for name, t, dt in (("xs", xs, torch.float64), ("xm", xm, torch.float64), ("conn_s", conn_s, torch.int32),
                        ("conn_m", conn_m, torch.int32), ("pair_s", pair_s, torch.int32),
                        ("pair_m", pair_m, torch.int32)):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dt and t.is_contiguous()):
            raise TypeError(f"{name} must be a contiguous CUDA tensor of {dt}")
    if xs.dim() != 2 or xs.shape[1] != 3 or xm.dim() != 2 or xm.shape[1] != 3:
        raise ValueError("xs and xm must be (N, 3)")
    for name, c in (("conn_s", conn_s), ("conn_m", conn_m)):
        if c.dim() != 2 or c.shape[1] not in (TRI3, QUAD4):
            raise ValueError(f"{name} must be (E, 3) (tri3) or (E, 4) (quad4)")
    if pair_s.shape != pair_m.shape or pair_s.dim() != 1:
        raise ValueError("pair_s and pair_m must be 1-D of equal length")
    o = default_options()
    o.lm, o.d_domain, o.search_inflation = lm, d_domain, delta
    P = int(pair_s.shape[0])
    Mb = torch.empty((max(P, 1), 4, 4), dtype=torch.float64, device="cuda")
    Db = torch.empty((max(P, 1), 4, 4), dtype=torch.float64, device="cuda") if d_domain == D_SEGMENT else None
    ne = torch.empty(max(P, 1), dtype=torch.uint8, device="cuda")
    st = stream if stream is not None else torch.cuda.current_stream().cuda_stream
    vp = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None  # noqa: E731
    call("mortar_integrate_pairs_static", ctypes.byref(o), ctypes.c_void_p(st), vp(xs), int(xs.shape[0]),
         vp(conn_s), int(conn_s.shape[0]), int(conn_s.shape[1]), vp(xm), int(xm.shape[0]), vp(conn_m),
         int(conn_m.shape[0]), int(conn_m.shape[1]), vp(pair_s), vp(pair_m), P, vp(Mb), vp(Db), vp(ne))
    return Mb[:P], (Db[:P] if Db is not None else None), ne[:P]


def status_string(code: int) -> str:
    return lib().mortar_status_string(code).decode()


class WeightedGap:
    """torch.autograd.Function for J = sum_j lam_j . ((D Xs)_j - (M Xm)_j).

    ``WeightedGap.apply(xs, xm, lam, mortar)`` returns J (a 0-d double tensor);
    its backward returns dJ/dXs and dJ/dXm from the library's adjoint kernel.
    ``lam`` is treated as a constant.  The connectivity is the one the
    ``mortar`` context was set up with.
    """

    @staticmethod
    def apply(xs, xm, lam, mortar: Mortar):
        return _weighted_gap_fn().apply(xs, xm, lam, mortar)


_WG = None


def _weighted_gap_fn():
    global _WG
    if _WG is None:
        torch = _torch()

        class _Fn(torch.autograd.Function):
            @staticmethod
            def forward(ctx, xs, xm, lam, mortar):
                mortar.set_coordinates(xs.detach(), xm.detach())
                J, gs, gm = mortar.weighted_gap_grad(lam.detach(), out_device=xs.is_cuda)
                if not xs.is_cuda:
                    gs = torch.from_numpy(gs)
                    gm = torch.from_numpy(gm)
                ctx.save_for_backward(gs, gm)
                return torch.tensor(J, dtype=torch.float64, device=xs.device)

            @staticmethod
            def backward(ctx, gJ):
                gs, gm = ctx.saved_tensors
                return gJ * gs, gJ * gm, None, None

        _WG = _Fn
    return _WG
