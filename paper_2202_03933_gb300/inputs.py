"""Seeded synthetic interface meshes shaped like the paper's workloads.

This module only *generates inputs*: node coordinates and connectivity of a
slave and a master surface mesh, plus the per-interface settings.  It holds
none of the mortar arithmetic (no shape functions, projections, clipping or
quadrature), so both the CUDA path and the CPU oracle can consume the very same
bits without sharing any of the method.

Random numbers come from a counter-based generator: value ``i`` of stream
``k`` under ``seed`` is SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) applied to
``seed + (k * 2**40 + i + 1) * 0x9E3779B97F4A7C15`` (mod 2**64), and the top
53 bits give a double in [0, 1).  Normal variates use the Box-Muller transform
of two such uniforms.

Workloads (the paper's own meshes need its in-house FEM code and are not
available; these stand in for them with the same element types and comparable
resolution ratios):

* ``planar_8x7``       -- 8x8 quad4 slave vs 7x7 quad4 master on the unit
  square, master nodes shifted in-plane by +-0.1 h_m (standard LMs).
* ``cylinder_200x173`` -- 90 degree cylinder patch r=1, length 2, 200x200 slave
  vs 173x173 master, master radius perturbed by N(0, (0.01 h)^2) (dual LMs).
* ``mixed_300x400``    -- 300x300 quad4 slave vs a 400x400 grid split into
  tri3 along random diagonals, rotated 7 degrees and offset (0.013, 0.029).
* ``batched_512``      -- 512 independent planar interfaces of n x n slave
  quads, n log-uniform in [4, 128], master ratio U(0.7, 1.3), offsets.
* ``planar_2000x1733`` -- 2000x2000 quad4 slave vs 1733x1733 noisy quad4
  master (dual LMs), about 1.4e7 candidate pairs.

Element nodes are numbered counter-clockwise about the surface normal; quad4
corners follow the parameter corners (-1,-1), (1,-1), (1,1), (-1,1).
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

QUAD4 = 4
TRI3 = 3
LM_STANDARD = 0
LM_DUAL = 1

SEED_BASE = 2202039330
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def uniform01(seed: int, stream: int, n: int) -> np.ndarray:
    """``n`` doubles in [0, 1) from stream ``stream`` of the counter generator."""
    with np.errstate(over="ignore"):
        ctr = np.arange(n, dtype=np.uint64) + np.uint64(stream * (1 << 40) + 1)
        z = np.uint64(seed % (1 << 64)) + ctr * _GOLDEN
        bits = _mix64(z) >> np.uint64(11)
    return bits.astype(np.float64) * (1.0 / (1 << 53))


def uniform(seed: int, stream: int, n: int, lo: float, hi: float) -> np.ndarray:
    return lo + (hi - lo) * uniform01(seed, stream, n)


def normal(seed: int, stream: int, n: int) -> np.ndarray:
    """Standard normal variates (Box-Muller on two uniform streams)."""
    u1 = uniform01(seed, stream, n)
    u2 = uniform01(seed, stream + 1, n)
    r = np.sqrt(-2.0 * np.log1p(-u1))   # 1 - u1 is in (0, 1]
    return r * np.cos(2.0 * math.pi * u2)


@dataclass
class Interface:
    """One slave/master pair of surface meshes (inputs only)."""
    name: str
    xs: np.ndarray          # (Ns, 3) float64 slave node coordinates
    conn_s: np.ndarray      # (Es, 4, 3, 8 or 6) int32 slave connectivity (0-based)
    type_s: int             # QUAD4, TRI3, QUAD8 or TRI6
    xm: np.ndarray          # (Nm, 3) float64 master node coordinates
    conn_m: np.ndarray      # (Em, 4 or 3) int32 master connectivity
    type_m: int
    lm: int = LM_STANDARD   # Lagrange multiplier shape functions
    delta: float = 1e-9     # search inflation (absolute length)
    info: dict = field(default_factory=dict)

    @property
    def n_slave_nodes(self) -> int:
        return int(self.xs.shape[0])

    @property
    def n_master_nodes(self) -> int:
        return int(self.xm.shape[0])


def grid_nodes(nx: int, ny: int, x0=0.0, y0=0.0, x1=1.0, y1=1.0) -> np.ndarray:
    """(nx+1)*(ny+1) nodes of a uniform grid, id = j*(nx+1) + i, z = 0."""
    xi = x0 + (x1 - x0) * (np.arange(nx + 1, dtype=np.float64) / nx)
    yj = y0 + (y1 - y0) * (np.arange(ny + 1, dtype=np.float64) / ny)
    X, Y = np.meshgrid(xi, yj, indexing="xy")
    out = np.zeros(((nx + 1) * (ny + 1), 3))
    out[:, 0] = X.ravel()
    out[:, 1] = Y.ravel()
    return out


def grid_quad4(nx: int, ny: int) -> np.ndarray:
    """Connectivity of the nx*ny quads of :func:`grid_nodes`, CCW about +z."""
    i, j = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    i = i.ravel()
    j = j.ravel()
    n00 = j * (nx + 1) + i
    conn = np.stack([n00, n00 + 1, n00 + nx + 2, n00 + nx + 1], axis=1)
    return conn.astype(np.int32)


def perturb_grid_inplane(x: np.ndarray, n: int, amp: float, seed: int, stream: int) -> np.ndarray:
    """Shift nodes of an n x n grid of the unit square in-plane by U(-amp, amp).

    Interior nodes move in both in-plane components, nodes on an edge of the
    square only along that edge, and the four corners stay fixed, so the
    perturbed mesh still covers the unit square exactly.
    """
    x = x.copy()
    m = x.shape[0]
    du = uniform(seed, stream, m, -amp, amp)
    dv = uniform(seed, stream + 1, m, -amp, amp)
    ids = np.arange(m)
    i = ids % (n + 1)
    j = ids // (n + 1)
    move_x = (i > 0) & (i < n)
    move_y = (j > 0) & (j < n)
    x[:, 0] += np.where(move_x, du, 0.0)
    x[:, 1] += np.where(move_y, dv, 0.0)
    return x


def planar_noisy(ns: int, nm: int, lm: int, seed: int, name: str, noise: float = 0.1,
                 delta: float = 1e-9) -> Interface:
    """ns x ns quad4 slave vs nm x nm noisy quad4 master on the unit square."""
    xs = grid_nodes(ns, ns)
    cs = grid_quad4(ns, ns)
    hm = 1.0 / nm
    xm = perturb_grid_inplane(grid_nodes(nm, nm), nm, noise * hm, seed, 0) if noise > 0 \
        else grid_nodes(nm, nm)
    cm = grid_quad4(nm, nm)
    return Interface(name, xs, cs, QUAD4, xm, cm, QUAD4, lm=lm, delta=delta,
                     info={"ns": ns, "nm": nm, "noise": noise, "seed": seed})


def kite_master(ns: int, nm: int, d: float, lm: int = LM_STANDARD, name: str = "kite") -> Interface:
    """ns x ns quad4 slave vs an nm x nm master grid whose interior nodes with
    even i + j are moved by (d h_m, d h_m): every master quad keeps two opposite
    corners in place and has the other two moved along the same diagonal, a
    convex bilinear quad whose corner angle approaches 180 degrees as d -> 0.5
    (strongly distorted but valid elements)."""
    xs = grid_nodes(ns, ns)
    cs = grid_quad4(ns, ns)
    xm = grid_nodes(nm, nm)
    n = nm + 1
    i = np.arange(xm.shape[0]) % n
    j = np.arange(xm.shape[0]) // n
    sel = (i > 0) & (i < nm) & (j > 0) & (j < nm) & ((i + j) % 2 == 0)
    xm[sel, 0] += d / nm
    xm[sel, 1] += d / nm
    return Interface(name, xs, cs, QUAD4, xm, grid_quad4(nm, nm), QUAD4, lm=lm, delta=1e-9,
                     info={"ns": ns, "nm": nm, "kite_d": d})


QUAD8, TRI6 = 8, 6


def quadratic_grid(n: int, kind: str):
    """Parameter-plane nodes (uv in [0,1]^2, z = 0) and connectivity of an n x n
    quad8 mesh, or of its tri6 split (each quad cut along the diagonal from its
    first to its third corner).  Node ids: corners j (n+1) + i, then the
    mid-points of the horizontal edges, of the vertical edges and (tri6) of the
    diagonals.  quad8 order: 4 corners counter-clockwise, then the mid-sides of
    edges 0-1, 1-2, 2-3, 3-0; tri6: 3 corners, then edges 0-1, 1-2, 2-0."""
    h = 1.0 / n
    corners = grid_nodes(n, n)
    i, j = np.meshgrid(np.arange(n), np.arange(n + 1), indexing="xy")
    hmid = np.stack([(i.ravel() + 0.5) * h, j.ravel() * h, np.zeros(i.size)], 1)
    i, j = np.meshgrid(np.arange(n + 1), np.arange(n), indexing="xy")
    vmid = np.stack([i.ravel() * h, (j.ravel() + 0.5) * h, np.zeros(i.size)], 1)
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    dmid = np.stack([(i.ravel() + 0.5) * h, (j.ravel() + 0.5) * h, np.zeros(i.size)], 1)
    nc, nh, nv = corners.shape[0], hmid.shape[0], vmid.shape[0]
    i = i.ravel()
    j = j.ravel()
    c00 = j * (n + 1) + i
    c10, c11, c01 = c00 + 1, c00 + n + 2, c00 + n + 1
    hb, ht = nc + j * n + i, nc + (j + 1) * n + i
    vl, vr = nc + nh + j * (n + 1) + i, nc + nh + j * (n + 1) + i + 1
    if kind == "quad8":
        x = np.concatenate([corners, hmid, vmid])
        conn = np.stack([c00, c10, c11, c01, hb, vr, ht, vl], 1)
    elif kind == "tri6":
        x = np.concatenate([corners, hmid, vmid, dmid])
        dg = nc + nh + nv + j * n + i
        lower = np.stack([c00, c10, c11, hb, vr, dg], 1)
        upper = np.stack([c00, c11, c01, dg, ht, vl], 1)
        conn = np.empty((2 * lower.shape[0], 6), dtype=np.int64)
        conn[0::2] = lower
        conn[1::2] = upper
    else:
        raise ValueError(kind)
    return x, conn.astype(np.int32)


def quadratic_planar(ns: int, nm: int, kind: str = "quad8", seed: int = SEED_BASE + 21,
                     noise: float = 0.1, warp: float = 0.0, name: str = "quadratic") -> Interface:
    """ns x ns quad8 (or tri6) slave mesh on the unit square against an nm x nm
    quad4 master with the in-plane node noise of planar_noisy.  warp > 0 moves
    every slave node (mid-sides included) in-plane by warp * h_s * sin(pi x)
    sin(pi y) along (1, 1): curved element edges, boundary unchanged."""
    xs, cs = quadratic_grid(ns, kind)
    if warp:
        f = warp / ns * np.sin(np.pi * xs[:, 0]) * np.sin(np.pi * xs[:, 1])
        xs = xs.copy()
        xs[:, 0] += f
        xs[:, 1] += f
    m = planar_noisy(2, nm, LM_STANDARD, seed, name, noise=noise)
    return Interface(name, xs, cs, QUAD8 if kind == "quad8" else TRI6, m.xm, m.conn_m, QUAD4, lm=LM_STANDARD,
                     delta=1e-9, info={"ns": ns, "nm": nm, "kind": kind, "noise": noise, "warp": warp})


def quadratic_cylinder(ns: int = 24, nm: int = 21, kind: str = "quad8", seed: int = SEED_BASE + 22,
                       name: str = "quadratic_cylinder") -> Interface:
    """Curved quadratic slave elements: the quad8 (tri6) mesh of the 90 degree
    cylinder patch r = 1, z in [0, 2] with every node (mid-sides included) on
    the cylinder, against the chord-quad4 master of cylinder_patch."""
    xs, cs = quadratic_grid(ns, kind)
    th = 0.5 * math.pi * xs[:, 0]
    z = 2.0 * xs[:, 1]
    xs = np.stack([np.cos(th), np.sin(th), z], 1)
    cyl = cylinder_patch(4, nm, LM_STANDARD, seed, name)
    return Interface(name, xs, cs, QUAD8 if kind == "quad8" else TRI6, cyl.xm, cyl.conn_m, QUAD4, lm=LM_STANDARD,
                     delta=0.05 / ns, info={"ns": ns, "nm": nm, "kind": kind})


def planar_8x7() -> Interface:
    """8x8 vs 7x7 quad4, +-0.1 h_m in-plane master noise, standard LMs."""
    return planar_noisy(8, 7, LM_STANDARD, SEED_BASE + 1, "planar_8x7")


def planar_2000x1733() -> Interface:
    """2000x2000 vs 1733x1733 quad4, +-0.1 h_m master noise, dual LMs."""
    return planar_noisy(2000, 1733, LM_DUAL, SEED_BASE + 5, "planar_2000x1733")


def cylinder_patch(ns: int = 200, nm: int = 173, lm: int = LM_DUAL,
                   seed: int = SEED_BASE + 2, name: str = "cylinder_200x173",
                   gap_rel: float = 0.01) -> Interface:
    """90 degree cylinder patch r=1, z in [0, 2]: chord quads, master radius noise.

    Slave nodes sit on r = 1 (each slave quad is a planar chord rectangle);
    master node radii are 1 + N(0, (gap_rel * h)^2) with h the largest master
    edge length.  Nodes are ordered so that the normal points outwards.
    """
    def nodes(n, radii=None):
        th = (0.5 * math.pi) * (np.arange(n + 1) / n)
        zz = 2.0 * (np.arange(n + 1) / n)
        T, Z = np.meshgrid(th, zz, indexing="xy")
        T = T.ravel()
        Z = Z.ravel()
        r = np.ones_like(T) if radii is None else radii
        return np.stack([r * np.cos(T), r * np.sin(T), Z], axis=1)

    xs = nodes(ns)
    cs = grid_quad4(ns, ns)
    h_m = max(2.0 * math.sin(0.25 * math.pi / nm), 2.0 / nm)
    radii = 1.0 + (gap_rel * h_m) * normal(seed, 0, (nm + 1) * (nm + 1))
    xm = nodes(nm, radii)
    cm = grid_quad4(nm, nm)
    h_s = max(2.0 * math.sin(0.25 * math.pi / ns), 2.0 / ns)
    return Interface(name, xs, cs, QUAD4, xm, cm, QUAD4, lm=lm, delta=0.05 * h_s,
                     info={"ns": ns, "nm": nm, "h_m": h_m, "h_s": h_s, "seed": seed})


def mixed_tri(ns: int = 300, nm: int = 400, lm: int = LM_STANDARD,
              seed: int = SEED_BASE + 3, name: str = "mixed_300x400",
              angle_deg: float = 7.0, offset=(0.013, 0.029)) -> Interface:
    """ns x ns quad4 slave vs an nm x nm grid of tri3 (random diagonals), rotated."""
    xs = grid_nodes(ns, ns)
    cs = grid_quad4(ns, ns)
    xm = grid_nodes(nm, nm)
    q = grid_quad4(nm, nm)
    flip = uniform01(seed, 0, q.shape[0]) < 0.5
    n00, n10, n11, n01 = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    t_a = np.where(flip[:, None], np.stack([n00, n10, n01], 1), np.stack([n00, n10, n11], 1))
    t_b = np.where(flip[:, None], np.stack([n10, n11, n01], 1), np.stack([n00, n11, n01], 1))
    cm = np.empty((2 * q.shape[0], 3), dtype=np.int32)
    cm[0::2] = t_a
    cm[1::2] = t_b
    a = math.radians(angle_deg)
    c, s = math.cos(a), math.sin(a)
    u = xm[:, 0] - 0.5
    v = xm[:, 1] - 0.5
    xm = np.stack([0.5 + c * u - s * v + offset[0], 0.5 + s * u + c * v + offset[1],
                   np.zeros_like(u)], axis=1)
    return Interface(name, xs, cs, QUAD4, xm, cm, TRI3, lm=lm, delta=1e-9,
                     info={"ns": ns, "nm": nm, "angle_deg": angle_deg,
                           "offset": list(offset), "seed": seed})


def batched_512(n_interfaces: int = 512, seed: int = SEED_BASE + 4,
                n_lo: float = 4.0, n_hi: float = 128.0) -> list[Interface]:
    """Independent planar quad4/quad4 interfaces of uneven size."""
    u_n = uniform01(seed, 0, n_interfaces)
    u_r = uniform01(seed, 1, n_interfaces)
    u_dx = uniform(seed, 2, n_interfaces, -0.05, 0.05)
    u_dy = uniform(seed, 3, n_interfaces, -0.05, 0.05)
    out = []
    for k in range(n_interfaces):
        n = int(round(math.exp(math.log(n_lo) + u_n[k] * (math.log(n_hi) - math.log(n_lo)))))
        nm = max(2, int(round(n * (0.7 + 0.6 * u_r[k]))))
        xs = grid_nodes(n, n)
        cs = grid_quad4(n, n)
        xm = grid_nodes(nm, nm, u_dx[k], u_dy[k], 1.0 + u_dx[k], 1.0 + u_dy[k])
        cm = grid_quad4(nm, nm)
        out.append(Interface(f"batched_{k}", xs, cs, QUAD4, xm, cm, QUAD4,
                             lm=LM_STANDARD, delta=1e-9,
                             info={"n": n, "nm": nm, "dx": float(u_dx[k]), "dy": float(u_dy[k])}))
    return out


def matching(n: int, lm: int, seed: int = SEED_BASE + 11, noise: float = 0.0) -> tuple[Interface, np.ndarray]:
    """Master = slave mesh with permuted node ids; returns (interface, perm).

    ``perm[i]`` is the master id of slave node ``i``.  With ``noise`` > 0 the
    shared nodes are moved in-plane (both sides identically).
    """
    xs = grid_nodes(n, n)
    if noise > 0:
        xs = perturb_grid_inplane(xs, n, noise / n, seed, 4)
    cs = grid_quad4(n, n)
    order = np.argsort(uniform01(seed, 2, xs.shape[0]), kind="stable")
    perm = np.empty_like(order)
    perm[order] = np.arange(order.size)
    xm = xs[order].copy()
    cm = perm[cs].astype(np.int32)
    # rotate each master element's node list by a random amount (same cycle)
    rot = (uniform01(seed, 3, cs.shape[0]) * 4).astype(np.int64) % 4
    idx = (np.arange(4)[None, :] + rot[:, None]) % 4
    cm = np.take_along_axis(cm, idx, axis=1).astype(np.int32)
    return Interface(f"matching_{n}", xs, cs, QUAD4, xm, cm, QUAD4, lm=lm, delta=1e-9), perm


def by_name(name: str):
    table = {
        "planar_8x7": planar_8x7,
        # smaller member of the planar family (profiling captures)
        "planar_600x520": lambda: planar_noisy(600, 520, LM_DUAL, SEED_BASE + 6, "planar_600x520"),
        "cylinder_200x173": cylinder_patch,
        "mixed_300x400": mixed_tri,
        "batched_512": batched_512,
        "planar_2000x1733": planar_2000x1733,
    }
    return table[name]()
