"""Mesh checks used by the tests (independent of both the oracle and the
CUDA library): shared-edge manifoldness, Euler characteristic, winding
number, exact point-in-union for the lattice solid."""
from __future__ import annotations

import numpy as np


def weld(tris):
    """tris[T,3,3] absolute coordinates -> (vertex ids [T,3], n_vertices),
    vertices matched by their exact bit pattern."""
    pts = np.ascontiguousarray(tris.reshape(-1, 3))
    view = pts.view(np.dtype((np.void, pts.dtype.itemsize * 3))).ravel()
    _, inv = np.unique(view, return_inverse=True)
    return inv.reshape(-1, 3), int(inv.max()) + 1 if inv.size else 0


def edge_report(ids):
    """Counts of undirected edges by multiplicity and whether every edge is
    used once in each direction (consistently oriented 2-manifold)."""
    a = ids[:, [0, 1, 2]].ravel()
    b = ids[:, [1, 2, 0]].ravel()
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    und = lo.astype(np.int64) * (ids.max() + 1) + hi
    uniq, cnt = np.unique(und, return_counts=True)
    directed = a.astype(np.int64) * (ids.max() + 1) + b
    dup_directed = directed.size - np.unique(directed).size
    return {"edges": uniq.size, "mult": dict(zip(*np.unique(cnt, return_counts=True))),
            "dup_directed": int(dup_directed), "degenerate": int(((a == b)).sum())}


def euler(ids, nv):
    rep = edge_report(ids)
    return nv - rep["edges"] + ids.shape[0], rep


def winding(tris, pts):
    """Generalised winding number of a triangle soup at pts (solid angles,
    Van Oosterom & Strackee)."""
    out = np.zeros(len(pts))
    for q, p in enumerate(pts):
        a = tris[:, 0] - p
        b = tris[:, 1] - p
        c = tris[:, 2] - p
        la, lb, lc = (np.linalg.norm(x, axis=1) for x in (a, b, c))
        det = np.einsum("ij,ij->i", a, np.cross(b, c))
        den = la * lb * lc + np.einsum("ij,ij->i", a, b) * lc + np.einsum("ij,ij->i", b, c) * la \
            + np.einsum("ij,ij->i", c, a) * lb
        out[q] = np.sum(2.0 * np.arctan2(det, den)) / (4 * np.pi)
    return out


def union_margin(lat, pts):
    """Signed lower bound on the distance from pts to the boundary of the
    lattice solid: positive inside, negative outside, |value| never above the
    true distance (max over the primitives of a per-primitive bound)."""
    xyz, ends, radii = lat["xyz"], lat["ends"], lat["radii"]
    node_r = np.zeros(len(xyz))
    node_r[ends[:, 0]] = radii[:, 0]
    node_r[ends[:, 1]] = radii[:, 1]
    m = np.full(len(pts), -np.inf)
    for c, r in zip(xyz, node_r):
        m = np.maximum(m, r - np.linalg.norm(pts - c, axis=1))
    for (a, b), (ra, rb) in zip(ends, radii):
        d = xyz[b] - xyz[a]
        L = np.linalg.norm(d)
        u = d / L
        s = (ra - rb) / L
        co = np.sqrt(1 - s * s)
        x = (pts - xyz[a]) @ u
        rad = np.linalg.norm((pts - xyz[a]) - np.outer(x, u), axis=1)
        mi = np.minimum(((ra - s * x) / co - rad) * co, np.minimum(x - ra * s, L + rb * s - x))
        m = np.maximum(m, mi)
    return m


def inside_union(lat, pts):
    """Exact membership in the union of nodal spheres and the frusta tangent
    to them (the lattice solid of Section 4.1)."""
    xyz, ends, radii = lat["xyz"], lat["ends"], lat["radii"]
    node_r = np.zeros(len(xyz))
    node_r[ends[:, 0]] = radii[:, 0]
    node_r[ends[:, 1]] = radii[:, 1]
    ins = np.zeros(len(pts), dtype=bool)
    for c, r in zip(xyz, node_r):
        ins |= np.linalg.norm(pts - c, axis=1) < r
    for (a, b), (ra, rb) in zip(ends, radii):
        d = xyz[b] - xyz[a]
        L = np.linalg.norm(d)
        u = d / L
        s = (ra - rb) / L
        co = np.sqrt(1 - s * s)
        x = (pts - xyz[a]) @ u
        rad = np.linalg.norm((pts - xyz[a]) - np.outer(x, u), axis=1)
        ok = (x >= ra * s) & (x <= L + rb * s) & (rad < (ra - s * x) / co)
        ins |= ok
    return ins
