"""Seeded synthetic lattice generators (inputs only).

This module builds the node coordinates, strut end indices and per-end radii
of the synthetic lattices used by the tests and the benchmark.  It holds no
part of the meta-meshing or triangulation arithmetic: it is shared by the
CUDA path and the oracle only as a source of inputs.

The paper's own models (tetgen lattices of Venus, Cow, Bunny, Dragon, Bone,
Teddy, Kitten and two GrabCAD parts, Section 6 and Table 1) are not
available; these generators stand in for them with the same kind of
structure: struts tangent to nodal spheres (Section 4.1), radius/length
ratios of 0.05-0.2, node valences from 1 to the mid twenties, cylinders and
cones, and sizes from thousands to a billion struts.

Every generator returns a dict with
  xyz   : (N, 3) float64 node centres
  ends  : (E, 2) int32 node ids of the two strut ends
  radii : (E, 2) float64 radius at end 0 / end 1 (a node property, so equal
          to the radius of the node each end sits on)
"""
from __future__ import annotations

import numpy as np

SEED = 20240524


def _pack(xyz, ends, node_r, name):
    ends = np.ascontiguousarray(ends, dtype=np.int32)
    radii = np.ascontiguousarray(node_r[ends], dtype=np.float64)
    return {"xyz": np.ascontiguousarray(xyz, dtype=np.float64), "ends": ends,
            "radii": radii, "name": name}


def bcc(nx: int, ny: int | None = None, nz: int | None = None, radius=0.08,
        jitter: float = 0.0, radius_range=None, seed: int = SEED):
    """Body-centred-cubic lattice of nx*ny*nz unit cells.

    Corner nodes (i, j, k) in [0,nx]x[0,ny]x[0,nz] come first (id
    i + (nx+1)(j + (ny+1)k)), then the cell centres (i+.5, j+.5, k+.5) with
    id (nx+1)(ny+1)(nz+1) + i + nx(j + ny k).  Each cell contributes 8
    struts centre -> corner, ordered by cell id then by corner bit
    (bit0 = +x, bit1 = +y, bit2 = +z).  Optional Gaussian jitter of every
    node coordinate and a per-node radius drawn uniformly from radius_range.
    """
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    ci = np.arange(nx + 1)
    cj = np.arange(ny + 1)
    ck = np.arange(nz + 1)
    K, J, I = np.meshgrid(ck, cj, ci, indexing="ij")
    corners = np.stack([I.ravel(), J.ravel(), K.ravel()], 1).astype(np.float64)
    K, J, I = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    I, J, K = I.ravel(), J.ravel(), K.ravel()
    centres = np.stack([I, J, K], 1).astype(np.float64) + 0.5
    n_corner = corners.shape[0]
    xyz = np.concatenate([corners, centres], 0)
    cell = np.arange(nx * ny * nz)
    bits = np.arange(8)
    ox, oy, oz = bits & 1, (bits >> 1) & 1, (bits >> 2) & 1
    cid = ((I[:, None] + ox[None]) + (nx + 1) * ((J[:, None] + oy[None]) + (ny + 1) * (K[:, None] + oz[None])))
    ends = np.stack([np.repeat(n_corner + cell, 8), cid.ravel()], 1)
    rng = np.random.default_rng(seed)
    n = xyz.shape[0]
    if jitter > 0:
        xyz = xyz + rng.normal(0.0, jitter, size=xyz.shape)
    if radius_range is not None:
        node_r = rng.uniform(radius_range[0], radius_range[1], size=n)
    else:
        node_r = np.full(n, float(radius))
    return _pack(xyz, ends, node_r, f"bcc{nx}x{ny}x{nz}")


OCTET_OFFSETS = np.array([(1, 1, 0), (1, -1, 0), (1, 0, 1), (1, 0, -1), (0, 1, 1), (0, 1, -1)])


def octet(n: int, radius_range=(0.04, 0.08), seed: int = SEED, ncells=None):
    """Octet-truss (FCC) lattice of n^3 unit cells.

    Nodes are the cube corners and face centres: the doubled-integer points
    (a, b, c) in [0, 2n]^3 with a+b+c even, ordered c-major then b then a;
    coordinates are (a, b, c)/2.  Struts join every pair at distance
    1/sqrt(2), listed by lower node id then by offset in OCTET_OFFSETS.
    Node radii are uniform in radius_range, so struts between nodes of
    different radius are cones.
    """
    nx, ny, nz = (n, n, n) if ncells is None else ncells
    A, B, C = 2 * nx + 1, 2 * ny + 1, 2 * nz + 1
    cc, bb, aa = np.meshgrid(np.arange(C), np.arange(B), np.arange(A), indexing="ij")
    keep = ((aa + bb + cc) % 2) == 0
    ids = -np.ones((C, B, A), dtype=np.int64)
    ids[keep] = np.arange(int(keep.sum()))
    pts = np.stack([aa[keep], bb[keep], cc[keep]], 1)
    struts = []
    for oi, (da, db, dc) in enumerate(OCTET_OFFSETS):
        a2, b2, c2 = pts[:, 0] + da, pts[:, 1] + db, pts[:, 2] + dc
        ok = (a2 >= 0) & (a2 < A) & (b2 >= 0) & (b2 < B) & (c2 >= 0) & (c2 < C)
        src = np.nonzero(ok)[0]
        dst = ids[c2[ok], b2[ok], a2[ok]]
        struts.append(np.stack([src, dst, np.full(src.shape, oi)], 1))
    s = np.concatenate(struts, 0)
    order = np.lexsort((s[:, 2], s[:, 0]))
    ends = s[order, :2]
    rng = np.random.default_rng(seed)
    node_r = rng.uniform(radius_range[0], radius_range[1], size=pts.shape[0])
    return _pack(pts.astype(np.float64) * 0.5, ends, node_r, f"octet{nx}x{ny}x{nz}")


def irregular(n_nodes: int, kmin=4, kmax=16, sigma=0.25, seed: int = SEED, r_scale=0.3):
    """Irregular lattice: i.i.d. uniform points in the unit cube, each joined
    to its k_v nearest neighbours with k_v uniform in {kmin..kmax}; the
    directed kNN graph is symmetrised.  Node radius is lognormal with median
    r_scale (0.3) x mean strut length and log-sd sigma, clipped to 0.45 x the node's
    shortest incident strut so that adjacent spheres never overlap.  Struts
    are listed by (lower id, higher id)."""
    from scipy.spatial import cKDTree

    rng = np.random.default_rng(seed)
    pts = rng.random((n_nodes, 3))
    kv = rng.integers(kmin, kmax + 1, size=n_nodes)
    tree = cKDTree(pts)
    _, nb = tree.query(pts, k=kmax + 1, workers=-1)
    nb = nb[:, 1:]
    cols = np.arange(kmax)[None, :] < kv[:, None]
    src = np.repeat(np.arange(n_nodes), kv)
    dst = nb[cols]
    lo, hi = np.minimum(src, dst), np.maximum(src, dst)
    key = np.unique(lo.astype(np.int64) * n_nodes + hi)
    ends = np.stack([key // n_nodes, key % n_nodes], 1)
    L = np.linalg.norm(pts[ends[:, 0]] - pts[ends[:, 1]], axis=1)
    r = np.exp(rng.normal(np.log(r_scale * L.mean()), sigma, size=n_nodes))
    minL = np.full(n_nodes, np.inf)
    np.minimum.at(minL, ends[:, 0], L)
    np.minimum.at(minL, ends[:, 1], L)
    node_r = np.minimum(r, 0.45 * minL)
    return _pack(pts, ends, node_r, f"irregular{n_nodes}")


def single_strut(p0, p1, r0, r1):
    """Two nodes joined by one strut (radius r0 at p0, r1 at p1)."""
    xyz = np.array([p0, p1], dtype=np.float64)
    return _pack(xyz, np.array([[0, 1]]), np.array([r0, r1], dtype=np.float64), "strut")


def star(directions, radius=0.1, far_radii=None, length=1.0, centre=(0.0, 0.0, 0.0)):
    """One centre node (id 0) with struts to nodes at centre + length*d_i."""
    d = np.asarray(directions, dtype=np.float64)
    d = d / np.linalg.norm(d, axis=1, keepdims=True)
    c = np.asarray(centre, dtype=np.float64)
    xyz = np.concatenate([c[None], c[None] + length * d], 0)
    ends = np.stack([np.zeros(len(d), dtype=np.int64), np.arange(1, len(d) + 1)], 1)
    node_r = np.full(len(d) + 1, float(radius))
    if far_radii is not None:
        node_r[1:] = far_radii
    return _pack(xyz, ends, node_r, "star")


def sub_lattice(lat, node_ids):
    """The struts incident to `node_ids` with their end nodes, keeping the
    relative order of both node ids and strut ids.  Returns (sub, node_map,
    strut_map) where node_map / strut_map give the original ids."""
    node_ids = np.asarray(node_ids)
    ends = lat["ends"]
    sel = np.nonzero(np.isin(ends[:, 0], node_ids) | np.isin(ends[:, 1], node_ids))[0]
    nodes = np.unique(ends[sel].ravel())
    remap = {int(v): i for i, v in enumerate(nodes)}
    sub_ends = np.vectorize(remap.__getitem__)(ends[sel]).reshape(-1, 2)
    sub = {"xyz": lat["xyz"][nodes], "ends": sub_ends.astype(np.int32),
           "radii": lat["radii"][sel], "name": lat.get("name", "") + "-sub"}
    return sub, nodes, sel


def bcc_device(n: int, radius: float, device, dtype=None):
    """BCC n^3 lattice built directly on a CUDA device with torch (same ids
    and strut order as `bcc`).  Returns (xyz, ends, radii) tensors."""
    import torch

    dtype = torch.float32 if dtype is None else dtype
    n1 = n + 1
    nc = n1 ** 3
    ncell = n ** 3
    xyz = torch.empty((nc + ncell, 3), dtype=dtype, device=device)
    ar = torch.arange(nc, device=device, dtype=torch.int64)
    xyz[:nc, 0] = (ar % n1).to(dtype)
    xyz[:nc, 1] = ((ar // n1) % n1).to(dtype)
    xyz[:nc, 2] = (ar // (n1 * n1)).to(dtype)
    del ar
    ends = torch.empty((ncell * 8, 2), dtype=torch.int32, device=device)
    chunk = 1 << 24
    bits = torch.arange(8, device=device, dtype=torch.int64)
    ox, oy, oz = bits & 1, (bits >> 1) & 1, (bits >> 2) & 1
    for c0 in range(0, ncell, chunk):
        c1 = min(ncell, c0 + chunk)
        cell = torch.arange(c0, c1, device=device, dtype=torch.int64)
        i, j, k = cell % n, (cell // n) % n, cell // (n * n)
        xyz[nc + c0:nc + c1, 0] = i.to(dtype) + 0.5
        xyz[nc + c0:nc + c1, 1] = j.to(dtype) + 0.5
        xyz[nc + c0:nc + c1, 2] = k.to(dtype) + 0.5
        cid = (i[:, None] + ox) + n1 * ((j[:, None] + oy) + n1 * (k[:, None] + oz))
        ends[8 * c0:8 * c1, 0] = (nc + cell).repeat_interleave(8).to(torch.int32)
        ends[8 * c0:8 * c1, 1] = cid.reshape(-1).to(torch.int32)
        del cell, i, j, k, cid
    radii = torch.full((ncell * 8, 2), float(radius), dtype=dtype, device=device)
    return xyz, ends, radii
