"""GPU-vs-oracle comparison helpers for the parity tests.

Node flags must agree on every node.  Index data (vertex keys and
generators, arc records, loops, holes, triangle counts per item) must match
bit-exactly on every node that is not flagged near-tangent (a strut pair
within 1e-6 of tangency, the one exemption the parity contract allows);
nodes flagged degenerate (the lattice model is violated there, e.g. a
vertex past a strut's far end) run the same per-node algorithm on both sides
and are compared like any other.  Coordinates agree within 2e-5 relative for
FP32 (vertex offsets relative to their length plus the nodal radius, angles
relative to 2 pi,
absolute STL coordinates relative to their magnitude plus the radius), and
1e-12 for the FP64 instantiation's meta-mesh data.
"""
from __future__ import annotations

import numpy as np

import oracle

NEAR_TANGENT = 1
DEGENERATE = 2
EXEMPT = NEAR_TANGENT


def lattice_as(lat, dtype):
    """The lattice rounded to `dtype` (both sides then see identical inputs)."""
    return {"xyz": lat["xyz"].astype(dtype).astype(np.float64), "ends": lat["ends"],
            "radii": lat["radii"].astype(dtype).astype(np.float64), "name": lat.get("name", "")}


def to_device(lat, dtype):
    import torch
    td = torch.float32 if dtype == np.float32 else torch.float64
    return (torch.tensor(lat["xyz"], dtype=td, device="cuda").contiguous(),
            torch.tensor(lat["ends"], dtype=torch.int32, device="cuda").contiguous(),
            torch.tensor(lat["radii"], dtype=td, device="cuda").contiguous())


class Report:
    def __init__(self):
        self.errors = []
        self.checked_nodes = 0
        self.exempt_nodes = 0
        self.max_dz = 0.0
        self.max_dphi = 0.0
        self.bad_nodes = []

    def fail(self, msg, node=None):
        if node is not None:
            self.bad_nodes.append(node)
        if len(self.errors) < 50:
            self.errors.append(msg)

    def ok(self):
        return not self.errors


def compare_metamesh(g, o: oracle.Oracle, nodes=None, z_tol=2e-5, phi_tol=2e-5, node_map=None,
                     exempt=EXEMPT, degenerate_tol=None):
    """Compare the GPU download `g` with oracle `o` node by node.
    node_map: oracle node id -> GPU node id (sub-lattice comparisons).
    exempt: node-flag bits that exempt a node from the data comparison (its
    flags are still compared; on an exempt node only the exempting bits).
    degenerate_tol: coordinate tolerance on nodes flagged degenerate (their
    steep sections are ill-conditioned), default z_tol / phi_tol."""
    rep = Report()
    row_o, adj_o, R_o = o.csr()
    nodes = range(o.N) if nodes is None else nodes
    for n in nodes:
        n = int(n)
        gn = n if node_map is None else int(node_map[n])
        nd = o.node(n)
        fo = nd["flags"]
        fg = int(g["node_flags"][gn])
        if (fo & exempt) != (fg & exempt) or (not fo & exempt and fo != fg):
            rep.fail(f"node {n}: flags oracle {fo} gpu {fg}", n)
            continue
        if fo & exempt:
            rep.exempt_nodes += 1
            rep.exempt_flags = getattr(rep, "exempt_flags", 0) | fo
            continue
        rep.checked_nodes += 1
        ztol, ptol = z_tol, phi_tol
        if degenerate_tol is not None and fo & DEGENERATE:
            ztol = ptol = degenerate_tol
        R = R_o[n]
        v0, v1 = g["vtx_off"][gn], g["vtx_off"][gn + 1]
        if v1 - v0 != len(nd["vz"]):
            rep.fail(f"node {n}: V oracle {len(nd['vz'])} gpu {v1 - v0}", n)
            continue
        if not np.array_equal(g["vtx_key"][v0:v1], nd["vkey"]) or \
           not np.array_equal(g["vtx_flags"][v0:v1], nd["vflags"]) or \
           not np.array_equal(g["vtx_gen"][v0:v1], nd["vgen"]):
            rep.fail(f"node {n}: vertex keys/flags/generators differ\n  o {nd['vkey']} {nd['vgen']}\n  g {g['vtx_key'][v0:v1]} {g['vtx_gen'][v0:v1]}", n)
            continue
        # relative to |z| + R: a vertex far from its node (degenerate nodes)
        # is stored to FP32 precision of its magnitude
        scale = np.linalg.norm(nd["vz"], axis=1) + R
        dz = (np.abs(g["vtx_z"][v0:v1].astype(np.float64) - nd["vz"]).max(axis=1, initial=0.0) / scale).max(initial=0.0)
        rep.max_dz = max(rep.max_dz, dz)
        if dz > ztol:
            rep.fail(f"node {n}: vertex positions differ by {dz:.3g} (|z| + R)", n)
        a0, a1 = g["arc_off"][gn], g["arc_off"][gn + 1]
        if a1 - a0 != len(nd["arc_i"]):
            rep.fail(f"node {n}: arcs oracle {len(nd['arc_i'])} gpu {a1 - a0}", n)
            continue
        ga = g["arc_ends"][a0:a1]
        av = g["arc_vtx"][a0:a1]
        gmap = None
        if node_map is not None:
            gmap = g["_end_map"]
        oe = nd["arc_i"][:, :2].copy()
        if gmap is not None:
            oe = np.where(oe >= 0, gmap[np.maximum(oe, 0)], -1)
        if not np.array_equal(ga, oe) or not np.array_equal(av & 255, nd["arc_i"][:, 2]) or \
           not np.array_equal((av >> 8) & 255, nd["arc_i"][:, 3]):
            rep.fail(f"node {n}: arc records differ\n  o {nd['arc_i'].tolist()}\n  g {np.c_[ga, av & 255, (av >> 8) & 255].tolist()}", n)
            continue
        dp = np.abs(g["arc_phi"][a0:a1].astype(np.float64) - nd["arc_f"]).max(initial=0.0) / (2 * np.pi)
        rep.max_dphi = max(rep.max_dphi, dp)
        if dp > ptol:
            rep.fail(f"node {n}: arc angles differ by {dp:.3g} x 2pi", n)
        # loops, per local strut end
        p = 0
        b = row_o[n]
        for li, ln in enumerate(nd["loop_len"]):
            eid = adj_o[b + li]
            geid = eid if gmap is None else gmap[eid]
            e0, e1 = g["end_off"][geid], g["end_off"][geid + 1]
            if not np.array_equal(g["loop_ent"][e0:e1], nd["loop_ent"][p:p + ln]):
                rep.fail(f"node {n} end {eid}: loop entries differ\n  o {nd['loop_ent'][p:p + ln]}\n  g {g['loop_ent'][e0:e1]}", n)
            p += ln
        h0, h1 = g["hole_off_n"][gn], g["hole_off_n"][gn + 1]
        if h1 - h0 != len(nd["hole_len"]):
            rep.fail(f"node {n}: holes oracle {len(nd['hole_len'])} gpu {h1 - h0}", n)
            continue
        p = 0
        for hh, ln in enumerate(nd["hole_len"]):
            q0, q1 = g["hole_off"][h0 + hh], g["hole_off"][h0 + hh + 1]
            if not np.array_equal(g["hole_ent"][q0:q1], nd["hole_ent"][p:p + ln]):
                rep.fail(f"node {n} hole {hh}: entries differ", n)
            p += ln
    return rep


def parse_stl(records):
    """uint8 [T, 50] -> (normals [T,3], vertices [T,3,3]) float32."""
    r = np.ascontiguousarray(records)
    f = r[:, :48].copy().view(np.float32).reshape(-1, 12)
    return f[:, :3], f[:, 3:].reshape(-1, 3, 3)


def compare_triangles(gn, gv, otris, R_max, tol=2e-5):
    """Per-triangle comparison of the GPU STL records with the oracle's
    triangles (same order): vertices within tol relative (magnitude + R);
    normals within the bound that the vertex tolerance implies for the
    triangle's conditioning."""
    ov = otris[:, 1:]
    on = otris[:, 0]
    if gv.shape[0] != ov.shape[0]:
        return [f"triangle count gpu {gv.shape[0]} oracle {ov.shape[0]}"], 0.0, 0.0
    scale = np.abs(ov) + R_max
    dv = (np.abs(gv.astype(np.float64) - ov) / scale).max(axis=(1, 2))
    e = [ov[:, 1] - ov[:, 0], ov[:, 2] - ov[:, 1], ov[:, 0] - ov[:, 2]]
    emax = np.max([np.linalg.norm(x, axis=1) for x in e], axis=0)
    area2 = np.linalg.norm(np.cross(e[0], -e[2]), axis=1)
    smax = np.abs(ov).max(axis=(1, 2)) + R_max
    cond = np.where(area2 > 0, smax * emax / np.maximum(area2, 1e-300), np.inf)
    # a vertex error d moves the normal by about d / height, and the height
    # of a triangle is area2 / emax: the vertex tolerance tol (|x| + R) allows
    # normal errors up to about 2 tol (|x| + R) emax / area2 = 2 tol cond
    # (two vertices moving)
    ntol = 1e-4 + 2.0 * tol * cond
    dn = np.linalg.norm(gn.astype(np.float64) - on, axis=1)
    good = np.isfinite(cond)
    errs = []
    bad_v = np.nonzero(dv > tol)[0]
    if bad_v.size:
        errs.append(f"{bad_v.size} triangles with vertices off by up to {dv.max():.3g} (first {bad_v[:5]})")
    bad_n = np.nonzero(good & (dn > ntol))[0]
    if bad_n.size:
        errs.append(f"{bad_n.size} triangles with normals off (first {bad_n[:5]}, dn {dn[bad_n[:5]]})")
    return errs, float(dv.max(initial=0)), float(np.where(good, dn / ntol, 0).max(initial=0))
