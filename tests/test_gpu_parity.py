"""CUDA path vs FP64 oracle, element by element, through the C ABI.

Meta-mesh (Section 4.3 of arXiv 2405.15197) and triangulation (Section 5,
Algorithm 1) on seeded synthetic lattices: BCC (the 10^3 closed-form case,
FP64 and FP32), octet-truss cones, jittered BCC, irregular kNN lattices,
single struts and stars, plus invalid inputs.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_2405_15197_gb300 import lattices as L  # noqa: E402
from paper_2405_15197_gb300 import liblm  # noqa: E402
from tests import parity as P  # noqa: E402

LATTICES = {
    "bcc10": lambda: L.bcc(10, radius=0.08),
    "bcc3": lambda: L.bcc(3, radius=0.1),
    "octet3": lambda: L.octet(3),
    "bccjit4": lambda: L.bcc(4, jitter=0.05, radius_range=(0.05, 0.09)),
    "irregular": lambda: L.irregular(1500, seed=9, r_scale=0.06),
    # the irregular configuration's radius law (median 0.3 x mean strut):
    # nearly every node violates the lattice model (sections past a strut's
    # length, steep sections) and is compared like any other
    "irr03": lambda: L.irregular(1500, seed=9, r_scale=0.3),
    "strut": lambda: L.single_strut((0.1, 0.2, 0.3), (1.0, 0.7, 0.5), 0.1, 0.1),
    "cone": lambda: L.single_strut((0.1, 0.2, 0.3), (1.0, 0.7, 0.5), 0.12, 0.05),
    "star5": lambda: L.star([(1, 0, 0), (0, 1, 0.2), (-1, 0.3, 0), (0.2, -1, 0.5), (0, 0, 1)],
                            radius=0.12, far_radii=[0.05, 0.09, 0.12, 0.07, 0.1]),
    # annular exposed spheres (reading 10): two narrowing cones with disjoint
    # caps, their two contours stitched as one band
    "annular": lambda: L.star([(1, 0, 0), (-1, 0, 0)], radius=0.2, far_radii=[0.1, 0.1]),
    "annular150": lambda: L.star([(1, 0, 0), (math.cos(math.radians(150)), math.sin(math.radians(150)), 0.0)],
                                 radius=0.2, far_radii=[0.05, 0.05], length=0.5),
    "annular_asym": lambda: L.star([(1, 0.05, 0.02), (-1, 0.03, -0.04)], radius=0.2, far_radii=[0.08, 0.12]),
}
_cache = {}


def build(name, dtype):
    key = (name, dtype)
    if key not in _cache:
        lat = P.lattice_as(LATTICES[name](), dtype)
        xyz, ends, radii = P.to_device(lat, dtype)
        mm = liblm.MetaMesh(xyz, ends, radii)
        _cache[key] = (lat, mm, mm.download(), oracle.Oracle(lat))
    return _cache[key]


IRREGULAR = ("irregular", "irr03")


@pytest.mark.parametrize("name,dtype", [("bcc10", np.float64), ("bcc10", np.float32), ("bcc3", np.float32),
                                        ("octet3", np.float32), ("bccjit4", np.float32),
                                        ("irregular", np.float32), ("irr03", np.float32), ("strut", np.float32),
                                        ("cone", np.float32), ("star5", np.float32),
                                        ("octet3", np.float64), ("irregular", np.float64), ("irr03", np.float64)])
def test_metamesh_parity(name, dtype):
    """Flags agree on every node; only near-tangent nodes are exempt from the
    data comparison.  FP64 coordinates within 1e-12 R, or 1e-9 R on nodes
    flagged degenerate (steep sections: condition numbers up to about 1e5)."""
    lat, mm, g, o = build(name, dtype)
    tol = 1e-12 if dtype == np.float64 else 2e-5
    rep = P.compare_metamesh(g, o, z_tol=tol, phi_tol=tol,
                             degenerate_tol=1e-9 if dtype == np.float64 else None)
    assert rep.ok(), "\n".join(rep.errors[:8])
    assert rep.checked_nodes + rep.exempt_nodes == o.N
    if name in IRREGULAR:
        deg = sum(1 for n in range(o.N) if o.node(n)["flags"] & P.DEGENERATE)
        print(f"{name}: {rep.exempt_nodes}/{o.N} nodes exempt (near-tangent), {deg} degenerate")
        assert rep.exempt_nodes <= 0.01 * o.N
    else:
        assert rep.exempt_nodes == 0
    cnt = mm.counts()
    V, ne, nc, H = o.totals()
    if rep.exempt_nodes == 0:
        assert cnt[:4] == [V, ne, nc, H]


def test_bcc10_totals_gpu():
    """BCC 10^3, R = 0.08 (closed form): V 13,028, 22,800 elliptical and
    2,168 circular arcs, 602 holes, 293,296 triangles at k = 16."""
    for dt in (np.float64, np.float32):
        lat, mm, g, o = build("bcc10", dt)
        assert mm.counts()[:4] == [13028, 22800, 2168, 602]
        assert mm.tri_count(16) == 293296


def item_counts(mm, n_items):
    return np.array([liblm.lm_tri_range(mm.h, i, i + 1)[1] for i in range(n_items)])


@pytest.mark.parametrize("name,dtype,k", [("bcc10", np.float64, 16), ("bcc10", np.float32, 16),
                                          ("bcc3", np.float32, 8), ("octet3", np.float32, 8),
                                          ("octet3", np.float32, 32), ("bccjit4", np.float32, 32),
                                          ("irregular", np.float32, 16), ("irr03", np.float32, 16),
                                          ("irregular", np.float64, 16), ("irr03", np.float64, 8),
                                          ("strut", np.float32, 8),
                                          ("cone", np.float32, 33), ("star5", np.float32, 16),
                                          ("octet3", np.float64, 32), ("annular", np.float32, 16),
                                          ("annular150", np.float32, 32), ("annular_asym", np.float32, 8),
                                          ("annular150", np.float64, 16)])
def test_triangles_parity(name, dtype, k):
    """Triangle counts per item bit-exact and every record of every item
    that touches no near-tangent node within tolerance (vertices 2e-5
    relative to |x| + R for FP32, 1e-7 for FP64)."""
    lat, mm, g, o = build(name, dtype)
    exempt = {n for n in range(o.N) if (o.node(n)["flags"] | int(g["node_flags"][n])) & P.EXEMPT}
    total = mm.tri_count(k)
    oc = o.tri_counts(k)
    n_items = o.E + o.N
    gc = item_counts(mm, n_items) if n_items <= 20000 else None
    ends = lat["ends"]
    if not exempt:
        assert total == int(oc.sum())
        if gc is not None:
            assert np.array_equal(gc, oc)
        rec = mm.triangulate(k).cpu().numpy()
        gn, gv = P.parse_stl(rec)
        ot, oa, ov = o.triangulate(k)
        errs, dv, dn = P.compare_triangles(gn, gv, ot, float(lat["radii"].max()),
                                           tol=2e-5 if dtype == np.float32 else 1e-7)
        assert not errs, errs
        ga, gvol = mm.objective(k)
        assert ga == pytest.approx(oa, rel=1e-5) and gvol == pytest.approx(ov, rel=1e-5)
    else:
        # compare item by item, skipping items touching an exempt node
        assert gc is not None
        ok_items = [i for i in range(n_items)
                    if (i < o.E and ends[i, 0] not in exempt and ends[i, 1] not in exempt)
                    or (i >= o.E and (i - o.E) not in exempt)]
        assert np.array_equal(gc[ok_items], oc[ok_items])
        rec = mm.triangulate(k).cpu().numpy()
        gn, gv = P.parse_stl(rec)
        ot, _, _ = o.triangulate(k)
        goff = np.concatenate([[0], np.cumsum(gc)])
        ooff = np.concatenate([[0], np.cumsum(oc)])
        gi = np.concatenate([np.arange(goff[i], goff[i + 1]) for i in ok_items])
        oi = np.concatenate([np.arange(ooff[i], ooff[i + 1]) for i in ok_items])
        errs, dv, dn = P.compare_triangles(gn[gi], gv[gi], ot[oi], float(lat["radii"].max()),
                                           tol=2e-5 if dtype == np.float32 else 1e-7)
        assert not errs, errs
        print(f"{name} k={k}: {len(ok_items)}/{n_items} items compared, max dv {dv:.3g}")


@pytest.mark.parametrize("name,dtype,k", [("bcc3", np.float32, 8), ("bcc10", np.float32, 16),
                                          ("octet3", np.float32, 8), ("octet3", np.float32, 32),
                                          ("bccjit4", np.float32, 32), ("octet3", np.float64, 32),
                                          ("star5", np.float32, 16), ("annular", np.float32, 16),
                                          ("annular150", np.float32, 32), ("annular_asym", np.float32, 8)])
def test_gpu_mesh_is_watertight(name, dtype, k):
    """The GPU's triangles weld bitwise into a closed, consistently oriented
    2-manifold (every edge used once in each direction) with chi = 2 (nodes -
    struts): points shared by two struts, by a strut and a hole fan, or by a
    strut of the FP32 pass and one of the FP64 pass carry the same bits."""
    from tests import meshcheck as mc
    lat, mm, g, o = build(name, dtype)
    mm.tri_count(k)
    _, gv = P.parse_stl(mm.triangulate(k).cpu().numpy())
    ids, nv = mc.weld(gv)
    chi, rep = mc.euler(ids, nv)
    assert rep["mult"] == {2: rep["edges"]}, rep["mult"]
    assert rep["dup_directed"] == 0 and rep["degenerate"] == 0
    assert chi == 2 * (o.N - o.E)


def test_stl_layout_and_header():
    """Binary STL records: 50 bytes, normal + 3 vertices f32, attribute 0;
    header count field little-endian, saturating at 2^32 - 1."""
    lat, mm, g, o = build("bcc3", np.float32)
    k = 8
    n = mm.tri_count(k)
    rec = mm.triangulate(k).cpu().numpy()
    assert rec.shape == (n, 50)
    assert np.all(rec[:, 48:] == 0)
    h = liblm.lm_stl_header(n)
    assert len(h) == 84 and int.from_bytes(h[80:], "little") == n
    assert int.from_bytes(liblm.lm_stl_header(5_000_000_000)[80:], "little") == 0xFFFFFFFF


def test_item_ranges_and_capacity():
    """Sub-ranges of items write the same records as the whole; a short
    output buffer is reported as LM_ERR_CAPACITY without writing past it."""
    lat, mm, g, o = build("octet3", np.float32)
    k = 8
    n = mm.tri_count(k)
    full = mm.triangulate(k).cpu().numpy()
    E, N = mm.n_struts, mm.n_nodes
    for b, e in [(0, 7), (5, E + 3), (E - 1, E + N), (E + 10, E + 11)]:
        first, cnt = liblm.lm_tri_range(mm.h, b, e)
        part = mm.triangulate(k, b, e).cpu().numpy()
        assert np.array_equal(part, full[first:first + cnt])
    out = torch.full((11, 50), 7, dtype=torch.uint8, device="cuda")
    liblm.lm_triangulate(mm.h, k, 0, E, out.data_ptr(), 10, None)
    assert liblm.lm_last_error(mm.h) == 4
    assert torch.all(out[10] == 7)


def test_empty_and_invalid_inputs():
    dev = "cuda"
    # no struts: an empty meta-mesh, no triangles
    xyz = torch.zeros((3, 3), dtype=torch.float32, device=dev)
    ends = torch.zeros((0, 2), dtype=torch.int32, device=dev)
    radii = torch.zeros((0, 2), dtype=torch.float32, device=dev)
    mm = liblm.MetaMesh(xyz, ends, radii)
    assert mm.counts()[:4] == [0, 0, 0, 0]
    assert mm.tri_count(8) == 0
    base = L.bcc(1, radius=0.1)

    def status(mut):
        lat = {k: v.copy() for k, v in base.items() if k != "name"}
        mut(lat)
        x, e, r = P.to_device(lat, np.float32)
        with pytest.raises(liblm.LmError) as ei:
            liblm.MetaMesh(x, e, r)
        return ei.value.status

    assert status(lambda l: l["radii"].__setitem__((0, 0), 0.2)) == 2          # radius mismatch
    assert status(lambda l: l["ends"].__setitem__((0, 1), 999)) == 1           # node out of range
    assert status(lambda l: l["ends"].__setitem__((0, 1), l["ends"][0, 0])) == 1  # self loop
    assert status(lambda l: l["radii"].__setitem__((1, 1), np.nan)) == 1       # NaN radius
    assert status(lambda l: l["xyz"].__setitem__((0, 0), np.nan)) == 1         # NaN coordinate

    def taper(l):
        l["radii"][:, 0] = 0.99
    assert status(taper) == 3                                                 # cone taper >= length
    star = L.star(np.random.default_rng(0).normal(size=(65, 3)), radius=0.01)
    x, e, r = P.to_device(star, np.float32)
    with pytest.raises(liblm.LmError) as ei:
        liblm.MetaMesh(x, e, r)
    assert ei.value.status == 8                                               # valence > 64
    with pytest.raises(liblm.LmError):
        liblm.lm_triangulate(mm.h, 9, 0, 1, 0, 0, None)                       # k without count


@pytest.mark.parametrize("name,dtype,k,chunk", [("octet3", np.float32, 32, 97), ("irregular", np.float32, 16, 1000),
                                                ("octet3", np.float64, 8, 61)])
def test_streaming_matches_direct(name, dtype, k, chunk):
    """Chunked triangulation streamed to pinned host slots (overlapped
    device-to-host copies; the per-chunk work replayed from two CUDA graphs)
    reproduces the direct output, including struts stitched by the FP64 pass."""
    lat, mm, g, o = build(name, dtype)
    n = mm.tri_count(k)
    full = mm.triangulate(k).cpu().numpy()
    n_items = mm.n_struts + mm.n_nodes
    max_chunk = max(liblm.lm_tri_range(mm.h, c, min(n_items, c + chunk))[1] for c in range(0, n_items, chunk))
    slot = 50 * max_chunk
    ring = torch.empty(3 * slot, dtype=torch.uint8, pin_memory=True)
    got = []

    def cb(ci, first_item, ntri, ptr, user):
        off = ptr - ring.data_ptr()
        got.append((ci, ring[off:off + 50 * ntri].numpy().copy()))

    tot = liblm.lm_triangulate_stream(mm.h, k, chunk, ring.data_ptr(), slot, 3, cb)
    assert tot == n
    got.sort(key=lambda x: x[0])
    cat = np.concatenate([x[1] for x in got]).reshape(-1, 50)
    assert np.array_equal(cat, full)


def test_autotuned_build_is_identical():
    """The autotuner (lm_options.autotune) only changes the launch shape of the
    persistent meta-mesh kernel: the meta-mesh is the same array for array."""
    lat = P.lattice_as(LATTICES["irregular"](), np.float32)
    xyz, ends, radii = P.to_device(lat, np.float32)
    ref = liblm.MetaMesh(xyz, ends, radii)
    opt = liblm.lm_options()
    opt.autotune = 1
    tuned = liblm.MetaMesh(xyz, ends, radii, options=opt)
    a, b = ref.download(), tuned.download()
    for key in a:
        assert np.array_equal(a[key], b[key]), key
    shape = liblm.lm_metamesh_launch_shape(tuned.h)
    for bw, npt in shape:
        assert (bw, npt) == (0, 0) or (bw in (1, 2, 4) and npt in (1, 2, 4, 8))
    assert shape[0][0] > 0
    assert liblm.lm_fp64_counts(tuned.h)[:8] == liblm.lm_fp64_counts(ref.h)[:8]


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_arena_gather_is_identical(dtype):
    """The count pass keeps each node's meta-mesh in an arena that a gather
    copies into the CSR layout, and nodes that do not fit go through the emit
    pass: with no arena, a small one (most nodes emitted) and the default one
    (every node gathered) the meta-mesh and the triangles are the same."""
    lat = P.lattice_as(LATTICES["irregular"](), dtype)
    xyz, ends, radii = P.to_device(lat, dtype)
    meshes = []
    for nbytes in (-1, 1 << 17, 3 << 18, 0):
        opt = liblm.lm_options()
        opt.arena_bytes = nbytes
        meshes.append(liblm.MetaMesh(xyz, ends, radii, options=opt))
    # the emit pass went over every node (no arena; a tiny one whose missed
    # nodes overflow the lists) and over the listed missed nodes only
    shapes = [liblm.lm_metamesh_emit_nodes(mm.h, listed=True) for mm in meshes]
    n_nodes = int(xyz.shape[0])
    assert shapes[0] == (n_nodes, False)
    assert shapes[1][1] is False and shapes[1][0] > n_nodes // 16 + 1024
    assert shapes[2][1] is True and 0 < shapes[2][0] < n_nodes
    assert shapes[3] == (0, False)
    ref = meshes[0].download()
    for mm in meshes[1:]:
        got = mm.download()
        for key in ref:
            assert np.array_equal(ref[key], got[key]), key
    recs = []
    for mm in meshes:
        mm.tri_count(8)
        recs.append(mm.triangulate(8).cpu().numpy())
    for r in recs[1:]:
        assert np.array_equal(recs[0], r)
    for mm in meshes:
        mm.close()
