"""Pins of the FP64 oracle against facts fixed by the paper and by geometry
(not against the oracle itself): closed forms, invariants, brute force.

Paper: arXiv 2405.15197.  Each test names the passage it pins.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2405_15197_gb300 import lattices as L
from tests import meshcheck as mc


# ---------------------------------------------------------------- helpers
def loops_of(o, n):
    """[(label_end_id or -1, dphi)] per local strut end of node n."""
    nd = o.node(n)
    out, p = [], 0
    for ln in nd["loop_len"]:
        ents = nd["loop_ent"][p:p + ln]
        p += ln
        lst = []
        for e in ents:
            a = int(e & 0x7FFFFFFF)
            lst.append((int(nd["arc_i"][a, 1]), float(nd["arc_f"][a, 1])))
        out.append(lst)
    return nd, out


# ------------------------------------------------------ P4: BCC 10^3 totals
def test_bcc10_closed_form_totals():
    """BCC 10x10x10, R=0.08, k=16 (derived closed form of the meta-mesh of
    Section 4.1 / 4.3.1 and the counts of Section 5 Eq. sampling)."""
    lat = L.bcc(10, radius=0.08)
    o = oracle.Oracle(lat)
    assert (o.N, o.E) == (2331, 8000)
    assert o.totals() == (13028, 22800, 2168, 602)
    assert (o.node_sizes()[:, 0] == 0).all()
    cnt = o.tri_counts(16)
    assert cnt.sum() == 293296
    assert 84 + 50 * int(cnt.sum()) == 14_664_884
    lat_cnt = cnt[:o.E]
    vals, num = np.unique(lat_cnt, return_counts=True)
    assert dict(zip(vals.tolist(), num.tolist())) == {34: 224, 35: 1944, 36: 5832}
    assert cnt[o.E:].sum() == 7688


# ------------------------------------------- P3: BCC node-level structures
@pytest.fixture(scope="module")
def bcc2():
    lat = L.bcc(2, radius=0.08)
    return lat, oracle.Oracle(lat)


def _node_at(lat, p):
    return int(np.nonzero(np.all(np.isclose(lat["xyz"], p), axis=1))[0][0])


def test_bcc_interior_node(bcc2):
    """Interior node (valence 8): 3 elliptical arcs of 2pi/3 per loop on the
    coordinate planes, 6 vertices at R sqrt(3/2) on the axes, 4 struts each."""
    lat, o = bcc2
    R = 0.08
    for p in [(1, 1, 1), (0.5, 0.5, 0.5)]:
        n = _node_at(lat, p)
        nd, lp = loops_of(o, n)
        assert nd["d"] == 8 and len(nd["vz"]) == 6 and len(nd["hole_len"]) == 0
        assert (nd["arc_i"][:, 1] >= 0).all() and len(nd["arc_i"]) == 12
        for loop in lp:
            assert len(loop) == 3
            for lab, dphi in loop:
                assert lab >= 0 and abs(dphi - 2 * math.pi / 3) < 1e-12
        vz = nd["vz"]
        assert np.allclose(np.sort(np.abs(vz).max(1)), R * math.sqrt(1.5), atol=1e-14)
        assert np.allclose(np.sort(np.abs(vz), 1)[:, :2], 0, atol=1e-14)
        for key in nd["vkey"]:
            assert bin(int(key)).count("1") == 4


def test_bcc_boundary_nodes(bcc2):
    """Face (valence 4), edge (2) and corner (1) nodes: loops of 5pi/6+5pi/6+pi/3,
    pi+pi and a full circle; vertex / arc / hole counts."""
    lat, o = bcc2
    cases = {(0, 1, 1): (4, 5, 4, 4, 1, [5 / 6, 5 / 6, 1 / 3]),
             (0, 0, 1): (2, 2, 1, 2, 1, [1, 1]),
             (0, 0, 0): (1, 1, 0, 1, 1, [2])}
    for p, (d, V, nell, ncirc, H, dph) in cases.items():
        n = _node_at(lat, p)
        nd, lp = loops_of(o, n)
        assert nd["d"] == d and len(nd["vz"]) == V and len(nd["hole_len"]) == H
        assert int((nd["arc_i"][:, 1] >= 0).sum()) == nell
        assert int((nd["arc_i"][:, 1] < 0).sum()) == ncirc
        for loop in lp:
            assert sorted(x[1] for x in loop) == pytest.approx(sorted(math.pi * f for f in dph), abs=1e-12)


# ------------------------------------------------ P5: topological invariants
@pytest.mark.parametrize("name", ["bcc3", "octet2", "bccjit3", "conestar"])
def test_euler_and_watertight(name):
    """Per node V - A + H = 2 - d; the triangulated surface is a closed,
    consistently oriented 2-manifold (every edge used once in each direction,
    vertices matched bitwise) with chi = 2 (nodes - struts), and encloses a
    positive volume (Section 5: strut stitching plus hole filling)."""
    lat = {"bcc3": lambda: L.bcc(3, radius=0.1),
           "octet2": lambda: L.octet(2),
           "bccjit3": lambda: L.bcc(3, jitter=0.05, radius_range=(0.05, 0.09)),
           "conestar": lambda: L.star([(1, 0, 0), (0, 1, 0.2), (-1, 0.3, 0), (0.2, -1, 0.5), (0, 0, 1)],
                                      radius=0.12, far_radii=[0.05, 0.09, 0.12, 0.07, 0.1])}[name]()
    o = oracle.Oracle(lat)
    s = o.node_sizes()
    assert (s[:, 0] == 0).all(), "lattice must be non-degenerate for this pin"
    row, _, _ = o.csr()
    deg = np.diff(row)
    assert np.all(s[:, 1] - s[:, 2] + s[:, 4] == 2 - deg)
    for k in (8, 16):
        tris, area, vol = o.triangulate(k)
        ids, nv = mc.weld(tris[:, 1:])
        chi, rep = mc.euler(ids, nv)
        assert rep["mult"] == {2: rep["edges"]}
        assert rep["dup_directed"] == 0 and rep["degenerate"] == 0
        assert chi == 2 * (o.N - o.E)
        assert vol > 0 and area > 0


# ------------------------------------- annular holes (reading 10): a band
def _annular_stars():
    c150 = (math.cos(math.radians(150)), math.sin(math.radians(150)), 0.0)
    return {
        # two antipodal narrowing cones: the exposed sphere between their
        # tangency circles is one band with two contours
        "antipodal": (L.star([(1, 0, 0), (-1, 0, 0)], radius=0.2, far_radii=[0.1, 0.1]), 0.4),
        # 150 degrees apart, cap half-angles 72.5 degrees: disjoint caps
        "tilted150": (L.star([(1, 0, 0), c150], radius=0.2, far_radii=[0.05, 0.05], length=0.5), 0.22),
        "asym": (L.star([(1, 0.05, 0.02), (-1, 0.03, -0.04)], radius=0.2, far_radii=[0.08, 0.12]), 0.4),
    }


@pytest.mark.parametrize("name", ["antipodal", "tilted150", "asym"])
def test_annular_band_closed_manifold(name):
    """A centre node whose two strut caps are disjoint: its exposed sphere is
    one component bounded by two contours (V - A + d + 2F - H = 2 with V = A
    = H = d = 2 gives F = 1), stitched as one band, so the mesh is a single
    closed, consistently oriented 2-manifold with chi = 2 (N - E) and a
    positive volume, the band having as many triangles as the two contours
    have points."""
    lat, _ = _annular_stars()[name]
    o = oracle.Oracle(lat)
    s = o.node_sizes()
    assert (s[:, 0] == 0).all()
    assert s[0, 1:].tolist() == [2, 2, 2, 2, 2]
    V, A, H, d = s[0, 1], s[0, 2], s[0, 4], 2
    assert (2 - V + A - d + H) // 2 == 1
    for k in (8, 16, 32):
        tris, area, vol = o.triangulate(k)
        ids, nv = mc.weld(tris[:, 1:])
        chi, rep = mc.euler(ids, nv)
        assert rep["mult"] == {2: rep["edges"]}
        assert rep["dup_directed"] == 0 and rep["degenerate"] == 0
        assert chi == 2 * (o.N - o.E)
        assert vol > 0 and area > 0
        cnt = o.tri_counts(k)
        assert cnt[o.E] == 2 * k


@pytest.mark.parametrize("k", [8, 16, 48])
def test_annular_band_area_closed_form(k):
    """Two antipodal cones with one half-angle (sin a = (R - r)/L): the two
    tangency circles are coaxial, radius R cos a at heights +-R sin a, and
    their k points lie at the same angles (both strut frames are built from
    the same axis), so the band is k rectangles of 2 R cos a sin(pi/k) by
    2 R sin a: area 4 k R^2 cos a sin a sin(pi/k), and every band vertex lies
    on one of the circles."""
    lat, _ = _annular_stars()["antipodal"]
    R, r, Ls = 0.2, 0.1, 1.0
    sa = (R - r) / Ls
    ca = math.sqrt(1 - sa * sa)
    o = oracle.Oracle(lat)
    tris, _, _ = o.triangulate(k)
    cnt = o.tri_counts(k)
    off = int(cnt[:o.E].sum())
    band = tris[off:off + int(cnt[o.E])]
    assert len(band) == 2 * k
    pts = band[:, 1:].reshape(-1, 3)
    assert np.allclose(np.abs(pts[:, 0]), R * sa, rtol=0, atol=1e-14)
    assert np.allclose(np.hypot(pts[:, 1], pts[:, 2]), R * ca, rtol=0, atol=1e-14)
    e1, e2 = band[:, 2] - band[:, 1], band[:, 3] - band[:, 1]
    area = 0.5 * np.linalg.norm(np.cross(e1, e2), axis=1).sum()
    assert area == pytest.approx(4 * k * R * R * ca * sa * math.sin(math.pi / k), rel=1e-12)
    # outward: every band normal points away from the axis
    mid = band[:, 1:].mean(1)
    nrm = np.cross(e1, e2)
    assert np.all(nrm[:, 1] * mid[:, 1] + nrm[:, 2] * mid[:, 2] > 0)


@pytest.mark.parametrize("name", ["antipodal", "tilted150", "asym"])
def test_annular_point_in_union_vs_winding(name):
    """Monte-Carlo points around the centre node (away from the far nodes'
    hole caps): inside the exact solid iff the mesh winds around them once,
    for points farther from the surface than the band's and the struts'
    sagittas.  Fanning each contour on its own would close each strut and
    leave the band of sphere between them outside the mesh."""
    lat, box = _annular_stars()[name]
    o = oracle.Oracle(lat)
    k = 48
    tris, _, _ = o.triangulate(k)
    rng = np.random.default_rng(3)
    pts = rng.uniform(-box, box, size=(4000, 3))
    ins = mc.inside_union(lat, pts)
    marg = mc.union_margin(lat, pts)
    assert np.all((marg > 0) == ins)
    # the band's chords sit at most R (1 - cos(g / 2)) inside the sphere,
    # g the widest angular gap between the two circles
    R = 0.2
    safe = np.abs(marg) > 0.2 * R + 4 * R * (1 - math.cos(math.pi / k))
    w = mc.winding(tris[:, 1:], pts[safe])
    assert safe.sum() > 1000 and ins[safe].sum() > 100
    assert np.all(np.abs(w - ins[safe]) < 1e-6)
    # points of the band region itself (inside the sphere, outside both
    # cones' caps, near the sphere) are inside the mesh
    band_pts = pts[safe & ins & (np.linalg.norm(pts, axis=1) < R) & (np.linalg.norm(pts, axis=1) > 0.5 * R)]
    assert len(band_pts) > 10


# --------------------------------------------- P2: isolated straight strut
@pytest.mark.parametrize("k", [6, 8, 16, 32, 64, 256])
def test_isolated_cylinder(k):
    """Single cylinder r, L: lateral area 2 k r sin(pi/k) L (-> 2 pi r L) and
    total volume L (k/2) r^2 sin(2pi/k) + 2 (1/3)(k/2) r^2 sin(2pi/k) r: two
    regular k-gons joined by a band, capped by fans to the projected
    barycentre of each hole (Section 5)."""
    r, Lh = 0.2, 1.7
    lat = L.single_strut((0.3, -0.2, 0.5), (0.3 + Lh * 0.6, -0.2 + Lh * 0.8, 0.5), r, r)
    o = oracle.Oracle(lat)
    _, a_lat, _ = o.triangulate(k, 0, 1, want_tris=False)
    assert a_lat == pytest.approx(2 * k * r * math.sin(math.pi / k) * Lh, rel=1e-12)
    _, _, vol = o.triangulate(k, want_tris=False)
    poly = 0.5 * k * r * r * math.sin(2 * math.pi / k)
    assert vol == pytest.approx(Lh * poly + 2 * poly * r / 3, rel=1e-10)
    if k == 256:
        assert a_lat == pytest.approx(2 * math.pi * r * Lh, rel=1e-4)


# ------------------------------------------------ P1: planar conic sections
@pytest.mark.parametrize("theta_deg", [60, 90, 120, 150])
def test_equal_cylinder_ellipse(theta_deg):
    """Two equal cylinders whose axes meet at angle theta intersect in a
    planar ellipse with semi-axes r and r/sin(theta/2) (Section 4.3.1)."""
    th = math.radians(theta_deg)
    r = 0.1
    u1 = np.array([1.0, 0, 0])
    u2 = np.array([math.cos(th), math.sin(th), 0])
    lat = L.star([u1, u2], radius=r, length=1.5)
    o = oracle.Oracle(lat)
    nd = o.node(0)
    ell = [a for a in range(len(nd["arc_i"])) if nd["arc_i"][a, 1] >= 0]
    assert len(ell) == 1
    P = o.arc_points(0, ell[0], 64)
    amaj = (u1 + u2) / np.linalg.norm(u1 + u2)
    bmin = np.cross(u1, u2) / np.linalg.norm(np.cross(u1, u2))
    x, y = P @ amaj, P @ bmin
    assert np.allclose((x * math.sin(th / 2) / r) ** 2 + (y / r) ** 2, 1.0, atol=1e-12)
    assert np.allclose(P @ (u1 - u2), 0, atol=1e-14)


@pytest.mark.parametrize("theta_deg,beyond", [(8.0, True), (10.0, True), (13.0, False), (16.0, False)])
def test_section_past_strut_length(theta_deg, beyond):
    """Lattice model (Section 4.1): a plane section must stay within the
    struts it joins.  For two equal cylinders of radius r at angle theta the
    section reaches the generator coordinate r cot(theta/2) (the end of the
    ellipse's major axis); the node is flagged degenerate (past a strut's
    length) exactly when that exceeds the strut length."""
    th = math.radians(theta_deg)
    r, length = 0.1, 1.0
    u1 = np.array([1.0, 0, 0])
    u2 = np.array([math.cos(th), math.sin(th), 0])
    lat = L.star([u1, u2], radius=r, length=length)
    o = oracle.Oracle(lat)
    tmax = r / math.tan(th / 2)
    # the envelope on strut 0 peaks at the closed form (dense sampling)
    phi = np.linspace(0, 2 * np.pi, 20001)
    t, lab = o.envelope(0, 0, phi)
    assert abs(t.max() - tmax) < 1e-6 * tmax
    fl = o.node(0)["flags"]
    assert bool(fl & 8) == beyond and bool(fl & 2) == beyond
    assert (tmax > length) == beyond


def _rot(axis, ang, v):
    axis = axis / np.linalg.norm(axis)
    return v * math.cos(ang) + np.cross(axis, v) * math.sin(ang) + axis * (axis @ v) * (1 - math.cos(ang))


@pytest.mark.parametrize("seed", range(6))
def test_paper_ellipse_construction(seed):
    """The paper's strut-plane ellipse (Section 4.3.1: o = (E1+E2)/2,
    a = (E1-E2)/2, b = lambda a^n, with F1, F2, E1, E2 built by rotations of
    the strut direction) with the cone angle read as
    alpha = asin((r^1 - r^0)/|v^1 - v^0|) describes the oracle's elliptical
    arc points exactly.  The plane is fitted to the arc points, so this also
    pins that two strut surfaces meet in a plane."""
    rng = np.random.default_rng(seed)
    R = 0.1
    u1 = rng.normal(size=3)
    u1 /= np.linalg.norm(u1)
    while True:
        u2 = rng.normal(size=3)
        u2 /= np.linalg.norm(u2)
        if 0.4 < math.acos(u1 @ u2) < 2.6:
            break
    far = rng.uniform(0.06, 0.14, size=2)
    lat = L.star([u1, u2], radius=R, far_radii=far, length=1.0)
    o = oracle.Oracle(lat)
    nd = o.node(0)
    ell = [a for a in range(len(nd["arc_i"])) if nd["arc_i"][a, 1] >= 0]
    assert len(ell) == 1
    P = o.arc_points(0, ell[0], 128)
    cen = P.mean(0)
    _, sv, vt = np.linalg.svd(P - cen)
    n = vt[2]
    assert sv[2] < 1e-12
    for strut, u, rf in ((0, u1, far[0]), (1, u2, far[1])):
        v0 = np.zeros(3)
        v1 = u * 1.0
        d = (v0 - v1) / np.linalg.norm(v0 - v1)
        dp = np.cross(d, n)
        dp /= np.linalg.norm(dp)
        alpha = math.asin((rf - R) / 1.0)
        F1 = v0 + _rot(dp, alpha - math.pi / 2, d) * R
        F2 = v0 + _rot(dp, math.pi / 2 - alpha, d) * R
        g1, g2 = _rot(dp, alpha, d), _rot(dp, -alpha, d)
        E1 = (n @ (cen - F1)) / (n @ g1) * g1 + F1
        E2 = (n @ (cen - F2)) / (n @ g2) * g2 + F2
        oc = 0.5 * (E1 + E2)
        a = 0.5 * (E1 - E2)
        lam = math.sqrt(1 - (a @ d) ** 2 / (math.cos(alpha) * np.linalg.norm(a)) ** 2)
        b = lam * np.cross(a, n)
        Q = P - oc
        x = Q @ a / (a @ a)
        y = Q @ b / (b @ b)
        assert np.allclose(x * x + y * y, 1.0, atol=1e-10), strut
        assert np.allclose(Q @ n, 0, atol=1e-12)


# ----------------------------------------------------- segment count reading
def test_segment_count_reading():
    """Eq. sampling N = floor(dt / (2 acos(1-CE))) + 1 with CE = 1-cos(pi/k)
    equals the oracle's count except on exact multiples of 2pi/k (where a
    full circle gets k segments, not k+1): BCC arcs of 2pi/3, 5pi/6, pi/3,
    pi, 2pi at k = 16 get 6, 7, 3, 8, 16."""
    lat = L.bcc(2, radius=0.08)
    o = oracle.Oracle(lat)
    seen = {}
    for n in range(o.N):
        nd = o.node(n)
        for dphi in nd["arc_f"][:, 1]:
            # 2 acos(1 - CE) = 2 pi / k exactly, so the paper's N is
            # floor((dphi/pi) * k / 2) + 1, evaluated in exact rationals
            frac = Fraction(round(dphi / math.pi, 6)).limit_denominator(12)
            paper = math.floor(frac * 16 / 2) + 1
            seen[round(dphi / math.pi, 6)] = paper
    n_of = {round(2 / 3, 6): 6, round(5 / 6, 6): 7, round(1 / 3, 6): 3, 1.0: 8, 2.0: 16}
    for frac, want in n_of.items():
        assert frac in seen
        paper = seen[frac]
        assert paper == (want + 1 if frac in (1.0, 2.0) else want)
    cnt = o.tri_counts(16)
    # corner strut: centre loop 18 + corner loop 16; edge: 18 + 8 + 8
    assert set(cnt[:o.E].tolist()) <= {34, 35, 36}


@pytest.mark.parametrize("excess,want", [(2.0 ** -11, 10), (2.0 ** -9, 11), (1e-9, 10)])
def test_segment_count_offset_band(excess, want):
    """The segment-count offset 2^-10 in N = ceil(dphi k / 2pi - 2^-10): an
    arc whose ratio dphi k / 2pi exceeds the integer 10 by 2^-11 gets 10
    segments (a 1e-6 offset would give 11), by 2^-9 gets 11, by 1e-9 gets
    10 under either reading.

    The arc is built from a closed form.  A node with a cylinder (strut 0,
    s_0 = 0) and a cone (strut 1, s_1 = (R - R_far)/L) whose axes meet at a
    right angle has two circle points n = a u_0 + b u_1 +- g w with
    u_0.n = 0 and u_1.n = s_1, i.e. at angles +-acos(s_1) from u_1 around
    u_0, so the elliptical arc of strut 0 spans dphi = 2 acos(s_1 / sin 90deg).
    Choosing s_1 = cos(dphi / 2) puts the ratio where the test wants it."""
    R, k = 0.1, 16
    x = 10.0 + excess
    dphi = x * 2.0 * math.pi / k
    s1 = math.cos(dphi / 2.0)
    lat = L.star([(1, 0, 0), (0, 1, 0)], radius=R, far_radii=[R, R - s1])
    o = oracle.Oracle(lat)
    nd = o.node(0)
    ell = [a for a in range(len(nd["arc_i"])) if nd["arc_i"][a, 1] >= 0]
    assert len(ell) == 1 and nd["arc_i"][ell[0], 0] == 0       # owned by strut 0's end
    a = ell[0]
    assert nd["arc_f"][a, 1] == pytest.approx(2.0 * math.acos(s1), abs=1e-12)
    assert len(o.arc_points(0, a, k)) - 1 == want
    # strut 0's band: its loop at the centre (elliptical + circular arc of
    # 2pi - dphi, ratio 16 - x) and the far end's full circle (16)
    n_circ = math.ceil(k - x - 2.0 ** -10)
    assert o.tri_counts(k)[0] == want + n_circ + k


# ------------------------------------------------------- P6: brute force
@pytest.mark.parametrize("name", ["bccjit2", "octet1", "irregular"])
def test_envelope_dense_sampling(name):
    """Dense angle sampling of every strut end: the direct arg-max of
    max(0, max_j h_j) (the kept surface of Section 4.3.1) matches each arc's
    label and span; the loops cover exactly 2 pi."""
    lat = {"bccjit2": lambda: L.bcc(2, jitter=0.05, radius_range=(0.05, 0.09)),
           "octet1": lambda: L.octet(1),
           "irregular": lambda: L.irregular(120, seed=3, r_scale=0.06)}[name]()
    o = oracle.Oracle(lat)
    row, adj, _ = o.csr()
    sizes = o.node_sizes()
    checked = 0
    for n in range(o.N):
        if sizes[n, 0] != 0:
            continue
        nd = o.node(n)
        p = 0
        for li, ln in enumerate(nd["loop_len"]):
            ents = nd["loop_ent"][p:p + ln]
            p += ln
            fr = o.end_frame(n, li)
            total = 0.0
            for e in ents:
                a = int(e & 0x7FFFFFFF)
                rev = bool(e >> 31)
                owner, other, v0, v1 = nd["arc_i"][a]
                dphi = nd["arc_f"][a, 1]
                vs, ve = (v1, v0) if rev else (v0, v1)
                z0, z1 = nd["vz"][vs], nd["vz"][ve]
                ph0 = math.atan2(z0 @ fr["e2"], z0 @ fr["e1"])
                ph1 = math.atan2(z1 @ fr["e2"], z1 @ fr["e1"])
                span = (ph1 - ph0) % (2 * math.pi)
                if span < 1e-9:
                    span = 2 * math.pi
                total += span
                phis = ph0 + span * np.linspace(0.02, 0.98, 200)
                _, lab = o.envelope(n, li, phis)
                me = adj[row[n] + li]
                lab_end = other if owner == me else owner
                want = -1 if other < 0 else int(np.nonzero(adj[row[n]:row[n + 1]] == lab_end)[0][0])
                assert np.all(lab == want), (n, li, want, np.unique(lab))
                if owner == adj[row[n] + li]:
                    assert span == pytest.approx(dphi, abs=1e-9)
            assert total == pytest.approx(2 * math.pi, abs=1e-9)
            checked += 1
    assert checked > 20


def test_point_in_union_vs_winding():
    """Monte-Carlo points away from the surface: inside the exact lattice
    solid (spheres and tangent frusta) iff the triangulated mesh winds
    around them once (region free of hole caps)."""
    lat = L.bcc(3, jitter=0.03, radius_range=(0.1, 0.16), seed=7)
    o = oracle.Oracle(lat)
    assert (o.node_sizes()[:, 0] == 0).all()
    tris, _, _ = o.triangulate(48)
    rng = np.random.default_rng(1)
    pts = rng.uniform(0.6, 2.4, size=(1500, 3))
    ins = mc.inside_union(lat, pts)
    marg = mc.union_margin(lat, pts)
    assert np.all((marg > 0) == ins)
    # keep points farther from the surface than 4 chord sagittas at k = 48
    safe = np.abs(marg) > 4 * 0.16 * (1 - math.cos(math.pi / 48))
    w = mc.winding(tris[:, 1:], pts[safe])
    assert safe.sum() > 1000 and ins[safe].sum() > 50
    assert np.all(np.abs(w - ins[safe]) < 1e-6)


def test_volume_second_order_convergence():
    """Enclosed volume converges as O(k^-2) (uniform chord subdivision,
    Section 5): successive differences shrink by 4 under doubling k."""
    lat = L.bcc(2, jitter=0.04, radius_range=(0.06, 0.1), seed=5)
    o = oracle.Oracle(lat)
    ks = [32, 64, 128, 256, 512]
    vol = [o.triangulate(k, want_tris=False)[2] for k in ks]
    dv = np.diff(vol)
    ratios = dv[:-1] / dv[1:]
    assert np.all(dv > 0)
    assert np.all((ratios > 3.5) & (ratios < 4.5))
    assert np.all(np.diff(np.abs(ratios - 4)) < 0) and abs(ratios[-1] - 4) < 0.1


@pytest.mark.parametrize("k", [8, 32])
def test_lateral_band_is_local(k):
    """Strut stitching (Section 5, 'connecting these vertices') joins points
    that are neighbours in the strut angle: no lateral triangle spans more
    than two sampling steps of the coarsest arc around the axis."""
    lat = L.bcc(3, jitter=0.04, radius_range=(0.06, 0.12), seed=11)
    o = oracle.Oracle(lat)
    tris, _, _ = o.triangulate(k, 0, o.E)
    off = np.concatenate([[0], np.cumsum(o.tri_counts(k, 0, o.E))])
    xyz, ends = lat["xyz"], lat["ends"]
    worst = 0.0
    for e in range(o.E):
        lo, hi = sorted(ends[e])
        u = xyz[hi] - xyz[lo]
        u /= np.linalg.norm(u)
        T = tris[off[e]:off[e + 1], 1:].reshape(-1, 3) - xyz[lo]
        perp = T - np.outer(T @ u, u)
        perp /= np.linalg.norm(perp, axis=1, keepdims=True)
        P = perp.reshape(-1, 3, 3)
        for a_, b_ in ((0, 1), (1, 2), (2, 0)):
            cosang = np.clip(np.einsum("ij,ij->i", P[:, a_], P[:, b_]), -1, 1)
            worst = max(worst, float(np.arccos(cosang).max()))
    assert worst < 2 * (2 * math.pi / k) + 1e-9


# ------------------------------------------- P7: adjoint reference (oracle)
def _node_R(o):
    return o.csr()[2]


def test_frozen_objective_matches_triangulation():
    """The recorded structure re-evaluated at the unperturbed parameters gives
    the triangulation's own area and volume (objective of Section 5's mesh)."""
    lat = L.bcc(3, jitter=0.05, radius_range=(0.05, 0.09), seed=5)
    o = oracle.Oracle(lat)
    for k in (8, 32):
        _, a, v = o.triangulate(k, want_tris=False)
        fz = oracle.Frozen(o, k)
        a2, v2 = fz.objective(o.xyz, _node_R(o))
        assert a2 == pytest.approx(a, rel=1e-13) and v2 == pytest.approx(v, rel=1e-13)


@pytest.mark.parametrize("k", [8, 13])
def test_frozen_gradient_straight_strut(k):
    """Isolated cylinder of radius r and length L (both ends valence 1): the
    lateral band is N rectangles and each cap an N-triangle fan to the point
    at distance r along -u, so area = 2 N r L sin(pi/N) + 2 N r^2 sin(pi/N)
    sqrt(1 + cos^2(pi/N)) and volume = (N/2) r^2 sin(2 pi/N) (L + 2r/3).
    Central differences of the frozen objective give d/dL along the axis,
    zero across it, and half of d/dr for each node radius."""
    p0, p1 = np.array([0.1, 0.2, 0.3]), np.array([1.0, 0.7, 0.5])
    r = 0.1
    lat = L.single_strut(p0, p1, r, r)
    o = oracle.Oracle(lat)
    fz = oracle.Frozen(o, k)
    N = k
    Ls = np.linalg.norm(p1 - p0)
    u = (p1 - p0) / Ls
    sn, cs = math.sin(math.pi / N), math.cos(math.pi / N)
    area = 2 * N * r * Ls * sn + 2 * N * r * r * sn * math.sqrt(1 + cs * cs)
    vol = 0.5 * N * r * r * math.sin(2 * math.pi / N) * (Ls + 2 * r / 3)
    a0, v0 = fz.objective(o.xyz, _node_R(o))
    assert a0 == pytest.approx(area, rel=1e-12) and v0 == pytest.approx(vol, rel=1e-12)
    dA_dL = 2 * N * r * sn
    dA_dr = 2 * N * Ls * sn + 4 * N * r * sn * math.sqrt(1 + cs * cs)
    dV_dL = 0.5 * N * r * r * math.sin(2 * math.pi / N)
    dV_dr = N * r * math.sin(2 * math.pi / N) * (Ls + 2 * r / 3) + N * r * r * math.sin(2 * math.pi / N) / 3
    ga, gv = fz.fd(1e-5, [0, 1])
    for q, sgn in ((0, -1.0), (1, 1.0)):
        assert np.allclose(ga[q, :3], sgn * dA_dL * u, rtol=1e-7, atol=1e-8)
        assert np.allclose(gv[q, :3], sgn * dV_dL * u, rtol=1e-7, atol=1e-8)
        assert ga[q, 3] == pytest.approx(dA_dr / 2, rel=1e-7)
        assert gv[q, 3] == pytest.approx(dV_dr / 2, rel=1e-7)


@pytest.mark.parametrize("name", ["tilted150", "asym"])
def test_frozen_band_objective_and_gradient(name):
    """The frozen structure replays an annular band (reading 10) too: it
    reproduces the triangulation's area and volume, and its central
    differences agree at h and h/2 to O(h^2)."""
    lat, _ = _annular_stars()[name]
    o = oracle.Oracle(lat)
    for k in (8, 24):
        _, a, v = o.triangulate(k, want_tris=False)
        fz = oracle.Frozen(o, k)
        a2, v2 = fz.objective(o.xyz, _node_R(o))
        assert a2 == pytest.approx(a, rel=1e-13) and v2 == pytest.approx(v, rel=1e-13)
        ga1, gv1 = fz.fd(1e-4, np.arange(o.N))
        ga2, gv2 = fz.fd(5e-5, np.arange(o.N))
        assert np.abs(ga1 - ga2).max() < 1e-6 * np.abs(ga1).max()
        assert np.abs(gv1 - gv2).max() < 1e-6 * np.abs(gv1).max()


def test_frozen_gradient_smooth_and_local():
    """With the structure frozen the objective is smooth: central differences
    at h and h/2 agree to O(h^2) (Richardson), and the locally re-evaluated
    difference equals the difference of whole-lattice evaluations."""
    lat = L.bcc(2, jitter=0.05, radius_range=(0.05, 0.09), seed=11)
    o = oracle.Oracle(lat)
    fz = oracle.Frozen(o, 16)
    nodes = np.arange(o.N)
    ga1, gv1 = fz.fd(1e-4, nodes)
    ga2, gv2 = fz.fd(5e-5, nodes)
    sa, sv = np.abs(ga1).max(), np.abs(gv1).max()
    assert np.abs(ga1 - ga2).max() < 1e-6 * sa and np.abs(gv1 - gv2).max() < 1e-6 * sv
    # whole-lattice central difference for a few parameters
    R = _node_R(o)
    for v, p in ((3, 0), (9, 2), (13, 3)):
        xp, xm = o.xyz.copy(), o.xyz.copy()
        Rp, Rm = R.copy(), R.copy()
        if p < 3:
            xp[v, p] += 1e-4
            xm[v, p] -= 1e-4
        else:
            Rp[v] += 1e-4
            Rm[v] -= 1e-4
        ap, vp = fz.objective(xp, Rp)
        am, vm = fz.objective(xm, Rm)
        # whole sums of ~1 differenced at 1e-4: rounding near 1e-11
        assert (ap - am) / 2e-4 == pytest.approx(ga1[v, p], rel=1e-7, abs=1e-9)
        assert (vp - vm) / 2e-4 == pytest.approx(gv1[v, p], rel=1e-7, abs=1e-9)


# ------------------------------------------------- the library's arctangent
def test_atan_coefficients_reproduce_from_the_fit():
    """The coefficients of lm_atan2 (csrc/lm_geom.cuh) are the FP32-rounded
    output of the committed minimax fit, whose FP32 evaluation stays within
    1.23e-7 rad of atan on [0, 1]."""
    import os
    import re
    from paper_2405_15197_gb300 import fit_atan
    src = open(os.path.join(os.path.dirname(fit_atan.__file__), "csrc", "lm_geom.cuh")).read()
    body = src[src.index("__device__ __forceinline__ float lm_atan2(float y, float x)"):]
    body = body[body.index("float p ="):body.index("float a = r * p;")]
    got = [float(x) for x in re.findall(r"(-?\d+\.\d+(?:e-?\d+)?)f", body)]
    want = fit_atan.coefficients_f32()
    assert np.array_equal(np.array(got[::-1], dtype=np.float32), want)
    assert fit_atan.max_error_f32(want, n=200_001) <= 1.23e-7
