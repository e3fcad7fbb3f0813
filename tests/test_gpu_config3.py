"""The irregular configuration at full size, GPU vs oracle on a slice.

2e6 uniform nodes in the unit cube, kNN k_v ~ U{4..16} symmetrised,
lognormal radii with median 0.3 x mean strut length (the configured radius
law), FP32.  The GPU meta-meshes the whole lattice with the launch the
benchmark uses; the oracle meta-meshes the ~1e5 nodes of the sub-cube
[0, 0.368)^3, which are compared node by node (flags on every node, data on
every node but the near-tangent ones), and the triangles of a seeded sample
of 20,000 struts and 5,000 nodes inside the sub-cube are compared record by
record at k = 16.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_2405_15197_gb300 import lattices as L  # noqa: E402
from paper_2405_15197_gb300 import liblm  # noqa: E402
from tests import parity as P  # noqa: E402


def test_irregular_2e6_slice_parity():
    lat = P.lattice_as(L.irregular(2_000_000, r_scale=0.3), np.float32)
    xyz, ends, radii = P.to_device(lat, np.float32)
    opt = liblm.lm_options()
    opt.autotune = 1
    mm = liblm.MetaMesh(xyz, ends, radii, options=opt)
    g = mm.download()
    sub = np.nonzero(np.all(lat["xyz"] < 0.368, axis=1))[0]
    assert sub.size >= 90_000
    o = oracle.Oracle(lat, nodes=sub)
    rep = P.compare_metamesh(g, o, nodes=sub)
    assert rep.ok(), "\n".join(rep.errors[:8])
    assert rep.exempt_nodes <= 0.01 * sub.size
    deg = np.mean((g["node_flags"][sub] & P.DEGENERATE) != 0)
    print(f"sub-cube {sub.size} nodes: {rep.exempt_nodes} near-tangent, degenerate fraction {deg:.3f}, "
          f"max vertex error {rep.max_dz:.3g} R")
    # triangles of a sample of items inside the sub-cube
    k = 16
    total = mm.tri_count(k)
    of = o.node_sizes()[:, 0]
    insub = np.zeros(o.N, bool)
    insub[sub] = True
    nt = (of & P.NEAR_TANGENT) != 0
    e_ = lat["ends"]
    struts = np.nonzero(insub[e_[:, 0]] & insub[e_[:, 1]] & ~nt[e_[:, 0]] & ~nt[e_[:, 1]])[0]
    nodes = sub[~nt[sub]]
    rng = np.random.default_rng(1)
    items = np.sort(np.concatenate([rng.choice(struts, 20000, replace=False),
                                    o.E + rng.choice(nodes, 5000, replace=False)]))
    rec = torch.empty((total, 50), dtype=torch.uint8, device="cuda")
    liblm.lm_triangulate(mm.h, k, 0, o.E + o.N, rec.data_ptr(), total)
    assert liblm.lm_last_error(mm.h) == 0
    R = float(lat["radii"].max())
    bad = []
    for it in items:
        f0, c = liblm.lm_tri_range(mm.h, int(it), int(it) + 1)
        ot, _, _ = o.triangulate(k, int(it), int(it) + 1)
        assert c == ot.shape[0], (it, c, ot.shape[0])
        gn, gv = P.parse_stl(rec[f0:f0 + c].cpu().numpy())
        errs, dv, dn = P.compare_triangles(gn, gv, ot, R)
        if errs:
            bad.append((int(it), errs))
    assert not bad, bad[:5]
    mm.close()
