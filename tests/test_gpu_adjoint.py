"""Adjoint (lm_metamesh_backward) against central finite differences of the
FP64 oracle with the discrete structure frozen, on a jittered BCC 4^3
lattice (189 nodes, 512 struts, 756 parameters) at k = 32."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_2405_15197_gb300 import lattices as L  # noqa: E402
from paper_2405_15197_gb300 import liblm  # noqa: E402
from paper_2405_15197_gb300.adjoint import lattice_objective  # noqa: E402
from tests import parity as P  # noqa: E402

K = 32
_cache = {}


def setup(dtype):
    """Central differences of the frozen-structure FP64 objective, h = 1e-4,
    Richardson-extrapolated with h / 2 ((4 D(h/2) - D(h)) / 3: truncation
    error O(h^4) instead of O(h^2))."""
    if dtype not in _cache:
        lat = P.lattice_as(L.bcc(4, jitter=0.05, radius_range=(0.05, 0.09)), dtype)
        o = oracle.Oracle(lat)
        fz = oracle.Frozen(o, K)
        ga1, gv1 = fz.fd(1e-4, np.arange(o.N))
        ga2, gv2 = fz.fd(5e-5, np.arange(o.N))
        ga, gv = (4.0 * ga2 - ga1) / 3.0, (4.0 * gv2 - gv1) / 3.0
        _cache[dtype] = (lat, o, ga, gv)
    return _cache[dtype]


def rel_err(g, ref):
    return np.abs(g - ref).max() / np.abs(ref).max()


def elementwise_err(g, ref, floor_frac=1e-3):
    """max |g - ref| / max(|ref|, floor_frac max|ref|): relative error of every
    entry above the floor, absolute below it."""
    floor = floor_frac * np.abs(ref).max()
    return (np.abs(g - ref) / np.maximum(np.abs(ref), floor)).max()


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_adjoint_vs_frozen_fd(dtype):
    lat, o, ga, gv = setup(dtype)
    xyz, ends, radii = P.to_device(lat, dtype)
    mm = liblm.MetaMesh(xyz, ends, radii)
    _, oa, ov = o.triangulate(K, want_tris=False)
    for w, ref in (((1.0, 0.0), ga), ((0.0, 1.0), gv)):
        gx, gr, a, v = mm.backward(K, *w)
        assert a == pytest.approx(oa, rel=1e-5) and v == pytest.approx(ov, rel=1e-5)
        g = np.concatenate([gx.cpu().numpy(), gr.cpu().numpy()[:, None]], 1).astype(np.float64)
        e = rel_err(g, ref)
        ee = elementwise_err(g, ref)
        print(f"w={w}: max |adjoint - FD| / max |FD| = {e:.2e}, element-wise {ee:.2e}")
        if dtype == np.float64:
            assert ee < 1e-6
        else:
            assert e < 1e-3


@pytest.mark.parametrize("name,dtype", [("annular150", np.float64), ("annular_asym", np.float64),
                                        ("annular150", np.float32)])
def test_adjoint_annular_band(name, dtype):
    """A node whose two contours are stitched as a band (reading 10): the
    adjoint of its triangles against the frozen-structure FD of the oracle."""
    from tests.test_gpu_parity import LATTICES
    lat = P.lattice_as(LATTICES[name](), dtype)
    o = oracle.Oracle(lat)
    fz = oracle.Frozen(o, 24)
    ga1, gv1 = fz.fd(1e-4, np.arange(o.N))
    ga2, gv2 = fz.fd(5e-5, np.arange(o.N))
    ga, gv = (4.0 * ga2 - ga1) / 3.0, (4.0 * gv2 - gv1) / 3.0
    xyz, ends, radii = P.to_device(lat, dtype)
    mm = liblm.MetaMesh(xyz, ends, radii)
    _, oa, ov = o.triangulate(24, want_tris=False)
    for w, ref in (((1.0, 0.0), ga), ((0.0, 1.0), gv)):
        gx, gr, a, v = mm.backward(24, *w)
        assert a == pytest.approx(oa, rel=1e-5) and v == pytest.approx(ov, rel=1e-5)
        g = np.concatenate([gx.cpu().numpy(), gr.cpu().numpy()[:, None]], 1).astype(np.float64)
        if dtype == np.float64:
            assert elementwise_err(g, ref) < 1e-6
        else:
            assert rel_err(g, ref) < 1e-3
    mm.close()


def test_adjoint_accumulates_and_autograd():
    lat, o, ga, gv = setup(np.float32)
    xyz, ends, radii = P.to_device(lat, np.float32)
    node_R = torch.tensor(o.csr()[2], dtype=torch.float32, device="cuda")
    x = xyz.clone().requires_grad_(True)
    r = node_R.clone().requires_grad_(True)
    J = lattice_objective(x, r, ends, K, 0.5, 2.0)
    _, oa, ov = o.triangulate(K, want_tris=False)
    assert J.item() == pytest.approx(0.5 * oa + 2.0 * ov, rel=1e-5)
    gx, gr = torch.autograd.grad(J * 3.0, (x, r))
    ref = 3.0 * (0.5 * ga + 2.0 * gv)
    g = np.concatenate([gx.cpu().numpy(), gr.cpu().numpy()[:, None]], 1).astype(np.float64)
    assert rel_err(g, ref) < 1e-3
    # gradients are added into the caller's buffers
    mm = liblm.MetaMesh(xyz, ends, radii)
    g1 = torch.ones((o.N, 3), device="cuda")
    g2 = torch.ones((o.N,), device="cuda")
    liblm.lm_metamesh_backward(mm.h, K, 1.0, 0.0, g1.data_ptr(), g2.data_ptr())
    assert np.allclose(g1.cpu().numpy() - 1.0, ga[:, :3], rtol=0, atol=1e-3 * np.abs(ga).max())
