"""CUDA paths that the standard parity lattices do not reach, through the
C ABI and against the FP64 oracle where there is a result to compare:

* the thread-per-strut stitching kernel, taken at resolutions whose loops
  no longer fit the tile kernel's shared memory (k = 4096);
* the meta-mesh launch of the d <= 64 valence bucket (a node of valence 40);
* the deferred-strut list overflowing into the deferral-bitmap scan;
* an allocation failure (a host-side device-memory budget, no GPU fault);
* the library's FP32 arctangent and sine / cosine against FP64 references;
* builds with the pool's freed memory retained (lm_pool_retain).
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


def _build(lat, dtype, options=None):
    lat = P.lattice_as(lat, dtype)
    xyz, ends, radii = P.to_device(lat, dtype)
    return lat, liblm.MetaMesh(xyz, ends, radii, options=options)


def _all_records(lat, mm, o, k, dtype):
    n = mm.tri_count(k)
    assert n == int(o.tri_counts(k).sum())
    rec = mm.triangulate(k).cpu().numpy()
    assert liblm.lm_last_error(mm.h) == 0
    gn, gv = P.parse_stl(rec)
    ot, oa, ov = o.triangulate(k)
    errs, dv, dn = P.compare_triangles(gn, gv, ot, float(lat["radii"].max()),
                                       tol=2e-5 if dtype == np.float32 else 1e-7)
    assert not errs, errs
    return rec


def test_thread_stitching_at_fine_resolution():
    """k = 4096: a loop holds about 4,100 points, more than two stitching
    tiles fit in shared memory, so the struts go through the thread-per-strut
    kernel (sequential zipper, points computed once per loop iterator)."""
    for dtype in (np.float32, np.float64):
        lat, mm = _build(L.bcc(2, radius=0.1), dtype)
        o = oracle.Oracle(lat)
        _all_records(lat, mm, o, 4096, dtype)
        mm.close()


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_valence_40_node(dtype):
    """A node of valence 40 (the d <= 64 bucket of the meta-mesh launch):
    meta-mesh and triangles against the oracle."""
    d = np.random.default_rng(4).normal(size=(40, 3))
    lat, mm = _build(L.star(d, radius=0.04, length=1.0), dtype)
    assert mm.counts()[6] == 40
    o = oracle.Oracle(lat)
    g = mm.download()
    tol = 2e-5 if dtype == np.float32 else 1e-12
    rep = P.compare_metamesh(g, o, z_tol=tol, phi_tol=tol, degenerate_tol=1e-9 if dtype == np.float64 else None)
    assert rep.ok(), rep.errors[:4]
    assert rep.exempt_nodes == 0
    _all_records(lat, mm, o, 8, dtype)
    mm.close()


def test_deferred_list_overflow_scans_the_bitmap():
    """With room for one listed deferred strut, the FP64 stitching pass scans
    the deferral bitmap instead of the list: the same records, byte for byte."""
    lat = L.irregular(1500, seed=9, r_scale=0.3)
    k = 16
    _, ref = _build(lat, np.float32)
    ref.tri_count(k)
    a = ref.triangulate(k).cpu().numpy()
    opt = liblm.lm_options()
    opt.redo_list_cap = 1
    _, small = _build(lat, np.float32, opt)
    small.tri_count(k)
    b = small.triangulate(k).cpu().numpy()
    assert liblm.lm_last_error(small.h) == 0
    deferred = sum(liblm.lm_fp64_counts(small.h)[i] for i in (12, 13, 14, 16, 17))
    assert deferred > 1
    assert np.array_equal(a, b)


def test_allocation_failure_is_reported():
    """A device-memory budget smaller than the build needs makes an
    allocation fail as on a full device: LM_ERR_OOM, nothing leaked (the
    next build in the same process succeeds)."""
    lat = L.octet(3)
    opt = liblm.lm_options()
    opt.mem_budget = 4096
    with pytest.raises(liblm.LmError) as ei:
        _build(lat, np.float32, opt)
    assert ei.value.status == 5
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        with pytest.raises(liblm.LmError):
            _build(lat, np.float32, opt)
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) < (64 << 20)
    _, mm = _build(lat, np.float32)
    assert mm.counts()[0] > 0
    mm.close()


def test_angle_functions_error_bounds():
    """lm_atan2 (degree-7 minimax polynomial in r^2, fit in fit_atan.py):
    within 2.5e-7 rad of atan2 when |y| <= x (the polynomial's 1.23e-7, the
    rounding of r = y / x and of r P), within 5e-7 rad everywhere (the
    octant identities add the FP32 constants pi/2, pi and a rounding each).
    lm_sincos: within 7e-7 of sin / cos over four turns."""
    rng = np.random.default_rng(11)
    n = 1 << 20
    th = np.linspace(-math.pi, math.pi, n)
    rad = np.exp(rng.uniform(-8, 8, n))
    y = (rad * np.sin(th)).astype(np.float32)
    x = (rad * np.cos(th)).astype(np.float32)
    a = np.linspace(-4 * math.pi, 4 * math.pi, n).astype(np.float32)
    at, sn, cs = liblm.lm_eval_angle_fns(torch.tensor(y, device="cuda"), torch.tensor(x, device="cuda"),
                                         torch.tensor(a, device="cuda"))
    at, sn, cs = at.cpu().numpy(), sn.cpu().numpy(), cs.cpu().numpy()
    ref = np.arctan2(y.astype(np.float64), x.astype(np.float64))
    err = np.abs(at.astype(np.float64) - ref)
    err = np.minimum(err, 2 * math.pi - err)  # +-pi
    first = (np.abs(y) <= x)
    assert err[first].max() <= 2.5e-7, err[first].max()
    assert err.max() <= 5e-7, err.max()
    a64 = a.astype(np.float64)
    assert np.abs(sn - np.sin(a64)).max() <= 7e-7
    assert np.abs(cs - np.cos(a64)).max() <= 7e-7


def test_pool_retain_and_build_times():
    """lm_pool_retain keeps freed device memory mapped in the default pool
    between builds (the arena's room counts it): builds after it are the same
    array for array; lm_metamesh_build_times reports five non-negative
    phases; the default is restored afterwards."""
    from tests.test_gpu_parity import LATTICES
    lat = P.lattice_as(LATTICES["irregular"](), np.float32)
    xyz, ends, radii = P.to_device(lat, np.float32)
    ref = liblm.MetaMesh(xyz, ends, radii)
    a = ref.download()
    ref.close()
    liblm.lm_pool_retain((1 << 64) - 1)
    try:
        for _ in range(2):
            mm = liblm.MetaMesh(xyz, ends, radii)
            b = mm.download()
            for key in a:
                assert np.array_equal(a[key], b[key]), key
            t = liblm.lm_metamesh_build_times(mm.h)
            assert len(t) == 5 and all(x >= 0 for x in t)
            mm.close()
    finally:
        liblm.lm_pool_retain(0)
