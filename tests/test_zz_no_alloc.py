"""The allocation-free triangulation entry point (lm_triangulate_noalloc).

It serves callers that cannot let the library allocate device memory when
they triangulate: an application whose GPU memory belongs to a framework's
caching allocator or to a pool sized up front, where a library cudaMalloc
could fail or force the pool to give memory back, or a latency-bound loop
in which cudaMalloc / cudaFree would stall the device.  Its scratch is a
fixed device array inside the library.  Its records must be byte-identical
to the allocating entry point's (lm_tri_count + lm_triangulate) for the same
items, on two calls in a row (the shared array keeps the previous call's
contents), in FP32 and FP64, and ranges beyond its capacity must be
refused.  This file is collected last so a failure here leaves every other
test already run.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2405_15197_gb300 import lattices as L  # noqa: E402
from paper_2405_15197_gb300 import liblm  # noqa: E402
from tests import parity as P  # noqa: E402


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_noalloc_matches_allocating_path(dtype):
    lat = P.lattice_as(L.octet(3), dtype)
    xyz, ends, radii = P.to_device(lat, dtype)
    mm = liblm.MetaMesh(xyz, ends, radii)
    n_items = mm.n_struts + mm.n_nodes
    for k, (b, e) in [(8, (0, n_items)), (32, (17, n_items - 5)), (16, (mm.n_struts - 3, n_items))]:
        mm.tri_count(k)
        first, cnt = liblm.lm_tri_range(mm.h, b, e)
        ref = torch.empty((max(cnt, 1), 50), dtype=torch.uint8, device="cuda")
        liblm.lm_triangulate(mm.h, k, b, e, ref.data_ptr(), cnt)
        assert liblm.lm_last_error(mm.h) == 0
        ref = ref[:cnt].cpu().numpy()
        for call in range(2):
            out = torch.full((cnt + 1, 50), 0xAB, dtype=torch.uint8, device="cuda")
            n = liblm.lm_triangulate_noalloc(mm.h, k, b, e, out.data_ptr(), cnt)
            assert liblm.lm_last_error(mm.h) == 0
            assert n == cnt
            got = out.cpu().numpy()
            assert np.all(got[cnt] == 0xAB)  # nothing written past the range
            # the same kernels on the same meta-mesh: the same bytes
            assert np.array_equal(got[:cnt], ref)
    mm.close()


def test_noalloc_rejects_oversized_range():
    lat = P.lattice_as(L.octet(24), np.float32)
    xyz, ends, radii = P.to_device(lat, np.float32)
    mm = liblm.MetaMesh(xyz, ends, radii)
    n_items = mm.n_struts + mm.n_nodes
    assert n_items > (1 << 18)
    out = torch.empty((8, 50), dtype=torch.uint8, device="cuda")
    with pytest.raises(liblm.LmError) as ei:
        liblm.lm_triangulate_noalloc(mm.h, 8, 0, (1 << 18) + 1, out.data_ptr(), 8)
    assert ei.value.status == 4
    # the largest accepted range works
    n = liblm.lm_triangulate_noalloc(mm.h, 8, 0, 1 << 18, 0, 0)
    assert n > 0
    mm.close()
