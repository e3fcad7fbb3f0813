"""Chunked meta-meshing with overlapped streaming (lm_stream_chunked): the
lattice built chunk by chunk (each chunk's struts with the halo of struts
incident to their end nodes), the next chunk's build beside the current
chunk's streaming (Section 4.2.2's pipeline at the meta-mesh level).  The
records of every k are the records of a whole-lattice build, as a set (and
in order when one chunk holds the whole lattice)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2405_15197_gb300 import liblm  # noqa: E402
from tests import parity as P  # noqa: E402
from tests.test_gpu_parity import LATTICES  # noqa: E402


def _chunked(xyz, ends, radii, ks, build_struts, slot=1 << 22, n_slots=3):
    ring = torch.empty(n_slots * slot, dtype=torch.uint8, pin_memory=True)
    got = {k: [] for k in ks}

    def cb(seq, k, first, ntri, ptr, user):
        off = ptr - ring.data_ptr()
        got[k].append((seq, ring[off:off + 50 * ntri].numpy().copy()))

    tris = liblm.lm_stream_chunked(xyz, ends, radii, ks, build_struts, ring.data_ptr(), slot, n_slots, cb)
    out = {}
    for q, k in enumerate(ks):
        parts = [a for _, a in sorted(got[k], key=lambda x: x[0])]
        rec = np.concatenate(parts).reshape(-1, 50) if parts else np.zeros((0, 50), np.uint8)
        assert rec.shape[0] == tris[q]
        out[k] = rec
    return out


def _sorted_rows(a):
    return np.sort(np.ascontiguousarray(a).view(np.dtype((np.void, 50))).ravel())


@pytest.mark.parametrize("name,dtype,parts", [("bcc10", np.float32, 5), ("octet3", np.float32, 3),
                                              ("irregular", np.float32, 4), ("irr03", np.float64, 3),
                                              ("bccjit4", np.float32, 6), ("annular150", np.float32, 2),
                                              ("star5", np.float32, 2)])
def test_chunked_records_equal_whole_build(name, dtype, parts):
    lat = P.lattice_as(LATTICES[name](), dtype)
    xyz, ends, radii = P.to_device(lat, dtype)
    E = ends.shape[0]
    ks = (8, 16)
    mm = liblm.MetaMesh(xyz, ends, radii)
    full = {}
    for k in ks:
        mm.tri_count(k)
        full[k] = mm.triangulate(k).cpu().numpy()
    mm.close()
    # uneven chunks, and one chunk holding the whole lattice
    got = _chunked(xyz, ends, radii, ks, E // parts + 7)
    for k in ks:
        assert got[k].shape == full[k].shape
        assert np.array_equal(_sorted_rows(got[k]), _sorted_rows(full[k]))
    one = _chunked(xyz, ends, radii, ks, E)
    for k in ks:
        assert np.array_equal(one[k], full[k])


def test_chunked_rejects_invalid_ends():
    lat = P.lattice_as(LATTICES["octet3"](), np.float32)
    xyz, ends, radii = P.to_device(lat, np.float32)
    bad = ends.clone()
    bad[3, 1] = xyz.shape[0] + 5
    ring = torch.empty(2 << 20, dtype=torch.uint8, pin_memory=True)
    with pytest.raises(liblm.LmError, match="LM_ERR_INVALID_ARG"):
        liblm.lm_stream_chunked(xyz, bad, radii, (8,), 50, ring.data_ptr(), 1 << 20, 2)
