"""Binary-STL file output through the three-stage pipeline (GPU
triangulation, device-to-host copy into a pinned ring, file writes by a host
thread; Section 4.2.2 of arXiv 2405.15197) against the direct device output
of the same meta-mesh, through the C ABI."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2405_15197_gb300 import liblm  # noqa: E402
from tests.test_gpu_parity import build  # noqa: E402


def _check_file(path, n, full):
    data = np.fromfile(path, dtype=np.uint8)
    assert data.size == 84 + 50 * n
    assert bytes(data[:84]) == liblm.lm_stl_header(n)
    assert int.from_bytes(bytes(data[80:84]), "little") == n
    assert np.array_equal(data[84:].reshape(-1, 50), full)


@pytest.mark.parametrize("name,dtype,k,chunk", [("bcc10", np.float64, 16, 97), ("octet3", np.float32, 32, 61),
                                                ("irregular", np.float32, 16, 1000)])
def test_stl_file_matches_direct(tmp_path, name, dtype, k, chunk):
    """Fixed chunks, a three-slot ring (every slot reused): the file is the
    header and every record of lm_triangulate in order."""
    _, mm, _, _ = build(name, dtype)
    n = mm.tri_count(k)
    full = mm.triangulate(k).cpu().numpy()
    n_items = mm.n_struts + mm.n_nodes
    max_chunk = max(liblm.lm_tri_range(mm.h, c, min(n_items, c + chunk))[1] for c in range(0, n_items, chunk))
    slot = 50 * max_chunk
    ring = torch.empty(3 * slot, dtype=torch.uint8, pin_memory=True)
    path = tmp_path / f"{name}_k{k}.stl"
    got, st = liblm.lm_triangulate_to_file(mm.h, k, str(path), ring.data_ptr(), slot, 3, chunk_items=chunk)
    assert got == n
    assert st["total_s"] > 0 and st["write_s"] >= 0 and st["wait_s"] >= 0 and st["fsync_s"] == 0
    _check_file(path, n, full)


def test_stl_file_chunk_size_rule_and_sync(tmp_path):
    """Chunks sized by Eq. chunk-size from the slot (chunk_items = 0), file
    synced before the call returns; a second call truncates and rewrites."""
    _, mm, _, _ = build("bcc10", np.float32)
    k = 8
    n = mm.tri_count(k)
    full = mm.triangulate(k).cpu().numpy()
    slot = 50 * (n // 5)
    ring = torch.empty(2 * slot, dtype=torch.uint8, pin_memory=True)
    path = tmp_path / "bcc10.stl"
    path.write_bytes(b"x" * (100 + 84 + 50 * n))  # longer than the result: truncated
    for _ in range(2):
        got, st = liblm.lm_triangulate_to_file(mm.h, k, str(path), ring.data_ptr(), slot, 2, sync=True)
        assert got == n and st["fsync_s"] >= 0
        _check_file(path, n, full)


def test_stl_file_errors(tmp_path):
    """A path that cannot be created returns LM_ERR_IO; a slot smaller than
    one chunk's records returns LM_ERR_CAPACITY; both leave the handle usable."""
    _, mm, _, _ = build("octet3", np.float32)
    k = 8
    n = mm.tri_count(k)
    ring = torch.empty(2 * 50 * n, dtype=torch.uint8, pin_memory=True)
    with pytest.raises(liblm.LmError, match="LM_ERR_IO"):
        liblm.lm_triangulate_to_file(mm.h, k, str(tmp_path / "no_dir" / "x.stl"), ring.data_ptr(), 50 * n, 2)
    with pytest.raises(liblm.LmError, match="LM_ERR_CAPACITY"):
        liblm.lm_triangulate_to_file(mm.h, k, str(tmp_path / "small.stl"), ring.data_ptr(), 500, 2,
                                     chunk_items=mm.n_struts + mm.n_nodes)
    got, _ = liblm.lm_triangulate_to_file(mm.h, k, str(tmp_path / "ok.stl"), ring.data_ptr(), 50 * n, 2)
    assert got == n
    _check_file(tmp_path / "ok.stl", n, mm.triangulate(k).cpu().numpy())
