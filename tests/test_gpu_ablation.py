"""Warp-centric vs thread-centric trimming (Section 6 of arXiv 2405.15197,
Fig. thread-vs-warp): the envelope t*(phi) = max(0, max_j h_j(phi)) of
Section 4.3.1 and its arg-max at sample angles of every strut end, in both
work mappings, against the FP64 oracle's direct evaluation and against each
other, through the C ABI."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2405_15197_gb300 import liblm  # noqa: E402
from tests.test_gpu_parity import build  # noqa: E402

S = 24


def _run(mm, dtype, mode):
    n_ends = 2 * mm.n_struts
    t = torch.empty(n_ends * S, dtype=torch.float32 if dtype == np.float32 else torch.float64, device="cuda")
    lab = torch.empty(n_ends * S, dtype=torch.int16, device="cuda")
    liblm.lm_envelope_samples(mm.h, S, mode, t.data_ptr(), lab.data_ptr())
    assert liblm.lm_last_error(mm.h) == 0
    return t.cpu().numpy().astype(np.float64).reshape(n_ends, S), lab.cpu().numpy().reshape(n_ends, S)


@pytest.mark.parametrize("name,dtype", [("octet3", np.float32), ("bccjit4", np.float32), ("star5", np.float32),
                                        ("octet3", np.float64), ("irregular", np.float64), ("irr03", np.float64)])
def test_envelope_both_mappings_match_oracle(name, dtype):
    lat, mm, g, o = build(name, dtype)
    row, adj, node_R = o.csr()
    ends = np.asarray(lat["ends"]).reshape(-1)
    tw, lw = _run(mm, dtype, liblm.LM_ENV_WARP)
    tt, lt = _run(mm, dtype, liblm.LM_ENV_THREAD)
    # the two mappings: same arithmetic, so the same results up to how the
    # compiler contracted each copy (amplified by steep sections on the
    # irregular lattices' degenerate nodes)
    rtol = 1e-6 if dtype == np.float32 else 1e-9
    assert np.allclose(tw, tt, rtol=rtol, atol=rtol * float(node_R.max()))
    assert (lw == lt).mean() > 0.9999
    # against the oracle (FP64, direct evaluation), every strut end; the
    # ablation evaluates h_j in plain arithmetic (none of the meta-mesh
    # kernel's conditioning for nearly parallel struts), whose FP32 error
    # reaches about 6e-5 (R + |t|) on the irregular lattice
    # (steep sections, with a denominator near zero, lose more: a few
    # samples in a thousand, bounded by 1e-2 (R + |t|))
    phi = 2 * math.pi * np.arange(S) / S
    tol = (2e-4 if dtype == np.float32 else 1e-9)
    agree = total = over = 0
    for e in range(2 * mm.n_struts):
        n = int(ends[e])
        li = int(np.nonzero(adj[row[n]:row[n + 1]] == e)[0][0])
        ot, ol = o.envelope(n, li, phi)
        rel = np.abs(tw[e] - ot) / (float(node_R[n]) + np.abs(ot))
        if dtype == np.float64:
            assert np.all(rel <= tol), (e, rel.max())
        over += int((rel > tol).sum())
        agree += int((lw[e] == ol).sum())
        total += S
    assert over <= 1e-3 * total
    assert agree >= 0.999 * total


def test_envelope_mappings_agree_on_degenerate_nodes():
    """The irregular lattice (many nodes outside the lattice model: steep
    sections whose t runs off to infinity, where plain FP32 is meaningless
    against FP64) in FP32: the two mappings give the same values."""
    lat, mm, g, o = build("irregular", np.float32)
    tw, lw = _run(mm, np.float32, liblm.LM_ENV_WARP)
    tt, lt = _run(mm, np.float32, liblm.LM_ENV_THREAD)
    fin = np.isfinite(tw) & np.isfinite(tt)
    assert fin.mean() > 0.999
    assert np.allclose(tw[fin], tt[fin], rtol=1e-5, atol=1e-7)
    assert (lw == lt).mean() > 0.999
