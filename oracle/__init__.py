"""FP64 CPU oracle (test infrastructure only).

Plain, slow, single-threaded C++ implementation of what the lattice
meta-meshing and triangulation path computes (arXiv 2405.15197, Sections 4.1,
4.3.1 and 5, Algorithm 1), compiled from ``lm_oracle.cpp`` with g++.  Only
the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg
use it; the CUDA library never imports or links it, and it shares no code
with the CUDA library.

Pins: see tests/test_oracle_*.py (closed forms, invariants, brute force).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lm_oracle.cpp")
_LIB = os.path.join(_HERE, "_lm_oracle.so")
_lib = None

c_i64p = ctypes.POINTER(ctypes.c_int64)
c_i32p = ctypes.POINTER(ctypes.c_int32)
c_u32p = ctypes.POINTER(ctypes.c_uint32)
c_u64p = ctypes.POINTER(ctypes.c_uint64)
c_dp = ctypes.POINTER(ctypes.c_double)

NF_NEAR_TANGENT, NF_DEGENERATE, NF_INCONSISTENT = 1, 2, 4
VF_SPHERE, VF_SEAM = 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle shared library (plain g++, no GPU code)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.lmo_build.restype = ctypes.c_void_p
        lib.lmo_build.argtypes = [ctypes.c_int64, ctypes.c_int64, c_dp, c_i32p, c_dp,
                                  ctypes.POINTER(ctypes.c_int)]
        lib.lmo_metamesh.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64]
        lib.lmo_free.argtypes = [ctypes.c_void_p]
        lib.lmo_node_sizes.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, c_i64p]
        lib.lmo_node_export.argtypes = [ctypes.c_void_p, ctypes.c_int64, c_dp, c_u64p, c_u32p,
                                        c_u32p, c_i32p, c_dp, c_i32p, c_u32p, c_i32p, c_u32p]
        lib.lmo_tri_counts.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64,
                                       ctypes.c_int64, c_i64p]
        lib.lmo_triangulate.restype = ctypes.c_int64
        lib.lmo_triangulate.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64,
                                        ctypes.c_int64, c_dp, c_dp]
        lib.lmo_csr.argtypes = [ctypes.c_void_p, c_i64p, c_i32p, c_dp]
        lib.lmo_end_frame.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, c_dp]
        lib.lmo_arc_points.restype = ctypes.c_int
        lib.lmo_arc_points.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int,
                                       ctypes.c_int, c_dp]
        lib.lmo_envelope.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int,
                                     ctypes.c_int64, c_dp, c_dp, c_i32p]
        lib.lmo_frozen_record.restype = ctypes.c_void_p
        lib.lmo_frozen_record.argtypes = [ctypes.c_void_p, ctypes.c_int]
        lib.lmo_frozen_free.argtypes = [ctypes.c_void_p]
        lib.lmo_frozen_objective.argtypes = [ctypes.c_void_p, ctypes.c_void_p, c_dp, c_dp, c_dp]
        lib.lmo_frozen_fd.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, c_i64p,
                                      ctypes.c_int64, c_dp]
        _lib = lib
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


class OracleError(RuntimeError):
    pass


class Oracle:
    """Meta-mesh of a whole lattice, node by node (Section 4.3.1)."""

    def __init__(self, lat, nodes=None):
        lib = _load()
        self.xyz = np.ascontiguousarray(lat["xyz"], dtype=np.float64)
        self.ends = np.ascontiguousarray(lat["ends"], dtype=np.int32)
        self.radii = np.ascontiguousarray(lat["radii"], dtype=np.float64)
        self.N, self.E = self.xyz.shape[0], self.ends.shape[0]
        st = ctypes.c_int(0)
        self.h = lib.lmo_build(self.N, self.E, _p(self.xyz, c_dp), _p(self.ends, c_i32p),
                               _p(self.radii, c_dp), ctypes.byref(st))
        self.status = st.value
        if self.status != 0:
            lib.lmo_free(self.h)
            self.h = None
            raise OracleError(f"oracle rejected the lattice (status {self.status})")
        if nodes is None:
            lib.lmo_metamesh(self.h, 0, self.N)
        else:
            self.metamesh_nodes(nodes)

    def metamesh_nodes(self, nodes):
        """Meta-mesh the listed nodes (one call per run of consecutive ids)."""
        lib = _load()
        ids = np.unique(np.asarray(nodes, dtype=np.int64).ravel())
        if ids.size == 0:
            return
        cut = np.nonzero(np.diff(ids) != 1)[0] + 1
        for run in np.split(ids, cut):
            lib.lmo_metamesh(self.h, int(run[0]), int(run[-1]) + 1)

    def __del__(self):
        if getattr(self, "h", None):
            _load().lmo_free(self.h)
            self.h = None

    def csr(self):
        row = np.zeros(self.N + 1, dtype=np.int64)
        adj = np.zeros(2 * self.E, dtype=np.int32)
        R = np.zeros(self.N, dtype=np.float64)
        _load().lmo_csr(self.h, _p(row, c_i64p), _p(adj, c_i32p), _p(R, c_dp))
        return row, adj, R

    def end_frame(self, n, li):
        out = np.zeros(11)
        _load().lmo_end_frame(self.h, int(n), int(li), _p(out, c_dp))
        return {"u": out[0:3], "e1": out[3:6], "e2": out[6:9], "s": out[9], "co": out[10]}

    def arc_points(self, n, a, k):
        """Node-relative points of node-local arc a at resolution k."""
        buf = np.zeros((4 * int(k) + 8, 3))
        N = _load().lmo_arc_points(self.h, int(n), int(a), int(k), _p(buf, c_dp))
        return buf[:N + 1].copy()

    def envelope(self, n, li, phi):
        """Direct evaluation of max(0, max_j h_j(phi)) and its arg-max."""
        phi = np.ascontiguousarray(phi, dtype=np.float64)
        t = np.zeros_like(phi)
        lab = np.zeros(phi.shape, dtype=np.int32)
        _load().lmo_envelope(self.h, int(n), int(li), phi.size, _p(phi, c_dp), _p(t, c_dp),
                             _p(lab, c_i32p))
        return t, lab

    def node_sizes(self, n0=0, n1=None):
        n1 = self.N if n1 is None else n1
        out = np.zeros((n1 - n0, 6), dtype=np.int64)
        _load().lmo_node_sizes(self.h, n0, n1, _p(out, c_i64p))
        return out

    def node(self, n):
        """All meta-mesh data of node n (node-local ids)."""
        fl, V, A, LE, H, HE = self.node_sizes(n, n + 1)[0]
        row, _, _ = self._csr_cache()
        d = int(row[n + 1] - row[n])
        vz = np.zeros((V, 3))
        vkey = np.zeros(V, dtype=np.uint64)
        vfl = np.zeros(V, dtype=np.uint32)
        vgen = np.zeros(V, dtype=np.uint32)
        arc_i = np.zeros((A, 4), dtype=np.int32)
        arc_f = np.zeros((A, 2))
        loop_len = np.zeros(d, dtype=np.int32)
        loop_ent = np.zeros(LE, dtype=np.uint32)
        hole_len = np.zeros(H, dtype=np.int32)
        hole_ent = np.zeros(HE, dtype=np.uint32)
        _load().lmo_node_export(self.h, n, _p(vz, c_dp), _p(vkey, c_u64p), _p(vfl, c_u32p),
                                _p(vgen, c_u32p), _p(arc_i, c_i32p), _p(arc_f, c_dp),
                                _p(loop_len, c_i32p), _p(loop_ent, c_u32p), _p(hole_len, c_i32p),
                                _p(hole_ent, c_u32p))
        return {"flags": int(fl), "vz": vz, "vkey": vkey, "vflags": vfl, "vgen": vgen,
                "arc_i": arc_i, "arc_f": arc_f, "loop_len": loop_len, "loop_ent": loop_ent,
                "hole_len": hole_len, "hole_ent": hole_ent, "d": d}

    def _csr_cache(self):
        if not hasattr(self, "_csr"):
            self._csr = self.csr()
        return self._csr

    def totals(self):
        """(V, elliptical arcs, circular arcs, holes) over all nodes."""
        s = self.node_sizes()
        V = int(s[:, 1].sum())
        H = int(s[:, 4].sum())
        n_ell = n_circ = 0
        for n in range(self.N):
            if s[n, 2] == 0:
                continue
            a = self.node(n)["arc_i"]
            n_circ += int((a[:, 1] < 0).sum())
            n_ell += int((a[:, 1] >= 0).sum())
        return V, n_ell, n_circ, H

    def tri_counts(self, k, i0=0, i1=None):
        i1 = self.E + self.N if i1 is None else i1
        out = np.zeros(i1 - i0, dtype=np.int64)
        _load().lmo_tri_counts(self.h, int(k), i0, i1, _p(out, c_i64p))
        return out

    def triangulate(self, k, i0=0, i1=None, want_tris=True):
        """Triangles of items [i0, i1) (struts first, then node hole fans):
        returns (tris[T,4,3] = normal, v0, v1, v2; area; volume)."""
        i1 = self.E + self.N if i1 is None else i1
        T = int(self.tri_counts(k, i0, i1).sum())
        tris = np.zeros((T, 12)) if want_tris else None
        acc = np.zeros(2)
        got = _load().lmo_triangulate(self.h, int(k), i0, i1,
                                      _p(tris, c_dp) if want_tris else None, _p(acc, c_dp))
        assert got == T, (got, T)
        return (tris.reshape(T, 4, 3) if want_tris else None), float(acc[0]), float(acc[1])


class Frozen:
    """The discrete structure of an oracle triangulation at resolution k
    (vertex generators, arcs, loops, holes, segment counts, stitching order,
    fan-centre rule), re-evaluated at perturbed node positions and radii:
    the function whose derivative the adjoint computes."""

    def __init__(self, o, k):
        self.o = o
        self.k = int(k)
        self.h = _load().lmo_frozen_record(o.h, self.k)

    def __del__(self):
        if getattr(self, "h", None):
            _load().lmo_frozen_free(self.h)
            self.h = None

    def objective(self, xyz, node_R):
        """(area, volume) at node positions xyz [N,3] and node radii [N]."""
        xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        node_R = np.ascontiguousarray(node_R, dtype=np.float64)
        out = np.zeros(2)
        _load().lmo_frozen_objective(self.o.h, self.h, _p(xyz, c_dp), _p(node_R, c_dp), _p(out, c_dp))
        return float(out[0]), float(out[1])

    def fd(self, step, nodes):
        """Central differences: arrays (d_area, d_volume), each [len(nodes), 4]
        with columns d/dx, d/dy, d/dz, d/dR of the listed nodes."""
        nodes = np.ascontiguousarray(nodes, dtype=np.int64)
        g = np.zeros((nodes.size, 8))
        _load().lmo_frozen_fd(self.o.h, self.h, float(step), _p(nodes, c_i64p), nodes.size, _p(g, c_dp))
        return g[:, :4].copy(), g[:, 4:].copy()
