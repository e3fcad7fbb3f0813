"""Thin ctypes binding of the liblm C ABI (include/liblm.h).

Argument marshalling only: every step of the meta-meshing / triangulation
path runs in the CUDA library ``_liblm.so`` built from ``csrc/``.  There is
no CPU fallback: if the library or a CUDA device is missing, calls raise.
PyTorch is used for device memory and streams.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_liblm.so")

LM_F32, LM_F64 = 0, 1
STATUS = {0: "LM_OK", 1: "LM_ERR_INVALID_ARG", 2: "LM_ERR_RADIUS_MISMATCH", 3: "LM_ERR_DEGENERATE",
          4: "LM_ERR_CAPACITY", 5: "LM_ERR_OOM", 6: "LM_ERR_CUDA", 7: "LM_ERR_TIMEOUT",
          8: "LM_ERR_VALENCE", 9: "LM_ERR_STATE", 10: "LM_ERR_IO"}
EXPORTS = ["lm_build_metamesh", "lm_metamesh_counts", "lm_metamesh_export", "lm_tri_count",
           "lm_tri_range", "lm_triangulate", "lm_triangulate_stream", "lm_stl_header",
           "lm_objective", "lm_metamesh_backward", "lm_last_error", "lm_metamesh_free",
           "lm_status_string", "lm_copy_to_host", "lm_launch_count", "lm_triangulate_noalloc",
           "lm_fp64_counts", "lm_metamesh_launch_shape", "lm_metamesh_build_times", "lm_eval_angle_fns",
           "lm_cuda_error_string", "lm_pool_retain", "lm_triangulate_to_file", "lm_envelope_samples",
           "lm_stream_chunked"]


class LmError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = int(status)
        msg = f"{where}: {STATUS.get(self.status, self.status)}"
        if self.status in (5, 6) and _lib is not None:
            msg += f" ({_lib.lm_cuda_error_string().decode()})"
        super().__init__(msg)


class lm_lattice(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int64), ("n_struts", ctypes.c_int64), ("dtype", ctypes.c_int32),
                ("pad_", ctypes.c_int32), ("node_xyz", ctypes.c_void_p),
                ("strut_ends", ctypes.c_void_p), ("end_radii", ctypes.c_void_p)]


class lm_options(ctypes.Structure):
    _fields_ = [("autotune", ctypes.c_int32), ("block_warps", ctypes.c_int32),
                ("grid_ctas", ctypes.c_int32), ("nodes_per_task", ctypes.c_int32),
                ("arena_bytes", ctypes.c_int64), ("redo_list_cap", ctypes.c_int64),
                ("mem_budget", ctypes.c_int64), ("reserved", ctypes.c_int64 * 1)]


class lm_metamesh_view(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("n_nodes", "n_struts", "n_vtx", "n_arcs", "n_loop_ent",
                                              "n_holes", "n_hole_ent")] + \
               [("dtype", ctypes.c_int32), ("pad_", ctypes.c_int32)] + \
               [(n, ctypes.c_void_p) for n in ("row_ptr", "adj", "node_R", "node_flags", "node_vtx_off",
                                               "vtx_z", "vtx_key", "vtx_flags", "vtx_gen", "node_arc_off",
                                               "arc_ends", "arc_vtx", "arc_phi", "end_loop_off", "loop_ent",
                                               "node_hole_off", "hole_off", "hole_ent")]


CHUNK_CB = ctypes.CFUNCTYPE(None, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p,
                            ctypes.c_void_p)
KCHUNK_CB = ctypes.CFUNCTYPE(None, ctypes.c_int64, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64,
                             ctypes.c_void_p, ctypes.c_void_p)
_lib = None


def load():
    """Load _liblm.so (build it with paper_2405_15197_gb300.build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library not built: {LIB_PATH} (run __graft_entry__.build())")
    lib = ctypes.CDLL(LIB_PATH)
    V, I32, I64, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    P64 = ctypes.POINTER(ctypes.c_int64)
    PD = ctypes.POINTER(ctypes.c_double)
    sig = {
        "lm_build_metamesh": ([ctypes.POINTER(lm_lattice), ctypes.POINTER(lm_options), V,
                               ctypes.POINTER(V)], ctypes.c_int),
        "lm_metamesh_counts": ([V, P64], ctypes.c_int),
        "lm_metamesh_export": ([V, ctypes.POINTER(lm_metamesh_view)], ctypes.c_int),
        "lm_tri_count": ([V, I32, V, P64], ctypes.c_int),
        "lm_tri_range": ([V, I64, I64, P64, P64], ctypes.c_int),
        "lm_triangulate": ([V, I32, I64, I64, V, I64, V], ctypes.c_int),
        "lm_triangulate_stream": ([V, I32, I64, V, I64, I32, CHUNK_CB, V, V, P64], ctypes.c_int),
        "lm_stl_header": ([ctypes.c_char_p, I64], None),
        "lm_objective": ([V, I32, V, PD, PD], ctypes.c_int),
        "lm_metamesh_backward": ([V, I32, D, D, V, V, V, PD, PD], ctypes.c_int),
        "lm_last_error": ([V, V], ctypes.c_int),
        "lm_metamesh_free": ([V], None),
        "lm_status_string": ([ctypes.c_int], ctypes.c_char_p),
        "lm_copy_to_host": ([V, V, I64], ctypes.c_int),
        "lm_launch_count": ([], ctypes.c_longlong),
        "lm_fp64_counts": ([V, P64], ctypes.c_int),
        "lm_triangulate_noalloc": ([V, I32, I64, I64, V, I64, V, P64], ctypes.c_int),
        "lm_metamesh_launch_shape": ([V, ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
        "lm_metamesh_build_times": ([V, ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
        "lm_eval_angle_fns": ([V, V, V, I64, V, V, V, V], ctypes.c_int),
        "lm_cuda_error_string": ([], ctypes.c_char_p),
        "lm_pool_retain": ([ctypes.c_uint64], ctypes.c_int),
        "lm_stream_chunked": ([ctypes.POINTER(lm_lattice), ctypes.POINTER(lm_options), ctypes.POINTER(ctypes.c_int32),
                               ctypes.c_int32, ctypes.c_int64, V, ctypes.c_int64, ctypes.c_int32, KCHUNK_CB, V, V,
                               ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
        "lm_envelope_samples": ([V, ctypes.c_int32, ctypes.c_int32, V, V, V], ctypes.c_int),
        "lm_triangulate_to_file": ([V, ctypes.c_int32, ctypes.c_char_p, ctypes.c_int64, V, ctypes.c_int64,
                                    ctypes.c_int32, ctypes.c_int32, V, ctypes.POINTER(ctypes.c_int64),
                                    ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _ck(s, where):
    if s != 0:
        raise LmError(s, where)


def _stream_ptr(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def lm_build_metamesh(xyz, ends, radii, options=None, stream=None):
    """Handle of the meta-mesh of a lattice given as CUDA tensors
    (xyz [N,3] and radii [E,2] float32/float64, ends [E,2] int32)."""
    import torch
    for t in (xyz, ends, radii):
        if not (t.is_cuda and t.is_contiguous()):
            raise ValueError("lattice tensors must be contiguous CUDA tensors")
    if ends.dtype != torch.int32 or xyz.dtype != radii.dtype or xyz.dtype not in (torch.float32, torch.float64):
        raise ValueError("ends must be int32; xyz and radii float32 or float64 of one dtype")
    lat = lm_lattice(xyz.shape[0], ends.shape[0], LM_F32 if xyz.dtype == torch.float32 else LM_F64, 0,
                     xyz.data_ptr(), ends.data_ptr(), radii.data_ptr())
    opt = options if options is not None else lm_options()
    h = ctypes.c_void_p()
    _ck(load().lm_build_metamesh(ctypes.byref(lat), ctypes.byref(opt), _stream_ptr(stream), ctypes.byref(h)),
        "lm_build_metamesh")
    return h


def lm_stream_chunked(xyz, ends, radii, ks, build_struts, ring_ptr, slot_bytes, n_slots, callback=None,
                      options=None, stream=None):
    """Meta-mesh and triangulate the lattice chunk by chunk (the next chunk's
    build beside the current chunk's streaming) through the pinned ring;
    callback(seq, k, first_item, n_tris, slot_ptr, user).  Returns the
    triangles emitted per k."""
    import torch
    for t in (xyz, ends, radii):
        if not (t.is_cuda and t.is_contiguous()):
            raise ValueError("lattice tensors must be contiguous CUDA tensors")
    if ends.dtype != torch.int32 or xyz.dtype != radii.dtype or xyz.dtype not in (torch.float32, torch.float64):
        raise ValueError("ends must be int32; xyz and radii float32 or float64 of one dtype")
    lat = lm_lattice(xyz.shape[0], ends.shape[0], LM_F32 if xyz.dtype == torch.float32 else LM_F64, 0,
                     xyz.data_ptr(), ends.data_ptr(), radii.data_ptr())
    opt = options if options is not None else lm_options()
    kk = (ctypes.c_int32 * len(ks))(*[int(k) for k in ks])
    tris = (ctypes.c_int64 * len(ks))()
    cb = KCHUNK_CB(callback) if callback is not None else KCHUNK_CB()
    _ck(load().lm_stream_chunked(ctypes.byref(lat), ctypes.byref(opt), kk, len(ks), int(build_struts),
                                 ctypes.c_void_p(int(ring_ptr)), int(slot_bytes), int(n_slots), cb, None,
                                 _stream_ptr(stream), tris), "lm_stream_chunked")
    return list(tris)


def lm_metamesh_counts(h):
    out = (ctypes.c_int64 * 8)()
    _ck(load().lm_metamesh_counts(h, out), "lm_metamesh_counts")
    return list(out)


def lm_metamesh_export(h):
    v = lm_metamesh_view()
    _ck(load().lm_metamesh_export(h, ctypes.byref(v)), "lm_metamesh_export")
    return v


def lm_tri_count(h, k, stream=None):
    tot = ctypes.c_int64()
    _ck(load().lm_tri_count(h, int(k), _stream_ptr(stream), ctypes.byref(tot)), "lm_tri_count")
    return tot.value


def lm_tri_range(h, item_begin, item_end):
    a, b = ctypes.c_int64(), ctypes.c_int64()
    _ck(load().lm_tri_range(h, int(item_begin), int(item_end), ctypes.byref(a), ctypes.byref(b)),
        "lm_tri_range")
    return a.value, b.value


def lm_triangulate(h, k, item_begin, item_end, out_ptr, capacity_tris, stream=None):
    _ck(load().lm_triangulate(h, int(k), int(item_begin), int(item_end), ctypes.c_void_p(int(out_ptr)),
                              int(capacity_tris), _stream_ptr(stream)), "lm_triangulate")


def lm_triangulate_stream(h, k, chunk_items, ring_ptr, slot_bytes, n_slots, callback=None, stream=None):
    cb = CHUNK_CB(callback) if callback is not None else CHUNK_CB()
    tot = ctypes.c_int64()
    _ck(load().lm_triangulate_stream(h, int(k), int(chunk_items), ctypes.c_void_p(int(ring_ptr)),
                                     int(slot_bytes), int(n_slots), cb, None, _stream_ptr(stream),
                                     ctypes.byref(tot)), "lm_triangulate_stream")
    return tot.value


LM_FILE_SYNC = 1
LM_ENV_WARP, LM_ENV_THREAD = 0, 1


def lm_envelope_samples(h, samples, mode, t_ptr, label_ptr, stream=None):
    """Trimming envelope t*(phi_q) and its arg-max at `samples` angles of
    every strut end, warp-centric (LM_ENV_WARP) or thread-centric
    (LM_ENV_THREAD); outputs [2E][samples] at the given device pointers."""
    _ck(load().lm_envelope_samples(h, int(samples), int(mode), ctypes.c_void_p(int(t_ptr)),
                                   ctypes.c_void_p(int(label_ptr)), _stream_ptr(stream)), "lm_envelope_samples")


def lm_triangulate_to_file(h, k, path, ring_ptr, slot_bytes, n_slots, chunk_items=0, sync=False, stream=None):
    """Binary-STL file of the triangulation at k through the pinned ring
    (GPU triangulation, device-to-host copy and file writes overlapped).
    Returns (triangles, {"total_s", "write_s", "wait_s", "fsync_s"})."""
    tot = ctypes.c_int64()
    st = (ctypes.c_double * 4)()
    _ck(load().lm_triangulate_to_file(h, int(k), os.fsencode(path), int(chunk_items), ctypes.c_void_p(int(ring_ptr)),
                                      int(slot_bytes), int(n_slots), LM_FILE_SYNC if sync else 0,
                                      _stream_ptr(stream), ctypes.byref(tot), st), "lm_triangulate_to_file")
    return tot.value, {"total_s": st[0], "write_s": st[1], "wait_s": st[2], "fsync_s": st[3]}


def lm_triangulate_noalloc(h, k, item_begin, item_end, out_ptr, capacity_tris, stream=None):
    """Allocation-free triangulation of items [begin, end) (at most 262,144
    items per call); returns the range's triangle count.  See liblm.h."""
    n = ctypes.c_int64()
    _ck(load().lm_triangulate_noalloc(h, int(k), int(item_begin), int(item_end), ctypes.c_void_p(int(out_ptr)),
                                      int(capacity_tris), _stream_ptr(stream), ctypes.byref(n)),
        "lm_triangulate_noalloc")
    return n.value


def lm_stl_header(n_tris):
    buf = ctypes.create_string_buffer(84)
    load().lm_stl_header(buf, int(n_tris))
    return buf.raw


def lm_objective(h, k, stream=None):
    a, v = ctypes.c_double(), ctypes.c_double()
    _ck(load().lm_objective(h, int(k), _stream_ptr(stream), ctypes.byref(a), ctypes.byref(v)), "lm_objective")
    return a.value, v.value


def lm_metamesh_backward(h, k, w_area, w_vol, grad_xyz_ptr, grad_r_ptr, stream=None):
    a, v = ctypes.c_double(), ctypes.c_double()
    _ck(load().lm_metamesh_backward(h, int(k), float(w_area), float(w_vol), ctypes.c_void_p(int(grad_xyz_ptr)),
                                    ctypes.c_void_p(int(grad_r_ptr)), _stream_ptr(stream), ctypes.byref(a),
                                    ctypes.byref(v)), "lm_metamesh_backward")
    return a.value, v.value


def lm_last_error(h, stream=None):
    return load().lm_last_error(h, _stream_ptr(stream))


def lm_metamesh_free(h):
    if h:
        load().lm_metamesh_free(h)


def lm_status_string(s):
    return load().lm_status_string(int(s)).decode()


N_FP64_COUNTS = 18


def lm_fp64_counts(h):
    out = (ctypes.c_int64 * N_FP64_COUNTS)()
    _ck(load().lm_fp64_counts(h, out), "lm_fp64_counts")
    return list(out)


def lm_eval_angle_fns(y, x, a, stream=None):
    """(lm_atan2(y, x), sin a, cos a) of float32 CUDA tensors, as computed by
    the library's FP32 angle functions."""
    import torch
    n = y.numel()
    at, sn, cs = (torch.empty(n, dtype=torch.float32, device=y.device) for _ in range(3))
    _ck(load().lm_eval_angle_fns(y.data_ptr(), x.data_ptr(), a.data_ptr(), n, at.data_ptr(), sn.data_ptr(),
                                 cs.data_ptr(), _stream_ptr(stream)), "lm_eval_angle_fns")
    return at, sn, cs


def lm_launch_count():
    return int(load().lm_launch_count())


def lm_pool_retain(nbytes):
    """Let the current device's default memory pool keep up to `nbytes` of
    the memory the library frees (0: give it back at every synchronisation)."""
    _ck(load().lm_pool_retain(int(nbytes)), "lm_pool_retain")


def lm_copy_to_host(dptr, nbytes, dtype):
    """Download `nbytes` from a device pointer into a new numpy array."""
    arr = np.empty(int(nbytes) // np.dtype(dtype).itemsize, dtype=dtype)
    if arr.size:
        _ck(load().lm_copy_to_host(arr.ctypes.data_as(ctypes.c_void_p), ctypes.c_void_p(dptr), arr.nbytes),
            "lm_copy_to_host")
    return arr


class MetaMesh:
    """Owning wrapper: keeps the lattice tensors alive for the handle's life."""

    def __init__(self, xyz, ends, radii, options=None, stream=None):
        self._keep = (xyz, ends, radii)
        self.dtype = xyz.dtype
        self.h = lm_build_metamesh(xyz, ends, radii, options, stream)
        self.n_nodes, self.n_struts = xyz.shape[0], ends.shape[0]

    def close(self):
        if getattr(self, "h", None):
            lm_metamesh_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def counts(self):
        return lm_metamesh_counts(self.h)

    def tri_count(self, k, stream=None):
        return lm_tri_count(self.h, k, stream)

    def triangulate(self, k, item_begin=0, item_end=None, out=None, stream=None):
        """STL records (uint8 CUDA tensor [T, 50]) of items [begin, end)."""
        import torch
        item_end = self.n_struts + self.n_nodes if item_end is None else item_end
        first, cnt = lm_tri_range(self.h, item_begin, item_end)
        if out is None:
            out = torch.empty((max(cnt, 1), 50), dtype=torch.uint8, device="cuda")
        lm_triangulate(self.h, k, item_begin, item_end, out.data_ptr(), out.shape[0], stream)
        return out[:cnt]

    def objective(self, k, stream=None):
        return lm_objective(self.h, k, stream)

    def backward(self, k, w_area=1.0, w_vol=0.0, stream=None):
        """Adjoint at k: (d/d node xyz [N,3], d/d node radius [N], area,
        volume) of w_area*area + w_vol*volume, as CUDA tensors of the
        lattice dtype."""
        import torch
        gx = torch.zeros((self.n_nodes, 3), dtype=self.dtype, device="cuda")
        gr = torch.zeros((self.n_nodes,), dtype=self.dtype, device="cuda")
        a, v = lm_metamesh_backward(self.h, k, w_area, w_vol, gx.data_ptr(), gr.data_ptr(), stream)
        return gx, gr, a, v

    def download(self):
        """Host copies of every meta-mesh array (numpy)."""
        v = lm_metamesh_export(self.h)
        fdt = np.float32 if v.dtype == LM_F32 else np.float64
        N, E = v.n_nodes, v.n_struts
        g = lm_copy_to_host
        return {
            "row_ptr": g(v.row_ptr, 8 * (N + 1), np.int64), "adj": g(v.adj, 4 * 2 * E, np.int32),
            "node_R": g(v.node_R, np.dtype(fdt).itemsize * N, fdt),
            "node_flags": g(v.node_flags, 4 * N, np.uint32),
            "vtx_off": g(v.node_vtx_off, 8 * (N + 1), np.int64),
            "vtx_z": g(v.vtx_z, np.dtype(fdt).itemsize * 3 * v.n_vtx, fdt).reshape(-1, 3),
            "vtx_key": g(v.vtx_key, 8 * v.n_vtx, np.uint64), "vtx_flags": g(v.vtx_flags, 4 * v.n_vtx, np.uint32),
            "vtx_gen": g(v.vtx_gen, 4 * v.n_vtx, np.uint32),
            "arc_off": g(v.node_arc_off, 8 * (N + 1), np.int64),
            "arc_ends": g(v.arc_ends, 8 * v.n_arcs, np.int32).reshape(-1, 2),
            "arc_vtx": g(v.arc_vtx, 4 * v.n_arcs, np.uint32),
            "arc_phi": g(v.arc_phi, np.dtype(fdt).itemsize * 2 * v.n_arcs, fdt).reshape(-1, 2),
            "end_off": g(v.end_loop_off, 8 * (2 * E + 1), np.int64),
            "loop_ent": g(v.loop_ent, 4 * v.n_loop_ent, np.uint32),
            "hole_off_n": g(v.node_hole_off, 8 * (N + 1), np.int64),
            "hole_off": g(v.hole_off, 8 * (v.n_holes + 1), np.int64),
            "hole_ent": g(v.hole_ent, 4 * v.n_hole_ent, np.uint32),
        }


def lm_metamesh_launch_shape(h):
    """[(warps per block, nodes per queue access)] per valence bucket."""
    out = (ctypes.c_int32 * 8)()
    _ck(load().lm_metamesh_launch_shape(h, out), "lm_metamesh_launch_shape")
    return [(out[2 * b], out[2 * b + 1]) for b in range(3)]


def lm_metamesh_build_times(h):
    """Device ms of the build: (CSR and tuning, count-pass kernel, sizing and
    output allocation, arena gather, emit pass)."""
    out = (ctypes.c_float * 5)()
    _ck(load().lm_metamesh_build_times(h, out), "lm_metamesh_build_times")
    return tuple(float(x) for x in out)


def lm_metamesh_emit_nodes(h, listed=False):
    """Nodes the build computed a second time (not held by its arena); with
    listed=True also whether the emit pass took only those from the count
    pass's lists (True) or went over every node (False)."""
    out = (ctypes.c_int32 * 8)()
    _ck(load().lm_metamesh_launch_shape(h, out), "lm_metamesh_launch_shape")
    return (int(out[6]), bool(out[7])) if listed else int(out[6])
