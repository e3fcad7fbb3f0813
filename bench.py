"""Benchmark of the lattice meta-meshing + triangulation hot path on GB300.

One step = one pass of the whole path over the workload: node-sorted CSR
build, persistent meta-mesh (count + emit passes), then triangulation at
k = 8 and k = 32 from that one meta-mesh, STL records written to HBM.

Workload (default): octet-truss 100x100x100 cells, 4,060,301 nodes,
24,120,000 struts, node radii uniform in [0.04, 0.08] (cones), FP32 with FP64
stability steps; inputs are synthetic (seeded) and resident in HBM before the
timed region (they are larger than L2).  `value` = struts per second through
the whole step.  `e2e` runs the same step through the C ABI from pinned host
inputs, streaming every triangle back into a pinned host ring.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload octet100|bcc500|...]
  python bench.py --impl reference   # the FP64 CPU oracle on a bounded sample
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "octet100": {"kind": "octet", "n": 100, "ks": (8, 32),
                 "desc": "octet-truss 100^3 cells, radii U[0.04,0.08] per node (cones), k=8 and k=32 from one meta-mesh"},
    "octet40": {"kind": "octet", "n": 40, "ks": (8, 32),
                "desc": "octet-truss 40^3 cells (smaller case), k=8 and k=32"},
    "octet24": {"kind": "octet", "n": 24, "ks": (8, 32),
                "desc": "octet-truss 24^3 cells (profiling case), k=8 and k=32"},
    "bcc500": {"kind": "bcc", "n": 500, "ks": (8, 32), "R": 0.05,
               "desc": "BCC 500^3 cells, 1.0e9 struts, R=0.05, k=8 and k=32"},
    "bcc40": {"kind": "bcc", "n": 40, "ks": (8, 32), "R": 0.05,
              "desc": "BCC 40^3 cells (profiling case of the 500^3 lattice), R=0.05, k=8 and k=32"},
}

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum of the stitching,
# FP64 and hole-fan launches) per triangle of the k = 32 emit, measured with
# ncu on the profiling case of the lattice family (octet 24^3) with the
# current kernels; the benchmark scales it by the triangles of its own emit
# (no entry: not measured with the current kernels, reported as null)
TRAFFIC_PER_TRI_K32 = {"octet": 52.4}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev = dev
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"lm_bench_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    mx.append(float(f[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, f[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def make_lattice_device(wl, device, torch):
    from paper_2405_15197_gb300 import lattices as L
    if wl["kind"] == "bcc":
        return L.bcc_device(wl["n"], wl["R"], device)
    lat = L.octet(wl["n"])
    return (torch.tensor(lat["xyz"], dtype=torch.float32, device=device),
            torch.tensor(lat["ends"], dtype=torch.int32, device=device),
            torch.tensor(lat["radii"], dtype=torch.float32, device=device))


_chunk_cache = {}


def emit_chunks(liblm, mm, k, cap_tris):
    """Item ranges whose records fit the device output buffer (one range when
    the whole triangulation fits; the 1e9-strut lattice reuses a bounded
    buffer chunk after chunk).  Sized once per (lattice, k) from the counts."""
    n_items = mm.n_struts + mm.n_nodes
    key = (mm.n_struts, mm.n_nodes, k, cap_tris)
    if key not in _chunk_cache:
        _, total = liblm.lm_tri_range(mm.h, 0, n_items)
        if total <= cap_tris:
            _chunk_cache[key] = [(0, n_items)]
        else:
            step = max(1, int(0.5 * cap_tris * n_items / total))
            ranges, b = [], 0
            while b < n_items:
                e = min(n_items, b + step)
                while liblm.lm_tri_range(mm.h, b, e)[1] > cap_tris:
                    e = b + max(1, (e - b) // 2)
                ranges.append((b, e))
                b = e
            _chunk_cache[key] = ranges
    return _chunk_cache[key]


def tuned_options(liblm):
    """Build options with the launch-shape autotuner on (cached per process)."""
    opt = liblm.lm_options()
    opt.autotune = 1
    return opt


def run_step(torch, liblm, xyz, ends, radii, ks, out, stream, want_times=False):
    """One full step on device-resident inputs.  Returns (struts, tris per k,
    per-phase times in ms) ."""
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 + 2 * len(ks))]
    ev[0].record(stream)
    mm = liblm.MetaMesh(xyz, ends, radii, options=tuned_options(liblm), stream=stream)
    ev[1].record(stream)
    tris = []
    for q, k in enumerate(ks):
        n = mm.tri_count(k, stream)
        ev[2 + 2 * q].record(stream)
        for b, e in emit_chunks(liblm, mm, k, out.numel() // 50):
            liblm.lm_triangulate(mm.h, k, b, e, out.data_ptr(), out.numel() // 50, stream)
        ev[3 + 2 * q].record(stream)
        tris.append(n)
    err = liblm.lm_last_error(mm.h, stream)
    if err:
        raise RuntimeError(f"device error {liblm.lm_status_string(err)}")
    times = None
    if want_times:
        stream.synchronize()
        times = {"metamesh_ms": ev[0].elapsed_time(ev[1])}
        for q, k in enumerate(ks):
            times[f"tri_k{k}_ms"] = ev[2 + 2 * q].elapsed_time(ev[3 + 2 * q])
            times[f"count_k{k}_ms"] = (ev[1] if q == 0 else ev[1 + 2 * q]).elapsed_time(ev[2 + 2 * q])
    mm.close()
    return ends.shape[0], tris, times


def max_over_ranks(torch, ms, dev):
    """Largest per-step time over the ranks (one all-reduce; the time itself
    when there is one process)."""
    dist = torch.distributed
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms
    t = torch.tensor([ms], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, n_struts, ms):
    """Whole-job struts/s: every replica meta-meshes and triangulates a lattice
    of n_struts struts per step (weak scaling), the slowest sets the time."""
    return world * n_struts / (ms / 1e3)


def bench_gpu(args):
    import torch

    from paper_2405_15197_gb300 import build, liblm

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build.build()
    liblm.load()
    wl = WORKLOADS[args.workload]
    ks = wl["ks"]
    xyz, ends, radii = make_lattice_device(wl, dev, torch)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    # output buffer sized for the larger k (this first build also runs the
    # launch-shape autotuner; later builds reuse its choice)
    mm = liblm.MetaMesh(xyz, ends, radii, options=tuned_options(liblm), stream=stream)
    totals = [mm.tri_count(k, stream) for k in ks]
    counts = mm.counts()
    launch_shape = liblm.lm_metamesh_launch_shape(mm.h)
    fb = liblm.lm_fp64_counts(mm.h)
    fp64 = dict(zip(["pair", "candidate", "position_refine", "dedup", "seam", "loop_angle", "label",
                     "arc_extent", "tri_segments", "tri_start_angle", "tri_stitch_order", "tri_fan_centre"],
                    fb[:12]))
    t_build = {"csr": None}
    mm.close()
    # device output buffer: the whole triangulation when it fits in 64 GB,
    # else a reused 16 GB chunk buffer
    out_bytes = max(totals) * 50
    if out_bytes > (64 << 30):
        out_bytes = 16 << 30
    out = torch.empty(out_bytes, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        run_step(torch, liblm, xyz, ends, radii, ks, out, stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    phase = []
    with Clocks(local) as clk:
        l0 = liblm.lm_launch_count()
        start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        start.record(stream)
        for s in range(args.steps):
            _, tris, tm = run_step(torch, liblm, xyz, ends, radii, ks, out, stream, want_times=False)
        stop.record(stream)
        torch.cuda.synchronize()
        l1 = liblm.lm_launch_count()
    ms = max_over_ranks(torch, start.elapsed_time(stop) / args.steps, dev)
    # per-phase times of one extra step (not part of the timed region)
    _, _, phase = run_step(torch, liblm, xyz, ends, radii, ks, out, stream, want_times=True)
    E = ends.shape[0]
    value = job_value(world, E, ms)
    peaks, peak_kind = load_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    # dominant kernel: largest phase
    k_big = max(ks)
    tri_ms = phase[f"tri_k{k_big}_ms"]
    tri_bytes = 50.0 * totals[ks.index(k_big)]
    roof_tri = {"bound": "hbm", "achieved": tri_bytes / (tri_ms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                "frac": tri_bytes / (tri_ms / 1e3) / 1e9 / hbm,
                "traffic": (TRAFFIC_PER_TRI_K32[wl["kind"]] * totals[ks.index(k_big)]
                            if k_big == 32 and wl["kind"] in TRAFFIC_PER_TRI_K32 else None),
                "kernel": f"triangulation emit at k={k_big} (k_tri_tiles FP32 pass + FP64 pass + k_tri_holes)",
                "algorithmic_bytes": "50 B written per triangle", "peak_kind": f"{peak_kind} hbm_gbs"}
    # end-to-end: pinned host inputs -> device -> meta-mesh -> triangles streamed to a pinned ring
    del out
    torch.cuda.empty_cache()
    e2e = bench_e2e(torch, liblm, xyz, ends, radii, ks, stream, dev, args) if not args.no_e2e else None
    adjoint = bench_adjoint(torch, liblm, dev, stream) if not args.no_adjoint else None
    res = {
        "metric": "meta-mesh struts/s; triangles/s & write GB/s vs HBM peak; adjoint struts/s",
        "value": value, "unit": "struts/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 (f64 stability steps)", "data": "synthetic",
        "config": {"workload": wl["desc"], "name": args.workload, "n_nodes": int(xyz.shape[0]),
                   "n_struts": int(E), "ks": list(ks), "triangles": dict(zip([f"k{k}" for k in ks], totals)),
                   "l2": "inputs (and outputs) larger than L2", "parallelism": f"replicas x{world}"},
        "phases_ms": phase,
        "metamesh_struts_per_s": E / (phase["metamesh_ms"] / 1e3),
        "triangles_per_s": {f"k{k}": totals[i] / (phase[f"tri_k{k}_ms"] / 1e3) for i, k in enumerate(ks)},
        "write_gbs": {f"k{k}": 50.0 * totals[i] / (phase[f"tri_k{k}_ms"] / 1e3) / 1e9 for i, k in enumerate(ks)},
        "meta_mesh_counts": {"vertices": counts[0], "elliptical_arcs": counts[1], "circular_arcs": counts[2],
                             "holes": counts[3], "degenerate_nodes": counts[5], "max_valence": counts[6]},
        "fp64_stability_steps": fp64,
        "metamesh_launch_shape": {"buckets": ["d<=16", "d<=32", "d<=64"],
                                  "warps_per_block_nodes_per_pop": launch_shape, "autotuned": True},
        "roofline": roof_tri,
        "gpu_launches": int((l1 - l0) // max(1, args.steps)) * args.steps,
        "clocks": clk.summary(),
        "e2e": e2e,
        "adjoint": adjoint,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        res["cpu_baseline"] = cpu_baseline(args, quick=True)
    if rank == 0:
        print(json.dumps(res))
    if world > 1:
        torch.distributed.destroy_process_group()


def bench_e2e(torch, liblm, xyz, ends, radii, ks, stream, dev, args):
    hx = xyz.cpu().pin_memory()
    he = ends.cpu().pin_memory()
    hr = radii.cpu().pin_memory()
    slot = 1 << 30
    n_slots = 4
    ring = torch.empty(n_slots * slot, dtype=torch.uint8, pin_memory=True)
    mm_tris = {}
    probe = liblm.MetaMesh(xyz, ends, radii, stream=stream)
    for k in ks:
        mm_tris[k] = probe.tri_count(k, stream)
    probe.close()

    def one():
        dx = hx.to(dev, non_blocking=True)
        de = he.to(dev, non_blocking=True)
        dr = hr.to(dev, non_blocking=True)
        mm = liblm.MetaMesh(dx, de, dr, options=tuned_options(liblm), stream=stream)
        tot = 0
        for k in ks:
            mm.tri_count(k, stream)
            # ~(slot / 50 / 80) items per chunk keeps a chunk inside one slot
            per_item = max(1.0, mm_tris[k] / (mm.n_struts + mm.n_nodes))
            chunk = int(0.8 * slot / 50 / (4 * per_item))
            tot += liblm.lm_triangulate_stream(mm.h, k, chunk, ring.data_ptr(), slot, n_slots, None, stream)
        mm.close()
        return tot

    one()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    steps = max(1, min(args.steps, 3))
    for _ in range(steps):
        tot = one()
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / steps
    E = ends.shape[0]
    return {"value": E / dt, "unit": "struts/s", "ms_per_step": dt * 1e3,
            "h2d_bytes_per_step": int(hx.numel() * hx.element_size() + he.numel() * he.element_size()
                                      + hr.numel() * hr.element_size()),
            "d2h_bytes_per_step": int(50 * tot), "steps": steps,
            "path": "pinned host lattice -> lm_build_metamesh -> lm_triangulate_stream (pinned ring)"}


def bench_adjoint(torch, liblm, dev, stream):
    """Adjoint throughput on the differentiation workload: BCC 64^3 cells with
    Gaussian node jitter 0.05 and node radii U[0.05, 0.09], objective area +
    volume at k = 32 (lm_metamesh_backward, device-resident lattice)."""
    from paper_2405_15197_gb300 import lattices as L
    lat = L.bcc(64, jitter=0.05, radius_range=(0.05, 0.09))
    xyz = torch.tensor(lat["xyz"], dtype=torch.float32, device=dev)
    ends = torch.tensor(lat["ends"], dtype=torch.int32, device=dev)
    radii = torch.tensor(lat["radii"], dtype=torch.float32, device=dev)
    mm = liblm.MetaMesh(xyz, ends, radii, stream=stream)
    mm.tri_count(32, stream)
    gx = torch.zeros((xyz.shape[0], 3), dtype=torch.float32, device=dev)
    gr = torch.zeros((xyz.shape[0],), dtype=torch.float32, device=dev)
    liblm.lm_metamesh_backward(mm.h, 32, 1.0, 1.0, gx.data_ptr(), gr.data_ptr(), stream)
    ts = []
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        liblm.lm_metamesh_backward(mm.h, 32, 1.0, 1.0, gx.data_ptr(), gr.data_ptr(), stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    mm.close()
    ms = statistics.median(ts)
    E = int(ends.shape[0])
    return {"struts_per_s": E / (ms / 1e3), "ms": ms, "n_struts": E, "k": 32,
            "workload": "BCC 64^3 cells, node jitter N(0, 0.05), radii U[0.05, 0.09], d(area + volume)/d(xyz, R)",
            "includes": "objective evaluation + point adjoints + per-node forward-mode pass"}


def cpu_baseline(args, quick=False):
    """The FP64 oracle, as it stands, single-threaded, on a bounded sample of
    the workload: an octet 32^3 sub-block (same generator and radii law) for
    the octet workloads, a BCC 40x40x8 slab for BCC; meta-mesh + both k."""
    import oracle
    from paper_2405_15197_gb300 import lattices as L
    wl = WORKLOADS[args.workload]
    if wl["kind"] == "octet":
        n = 32 if not quick else 16
        lat = L.octet(n)
        sample = f"octet {n}^3 cells ({lat['ends'].shape[0]} struts), meta-mesh + k=8 + k=32"
    else:
        lat = L.bcc(40, 40, 8 if not quick else 4, radius=wl["R"])
        sample = f"BCC slab ({lat['ends'].shape[0]} struts), meta-mesh + k=8 + k=32"
    lat = {k: (v.astype(np.float32).astype(np.float64) if k in ("xyz", "radii") else v) for k, v in lat.items()}
    oracle.build()
    t0 = time.perf_counter()
    o = oracle.Oracle(lat)
    for k in wl["ks"]:
        o.triangulate(k, want_tris=False)
    dt = time.perf_counter() - t0
    E = lat["ends"].shape[0]
    return {"value": E / dt, "unit": "struts/s", "cores": 1, "kind": "oracle", "sample": sample,
            "seconds": dt}


def bench_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    t_steps = []
    cb = None
    for _ in range(args.warmup):
        cpu_baseline(args, quick=True)
    for _ in range(args.steps):
        cb = cpu_baseline(args, quick=True)
        t_steps.append(cb["seconds"])
    wl = WORKLOADS[args.workload]
    res = {"impl": "reference", "metric": "meta-mesh struts/s; triangles/s & write GB/s vs HBM peak; adjoint struts/s",
           "value": cb["value"], "unit": "struts/s", "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * statistics.mean(t_steps), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": wl["desc"], "name": args.workload},
           "cpu_baseline": {"value": cb["value"], "unit": "struts/s", "cores": 1, "kind": "oracle",
                            "sample": cb["sample"]},
           "e2e": {"value": cb["value"], "unit": "struts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(res))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="octet100", choices=sorted(WORKLOADS))
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        bench_reference(args)
    else:
        bench_gpu(args)


if __name__ == "__main__":
    main()
