"""Benchmark of the lattice meta-meshing + triangulation hot path on GB300.

One step = one pass of the whole path over the workload: node-sorted CSR
build, persistent meta-mesh (count pass, arena gather, emit pass), then
triangulation at k = 8 and k = 32 from that one meta-mesh, STL records
written to HBM (a reused 16 GB device buffer, chunk after chunk, when the
records of one k do not fit in 64 GB).

Workload (default): billion-scale BCC 500x500x500 cells, 250,751,501 nodes,
1.0e9 struts, R = 0.05, FP32 with FP64 stability steps; inputs are synthetic
(generated on the device) and resident in HBM before the timed region (they
are larger than L2).  `value` = struts per second through the whole step.
`e2e` runs the same step through the C ABI from pinned host inputs,
streaming every triangle back into a pinned host ring.  The line also
carries the octet-truss 100^3 and the 2e6-node irregular configurations
(extra keys), the adjoint on jittered BCC 64^3, and the FP64 oracle timed on
the host cores (one core and every core).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload bcc500|octet100|...]
  python bench.py --impl reference   # the FP64 CPU oracle on a bounded sample
  python bench.py --cpu-configs      # the oracle on every configuration (host cores)
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

# cpu_one / cpu_all: oracle samples timed on one core and on every core;
# cpu_ref: the reference arm's per-step sample (all cores); cpu_extrapolate:
# whole workload / cpu_all sample
WORKLOADS = {
    "bcc500": {"kind": "bcc", "n": 500, "ks": (8, 32), "R": 0.05,
               "desc": "billion-scale BCC 500^3 cells (1.0e9 struts), R=0.05, meta-mesh once, "
                       "triangulated at k=8 and k=32",
               "cpu_one": ("bcc", 500, 50, 4, 0.05), "cpu_all": ("bcc", 500, 500, 4, 0.05),
               "cpu_ref": ("bcc", 500, 100, 4, 0.05), "cpu_extrapolate": 125},
    "octet100": {"kind": "octet", "n": 100, "ks": (8, 32),
                 "desc": "octet-truss 100^3 cells, radii U[0.04,0.08] per node (cones), k=8 and k=32 from one meta-mesh",
                 "cpu_one": ("octet", 24, 24, 24), "cpu_all": ("octet", 100, 100, 8),
                 "cpu_ref": ("octet", 100, 100, 4), "cpu_extrapolate": 12.5},
    "octet40": {"kind": "octet", "n": 40, "ks": (8, 32),
                "desc": "octet-truss 40^3 cells (smaller case), k=8 and k=32",
                "cpu_one": ("octet", 16, 16, 16), "cpu_all": ("octet", 40, 40, 40), "cpu_ref": ("octet", 40, 40, 8)},
    "octet24": {"kind": "octet", "n": 24, "ks": (8, 32),
                "desc": "octet-truss 24^3 cells (profiling case), k=8 and k=32",
                "cpu_one": ("octet", 16, 16, 16), "cpu_all": ("octet", 24, 24, 24), "cpu_ref": ("octet", 24, 24, 8)},
    "bcc40": {"kind": "bcc", "n": 40, "ks": (8, 32), "R": 0.05,
              "desc": "BCC 40^3 cells (profiling case of the 500^3 lattice), R=0.05, k=8 and k=32",
              "cpu_one": ("bcc", 40, 40, 8, 0.05), "cpu_all": ("bcc", 40, 40, 40, 0.05),
              "cpu_ref": ("bcc", 40, 40, 8, 0.05)},
}

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per triangle of
# the FP32 stitching launch k_tri_tiles at k = 32 (its FP64 and hole-fan
# launches take 1.4 % of the emit's time on BCC), measured with ncu on the
# profiling case of the lattice family (BCC 40^3: 1,727.8 MB over 32.7 M
# triangles of one launch) with the current kernels; the benchmark scales it
# by the triangles of its own emit (no entry: not measured with the current
# kernels, reported as null)
TRAFFIC_PER_TRI_K32 = {"bcc": 52.8}


METRIC = "meta-mesh struts/s; triangles/s & write GB/s vs HBM peak; adjoint struts/s"


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
        bt = liblm.lm_metamesh_build_times(mm.h)
        (times["metamesh_csr_tune_ms"], times["metamesh_count_kernel_ms"], times["metamesh_size_alloc_ms"],
         times["metamesh_gather_ms"], times["metamesh_emit_ms"]) = bt
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


# FP32 lanes per SM (Blackwell): the ALU peak of the meta-mesh kernel is
# SMs x lanes x 2 (an FMA counts two flops) x the maximum SM clock
FP32_LANES_PER_SM = 128
N_SMS = 152


def fp32_peak_tflops(peaks):
    mhz = float(peaks.get("sm_max_mhz", 2070.0))
    return N_SMS * FP32_LANES_PER_SM * 2.0 * mhz * 1e6 / 1e12


def metamesh_flops(vhist):
    """Algorithmic FP32 work of the meta-mesh: per node of valence d,
    15 d(d-1) for the pair classification, (40 + 16 d) per circle-point
    generator (d(d-1)/2 of them: setup + two roots screened against d ends)
    and (170 + 16 d) per triple-point generator (d(d-1)(d-2)/6: the line of
    two planes, the quadratic on the cone, its conditioning estimate, two
    roots screened against d ends)."""
    tot = 0
    for d, cnt in vhist.items():
        c2, c3 = d * (d - 1) // 2, d * (d - 1) * (d - 2) // 6
        tot += cnt * (15 * d * (d - 1) + c2 * (40 + 16 * d) + c3 * (170 + 16 * d))
    return float(tot)


def metamesh_bytes(counts, N, E, tsz=4):
    """Algorithmic DRAM bytes of the meta-mesh build: inputs read once
    (xyz, strut ends, end radii) and every output written once (vertices
    28 B, arcs 20 B, loop and hole entries 4 B, hole offsets 8 B, per-node
    flags / offsets / radius / CSR row, per-end CSR entry and loop offset)."""
    V, ell, circ, H = counts[:4]
    A, LE, HE = ell + circ, 2 * ell + circ, circ
    rd = 3 * tsz * N + 8 * E + 2 * tsz * E
    wr = (V * (3 * tsz + 16) + A * (12 + 2 * tsz) + 4 * LE + 8 * H + 4 * HE
          + N * (4 + 4 * 8 + tsz + 8) + 2 * E * (4 + 8))
    return float(rd + wr)


def valence_hist(torch, ends, n_nodes):
    """{valence: nodes} of a device lattice (chunked bincount)."""
    deg = torch.zeros(n_nodes, dtype=torch.int64, device=ends.device)
    flat = ends.view(-1)
    for c in flat.split(1 << 27):
        deg += torch.bincount(c.long(), minlength=n_nodes)
    h = torch.bincount(deg).cpu().tolist()
    del deg
    return {d: int(c) for d, c in enumerate(h) if c and d}


# ncu-measured figures of the meta-mesh count pass on the profiling case of
# each lattice family (BCC 40^3, 132,921 nodes, one launch): DRAM bytes per
# node (read + write, scaled by the benchmark's node count), FMA / ALU / FP64
# pipe fractions, issue-active fraction, active lanes per warp instruction,
# instruction-cache (GCC) hit rate.  Absent: not measured with the current
# kernel (reported as null).
METAMESH_NCU = {"bcc": {"dram_bytes_per_node": 527.8, "fp32_issue_frac_ncu": 0.131, "alu_pipe_frac_ncu": 0.256,
                        "fp64_pipe_frac_ncu": 0.013, "issue_active_ncu": 0.371, "lanes_per_inst_ncu": 11.5,
                        "icache_gcc_hit_ncu": 0.871}}


def rooflines(wl, ks, totals, phase, counts, vhist, N, E, peaks, peak_kind):
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    k_big = max(ks)
    tri_ms = phase[f"tri_k{k_big}_ms"]
    tri_bytes = 50.0 * totals[ks.index(k_big)]
    tri = {"bound": "hbm", "achieved": tri_bytes / (tri_ms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
           "frac": tri_bytes / (tri_ms / 1e3) / 1e9 / hbm,
           "traffic": (TRAFFIC_PER_TRI_K32[wl["kind"]] * totals[ks.index(k_big)]
                       if k_big == 32 and wl["kind"] in TRAFFIC_PER_TRI_K32 else None),
           "kernel": f"triangulation emit at k={k_big} (k_tri_tiles FP32 pass + FP64 pass + k_tri_holes)",
           "algorithmic_bytes": f"50 B written per triangle x {totals[ks.index(k_big)]} triangles",
           "peak_kind": f"{peak_kind} hbm_gbs (copy burst)"}
    mm_ms = phase["metamesh_ms"]
    kern_ms = phase["metamesh_count_kernel_ms"]
    fl = metamesh_flops(vhist)
    pk = fp32_peak_tflops(peaks)
    ach = fl / (kern_ms / 1e3) / 1e12
    by = metamesh_bytes(counts, N, E)
    ncu = METAMESH_NCU.get(wl["kind"], {})
    mm = {"bound": "alu", "achieved": ach, "peak": pk, "unit": "TFLOP/s", "frac": ach / pk,
          "traffic": ncu["dram_bytes_per_node"] * N if "dram_bytes_per_node" in ncu else None,
          "kernel": "k_metamesh count pass (persistent launch, every node computed once; CUDA events "
                    "around the launch inside the library)",
          "launch_ms": kern_ms,
          "build_achieved": fl / (mm_ms / 1e3) / 1e12, "build_ms": mm_ms,
          "algorithmic_flops": fl, "flops_per_strut": fl / max(E, 1),
          "flop_model": "per node of valence d: 15 d(d-1) + C(d,2)(40 + 16 d) + C(d,3)(170 + 16 d)",
          "peak_kind": f"derived: {N_SMS} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x "
                       f"{float(peaks.get('sm_max_mhz', 2070.0)):.0f} MHz",
          "dram_gbs_algorithmic": by / (mm_ms / 1e3) / 1e9, "algorithmic_bytes": by,
          "dram_frac_algorithmic": by / (mm_ms / 1e3) / 1e9 / hbm,
          "traffic_note": "ncu dram bytes per node of the BCC 40^3 count-pass launch x nodes"}
    mm.update({k: v for k, v in ncu.items() if k != "dram_bytes_per_node"})
    dominant = mm if mm_ms >= tri_ms else tri
    return dominant, {"metamesh": mm, f"triangulation_k{k_big}": tri}


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
    if not args.no_pool_retain:
        # builds of the same size reuse the pool's mapped memory from step to
        # step (as a service that rebuilds meta-meshes would configure it)
        liblm.lm_pool_retain((1 << 64) - 1)
    wl = WORKLOADS[args.workload]
    ks = wl["ks"]
    xyz, ends, radii = make_lattice_device(wl, dev, torch)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    N, E = int(xyz.shape[0]), int(ends.shape[0])
    vhist = valence_hist(torch, ends, N)
    # output buffer sized for the larger k (this first build also runs the
    # launch-shape autotuner; later builds reuse its choice)
    mm = liblm.MetaMesh(xyz, ends, radii, options=tuned_options(liblm), stream=stream)
    totals = [mm.tri_count(k, stream) for k in ks]
    counts = mm.counts()
    launch_shape = liblm.lm_metamesh_launch_shape(mm.h)
    twice = liblm.lm_metamesh_emit_nodes(mm.h)
    fb = liblm.lm_fp64_counts(mm.h)
    fp64 = dict(zip(["pair", "candidate", "position_refine", "dedup", "seam", "loop_angle", "label",
                     "arc_extent", "tri_segments", "tri_start_angle", "tri_stitch_order", "tri_fan_centre"],
                    fb[:12]))
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
    with Clocks(local) as clk:
        l0 = liblm.lm_launch_count()
        start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        start.record(stream)
        for s in range(args.steps):
            run_step(torch, liblm, xyz, ends, radii, ks, out, stream, want_times=False)
        stop.record(stream)
        torch.cuda.synchronize()
        l1 = liblm.lm_launch_count()
    ms = max_over_ranks(torch, start.elapsed_time(stop) / args.steps, dev)
    # per-phase times of one extra step (not part of the timed region)
    _, _, phase = run_step(torch, liblm, xyz, ends, radii, ks, out, stream, want_times=True)
    value = job_value(world, E, ms)
    peaks, peak_kind = load_peaks()
    roof, roofs = rooflines(wl, ks, totals, phase, counts, vhist, N, E, peaks, peak_kind)
    del out
    torch.cuda.empty_cache()
    e2e = bench_e2e(torch, liblm, xyz, ends, radii, ks, stream, dev, args) if not args.no_e2e else None
    del xyz, ends, radii
    torch.cuda.empty_cache()
    adjoint = bench_adjoint(torch, liblm, dev, stream) if not args.no_adjoint else None
    extras = {}
    if world == 1 and not args.no_extras:
        if args.workload != "octet100":
            extras["octet100"] = bench_other(torch, liblm, dev, stream, "octet100")
        extras["irregular2m"] = bench_irregular(torch, liblm, dev, stream)
        extras["stl_file"] = bench_stl_file(torch, liblm, dev, stream)
        extras["ablation_warp_vs_thread"] = bench_ablation(torch, liblm, dev, stream)
    res = {
        "metric": METRIC,
        "value": value, "unit": "struts/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 (f64 stability steps)", "data": "synthetic",
        "config": {"workload": wl["desc"], "name": args.workload, "n_nodes": N,
                   "n_struts": E, "ks": list(ks), "triangles": dict(zip([f"k{k}" for k in ks], totals)),
                   "l2": "inputs (and outputs) larger than L2", "parallelism": f"replicas x{world}"},
        "phases_ms": phase,
        "metamesh_struts_per_s": E / (phase["metamesh_ms"] / 1e3),
        "triangles_per_s": {f"k{k}": totals[i] / (phase[f"tri_k{k}_ms"] / 1e3) for i, k in enumerate(ks)},
        "write_gbs": {f"k{k}": 50.0 * totals[i] / (phase[f"tri_k{k}_ms"] / 1e3) / 1e9 for i, k in enumerate(ks)},
        "meta_mesh_counts": {"vertices": counts[0], "elliptical_arcs": counts[1], "circular_arcs": counts[2],
                             "holes": counts[3], "degenerate_nodes": counts[5], "max_valence": counts[6]},
        "valence_histogram": {str(d): c for d, c in sorted(vhist.items())},
        "fp64_stability_steps": fp64,
        "metamesh_launch_shape": {"buckets": ["d<=16", "d<=32", "d<=64"],
                                  "warps_per_block_nodes_per_pop": launch_shape, "autotuned": True,
                                  "nodes_computed_twice": twice},
        "roofline": roof,
        "rooflines": roofs,
        "gpu_launches": int((l1 - l0) // max(1, args.steps)) * args.steps,
        "clocks": clk.summary(),
        "e2e": e2e,
        "adjoint": adjoint,
    }
    res.update(extras)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        res["cpu_baseline"] = cpu_baseline(args)
    if rank == 0:
        print(json.dumps(res))
    if world > 1:
        torch.distributed.destroy_process_group()


def bench_other(torch, liblm, dev, stream, name, steps=3):
    """Device-resident step rate of another workload (a few steps after one
    warm-up), with its triangulation roofline."""
    wl = WORKLOADS[name]
    ks = wl["ks"]
    xyz, ends, radii = make_lattice_device(wl, dev, torch)
    mm = liblm.MetaMesh(xyz, ends, radii, options=tuned_options(liblm), stream=stream)
    totals = [mm.tri_count(k, stream) for k in ks]
    counts = mm.counts()
    mm.close()
    out = torch.empty(max(totals) * 50, dtype=torch.uint8, device=dev)
    run_step(torch, liblm, xyz, ends, radii, ks, out, stream)
    ph = []
    for _ in range(steps):
        ph.append(run_step(torch, liblm, xyz, ends, radii, ks, out, stream, want_times=True)[2])
    phase = {key: statistics.median(p[key] for p in ph) for key in ph[0]}
    N, E = int(xyz.shape[0]), int(ends.shape[0])
    vhist = valence_hist(torch, ends, N)
    peaks, peak_kind = load_peaks()
    _, roofs = rooflines(wl, ks, totals, phase, counts, vhist, N, E, peaks, peak_kind)
    step_ms = phase["metamesh_ms"] + sum(phase[f"count_k{k}_ms"] + phase[f"tri_k{k}_ms"] for k in ks)
    del out, xyz, ends, radii
    torch.cuda.empty_cache()
    return {"workload": wl["desc"], "n_struts": E, "ms_per_step": step_ms, "struts_per_s": E / (step_ms / 1e3),
            "phases_ms": phase, "metamesh_struts_per_s": E / (phase["metamesh_ms"] / 1e3),
            "triangles": dict(zip([f"k{k}" for k in ks], totals)),
            "write_gbs": {f"k{k}": 50.0 * totals[i] / (phase[f"tri_k{k}_ms"] / 1e3) / 1e9 for i, k in enumerate(ks)},
            "rooflines": roofs, "timing": f"median of {steps} device-resident steps (CUDA events)"}


def bench_irregular(torch, liblm, dev, stream, k=16, reps=3):
    """The irregular configuration: 2e6 uniform nodes, kNN k_v ~ U{4..16}
    symmetrised, lognormal radii (median 0.3 x mean strut length), FP32;
    persistent autotuned meta-mesh launch, triangulated at k = 16."""
    from paper_2405_15197_gb300 import lattices as L
    t0 = time.perf_counter()
    lat = L.irregular(2_000_000, r_scale=0.3)
    gen_s = time.perf_counter() - t0
    xyz = torch.tensor(lat["xyz"], dtype=torch.float32, device=dev)
    ends = torch.tensor(lat["ends"], dtype=torch.int32, device=dev)
    radii = torch.tensor(lat["radii"], dtype=torch.float32, device=dev)
    N, E = int(xyz.shape[0]), int(ends.shape[0])
    vhist = valence_hist(torch, ends, N)
    mm = liblm.MetaMesh(xyz, ends, radii, options=tuned_options(liblm), stream=stream)
    shape = liblm.lm_metamesh_launch_shape(mm.h)
    mm.close()
    bt, et, ct, ntri, counts, flags = [], [], [], 0, None, None
    for r in range(reps):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record(stream)
        mm = liblm.MetaMesh(xyz, ends, radii, options=tuned_options(liblm), stream=stream)
        ev[1].record(stream)
        ntri = mm.tri_count(k, stream)
        ev[2].record(stream)
        out = torch.empty((max(ntri, 1), 50), dtype=torch.uint8, device=dev)
        liblm.lm_triangulate(mm.h, k, 0, E + N, out.data_ptr(), ntri, stream)
        ev[3].record(stream)
        if liblm.lm_last_error(mm.h, stream):
            raise RuntimeError("device error in the irregular triangulation")
        torch.cuda.synchronize()
        bt.append(ev[0].elapsed_time(ev[1]))
        ct.append(ev[1].elapsed_time(ev[2]))
        et.append(ev[2].elapsed_time(ev[3]))
        if r == reps - 1:
            counts = mm.counts()
            v = liblm.lm_metamesh_export(mm.h)
            flags = liblm.lm_copy_to_host(v.node_flags, 4 * N, np.uint32)
            fb = liblm.lm_fp64_counts(mm.h)
        del out
        mm.close()
    torch.cuda.empty_cache()
    b_ms, e_ms = statistics.median(bt), statistics.median(et)
    return {"workload": "irregular: 2e6 uniform nodes in the unit cube, kNN k_v ~ U{4..16} symmetrised, "
                        "radii lognormal(ln 0.3 mean strut length, 0.25) clipped to 0.45 x shortest strut, FP32, k=16",
            "n_nodes": N, "n_struts": E, "generation_s": gen_s,
            "valence_histogram": {str(d): c for d, c in sorted(vhist.items())},
            "metamesh_ms": b_ms, "metamesh_struts_per_s": E / (b_ms / 1e3),
            "count_k16_ms": statistics.median(ct), "tri_k16_ms": e_ms, "triangles_k16": ntri,
            "triangles_per_s": ntri / (e_ms / 1e3), "write_gbs": 50.0 * ntri / (e_ms / 1e3) / 1e9,
            "degenerate_fraction": float(np.mean((flags & 2) != 0)),
            "near_tangent_fraction": float(np.mean((flags & 1) != 0)),
            "meta_mesh_counts": counts[:6], "fp64_stability_steps": fb,
            "metamesh_launch_shape": {"buckets": ["d<=16", "d<=32", "d<=64"],
                                      "warps_per_block_nodes_per_pop": shape, "autotuned": True},
            "timing": f"median of {reps} (CUDA events)"}


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

    phases = {}

    def one():
        t_a = time.perf_counter()
        dx = hx.to(dev, non_blocking=True)
        de = he.to(dev, non_blocking=True)
        dr = hr.to(dev, non_blocking=True)
        mm = liblm.MetaMesh(dx, de, dr, options=tuned_options(liblm), stream=stream)
        torch.cuda.synchronize()
        phases["h2d_and_build_s"] = time.perf_counter() - t_a
        tot = 0
        for k in ks:
            t_k = time.perf_counter()
            mm.tri_count(k, stream)
            # ~(slot / 50 / 80) items per chunk keeps a chunk inside one slot
            per_item = max(1.0, mm_tris[k] / (mm.n_struts + mm.n_nodes))
            chunk = int(0.8 * slot / 50 / (4 * per_item))
            n = liblm.lm_triangulate_stream(mm.h, k, chunk, ring.data_ptr(), slot, n_slots, None, stream)
            torch.cuda.synchronize()
            phases[f"count_and_stream_k{k}_s"] = time.perf_counter() - t_k
            phases[f"d2h_gbs_k{k}"] = 50.0 * n / phases[f"count_and_stream_k{k}_s"] / 1e9
            tot += n
        mm.close()
        return tot

    E = ends.shape[0]
    steps = 1 if E > 100_000_000 else max(1, min(args.steps, 3))
    # the whole-lattice path (the headline): build once, then stream each k
    one()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        tot = one()
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / steps
    # the chunked path (memory bounded by the chunk): the lattice meta-meshed
    # in ten strut chunks with their halo struts, each chunk's triangles
    # streamed while the next chunk builds
    build_struts = max(1, -(-E // 10))

    def one_chunked():
        dx = hx.to(dev, non_blocking=True)
        de = he.to(dev, non_blocking=True)
        dr = hr.to(dev, non_blocking=True)
        tris = liblm.lm_stream_chunked(dx, de, dr, ks, build_struts, ring.data_ptr(), slot, n_slots, None,
                                       tuned_options(liblm), stream)
        torch.cuda.synchronize()
        return sum(tris)

    one_chunked()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        tot_c = one_chunked()
    torch.cuda.synchronize()
    dt_chunked = (time.perf_counter() - t0) / steps
    assert tot_c == tot, (tot_c, tot)
    # the device-to-host bandwidth this link gives large copies into the
    # (already written) pinned ring: best of several 4 x 1 GiB copies, timed
    # with CUDA events on the stream (the bound of the streaming phases)
    probe_d = torch.empty(slot, dtype=torch.uint8, device=dev)
    probe_d.fill_(1)
    c2c = 0.0
    for _ in range(4):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for q in range(n_slots):
            ring[q * slot:(q + 1) * slot].copy_(probe_d, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        c2c = max(c2c, n_slots * slot / (e0.elapsed_time(e1) / 1e3) / 1e9)
    del probe_d
    return {"value": E / dt, "unit": "struts/s", "ms_per_step": dt * 1e3, "phases": phases,
            "path": "pinned host lattice -> lm_build_metamesh -> lm_triangulate_stream per k (pinned ring)",
            "chunked": {"ms_per_step": dt_chunked * 1e3, "value": E / dt_chunked,
                        "path": "pinned host lattice -> lm_stream_chunked (ten strut chunks with their halo "
                                "struts, the next chunk built while the current one streams) -> pinned ring"},
            "h2d_bytes_per_step": int(hx.numel() * hx.element_size() + he.numel() * he.element_size()
                                      + hr.numel() * hr.element_size()),
            "d2h_bytes_per_step": int(50 * tot), "steps": steps,
            "d2h_copy_gbs_measured": c2c,
            "d2h_bound_s": 50.0 * tot / (c2c * 1e9),
            "d2h_link_frac": {f"k{k}": phases[f"d2h_gbs_k{k}"] / c2c for k in ks}}


def bench_stl_file(torch, liblm, dev, stream, n=80, k=32):
    """Binary-STL file through the three-stage pipeline (GPU triangulation,
    device-to-host copy into a pinned ring, file writes by a host thread),
    synced to disk before the clock stops: BCC n^3 cells, R = 0.05, k."""
    wl = {"kind": "bcc", "n": n, "R": 0.05}
    xyz, ends, radii = make_lattice_device(wl, dev, torch)
    mm = liblm.MetaMesh(xyz, ends, radii, options=tuned_options(liblm), stream=stream)
    slot = 1 << 30
    ring = torch.empty(4 * slot, dtype=torch.uint8, pin_memory=True)
    d = tempfile.mkdtemp(prefix="lm_stl_")
    path = os.path.join(d, f"bcc{n}_k{k}.stl")
    try:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ntri, st = liblm.lm_triangulate_to_file(mm.h, k, path, ring.data_ptr(), slot, 4, sync=True, stream=stream)
        dt = time.perf_counter() - t0
        size = os.path.getsize(path)
    finally:
        if os.path.exists(path):
            os.remove(path)
        os.rmdir(d)
        mm.close()
    return {"workload": f"BCC {n}^3 cells, R=0.05, k={k}, binary STL to the local disk (fsync before the clock stops)",
            "triangles": ntri, "file_bytes": size, "seconds": dt, "file_gbs": size / dt / 1e9,
            "writer": st, "ring": "4 x 1 GiB pinned slots, chunks by Eq. chunk-size"}


def bench_ablation(torch, liblm, dev, stream, name="octet100", samples=32, reps=3):
    """Warp-centric vs thread-centric trimming (the paper's Section 6
    ablation): the envelope of Section 4.3.1 at `samples` angles of every
    strut end, in both work mappings, same arithmetic (lm_envelope_samples)."""
    wl = WORKLOADS[name]
    xyz, ends, radii = make_lattice_device(wl, dev, torch)
    mm = liblm.MetaMesh(xyz, ends, radii, options=tuned_options(liblm), stream=stream)
    n_ends = 2 * mm.n_struts
    t = torch.empty(n_ends * samples, dtype=torch.float32, device=dev)
    lab = torch.empty(n_ends * samples, dtype=torch.int16, device=dev)
    deg = torch.bincount(ends.reshape(-1).long(), minlength=mm.n_nodes).double()
    evals = float((deg * (deg - 1)).sum().item()) * samples  # h_j evaluations
    res = {}
    for mode, key in ((liblm.LM_ENV_WARP, "warp_centric"), (liblm.LM_ENV_THREAD, "thread_centric")):
        liblm.lm_envelope_samples(mm.h, samples, mode, t.data_ptr(), lab.data_ptr(), stream)
        ms = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            liblm.lm_envelope_samples(mm.h, samples, mode, t.data_ptr(), lab.data_ptr(), stream)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        m = statistics.median(ms)
        res[key] = {"ms": m, "h_evals_per_s": evals / (m / 1e3)}
    mm.close()
    return {"workload": f"{wl['desc']}: envelope t*(phi) = max(0, max_j h_j(phi)) at {samples} angles of each "
                        f"of {n_ends} strut ends (trimming, Section 4.3.1)",
            **res, "thread_over_warp": res["thread_centric"]["ms"] / res["warp_centric"]["ms"],
            "paper": "35x (warp-centric over thread-centric meta-meshing, RTX 3090, Section 6)"}


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


# ------------------------------------------------------------ CPU oracle timing
# The FP64 oracle runs unchanged; only the work is split across processes.
# Worker w of P takes struts [E w / P, E (w+1) / P), meta-meshes every node
# those struts touch (nodes on a range boundary are meta-meshed twice), and
# triangulates its struts and the hole fans of the nodes it owns (a node is
# owned by the worker holding its lowest-id strut).  Processes are spawned
# (never forked after CUDA initialisation) and start their timed region
# together at a barrier; the rate is all struts / the slowest worker's time.


def sample_lattice(spec):
    """Lattice of a CPU-timing spec: ('bcc', nx, ny, nz, R), ('octet', nx, ny,
    nz), ('bccjit', n) or ('npz', path).  FP32-rounded coordinates and radii
    (the GPU workloads are FP32)."""
    from paper_2405_15197_gb300 import lattices as L
    kind = spec[0]
    if kind == "bcc":
        lat = L.bcc(spec[1], spec[2], spec[3], radius=spec[4])
    elif kind == "bcc64":
        lat = L.bcc(spec[1], spec[1], spec[1], radius=spec[2])
    elif kind == "octet":
        lat = L.octet(0, ncells=(spec[1], spec[2], spec[3]))
    elif kind == "bccjit":
        lat = L.bcc(spec[1], jitter=0.05, radius_range=(0.05, 0.09))
    elif kind == "npz":
        d = np.load(spec[1])
        lat = {"xyz": d["xyz"], "ends": d["ends"], "radii": d["radii"]}
    else:
        raise ValueError(spec)
    if kind != "bcc64":
        lat = {k: (v.astype(np.float32).astype(np.float64) if k in ("xyz", "radii") else v)
               for k, v in lat.items() if k in ("xyz", "ends", "radii")}
    return lat


def _worker_items(lat, w, procs, nodes=None):
    """Struts (ranges), node-item runs and the nodes to meta-mesh of worker w.
    nodes: restrict the work to these nodes (struts whose lower-id end is in
    the set, hole fans of the set), else the whole lattice."""
    ends = lat["ends"]
    E, N = ends.shape[0], lat["xyz"].shape[0]
    if nodes is None:
        e0, e1 = E * w // procs, E * (w + 1) // procs
        first = np.full(N, E, dtype=np.int64)
        sid = np.arange(E, dtype=np.int64)
        np.minimum.at(first, ends[:, 0], sid)
        np.minimum.at(first, ends[:, 1], sid)
        owned = np.nonzero((first >= e0) & (first < e1))[0]
        strut_runs = [(e0, e1)] if e1 > e0 else []
        need = np.unique(ends[e0:e1].ravel())
    else:
        mine = np.sort(np.asarray(nodes))[w::procs]
        lo = np.minimum(ends[:, 0], ends[:, 1])
        sel = np.nonzero(np.isin(lo, mine))[0]
        cut = np.nonzero(np.diff(sel) != 1)[0] + 1
        strut_runs = [(int(r[0]), int(r[-1]) + 1) for r in np.split(sel, cut) if r.size]
        owned = mine
        need = np.unique(np.concatenate([ends[sel].ravel(), mine]))
    cut = np.nonzero(np.diff(owned) != 1)[0] + 1
    node_runs = [(E + int(r[0]), E + int(r[-1]) + 1) for r in np.split(owned, cut) if r.size]
    n_struts = sum(b - a for a, b in strut_runs)
    return strut_runs, node_runs, need, n_struts


def _oracle_worker(w, procs, inq, outq, barrier):
    import oracle
    cache = {}
    while True:
        job = inq.get()
        if job is None:
            return
        spec, ks, nodes_path = job
        key = (spec, nodes_path)
        if key not in cache:
            cache.clear()
            lat = sample_lattice(spec)
            nodes = np.load(nodes_path) if nodes_path else None
            cache[key] = (lat, _worker_items(lat, w, procs, nodes))
        lat, (sruns, nruns, need, n_struts) = cache[key]
        barrier.wait()
        t0 = time.perf_counter()
        o = oracle.Oracle(lat, nodes=[])
        o.metamesh_nodes(need)
        for k in ks:
            for a, b in sruns + nruns:
                o.triangulate(k, a, b, want_tris=False)
        dt = time.perf_counter() - t0
        del o
        outq.put((w, dt, n_struts))


class OraclePool:
    """`procs` spawned processes that time the oracle together."""

    def __init__(self, procs):
        import multiprocessing as mp
        import oracle
        oracle.build()
        ctx = mp.get_context("spawn")
        self.procs = procs
        self.barrier = ctx.Barrier(procs)
        self.outq = ctx.Queue()
        self.inqs = [ctx.Queue() for _ in range(procs)]
        self.ps = [ctx.Process(target=_oracle_worker, args=(w, procs, self.inqs[w], self.outq, self.barrier),
                               daemon=True) for w in range(procs)]
        for p in self.ps:
            p.start()

    def run(self, spec, ks, nodes_path=None):
        """(struts meta-meshed and triangulated, seconds of the slowest worker)."""
        import queue
        for q in self.inqs:
            q.put((spec, tuple(ks), nodes_path))
        res = []
        while len(res) < self.procs:
            try:
                res.append(self.outq.get(timeout=5))
            except queue.Empty:
                if not all(p.is_alive() for p in self.ps):
                    raise RuntimeError("an oracle worker process died")
        return sum(r[2] for r in res), max(r[1] for r in res)

    def close(self):
        for q in self.inqs:
            q.put(None)
        for p in self.ps:
            p.join(timeout=30)


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline(args, quick=False):
    """The FP64 oracle as it stands, on the machine's host cores: one core on a
    block of the workload and every core (one process each) on a larger
    block; for the billion-strut lattice the all-core time of its
    500x500x4-cell slab is also scaled by 125 (extrapolated)."""
    wl = WORKLOADS[args.workload]
    cores = host_cores()
    one_spec, all_spec = wl["cpu_one"], wl["cpu_all"]
    pool = OraclePool(1)
    e1, t1 = pool.run(one_spec, wl["ks"])
    pool.close()
    pool = OraclePool(cores)
    ea, ta = pool.run(all_spec, wl["ks"])
    pool.close()
    out = {"value": ea / ta, "unit": "struts/s", "cores": cores, "kind": "oracle",
           "sample": f"{_spec_desc(all_spec)} ({ea} struts) on {cores} processes, meta-mesh + "
                     + " + ".join(f"k={k}" for k in wl["ks"]),
           "seconds": ta,
           "one_core": {"value": e1 / t1, "unit": "struts/s", "cores": 1, "seconds": t1,
                        "sample": f"{_spec_desc(one_spec)} ({e1} struts)"},
           "nproc": cores}
    if wl.get("cpu_extrapolate"):
        f = wl["cpu_extrapolate"]
        out["extrapolated"] = {"factor": f, "seconds_all_cores": ta * f, "seconds_one_core": t1 * f * ea / e1,
                               "note": f"whole workload = the slab x {f} (extrapolated, not run)"}
    return out


def _spec_desc(spec):
    if spec[0] == "bcc":
        return f"BCC {spec[1]}x{spec[2]}x{spec[3]} cells, R={spec[4]}"
    if spec[0] == "octet":
        return f"octet-truss {spec[1]}x{spec[2]}x{spec[3]} cells"
    if spec[0] == "bccjit":
        return f"jittered BCC {spec[1]}^3 cells"
    if spec[0] == "bcc64":
        return f"BCC {spec[1]}^3 cells, R={spec[2]} (FP64)"
    return str(spec[0])


def bench_reference(args):
    """Reference arm: the FP64 oracle as it stands, on every host core (one
    spawned process each), each step a bounded sample of the workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = WORKLOADS[args.workload]
    cores = host_cores()
    spec = wl["cpu_ref"]
    pool = OraclePool(cores)
    try:
        for _ in range(args.warmup):
            pool.run(spec, wl["ks"])
        t_steps, n = [], 0
        for _ in range(args.steps):
            n, dt = pool.run(spec, wl["ks"])
            t_steps.append(dt)
    finally:
        pool.close()
    ms = 1e3 * statistics.mean(t_steps)
    value = n / (ms / 1e3)
    sample = f"{_spec_desc(spec)} ({n} struts) per step on {cores} processes, meta-mesh + " + \
        " + ".join(f"k={k}" for k in wl["ks"])
    res = {"impl": "reference", "metric": METRIC,
           "value": value, "unit": "struts/s", "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": wl["desc"], "name": args.workload},
           "cpu_baseline": {"value": value, "unit": "struts/s", "cores": cores, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": "struts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(res))


def cpu_configs(args):
    """The oracle on every host core over each configuration of the
    benchmark suite: BCC 10^3 (FP64, k=16), octet 100^3 (k=8, 32) and jittered
    BCC 64^3 (k=32) whole; the 2e6-node irregular lattice (k=16) on a
    1e5-node sub-cube and BCC 500^3 (k=8, 32) on its 500x500x4-cell slab,
    both scaled to the whole lattice (extrapolated).  Prints one JSON line."""
    from paper_2405_15197_gb300 import lattices as L
    cores = host_cores()
    pool = OraclePool(cores)
    out = {"cores": cores, "configs": {}}
    try:
        for name, spec, ks, factor in [("bcc10_fp64", ("bcc64", 10, 0.08), (16,), 1.0),
                                       ("octet100", ("octet", 100, 100, 100), (8, 32), 1.0),
                                       ("bccjit64", ("bccjit", 64), (32,), 1.0),
                                       ("bcc500_slab", ("bcc", 500, 500, 4, 0.05), (8, 32), 125.0)]:
            n, dt = pool.run(spec, ks)
            out["configs"][name] = {"struts": n, "seconds": dt, "struts_per_s": n / dt, "ks": list(ks),
                                    "whole_seconds": dt * factor, "extrapolated": factor != 1.0}
        lat = L.irregular(2_000_000, r_scale=0.3)
        lat = {k: (v.astype(np.float32).astype(np.float64) if k in ("xyz", "radii") else v)
               for k, v in lat.items() if k in ("xyz", "ends", "radii")}
        sub = np.nonzero(np.all(lat["xyz"] < 0.368, axis=1))[0]
        with tempfile.TemporaryDirectory() as td:
            lp, npth = os.path.join(td, "irr.npz"), os.path.join(td, "sub.npy")
            np.savez(lp, **lat)
            np.save(npth, sub)
            n, dt = pool.run(("npz", lp), (16,), npth)
        f = lat["xyz"].shape[0] / sub.size
        out["configs"]["irregular2m_subcube"] = {"struts": n, "nodes": int(sub.size), "seconds": dt,
                                                 "struts_per_s": n / dt, "ks": [16], "whole_seconds": dt * f,
                                                 "extrapolated": True}
    finally:
        pool.close()
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="bcc500", choices=sorted(WORKLOADS))
    ap.add_argument("--cpu-configs", action="store_true",
                    help="time the oracle on every configuration (all host cores) and exit")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-pool-retain", action="store_true",
                    help="let the memory pool give freed memory back at every synchronisation")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the octet 100^3 and irregular 2e6-node lines")
    args = ap.parse_args()
    if args.cpu_configs:
        cpu_configs(args)
    elif args.impl == "reference":
        bench_reference(args)
    else:
        bench_gpu(args)


if __name__ == "__main__":
    main()
