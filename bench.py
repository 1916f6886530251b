#!/usr/bin/env python
"""Benchmark of the Voronoi-cell hot path on GB300.

One step = the whole path over one synthetic point set: vt_build (Morton key,
radix sort, gather, bucket tree, clipping with the security-radius test and
exact fallback, facet emission), vt_cells (volumes and the neighbour CSR),
vt_density, vt_gradient, vt_grid_density (256^3) and vt_backward.

Workload (default): 16,777,216 FP32 points, the clustered generator (60 % in
2000 NFW halos, 25 % on filaments, 15 % uniform), seed 2, periodic box of side
200; FP32-filtered clipping.  Inputs (201 MB) and every workspace exceed the
129 MB L2, so no flush is needed between steps.

Prints one JSON line.  ``value`` is cells/s of the full step with inputs
resident on the device; ``e2e`` the same through the C ABI with the positions
copied from pinned host memory and every output copied back inside the timed
region; ``roofline`` is the clipping kernel (the dominant one) against the
FP32 issue peak; ``cpu_baseline`` the FP64 oracle on a bounded sample.
``--impl reference`` times the oracle alone (the reference arm).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Voronoi cells/sec (fwd, bwd) at 16.7M clustered pts on 1 GB300; roofline fraction"
UNIT = "cells/s"

# Algorithmic work of one cell, from the oracle on a 2048-cell sample of each workload (seed 7; the table is
# the output of tests/work_per_cell.py):
# W = n_cert * V * 6 + V * 40 + F * 30 flops with n_cert the sites examined before the security stop (every
# one must be tested against the cell's vertices, 3 FMA each), V the vertices (a vertex from three planes costs
# about 40 flops) and F the facets of the final cell (about 30 flops each for area, centroid and volume).
WORK = {
    "uniform4096": {"n_cert": 42.75, "verts": 27.05, "faces": 15.53},
    "clustered64k": {"n_cert": 177.45, "verts": 26.50, "faces": 15.25},
    "clustered2M": {"n_cert": 213.01, "verts": 26.64, "faces": 15.32},
    "clustered16M": {"n_cert": 163.17, "verts": 26.74, "faces": 15.37},
    "halosets4096": {"n_cert": 147.19, "verts": 26.55, "faces": 15.27},
}
# DRAM bytes (read + write) of one launch of the clipping kernel: dram__bytes_read.sum + dram__bytes_write.sum of
# one launch on the 2,097,152-point clustered set (543 B per cell, profiles/k_clip_clustered2M_dram.md) times the
# cells of the launch (the facet records that dominate it grow with the cells)
CLIP_TRAFFIC_PER_CELL = {"filter32": 543.3}
CLIP_TRAFFIC = {("clustered16M", "filter32"): CLIP_TRAFFIC_PER_CELL["filter32"] * 16777216,
                ("clustered2M", "filter32"): CLIP_TRAFFIC_PER_CELL["filter32"] * 2097152}
# FMA lanes per SM of the GB300 (sm_103): 128 FP32; the FP64 rate is 1/64 of it (2 FP64 FMA per clock per SM)
FP32_LANES_PER_SM = 128
FP64_LANES_PER_SM = 2


def flops_per_cell(w):
    return w["n_cert"] * w["verts"] * 6 + w["verts"] * 40 + w["faces"] * 30


def _inputs_tag():
    """Short hash of the generator module: a cached point set is reused only while its generator is unchanged."""
    import hashlib

    from paper_1601_06429_gb300 import inputs

    with open(inputs.__file__, "rb") as f:
        return hashlib.sha1(f.read()).hexdigest()[:10]


def workload(name):
    from paper_1601_06429_gb300 import inputs

    cache = os.path.join(tempfile.gettempdir(), "vt_bench_%s_%s.npy" % (name, _inputs_tag()))
    if name == "clustered16M":
        L = 200.0
        gen = lambda: inputs.clustered(16777216, L=L, seed=2)  # noqa: E731
        desc = dict(workload="clustered 16,777,216 FP32 points, periodic box L=200, seed 2", N=16777216, L=L,
                    grid=256)
    elif name == "clustered2M":
        L = 100.0
        gen = lambda: inputs.clustered(2097152, L=L, seed=1)  # noqa: E731
        desc = dict(workload="clustered 2,097,152 FP32 points, periodic box L=100, seed 1", N=2097152, L=L, grid=256)
    elif name == "clustered64k":
        L = float(np.float32(100.0 * (65536 / 2097152) ** (1.0 / 3.0)))
        gen = lambda: inputs.clustered(65536, L=L, seed=1)  # noqa: E731
        desc = dict(workload="clustered 65,536 FP32 points (the 2M recipe scaled), periodic box L=%.4f, seed 1" % L,
                    N=65536, L=L, grid=64)
    elif name == "halosets4096":
        x, off = _cached(cache, lambda: inputs.halo_sets())
        desc = dict(workload="4096 independent NFW halos (c ~ U(5,15), r_vir = 1), sizes log-uniform in "
                             "[64, 65536], %d FP32 points in all, each set in its own bounded box [-1,1]^3, seed 6"
                             % len(x), N=len(x), L=2.0, grid=0, set_off=off)
        return x, desc
    elif name == "uniform4096":
        L = 1.0
        gen = lambda: inputs.uniform(4096, seed=0, dtype=np.float32)  # noqa: E731
        desc = dict(workload="uniform 4096 FP32 points, unit periodic box, seed 0", N=4096, L=L, grid=32)
    else:
        raise SystemExit("unknown workload " + name)
    if os.path.exists(cache):
        x = np.load(cache)
    else:
        x = gen()
        try:
            np.save(cache + ".tmp.npy", x)
            os.replace(cache + ".tmp.npy", cache)
        except OSError:
            pass
    return x, desc


def _cached(cache, gen):
    """(points, set offsets) from the cache files, else generated and cached."""
    cache_off = cache[:-4] + "_off.npy"
    if os.path.exists(cache) and os.path.exists(cache_off):
        return np.load(cache), np.load(cache_off)
    x, off = gen()
    try:
        np.save(cache + ".tmp.npy", x)
        np.save(cache_off + ".tmp.npy", off)
        os.replace(cache + ".tmp.npy", cache)
        os.replace(cache_off + ".tmp.npy", cache_off)
    except OSError:
        pass
    return x, off


class Clocks:
    """Samples nvidia-smi every 200 ms while active."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        return self.summarise(self.lines)

    @staticmethod
    def summarise(lines):
        """Median SM clock, the largest maximum clock and the throttle reasons seen Active, from nvidia-smi's
        csv lines (fields in the order of Q)."""
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in lines:
            f = [v.strip() for v in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for k, n in enumerate(names):
                if f[5 + k].strip() == "Active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(v, ws, device=None):
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist

    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _measured(key, default):
    """A field of MEASURED_PEAKS.json (measured on the same kind of GPU), else ``default``."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)[key])
    except (OSError, ValueError, KeyError, TypeError):
        return default


def alu_peaks(sm_count, sm_max_mhz):
    """Derived FMA-issue peaks (TFLOP/s) from the unit counts and the maximum SM clock: (FP32, FP64)."""
    f = sm_count * 2 * sm_max_mhz * 1e6 / 1e12
    return f * FP32_LANES_PER_SM, f * FP64_LANES_PER_SM


def _hbm_gbs(default=6688.8):
    """Measured copy bandwidth of the GB300 in GB/s: MEASURED_PEAKS.json's hbm_gbs when the file is present
    (a STREAM-style copy timed on the same kind of GPU), else the value last measured there."""
    return _measured("hbm_gbs", default)


HBM_GBS = _hbm_gbs()


def step_roofline(N, G, faces, fpc, peak_tflops, t_ms):
    """Time-based roofline of the whole step: per stage max(bytes / HBM bandwidth, flops / ALU peak), summed,
    against the measured time (the forward, grid and backward events).  Bytes per cell, algorithmic:
    key 24, radix sort 6 passes x 32, gather 40, clipping (facet records 32 B each, cell record 24, position 16),
    neighbour CSR 36 per facet + 8, density 40, gradient 40 per facet + 12, backward 36 per facet + 12; the grid
    writes 4 B per node.  Only the clipping stage has a flop count; every other stage is bound by its bytes."""
    clip_bytes = 32 * faces + 24 + 16
    per_cell = 24 + 6 * 32 + 40 + clip_bytes + (36 * faces + 8) + 40 + (40 * faces + 12) + (36 * faces + 12)
    to_ms = 1e3 / (HBM_GBS * 1e9)
    t_hbm = (per_cell * N + 4.0 * G ** 3) * to_ms
    t_clip_hbm = clip_bytes * N * to_ms
    t_alu = fpc * N / (peak_tflops * 1e12) * 1e3
    t_roof = (t_hbm - t_clip_hbm) + max(t_clip_hbm, t_alu)
    return {"t_roof_ms": t_roof, "t_hbm_ms": t_hbm, "t_clip_hbm_ms": t_clip_hbm, "t_clip_alu_ms": t_alu,
            "t_measured_ms": t_ms, "frac": t_roof / t_ms, "bytes_per_cell": per_cell, "hbm_gbs": HBM_GBS}


class OracleTimer:
    """The FP64 oracle (certified mode, all host cores) on random samples of cells of one workload.  The k-d tree
    over every point is built once, outside the timed region, and its build time is reported beside the rate;
    each sample is then timed alone, so the rate is cells per second of cell work."""

    def __init__(self, x, desc):
        import oracle

        oracle.build()
        self.N = len(x)
        self.off = desc.get("set_off")
        t0 = time.perf_counter()
        if self.off is None:
            self.trees = [oracle.Tree(x.astype(np.float64), 0.0, desc["L"], True)]
        else:
            # bounded sets: one tree per set, each in its box [-1,1]^3
            self.trees = [oracle.Tree(x[self.off[s]:self.off[s + 1]].astype(np.float64), -1.0, 1.0, False)
                          for s in range(len(self.off) - 1)]
        self.tree_seconds = time.perf_counter() - t0

    def rate(self, n_sample, seed):
        """(cells/s, info) on n_sample random cells."""
        pick = np.sort(np.random.default_rng(seed).choice(self.N, n_sample, replace=False))
        t0 = time.perf_counter()
        if self.off is None:
            self.trees[0].cells(pick)
        else:
            sid = np.searchsorted(self.off, pick, side="right") - 1
            for s in np.unique(sid):
                self.trees[s].cells(pick[sid == s] - self.off[s])
        dt = time.perf_counter() - t0
        what = ("%d random cells of the same point set, certified mode, FP64; the k-d tree over all %d points "
                "(%.1f s, built once outside the timed region) is not in the rate" % (n_sample, self.N,
                                                                                        self.tree_seconds))
        if self.off is not None:
            what = what.replace("the k-d tree over all", "the k-d trees of all sets over")
        return n_sample / dt, dict(cores=os.cpu_count(), seconds=dt, tree_seconds=self.tree_seconds, sample=what)


def parity_report(x, L, tree, out, flags, n_sample=2048, n_grad=256, seed=21):
    """Per-particle errors of one step's outputs against the FP64 oracle (certified mode, on the kept tree) on
    n_sample random cells plus every cell the exact kernel finished (and up to 256 that needed FP64 decisions):
    the largest relative volume and density errors, neighbour lists that differ, and for n_grad of the cells
    (whose neighbours' oracle cells are computed too) the least-squares gradient error
    |dg| / max(|g_ref|, 1e-3 rho / l), l = V^(1/3), and |dg| / (rho / l) alone.  ``out``: numpy vol, dens, grad,
    off, ids in input order; ``flags``: vt_cell_flags."""
    import oracle

    N = len(x)
    rng = np.random.default_rng(seed)
    exact = np.nonzero(flags & 2)[0]
    fp64 = np.nonzero(flags & 1)[0]
    fp64 = rng.choice(fp64, min(256, len(fp64)), replace=False) if len(fp64) else fp64
    which = np.unique(np.concatenate([rng.choice(N, n_sample, replace=False), exact, fp64])).astype(np.int64)
    o = tree.cells(which)
    vr = np.abs(out["vol"][which] - o["vol"]) / o["vol"]
    dr = np.abs(out["dens"][which] - 1.0 / o["vol"]) * o["vol"]
    ooff, oids = oracle.neighbours(o)
    bad = sum(not np.array_equal(out["ids"][out["off"][i]:out["off"][i + 1]], oids[ooff[k]:ooff[k + 1]])
              for k, i in enumerate(which))
    gw = np.sort(rng.choice(which, min(n_grad, len(which)), replace=False))
    nb = np.unique(np.concatenate([out["ids"][out["off"][i]:out["off"][i + 1]] for i in gw] + [gw]))
    on = tree.cells(nb)
    dens_all = np.zeros(N)
    dens_all[nb] = 1.0 / on["vol"]
    og = tree.cells(gw)
    noff, nids, disp = oracle.neighbour_displacements(og, x.astype(np.float64), 0.0, L)
    g_ref = oracle.gradient(dens_all[gw], noff, nids, disp, dens_all)
    rho, ell = 1.0 / og["vol"], og["vol"] ** (1.0 / 3.0)
    dg = np.linalg.norm(out["grad"][gw] - g_ref, axis=1)
    return {"cells": int(len(which)), "exact_cells": int(len(exact)), "fp64_cells_in_sample": int(len(fp64)),
            "vol_max_rel": float(vr.max()), "vol_p99_rel": float(np.quantile(vr, 0.99)),
            "dens_max_rel": float(dr.max()), "nbr_lists_different": int(bad), "grad_cells": int(len(gw)),
            "grad_max_err_floor_1e-3": float((dg / np.maximum(np.linalg.norm(g_ref, axis=1), 1e-3 * rho / ell)).max()),
            "grad_max_abs_over_rho_per_l": float((dg / (rho / ell)).max())}


def workload_config(desc, ws):
    """The workload keys both arms report in ``config``."""
    G = desc.get("grid", 0)
    return {"workload": desc["workload"], "grid": "%d^3" % G if G else "none (no single box)",
            "parallelism": "replicas" if ws > 1 else "1 GPU"}


def run_reference(args):
    ws, rank, local = dist_setup(args)
    if rank != 0:
        return 0
    x, desc = workload(args.workload)
    timer = OracleTimer(x, desc)
    rates = []
    info = None
    for k in range(args.warmup + args.steps):
        r, info = timer.rate(args.cpu_sample, seed=100 + k)
        if k >= args.warmup:
            rates.append(r)
    value = statistics.median(rates)
    N = desc["N"]
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            # one whole step would be every cell of the workload: extrapolated from the sampled per-cell rate,
            # plus the one tree build
            "ms_per_step": 1000.0 * (N / value + timer.tree_seconds),
            "ms_per_step_kind": "extrapolated: %d cells at the sampled rate + the k-d tree build (%.1f s); each timed "
                                "step ran %d cells" % (N, timer.tree_seconds, args.cpu_sample),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(workload_config(desc, ws), precision="fp64 oracle, exact predicates (certified mode)"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": info["cores"], "kind": "oracle",
                             "sample": info["sample"], "tree_seconds": timer.tree_seconds},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_ours(args):
    import torch

    from paper_1601_06429_gb300 import binding as vt
    from paper_1601_06429_gb300.build import build

    ws, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0:
        build()
    barrier(ws)
    vt.load_library()
    x, desc = workload(args.workload)
    N, L, G = desc["N"], desc["L"], desc["grid"]
    box = ((0.0,) * 3, (L,) * 3)
    set_off = desc.get("set_off")
    boxes = None if set_off is None else np.tile([-1.0, -1.0, -1.0, 1.0, 1.0, 1.0], (len(set_off) - 1, 1))
    set_k = set_tpc = None
    tuned = None
    if set_off is not None and not args.no_autotune:
        # per size class: k_target and threads per cell from timed trial builds (untimed here)
        t0 = time.perf_counter()
        set_k, set_tpc = vt.vt_autotune_batched(torch.from_numpy(x).to(dev), set_off, boxes, precision=args.precision)
        sizes = np.diff(set_off)
        cls = np.floor(np.log2(np.maximum(sizes, 1))).astype(int)
        tuned = {"seconds": time.perf_counter() - t0,
                 "per_size_class": {"%d..%d" % (2 ** cc, 2 ** (cc + 1) - 1):
                                    {"k_target": int(set_k[cls == cc][0]), "threads_per_cell": int(set_tpc[cls == cc][0])}
                                    for cc in np.unique(cls)}}
    stream = torch.cuda.current_stream(dev)
    xd = torch.from_numpy(x).to(dev)
    w = torch.from_numpy(np.random.default_rng(4).random(N).astype(np.float32)).to(dev)  # dL/dV weights
    def outputs():
        """Device buffers of one step's outputs."""
        return dict(vol=torch.empty(N, dtype=torch.float32, device=dev),
                    dens=torch.empty(N, dtype=torch.float32, device=dev),
                    grad=torch.empty(N, 3, dtype=torch.float32, device=dev),
                    off=torch.empty(N + 1, dtype=torch.int64, device=dev),
                    ids=torch.empty(24 * N, dtype=torch.int32, device=dev),
                    grid=torch.empty(G, G, G, dtype=torch.float32, device=dev) if G else None,
                    dpos=torch.empty(N, 3, dtype=torch.float32, device=dev))

    out0 = outputs()
    stats = []
    marks = []  # per timed step: events after the forward (build, cells, density, gradient), grid, backward

    def step(pos_dev, mark=False, o=out0):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)] if mark else None
        if ev:
            ev[0].record(stream)
        if set_off is None:
            h = vt.vt_build(pos_dev, None, box[0], box[1], True, args.precision)
        else:
            h = vt.vt_build_batched(pos_dev, set_off, boxes, precision=args.precision, set_k=set_k, set_tpc=set_tpc)
        nnz = vt.vt_cells(h)
        if nnz > o["ids"].numel():
            o["ids"] = torch.empty(int(nnz * 1.2), dtype=torch.int32, device=dev)
        vt.vt_cells(h, o["vol"], o["off"], o["ids"])
        vt.vt_density(h, o["dens"])
        vt.vt_gradient(h, o["grad"])
        if ev:
            ev[1].record(stream)
        if G:
            vt.vt_grid_density(h, G, 1, o["grid"])
        if ev:
            ev[2].record(stream)
        vt.vt_backward(h, w, 0.0, o["dpos"])
        if ev:
            ev[3].record(stream)
            marks.append(ev)
        st = vt.vt_status(h)
        vt.vt_destroy(h)
        if st["rc"] != 0:
            raise RuntimeError("device error %d" % st["rc"])
        stats.append(st)
        return nnz

    # measured FMA throughput (reported beside the derived peaks)
    probe_tflops = vt.vt_probe_fp32_tflops() if args.precision == "filter32" else vt.vt_probe_fp64_tflops()
    # ---------------- device-resident inputs
    for _ in range(args.warmup):
        step(xd)
    stats.clear()
    torch.cuda.synchronize()
    barrier(ws)
    clk = Clocks(local)
    clk.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        nnz = step(xd, mark=True)
    e1.record(stream)
    torch.cuda.synchronize()
    t_ms = e0.elapsed_time(e1)
    clocks = clk.stop()
    barrier(ws)
    t_ms = max_over_ranks(t_ms, ws, dev)
    ms_step = t_ms / args.steps
    value = ws * N * args.steps / (t_ms / 1000.0)
    clip_ms = statistics.mean(s["t_clip_ms"] for s in stats)
    sort_ms = statistics.mean(s["t_sort_ms"] for s in stats)
    launches = sum(s["n_launches"] for s in stats)
    fwd_ms = statistics.mean(m[0].elapsed_time(m[1]) for m in marks)
    grid_ms = statistics.mean(m[1].elapsed_time(m[2]) for m in marks)
    bwd_ms = statistics.mean(m[2].elapsed_time(m[3]) for m in marks)

    # ---------------- the exact volume-averaged grid (an extra output, outside the timed step)
    grid_volume_ms = None
    if G and set_off is None:
        h = vt.vt_build(xd, None, box[0], box[1], True, args.precision)
        gv = torch.empty(G, G, G, dtype=torch.float32, device=dev)
        vt.vt_grid_density_volume(h, G, gv)  # first call allocates its accumulator
        torch.cuda.synchronize()
        g0 = torch.cuda.Event(enable_timing=True)
        g1 = torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        vt.vt_grid_density_volume(h, G, gv)
        g1.record(stream)
        torch.cuda.synchronize()
        grid_volume_ms = g0.elapsed_time(g1)
        if vt.vt_status(h)["n_grid_failed"]:
            raise RuntimeError("volume-averaged grid: parts not computed")
        vt.vt_destroy(h)
        del gv

    # ---------------- end to end through the ABI with host buffers
    # Every step's positions come from pinned host memory (H2D stream) and every output goes back to pinned host
    # memory (D2H stream).  Two sets of device buffers alternate: the next step's positions are copied in during
    # this step, and this step's outputs are copied out during the next one (the library reads its status words
    # through mapped memory, so its builds never wait behind these copies); events order each buffer's reuse.
    xh = torch.from_numpy(x).pin_memory()
    outs_h = dict(vol=torch.empty(N, dtype=torch.float32).pin_memory(),
                  dens=torch.empty(N, dtype=torch.float32).pin_memory(),
                  grad=torch.empty(N, 3, dtype=torch.float32).pin_memory(),
                  off=torch.empty(N + 1, dtype=torch.int64).pin_memory(),
                  grid=torch.empty(G, G, G, dtype=torch.float32).pin_memory() if G else None,
                  dpos=torch.empty(N, 3, dtype=torch.float32).pin_memory())
    ids_h = torch.empty(out0["ids"].numel(), dtype=torch.int32).pin_memory()
    bufs = [dict(x=torch.empty_like(xd), o=out0), dict(x=torch.empty_like(xd), o=outputs())]
    s_h2d = torch.cuda.Stream(device=dev)
    s_d2h = torch.cuda.Stream(device=dev)
    for b in bufs:
        b["in"] = torch.cuda.Event()      # positions on the device
        b["done"] = torch.cuda.Event()    # the step that used this buffer has computed its outputs
        b["copied"] = torch.cuda.Event()  # its outputs are back on the host
        b["done"].record(stream)
        b["copied"].record(stream)

    def copy_out(o, n):
        nonlocal ids_h
        if n > ids_h.numel():
            ids_h = torch.empty(int(n * 1.2), dtype=torch.int32).pin_memory()
        for k in ("vol", "dens", "grad", "off", "dpos") + (("grid",) if G else ()):
            outs_h[k].copy_(o[k], non_blocking=True)
        ids_h[:n].copy_(o["ids"][:n], non_blocking=True)

    def copy_in(b):
        with torch.cuda.stream(s_h2d):
            s_h2d.wait_event(b["done"])  # the step two back has read these positions
            b["x"].copy_(xh, non_blocking=True)
            b["in"].record(s_h2d)

    def e2e_step(k, prefetch):
        b = bufs[k % 2]
        if prefetch:
            copy_in(bufs[(k + 1) % 2])  # the next step's positions, during this step
        stream.wait_event(b["in"])
        stream.wait_event(b["copied"])  # the outputs two steps back are on the host
        n = step(b["x"], o=b["o"])
        b["done"].record(stream)
        with torch.cuda.stream(s_d2h):
            s_d2h.wait_event(b["done"])
            copy_out(b["o"], n)
            b["copied"].record(s_d2h)
        return n

    copy_in(bufs[0])
    n = e2e_step(0, False)
    torch.cuda.synchronize()
    barrier(ws)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s_h2d.wait_event(e0)
    copy_in(bufs[0])
    for k in range(args.steps):
        n = e2e_step(k, k + 1 < args.steps)
    stream.wait_stream(s_d2h)
    e1.record(stream)
    torch.cuda.synchronize()
    te_ms = max_over_ranks(e0.elapsed_time(e1), ws, dev)
    e2e_value = ws * N * args.steps / (te_ms / 1000.0)
    h2d = N * 12
    d2h = N * 4 + N * 4 + N * 12 + (N + 1) * 8 + G ** 3 * 4 + N * 12 + n * 4
    # the same copies alone, on one stream: the host<->device part of the e2e step
    e0.record(stream)
    for _ in range(args.steps):
        bufs[0]["x"].copy_(xh, non_blocking=True)
        copy_out(out0, n)
    e1.record(stream)
    torch.cuda.synchronize()
    copy_ms = e0.elapsed_time(e1) / args.steps

    # ---------------- roofline of the clipping kernel (FP32 issue bound)
    wk = WORK.get(args.workload, WORK["clustered16M"])
    fpc = flops_per_cell(wk)
    achieved = fpc * N / (clip_ms / 1000.0) / 1e12
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    peak_mhz = clocks.get("sm_max_mhz") or _measured("sm_max_mhz", 2070.0)
    peak32, peak64 = alu_peaks(sm_count, peak_mhz)
    peak = peak32 if args.precision == "filter32" else peak64

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if args.precision == "filter32" else "f64",
            "data": "synthetic",
            "config": dict(workload_config(desc, ws), precision=args.precision,
                           l2="inputs and workspaces larger than L2 (no flush)"),
            "fwd_bwd_breakdown_ms": {"build_sort_tree": sort_ms, "build_clip": clip_ms,
                                     "rest_of_step": ms_step - sort_ms - clip_ms,
                                     "forward": fwd_ms, "grid": grid_ms, "backward": bwd_ms},
            "fwd_cells_per_s": N / (fwd_ms / 1000.0), "bwd_cells_per_s": N / (bwd_ms / 1000.0),
            "grid_volume_ms": grid_volume_ms,
            "step_roofline": step_roofline(N, G, nnz / N, fpc, peak, fwd_ms + grid_ms + bwd_ms),
            "faces_per_cell": nnz / N,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "e2e_copies": {"ms_per_step": copy_ms, "gb_per_s": (h2d + d2h) / (copy_ms * 1e6),
                           "note": "the e2e step's copies alone, back to back (pinned host buffers, one stream)"},
            "gpu_launches": launches,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": CLIP_TRAFFIC.get((args.workload, args.precision)),
                         "kernel": "k_clip (clipping, security test, facet emission)",
                         "work": "%.0f algorithmic flops/cell x %d cells per launch" % (fpc, N),
                         "peak_note": "%s FMA issue: %d SMs x %d lanes x 2 flop x %.0f MHz (derived)"
                                      % ("FP32" if args.precision == "filter32" else "FP64", sm_count,
                                         FP32_LANES_PER_SM if args.precision == "filter32" else FP64_LANES_PER_SM,
                                         peak_mhz),
                         "peak_probe": probe_tflops,
                         "frac_of_probe": achieved / probe_tflops if probe_tflops > 0 else None},
            "clocks": clocks,
            "device_counters": {k: stats[-1][k] for k in ("n_cut", "n_tested", "n_passes", "n_fp64_fallbacks",
                                                          "n_exact_cells", "n_exact_preds", "n_exact_zero", "max_faces",
                                                          "n_handed_over", "n_bucket_passes")}}
    if tuned is not None:
        line["config"]["autotune"] = tuned
    if set_off is not None and not args.no_loop_baseline:
        line["per_set_loop"] = per_set_loop(vt, x, set_off, args.precision, dev, stream, N)
    if set_off is not None:
        line["graph_replay"] = graph_replay(vt, xd, set_off, boxes, set_k, set_tpc, args, dev, w)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        timer = OracleTimer(x, desc)
        r, info = timer.rate(args.cpu_sample, seed=11)
        line["cpu_baseline"] = {"value": r, "unit": UNIT, "cores": info["cores"], "kind": "oracle",
                                "sample": info["sample"], "tree_seconds": info["tree_seconds"]}
        if set_off is None and not args.no_parity:
            # per-output error against the oracle: the timed step's outputs, and the other precision's
            t0 = time.perf_counter()
            host = lambda t: t.double().cpu().numpy() if t.is_floating_point() else t.cpu().numpy()  # noqa: E731
            par = {}
            h = vt.vt_build(xd, None, box[0], box[1], True, args.precision)
            nnz_last = vt.vt_cells(h)
            out = dict(vol=host(out0["vol"]), dens=host(out0["dens"]), grad=host(out0["grad"]), off=host(out0["off"]),
                       ids=host(out0["ids"][:nnz_last]))
            par[args.precision] = parity_report(x, L, timer.trees[0], out, vt.cell_flags(h).cpu().numpy())
            vt.vt_destroy(h)
            other = "plain64" if args.precision == "filter32" else "filter32"
            h = vt.vt_build(xd, None, box[0], box[1], True, other)
            v2, o2, i2 = vt.cells(h)
            out = dict(vol=host(v2), dens=host(vt.density(h)), grad=host(vt.gradient(h)), off=host(o2), ids=host(i2))
            par[other] = parity_report(x, L, timer.trees[0], out, vt.cell_flags(h).cpu().numpy())
            st2 = vt.vt_status(h)
            par[other]["clip_ms"] = st2["t_clip_ms"]
            vt.vt_destroy(h)
            par["seconds"] = time.perf_counter() - t0
            line["parity"] = par
    if rank == 0:
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


def graph_replay(vt, xd, set_off, boxes, set_k, set_tpc, args, dev, w):
    """The batched step as one CUDA graph: a batched handle built once, then vt_rebuild (sort, tree, persistent
    clipping launch), vt_cells (volumes and CSR offsets), vt_density, vt_gradient and vt_backward captured and
    replayed on the resident positions; cells/s over args.steps replays (CUDA events)."""
    import torch

    N = xd.shape[0]
    s = torch.cuda.Stream(device=dev)
    vol = torch.empty(N, dtype=torch.float32, device=dev)
    off = torch.empty(N + 1, dtype=torch.int64, device=dev)
    dens = torch.empty(N, dtype=torch.float32, device=dev)
    grad = torch.empty(N, 3, dtype=torch.float32, device=dev)
    dpos = torch.empty(N, 3, dtype=torch.float32, device=dev)
    torch.cuda.synchronize(dev)
    with torch.cuda.stream(s):
        h = vt.vt_build_batched(xd, set_off, boxes, precision=args.precision, set_k=set_k, set_tpc=set_tpc, stream=s)
        vt.vt_rebuild(h, xd)
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        vt.vt_rebuild(h, xd)
        vt.vt_cells(h, vol, off, None, count=False)
        vt.vt_density(h, dens)
        vt.vt_gradient(h, grad)
        vt.vt_backward(h, w, 0.0, dpos)
    with torch.cuda.stream(s):
        for _ in range(args.warmup):
            g.replay()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    s.synchronize()
    e0.record(s)
    with torch.cuda.stream(s):
        for _ in range(args.steps):
            g.replay()
    e1.record(s)
    s.synchronize()
    st = vt.vt_status(h)
    vt.vt_destroy(h)
    if st["rc"] != 0:
        raise RuntimeError("device error %d in the graph replay" % st["rc"])
    t = e0.elapsed_time(e1) / args.steps
    return {"value": N / (t / 1000.0), "unit": UNIT, "ms_per_step": t,
            "what": "one CUDA graph per step: vt_rebuild + vt_cells (volumes, offsets) + vt_density + vt_gradient + "
                    "vt_backward on a batched handle built once"}


def per_set_loop(vt, x, set_off, precision, dev, stream, N):
    """The same batch as a host loop of one vt_build (and the same outputs) per set, timed once after one
    untimed pass; returns its cells/s."""
    import torch

    xd = torch.from_numpy(x).to(dev)
    w = torch.from_numpy(np.random.default_rng(4).random(N).astype(np.float32)).to(dev)
    vol = torch.empty(N, dtype=torch.float32, device=dev)
    dens = torch.empty(N, dtype=torch.float32, device=dev)
    grad = torch.empty(N, 3, dtype=torch.float32, device=dev)
    dpos = torch.empty(N, 3, dtype=torch.float32, device=dev)
    lo, hi = (-1.0,) * 3, (1.0,) * 3

    def one_pass():
        for s in range(len(set_off) - 1):
            a, b = int(set_off[s]), int(set_off[s + 1])
            if b == a:
                continue
            h = vt.vt_build(xd[a:b], None, lo, hi, False, precision)
            n = vt.vt_cells(h)
            off = torch.empty(b - a + 1, dtype=torch.int64, device=dev)
            ids = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
            vt.vt_cells(h, vol[a:b], off, ids)
            vt.vt_density(h, dens[a:b])
            vt.vt_gradient(h, grad[a:b])
            vt.vt_backward(h, w[a:b], 0.0, dpos[a:b])
            st = vt.vt_status(h)
            vt.vt_destroy(h)
            if st["rc"] != 0:
                raise RuntimeError("device error %d in set %d" % (st["rc"], s))

    one_pass()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    one_pass()
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1)
    return {"value": N / (t / 1000.0), "unit": UNIT, "ms": t,
            "what": "host loop of vt_build + vt_cells + vt_density + vt_gradient + vt_backward per set"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="clustered16M")
    ap.add_argument("--precision", choices=["filter32", "plain64"], default="filter32")
    ap.add_argument("--cpu-sample", type=int, default=16384,
                    help="oracle cells per timed sample, in cpu_baseline and in each step of --impl reference")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-parity", action="store_true", help="skip the per-output error report against the oracle")
    ap.add_argument("--no-loop-baseline", action="store_true", help="batched workloads: skip the per-set loop")
    ap.add_argument("--no-autotune", action="store_true", help="batched workloads: default k_target, one warp per cell")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    return run_reference(args) if args.impl == "reference" else run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
