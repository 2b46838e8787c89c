#!/usr/bin/env python
"""Benchmark of the reverse ray tracing hot path (Altay & Theuns,
arXiv:1304.4235) on the large log-normal box: 2^24 SPH particles (256^3)
sampling a log-normal density field (sigma_ln rho = 2.5, P(k) ~ k^-2.5, mean
n_H = 1e-5 cm^-3, T = 1e4 (rho/rho_mean)^0.6 K) in a periodic 8 Mpc box, h
from 32 neighbours, 12 HEALPix rays of 100 kpc per particle with periodic
wrapping, 400 frequency bins (nu^-1.5, 13.6-54.4 eV), FP32 columns and
spectral sum, FP64 equilibrium.

One step = one full solve of the hot path: BVH build, then the Sec. 4
iteration from x_thin to the paper's stopping test (max |dx|/x < 1e-3), each
sweep tracing every active particle's 12 rays (Eq. colden, FP32 columns),
folding them through the spectrum (Eq. gamma_shld) and updating x in FP64
(Eq. xroots).  Sweep 0's traversal also keeps every ray's segment list
where it fits in HBM, and later sweeps read their columns from the lists
(the box converges in two sweeps: one traversal and one product).  Metric:
rays/s and particle-updates/s, whole job.  Beside it (untimed by the step
count, CUDA events): wall time to x within rel 1e-3 of a tightly converged
x* for plain sweeps and for Newton-Krylov, the adjoint gradient with
recomputed and with stored segments, the 262144-particle halo, the
differentiation workload, the 128^3 box with helium, and the plain FP64
method on the 4096-particle lattice beside the oracle solving it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload c5|halo|c5_eighth|halo_65536] [--no-compare] [--no-cpu-baseline] [--no-e2e]

Under torchrun every rank solves its own copy (replicas; independent boxes
need no exchange) and rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "rays/s and particle-updates/s to converged x (rel 1e-3), Newton+adjoint vs plain"

# The benchmark workloads (seeded generators of workloads/): the large
# log-normal box (default) and the 262144-particle self-shielding halo.
WORKLOADS = {
    "c5": ("lognormal_box", dict(n_side=256, box_kpc=8000.0, sigma_ln=2.5, nside=1, F=400)),
    "halo": ("halo", dict()),
    # the same density field at 1/8 of the particles (profiling captures)
    "c5_eighth": ("lognormal_box", dict(n_side=128, box_kpc=4000.0, sigma_ln=2.5, nside=1, F=400)),
    # the halo at 1/4 of the particles (profiling captures of the stored-segment path)
    "halo_65536": ("halo", dict(n=65536)),
}

# Grid cell (kpc) of the oracle's uniform-grid search for each workload.
GRID_CELL = {"c5": 80.0, "halo": 4.0, "c5_eighth": 80.0, "halo_65536": 4.0}


def workload_name(key: str, w) -> str:
    if w.name == "lognormal_box":
        side = round(w.n ** (1 / 3))
        sig = WORKLOADS[key][1].get("sigma_ln", 2.0)
        return f"lognormal_{side}cube_sigma{sig:g}_L{w.box:g}kpc_nside{w.nside}_l{w.l_ray:g}kpc_F{w.F}"
    return f"halo_{w.n}_nside{w.nside}_l{w.l_ray:g}kpc_F{w.F}"


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per unit of work
# of a kernel from one ncu capture, keyed by the hash of the kernel's source
# files at capture time; a changed kernel reports traffic null.
#   k_trace: bytes per ray-sphere hit;  k_spmv: bytes per stored segment
MEASURED_TRAFFIC = {
    # the 256^3 box's own traversal (one-pass capture), which also stores the
    # segment lists: 34.2e9 + 180.7e9 DRAM bytes for 1.762e10 hits (captured
    # at source hash 7f3194b2267f46f1, which differs from this key's source
    # in one duplicated comment only)
    "k_trace": {"510ddac9de652e18": 12.20},
    # k_spmv8 on the 65536-particle halo (one-pass capture): 2.273e9 + 3.8e6
    # DRAM bytes for 3.23e8 padded segments, captured at source hash
    # 87756054aa5bee94; the files have since gained the chunk kernels and
    # trailing argument fields, the body of k_spmv8 is unchanged
    "k_spmv": {"92fdf220e9a3969d": 7.04},
}
KERNEL_SOURCES = {"k_trace": ("trace.cu", "common.cuh"), "k_spmv": ("linalg.cu", "linalg.cuh")}


def source_hash(kernel: str) -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_1304_4235_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=list(WORKLOADS), default="c5")
    ap.add_argument("--no-compare", action="store_true", help="skip the untimed convergence / adjoint runs")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU time of the oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--max-iter", type=int, default=4000, help="sweep / Newton-step limit of one solve")
    ap.add_argument("--cache-dir", default=os.path.join(ROOT, "_cache"), help="generated inputs")
    return ap.parse_args()


def load_workload(key: str, cache_dir: str):
    import workloads as W
    fn, kw = WORKLOADS[key]
    return W.cached(getattr(W, fn), cache_dir, **kw)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [v.strip() for v in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def combine_ranks(total_ms: float, counts, device=None):
    """Replicas: the job's time is the slowest rank's, its work the sum over
    ranks.  Returns (max total_ms, [summed counts]); a no-op without a
    process group."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return total_ms, list(counts)
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([float(v) for v in counts], dtype=torch.float64, device=device)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t.item()), [float(v) for v in c.tolist()]


class OracleSample:
    """The FP64 oracle (test infrastructure) on a bounded sample of the
    workload: its uniform-grid search (equal to the brute-force sums of Eq.
    colden to rounding order) built once, then one sweep -- columns of every
    ray, Gamma and the equilibrium x -- for seeded samples of origins sized to
    take about `seconds` of CPU time."""

    def __init__(self, w, cell: float):
        import oracle as O

        self.O, self.w = O, w
        e, J = w.spectrum()
        self.s, self.wts = O.spectrum(e, J, w.gamma_thin)
        self.dirs = O.healpix(w.nside)
        self.x0 = O.xeq(self.wts.sum(), w.nH, w.T, 0.0, False)
        t0 = time.perf_counter()
        self.grid = O.Grid(w, cell)
        self.build_s = time.perf_counter() - t0
        self.cell = cell
        self.count = 64

    def run(self, count: int, seed: int) -> float:
        import workloads as W

        O, w = self.O, self.w
        org = W.random_origins(w.n, count, seed)
        t0 = time.perf_counter()
        tau = self.grid.columns(self.x0, self.dirs, origins=org)
        g, te = O.gamma(tau, self.s, self.wts)
        O.xeq(g, w.nH[org], w.T[org], 0.0, te >= 1)
        return time.perf_counter() - t0

    def sample(self, seconds: float, seed: int):
        """One sample of about `seconds`; the size is calibrated on the first
        call (twice: the first small run also pays the threads' start-up)."""
        if self.count == 64:
            for c in (64, 1024):
                t = self.run(c, seed + 1000 + c)
                self.count = int(min(self.w.n, max(64, c * seconds / max(t, 1e-3))))
        dt = self.run(self.count, seed)
        return {"rays": self.count * self.dirs.shape[0], "origins": self.count, "seconds": dt,
                "cores": self.O.num_threads()}

    def describe(self, r) -> str:
        return (f"{r['origins']} seeded origins x {self.dirs.shape[0]} rays, one sweep (columns by the "
                f"oracle's uniform-grid search, {self.cell:g} kpc cells, {self.grid.entries} entries, built once "
                f"in {self.build_s:.1f} s and not counted; FP64 Gamma and x) per sample")


def reference_arm(args, key, w):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    ors = OracleSample(w, GRID_CELL[key])
    per = max(2.0, args.cpu_seconds / max(1, args.steps + args.warmup))
    for i in range(args.warmup):
        ors.sample(per, 1 + i)
    runs = [ors.sample(per, 100 + i) for i in range(args.steps)]
    rays = sum(r["rays"] for r in runs)
    secs = sum(r["seconds"] for r in runs)
    value = rays / secs
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "rays/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": workload_name(key, w), "l2": "n/a (CPU)"},
        "particle_updates_per_s": sum(r["origins"] for r in runs) / secs,
        "cpu_baseline": {"value": value, "unit": "rays/s", "cores": runs[0]["cores"], "kind": "oracle-grid",
                         "sample": ors.describe(runs[0])},
        "e2e": {"value": value, "unit": "rays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


class Device:
    """The workload's inputs as pinned host tensors and on the device, the
    spectrum and the ray set."""

    def __init__(self, w, dev):
        import torch
        from paper_1304_4235_gb300 import urchin as U

        self.w, self.dev, self.U = w, dev, U
        pos = w.pos.astype(np.float32)
        host = {
            "px": np.ascontiguousarray(pos[:, 0]), "py": np.ascontiguousarray(pos[:, 1]),
            "pz": np.ascontiguousarray(pos[:, 2]), "h": np.ascontiguousarray(w.h, dtype=np.float32),
            "m": np.ascontiguousarray(w.mass_H), "nH": np.ascontiguousarray(w.nH),
            "T": np.ascontiguousarray(w.T),
        }
        self.pinned = {k: torch.from_numpy(v).pin_memory() for k, v in host.items()}
        self.d = {k: v.to(dev) for k, v in self.pinned.items()}
        e, J = w.spectrum()
        s_h, w_h = U.urchin_spectrum_weights(e, J, w.gamma_thin)
        self.s, self.wts = torch.from_numpy(s_h).to(dev), torch.from_numpy(w_h).to(dev)
        self.dirs = U.urchin_healpix_dirs(w.nside)

    def bvh(self, d=None):
        d = self.d if d is None else d
        w = self.w
        return self.U.urchin_build_bvh(d["px"], d["py"], d["pz"], d["h"], d["m"], w.periodic, w.box, w.unit_cm)

    def solve(self, bvh, d=None, s=None, wts=None, **kw):
        d = self.d if d is None else d
        kw.setdefault("precision", self.U.F32)
        kw.setdefault("raise_not_converged", False)
        return self.U.urchin_solve(bvh, self.dirs, self.w.l_ray, self.s if s is None else s,
                                   self.wts if wts is None else wts, d["nH"], d["T"], **kw)

    def solve_step(self, d=None, max_iter=4000):
        """One full solve: BVH build, then plain sweeps from x_thin to
        max |dx|/x < 1e-3 (segments stored where a long solve pays for them)."""
        bvh = self.bvh(d)
        x, st = self.solve(bvh, d, tol=1e-3, max_iter=max_iter, segments=self.U.SEG_AUTO, profile=True)
        bvh.close()
        return x, st


def events():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def timed(stream, fn):
    """(result, seconds) of fn() bracketed by CUDA events on `stream`."""
    a, b = events()
    a.record(stream)
    r = fn()
    b.record(stream)
    b.synchronize()
    return r, a.elapsed_time(b) * 1e-3


def roofline_spmv(stats, hbm, peak_kind):
    """k_spmv8 (stored-segment columns) against the HBM roofline: 8
    algorithmic bytes per segment (a 4-byte particle index and a 4-byte
    value; the kernel moves 7, the index split in 16 + 8 bits), plus each
    ray's 4-byte column and the 4-byte x gather per particle, over the
    launch's mean duration."""
    launches = sum(st["spmv_launches"] for st in stats)
    spmv_s = sum(st["spmv_s"] for st in stats)
    moved = sum(st["spmv_bytes"] for st in stats)          # 7 per segment + columns + x
    st0 = stats[-1]
    extra = launches * (st0["n_active"] * 12 * 4 + st0["n_active"] * 4)
    seg = max(moved - extra, 0) / 7.0
    per_bytes = (seg * 8 + extra) / max(launches, 1)
    per_s = spmv_s / max(launches, 1)
    achieved = per_bytes / per_s / 1e9 if per_s > 0 else None
    t = MEASURED_TRAFFIC["k_spmv"].get(source_hash("k_spmv"))
    return {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": achieved / hbm if achieved else None, "traffic": (t * seg / max(launches, 1)) if t else None,
            "kernel": "k_spmv8 (FP32 stored segments)", "peak_kind": peak_kind, "alg_bytes_per_launch": per_bytes,
            "launch_ms": per_s * 1e3, "segments_per_launch": seg / max(launches, 1)}


def roofline(stats, trace_launches_total, hbm, peak_kind, rays_per_sweep):
    """k_trace against the HBM roofline: algorithmic bytes per launch (every
    ray-sphere hit reads a 16-byte particle record and its 4-byte weight; every
    ray writes its 4-byte column) over the launch's mean duration.  When the
    solve's one traversal also stored the segment lists (one per step, over
    every particle's rays), it writes each ray's 4-byte hit count and every
    stored entry (8 bytes: particle index and value, the padding included)."""
    hits = sum(st["hits"] for st in stats)
    trace_s = sum(st["trace_s"] for st in stats)
    n = max(trace_launches_total, 1)
    if all(st["trace_launches"] == 1 and st["segments_stored"] for st in stats):
        rays = rays_per_sweep * len(stats)
        stored = sum(st["nnz"] for st in stats)
        per_bytes = (hits * 20 + rays * 8 + stored * 8) / n
    else:
        rays = sum(st["rays"] for st in stats)
        per_bytes = (hits * 20 + rays * 4) / n
    per_s = trace_s / n
    achieved = per_bytes / per_s / 1e9 if per_s > 0 else None
    t = MEASURED_TRAFFIC["k_trace"].get(source_hash("k_trace"))
    return {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": achieved / hbm if achieved else None,
            "traffic": (t * hits / n) if t else None,
            "kernel": "k_trace<float,M4> (FP32 columns; segment lists stored while tracing where the solve "
                      "keeps them)", "peak_kind": peak_kind,
            "alg_bytes_per_launch": per_bytes, "launch_ms": per_s * 1e3,
            "hits_per_launch": hits / n, "rays_per_launch": rays / n,
            "sphere_tests_per_hit": sum(st["sphere_tests"] for st in stats) / max(hits, 1),
            "node_visits_per_hit": sum(st["node_visits"] for st in stats) / max(hits, 1)}


def main():
    args = parse()
    key = args.workload
    w = load_workload(key, args.cache_dir)
    if args.impl == "reference":
        reference_arm(args, key, w)
        return

    import torch
    import torch.distributed as dist

    from paper_1304_4235_gb300 import urchin as U

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    U.load()
    D = Device(w, dev)
    stream = torch.cuda.current_stream(dev)
    # inputs larger than L2 (129 MB) on the largest box; the halo's are
    # smaller, so a 256 MB write flushes L2 before every timed step
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    for _ in range(args.warmup):
        D.solve_step(max_iter=args.max_iter)
    clocks = Clocks(dev.index if dev.index is not None else 0)
    stats, step_s = [], []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    launches0 = U.urchin_kernel_launches()
    clocks.start()
    for _ in range(args.steps):
        flush.zero_()
        (_, st), dt = timed(stream, lambda: D.solve_step(max_iter=args.max_iter))
        step_s.append(dt)
        stats.append(st)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    launches = U.urchin_kernel_launches() - launches0
    total_ms = 1e3 * sum(step_s)
    rays = sum(st["rays"] for st in stats)
    updates = sum(st["particle_updates"] for st in stats)
    total_ms, (rays, updates) = combine_ranks(total_ms, (rays, updates), device=dev)

    # end to end through the public API with host buffers: pinned H2D of the
    # inputs, build, sweep, D2H of x, all inside the timed region
    e2e = None
    if not args.no_e2e:
        x_host = torch.empty(w.n, dtype=torch.float64).pin_memory()
        h2d = sum(v.numel() * v.element_size() for v in D.pinned.values())
        d2h = x_host.numel() * x_host.element_size()
        e2e_s, e2e_rays = [], 0

        def e2e_step():
            dd = {k: v.to(dev, non_blocking=True) for k, v in D.pinned.items()}
            x, st = D.solve_step(dd, max_iter=args.max_iter)
            x_host.copy_(x, non_blocking=True)
            return st

        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize(dev)
            st, dt = timed(stream, e2e_step)
            e2e_s.append(dt)
            e2e_rays += st["rays"]
        e2e = {"value": e2e_rays / sum(e2e_s) * world, "unit": "rays/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    hbm, peak_kind = peaks()
    trace_s = sum(st["trace_s"] for st in stats)
    sweep_s = sum(st["sweep_s"] for st in stats)
    trace_launches = sum(st["trace_launches"] for st in stats)
    kernels = {
        "k_trace": {"s": trace_s, "launches": trace_launches},
        "k_sweep_pp": {"s": sweep_s, "launches": sum(st["sweep_launches"] for st in stats)},
        "stored_columns": {"s": sum(st["spmv_s"] for st in stats),
                           "launches": sum(st["spmv_launches"] for st in stats)},
    }
    for k in kernels.values():
        k["share_of_step"] = k["s"] / (total_ms * 1e-3 / world) if total_ms > 0 else None
    st0 = stats[-1]
    line = {
        "metric": METRIC, "value": rays / (total_ms * 1e-3), "unit": "rays/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": workload_name(key, w), "particles": w.n, "rays_per_particle": w.R,
                   "l_ray_kpc": w.l_ray, "bins": w.F, "method": "plain", "tol": 1e-3, "segments": "auto",
                   "step": "BVH build + plain sweeps from x_thin to max |dx|/x < 1e-3",
                   "l2": "inputs > L2 (129 MB); a 256 MB write before each step"},
        "particle_updates_per_s": updates / (total_ms * 1e-3),
        "iterations": st0["iterations"], "converged": bool(st0["converged"]),
        "segments_stored": bool(st0["segments_stored"]), "n_active": st0["n_active"], "hits_per_step": st0["hits"],
        "wall_s_to_converged": total_ms * 1e-3 / args.steps,
        "gpu_launches": int(launches),
        "roofline": (roofline_spmv(stats, hbm, peak_kind) if sum(st["spmv_s"] for st in stats) > trace_s
                     else roofline(stats, trace_launches, hbm, peak_kind, w.n * len(D.dirs))),
        "kernels": kernels,
        "clocks": clk,
        "e2e": e2e,
    }
    if not args.no_compare and world == 1:
        line["compare"] = compare(args, key, w, D, stream)
    if world == 1 and not args.no_cpu_baseline:
        ors = OracleSample(w, GRID_CELL[key])
        r = ors.sample(args.cpu_seconds, 7)
        line["cpu_baseline"] = {"value": r["rays"] / r["seconds"], "unit": "rays/s", "cores": r["cores"],
                                "kind": "oracle-grid", "sample": ors.describe(r) + f", {r['seconds']:.1f} s"}
        if "compare" in line:
            line["compare"]["lattice_fp64"] = lattice_fp64(args, dev, stream)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def convergence(D, stream, max_iter: int):
    """Wall time to x within rel 1e-3 of a tightly converged x* (plain sweeps
    to dx_tol 1e-6), for plain sweeps at decreasing dx_tol and for
    Newton-Krylov (plain sweeps until at most 1 % of the particles move by
    >= 1e-5, then GMRES(60) to relative residual 1e-4); stored segments where
    they fit (SEG_AUTO).  Each run: BVH build + solve, CUDA events."""
    U = D.U
    out = {}

    def run(**kw):
        def go():
            bvh = D.bvh()
            x, st = D.solve(bvh, segments=U.SEG_AUTO, profile=True, **kw)
            bvh.close()
            return x, st
        (x, st), dt = timed(stream, go)
        return x.cpu().numpy(), st, dt

    xr, sr, dtr = run(tol=1e-6, max_iter=max_iter * 5)
    out["xstar"] = {"method": "plain", "dx_tol": 1e-6, "iterations": sr["iterations"],
                    "converged": bool(sr["converged"]), "wall_s": dtr}
    runs = [("plain", U.METHOD_PLAIN, 1e-3, {}), ("plain_tol1e-4", U.METHOD_PLAIN, 1e-4, {}),
            ("plain_tol1e-5", U.METHOD_PLAIN, 1e-5, {}),
            ("newton", U.METHOD_NEWTON, 1e-5, dict(gmres_m=60, newton_eta=1e-4))]
    for name, meth, tol, extra in runs:
        xm, sm, dt = run(method=meth, tol=tol, max_iter=max_iter, **extra)
        dist = np.abs(xm - xr) / xr
        out[name] = {"wall_s": dt, "dx_tol": tol, "iterations": sm["iterations"], "converged": bool(sm["converged"]),
                     "rays": sm["rays"], "rays_per_s": sm["rays"] / dt,
                     "particle_updates_per_s": sm["particle_updates"] / dt,
                     "segments_stored": bool(sm["segments_stored"]), "nnz": sm["nnz"],
                     "trace_s": sm["trace_s"], "spmv_s": sm["spmv_s"], "sweep_s": sm["sweep_s"],
                     "newton_start": sm["newton_start"], "newton_fallbacks": sm["newton_fallbacks"],
                     "max_rel_to_xstar": float(dist.max()), "p999_rel_to_xstar": float(np.quantile(dist, 0.999))}
    ok = [v["wall_s"] for k, v in out.items() if k.startswith("plain") and v["max_rel_to_xstar"] < 1e-3]
    t = {"plain_wall_s": min(ok) if ok else None,
         "newton_wall_s": out["newton"]["wall_s"] if out["newton"]["max_rel_to_xstar"] < 1e-3 else None}
    t["newton_speedup"] = (t["plain_wall_s"] / t["newton_wall_s"]) if (t["plain_wall_s"] and t["newton_wall_s"]) else None
    out["to_rel_1e-3_of_xstar"] = t
    return out


def adjoint(D, stream, max_iter: int, segments):
    """Reverse mode at the converged state (plain sweeps to dx_tol 1e-3):
    gradient of L = sum_i ln x*_i with respect to the spectrum weights
    (adjoint GMRES(30) to 1e-6, one transposed column pass per product)."""
    import torch
    U = D.U
    bvh = D.bvh()
    state = torch.empty(D.w.n, dtype=torch.uint8, device=D.dev)
    xs, ss = D.solve(bvh, tol=1e-3, max_iter=max_iter, segments=U.SEG_AUTO, state=state)
    torch.cuda.synchronize(D.dev)

    def go():
        return U.urchin_solve_vjp(bvh, D.dirs, D.w.l_ray, D.s, D.wts, D.d["nH"], D.d["T"], xs, state, 1.0 / xs,
                                  tol=1e-6, max_iter=600, gmres_m=30, segments=segments, precision=U.F32,
                                  raise_not_converged=False, profile=True)
    (wb, vs), dt = timed(stream, go)
    bvh.close()
    return {"loss": "sum ln x*", "segments": "recompute" if segments == U.SEG_RECOMPUTE else "auto",
            "segments_stored": bool(vs["segments_stored"]),
            "wall_s": dt, "products": vs["iterations"], "rel_residual": vs["max_rel_dx"],
            "converged": bool(vs["converged"]), "rays": vs["rays"], "grad_norm": float(wb.norm()),
            "trace_s": vs["trace_s"], "spmv_s": vs["spmv_s"]}


def gradient_workload(D, stream, max_iter: int):
    """The differentiation workload on the halo: 200 bins, loss = sum over all
    rays of (log10 N_HI - log10 N_target)^2, the target from seeded +-20 %
    bin weights; x* by Newton-Krylov, gradient by autograd (adjoint solve +
    column transpose).  Reports the solves' segment mode, sweeps and Newton
    fallbacks beside the times."""
    import torch
    import workloads as W
    from paper_1304_4235_gb300 import autograd as UA
    U, w, dev = D.U, D.w, D.dev
    e2, J2 = W.powerlaw_spectrum(200, w.e_lo, w.e_hi)
    s2h, w2h = U.urchin_spectrum_weights(e2, J2, w.gamma_thin)
    s2, w2 = torch.from_numpy(s2h).to(dev), torch.from_numpy(w2h).to(dev)
    kw = dict(tol=1e-5, tau_skip=1e-4, max_iter=max_iter, method=U.METHOD_NEWTON, gmres_m=60, newton_eta=1e-4,
              segments=U.SEG_AUTO, precision=U.F32, raise_not_converged=False, profile=True)
    clocks = Clocks(dev.index if dev.index is not None else 0)
    clocks.start()
    bvh = D.bvh()
    w2t = w2 * torch.from_numpy(np.random.default_rng(1308).uniform(0.8, 1.2, 200)).to(dev)
    xt, stt = U.urchin_solve(bvh, D.dirs, w.l_ray, s2, w2t, D.d["nH"], D.d["T"], **kw)
    target = torch.log10(U.urchin_trace_columns(bvh, xt, D.dirs, w.l_ray).double())
    wv = w2.clone().requires_grad_(True)
    # The loss's torch kernels (log10, square and sum in double, and their
    # backward) are loaded on their first use in the process, which took
    # 4.9 s + 0.7 s with the GPU idle on a fresh box: run them once here,
    # outside the timed region.
    cw = torch.ones_like(target, dtype=torch.float32).requires_grad_(True)
    ((torch.log10(cw.double()) - target) ** 2).sum().backward()
    del cw
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    free0 = torch.cuda.mem_get_info(dev)[0]
    torch.cuda.synchronize(dev)
    host = [time.perf_counter()]
    ev[0].record(stream)
    info = {}
    xg = UA.converged_x(wv, bvh, D.dirs, w.l_ray, s2, D.d["nH"], D.d["T"], solve_kw=kw,
                        vjp_kw=dict(tol=1e-6, max_iter=600, gmres_m=30, raise_not_converged=False, profile=True),
                        info=info)
    ev[3].record(stream)
    host.append(time.perf_counter())
    cols = UA.columns(xg, bvh, D.dirs, w.l_ray)
    ev[4].record(stream)
    host.append(time.perf_counter())
    L = ((torch.log10(cols.double()) - target) ** 2).sum()
    ev[1].record(stream)
    host.append(time.perf_counter())
    L.backward()
    ev[2].record(stream)
    ev[2].synchronize()
    host.append(time.perf_counter())
    bvh.close()
    clk = clocks.stop()
    fs = info.get("forward_stats", {})
    bs = info.get("vjp_stats", {})
    # where the time goes, to tell a slow GPU from host-side waits
    phases = {f"{tag}_{k}": st.get(k) for tag, st in (("forward", fs), ("backward", bs), ("target", stt))
              for k in ("wall_s", "trace_s", "spmv_s", "sweep_s", "spmv_launches", "trace_launches")}
    phases.update({"gpu_solve_s": ev[0].elapsed_time(ev[3]) * 1e-3, "gpu_columns_s": ev[3].elapsed_time(ev[4]) * 1e-3,
                   "gpu_loss_s": ev[4].elapsed_time(ev[1]) * 1e-3, "host_solve_s": host[1] - host[0],
                   "host_columns_s": host[2] - host[1], "host_loss_s": host[3] - host[2],
                   "host_backward_s": host[4] - host[3], "free_bytes_at_start": free0})
    return {"loss": float(L.detach()), "forward_s": ev[0].elapsed_time(ev[1]) * 1e-3,
            "backward_s": ev[1].elapsed_time(ev[2]) * 1e-3, "grad_norm": float(wv.grad.norm()),
            "forward": "Newton-Krylov to dx_tol 1e-5 + columns of x*",
            "backward": "adjoint GMRES(30) to 1e-6 + column transpose",
            "forward_iterations": fs.get("iterations"), "forward_segments_stored": fs.get("segments_stored"),
            "forward_newton_start": fs.get("newton_start"), "forward_newton_fallbacks": fs.get("newton_fallbacks"),
            "backward_products": bs.get("iterations"), "target_solve_iterations": stt["iterations"],
            "phases": phases, "clocks": clk}


def cosmological_box(args, dev, stream):
    """The cosmological-like box with helium: 128^3 particles in 4 Mpc,
    sigma_ln 2, 48 rays of 100 kpc with periodic wrapping, 200 bins over
    13.6-136 eV, H I iterated with fixed He I / He II columns (seeded
    abundances, a stand-in He I cross section: the paper has no He I fit),
    plain sweeps to max |dx|/x < 1e-3 (BVH build + solve, CUDA events)."""
    import torch
    import workloads as W
    w = W.cached(W.lognormal_box, args.cache_dir, e_hi=136.0)
    D = Device(w, dev)
    U = D.U
    e, J = w.spectrum()
    s2 = torch.from_numpy(U.urchin_cross_section_ratio(e, U.XSEC_HEII)).to(dev)
    s1 = torch.from_numpy(W.hei_cross_section_standin(e)).to(dev)
    he1, he2 = (torch.from_numpy(a).to(dev) for a in W.helium_fractions(w, 1309))

    def go():
        bvh = D.bvh()
        x, st = D.solve(bvh, tol=1e-3, max_iter=args.max_iter, segments=U.SEG_AUTO, profile=True,
                        s_he1=s1, s_he2=s2, he1=he1, he2=he2)
        bvh.close()
        return st
    go()
    st, dt = timed(stream, go)
    return {"workload": f"lognormal_128cube_sigma2_L4000kpc_nside2_l100kpc_F200_13.6-136eV_HI+HeI+HeII",
            "wall_s": dt, "iterations": st["iterations"], "converged": bool(st["converged"]),
            "rays": st["rays"], "rays_per_s": st["rays"] / dt, "particle_updates_per_s": st["particle_updates"] / dt,
            "segments_stored": bool(st["segments_stored"]), "trace_s": st["trace_s"], "spmv_s": st["spmv_s"],
            "sweep_s": st["sweep_s"], "hits": st["hits"]}


def lattice_fp64(args, dev, stream):
    """The plain FP64 method on the 4096-particle jittered lattice (16^3 in a
    periodic 1 Mpc box, n_H 1.5e-3 cm^-3, 12 rays of 500 kpc, 50 bins): BVH
    build + FP64 plain sweeps from x_thin to max |dx|/x < 1e-3 on the GPU
    (CUDA events), and beside it, as this workload's CPU baseline, the FP64
    oracle solving the same problem to the same tolerance by brute force on
    all host cores, with the largest relative difference of the two x."""
    import traceback

    import oracle as O
    import workloads as W
    out = {"workload": "lattice_16cube_L1000kpc_nside1_l500kpc_F50", "precision": "f64", "method": "plain",
           "tol": 1e-3}
    try:
        w = W.lattice_box()
        D = Device(w, dev)
        U = D.U

        def go():
            bvh = D.bvh()
            x, st = D.solve(bvh, tol=1e-3, max_iter=args.max_iter, precision=U.F64, profile=True)
            bvh.close()
            return x, st
        go()
        (x, st), dt = timed(stream, go)
        xg = x.cpu().numpy()
        out.update({"wall_s": dt, "iterations": st["iterations"], "converged": bool(st["converged"]),
                    "rays": st["rays"], "rays_per_s": st["rays"] / dt,
                    "particle_updates_per_s": st["particle_updates"] / dt})
        e, J = w.spectrum()
        s, wts = O.spectrum(e, J, w.gamma_thin)
        t0 = time.perf_counter()
        xo, _, info = O.solve(w, s, wts, O.healpix(w.nside), tol=1e-3)
        to = time.perf_counter() - t0
        out["oracle"] = {"kind": "oracle", "search": "brute force", "cores": O.num_threads(), "wall_s": to,
                         "iterations": int(info["sweeps"]), "converged": bool(info["converged"]),
                         "rays": float(info["rays"]), "rays_per_s": float(info["rays"]) / to}
        out["max_rel_gpu_vs_oracle"] = float(np.max(np.abs(xg - xo) / xo))
    except Exception as exc:       # a failed side comparison must not cost the benchmark line
        traceback.print_exc()
        out["error"] = f"{type(exc).__name__}: {exc}"
    return out


def compare(args, key, w, D, stream):
    import torch
    comp = {"workload": workload_name(key, w)}
    comp.update(convergence(D, stream, args.max_iter))
    comp["adjoint_recompute"] = adjoint(D, stream, args.max_iter, D.U.SEG_RECOMPUTE)
    # the same gradient with the segment lists stored once (count + fill)
    # and every transposed product read from them
    comp["adjoint_stored"] = adjoint(D, stream, args.max_iter, D.U.SEG_AUTO)
    if key.startswith("c5"):
        # the 262144-particle halo beside it
        wh = load_workload("halo", args.cache_dir)
        Dh = Device(wh, D.dev)
        comp["halo"] = {"workload": workload_name("halo", wh)}
        comp["halo"].update(convergence(Dh, stream, args.max_iter))
        comp["halo"]["adjoint"] = adjoint(Dh, stream, args.max_iter, D.U.SEG_AUTO)
        comp["gradient_column_misfit_200_bins"] = gradient_workload(Dh, stream, args.max_iter)
        del Dh
        torch.cuda.empty_cache()
        comp["cosmological_box_helium"] = cosmological_box(args, D.dev, stream)
        torch.cuda.empty_cache()
    else:
        comp["gradient_column_misfit_200_bins"] = gradient_workload(D, stream, args.max_iter)
    return comp


if __name__ == "__main__":
    main()
