#!/usr/bin/env python
"""Benchmark of the reverse ray tracing solve (Altay & Theuns, arXiv:1304.4235)
on the 262144-particle self-shielding halo: n_H = 10 (r/kpc)^-2 cm^-3 over
r = 1-100 kpc, T = 1e4 K, h from 48 neighbours, 12 HEALPix rays per particle
of length 200 kpc, 100 frequency bins (nu^-1.5, 13.6-54.4 eV), FP32 columns
and spectral sum, FP64 equilibrium; iterate to max |dx|/x < 1e-3.

One step = one full pass of the hot path on a fresh copy of the inputs:
BVH build, then the solve from x_thin to convergence.  Metric: rays/s (all
rays traced, value and tangent) and particle-updates/s, whole job.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--method plain|newton]
                  [--segments recompute|store|auto] [--impl ours|reference]

Under torchrun every rank solves its own copy of the halo (replicas; the
method needs no exchange between independent halos) and rank 0 prints one
JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
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
def workload_name(w) -> str:
    """The halo as benchmarked: particles, HEALPix N_side, ray length, bins."""
    return f"halo_{w.n}_nside{w.nside}_l{w.l_ray:g}kpc_F{w.F}"

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per unit of work
# of a kernel, from one ncu capture, keyed by the hash of the kernel's source
# files at capture time; a changed kernel reports traffic null.
#   k_spmv: bytes per stored segment read;  k_trace: bytes per ray-sphere hit
MEASURED_TRAFFIC = {
    # 65536-particle halo: 2.2773e9 DRAM bytes for 3.2360e8 segments (rays padded
    # to multiples of 8) in one launch of k_spmv8 (7 algorithmic bytes per segment);
    # captured at 41377b11515427e3, whose sources differ from 87756054aa5bee94
    # only in the rewrapped file comment of linalg.cu
    "k_spmv": {"41377b11515427e3": 7.038, "87756054aa5bee94": 7.038},
    "k_trace": {},
}
KERNEL_SOURCES = {"k_spmv": ("linalg.cu", "linalg.cuh"),
                  "k_trace": ("trace.cu", "common.cuh")}


def source_hash(kernel: str) -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_1304_4235_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--method", choices=["plain", "newton"], default="plain")
    ap.add_argument("--segments", choices=["recompute", "store", "auto"], default="auto")
    ap.add_argument("--blocks", type=int, default=1, help="update order: 1 Jacobi, B>1 density blocks")
    ap.add_argument("--no-compare", action="store_true", help="skip the untimed Newton / tight-tolerance runs")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU time of the oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--max-iter", type=int, default=1000, help="sweep / Newton-step limit of one solve")
    ap.add_argument("--halo-n", type=int, default=262144, help="particles (profiling of smaller cases)")
    return ap.parse_args()


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


def oracle_sample(w, s, wts, dirs, seconds: float):
    """The FP64 oracle on a bounded sample of the workload: one sweep (columns
    of every ray, Gamma and the equilibrium x) for a seeded sample of origins
    sized to take about `seconds` of CPU time."""
    import oracle as O
    import workloads as W

    x0 = O.xeq(wts.sum(), w.nH, w.T, 0.0, False)

    def run(count, seed):
        org = W.random_origins(w.n, count, seed)
        t0 = time.perf_counter()
        tau = O.columns(w, x0, dirs, origins=org)
        g, te = O.gamma(tau, s, wts)
        O.xeq(g, w.nH[org], w.T[org], 0.0, te >= 1)
        return time.perf_counter() - t0

    t = run(32, 1)
    count = int(min(w.n, max(32, 32 * seconds / max(t, 1e-3))))
    dt = run(count, 2)
    rays = count * dirs.shape[0]
    return {"rays": rays, "origins": count, "seconds": dt, "cores": O.num_threads()}


def reference_arm(args, w):
    import oracle as O

    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    e, J = w.spectrum()
    s, wts = O.spectrum(e, J, w.gamma_thin)
    dirs = O.healpix(w.nside)
    per = max(2.0, args.cpu_seconds / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        oracle_sample(w, s, wts, dirs, per)
    runs = [oracle_sample(w, s, wts, dirs, per) for _ in range(args.steps)]
    rays = sum(r["rays"] for r in runs)
    secs = sum(r["seconds"] for r in runs)
    value = rays / secs
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "rays/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": workload_name(w), "l2": "n/a (CPU)"},
        "particle_updates_per_s": sum(r["origins"] for r in runs) / secs,
        "cpu_baseline": {"value": value, "unit": "rays/s", "cores": runs[0]["cores"], "kind": "oracle",
                         "sample": f"{runs[0]['origins']} seeded origins x {dirs.shape[0]} rays, one sweep "
                                   f"(brute-force columns over all {w.n} particles, Gamma, x) per step"},
        "e2e": {"value": value, "unit": "rays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    import workloads as W

    w = W.halo(n=args.halo_n)
    if args.impl == "reference":
        reference_arm(args, w)
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

    method = U.METHOD_NEWTON if args.method == "newton" else U.METHOD_PLAIN
    segs = {"recompute": U.SEG_RECOMPUTE, "store": U.SEG_STORE, "auto": U.SEG_AUTO}[args.segments]
    pos = w.pos.astype(np.float32)
    host = {
        "px": np.ascontiguousarray(pos[:, 0]), "py": np.ascontiguousarray(pos[:, 1]),
        "pz": np.ascontiguousarray(pos[:, 2]), "h": np.ascontiguousarray(w.h, dtype=np.float32),
        "m": np.ascontiguousarray(w.mass_H), "nH": np.ascontiguousarray(w.nH),
        "T": np.ascontiguousarray(w.T),
    }
    pinned = {k: torch.from_numpy(v).pin_memory() for k, v in host.items()}
    d = {k: v.to(dev) for k, v in pinned.items()}
    e, J = w.spectrum()
    s_h, w_h = U.urchin_spectrum_weights(e, J, w.gamma_thin)
    s_d, w_d = torch.from_numpy(s_h).to(dev), torch.from_numpy(w_h).to(dev)
    dirs = U.urchin_healpix_dirs(w.nside)
    stream = torch.cuda.current_stream(dev)

    # the timed method: plain sweeps to the paper's dx_tol = 1e-3, or
    # Newton-Krylov to dx_tol = 1e-5 (GMRES(60) to relative residual 1e-4)
    timed = dict(tol=1e-3) if method == U.METHOD_PLAIN else dict(tol=1e-5, gmres_m=60, newton_eta=1e-4)

    def step(dd, x_out=None, meth=None, tol=None, max_iter=None, gmres_m=None, newton_eta=None):
        tol = timed["tol"] if tol is None else tol
        gmres_m = timed.get("gmres_m", 20) if gmres_m is None else gmres_m
        newton_eta = timed.get("newton_eta", 0.0) if newton_eta is None else newton_eta
        bvh = U.urchin_build_bvh(dd["px"], dd["py"], dd["pz"], dd["h"], dd["m"], w.periodic, w.box, w.unit_cm)
        x = torch.empty(w.n, dtype=torch.float64, device=dev) if x_out is None else x_out
        x, st = U.urchin_solve(bvh, dirs, w.l_ray, s_d, w_d, dd["nH"], dd["T"], x, tol=tol, tau_skip=1e-4,
                               max_iter=max_iter or args.max_iter, method=method if meth is None else meth,
                               segments=segs, precision=U.F32, case_rule=U.CASE_AUTO, profile=True,
                               raise_not_converged=False, blocks=args.blocks, gmres_m=gmres_m,
                               newton_eta=newton_eta)
        bvh.close()
        return x, st

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > L2 (129 MB)
    for _ in range(args.warmup):
        step(d)

    clocks = Clocks(dev.index if dev.index is not None else 0)
    stats = []
    step_ms = []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    launches0 = U.urchin_kernel_launches()
    clocks.start()
    for _ in range(args.steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        _, st = step(d)
        b.record(stream)
        b.synchronize()
        step_ms.append(a.elapsed_time(b))
        stats.append(st)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    launches = U.urchin_kernel_launches() - launches0

    total_ms = sum(step_ms)
    rays = sum(st["rays"] for st in stats)
    updates = sum(st["particle_updates"] for st in stats)
    hits = sum(st["hits"] for st in stats)
    trace_s = sum(st["trace_s"] for st in stats)
    trace_launches = sum(st["trace_launches"] for st in stats)
    total_ms, (rays, updates) = combine_ranks(total_ms, (rays, updates), device=dev)

    # end to end through the public API with host buffers: pinned H2D of the
    # inputs, build, solve, D2H of x, all inside the timed region
    e2e = None
    if not args.no_e2e:
        x_host = torch.empty(w.n, dtype=torch.float64).pin_memory()
        e2e_ms, e2e_rays = [], 0
        h2d = sum(v.numel() * v.element_size() for v in pinned.values())
        d2h = x_host.numel() * x_host.element_size()
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize(dev)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            dd = {k: v.to(dev, non_blocking=True) for k, v in pinned.items()}
            x, st = step(dd)
            x_host.copy_(x, non_blocking=True)
            b.record(stream)
            b.synchronize()
            e2e_ms.append(a.elapsed_time(b))
            e2e_rays += st["rays"]
        e2e = {"value": e2e_rays / (sum(e2e_ms) * 1e-3) * world, "unit": "rays/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    hbm, peak_kind = peaks()
    # per-kernel GPU time of the timed steps (CUDA events on the solve's stream)
    spmv_s = sum(st["spmv_s"] for st in stats)
    sweep_s = sum(st["sweep_s"] for st in stats)
    spmv_launches = sum(st["spmv_launches"] for st in stats)
    spmv_bytes = sum(st["spmv_bytes"] for st in stats)
    trace_bytes = hits * 20 + sum(st["rays"] for st in stats if st["spmv_launches"] == 0) * 4
    kernels = {
        "k_spmv": {"s": spmv_s, "launches": spmv_launches},
        "k_trace": {"s": trace_s, "launches": trace_launches},
        "k_sweep": {"s": sweep_s, "launches": sum(st["sweep_launches"] for st in stats)},
    }
    for k in kernels.values():
        k["share_of_step"] = k["s"] / (total_ms * 1e-3 / world) if total_ms > 0 else None
    if spmv_s >= trace_s and spmv_launches > 0:
        per_bytes = spmv_bytes / spmv_launches
        per_s = spmv_s / spmv_launches
        # 4-byte value + 3-byte split particle index per FP32 segment (n <= 2^24);
        # the per-ray output and per-particle gather bytes are ~0.1 % of a launch
        seg_per_launch = (spmv_bytes / spmv_launches) / (7.0 if w.n <= (1 << 24) else 8.0)
        t = MEASURED_TRAFFIC["k_spmv"].get(source_hash("k_spmv"))
        roof = {"bound": "hbm", "achieved": per_bytes / per_s / 1e9, "peak": hbm, "unit": "GB/s",
                "frac": per_bytes / per_s / 1e9 / hbm,
                "traffic": (t * seg_per_launch) if t else None,
                "kernel": "k_spmv8 (FP32 stored segments)", "peak_kind": peak_kind,
                "alg_bytes_per_launch": per_bytes, "launch_ms": per_s * 1e3}
    else:
        per_bytes = trace_bytes / max(trace_launches, 1)
        per_s = trace_s / max(trace_launches, 1)
        t = MEASURED_TRAFFIC["k_trace"].get(source_hash("k_trace"))
        roof = {"bound": "hbm", "achieved": per_bytes / per_s / 1e9 if per_s > 0 else None, "peak": hbm,
                "unit": "GB/s", "frac": (per_bytes / per_s / 1e9 / hbm) if per_s > 0 else None,
                "traffic": (t * hits / max(trace_launches, 1)) if t else None,
                "kernel": "k_trace<float,M4>", "peak_kind": peak_kind,
                "alg_bytes_per_launch": per_bytes, "launch_ms": per_s * 1e3}
    roof["traversal"] = {"hits_per_launch": hits / max(trace_launches, 1), "launch_ms": 1e3 * trace_s / max(trace_launches, 1),
                         "sphere_tests_per_hit": sum(st["sphere_tests"] for st in stats) / max(hits, 1),
                         "node_visits_per_hit": sum(st["node_visits"] for st in stats) / max(hits, 1)}
    st0 = stats[-1]
    line = {
        "metric": METRIC, "value": rays / (total_ms * 1e-3), "unit": "rays/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": workload_name(w), "particles": w.n, "rays_per_particle": w.R, "l_ray_kpc": w.l_ray,
                   "bins": w.F, "method": args.method, "segments": args.segments, "blocks": args.blocks,
                   "tol": timed["tol"], "l2": "flushed before each step (256 MB write); stored segments >> L2"},
        "particle_updates_per_s": updates / (total_ms * 1e-3),
        "iterations": st0["iterations"], "n_active": st0["n_active"], "converged": bool(st0["converged"]),
        "segments_stored": bool(st0["segments_stored"]), "nnz": st0["nnz"],
        "wall_s_to_converged": total_ms * 1e-3 / args.steps,
        "gpu_launches": int(launches),
        "roofline": roof,
        "kernels": kernels,
        "clocks": clk,
        "e2e": e2e,
    }
    if not args.no_compare and world == 1:
        # untimed: wall time to x within rel 1e-3 of a tightly converged x*
        # (max over particles), for plain sweeps at decreasing step
        # tolerances and for Newton-Krylov (plain sweeps until at most 1 % of
        # the particles move by >= 1e-5, then Newton steps with GMRES(60) to
        # relative residual 1e-4)
        comp = {}
        xr, sr = step(d, meth=U.METHOD_PLAIN, tol=1e-6, max_iter=20000)
        xr = xr.cpu().numpy()
        runs = [("plain", U.METHOD_PLAIN, 1e-3, {}), ("plain_tol1e-4", U.METHOD_PLAIN, 1e-4, {}),
                ("plain_tol1e-5", U.METHOD_PLAIN, 1e-5, {}),
                ("newton", U.METHOD_NEWTON, 1e-5, dict(gmres_m=60, newton_eta=1e-4))]
        for name, meth, tol, extra in runs:
            torch.cuda.synchronize(dev)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            xm, sm = step(d, meth=meth, tol=tol, max_iter=args.max_iter * 3, **extra)
            b.record(stream)
            b.synchronize()
            dist = np.abs(xm.cpu().numpy() - xr) / xr
            comp[name] = {"wall_s": a.elapsed_time(b) * 1e-3, "dx_tol": tol, "iterations": sm["iterations"],
                          "converged": bool(sm["converged"]), "rays": sm["rays"],
                          "newton_start": sm["newton_start"], "newton_fallbacks": sm["newton_fallbacks"],
                          "max_rel_to_xstar": float(dist.max()), "p999_rel_to_xstar": float(np.quantile(dist, 0.999))}
        comp["xstar"] = {"method": "plain", "dx_tol": 1e-6, "iterations": sr["iterations"],
                         "converged": bool(sr["converged"])}
        ok = [v["wall_s"] for k, v in comp.items() if k.startswith("plain") and v["max_rel_to_xstar"] < 1e-3]
        comp["to_rel_1e-3_of_xstar"] = {
            "plain_wall_s": min(ok) if ok else None,
            "newton_wall_s": comp["newton"]["wall_s"] if comp["newton"]["max_rel_to_xstar"] < 1e-3 else None}
        t = comp["to_rel_1e-3_of_xstar"]
        t["newton_speedup"] = (t["plain_wall_s"] / t["newton_wall_s"]) if (t["plain_wall_s"] and t["newton_wall_s"]) else None
        # the near/far split of the paper (a different model of the near
        # particles, so its x is not compared with the plain scheme's x*),
        # with the analytic (threshold) and the numerical (spectrum) slab
        for name, slab in (("near_far_threshold", U.SLAB_THRESHOLD), ("near_far_spectrum", U.SLAB_SPECTRUM)):
            bvh = U.urchin_build_bvh(d["px"], d["py"], d["pz"], d["h"], d["m"], w.periodic, w.box, w.unit_cm)
            torch.cuda.synchronize(dev)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            xnf, snf = U.urchin_solve(bvh, dirs, w.l_ray, s_d, w_d, d["nH"], d["T"], tol=1e-3, tau_skip=1e-4,
                                      max_iter=args.max_iter, segments=segs, precision=U.F32, near_far=slab,
                                      raise_not_converged=False, profile=True)
            b.record(stream)
            b.synchronize()
            bvh.close()
            xnf = xnf.cpu().numpy()
            comp[name] = {"wall_s": a.elapsed_time(b) * 1e-3, "dx_tol": 1e-3, "iterations": snf["iterations"],
                          "converged": bool(snf["converged"]), "rays": snf["rays"],
                          "trace_s": snf["trace_s"], "spmv_s": snf["spmv_s"], "sweep_s": snf["sweep_s"],
                          "median_x_over_plain_xstar": float(np.median(xnf / xr))}
        # reverse mode at the converged state: gradient of L = sum_i ln x*_i
        # with respect to the spectrum weights (adjoint GMRES, one transposed
        # column pass per product)
        bvh = U.urchin_build_bvh(d["px"], d["py"], d["pz"], d["h"], d["m"], w.periodic, w.box, w.unit_cm)
        state = torch.empty(w.n, dtype=torch.uint8, device=dev)
        xs, ss = U.urchin_solve(bvh, dirs, w.l_ray, s_d, w_d, d["nH"], d["T"], tol=1e-3, tau_skip=1e-4,
                                max_iter=args.max_iter, segments=segs, precision=U.F32, state=state,
                                raise_not_converged=False)
        torch.cuda.synchronize(dev)
        # the first call after the forward solve, then the same call again
        for name in ("adjoint", "adjoint_repeat"):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            wb, vs = U.urchin_solve_vjp(bvh, dirs, w.l_ray, s_d, w_d, d["nH"], d["T"], xs, state, 1.0 / xs,
                                        tol=1e-6, max_iter=600, gmres_m=30, segments=segs, precision=U.F32,
                                        raise_not_converged=False, profile=True)
            b.record(stream)
            b.synchronize()
            comp[name] = {"loss": "sum ln x*", "wall_s": a.elapsed_time(b) * 1e-3, "products": vs["iterations"],
                          "rel_residual": vs["max_rel_dx"], "converged": bool(vs["converged"]),
                          "rays": vs["rays"], "grad_norm": float(wb.norm()), "trace_s": vs["trace_s"],
                          "spmv_s": vs["spmv_s"]}
        # the differentiation workload on the same halo: 200 bins, loss = sum over
        # all rays of (log10 N_HI - log10 N_target)^2, the target from seeded
        # +-20 % bin weights; x* by Newton-Krylov, gradient by autograd (adjoint
        # solve + column transpose)
        from paper_1304_4235_gb300 import autograd as UA
        e2, J2 = W.powerlaw_spectrum(200, w.e_lo, w.e_hi)
        s2h, w2h = U.urchin_spectrum_weights(e2, J2, w.gamma_thin)
        s2, w2 = torch.from_numpy(s2h).to(dev), torch.from_numpy(w2h).to(dev)
        kw = dict(tol=1e-5, tau_skip=1e-4, max_iter=args.max_iter, method=U.METHOD_NEWTON, gmres_m=60,
                  newton_eta=1e-4, segments=segs, precision=U.F32, raise_not_converged=False)
        w2t = w2 * torch.from_numpy(np.random.default_rng(1308).uniform(0.8, 1.2, 200)).to(dev)
        xt, _ = U.urchin_solve(bvh, dirs, w.l_ray, s2, w2t, d["nH"], d["T"], **kw)
        target = torch.log10(U.urchin_trace_columns(bvh, xt, dirs, w.l_ray).double())
        wv = w2.clone().requires_grad_(True)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record(stream)
        xg = UA.converged_x(wv, bvh, dirs, w.l_ray, s2, d["nH"], d["T"], solve_kw=kw,
                            vjp_kw=dict(tol=1e-6, max_iter=600, gmres_m=30, raise_not_converged=False))
        L = ((torch.log10(UA.columns(xg, bvh, dirs, w.l_ray).double()) - target) ** 2).sum()
        ev[1].record(stream)
        L.backward()
        ev[2].record(stream)
        ev[2].synchronize()
        comp["gradient_column_misfit_200_bins"] = {
            "loss": float(L.detach()), "forward_s": ev[0].elapsed_time(ev[1]) * 1e-3,
            "backward_s": ev[1].elapsed_time(ev[2]) * 1e-3, "grad_norm": float(wv.grad.norm()),
            "forward": "Newton-Krylov to dx_tol 1e-5 + columns of x*",
            "backward": "adjoint GMRES(30) to 1e-6 + column transpose"}
        bvh.close()
        line["compare"] = comp
    if world == 1 and not args.no_cpu_baseline:
        import oracle as O
        e_, J_ = w.spectrum()
        so, wo = O.spectrum(e_, J_, w.gamma_thin)
        r = oracle_sample(w, so, wo, O.healpix(w.nside), args.cpu_seconds)
        line["cpu_baseline"] = {
            "value": r["rays"] / r["seconds"], "unit": "rays/s", "cores": r["cores"], "kind": "oracle",
            "sample": f"{r['origins']} seeded origins x {w.R} rays, one sweep (brute-force columns over all "
                      f"{w.n} particles, Gamma, x), {r['seconds']:.1f} s"}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
