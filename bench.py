"""Benchmark of the FHR hot path (Algorithm 1) on synthetic data shaped like the
paper's workloads.

One step = normalise -> NNDSVD start -> fast-HALS NMF -> MBIR of every subspace
channel -> expansion to all wavelength bins, on one batch of counts already
resident in HBM (the 128 x 128 x 64 volume, 90 views, 64 x 128 detector,
Nk = 1200, K = 5, 200 counts per bin, 4% dead bins).  The metric is
voxel*bins/s: Nx * Nk / step time.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints ONE JSON line (rank 0).  Under torchrun (N > 1) every rank runs its own
replica of the step (the path shards by independent volumes; no data-path
collective) and the time is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "voxel*bins/s end-to-end (normalise + NNDSVD + 200-iteration NMF + MBIR + expansion)"
UNIT = "voxel*bins/s"
NMF_ITERS = 200
MBIR_ITERS = 100
K = 5


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms in the background."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power) if power else None}


def max_over_ranks(x: float, device="cpu") -> float:
    """The slowest replica's value (a time): all-reduce MAX across the process group,
    or x itself outside one."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(world: int, units_per_rank: float, ms: float) -> float:
    """Units of all replicas per second over the max-over-ranks time (weak scaling)."""
    return world * units_per_rank / (ms / 1e3)


def make_inputs(device):
    from paper_2410_22500_gb300 import synth

    pb = synth.volume_3d_f32()
    y, y0 = synth.counts_torch(pb, device=device)
    return pb, y, y0


def algorithmic_pass_bytes(Np, Nk, K_):
    """One fused NMF pass reads P once (f32) and W once, writes W once."""
    return Np * Nk * 4 + 2 * Np * K_ * 4


# ---------------------------------------------------------------------------- CPU oracle
def oracle_sample(nmf_iters_run=10, mbir_iters_run=5):
    """The FP64 oracle on one detector row (one slice) of the same workload: every stage
    runs; NMF and MBIR run a few iterations and their time is scaled linearly to the
    full iteration counts.  Returns (voxel*bins/s, seconds, description)."""
    import oracle
    from paper_2410_22500_gb300 import synth

    pb = synth.scaled(synth.volume_3d_f32, Nr=1, seed=1001)
    g = pb.geom
    y, y0 = synth.counts_numpy(pb)
    th = g.angles()
    t0 = time.perf_counter()
    P = oracle.normalise(y, y0, dead=pb.dead_bins)
    t_norm = time.perf_counter() - t0
    t0 = time.perf_counter()
    D0, W0 = oracle.nndsvd(P, K)
    t_init = time.perf_counter() - t0
    t0 = time.perf_counter()
    D, W, obj = oracle.nmf(P, D0, W0, nmf_iters_run)
    t_nmf = (time.perf_counter() - t0) * NMF_ITERS / nmf_iters_run
    V = W.reshape(g.Nv, g.Nc, g.Nr * K)
    sv, sx = oracle.mbir_sigmas(W, K, g.Nc)
    t0 = time.perf_counter()
    xs = oracle.mbir(V, g.N, g.Nr, K, th, sv, sx, iters=mbir_iters_run, momentum=True)
    t_mbir = (time.perf_counter() - t0) * MBIR_ITERS / mbir_iters_run
    t0 = time.perf_counter()
    oracle.expand(xs, D, g.N, g.Nr)
    t_exp = time.perf_counter() - t0
    total = t_norm + t_init + t_nmf + t_mbir + t_exp
    vb = g.Nr * g.N * g.N * pb.Nk
    desc = ("one slice (Nr=1) of the 128x128x64 / Nk=1200 / K=5 workload, single-threaded FP64 oracle; "
            "NMF %d of %d and MBIR %d of %d iterations run, scaled linearly" % (nmf_iters_run, NMF_ITERS,
                                                                               mbir_iters_run, MBIR_ITERS))
    return vb / total, total, desc


# ---------------------------------------------------------------------------- GPU arm
def run_ours(args, rank, world, device):
    import torch
    from paper_2410_22500_gb300 import build as fbuild
    from paper_2410_22500_gb300 import fhr

    fbuild.build()
    torch.cuda.set_device(device)
    ctx = fhr.Context(device)
    pb, y, y0 = make_inputs("cuda:%d" % device)
    g = pb.geom
    dead = torch.from_numpy(pb.dead_bins).cuda(device)
    prm = ctx.pipeline_params(Nv=g.Nv, Nr=g.Nr, Nc=g.Nc, Nk=pb.Nk, N=g.N, K=K, nmf_iters=NMF_ITERS,
                              mbir_iters=MBIR_ITERS, momentum=True, seed=17)
    ws, ws_bytes = ctx.pipeline_workspace(prm)
    D = torch.empty((pb.Nk, K), dtype=torch.float32, device=device)
    xh = torch.empty((g.Nr, g.N, g.N, pb.Nk), dtype=torch.float32, device=device)
    obj = torch.empty(NMF_ITERS, dtype=torch.float64, device=device)
    stream = ctx.stream

    def step():
        ctx.pipeline(prm, y, y0, D, xh, obj=obj, dead=dead, ws=ws, ws_bytes=ws_bytes)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if ctx.status(ws) != 0:
        raise RuntimeError("device status after warm-up")

    dist = None
    if world > 1:
        import torch.distributed as dist_mod

        dist = dist_mod
        dist.barrier()
    clocks = ClockSampler(device)
    clocks.start()
    ctx.profile(True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    launches, _ = ctx.profile_read()
    pass_n, pass_ms = ctx.profile_read("nmf_pass")
    fams = {n: ctx.profile_read(n) for n in ("normalise", "nndsvd_pass", "nmf_pass", "nmf_reduce", "nmf_update",
                                             "proj_fwd", "mbir_update", "expand")}
    ctx.profile(False)
    clk = clocks.stop()
    if ctx.status(ws) != 0:
        raise RuntimeError("device status after timed steps")
    ms = max_over_ranks(ms, device)
    ms_step = ms / args.steps
    vb = g.Nr * g.N * g.N * pb.Nk
    value = whole_job_value(world, vb, ms_step)

    # ---- end to end through the C ABI with pinned host buffers
    prm_h = ctx.pipeline_params(Nv=g.Nv, Nr=g.Nr, Nc=g.Nc, Nk=pb.Nk, N=g.N, K=K, nmf_iters=NMF_ITERS,
                                mbir_iters=MBIR_ITERS, momentum=True, seed=17, host_io=True)
    del ws
    torch.cuda.empty_cache()
    ws_h, wsb_h = ctx.pipeline_workspace(prm_h)
    y_h = y.cpu().pin_memory()
    y0_h = y0.cpu().pin_memory()
    xh_h = torch.empty(xh.shape, dtype=torch.float32).pin_memory()
    del xh
    torch.cuda.empty_cache()
    h2d = y_h.numel() * 2 + y0_h.numel() * 2
    d2h = xh_h.numel() * 4

    def step_h():
        ctx.pipeline(prm_h, y_h, y0_h, D, xh_h, obj=obj, dead=dead, ws=ws_h, ws_bytes=wsb_h)

    step_h()
    torch.cuda.synchronize()
    e2e_steps = max(1, args.steps)
    if dist is not None:
        dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(e2e_steps):
        step_h()
    ctx.io_join()   # the last step's output copy is inside the timed region
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / e2e_steps
    e2e_ms = max_over_ranks(e2e_ms, device)
    if ctx.status(ws_h) != 0:
        raise RuntimeError("device status after end-to-end steps")

    peak, peak_kind = _peaks()
    pass_bytes = algorithmic_pass_bytes(g.Np, pb.Nk, K)
    achieved = pass_bytes / (pass_ms / pass_n / 1e3) / 1e9 if pass_n else None
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "nmf_pass_traffic.json")
    if os.path.exists(tpath):
        try:
            from paper_2410_22500_gb300 import build as fb

            with open(tpath) as f:
                tr = json.load(f)
            if tr.get("source_digest") == fb.kernel_digest("nmf_pass") and tr.get("workload") == "volume_3d_f32":
                traffic = tr["bytes_per_launch"]
        except Exception:
            traffic = None
    out = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded ellipsoid phantom, Bragg-edge spectra, Poisson counts)",
        "config": {"workload": "volume_3d_f32: 128x128x64 voxels, Nk=1200, 90 views, 64x128 detector, K=5, "
                               "I0=200, 4% dead bins",
                   "Np": g.Np, "Nk": pb.Nk, "Nx": g.Nx, "K": K, "nmf_iters": NMF_ITERS, "mbir_iters": MBIR_ITERS,
                   "init": "nndsvd", "mbir": "SQS + momentum, qGGMRF p=1.2 q=2 T=1",
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "l2": "inputs larger than L2 (P is 3.54 GB per step)"},
        "e2e": {"value": whole_job_value(world, vb, e2e_ms), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
        "gpu_launches": int(launches),
        "roofline": {"bound": "hbm", "kernel": "nmf_mma_kernel (fused fast-HALS pass, warp MMA)", "achieved": achieved,
                     "peak": peak, "peak_kind": "%s (MEASURED_PEAKS.json hbm_gbs)" % peak_kind
                     if peak_kind == "measured" else "fallback", "unit": "GB/s",
                     "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                     "frac_of_nominal_7900": (achieved / 7900.0) if achieved else None,
                     "algorithmic_bytes_per_launch": pass_bytes, "launches": pass_n,
                     "avg_launch_ms": pass_ms / pass_n if pass_n else None},
        "kernel_ms": {n: {"launches": c, "total_ms": t} for n, (c, t) in fams.items()},
        "clocks": clk,
    }
    ctx.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        # the reference arm is the FP64 CPU oracle, timed as it stands on the host cores
        if rank != 0:
            return
        import oracle

        oracle.build()
        vals = []
        desc = ""
        for _ in range(args.warmup):
            oracle_sample(2, 1)
        for _ in range(args.steps):
            v, secs, desc = oracle_sample(4, 2)
            vals.append(v)
        v = statistics.median(vals)
        print(json.dumps({"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 0,
                          "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
                          "dtype": "f64", "data": "synthetic", "config": {"workload": "volume_3d_f32 (one slice)"},
                          "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc},
                          "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
        return

    if world > 1:
        import torch
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    out = run_ours(args, rank, world, local)
    if rank == 0:
        if not args.no_cpu_baseline:
            import oracle

            oracle.build()
            v, secs, desc = oracle_sample()
            out["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc,
                                   "seconds": secs}
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist

        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
