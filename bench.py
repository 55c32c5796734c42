"""Benchmark of the FHR hot path (Algorithm 1) on synthetic data shaped like the
paper's workloads.

One step = normalise -> NNDSVD start -> 200 fast-HALS NMF iterations -> 100 MBIR
iterations of every subspace channel -> expansion to all wavelength bins, on one
batch of counts already resident in HBM.  The workload is the largest that the
single-GPU configurations name, the precision form on a 256^3 volume: 6
ellipsoid materials, Nk = 1500 wavelength bins, 120 views over 180 degrees, a
256 x 256 detector, 100 open-beam counts per bin, K = 6; P (7.86M x 1500) is
streamed as BF16 with FP32 accumulation and FP64 Gram matrices and objective;
x^h (256^3 x 1500) is written in FP32.  The metric is voxel*bins/s:
Nx * Nk / step time, valid when the path is within 1e-3 relative error of FP64,
which the line's `accuracy` field measures on a one-slice sample against the
FP64 oracle.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints ONE JSON line (rank 0).  Under torchrun (N > 1) every rank runs its own
replica of the step (the path shards by independent volumes; no data-path
collective) and the time is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
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

METRIC = "voxel*bins/s end-to-end (normalise + NNDSVD + 200-iteration NMF + 100-iteration MBIR + expansion)"
UNIT = "voxel*bins/s"
NMF_ITERS = 200
MBIR_ITERS = 100
K = 6
WORKLOAD = ("precision form, 256^3 volume: 6 ellipsoid materials, K=6, Nk=1500, 120 views, 256x256 detector, "
            "I0=100 counts/bin; P streamed as BF16 (FP32 accumulation, FP64 Grams/objective), x^h FP32")
# oracle samples: (NMF iterations, MBIR iterations) run on one slice, then scaled
SAMPLE_ALL_CORES = (20, 10)
SAMPLE_ONE_CORE = (4, 2)
SAMPLE_REFERENCE = (4, 2)


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


def workload():
    from paper_2410_22500_gb300 import synth

    return synth.volume_3d_bf16()


def one_slice():
    """One detector row (one slice) of the workload's shape: the same per-slice sizes,
    dose and materials count, seeded like the volume."""
    from paper_2410_22500_gb300 import synth

    return synth.scaled(synth.volume_3d_bf16, Nr=1, seed=1002)


def algorithmic_pass_bytes(Np, Nk, elem, K_):
    """One fused NMF pass reads the Nk live bins of every row of P once and W once, and
    writes W once (P's padding columns, streamed too, are not counted)."""
    return Np * Nk * elem + 2 * Np * K_ * 4


def cpu_info():
    cores = len(os.sched_getaffinity(0))
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                k = line.split(":")[0].strip().lower()
                if k in ("model name", "cpu model", "hardware") and ":" in line:
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if model is None:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    import platform

    return cores, "%s (%s)" % (model or "unknown", platform.machine())


# ---------------------------------------------------------------------------- CPU oracle
def oracle_sample(nmf_run, mbir_run, threads, save=None):
    """The FP64 oracle on one slice of the workload, every stage; NMF and MBIR run
    nmf_run and mbir_run iterations and their time is scaled linearly to the full
    counts.  Returns a dict with the scaled voxel*bins/s and the stage times."""
    import oracle

    threads = oracle.set_threads(threads)
    pb = one_slice()
    g = pb.geom
    y, y0 = synth_counts(pb)
    th = g.angles()
    t = {}
    t0 = time.perf_counter()
    P = oracle.normalise(y, y0)
    t["normalise"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    D0, W0 = oracle.nndsvd(P, K)
    t["nndsvd"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    D, W, obj = oracle.nmf(P, D0, W0, nmf_run)
    t["nmf_run"] = time.perf_counter() - t0
    V = W.reshape(g.Nv, g.Nc, g.Nr * K)
    sv, sx = oracle.mbir_sigmas(W, K, g.Nc)
    t0 = time.perf_counter()
    xs = oracle.mbir(V, g.N, g.Nr, K, th, sv, sx, iters=mbir_run, momentum=True)
    t["mbir_run"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    xh = oracle.expand(xs, D, g.N, g.Nr)
    t["expand"] = time.perf_counter() - t0
    total = (t["normalise"] + t["nndsvd"] + t["nmf_run"] * NMF_ITERS / nmf_run + t["mbir_run"] * MBIR_ITERS / mbir_run
             + t["expand"])
    vb = g.Nr * g.N * g.N * pb.Nk
    if save:
        # untimed: the same stages on P rounded to BF16 (through FP32, as the GPU stores it),
        # from the same start, so that the GPU's BF16 path can be compared on equal data
        import torch

        Pb = torch.from_numpy(P.astype(np.float32)).to(torch.bfloat16).double().numpy()
        Db, Wb, objb = oracle.nmf(Pb, D0, W0, nmf_run)
        svb, sxb = oracle.mbir_sigmas(Wb, K, g.Nc)
        xsb = oracle.mbir(Wb.reshape(g.Nv, g.Nc, g.Nr * K), g.N, g.Nr, K, th, svb, sxb, iters=mbir_run, momentum=True)
        np.savez(save, D0=D0, W0=W0, xh=xh, obj=obj, D=D, xh_bf16=oracle.expand(xsb, Db, g.N, g.Nr))
    return {"value": vb / total, "seconds_scaled": total, "seconds_run": sum(t.values()), "threads": threads,
            "stage_s": {k: round(v, 3) for k, v in t.items()}, "nmf_run": nmf_run, "mbir_run": mbir_run}


def synth_counts(pb):
    from paper_2410_22500_gb300 import synth

    return synth.counts_numpy(pb)


def _sample_desc(nmf_run, mbir_run, cores):
    return ("one slice (Nr=1) of the 256^3 / Nk=1500 / K=6 workload (256x256 image, 120 views, 256 bins), FP64 "
            "oracle on %d host thread%s, every stage; NMF %d of %d and MBIR %d of %d iterations run, scaled "
            "linearly" % (cores, "" if cores == 1 else "s", nmf_run, NMF_ITERS, mbir_run, MBIR_ITERS))


def run_oracle_subprocess(nmf_run, mbir_run, threads, save=None):
    """The oracle sample in a fresh interpreter, so that its thread count (OpenMP and
    the BLAS inside the SVD) is set before any library starts."""
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = str(threads)
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-sample", str(nmf_run), str(mbir_run), str(threads)]
    if save:
        cmd += ["--save", save]
    out = subprocess.run(cmd, env=env, capture_output=True, text=True, check=True)
    return json.loads(out.stdout.strip().splitlines()[-1])


# ---------------------------------------------------------------------------- GPU arm
def accuracy_check(ctx, ref_path, nmf_run, mbir_run):
    """x^h of the GPU path against the FP64 oracle on the one-slice sample: the same
    counts, the same start (the oracle's NNDSVD factors), the same iteration counts,
    through the library's normalise / decompose / reconstruct / expand calls in the
    benchmark's precision (BF16 P, FP32 x^h)."""
    import torch
    from paper_2410_22500_gb300 import fhr

    ref = np.load(ref_path)
    pb = one_slice()
    g = pb.geom
    y, y0 = synth_counts(pb)
    yd = torch.from_numpy(y.view(np.int16)).cuda()
    y0d = torch.from_numpy(y0.view(np.int16)).cuda()
    P = ctx.normalise(yd, y0d, p_dtype=fhr.BF16)
    D = torch.from_numpy(ref["D0"].astype(np.float32)).cuda()
    W = torch.from_numpy(ref["W0"].astype(np.float32)).cuda()
    D, W, obj = ctx.decompose(P, pb.Nk, K, nmf_run, D=D, W=W)
    xs = ctx.reconstruct(W.view(g.Nv, g.Nc, g.Nr * K), g.N, g.Nr, K, mbir_run, momentum=True)
    xh = ctx.expand(xs, D, g.N, g.Nr, xh_dtype=fhr.F32)
    torch.cuda.synchronize()
    got = xh.cpu().numpy().astype(np.float64)

    def errs(want):
        err = got - want
        return (float(np.linalg.norm(err) / np.linalg.norm(want)), float(np.abs(err).max() / np.abs(want).max()))

    rel_l2, max_rel = errs(ref["xh"])
    par_l2, par_max = errs(ref["xh_bf16"])
    o_gpu, o_ref = float(obj[-1].item()), float(ref["obj"][-1])
    return {"sample": "one slice (Nr=1) of the workload: 256x256 image, 120 views, 256 bins, Nk=1500, K=6, "
                      "I0=100, seeded counts",
            "start": "the oracle's NNDSVD factors (exact SVD), given to both sides",
            "path": "fhr_normalise (BF16 P) -> fhr_decompose -> fhr_reconstruct (momentum) -> fhr_expand (FP32)",
            "nmf_iters": nmf_run, "mbir_iters": mbir_run,
            "xh_rel_l2": rel_l2, "xh_max_abs_over_max": max_rel,
            "objective_rel": abs(o_gpu - o_ref) / o_ref,
            "parity_on_bf16_data": {"xh_rel_l2": par_l2, "xh_max_abs_over_max": par_max,
                                    "note": "against the FP64 oracle run on P rounded to BF16: what the GPU's "
                                            "arithmetic adds to the BF16 form's own error"},
            "bound": 1e-3,
            "within_bound": bool(rel_l2 <= 1e-3 and par_l2 <= 1e-3 and par_max <= 1e-3)}


def run_ours(args, rank, world, device):
    import torch
    from paper_2410_22500_gb300 import build as fbuild
    from paper_2410_22500_gb300 import fhr

    fbuild.build()
    torch.cuda.set_device(device)
    ctx = fhr.Context(device)
    pb = workload()
    g = pb.geom
    from paper_2410_22500_gb300 import synth

    y, y0 = synth.counts_torch(pb, device="cuda:%d" % device)
    prm = ctx.pipeline_params(Nv=g.Nv, Nr=g.Nr, Nc=g.Nc, Nk=pb.Nk, N=g.N, K=K, nmf_iters=NMF_ITERS,
                              mbir_iters=MBIR_ITERS, momentum=True, seed=17, p_dtype=fhr.BF16, xh_dtype=fhr.F32)
    ldP = prm.nmf.ldP
    ws, ws_bytes = ctx.pipeline_workspace(prm)
    D = torch.empty((pb.Nk, K), dtype=torch.float32, device=device)
    xh = torch.empty((g.Nr, g.N, g.N, pb.Nk), dtype=torch.float32, device=device)
    obj = torch.empty(NMF_ITERS, dtype=torch.float64, device=device)
    stream = ctx.stream

    def step():
        ctx.pipeline(prm, y, y0, D, xh, obj=obj, ws=ws, ws_bytes=ws_bytes)

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
    fams = {n: ctx.profile_read(n) for n in ("normalise", "nndsvd_pass", "nmf_pass", "nmf_reduce", "nmf_update",
                                             "proj_fwd", "mbir_update", "expand")}
    ctx.profile(False)
    clk = clocks.stop()
    if ctx.status(ws) != 0:
        raise RuntimeError("device status after timed steps")
    final_obj = float(obj[-1].item())
    ms = max_over_ranks(ms, device)
    ms_step = ms / args.steps
    vb = g.Nr * g.N * g.N * pb.Nk
    value = whole_job_value(world, vb, ms_step)

    # ---- end to end through the C ABI with pinned host buffers (counts in, x^h out)
    prm_h = ctx.pipeline_params(Nv=g.Nv, Nr=g.Nr, Nc=g.Nc, Nk=pb.Nk, N=g.N, K=K, nmf_iters=NMF_ITERS,
                                mbir_iters=MBIR_ITERS, momentum=True, seed=17, p_dtype=fhr.BF16, xh_dtype=fhr.F32,
                                host_io=True)
    del ws, xh
    torch.cuda.empty_cache()
    y_h = torch.empty(y.shape, dtype=y.dtype, pin_memory=True)
    y_h.copy_(y)
    y0_h = torch.empty(y0.shape, dtype=y0.dtype, pin_memory=True)
    y0_h.copy_(y0)
    del y, y0
    torch.cuda.empty_cache()
    ws_h, wsb_h = ctx.pipeline_workspace(prm_h)
    xh_h = torch.empty((g.Nr, g.N, g.N, pb.Nk), dtype=torch.float32, pin_memory=True)
    h2d = y_h.numel() * 2 + y0_h.numel() * 2
    d2h = xh_h.numel() * 4

    def step_h():
        ctx.pipeline(prm_h, y_h, y0_h, D, xh_h, obj=obj, ws=ws_h, ws_bytes=wsb_h)

    step_h()
    ctx.io_join()
    torch.cuda.synchronize()
    e2e_steps = max(2, min(args.steps, 5))
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
    del ws_h, xh_h, y_h, y0_h
    torch.cuda.empty_cache()

    peak, peak_kind = _peaks()
    pass_n, pass_ms = fams["nmf_pass"]
    pass_bytes = algorithmic_pass_bytes(g.Np, pb.Nk, 2, K)
    achieved = pass_bytes / (pass_ms / pass_n / 1e3) / 1e9 if pass_n else None
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "nmf_pass_traffic.json")
    if os.path.exists(tpath):
        try:
            with open(tpath) as f:
                tr = json.load(f)
            if (tr.get("source_digest") == fbuild.kernel_digest("nmf_pass") and tr.get("p_dtype") == "bf16"
                    and tr.get("ldP") == ldP):
                # scaled from the captured case by rows (traffic grows with the rows streamed)
                traffic = tr["bytes_per_row"] * g.Np
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
        "dtype": "bf16",
        "data": "synthetic (seeded ellipsoid phantom, Bragg-edge spectra, Poisson counts)",
        "config": {"workload": WORKLOAD, "Np": g.Np, "Nk": pb.Nk, "ldP": ldP, "Nx": g.Nx, "K": K,
                   "nmf_iters": NMF_ITERS, "mbir_iters": MBIR_ITERS, "init": "nndsvd",
                   "mbir": "SQS + momentum, qGGMRF p=1.2 q=2 T=1",
                   "precision": "P in BF16, FP32 accumulation in every contraction, FP64 Gram matrices, objective "
                                "and D normalisation; projector, MBIR and x^h in FP32",
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "l2": "inputs larger than L2 (P is 23.7 GB, x^h 100.7 GB per step)"},
        "e2e": {"value": whole_job_value(world, vb, e2e_ms), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms, "steps": e2e_steps,
                "note": "pinned host counts in, pinned host x^h (FP32) out, on two copy streams; consecutive "
                        "calls overlap their copies with each other's compute"},
        "gpu_launches": int(launches),
        "roofline": {"bound": "hbm", "kernel": "nmf_mma_kernel (fused fast-HALS pass, BF16 P)", "achieved": achieved,
                     "peak": peak, "peak_kind": "%s (MEASURED_PEAKS.json hbm_gbs)" % peak_kind
                     if peak_kind == "measured" else "fallback", "unit": "GB/s",
                     "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                     "frac_of_nominal_7900": (achieved / 7900.0) if achieved else None,
                     "algorithmic_bytes_per_launch": pass_bytes, "launches": pass_n,
                     "avg_launch_ms": pass_ms / pass_n if pass_n else None},
        "kernel_ms": {n: {"launches": c, "total_ms": t} for n, (c, t) in fams.items()},
        "final_objective": final_obj,
        "clocks": clk,
    }
    return ctx, out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--oracle-sample", nargs=3, type=int, default=None, help=argparse.SUPPRESS)
    ap.add_argument("--save", default=None, help=argparse.SUPPRESS)
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.oracle_sample:
        # one timed oracle sample (a child of this script, with its thread count fixed)
        import oracle

        oracle.build()
        n1, n2, th = args.oracle_sample
        print(json.dumps(oracle_sample(n1, n2, th, save=args.save)))
        return

    if args.impl == "reference":
        # the reference arm is the FP64 CPU oracle, timed as it stands on the host cores
        if rank != 0:
            return
        import oracle

        oracle.build()
        cores, model = cpu_info()
        n1, n2 = SAMPLE_REFERENCE
        oracle.set_threads(cores)
        for _ in range(args.warmup):
            oracle_sample(1, 1, cores)
        vals = [oracle_sample(n1, n2, cores)["value"] for _ in range(args.steps)]
        v = statistics.median(vals)
        print(json.dumps({"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 0,
                          "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
                          "dtype": "f64", "data": "synthetic",
                          "config": {"workload": WORKLOAD + " (one slice)"},
                          "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "cpu": model, "kind": "oracle",
                                           "sample": _sample_desc(n1, n2, cores)},
                          "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
        return

    if world > 1:
        import torch
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    ctx, out = run_ours(args, rank, world, local)
    if rank == 0 and not args.no_cpu_baseline:
        import oracle

        oracle.build()
        cores, model = cpu_info()
        with tempfile.TemporaryDirectory() as td:
            ref_path = os.path.join(td, "oracle_sample.npz")
            allc = run_oracle_subprocess(*SAMPLE_ALL_CORES, cores, save=ref_path)
            out["accuracy"] = accuracy_check(ctx, ref_path, *SAMPLE_ALL_CORES)
        one = run_oracle_subprocess(*SAMPLE_ONE_CORE, 1)
        out["cpu_baseline"] = {"value": allc["value"], "unit": UNIT, "cores": allc["threads"], "cpu": model,
                               "kind": "oracle", "sample": _sample_desc(*SAMPLE_ALL_CORES, allc["threads"]),
                               "seconds_scaled": allc["seconds_scaled"], "seconds_run": allc["seconds_run"],
                               "stage_s": allc["stage_s"],
                               "single_thread": {"value": one["value"], "cores": 1,
                                                 "sample": _sample_desc(*SAMPLE_ONE_CORE, 1),
                                                 "seconds_scaled": one["seconds_scaled"],
                                                 "seconds_run": one["seconds_run"], "stage_s": one["stage_s"]}}
    ctx.close()
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist

        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
