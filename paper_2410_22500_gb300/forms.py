"""Measurements of the added forms of the path on synthetic workloads (one JSON
line per case; device timing with CUDA events on the library's stream).

    python -m paper_2410_22500_gb300.forms precision
    python -m paper_2410_22500_gb300.forms batched [n_problems] [iters]

`precision`: the 256^3 volume (6 ellipsoids, Nk = 1500, 120 views, 256 x 256
detector, 100 counts per bin; P is 7.86M x 1500) through Algorithm 1 with P
streamed as BF16 and, for comparison, as FP32 (x^h written as BF16 in both):
whole-pipeline time, voxel*bins/s, per-kernel-family times and the fused
pass's HBM rate.  The error of the BF16 form against FP64 is measured by the
GPU tests (tests/test_gpu_forms.py), where the FP64 reference can run.

`batched`: 40 uneven 2-D problems (N in 64..512 step 16, Nc = N, 45..180
views, K in 3..8; problem i seeded with 2000 + i), sinograms made by the
library's projector from seeded disk phantoms.  Times the batched
reconstruction (one persistent launch, autotuned work-item size) against one
fhr_reconstruct call per problem, both including their set-up, and reports the
per-problem times of the latter.
"""
import json
import sys

import numpy as np
import torch

from . import build, fhr, synth

K_PRECISION = 6
NMF_ITERS = 200
MBIR_ITERS = 100


def _timed(ctx, fn):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(ctx.stream)
    fn()
    e1.record(ctx.stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def precision() -> None:
    build.build()
    ctx = fhr.Context(0)
    pb = synth.volume_3d_bf16()
    g = pb.geom
    y, y0 = synth.counts_torch(pb, device="cuda")
    D = torch.empty((pb.Nk, K_PRECISION), dtype=torch.float32, device="cuda")
    obj = torch.empty(NMF_ITERS, dtype=torch.float64, device="cuda")
    xh = torch.empty((g.Nr, g.N, g.N, pb.Nk), dtype=torch.bfloat16, device="cuda")
    for p_dtype, name in ((fhr.BF16, "bf16"), (fhr.F32, "f32")):
        prm = ctx.pipeline_params(Nv=g.Nv, Nr=g.Nr, Nc=g.Nc, Nk=pb.Nk, N=g.N, K=K_PRECISION, nmf_iters=NMF_ITERS,
                                  mbir_iters=MBIR_ITERS, momentum=True, seed=17, p_dtype=p_dtype,
                                  xh_dtype=fhr.BF16)
        ws, wsb = ctx.pipeline_workspace(prm)
        run = lambda: ctx.pipeline(prm, y, y0, D, xh, obj=obj, ws=ws, ws_bytes=wsb)
        run()   # warm-up
        ctx.check(ctx.status(ws))
        ctx.profile(True)
        ms = _timed(ctx, run)
        fams = {n: ctx.profile_read(n) for n in ("normalise", "nndsvd_pass", "nmf_pass", "nmf_reduce", "nmf_update",
                                                 "proj_fwd", "mbir_update", "expand")}
        ctx.profile(False)
        ctx.check(ctx.status(ws))
        es = 2 if p_dtype == fhr.BF16 else 4
        n, pms = fams["nmf_pass"]
        pass_bytes = g.Np * prm.nmf.ldP * es + 2 * g.Np * K_PRECISION * 4
        vb = g.Nr * g.N * g.N * pb.Nk
        print(json.dumps({
            "case": "precision", "p_dtype": name, "workload": "256^3 volume, Nk=1500, 120 views, K=6, 100 counts/bin",
            "nmf_iters": NMF_ITERS, "mbir_iters": MBIR_ITERS, "pipeline_ms": round(ms, 2),
            "voxel_bins_per_s": vb / (ms / 1e3),
            "nmf_pass_ms": round(pms / n, 4) if n else None,
            "nmf_pass_gbs": round(pass_bytes / (pms / n / 1e3) / 1e9, 1) if n else None,
            "kernel_ms": {k: round(v[1], 2) for k, v in fams.items()},
            "final_objective": float(obj[-1].item())}), flush=True)
        del ws
        torch.cuda.empty_cache()
    ctx.close()


def _batch_shapes(n_problems: int):
    out = []
    for i in range(n_problems):
        rng = np.random.default_rng(2000 + i)
        N = int(rng.integers(4, 33)) * 16
        Nv = int(rng.integers(45, 181))
        K = int(rng.integers(3, 9))
        out.append((N, Nv, K))
    return out


def batched(n_problems: int = 40, iters: int = 100) -> None:
    build.build()
    ctx = fhr.Context(0)
    shapes = _batch_shapes(n_problems)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(2000)
    sinos = []
    for N, Nv, K in shapes:
        yy, xx = torch.meshgrid(torch.arange(N, device="cuda"), torch.arange(N, device="cuda"), indexing="ij")
        r = ((yy - N / 2) ** 2 + (xx - N / 2) ** 2).sqrt()
        x = (r < 0.4 * N).float()[..., None] * (0.5 + torch.rand((1, 1, K), device="cuda", generator=gen))
        sinos.append(ctx.project(x.contiguous(), N, Nv))
    Ns, Ks = [s[0] for s in shapes], [s[2] for s in shapes]
    _, tile = ctx.reconstruct_batch(sinos, Ns, Ks, 4, autotune=True)
    out = {}
    t_batch = _timed(ctx, lambda: out.__setitem__("xb", ctx.reconstruct_batch(sinos, Ns, Ks, iters, tile=tile)[0]))
    t_setup = _timed(ctx, lambda: ctx.reconstruct_batch(sinos, Ns, Ks, 0, tile=tile))
    ctx.reconstruct(sinos[0], Ns[0], 1, Ks[0], 2)
    per, xs = [], []
    for s, N, K in zip(sinos, Ns, Ks):
        box = {}
        per.append(round(_timed(ctx, lambda: box.__setitem__("x", ctx.reconstruct(s, N, 1, K, iters))), 3))
        xs.append(box["x"])
    worst = max(float(((a - b).norm() / b.norm().clamp_min(1e-30)).item()) for a, b in zip(out["xb"], xs))
    vox = sum(N * N * K for N, _, K in shapes)
    t_seq = sum(per)
    print(json.dumps({"case": "batched", "problems": n_problems, "iters": iters, "tile": tile,
                      "batched_ms": round(t_batch, 2), "batched_setup_ms": round(t_setup, 2),
                      "per_problem_total_ms": round(t_seq, 2), "speedup": round(t_seq / t_batch, 3),
                      "voxel_channel_iters_per_s": vox * iters / (t_batch / 1e3),
                      "max_rel_diff_vs_per_problem": worst,
                      "per_problem": [{"N": N, "Nv": Nv, "K": K, "ms": t} for (N, Nv, K), t in zip(shapes, per)]}))
    ctx.close()


if __name__ == "__main__":
    case = sys.argv[1] if len(sys.argv) > 1 else "precision"
    if case == "precision":
        precision()
    elif case == "batched":
        batched(int(sys.argv[2]) if len(sys.argv) > 2 else 40, int(sys.argv[3]) if len(sys.argv) > 3 else 100)
    else:
        raise SystemExit("unknown case %r" % case)
