"""Measurements of the added forms of the path on synthetic workloads (one JSON
line per case; device timing with CUDA events on the library's stream).

    python -m paper_2410_22500_gb300.forms precision
    python -m paper_2410_22500_gb300.forms batched [n_problems] [iters]
    python -m paper_2410_22500_gb300.forms learned [n_train]
    python -m paper_2410_22500_gb300.forms fbp_fmd
    python -m paper_2410_22500_gb300.forms dhr
    python -m paper_2410_22500_gb300.forms ns_sweep

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

`learned`: the learned warm start with BF16 P against the plain FP32 form.
A 1500 -> 256 -> 128 -> 6 MLP (GELU, GELU, softplus; BF16 weights in the
forward, FP32 accumulation) is trained by the library's kernels on the plain
method's coefficients (NNDSVD start, 100 iterations) for n_train (default
2000) seeded 128x128x32 phantoms (120 views, 128 x 32 detector, 50
counts/bin; 2048 sampled pixel rows each) whose six materials share one
spectra library.  A held-out 256x256x128 volume
(Nk = 1500, 120 views, 256 x 128 detector, 50 counts/bin) is then run through
Algorithm 1 twice: the plain FP32 form (NNDSVD start, 200 iterations) and the
learned + BF16 form with the fewest iterations whose factors reach the plain
final objective within 1e-3 relative, both objectives evaluated against the
FP32 P.  Reports iterations, whole-pipeline times and the speedup; also the
plain form stopped at the iteration where it first came within 1e-3 of its own
final objective, and the BF16 form from the NNDSVD start with the fewest
iterations that reach the same target (what the learned start adds to BF16).

`dhr`: the comparison of the paper's Table II on the 3-D workload's shapes (no dead
bins): direct reconstruction of every wavelength bin by FBP (DHR; the bins in slabs
of 64, each slab one fhr_fbp call on P's columns viewed as a sinogram) against FHR
with FBP and FHR with MBIR; whole-path times and SNR_FHR (Eq. snr_fhr) of each x^h
over the phantom's pure voxels (per material) and air at least 3 pixels from any
material (background).  A timing reference for the per-bin path, not a product path.

`ns_sweep`: the subspace-dimension experiment of Sec. V-D on a synthetic 3-material
volume (128 x 128 x 32, Nk = 1200, 90 views, 200 counts/bin): for N_s = 1..8 (the
fused pass takes K <= 8) the path (NNDSVD start, 200 NMF and 100 MBIR iterations)
then semi-supervised FMD with the pure voxels as regions; the relative error of each
estimated material spectrum against the phantom's, and SNR_FMD (Eq. snr_fmd) of x^m.

`fbp_fmd`: the 3-D f32 workload (the benchmark's) through Algorithm 1 with the
MBIR and with the FBP reconstruction (200 NMF iterations; 100 SQS iterations),
whole-pipeline times and the FBP kernels' times; then the semi-supervised FMD
(Algorithm 2 after the reconstruction) of its MBIR subspace volume with the
phantom's pure voxels as the user regions: the time of fhr_fmd, its HBM rate
against the algorithmic bytes, and the relative error of each estimated
material spectrum D^m against the phantom's over the live bins.
"""
import ctypes
import json
import sys
import time

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
        pass_bytes = g.Np * pb.Nk * es + 2 * g.Np * K_PRECISION * 4   # the live bins (row padding not counted)
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
    _, tile, vw = ctx.reconstruct_batch(sinos, Ns, Ks, 4, autotune=True)
    out = {}
    t_batch = _timed(ctx, lambda: out.__setitem__("xb", ctx.reconstruct_batch(sinos, Ns, Ks, iters, tile=tile,
                                                                              vw=vw)[0]))
    t_setup = _timed(ctx, lambda: ctx.reconstruct_batch(sinos, Ns, Ks, 0, tile=tile, vw=vw))
    # the default tile shape, for comparison with the tuned one
    t_default = _timed(ctx, lambda: ctx.reconstruct_batch(sinos, Ns, Ks, iters))
    ctx.reconstruct(sinos[0], Ns[0], 1, Ks[0], 2)
    per, xs = [], []
    for s, N, K in zip(sinos, Ns, Ks):
        box = {}
        per.append(round(_timed(ctx, lambda: box.__setitem__("x", ctx.reconstruct(s, N, 1, K, iters))), 3))
        xs.append(box["x"])
    worst = max(float(((a - b).norm() / b.norm().clamp_min(1e-30)).item()) for a, b in zip(out["xb"], xs))
    vox = sum(N * N * K for N, _, K in shapes)
    t_seq = sum(per)
    print(json.dumps({"case": "batched", "problems": n_problems, "iters": iters, "tile": tile, "vw": vw,
                      "batched_ms": round(t_batch, 2), "batched_setup_ms": round(t_setup, 2),
                      "batched_default_tile_ms": round(t_default, 2),
                      "per_problem_total_ms": round(t_seq, 2), "speedup": round(t_seq / t_batch, 3),
                      "voxel_channel_iters_per_s": vox * iters / (t_batch / 1e3),
                      "max_rel_diff_vs_per_problem": worst,
                      "per_problem": [{"N": N, "Nv": Nv, "K": K, "ms": t} for (N, Nv, K), t in zip(shapes, per)]}))
    ctx.close()


def _objective(P, Nk, D, W, rows=131072):
    """||P - W D^T||_F^2 against the FP32 P, FP64 accumulation (evaluation only)."""
    tot = 0.0
    for r0 in range(0, P.shape[0], rows):
        R = P[r0:r0 + rows, :Nk].float() - W[r0:r0 + rows] @ D.T
        tot += float((R.double() ** 2).sum().item())
    return tot


def _first_within(obj, target):
    hit = np.nonzero(np.asarray(obj) <= target)[0]
    return int(hit[0]) + 1 if len(hit) else None


def learned(n_train: int = 2000, rows_per_phantom: int = 2048, target_iters: int = 100) -> None:
    from . import learned as lw

    build.build()
    torch.backends.cuda.matmul.allow_tf32 = False
    ctx = fhr.Context(0)
    Nk, K, H1, H2, iters = 1500, 6, 256, 128, 200
    lib = synth.spectra_library(Nk, K, seed=77)
    ldb = (Nk + 7) // 8 * 8
    # training set: plain-method coefficients (NNDSVD start, target_iters iterations) on the
    # BF16 P of n_train seeded 128x128x32 phantoms, rows_per_phantom pixel rows sampled from each
    gen = torch.Generator(device="cuda")
    gen.manual_seed(5)
    X = torch.empty((n_train * rows_per_phantom, ldb), dtype=torch.bfloat16, device="cuda")
    T = torch.empty((n_train * rows_per_phantom, K), dtype=torch.float32, device="cuda")
    t_gen = time.perf_counter()
    for i in range(n_train):
        pb = synth.make_problem(N=128, Nr=32, Nc=128, Nv=120, Nk=Nk, Nm=K, I0=50, seed=5000 + i, spectra=lib,
                                three_d=True, device="cuda")
        y, y0 = synth.counts_torch(pb, device="cuda")
        Pb = ctx.normalise(y, y0, p_dtype=fhr.BF16)
        D, W, _ = ctx.decompose(Pb, Nk, K, target_iters, init=fhr.INIT_NNDSVD, obj=False)
        perm = torch.as_tensor(lw.match_order(D.cpu().numpy(), lib), device="cuda")
        idx = torch.randint(0, Pb.shape[0], (rows_per_phantom,), device="cuda", generator=gen)
        X[i * rows_per_phantom:(i + 1) * rows_per_phantom] = Pb[idx]
        T[i * rows_per_phantom:(i + 1) * rows_per_phantom] = W[idx][:, perm]
        del y, y0, Pb, W
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t_gen
    dims = ctx.mlp_dims(Nk, H1, H2, K, ldx=ldb, x_bf16=True, weights_bf16=True)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0[0].record(ctx.stream)
    steps, batch = 6000, 8192
    prm, hist = lw.train(ctx, dims, X, T, steps=steps, batch=batch, lr=2e-3, log_every=1000)
    t0[1].record(ctx.stream)
    torch.cuda.synchronize()
    train_ms = t0[0].elapsed_time(t0[1])
    del X, T
    torch.cuda.empty_cache()

    held = synth.make_problem(N=256, Nr=128, Nc=256, Nv=120, Nk=Nk, Nm=K, I0=50, seed=6000, spectra=lib,
                              three_d=True)
    g = held.geom
    y, y0 = synth.counts_torch(held, device="cuda")
    # objectives against the FP32 P
    P32 = ctx.normalise(y, y0)
    Dp, Wp, obj_p = ctx.decompose(P32, Nk, K, iters, init=fhr.INIT_NNDSVD)
    f_plain = _objective(P32, Nk, Dp, Wp)
    obj_p = obj_p.cpu().numpy()
    n_plain_tol = _first_within(obj_p, obj_p[-1] * (1 + 1e-3))
    del Wp
    Pb = ctx.normalise(y, y0, p_dtype=fhr.BF16)
    target = f_plain * (1 + 1e-3)

    def reach(**kw):
        """Fewest iterations on the BF16 P whose factors reach the target on the FP32 P."""
        D_, W_, ob = ctx.decompose(Pb, Nk, K, iters, **kw)
        ob = ob.cpu().numpy()
        off = _objective(P32, Nk, D_, W_) - float(ob[-1])   # FP32-P minus BF16-P objective near the end
        del W_
        n_ = _first_within(ob + off, target) or iters
        f_ = None
        while n_ <= iters:
            D_, W_, _ = ctx.decompose(Pb, Nk, K, n_, obj=False, **kw)
            f_ = _objective(P32, Nk, D_, W_)
            del W_
            if f_ <= target:
                break
            n_ += 1
        return min(n_, iters), f_

    n, f_learn = reach(mlp=(dims, prm))
    n_pb, f_pb = reach(init=fhr.INIT_NNDSVD)
    reached = f_learn is not None and f_learn <= target
    del P32, Pb
    torch.cuda.empty_cache()

    xh = torch.empty((g.Nr, g.N, g.N, Nk), dtype=torch.bfloat16, device="cuda")
    Dout = torch.empty((Nk, K), dtype=torch.float32, device="cuda")

    def run_pipeline(p_dtype, init, nmf_iters):
        prm_p = ctx.pipeline_params(Nv=g.Nv, Nr=g.Nr, Nc=g.Nc, Nk=Nk, N=g.N, K=K, nmf_iters=nmf_iters,
                                    mbir_iters=MBIR_ITERS, momentum=True, p_dtype=p_dtype, xh_dtype=fhr.BF16,
                                    init=init)
        if init == fhr.INIT_LEARNED:
            # the network reads the pipeline's own P rows (its row stride)
            dims_p = ctx.mlp_dims(Nk, H1, H2, K, ldx=prm_p.norm.ldP, x_bf16=True, weights_bf16=True)
            prm_p.nmf.mlp = ctypes.addressof(dims_p)
            prm_p.nmf.mlp_params = prm.data_ptr()
        ws, wsb = ctx.pipeline_workspace(prm_p)
        ob = torch.empty(max(nmf_iters, 1), dtype=torch.float64, device="cuda")
        go = lambda: ctx.pipeline(prm_p, y, y0, Dout, xh, obj=ob, ws=ws, ws_bytes=wsb)
        go()
        ctx.check(ctx.status(ws))
        ctx.profile(True)
        ms = _timed(ctx, go)
        fams = {k: round(ctx.profile_read(k)[1], 2) for k in ("normalise", "nndsvd_pass", "nmf_pass", "mlp_forward",
                                                              "proj_fwd", "mbir_update", "expand")}
        ctx.profile(False)
        ctx.check(ctx.status(ws))
        del ws
        torch.cuda.empty_cache()
        return ms, fams

    t_plain, k_plain = run_pipeline(fhr.F32, fhr.INIT_NNDSVD, iters)
    t_plain_tol, _ = run_pipeline(fhr.F32, fhr.INIT_NNDSVD, n_plain_tol)
    t_lb, k_lb = run_pipeline(fhr.BF16, fhr.INIT_LEARNED, n)
    t_pb, _ = run_pipeline(fhr.BF16, fhr.INIT_NNDSVD, n_pb)
    vb = g.Nr * g.N * g.N * Nk
    print(json.dumps({
        "case": "learned", "workload": "256x256x128 volume, Nk=1500, 120 views, K=6, 50 counts/bin",
        "train": {"phantoms": n_train, "rows": n_train * rows_per_phantom, "target_iters": target_iters,
                  "set_s": round(t_gen, 1), "steps": steps, "batch": batch, "ms": round(train_ms, 1), "loss": hist},
        "plain_f32": {"iters": iters, "objective_fp32P": f_plain, "pipeline_ms": round(t_plain, 2),
                      "voxel_bins_per_s": vb / (t_plain / 1e3), "kernel_ms": k_plain},
        "plain_f32_own_tol": {"iters": n_plain_tol, "pipeline_ms": round(t_plain_tol, 2)},
        "learned_bf16": {"iters": n, "objective_fp32P": f_learn, "reached_plain_within_1e-3": bool(reached),
                         "rel_to_plain": (f_learn / f_plain - 1.0) if f_learn else None,
                         "pipeline_ms": round(t_lb, 2), "voxel_bins_per_s": vb / (t_lb / 1e3), "kernel_ms": k_lb},
        "plain_bf16_nndsvd": {"iters": n_pb, "objective_fp32P": f_pb,
                              "reached_plain_within_1e-3": bool(f_pb is not None and f_pb <= target),
                              "pipeline_ms": round(t_pb, 2)},
        "speedup_vs_plain_f32": round(t_plain / t_lb, 3),
        "speedup_vs_plain_f32_own_tol": round(t_plain_tol / t_lb, 3),
        "speedup_vs_bf16_nndsvd": round(t_pb / t_lb, 3)}), flush=True)
    ctx.close()


def fbp_fmd() -> None:
    build.build()
    ctx = fhr.Context(0)
    pb = synth.volume_3d_f32()
    g = pb.geom
    K = 5
    y, y0 = synth.counts_torch(pb, device="cuda")
    dead = torch.from_numpy(pb.dead_bins).cuda()
    D = torch.empty((pb.Nk, K), dtype=torch.float32, device="cuda")
    xh = torch.empty((g.Nr, g.N, g.N, pb.Nk), dtype=torch.float32, device="cuda")
    vb = g.Nr * g.N * g.N * pb.Nk
    out = {"case": "fbp_fmd", "workload": "128x128x64 volume, Nk=1200, 90 views, 64x128 detector, K=5"}
    for name, recon in (("mbir", fhr.RECON_MBIR), ("fbp", fhr.RECON_FBP)):
        prm = ctx.pipeline_params(Nv=g.Nv, Nr=g.Nr, Nc=g.Nc, Nk=pb.Nk, N=g.N, K=K, nmf_iters=NMF_ITERS,
                                  mbir_iters=MBIR_ITERS, momentum=True, seed=17, recon=recon)
        ws, wsb = ctx.pipeline_workspace(prm)
        run = lambda: ctx.pipeline(prm, y, y0, D, xh, dead=dead, ws=ws, ws_bytes=wsb)
        run()
        ctx.check(ctx.status(ws))
        ctx.profile(True)
        ms = _timed(ctx, run)
        fams = {k: round(ctx.profile_read(k)[1], 3) for k in ("nmf_pass", "proj_fwd", "mbir_update", "fbp_filter",
                                                              "proj_bwd", "expand")}
        ctx.profile(False)
        ctx.check(ctx.status(ws))
        out["pipeline_" + name] = {"ms": round(ms, 2), "voxel_bins_per_s": vb / (ms / 1e3), "kernel_ms": fams}
        del ws
        torch.cuda.empty_cache()
    # FMD of the MBIR subspace volume, the phantom's pure voxels as the user regions
    P = ctx.normalise(y, y0, dead=dead)
    Ds, W, _ = ctx.decompose(P, pb.Nk, K, NMF_ITERS, init=fhr.INIT_NNDSVD, obj=False)
    del P
    xs = ctx.reconstruct(W.view(g.Nv, g.Nc, g.Nr * K), g.N, g.Nr, K, MBIR_ITERS, momentum=True)
    frac = synth.volume_fractions(pb.phantom, g.N, g.Nr)             # [Nr][N][N][Nm]
    Nm = frac.shape[-1]
    lab = np.where(frac.max(axis=-1) >= 0.999, frac.argmax(axis=-1) + 1, 0).astype(np.uint8)
    labels = torch.from_numpy(np.ascontiguousarray(lab.transpose(1, 2, 0))).cuda()   # voxel order (iy, ix, r)
    T, xm, Dm = ctx.fmd(xs, labels, Ds, Nm)
    ctx.profile(True)
    ms = _timed(ctx, lambda: ctx.fmd(xs, labels, Ds, Nm, check_status=False))
    n_fmd, fmd_ms = ctx.profile_read("fmd")
    ctx.profile(False)
    Nx = g.N * g.N * g.Nr
    nbytes = 2 * Nx * K * 4 + 2 * Nx + Nx * Nm * 4      # x^s twice, labels twice, x^m once
    live = pb.dead_bins == 0
    Dm_h = Dm.cpu().numpy().astype(np.float64)[live]
    mu = pb.spectra[live]
    err = [float(np.linalg.norm(Dm_h[:, m] - mu[:, m]) / np.linalg.norm(mu[:, m])) for m in range(Nm)]
    out["fmd"] = {"voxels": Nx, "Ns": K, "Nm": Nm, "labelled_voxels": int((lab > 0).sum()),
                  "ms": round(fmd_ms / max(n_fmd, 1), 4), "gbs": round(nbytes / (fmd_ms / max(n_fmd, 1) / 1e3) / 1e9, 1),
                  "algorithmic_bytes": nbytes, "Dm_rel_err_per_material": [round(e, 4) for e in err]}
    print(json.dumps(out), flush=True)
    ctx.close()


def _rois(pb, margin=3):
    """Region labels in voxel order (r, iy, ix): m + 1 on the pure voxels of material m,
    background on air at least `margin` pixels (in-plane) from every material."""
    from scipy import ndimage

    g = pb.geom
    frac = synth.volume_fractions(pb.phantom, g.N, g.Nr)             # [Nr][N][N][Nm]
    lab = np.where(frac.max(axis=-1) >= 0.999, frac.argmax(axis=-1) + 1, 0).astype(np.uint8)
    any_mat = frac.sum(axis=-1) > 0
    near = ndimage.binary_dilation(any_mat, structure=np.ones((1, 2 * margin + 1, 2 * margin + 1), bool))
    yy, xx = np.mgrid[0:g.N, 0:g.N] - 0.5 * (g.N - 1)
    inside = (yy ** 2 + xx ** 2) < (0.5 * g.N - 2) ** 2
    lab[(~near) & inside[None]] = fhr.ROI_BACKGROUND
    return lab, frac


def dhr() -> None:
    build.build()
    ctx = fhr.Context(0)
    pb = synth.scaled(synth.volume_3d_f32, dead_frac=0.0)
    g = pb.geom
    K, Kb = 5, 64
    y, y0 = synth.counts_torch(pb, device="cuda")
    lab, frac = _rois(pb)
    Nm = frac.shape[-1]
    roi_r = torch.from_numpy(lab.reshape(-1)).cuda()                                   # (r, iy, ix)
    roi_y = torch.from_numpy(np.ascontiguousarray(lab.transpose(1, 2, 0)).reshape(-1)).cuda()   # (iy, ix, r)
    vb = g.Nr * g.N * g.N * pb.Nk
    out = {"case": "dhr", "workload": "128x128x64 volume, Nk=1200, 90 views, 64x128 detector, 200 counts/bin, "
                                      "5 materials, K=5 (FHR)",
           "roi": {"materials": Nm, "signal_voxels": int(((lab > 0) & (lab < 255)).sum()),
                   "background_voxels": int((lab == 255).sum())}}
    # DHR: every bin reconstructed by FBP, in slabs of Kb bins
    P = ctx.normalise(y, y0)
    slabs = [(k0, min(pb.Nk, k0 + Kb)) for k0 in range(0, pb.Nk, Kb)]
    xs_slab = torch.empty((g.N, g.N, g.Nr * Kb), dtype=torch.float32, device="cuda")
    sino = torch.empty((g.Np, Kb), dtype=torch.float32, device="cuda")

    def run_dhr(measure):
        acc = []
        for k0, k1 in slabs:
            kb = k1 - k0
            s_ = sino.view(-1)[:g.Np * kb].view(g.Np, kb)        # contiguous [Np][kb]
            s_.copy_(P[:, k0:k1])
            xs = ctx.fbp(s_.view(g.Nv, g.Nc, g.Nr * kb), g.N,
                         xs=xs_slab.view(-1)[:g.N * g.N * g.Nr * kb].view(g.N, g.N, g.Nr * kb))
            if measure:
                db = float(ctx.snr(xs.view(-1, kb), roi_y, Nm, fhr.SNR_FHR).item())
                acc.append((kb, 10 ** (db / 10)))
        return acc

    run_dhr(False)
    t_dhr = _timed(ctx, lambda: run_dhr(False))
    parts = run_dhr(True)
    snr_dhr = 10 * np.log10(sum(kb * q for kb, q in parts) / sum(kb for kb, _ in parts))
    out["dhr_fbp"] = {"ms": round(t_dhr, 2), "slabs": len(slabs), "voxel_bins_per_s": vb / (t_dhr / 1e3),
                      "snr_fhr_db": round(float(snr_dhr), 3),
                      "note": "normalised P given; per slab a column copy of P then fhr_fbp"}
    del P, sino, xs_slab
    torch.cuda.empty_cache()
    D = torch.empty((pb.Nk, K), dtype=torch.float32, device="cuda")
    xh = torch.empty((g.Nr, g.N, g.N, pb.Nk), dtype=torch.float32, device="cuda")
    for name, recon in (("fhr_fbp", fhr.RECON_FBP), ("fhr_mbir", fhr.RECON_MBIR)):
        prm = ctx.pipeline_params(Nv=g.Nv, Nr=g.Nr, Nc=g.Nc, Nk=pb.Nk, N=g.N, K=K, nmf_iters=NMF_ITERS,
                                  mbir_iters=MBIR_ITERS, momentum=True, seed=17, recon=recon)
        ws, wsb = ctx.pipeline_workspace(prm)
        run = lambda: ctx.pipeline(prm, y, y0, D, xh, ws=ws, ws_bytes=wsb)
        run()
        ctx.check(ctx.status(ws))
        ms = _timed(ctx, run)
        ctx.check(ctx.status(ws))
        db = float(ctx.snr(xh.view(-1, pb.Nk), roi_r, Nm, fhr.SNR_FHR).item())
        out[name] = {"ms": round(ms, 2), "voxel_bins_per_s": vb / (ms / 1e3), "snr_fhr_db": round(db, 3),
                     "note": "whole path from the counts (normalise, NNDSVD, 200 NMF iterations, reconstruction, "
                             "expansion)"}
        del ws
        torch.cuda.empty_cache()
    print(json.dumps(out), flush=True)
    ctx.close()


def ns_sweep(max_ns: int = 8) -> None:
    build.build()
    ctx = fhr.Context(0)
    pb = synth.make_problem(N=128, Nr=32, Nc=128, Nv=90, Nk=1200, Nm=3, I0=200, seed=3003)
    g = pb.geom
    y, y0 = synth.counts_torch(pb, device="cuda")
    lab, frac = _rois(pb)
    Nm = frac.shape[-1]
    labels = torch.from_numpy(np.ascontiguousarray(np.where(lab == fhr.ROI_BACKGROUND, 0, lab).transpose(1, 2, 0))
                              ).cuda()
    roi = torch.from_numpy(np.ascontiguousarray(lab.transpose(1, 2, 0)).reshape(-1)).cuda()   # (iy, ix, r)
    P = ctx.normalise(y, y0)
    rows = []
    for Ns in range(1, max_ns + 1):
        t0 = time.perf_counter()
        Ds, W, _ = ctx.decompose(P, pb.Nk, Ns, NMF_ITERS, init=fhr.INIT_NNDSVD, obj=False)
        xs = ctx.reconstruct(W.view(g.Nv, g.Nc, g.Nr * Ns), g.N, g.Nr, Ns, MBIR_ITERS, momentum=True)
        row = {"Ns": Ns}
        if Ns >= Nm:
            T, xm, Dm = ctx.fmd(xs, labels, Ds, Nm)
            Dm_h = Dm.cpu().numpy().astype(np.float64)
            err = [float(np.linalg.norm(Dm_h[:, m] - pb.spectra[:, m]) / np.linalg.norm(pb.spectra[:, m]))
                   for m in range(Nm)]
            row["Dm_rel_err"] = [round(e, 4) for e in err]
            row["Dm_rel_err_mean"] = round(float(np.mean(err)), 4)
            row["snr_fmd_db"] = round(float(ctx.snr(xm, roi, Nm, fhr.SNR_FMD).item()), 3)
        else:
            row["note"] = "Ns < Nm: FMD needs at least as many subspace channels as materials"
        torch.cuda.synchronize()
        row["s"] = round(time.perf_counter() - t0, 3)
        rows.append(row)
        del Ds, W, xs
    print(json.dumps({"case": "ns_sweep", "workload": "128x128x32 volume, Nk=1200, 90 views, 128x32 detector, "
                                                      "200 counts/bin, 3 materials", "rows": rows}), flush=True)
    ctx.close()


if __name__ == "__main__":
    case = sys.argv[1] if len(sys.argv) > 1 else "precision"
    if case == "precision":
        precision()
    elif case == "fbp_fmd":
        fbp_fmd()
    elif case == "learned":
        learned(int(sys.argv[2]) if len(sys.argv) > 2 else 2000)
    elif case == "dhr":
        dhr()
    elif case == "ns_sweep":
        ns_sweep()
    elif case == "batched":
        batched(int(sys.argv[2]) if len(sys.argv) > 2 else 40, int(sys.argv[3]) if len(sys.argv) > 3 else 100)
    else:
        raise SystemExit("unknown case %r" % case)
