"""Small, fixed cases for profiling single kernels (ncu captures must stay small).

    python -m paper_2410_22500_gb300.profcase nmf_pass [Np]
    python -m paper_2410_22500_gb300.profcase mbir_batch [n_problems] [iters]

`nmf_pass`: P of Np x 1200 uniform f32 (default Np = 92,160: 442 MB, larger than
L2), K = 5, three fast-HALS iterations from a fixed start.  Launch 0 is the first
pass; profile with `-k regex:nmf_pass -s 1 -c 1`.

`mbir_batch`: the uneven 2-D batch (40 problems by default: N in 64..512 step 16,
Nc = N, 45..180 views, K in 3..8, problem i seeded with 2000 + i), sinograms
made by the library's projector from seeded disk phantoms; times the batched
reconstruction (autotuned tile) against one fhr_reconstruct call per problem
and prints one JSON line.
"""
import json
import sys

import torch

from . import build, fhr


def nmf_pass(Np: int = 92160, Nk: int = 1200, K: int = 5, iters: int = 3) -> None:
    build.build()
    ctx = fhr.Context(0)
    g = torch.Generator(device="cuda")
    g.manual_seed(0)
    P = torch.rand((Np, Nk), device="cuda", generator=g)
    D = torch.rand((Nk, K), device="cuda", generator=g) + 0.1
    W = torch.rand((Np, K), device="cuda", generator=g) + 0.1
    ctx.decompose(P, Nk, K, iters, D=D, W=W)
    torch.cuda.synchronize()
    ctx.close()
    print("ok")


def _batch_shapes(n_problems: int):
    import numpy as np

    out = []
    for i in range(n_problems):
        rng = np.random.default_rng(2000 + i)
        N = int(rng.integers(4, 33)) * 16
        Nv = int(rng.integers(45, 181))
        K = int(rng.integers(3, 9))
        out.append((N, Nv, K))
    return out


def mbir_batch(n_problems: int = 40, iters: int = 100) -> None:
    build.build()
    ctx = fhr.Context(0)
    shapes = _batch_shapes(n_problems)
    g = torch.Generator(device="cuda")
    g.manual_seed(2000)
    sinos = []
    for N, Nv, K in shapes:
        yy, xx = torch.meshgrid(torch.arange(N, device="cuda"), torch.arange(N, device="cuda"), indexing="ij")
        r = ((yy - N / 2) ** 2 + (xx - N / 2) ** 2).sqrt()
        x = (r < 0.4 * N).float()[..., None] * (0.5 + torch.rand((1, 1, K), device="cuda", generator=g))
        sinos.append(ctx.project(x.contiguous(), N, Nv))
    Ns, Ks = [s[0] for s in shapes], [s[2] for s in shapes]
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    # batched: autotune once, then time a full run
    _, tile = ctx.reconstruct_batch(sinos, Ns, Ks, 4, autotune=True)
    torch.cuda.synchronize()
    ev[0].record()
    xb, _ = ctx.reconstruct_batch(sinos, Ns, Ks, iters, tile=tile)
    ev[1].record()
    torch.cuda.synchronize()
    t_batch = ev[0].elapsed_time(ev[1])
    # one call per problem
    ctx.reconstruct(sinos[0], Ns[0], 1, Ks[0], 2)
    torch.cuda.synchronize()
    ev[2].record()
    xs = [ctx.reconstruct(s, N, 1, K, iters) for s, N, K in zip(sinos, Ns, Ks)]
    ev[3].record()
    torch.cuda.synchronize()
    t_seq = ev[2].elapsed_time(ev[3])
    worst = max(float(((a - b).norm() / b.norm().clamp_min(1e-30)).item()) for a, b in zip(xb, xs))
    vox = sum(N * N * K for N, _, K in shapes)
    print(json.dumps({"case": "mbir_batch", "problems": n_problems, "iters": iters, "tile": tile,
                      "batched_ms": round(t_batch, 3), "per_problem_ms": round(t_seq, 3),
                      "speedup": round(t_seq / t_batch, 3), "voxel_channels": vox,
                      "max_rel_diff_vs_per_problem": worst}))
    ctx.close()


if __name__ == "__main__":
    case = sys.argv[1] if len(sys.argv) > 1 else "nmf_pass"
    if case == "nmf_pass":
        nmf_pass(int(sys.argv[2]) if len(sys.argv) > 2 else 92160)
    elif case == "mbir_batch":
        mbir_batch(int(sys.argv[2]) if len(sys.argv) > 2 else 40, int(sys.argv[3]) if len(sys.argv) > 3 else 100)
    else:
        raise SystemExit("unknown case %r" % case)
