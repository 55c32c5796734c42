"""Small, fixed cases for profiling single kernels (ncu captures must stay small).

    python -m paper_2410_22500_gb300.profcase nmf_pass [Np]
    python -m paper_2410_22500_gb300.profcase nmf_pass_bf16 [Np]
    python -m paper_2410_22500_gb300.profcase mbir
    python -m paper_2410_22500_gb300.profcase fmd
    python -m paper_2410_22500_gb300.profcase fbp
    python -m paper_2410_22500_gb300.profcase mlp [M]

`nmf_pass`: P of Np x 1200 uniform f32 (default Np = 92,160: 442 MB, larger than
L2), K = 5, three fast-HALS iterations from a fixed start.  Launch 0 is the first
pass; profile with `-k regex:nmf_ -s 1 -c 1` (the tensor-core kernel is
`nmf_mma_kernel`, the CUDA-core one `nmf_pass_kernel`).

`nmf_pass_bf16`: the same with P of Np rows of 1500 bf16 bins (default Np = 122,880)
in the row stride fhr_nmf_row_stride gives (1544 values, 380 MB), K = 6: the rows
and K of the 256^3 precision form as the pipeline lays them out.

`mbir`: the reconstruction of the 3-D workload's subspace sinograms (N = 128,
64 slices x K = 5, 90 views x 128 bins; uniform random sinogram), four SQS
iterations with momentum: launches of proj_fwd_kernel and mbir_update_kernel
at the benchmark's shapes (profile with `-k regex:"proj_fwd|mbir_update" -s 2 -c 2`).
`mbir_volume`: the same at the 256^3 precision form's shapes (N = 256, 256 slices x
K = 6, 120 views x 256 bins: a 403 MB image and a 189 MB sinogram), three SQS
iterations with momentum.
`normalise_expand`: the normalisation of counts shaped like 8 detector rows of the
256^3 precision form (120 views x 8 rows x 256 columns x 1500 bins, 100 counts per
bin, to BF16 P: 737 MB in, 737 MB out) and the expansion of 8 slices of that
volume (256 x 256 x 8 voxels, K = 6, to FP32 x^h: 3.1 GB), two calls each.
`fmd`: the semi-supervised material decomposition of 1,048,576 voxels (the 3-D
workload's volume), Ns = Nm = 5, seeded mixtures with 10% of the voxels labelled,
Nk = 1200; three calls (fmd_region_partials, fmd_finish_T, fmd_gram, fmd_spectra,
fmd_subset_inverses, fmd_nnls each).

`mlp`: the learned start's network forward (1500 -> 256 -> 128 -> 6, bf16 rows of
1504 bins and bf16 weights) on M rows (default 131,072: 394 MB of rows, 1024 row
tiles), three calls: launches of mlp_gemm_tc (layers 1 and 2) and the small last layer.

`fbp`: FBP of the 3-D workload's subspace sinograms (N = 128, 64 slices x K = 5, 90
views x 128 bins; uniform random sinogram), three calls (fbp_filter_kernel, then
proj_bwd_kernel each).
"""
import sys

import torch

from . import build, fhr


def nmf_pass(Np: int = 92160, Nk: int = 1200, K: int = 5, iters: int = 3, dtype=torch.float32, ldP=None) -> None:
    build.build()
    ctx = fhr.Context(0)
    g = torch.Generator(device="cuda")
    g.manual_seed(0)
    P = torch.zeros((Np, ldP or Nk), device="cuda", dtype=dtype)
    P[:, :Nk] = torch.rand((Np, Nk), device="cuda", generator=g).to(dtype)
    D = torch.rand((Nk, K), device="cuda", generator=g) + 0.1
    W = torch.rand((Np, K), device="cuda", generator=g) + 0.1
    ctx.decompose(P, Nk, K, iters, D=D, W=W)
    torch.cuda.synchronize()
    ctx.close()
    print("ok")


def mbir(iters: int = 4, N: int = 128, Nr: int = 64, K: int = 5, Nv: int = 90, Nc: int = 128) -> None:
    build.build()
    ctx = fhr.Context(0)
    g = torch.Generator(device="cuda")
    g.manual_seed(0)
    sino = torch.rand((Nv, Nc, Nr * K), device="cuda", generator=g)
    ctx.reconstruct(sino, N, Nr, K, iters, momentum=True)
    torch.cuda.synchronize()
    ctx.close()
    print("ok")


def fmd(calls: int = 3) -> None:
    import numpy as np

    build.build()
    ctx = fhr.Context(0)
    rng = np.random.default_rng(0)
    Nx, Ns, Nm, Nk = 1048576, 5, 5, 1200
    B = rng.normal(size=(Nm, Ns)) + 3 * np.eye(Nm, Ns)
    xm = rng.uniform(size=(Nx, Nm)) * (rng.uniform(size=(Nx, Nm)) > 0.4)
    xs = torch.from_numpy((xm @ B + 0.05 * rng.normal(size=(Nx, Ns))).astype(np.float32)).cuda()
    lab = (np.argmax(xm, axis=1) + 1).astype(np.uint8)
    lab[rng.uniform(size=Nx) < 0.9] = 0
    labels = torch.from_numpy(lab).cuda()
    D = torch.from_numpy(rng.uniform(size=(Nk, Ns)).astype(np.float32)).cuda()
    for _ in range(calls):
        ctx.fmd(xs, labels, D, Nm)
    torch.cuda.synchronize()
    ctx.close()
    print("ok")


def fbp(calls: int = 3) -> None:
    build.build()
    ctx = fhr.Context(0)
    g = torch.Generator(device="cuda")
    g.manual_seed(0)
    N, Nr, K, Nv, Nc = 128, 64, 5, 90, 128
    sino = torch.rand((Nv, Nc, Nr * K), device="cuda", generator=g)
    for _ in range(calls):
        ctx.fbp(sino, N)
    torch.cuda.synchronize()
    ctx.close()
    print("ok")


def normalise_expand(Nr: int = 8) -> None:
    build.build()
    ctx = fhr.Context(0)
    g = torch.Generator(device="cuda")
    g.manual_seed(0)
    Nv, Nc, Nk, N, K = 120, 256, 1500, 256, 6
    y = torch.poisson(torch.full((Nv, Nr, Nc, Nk), 60.0, device="cuda"), generator=g).to(torch.int32).to(torch.int16)
    y0 = torch.poisson(torch.full((Nr, Nc, Nk), 100.0, device="cuda"), generator=g).to(torch.int32).to(torch.int16)
    for _ in range(2):
        P = ctx.normalise(y, y0, p_dtype=fhr.BF16)
    del P, y
    xs = torch.rand((N, N, Nr * K), device="cuda", generator=g)
    D = torch.rand((Nk, K), device="cuda", generator=g)
    for _ in range(2):
        xh = ctx.expand(xs, D, N, Nr)
    torch.cuda.synchronize()
    ctx.close()
    print("ok")


def mlp(M: int = 131072, calls: int = 3) -> None:
    import math

    build.build()
    ctx = fhr.Context(0)
    g = torch.Generator(device="cuda")
    g.manual_seed(0)
    Nk, H1, H2, K, ldx = 1500, 256, 128, 6, 1504
    sizes = [H1 * Nk, H1, H2 * H1, H2, K * H2, K]
    scales = [1 / math.sqrt(Nk), 0.1, 1 / math.sqrt(H1), 0.1, 1 / math.sqrt(H2), 0.1]
    prm = torch.cat([torch.randn(n, device="cuda", generator=g) * sc for n, sc in zip(sizes, scales)])
    X = (torch.rand((M, ldx), device="cuda", generator=g) * 2).to(torch.bfloat16)
    d = ctx.mlp_dims(Nk, H1, H2, K, ldx=ldx, x_bf16=True, weights_bf16=True)
    Y = None
    for _ in range(calls):
        Y = ctx.mlp_forward(d, prm, X, Y=Y)
    torch.cuda.synchronize()
    ctx.close()
    print("ok")


if __name__ == "__main__":
    case = sys.argv[1] if len(sys.argv) > 1 else "nmf_pass"
    if case == "nmf_pass":
        nmf_pass(int(sys.argv[2]) if len(sys.argv) > 2 else 92160)
    elif case == "nmf_pass_bf16":
        nmf_pass(int(sys.argv[2]) if len(sys.argv) > 2 else 122880, Nk=1500, K=6, dtype=torch.bfloat16,
                 ldP=fhr.nmf_row_stride(1500, fhr.BF16))
    elif case == "mbir":
        mbir()
    elif case == "mbir_volume":
        mbir(3, N=256, Nr=256, K=6, Nv=120, Nc=256)
    elif case == "normalise_expand":
        normalise_expand(int(sys.argv[2]) if len(sys.argv) > 2 else 8)
    elif case == "fmd":
        fmd()
    elif case == "mlp":
        mlp(int(sys.argv[2]) if len(sys.argv) > 2 else 131072)
    elif case == "fbp":
        fbp()
    else:
        raise SystemExit("unknown case %r" % case)
