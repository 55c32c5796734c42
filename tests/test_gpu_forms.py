"""Error of the BF16 form (P streamed as bfloat16, FP32 accumulation, FP64 Grams
and objective) against the FP64 oracle on the 256^3 / Nk = 1500 / K = 6 workload:
on one detector row next to the FP32 form (both from the same NNDSVD factors,
objectives evaluated against the FP32 P), and on the 32-slice subset of the
full volume (from a shared seeded start, evaluated against the FP64 P)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ITERS = 10


def _obj(P, D, W):
    R = P - W @ D.T
    return float(np.sum(R * R))


def test_bf16_form_error_against_fp64(fx, orc):
    import torch

    from paper_2410_22500_gb300 import synth

    pb = synth.scaled(synth.volume_3d_bf16, Nr=1)
    y, y0 = synth.counts_numpy(pb)
    P64 = orc.normalise(y, y0)
    P32 = P64.astype(np.float32)
    Pr = P32.astype(np.float64)
    Np, Nk = P32.shape
    K = 6
    D0, W0 = orc.nndsvd(Pr, K)
    D0 = D0.astype(np.float32)
    W0 = W0.astype(np.float32)
    Do, Wo, _ = orc.nmf(Pr, D0.astype(np.float64), W0.astype(np.float64), ITERS)
    ref = Wo @ Do.T
    f_ref = _obj(Pr, Do, Wo)
    res = {}
    for name in ("f32", "bf16"):
        if name == "f32":
            ldP = (Nk + 3) // 4 * 4
            Pd = torch.zeros((Np, ldP), dtype=torch.float32)
            Pd[:, :Nk] = torch.from_numpy(P32)
        else:
            ldP = (Nk + 7) // 8 * 8
            Pd = torch.zeros((Np, ldP), dtype=torch.bfloat16)
            Pd[:, :Nk] = torch.from_numpy(P32).to(torch.bfloat16)
        D, W, _ = fx.decompose(Pd.cuda(), Nk, K, ITERS, D=torch.from_numpy(D0).cuda(), W=torch.from_numpy(W0).cuda())
        D = D.cpu().numpy().astype(np.float64)
        W = W.cpu().numpy().astype(np.float64)
        prod = W @ D.T
        res[name] = (np.linalg.norm(prod - ref) / np.linalg.norm(ref), abs(_obj(Pr, D, W) - f_ref) / f_ref)
    print("\nBF16 form vs FP64 after %d iterations: product rel err %.3e, objective rel err %.3e "
          "(FP32 form: %.3e, %.3e)" % (ITERS, res["bf16"][0], res["bf16"][1], res["f32"][0], res["f32"][1]))
    assert res["f32"][0] <= 1e-4 and res["f32"][1] <= 1e-4
    assert res["bf16"][1] <= 1e-3
    assert res["bf16"][0] <= 1e-2


def test_bf16_form_error_on_32_slices(fx, orc):
    # the precision form's error against FP64 on the 32-slice subset of the 256^3 / Nk = 1500 /
    # K = 6 workload: detector rows 112..143 of the full volume's counts (983,040 pixel rows).
    # The GPU streams P as BF16 (normalised on the GPU from the counts); the oracle normalises
    # the same counts in FP64.  Both run 10 iterations from one seeded GIVEN start; the GPU's
    # factors are then evaluated against the FP64 P by the oracle.
    import torch

    from paper_2410_22500_gb300 import fhr, synth

    pb = synth.volume_3d_bf16()
    y, y0 = synth.counts_torch(pb)
    r0, r1 = 112, 144
    ys = y[:, r0:r1].contiguous()
    y0s = y0[r0:r1].contiguous()
    del y, y0
    torch.cuda.empty_cache()
    Nv, Nr, Nc, Nk = ys.shape
    Np = Nv * Nr * Nc
    rng = np.random.default_rng(32)
    D0, W0 = synth.nmf_given_init(rng, Np, Nk, 6)
    D0 = D0.astype(np.float32)
    W0 = W0.astype(np.float32)
    Pb = fx.normalise(ys, y0s, p_dtype=fhr.BF16)
    D, W, obj = fx.decompose(Pb, Nk, 6, ITERS, D=torch.from_numpy(D0).cuda(), W=torch.from_numpy(W0).cuda())
    Dg = D.cpu().numpy().astype(np.float64)
    Wg = W.cpu().numpy().astype(np.float64)
    del Pb, D, W
    yh = ys.cpu().numpy().view(np.uint16)
    y0h = y0s.cpu().numpy().view(np.uint16)
    del ys, y0s
    torch.cuda.empty_cache()
    P64 = orc.normalise(yh, y0h)
    del yh
    Do, Wo, objo = orc.nmf(P64, D0.astype(np.float64), W0.astype(np.float64), ITERS)
    f_gpu = orc.objective(P64, Dg, Wg)
    num = den = 0.0
    for a in range(0, Np, 65536):
        ref = Wo[a:a + 65536] @ Do.T
        num += float(np.sum((Wg[a:a + 65536] @ Dg.T - ref) ** 2))
        den += float(np.sum(ref * ref))
    prod = (num / den) ** 0.5
    fo = float(objo[-1])
    print("\nBF16 form vs FP64 on 32 slices (983,040 x 1500), %d iterations from a shared start: "
          "product W D^T rel err %.3e, objective (against FP64 P) rel err %.3e" % (ITERS, prod, abs(f_gpu - fo) / fo))
    assert prod <= 2e-3
    assert abs(f_gpu - fo) <= 1e-3 * fo
