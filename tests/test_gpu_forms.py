"""Error of the BF16 form (P streamed as bfloat16, FP32 accumulation, FP64 Grams
and objective) against the FP64 oracle, next to the FP32 form, on one detector
row of the 256^3 / Nk = 1500 / K = 6 workload.  Both forms start from the same
NNDSVD factors; the objectives are evaluated against the FP32 P."""
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
