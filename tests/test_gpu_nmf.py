"""GPU parity of the subspace decomposition (Sec. III): fused fast-HALS pass, D update, NNDSVD start."""
import numpy as np
import pytest
from _parity import assert_close, rel_l2 as _rel

pytestmark = pytest.mark.gpu


def _dev(a, dtype=None):
    import torch

    t = torch.from_numpy(np.ascontiguousarray(a))
    return t.cuda() if dtype is None else t.to(dtype).cuda()


def _padded(P, ldP):
    out = np.zeros((P.shape[0], ldP), np.float32)
    out[:, :P.shape[1]] = P
    return out


def _run_pair(fx, orc, P64, K, iters, seed):
    rng = np.random.default_rng(seed)
    Np, Nk = P64.shape
    from paper_2410_22500_gb300 import synth

    D0, W0 = synth.nmf_given_init(rng, Np, Nk, K)
    D0 = D0.astype(np.float32).astype(np.float64)
    W0 = W0.astype(np.float32).astype(np.float64)
    ldP = (Nk + 3) // 4 * 4
    P32 = P64.astype(np.float32)
    Pd = _dev(_padded(P32, ldP))
    D, W, obj = fx.decompose(Pd, Nk, K, iters, D=_dev(D0.astype(np.float32)), W=_dev(W0.astype(np.float32)))
    Dr, Wr, objr = orc.nmf(P32.astype(np.float64), D0, W0, iters)
    return D.cpu().numpy().astype(np.float64), W.cpu().numpy().astype(np.float64), obj.cpu().numpy(), Dr, Wr, objr


@pytest.mark.parametrize("Np,Nk,K", [(203, 37, 3), (96, 128, 5), (1000, 64, 8), (57, 12, 1), (300, 200, 2)])
def test_first_ten_iterates(fx, orc, Np, Nk, K):
    # tolerance of the first 10 iterates: 1e-4 relative (FP32 pass vs FP64 oracle)
    rng = np.random.default_rng(Np + Nk)
    P = rng.uniform(0, 1, size=(Np, Nk)) * rng.uniform(0.5, 1.5, size=(Np, 1))
    for t in (1, 3, 10):
        D, W, obj, Dr, Wr, objr = _run_pair(fx, orc, P, K, t, seed=7)
        assert_close(D, Dr, 1e-4, what="D, %d iterations" % t)
        assert_close(W, Wr, 1e-4, what="W, %d iterations" % t)
        np.testing.assert_allclose(obj, objr, rtol=1e-4)


@pytest.mark.parametrize("dtype,ldP", [("bf16", 200), ("bf16", 256), ("f32", 228)])
def test_padded_row_stride_matches_oracle(fx, orc, dtype, ldP):
    # Nk = 96 live bins in rows of ldP: 200 bf16 / 228 f32 values are exactly the staged
    # row of the tensor-core pass (one bulk copy per 8-row tile), 256 is wider than it
    # (each row copy stops at the staged row); 500 rows leave a ragged last tile
    import torch
    from paper_2410_22500_gb300 import synth

    rng = np.random.default_rng(31)
    Np, Nk, K = 500, 96, 4
    P = rng.uniform(0, 1, size=(Np, Nk))
    tdt = torch.bfloat16 if dtype == "bf16" else torch.float32
    Pt = torch.zeros((Np, ldP), dtype=tdt)
    Pt[:, :Nk] = torch.from_numpy(P.astype(np.float32)).to(tdt)
    Pr = Pt[:, :Nk].float().numpy().astype(np.float64)
    D0, W0 = synth.nmf_given_init(rng, Np, Nk, K)
    D0 = D0.astype(np.float32)
    W0 = W0.astype(np.float32)
    D, W, obj = fx.decompose(Pt.cuda(), Nk, K, 10, D=_dev(D0), W=_dev(W0))
    Dr, Wr, objr = orc.nmf(Pr, D0.astype(np.float64), W0.astype(np.float64), 10)
    assert_close(D.cpu().numpy(), Dr, 1e-4, what="D")
    assert_close(W.cpu().numpy(), Wr, 1e-4, what="W")
    np.testing.assert_allclose(obj.cpu().numpy(), objr, rtol=1e-4)


def test_row_stride_does_not_change_results(fx):
    # the 256^3 form's rows (1500 bf16 bins): stored with the pipeline's stride (1544, one
    # bulk copy per 8-row tile) and with the plain one (1504, one copy per row), the pass
    # does the same arithmetic on the same live bins, so D, W and the objective agree bit
    # for bit; 98,305 rows leave a ragged last tile
    import torch
    from paper_2410_22500_gb300 import fhr, synth

    assert fhr.nmf_row_stride(1500, fhr.BF16) == 1544
    rng = np.random.default_rng(17)
    Np, Nk, K = 98305, 1500, 6
    g = torch.Generator(device="cuda")
    g.manual_seed(17)
    live = torch.rand((Np, Nk), device="cuda", generator=g).to(torch.bfloat16)
    D0, W0 = synth.nmf_given_init(rng, Np, Nk, K)
    out = []
    for ldP in (1504, 1544):
        P = torch.zeros((Np, ldP), dtype=torch.bfloat16, device="cuda")
        P[:, :Nk] = live
        D, W, obj = fx.decompose(P, Nk, K, 3, D=_dev(D0.astype(np.float32)), W=_dev(W0.astype(np.float32)))
        out.append((D.cpu().numpy(), W.cpu().numpy(), obj.cpu().numpy()))
        del P
    for a, b in zip(out[0], out[1]):
        np.testing.assert_array_equal(a, b)


def test_tiny_2d_workload_final_objective(fx, orc):
    # the 32x32 / 60-view / Nk=128 / K=3 workload, 200 iterations: final objective within 1e-3
    from paper_2410_22500_gb300 import synth

    pb = synth.tiny_2d()
    y, y0 = synth.counts_numpy(pb)
    P = orc.normalise(y, y0)
    D, W, obj, Dr, Wr, objr = _run_pair(fx, orc, P, 3, 200, seed=1000)
    assert abs(obj[-1] - objr[-1]) <= 1e-3 * objr[-1]
    assert abs(obj[-1] - orc.objective(P.astype(np.float32).astype(np.float64), D, W)) <= 1e-3 * objr[-1]
    assert np.all(np.diff(obj) <= 1e-6 * obj[:-1])        # monotone up to FP32 rounding
    assert np.all(D >= 0) and np.all(W >= 0)


def test_bf16_stream_matches_oracle_on_rounded_data(fx, orc):
    # BF16 inputs, FP32 accumulation: against the oracle run on the same bf16-rounded P the
    # iterates agree to the FP32 tolerance; the error from rounding P itself is reported too
    import torch
    from paper_2410_22500_gb300 import synth

    rng = np.random.default_rng(5)
    Np, Nk, K = 500, 96, 4
    P = rng.uniform(0, 1, size=(Np, Nk))
    Pb = torch.from_numpy(P.astype(np.float32)).to(torch.bfloat16)
    Pr = Pb.float().numpy().astype(np.float64)
    D0, W0 = synth.nmf_given_init(rng, Np, Nk, K)
    D0 = D0.astype(np.float32)
    W0 = W0.astype(np.float32)
    D, W, obj = fx.decompose(Pb.cuda(), Nk, K, 10, D=_dev(D0), W=_dev(W0))
    Dr, Wr, objr = orc.nmf(Pr, D0.astype(np.float64), W0.astype(np.float64), 10)
    assert_close(D.cpu().numpy(), Dr, 1e-4)
    assert_close(W.cpu().numpy(), Wr, 1e-4)
    Df, Wf, objf = orc.nmf(P, D0.astype(np.float64), W0.astype(np.float64), 10)
    print("bf16 data rounding: D rel err %.2e, objective rel err %.2e" % (_rel(Dr, Df), abs(objr[-1] - objf[-1]) / objf[-1]))


def test_dead_bins_give_zero_dictionary_rows(fx, orc):
    rng = np.random.default_rng(9)
    Np, Nk, K = 400, 50, 3
    P = rng.uniform(0, 1, size=(Np, Nk))
    P[:, [3, 17, 49]] = 0
    D, W, obj, Dr, Wr, objr = _run_pair(fx, orc, P, K, 5, seed=3)
    assert np.all(D[[3, 17, 49]] == 0)


def test_nndsvd_start_matches_exact_svd(fx, orc):
    # randomised subspace iteration vs the oracle's exact SVD: rank-K signal + noise,
    # so the K-th gap is large and the start agrees closely
    from paper_2410_22500_gb300 import fhr

    rng = np.random.default_rng(11)
    Np, Nk, K = 3000, 80, 4
    Dt = rng.uniform(0, 1, size=(Nk, K))
    Wt = rng.uniform(0, 1, size=(Np, K))
    P = Wt @ Dt.T + 0.01 * rng.uniform(0, 1, size=(Np, Nk))
    P32 = P.astype(np.float32)
    D, W, _ = fx.decompose(_dev(P32), Nk, K, 0, init=fhr.INIT_NNDSVD, seed=1, obj=False)
    Dr, Wr = orc.nndsvd(P32.astype(np.float64), K)
    assert_close(D.cpu().numpy(), Dr, 1e-3)
    assert_close(W.cpu().numpy(), Wr, 1e-3)
    assert float(D.min()) >= 0 and float(W.min()) >= 0


def test_nndsvd_then_iterations_reach_oracle_objective(fx, orc):
    from paper_2410_22500_gb300 import fhr, synth

    pb = synth.tiny_2d()
    y, y0 = synth.counts_numpy(pb)
    P = orc.normalise(y, y0).astype(np.float32)
    D, W, obj = fx.decompose(_dev(P), 128, 3, 200, init=fhr.INIT_NNDSVD, seed=2)
    D0r, W0r = orc.nndsvd(P.astype(np.float64), 3)
    Dr, Wr, objr = orc.nmf(P.astype(np.float64), D0r, W0r, 200)
    assert abs(obj.cpu().numpy()[-1] - objr[-1]) <= 1e-3 * objr[-1]


def test_full_size_one_iteration(fx, orc):
    # the 3-D workload at full size (737,280 pixels x 1200 bins, K = 5): one iteration from a
    # GIVEN start; every pixel row of W against the oracle's V half-step, D against the
    # oracle's D half-step over all pixels
    import torch
    from paper_2410_22500_gb300 import synth

    pb = synth.volume_3d_f32()
    y, y0 = synth.counts_torch(pb)
    P = fx.normalise(y, y0, dead=_dev(pb.dead_bins))
    del y
    K, Nk = 5, pb.Nk
    rng = np.random.default_rng(12)
    D0, W0 = synth.nmf_given_init(rng, P.shape[0], Nk, K)
    D0 = D0.astype(np.float32)
    W0 = W0.astype(np.float32)
    D, W, obj = fx.decompose(P, Nk, K, 1, D=_dev(D0), W=_dev(W0))
    torch.cuda.synchronize()
    Ph = P[:, :Nk].cpu().numpy().astype(np.float64)
    Wv = W0.astype(np.float64).copy()
    orc.hals_update_W(Ph, D0.astype(np.float64), Wv)
    Dv = D0.astype(np.float64).copy()
    orc.hals_update_D(Ph, Wv, Dv)
    n = orc.normalise_columns(Dv, Wv)
    assert_close(W.cpu().numpy().astype(np.float64), Wv, 1e-4, what="W, all 737,280 rows")
    assert_close(D.cpu().numpy().astype(np.float64), Dv, 1e-4)
