"""GPU parity of the clustering start of the decomposition (k-means++ seeding,
Lloyd iterations in FP64, D0 = centres, W0 = one HALS V step from zero)."""
import numpy as np
import pytest
from _parity import assert_close, rel_l2 as _rel

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _padded(P, ldP):
    out = np.zeros((P.shape[0], ldP), np.float32)
    out[:, :P.shape[1]] = P
    return out


def _gpu_start(fx, P32, K, S, iters, seed, nmf_iters=0):
    from paper_2410_22500_gb300 import fhr

    Np, Nk = P32.shape
    ldP = (Nk + 3) // 4 * 4
    D, W, obj = fx.decompose(_dev(_padded(P32, ldP)), Nk, K, nmf_iters, init=fhr.INIT_CLUSTER, seed=seed,
                             kmeans_samples=S, kmeans_iters=iters)
    return D.cpu().numpy().astype(np.float64), W.cpu().numpy().astype(np.float64), obj.cpu().numpy()


def _blobs(rng, K, per, Nk, spread=0.02):
    centres = rng.uniform(0.5, 2.0, size=(K, Nk)) * (1 + 2 * np.arange(K))[:, None]
    lab = np.repeat(np.arange(K), per)
    X = centres[lab] + spread * rng.normal(size=(K * per, Nk))
    return np.abs(X[rng.permutation(K * per)])


@pytest.mark.parametrize("Np,Nk,K,S", [(2000, 37, 4, 2000), (5000, 64, 6, 777), (900, 200, 3, 300)])
def test_separated_clusters_match_oracle(fx, orc, Np, Nk, K, S):
    rng = np.random.default_rng(Np + K)
    P32 = _blobs(rng, K, Np // K + 1, Nk)[:Np].astype(np.float32)
    D, W, _ = _gpu_start(fx, P32, K, S, 8, seed=3)
    Dr, Wr = orc.cluster_init(P32.astype(np.float64), K, S=S, iters=8, seed=3)
    assert_close(D, Dr, 1e-6)
    assert_close(W, Wr, 1e-5)


def test_workload_start_and_iterates_match_oracle(fx, orc):
    # the 32x32 / 60-view / Nk=128 / K=3 projection data: the start and the
    # first ten iterates from it, against the oracle's start and HALS
    from paper_2410_22500_gb300 import synth

    pb = synth.tiny_2d()
    y, y0 = synth.counts_numpy(pb)
    P32 = orc.normalise(y, y0).astype(np.float32)
    P64 = P32.astype(np.float64)
    K = 3
    D, W, _ = _gpu_start(fx, P32, K, 1024, 20, seed=11)
    Dr, Wr = orc.cluster_init(P64, K, S=1024, iters=20, seed=11)
    assert_close(D, Dr, 1e-6)
    assert_close(W, Wr, 1e-5)
    D10, W10, obj = _gpu_start(fx, P32, K, 1024, 20, seed=11, nmf_iters=10)
    Dr10, Wr10, objr = orc.nmf(P64, Dr.astype(np.float32).astype(np.float64), Wr, 10)
    assert_close(D10, Dr10, 1e-4)
    assert_close(W10, Wr10, 1e-4)
    np.testing.assert_allclose(obj, objr, rtol=1e-4)


def test_bf16_input(fx, orc):
    import torch

    from paper_2410_22500_gb300 import fhr

    rng = np.random.default_rng(21)
    Np, Nk, K = 1500, 48, 4
    P = _blobs(rng, K, Np // K + 1, Nk)[:Np]
    Pb = torch.from_numpy(P.astype(np.float32)).to(torch.bfloat16)
    Pr = Pb.float().numpy().astype(np.float64)
    D, W, _ = fx.decompose(Pb.cuda(), Nk, K, 0, init=fhr.INIT_CLUSTER, seed=5, kmeans_samples=600, kmeans_iters=5)
    Dr, Wr = orc.cluster_init(Pr, K, S=600, iters=5, seed=5)
    assert_close(D.cpu().numpy().astype(np.float64), Dr, 1e-6)
    assert_close(W.cpu().numpy().astype(np.float64), Wr, 1e-5)


def test_default_sample_and_iterations(fx, orc):
    # kmeans_samples = 0 -> min(Np, 32768); kmeans_iters = 0 -> 20
    rng = np.random.default_rng(22)
    P32 = _blobs(rng, 3, 400, 20)[:1000].astype(np.float32)
    D, _, _ = _gpu_start(fx, P32, 3, 0, 0, seed=1)
    Dr, _ = orc.cluster_init(P32.astype(np.float64), 3, S=1000, iters=20, seed=1)
    assert_close(D, Dr, 1e-6)


def test_rejects_bad_cluster_arguments(fx):
    from paper_2410_22500_gb300 import fhr

    P = _dev(np.ones((100, 8), np.float32))
    with pytest.raises(fhr.FhrError) as e:
        fx.decompose(P, 8, 3, 1, init=fhr.INIT_CLUSTER, kmeans_samples=(1 << 20) + 1)
    assert e.value.code == fhr.ERR_ARG
    with pytest.raises(fhr.FhrError) as e:
        fx.decompose(P, 8, 3, 1, init=fhr.INIT_CLUSTER, kmeans_samples=2)
    assert e.value.code == fhr.ERR_ARG
