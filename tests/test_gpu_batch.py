"""GPU parity of the batched MBIR form: many uneven problems of Eq. (recon) in one
persistent cooperative launch, against per-problem reconstruction and the oracle."""
import math

import numpy as np
import pytest
from _parity import assert_close, rel_l2 as _rel

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _angles(Nv):
    return np.arange(Nv) * (math.pi / Nv)


def _sino(orc, N, Nc, Nv, Nr, K, seed, noise=0.02):
    rng = np.random.default_rng(seed)
    xt = np.zeros((N, N, Nr * K))
    c = N // 2
    xt[c - N // 4:c + N // 4, c - N // 5:c + N // 3] = rng.uniform(0.5, 1.0, size=Nr * K)
    V = orc.project(xt, Nc, _angles(Nv))
    return (V + noise * rng.normal(size=V.shape) * V.max()).astype(np.float32)


# (N, Nc, Nv, Nr, K): uneven sizes, channel counts and ragged work-item tails
BATCH_2D = [(16, 24, 18, 1, 3), (24, 36, 30, 1, 2), (9, 13, 7, 1, 1), (20, 30, 12, 1, 5), (32, 32, 45, 1, 8)]
BATCH_3D = [(12, 18, 10, 3, 2), (16, 20, 14, 2, 3), (10, 15, 9, 4, 1)]


def _run(fx, orc, probs, iters, momentum=False, p=1.2, tile=0, vw=0, sigmas=False, x0=None):
    V = [_sino(orc, N, Nc, Nv, Nr, K, seed=100 + i) for i, (N, Nc, Nv, Nr, K) in enumerate(probs)]
    sg = None
    if sigmas:
        sg = [orc.mbir_sigmas(v.astype(np.float64).reshape(-1, K), K, Nc) for v, (N, Nc, Nv, Nr, K) in zip(V, probs)]
    xss = None if x0 is None else [_dev(x) for x in x0]
    out, t, _ = fx.reconstruct_batch([_dev(v) for v in V], [b[0] for b in probs], [b[4] for b in probs], iters,
                                     Nr=[b[3] for b in probs], xss=xss, sigmas=sg, momentum=momentum, p=p, tile=tile,
                                     vw=vw)
    return V, [o.cpu().numpy() for o in out], t


@pytest.mark.parametrize("probs", [BATCH_2D, BATCH_3D], ids=["2d", "3d"])
@pytest.mark.parametrize("momentum", [False, True])
def test_batch_matches_single_and_oracle(fx, orc, probs, momentum):
    iters = 12
    V, got, _ = _run(fx, orc, probs, iters, momentum=momentum)
    for v, g, (N, Nc, Nv, Nr, K) in zip(V, got, probs):
        single = fx.reconstruct(_dev(v), N, Nr, K, iters, momentum=momentum).cpu().numpy()
        assert_close(g, single, 1e-6)
        sv, sx = orc.mbir_sigmas(v.astype(np.float64).reshape(-1, K), K, Nc)
        ref = orc.mbir(v.astype(np.float64), N, Nr, K, _angles(Nv), sv, sx, iters=iters, momentum=momentum)
        assert_close(g, ref, 1e-4)


def test_wide_channel_vectors(fx, orc):
    # 3-D problems whose Nr*K exceeds a block's 256 threads: 320 and 260 values (multiples
    # of 4, so four values per thread), every tile width requested falls back to one that fits
    probs = [(12, 18, 10, 64, 5), (10, 15, 9, 52, 5)]
    iters = 5
    V, got, _ = _run(fx, orc, probs, iters, momentum=True, vw=1)
    for v, g, (N, Nc, Nv, Nr, K) in zip(V, got, probs):
        single = fx.reconstruct(_dev(v), N, Nr, K, iters, momentum=True).cpu().numpy()
        assert_close(g, single, 1e-6)


def test_batch_explicit_sigmas_and_warm_start(fx, orc):
    probs = BATCH_2D[:3]
    rng = np.random.default_rng(9)
    x0 = [rng.uniform(0, 0.5, size=(N, N, Nr * K)).astype(np.float32) for (N, Nc, Nv, Nr, K) in probs]
    V, got, _ = _run(fx, orc, probs, 10, p=1.5, sigmas=True, x0=x0)
    for v, g, x, (N, Nc, Nv, Nr, K) in zip(V, got, x0, probs):
        sv, sx = orc.mbir_sigmas(v.astype(np.float64).reshape(-1, K), K, Nc)
        ref = orc.mbir(v.astype(np.float64), N, Nr, K, _angles(Nv), sv, sx, p=1.5, iters=10,
                       x0=x.astype(np.float64))
        assert_close(g, ref, 1e-4)


@pytest.mark.parametrize("probs", [BATCH_2D, BATCH_3D], ids=["2d", "3d"])
def test_tile_shape_does_not_change_results(fx, orc, probs):
    # every channel of every pixel and ray is summed in the same order whatever the
    # work-item size and the values per thread
    _, a, _ = _run(fx, orc, probs, 6, tile=1)
    for tile, vw in ((8, 0), (2, 2), (4, 1)):
        _, b, _ = _run(fx, orc, probs, 6, tile=tile, vw=vw)
        for x, y in zip(a, b):
            np.testing.assert_array_equal(x, y)


def test_autotune_picks_a_candidate(fx, orc):
    V = [_sino(orc, N, Nc, Nv, Nr, K, seed=100 + i) for i, (N, Nc, Nv, Nr, K) in enumerate(BATCH_2D)]
    Ns, Ks = [b[0] for b in BATCH_2D], [b[4] for b in BATCH_2D]
    tuned, tile, vw = fx.reconstruct_batch([_dev(v) for v in V], Ns, Ks, 6, autotune=True)
    assert tile in (1, 2, 4, 8, 16) and vw in (1, 2, 4)
    plain, _, _ = fx.reconstruct_batch([_dev(v) for v in V], Ns, Ks, 6, tile=2)
    for x, y in zip(tuned, plain):
        np.testing.assert_array_equal(x.cpu().numpy(), y.cpu().numpy())


def test_autotune_leaves_volumes_alone(fx, orc):
    import ctypes

    import torch

    from paper_2410_22500_gb300 import fhr

    probs = BATCH_2D[:2]
    V = [_dev(_sino(orc, N, Nc, Nv, Nr, K, seed=7 + i)) for i, (N, Nc, Nv, Nr, K) in enumerate(probs)]
    xs = [torch.full((N, N, Nr * K), 0.25, device="cuda") for (N, Nc, Nv, Nr, K) in probs]
    arr = fx.batch_problems(V, [b[0] for b in probs], [b[4] for b in probs], xs)
    prm = fx.batch_params(8)
    n = ctypes.c_size_t()
    fx.check(fx.L.fhr_reconstruct_batch_workspace_size(fx._h, 2, arr, ctypes.byref(prm), ctypes.byref(n)))
    ws = fx.workspace(n.value)
    best, best_vw = ctypes.c_int(), ctypes.c_int()
    fx.check(fx.L.fhr_reconstruct_batch_autotune(fx._h, 2, arr, ctypes.byref(prm), fhr._ptr(ws), n.value,
                                                 ctypes.byref(best), ctypes.byref(best_vw)))
    assert fx.status(ws) == 0
    for x in xs:
        assert torch.all(x == 0.25)


def test_zero_iterations_keep_start(fx, orc):
    probs = BATCH_2D[:2]
    rng = np.random.default_rng(3)
    x0 = [rng.uniform(size=(N, N, Nr * K)).astype(np.float32) for (N, Nc, Nv, Nr, K) in probs]
    _, got, _ = _run(fx, orc, probs, 0, x0=x0)
    for g, x in zip(got, x0):
        np.testing.assert_array_equal(g, x)


def test_batch_rejects_bad_problems(fx, orc):
    import torch

    from paper_2410_22500_gb300 import fhr

    a = _dev(_sino(orc, 12, 18, 10, 1, 2, seed=1))
    b = _dev(_sino(orc, 12, 18, 10, 2, 2, seed=2))
    with pytest.raises(fhr.FhrError) as e:   # 2-D and 3-D in one batch
        fx.reconstruct_batch([a, b], [12, 12], [2, 2], 3, Nr=[1, 2])
    assert e.value.code == fhr.ERR_ARG
    with pytest.raises(fhr.FhrError) as e:   # K above the maximum
        fx.reconstruct_batch([a], [12], [9], 3)
    assert e.value.code == fhr.ERR_ARG
    big = torch.zeros((10, 18, 259), device="cuda")   # Nr*K = 259: odd, so one value per thread > 256 lanes
    with pytest.raises(fhr.FhrError) as e:
        fx.reconstruct_batch([big], [12], [7], 3, Nr=37)
    assert e.value.code == fhr.ERR_ARG
    with pytest.raises(fhr.FhrError) as e:
        fx.reconstruct_batch([a], [12], [2], 3, q=1.5)
    assert e.value.code == fhr.ERR_UNSUPPORTED
