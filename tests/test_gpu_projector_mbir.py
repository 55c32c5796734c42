"""GPU parity of the strip-area projector pair and of the MBIR (SQS, qGGMRF) reconstruction, Eq. (recon)."""
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


GEOMS = [(32, 48, 60, 3), (16, 23, 17, 8), (9, 13, 7, 1), (24, 40, 45, 12), (8, 12, 4, 5)]


@pytest.mark.parametrize("N,Nc,Nv,Wl", GEOMS)
def test_forward_matches_oracle(fx, orc, N, Nc, Nv, Wl):
    rng = np.random.default_rng(200 + N)
    x = rng.uniform(0, 1, size=(N, N, Wl)).astype(np.float32)
    y = fx.project(_dev(x), Nc, Nv).cpu().numpy()
    ref = orc.project(x.astype(np.float64), Nc, _angles(Nv))
    assert_close(y, ref, 1e-5)


@pytest.mark.parametrize("N,Nc,Nv,Wl", GEOMS)
def test_backward_matches_oracle(fx, orc, N, Nc, Nv, Wl):
    rng = np.random.default_rng(300 + N)
    e = rng.normal(size=(Nv, Nc, Wl)).astype(np.float32)
    x = fx.backproject(_dev(e), N).cpu().numpy()
    ref = orc.backproject(e.astype(np.float64), N, _angles(Nv))
    assert_close(x, ref, 1e-5)


def test_adjointness_fp32(fx):
    rng = np.random.default_rng(400)
    N, Nc, Nv, Wl = 40, 60, 50, 8
    x = rng.normal(size=(N, N, Wl)).astype(np.float32)
    y = rng.normal(size=(Nv, Nc, Wl)).astype(np.float32)
    Ax = fx.project(_dev(x), Nc, Nv).cpu().numpy().astype(np.float64)
    Aty = fx.backproject(_dev(y), N).cpu().numpy().astype(np.float64)
    lhs = np.sum(Ax * y)
    rhs = np.sum(x * Aty)
    scale = np.sqrt(np.sum(Ax * Ax) * np.sum(y * y))
    assert abs(lhs - rhs) <= 1e-6 * scale


def test_exact_transpose_on_unit_vectors(fx, orc):
    # the two tables hold bit-identical weights: A e_i (forward) equals row i of A^T
    # applied to unit sinogram vectors, compared through the dense oracle matrix
    N, Nc, Nv = 6, 10, 7
    th = _angles(Nv)
    A = orc.system_matrix(N, Nc, th)
    X = np.zeros((N, N, N * N), np.float32)
    for i in range(N * N):
        X[i // N, i % N, i] = 1
    Af = fx.project(_dev(X), Nc, Nv).cpu().numpy().reshape(Nv * Nc, N * N)
    Y = np.eye(Nv * Nc, dtype=np.float32).reshape(Nv, Nc, Nv * Nc)
    Ab = fx.backproject(_dev(Y), N).cpu().numpy().reshape(N * N, Nv * Nc)
    np.testing.assert_array_equal(Af, Ab.T)
    # each weight is the FP32 difference of two footprint-integral values in [0, 1],
    # evaluated at an FP64 offset (values under 2^-22 flushed to 0): within a few
    # FP32 ulps of 1 of the exact area
    np.testing.assert_allclose(Af, A, atol=3e-7)


def test_custom_angles(fx, orc):
    import torch

    rng = np.random.default_rng(401)
    N, Nc, Nv, Wl = 16, 24, 11, 4
    th = np.sort(rng.uniform(0, math.pi, Nv))
    x = rng.uniform(size=(N, N, Wl)).astype(np.float32)
    y = fx.project(_dev(x), Nc, Nv, angles=torch.from_numpy(th).cuda()).cpu().numpy()
    assert_close(y, orc.project(x.astype(np.float64), Nc, th), 1e-5)


def _sino(orc, N, Nc, Nv, Nr, K, seed, noise=0.02):
    rng = np.random.default_rng(seed)
    xt = np.zeros((N, N, Nr * K))
    c = N // 2
    xt[c - N // 4:c + N // 4, c - N // 5:c + N // 3] = rng.uniform(0.5, 1.0, size=Nr * K)
    V = orc.project(xt, Nc, _angles(Nv))
    return (V + noise * rng.normal(size=V.shape) * V.max()).astype(np.float32)


@pytest.mark.parametrize("N,Nc,Nv,Nr,K,momentum,p", [(20, 30, 24, 2, 3, False, 1.2), (16, 24, 18, 3, 2, True, 1.2),
                                                     (24, 36, 30, 1, 3, False, 1.5), (12, 18, 10, 4, 1, True, 2.0)])
def test_mbir_matches_oracle(fx, orc, N, Nc, Nv, Nr, K, momentum, p):
    V = _sino(orc, N, Nc, Nv, Nr, K, seed=N + Nr)
    sv, sx = orc.mbir_sigmas(V.astype(np.float64).reshape(-1, K), K, Nc)
    iters = 20
    ref = orc.mbir(V.astype(np.float64), N, Nr, K, _angles(Nv), sv, sx, p=p, iters=iters, momentum=momentum)
    got = fx.reconstruct(_dev(V), N, Nr, K, iters, p=p, momentum=momentum).cpu().numpy()
    assert_close(got, ref, 1e-4)
    # explicit sigmas take the same path
    got2 = fx.reconstruct(_dev(V), N, Nr, K, iters, p=p, momentum=momentum, sigma_v=sv, sigma_x=sx).cpu().numpy()
    assert_close(got2, ref, 1e-4)


def test_mbir_no_prior_and_warm_start(fx, orc):
    N, Nc, Nv, Nr, K = 12, 18, 16, 1, 2
    V = _sino(orc, N, Nc, Nv, Nr, K, seed=5)
    sv, sx = np.array([0.5, 1.0]), np.array([1.0, 1.0])
    rng = np.random.default_rng(6)
    x0 = rng.uniform(0, 0.5, size=(N, N, Nr * K)).astype(np.float32)
    ref = orc.mbir(V.astype(np.float64), N, Nr, K, _angles(Nv), sv, sx, beta=0.0, iters=15,
                   x0=x0.astype(np.float64))
    got = fx.reconstruct(_dev(V), N, Nr, K, 15, beta=0.0, sigma_v=sv, sigma_x=sx, xs=_dev(x0)).cpu().numpy()
    assert_close(got, ref, 1e-4)


def test_mbir_zero_channel(fx, orc):
    # an all-zero subspace channel reconstructs to zero (sigma defaults to 1 there)
    N, Nc, Nv, Nr, K = 10, 16, 12, 1, 2
    V = _sino(orc, N, Nc, Nv, Nr, K, seed=7)
    V[..., 1] = 0
    got = fx.reconstruct(_dev(V), N, Nr, K, 10).cpu().numpy()
    assert np.all(got[..., 1] == 0)
    assert np.all(got >= 0)


def test_channel_chunked_gathers_match_oracle(fx, orc):
    # a sinogram slab over the gathers' L2 budget (180 x 256 rays x 384 values = 71 MB):
    # the gathers run in channel chunks, chunk-major over the grid
    rng = np.random.default_rng(600)
    N, Nc, Nv, Wl = 40, 256, 180, 384
    th = _angles(Nv)
    x = rng.uniform(size=(N, N, Wl)).astype(np.float32)
    y = fx.project(_dev(x), Nc, Nv).cpu().numpy()
    assert_close(y, orc.project(x.astype(np.float64), Nc, th), 1e-5)
    e = rng.normal(size=(Nv, Nc, Wl)).astype(np.float32)
    xb = fx.backproject(_dev(e), N).cpu().numpy()
    assert_close(xb, orc.backproject(e.astype(np.float64), N, th), 1e-5)


def test_mbir_channel_chunked_matches_oracle(fx, orc):
    # 180 x 96 rays x 1024 values (71 MB): the MBIR gathers run in channel chunks.
    # (The detector is kept about 1.5 N wide: sigma_x ~ mean / Nc, so a detector much
    # wider than the image makes the p = 1.2 prior nearly non-smooth and the iterates
    # sensitive to rounding at the 1e-3 level, a property of the problem, not the chunks.)
    N, Nc, Nv, Nr, K = 64, 96, 180, 128, 8
    V = _sino(orc, N, Nc, Nv, Nr, K, seed=9)
    sv, sx = orc.mbir_sigmas(V.astype(np.float64).reshape(-1, K), K, Nc)
    ref = orc.mbir(V.astype(np.float64), N, Nr, K, _angles(Nv), sv, sx, iters=3, momentum=True)
    got = fx.reconstruct(_dev(V), N, Nr, K, 3, momentum=True).cpu().numpy()
    assert_close(got, ref, 1e-4)


def test_full_size_projector_pair_and_mbir(fx, orc):
    # the 3-D workload's shape in the benchmark's launch configuration (N = 128, 64 slices x
    # K = 5 channels = 320 values per pixel, 90 views x 128 bins): both gathers and two MBIR
    # iterations with momentum against the FP64 oracle over every output
    N, Nc, Nv, Nr, K = 128, 128, 90, 64, 5
    Wl = Nr * K
    rng = np.random.default_rng(700)
    x = rng.uniform(0, 1, size=(N, N, Wl)).astype(np.float32)
    y = fx.project(_dev(x), Nc, Nv).cpu().numpy()
    ref = orc.project(x.astype(np.float64), Nc, _angles(Nv))
    assert_close(y, ref, 1e-5)
    e = rng.normal(size=(Nv, Nc, Wl)).astype(np.float32)
    xb = fx.backproject(_dev(e), N).cpu().numpy()
    assert_close(xb, orc.backproject(e.astype(np.float64), N, _angles(Nv)), 1e-5)
    V = ref.astype(np.float32)
    sv, sx = orc.mbir_sigmas(V.astype(np.float64).reshape(-1, K), K, Nc)
    got = fx.reconstruct(_dev(V), N, Nr, K, 2, momentum=True).cpu().numpy()
    want = orc.mbir(V.astype(np.float64), N, Nr, K, _angles(Nv), sv, sx, iters=2, momentum=True)
    assert_close(got, want, 1e-4)


@pytest.mark.parametrize("Wl", [4096, 4092, 1023, 2056])
def test_wide_channel_vectors(fx, orc, Wl):
    # the widest channel vectors the projector takes (1..1024, or multiples of 4 up to
    # 4096) on a small image, where no L2 chunking splits them: up to 1023 threads per item
    N, Nc, Nv = 8, 12, 6
    rng = np.random.default_rng(800 + Wl)
    x = rng.uniform(0, 1, size=(N, N, Wl)).astype(np.float32)
    y = fx.project(_dev(x), Nc, Nv).cpu().numpy()
    assert_close(y, orc.project(x.astype(np.float64), Nc, _angles(Nv)), 1e-5)
    e = rng.normal(size=(Nv, Nc, Wl)).astype(np.float32)
    xb = fx.backproject(_dev(e), N).cpu().numpy()
    assert_close(xb, orc.backproject(e.astype(np.float64), N, _angles(Nv)), 1e-5)


def test_too_wide_channel_vectors_are_rejected(fx):
    from paper_2410_22500_gb300 import fhr

    for Wl in (4100, 1025):
        with pytest.raises(fhr.FhrError):
            fx.project(_dev(np.zeros((8, 8, Wl), np.float32)), 12, 6)


# Shapes that take the shared-memory staged gathers (Nc and Wl multiples of 4): ragged ray
# blocks (Nc not a multiple of 32), ragged 8 x 8 tiles (N not a multiple of 8), ragged channel
# chunks (Wl not a multiple of 64), runs and slabs clipped to small images and detectors.
TMA_GEOMS = [(61, 36, 50, 68), (256, 256, 120, 64), (5, 8, 9, 16), (13, 12, 33, 4), (100, 132, 77, 1540),
             (57, 60, 45, 200)]


@pytest.mark.parametrize("N,Nc,Nv,Wl", TMA_GEOMS)
def test_staged_gathers_match_oracle(fx, orc, N, Nc, Nv, Wl):
    rng = np.random.default_rng(900 + N + Wl)
    th = _angles(Nv)
    x = rng.uniform(0, 1, size=(N, N, Wl)).astype(np.float32)
    y = fx.project(_dev(x), Nc, Nv).cpu().numpy()
    assert_close(y, orc.project(x.astype(np.float64), Nc, th), 1e-5, what="forward")
    e = rng.normal(size=(Nv, Nc, Wl)).astype(np.float32)
    xb = fx.backproject(_dev(e), N).cpu().numpy()
    assert_close(xb, orc.backproject(e.astype(np.float64), N, th), 1e-5, what="backward")


def test_staged_gathers_custom_angles_and_adjoint(fx, orc):
    import torch

    rng = np.random.default_rng(950)
    N, Nc, Nv, Wl = 70, 100, 23, 8
    th = np.sort(rng.uniform(0, math.pi, Nv))
    ang = torch.from_numpy(th).cuda()
    x = rng.normal(size=(N, N, Wl)).astype(np.float32)
    yv = rng.normal(size=(Nv, Nc, Wl)).astype(np.float32)
    Ax = fx.project(_dev(x), Nc, Nv, angles=ang).cpu().numpy()
    Aty = fx.backproject(_dev(yv), N, angles=ang).cpu().numpy()
    assert_close(Ax, orc.project(x.astype(np.float64), Nc, th), 1e-5)
    assert_close(Aty, orc.backproject(yv.astype(np.float64), N, th), 1e-5)
    lhs = np.sum(Ax.astype(np.float64) * yv)
    rhs = np.sum(x.astype(np.float64) * Aty)
    assert abs(lhs - rhs) <= 1e-6 * np.sqrt(np.sum(Ax.astype(np.float64) ** 2) * np.sum(yv.astype(np.float64) ** 2))


@pytest.mark.parametrize("N,Nc,Nv,Nr,K,momentum,p", [(61, 36, 50, 4, 3, True, 1.2), (40, 64, 90, 2, 2, False, 1.5),
                                                     (29, 44, 31, 1, 8, True, 2.0)])
def test_staged_mbir_matches_oracle(fx, orc, N, Nc, Nv, Nr, K, momentum, p):
    V = _sino(orc, N, Nc, Nv, Nr, K, seed=N + 7 * Nr)
    sv, sx = orc.mbir_sigmas(V.astype(np.float64).reshape(-1, K), K, Nc)
    ref = orc.mbir(V.astype(np.float64), N, Nr, K, _angles(Nv), sv, sx, p=p, iters=12, momentum=momentum)
    got = fx.reconstruct(_dev(V), N, Nr, K, 12, p=p, momentum=momentum).cpu().numpy()
    assert_close(got, ref, 1e-4)
