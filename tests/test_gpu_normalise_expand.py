"""GPU parity of the normalisation (Eq. neglogattenuation, App. A) and expansion (Eq. sub_expansion) kernels."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch

    a = np.ascontiguousarray(a)
    if a.dtype == np.uint16:          # torch has partial uint16 support: move the bits as int16
        a = a.view(np.int16)
    return torch.from_numpy(a).cuda()


def _rows(P, Nk):
    return P[:, :Nk].float().cpu().numpy().astype(np.float64)


# GPU: p = (hi0 - hi) + (lo0 - lo) from FP32 pairs hi + lo of ln y0 and ln y (each pair
# within 2^-48 ln 65535 of the logarithm): error <= 1 ulp(p) plus a few 2^-24 of the pair
# differences, at most 1.5e-7 absolute near p = 0 and 2.4e-7 relative
ATOL, RTOL = 1.5e-7, 2.4e-7


# Nk % 8 == 0, 4, 2 and odd take the 16-, 8-, 4- and 2-byte count loads
@pytest.mark.parametrize("shape", [(3, 2, 5, 16), (4, 3, 7, 37), (2, 1, 48, 128), (1, 1, 1, 8), (3, 2, 5, 44),
                                   (2, 3, 7, 38), (2, 2, 9, 1500)])
def test_normalise_matches_oracle(fx, orc, shape):
    rng = np.random.default_rng(100 + shape[-1])
    Nv, Nr, Nc, Nk = shape
    y = rng.integers(0, 3000, size=shape).astype(np.uint16)
    y[0, 0, 0, :3] = [0, 65535, 1]          # zero count, maximum, one
    y0 = rng.integers(0, 3000, size=(Nr, Nc, Nk)).astype(np.uint16)
    y0[0, 0, :2] = [0, 65535]
    P = fx.normalise(_dev(y), _dev(y0))
    ref = orc.normalise(y, y0)
    got = _rows(P, Nk)
    np.testing.assert_allclose(got, ref, atol=ATOL, rtol=RTOL)
    if P.shape[1] > Nk:   # padding columns are written as zero
        assert float(P[:, Nk:].abs().max()) == 0.0


def test_normalise_dead_bins_and_offset(fx, orc):
    rng = np.random.default_rng(101)
    Nv, Nr, Nc, Nk = 5, 4, 9, 24
    y0 = rng.integers(800, 1200, size=(Nr, Nc, Nk)).astype(np.uint16)
    y = (y0[None] * rng.uniform(0.2, 1.1, size=(Nv, Nr, Nc, Nk))).astype(np.uint16)
    bg = np.zeros((Nr, Nc), np.uint8)
    bg[:, :2] = 1
    dead = np.zeros(Nk, np.uint8)
    dead[[0, 5, 23]] = 1
    P, b = fx.normalise(_dev(y), _dev(y0), bg=_dev(bg), dead=_dev(dead))
    ref, bref = orc.normalise(y, y0, bg=bg, dead=dead, return_offset=True)
    np.testing.assert_allclose(b.cpu().numpy(), bref, atol=5e-7, rtol=1e-6)
    np.testing.assert_allclose(_rows(P, Nk), ref, atol=2e-6, rtol=1e-6)
    assert float(P[:, [0, 5, 23]].abs().max()) == 0.0


@pytest.mark.parametrize("p_dtype", ["f32", "bf16"])
def test_normalise_dead_pixel_bins_and_offset(fx, orc, p_dtype):
    # a per-(detector pixel, bin) mask, also inside the background region (those entries
    # carry zero counts and must not enter the offset), a ragged Nk and a padded row
    from paper_2410_22500_gb300 import fhr

    rng = np.random.default_rng(102)
    Nv, Nr, Nc, Nk = 6, 3, 11, 37
    y0 = rng.integers(800, 1200, size=(Nr, Nc, Nk)).astype(np.uint16)
    y = (y0[None] * rng.uniform(0.2, 1.1, size=(Nv, Nr, Nc, Nk))).astype(np.uint16)
    bg = np.zeros((Nr, Nc), np.uint8)
    bg[:, :3] = 1
    dead = (rng.uniform(size=(Nr, Nc, Nk)) < 0.15).astype(np.uint8)
    dead[:, :3, 4] = 1                     # bin 4 dead across the whole background
    y[:, dead.astype(bool)] = 0
    y0[dead.astype(bool)] = 0
    pd = fhr.BF16 if p_dtype == "bf16" else fhr.F32
    P, b = fx.normalise(_dev(y), _dev(y0), bg=_dev(bg), dead=_dev(dead), p_dtype=pd)
    ref, bref = orc.normalise(y, y0, bg=bg, dead=dead, return_offset=True)
    np.testing.assert_allclose(b.cpu().numpy(), bref, atol=5e-7, rtol=1e-6)
    assert np.all(b.cpu().numpy()[:, 4] == 0)
    got = P.float().cpu().numpy()[:, :Nk]
    if p_dtype == "bf16":
        np.testing.assert_allclose(got, ref, atol=2e-6, rtol=2 ** -8)
    else:
        np.testing.assert_allclose(got, ref, atol=2e-6, rtol=1e-6)
    for v in range(Nv):
        for r in range(Nr):
            j = (v * Nc + np.arange(Nc)) * Nr + r
            assert np.all(got[j][dead[r].astype(bool)] == 0)


def test_normalise_bf16_rounding(fx, orc):
    import torch
    from paper_2410_22500_gb300 import fhr

    rng = np.random.default_rng(102)
    y = rng.integers(1, 2000, size=(3, 2, 6, 40)).astype(np.uint16)
    y0 = rng.integers(1000, 2000, size=(2, 6, 40)).astype(np.uint16)
    P = fx.normalise(_dev(y), _dev(y0), p_dtype=fhr.BF16)
    assert P.dtype == torch.bfloat16 and P.shape[1] == 40
    ref = orc.normalise(y, y0)
    # round-to-nearest bf16 (8 significant bits) of the f32 value: error <= half an ulp,
    # i.e. <= 2^-8 of the value (+ the f32 error)
    got = _rows(P, 40)
    assert np.all(np.abs(got - ref) <= 2.0 ** -8 * np.abs(ref) + 2 * ATOL)


def test_normalise_full_size_sampled(fx, orc):
    # the 3-D workload's full counts array (90 x 64 x 128 x 1200), checked on sampled rows
    import torch
    from paper_2410_22500_gb300 import synth

    pb = synth.volume_3d_f32()
    y, y0 = synth.counts_torch(pb)
    dead = _dev(pb.dead_bins)
    P = fx.normalise(y, y0, dead=dead)
    torch.cuda.synchronize()
    g = pb.geom
    rng = np.random.default_rng(103)
    rows = rng.choice(g.Np, size=64, replace=False)
    v = rows // (g.Nc * g.Nr)
    c = (rows // g.Nr) % g.Nc
    r = rows % g.Nr
    ys = y[torch.as_tensor(v), torch.as_tensor(r), torch.as_tensor(c)].cpu().numpy().view(np.uint16)
    y0s = y0[torch.as_tensor(r), torch.as_tensor(c)].cpu().numpy().view(np.uint16)
    for i in range(len(rows)):
        ref = orc.normalise(ys[i:i + 1].reshape(1, 1, 1, -1), y0s[i:i + 1].reshape(1, 1, -1), dead=pb.dead_bins)
        np.testing.assert_allclose(P[rows[i], :pb.Nk].double().cpu().numpy(), ref[0], atol=ATOL, rtol=RTOL)


@pytest.mark.parametrize("N,Nr,K,Nk,k0,k1", [(5, 3, 3, 17, 0, 0), (8, 2, 5, 64, 0, 0), (6, 1, 8, 40, 7, 31),
                                             (4, 4, 1, 12, 0, 0)])
def test_expand_matches_oracle(fx, orc, N, Nr, K, Nk, k0, k1):
    rng = np.random.default_rng(110 + Nk)
    xs = rng.uniform(0, 1, size=(N, N, Nr * K)).astype(np.float32)
    D = rng.uniform(0, 1, size=(Nk, K)).astype(np.float32)
    xh = fx.expand(_dev(xs), _dev(D), N, Nr, k0=k0, k1=k1).cpu().numpy()
    ref = orc.expand(xs.astype(np.float64), D.astype(np.float64), N, Nr)
    if k0 or k1:
        ref = ref[..., k0:k1]
    # K fused multiply-adds in FP32: |err| <= K * 2^-24 * sum |x d|
    np.testing.assert_allclose(xh, ref, rtol=K * 1.2e-7 * 4, atol=1e-7)


def test_expand_bf16(fx, orc):
    from paper_2410_22500_gb300 import fhr

    rng = np.random.default_rng(111)
    N, Nr, K, Nk = 7, 2, 4, 36
    xs = rng.uniform(0, 1, size=(N, N, Nr * K)).astype(np.float32)
    D = rng.uniform(0, 1, size=(Nk, K)).astype(np.float32)
    xh = fx.expand(_dev(xs), _dev(D), N, Nr, xh_dtype=fhr.BF16).float().cpu().numpy()
    ref = orc.expand(xs.astype(np.float64), D.astype(np.float64), N, Nr)
    assert np.all(np.abs(xh - ref) <= 2.0 ** -8 * np.abs(ref) + 1e-6)


def test_expand_full_size_sampled(fx, orc):
    # x^h for the 3-D workload (64 x 128 x 128 voxels x 1200 bins, 5 GB in f32), sampled pixels
    # (every slice and bin of each) against the oracle's expansion of that pixel
    import torch

    N, Nr, K, Nk = 128, 64, 5, 1200
    rng = np.random.default_rng(111)
    xs = rng.uniform(0, 1, size=(N, N, Nr * K)).astype(np.float32)
    D = rng.uniform(0, 1, size=(Nk, K)).astype(np.float32)
    xh = fx.expand(_dev(xs), _dev(D), N, Nr)
    pix = rng.choice(N * N, 48, replace=False)
    pix[:2] = [0, N * N - 1]
    for p in pix:
        i, j = divmod(int(p), N)
        got = xh[:, i, j, :].cpu().numpy()
        ref = orc.expand(xs[i:i + 1, j:j + 1].astype(np.float64), D.astype(np.float64), 1, Nr)[:, 0, 0, :]
        np.testing.assert_allclose(got, ref, rtol=K * 1.2e-7 * 4, atol=1e-7)
    del xh
    torch.cuda.empty_cache()
