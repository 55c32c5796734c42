"""Pins of the oracle's filtered back-projection (the FBP variant of FHR)."""
import math

import numpy as np

import oracle


def test_ramp_frequency_response_is_abs_f():
    # the sampled band-limited ramp has frequency response |f| on |f| <= 1/2
    M = 20000
    n = np.arange(-M, M + 1)
    h = np.array([oracle.ramp(int(k)) for k in n])
    for f in (0.0, 0.05, 0.13, 0.25, 0.37, 0.49):
        H = float(np.sum(h * np.cos(2 * math.pi * f * n)))
        assert abs(H - f) < 2e-4, (f, H)


def test_ramp_is_even_with_zero_even_taps():
    for k in range(1, 40):
        assert oracle.ramp(k) == oracle.ramp(-k)
        if k % 2 == 0:
            assert oracle.ramp(k) == 0.0
        else:
            assert oracle.ramp(k) < 0.0
    assert oracle.ramp(0) > 0.0


def test_filter_is_the_linear_convolution():
    rng = np.random.default_rng(1)
    Nv, Nc, Wl = 3, 17, 2
    p = rng.normal(size=(Nv, Nc, Wl))
    q = oracle.ramp_filter(p)
    h = np.array([oracle.ramp(k) for k in range(-(Nc - 1), Nc)])
    for v in range(Nv):
        for w in range(Wl):
            full = np.convolve(p[v, :, w], h)
            np.testing.assert_allclose(q[v, :, w], full[Nc - 1:2 * Nc - 1], rtol=1e-13, atol=1e-15)


def _disk_sinogram(R, Nc, Nv, sub=16):
    u = (np.arange(Nc) - (Nc - 1) / 2.0)[:, None] + (np.arange(sub) + 0.5)[None, :] / sub - 0.5
    chord = 2.0 * np.sqrt(np.maximum(R * R - u * u, 0.0)).mean(axis=1)
    return np.repeat(chord[None, :], Nv, axis=0)[..., None]


def test_fbp_inverts_the_disk_transform():
    # FBP of the analytic (bin-averaged) projections of a unit disk gives the disk
    N, Nc, Nv, R = 64, 96, 180, 20.0
    th = np.arange(Nv) * math.pi / Nv
    x = oracle.fbp(_disk_sinogram(R, Nc, Nv), N, th)[..., 0]
    c = (np.arange(N) - (N - 1) / 2.0)
    r = np.sqrt(c[:, None] ** 2 + c[None, :] ** 2)
    inside, outside = x[r < 0.8 * R], x[(r > 1.2 * R) & (r < 0.45 * N)]
    assert abs(inside.mean() - 1.0) < 0.02
    assert inside.std() < 0.03
    assert np.sqrt(np.mean(outside ** 2)) < 0.03


def test_fbp_channels_are_independent_and_linear():
    rng = np.random.default_rng(2)
    N, Nc, Nv = 12, 18, 10
    th = np.arange(Nv) * math.pi / Nv
    p = rng.uniform(size=(Nv, Nc, 3))
    x = oracle.fbp(p, N, th)
    for w in range(3):
        np.testing.assert_allclose(x[..., w], oracle.fbp(p[..., w:w + 1], N, th)[..., 0], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(oracle.fbp(2.5 * p, N, th), 2.5 * x, rtol=1e-12, atol=1e-14)
