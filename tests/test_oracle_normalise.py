"""Pins of the oracle's normalisation (Eq. neglogattenuation, Appendix A)."""
import math
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def _golden():
    rows = []
    with open(os.path.join(HERE, "golden", "normalise_cases.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                y, y0, p = line.split()
                rows.append((int(y), int(y0), float(p)))
    return rows


def test_golden_cases(orc):
    rows = _golden()
    n = len(rows)
    y = np.array([r[0] for r in rows], dtype=np.uint16).reshape(1, 1, 1, n)
    y0 = np.array([r[1] for r in rows], dtype=np.uint16).reshape(1, 1, n)
    P = orc.normalise(y, y0)
    np.testing.assert_allclose(P[0], [r[2] for r in rows], rtol=1e-15, atol=0)


def test_powers_of_two_exact(orc):
    # y0 = y * 2^m  =>  p = ln(y0) - ln(y) = m ln 2 (Eq. neglogattenuation); each log is
    # correctly rounded, so the difference is within a few ulp of ln(y0) <= ln(65535)
    rng = np.random.default_rng(1)
    Nv, Nr, Nc, Nk = 3, 2, 4, 16
    m = rng.integers(0, 6, size=(Nv, Nr, Nc, Nk))
    y0 = (rng.integers(1, 1000, size=(Nr, Nc, Nk)) << 5).astype(np.uint16)
    y = (y0[None].astype(np.int64) >> m).astype(np.uint16)
    P = orc.normalise(y, y0)
    tol = 4 * np.finfo(float).eps * math.log(65535)
    for v in range(Nv):
        for r in range(Nr):
            for c in range(Nc):
                j = (v * Nc + c) * Nr + r
                np.testing.assert_allclose(P[j], m[v, r, c] * math.log(2.0), rtol=0, atol=tol)


def test_pixel_order_vcr(orc):
    # P row j = (v*Nc + c)*Nr + r holds pixel (v, r, c): encode (v, r, c) into the counts
    Nv, Nr, Nc, Nk = 3, 4, 5, 2
    y0 = np.full((Nr, Nc, Nk), 60000, dtype=np.uint16)
    y = np.empty((Nv, Nr, Nc, Nk), dtype=np.uint16)
    for v in range(Nv):
        for r in range(Nr):
            for c in range(Nc):
                y[v, r, c, :] = 1 + v * 100 + r * 10 + c
    P = orc.normalise(y, y0)
    for v in range(Nv):
        for r in range(Nr):
            for c in range(Nc):
                j = (v * Nc + c) * Nr + r
                want = math.log(60000) - math.log(1 + v * 100 + r * 10 + c)
                assert abs(P[j, 0] - want) < 1e-13


def test_planted_offset_recovered(orc):
    # Appendix A: the background mean of -log(y/y0) is b_{v,k}; plant alpha = 2^-e
    rng = np.random.default_rng(2)
    Nv, Nr, Nc, Nk = 4, 3, 6, 8
    e = rng.integers(0, 3, size=(Nv, Nk))           # b = e ln 2
    a = rng.integers(0, 4, size=(Nv, Nr, Nc, Nk))   # object attenuation a ln 2
    bg = np.zeros((Nr, Nc), dtype=np.uint8)
    bg[:, 0] = 1
    bg[:, -1] = 1
    a[:, bg.astype(bool), :] = 0
    y0 = np.full((Nr, Nc, Nk), 4096, dtype=np.uint16)
    y = (4096 >> (a + e[:, None, None, :])).astype(np.uint16)
    P, b = orc.normalise(y, y0, bg=bg, return_offset=True)
    np.testing.assert_allclose(b, e * math.log(2.0), rtol=1e-15, atol=1e-15)
    for v in range(Nv):
        for r in range(Nr):
            for c in range(Nc):
                j = (v * Nc + c) * Nr + r
                np.testing.assert_allclose(P[j], a[v, r, c] * math.log(2.0), atol=1e-14)


def test_dead_bins_zero(orc):
    rng = np.random.default_rng(3)
    y = rng.integers(0, 500, size=(2, 2, 3, 10)).astype(np.uint16)
    y0 = rng.integers(400, 900, size=(2, 3, 10)).astype(np.uint16)
    dead = np.zeros(10, dtype=np.uint8)
    dead[[1, 7]] = 1
    P = orc.normalise(y, y0, dead=dead)
    assert np.all(P[:, [1, 7]] == 0)
    P2 = orc.normalise(y, y0)
    np.testing.assert_array_equal(P[:, dead == 0], P2[:, dead == 0])
    assert np.all(P2 >= 0)


def test_noise_free_projection_recovered(orc):
    # counts from the generator without noise: p recovered up to count rounding, |dp| <= ~1/(2y)
    from paper_2410_22500_gb300 import synth

    pb = synth.make_problem(N=16, Nr=2, Nc=24, Nv=6, Nk=12, Nm=2, I0=60000, seed=5)
    y, y0 = synth.counts_numpy(pb, noise=False)
    P = orc.normalise(y, y0)
    p = synth.noise_free_projection(pb)              # [Nv][Nr][Nc][Nk]
    pv = p.transpose(0, 2, 1, 3).reshape(-1, pb.Nk)  # (v, c, r) order
    bound = 0.6 / np.maximum(y.transpose(0, 2, 1, 3).reshape(-1, pb.Nk).astype(float), 1)
    assert np.all(np.abs(P - pv) <= bound + 1e-12)


def test_dead_pixel_bins_zero_and_rest_unchanged(orc):
    # a per-(detector pixel, bin) mask zeroes exactly those entries in every view
    rng = np.random.default_rng(4)
    Nv, Nr, Nc, Nk = 3, 2, 4, 9
    y = rng.integers(0, 500, size=(Nv, Nr, Nc, Nk)).astype(np.uint16)
    y0 = rng.integers(400, 900, size=(Nr, Nc, Nk)).astype(np.uint16)
    dead = (rng.uniform(size=(Nr, Nc, Nk)) < 0.2).astype(np.uint8)
    P = orc.normalise(y, y0, dead=dead)
    P2 = orc.normalise(y, y0)
    for v in range(Nv):
        for r in range(Nr):
            for c in range(Nc):
                j = (v * Nc + c) * Nr + r
                m = dead[r, c].astype(bool)
                assert np.all(P[j, m] == 0)
                np.testing.assert_array_equal(P[j, ~m], P2[j, ~m])


def test_per_bin_mask_equals_its_broadcast(orc):
    rng = np.random.default_rng(5)
    Nv, Nr, Nc, Nk = 2, 3, 4, 7
    y = rng.integers(0, 300, size=(Nv, Nr, Nc, Nk)).astype(np.uint16)
    y0 = rng.integers(200, 600, size=(Nr, Nc, Nk)).astype(np.uint16)
    bg = np.zeros((Nr, Nc), np.uint8)
    bg[:, 0] = 1
    dead = np.zeros(Nk, np.uint8)
    dead[[2, 5]] = 1
    Pa, ba = orc.normalise(y, y0, bg=bg, dead=dead, return_offset=True)
    Pb, bb = orc.normalise(y, y0, bg=bg, dead=np.broadcast_to(dead, (Nr, Nc, Nk)).copy(), return_offset=True)
    np.testing.assert_array_equal(Pa, Pb)
    np.testing.assert_array_equal(ba, bb)
    assert np.all(ba[:, [2, 5]] == 0)      # no live background entry


def test_background_mean_skips_dead_entries(orc):
    # App. A offset with two background pixels, one of them dead in bin 1 with zero counts:
    # b is then the other pixel's -log(y/y0) alone (worked by hand: ln(800/200) = 2 ln 2),
    # and the planted offset is removed from the object pixel
    y0 = np.full((1, 3, 2), 800, np.uint16)
    y = np.zeros((1, 1, 3, 2), np.uint16)
    y[0, 0, 0] = [400, 200]                 # background pixel 0: b = ln 2, 2 ln 2
    y[0, 0, 1] = [400, 0]                   # background pixel 1: bin 1 dead (no counts)
    y[0, 0, 2] = [100, 50]                  # object pixel
    bg = np.array([[1, 1, 0]], np.uint8)
    dead = np.zeros((1, 3, 2), np.uint8)
    dead[0, 1, 1] = 1
    P, b = orc.normalise(y, y0, bg=bg, dead=dead, return_offset=True)
    np.testing.assert_allclose(b[0], [math.log(2.0), 2 * math.log(2.0)], rtol=1e-15)
    np.testing.assert_allclose(P[2], [math.log(8.0) - math.log(2.0), math.log(16.0) - 2 * math.log(2.0)],
                               rtol=1e-15)
    assert P[1, 1] == 0.0
