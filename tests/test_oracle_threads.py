"""The oracle's parallel loops change nothing: every output is the same bit for bit
with one host thread and with several (each sum is taken in a fixed order)."""
import math

import numpy as np


def _run(orc, threads):
    orc.set_threads(threads)
    rng = np.random.default_rng(90)
    N, Nc, Nv, Nr, K = 12, 18, 20, 3, 2
    th = np.arange(Nv) * math.pi / Nv
    x = rng.uniform(size=(N, N, Nr * K))
    y = orc.project(x, Nc, th)
    xb = orc.backproject(y, N, th)
    sv, sx = orc.mbir_sigmas(y.reshape(-1, K), K, Nc)
    xm = orc.mbir(y, N, Nr, K, th, sv, sx, iters=4, momentum=True)
    P = rng.uniform(size=(300, 70))
    D0, W0 = rng.uniform(0.1, 1, size=(70, 3)), rng.uniform(0.1, 1, size=(300, 3))
    D, W, obj = orc.nmf(P, D0, W0, 3)
    xh = orc.expand(xm, D[:, :K], N, Nr)
    counts = rng.integers(0, 900, size=(4, 2, 5, 70)).astype(np.uint16)
    open_beam = rng.integers(500, 1000, size=(2, 5, 70)).astype(np.uint16)
    bg = np.zeros((2, 5), np.uint8)
    bg[:, 0] = 1
    Pn = orc.normalise(counts, open_beam, bg=bg)
    fb = orc.fbp(y, N, th)
    return [y, xb, xm, D, W, obj, xh, Pn, fb]


def test_thread_count_does_not_change_results(orc):
    prev = orc.set_threads(0)
    try:
        a = _run(orc, 1)
        b = _run(orc, 4)
    finally:
        orc.set_threads(prev)
    for u, v in zip(a, b):
        np.testing.assert_array_equal(u, v)
