"""Pins of the oracle's MBIR solve of Eq. (recon) (SQS iterations, qGGMRF prior)."""
import math

import numpy as np
import pytest


def _angles(Nv):
    return np.arange(Nv) * math.pi / Nv


@pytest.mark.parametrize("p,T,sx", [(1.2, 1.0, 0.3), (1.5, 2.0, 1.7), (1.0, 0.5, 0.05)])
def test_influence_is_derivative_over_delta(orc, p, T, sx):
    # rho'(d)/d by central differences of rho itself
    for d in [-3.0, -0.4, -1e-3, 2e-3, 0.1, 0.77, 5.0]:
        h = 1e-6 * max(abs(d), 1e-3)
        num = (orc.qggmrf_rho(d + h, sx, p, 2.0, T) - orc.qggmrf_rho(d - h, sx, p, 2.0, T)) / (2 * h)
        assert abs(num / d - orc.qggmrf_influence(d, sx, p, 2.0, T)) <= 1e-6 * abs(num / d)


def test_rho_reduces_to_gaussian_when_p_equals_q(orc):
    # u = 1 when q = p: rho = |d|^p / (2 p sx^p); p = q = 2 gives d^2 / (4 sx^2)
    for d in [-2.0, 0.3, 1.1]:
        assert abs(orc.qggmrf_rho(d, 0.7, 2.0, 2.0, 1.3) - d * d / (4 * 0.49)) < 1e-15
    assert orc.qggmrf_influence(0.0, 0.7, 1.2, 2.0, 1.0) > 0      # finite at 0 for q = 2


def test_no_prior_converges_to_least_squares(orc):
    # beta = 0 and consistent data from a positive image: the minimiser of Eq. (recon)
    # is the least-squares solution, i.e. the image itself (A has full column rank)
    rng = np.random.default_rng(42)
    N, Nc, Nv, Nr, K = 4, 8, 16, 1, 2
    th = _angles(Nv)
    A = orc.system_matrix(N, Nc, th)
    assert np.linalg.matrix_rank(A) == N * N
    xt = rng.uniform(0.5, 1.5, size=(N, N, Nr * K))
    V = orc.project(xt, Nc, th)
    # SQS with momentum converges slowly (cond(A^T A) ~ 7e3): 20000 steps reach ~1e-6
    x = orc.mbir(V, N, Nr, K, th, np.array([1.0, 0.5]), np.array([1.0, 1.0]), beta=0.0,
                 iters=20000, momentum=True)
    xl = np.linalg.lstsq(A, V.reshape(-1, K), rcond=None)[0].reshape(N, N, K)
    np.testing.assert_allclose(x, xl, atol=5e-6)


def _laplacian(N, Nr):
    """Weighted graph Laplacian of the prior's neighbourhood over (iy, ix, r)."""
    offs = [(-1, 0, 0, 1.0), (1, 0, 0, 1.0), (0, -1, 0, 1.0), (0, 1, 0, 1.0),
            (-1, -1, 0, 2 ** -0.5), (-1, 1, 0, 2 ** -0.5), (1, -1, 0, 2 ** -0.5), (1, 1, 0, 2 ** -0.5)]
    if Nr > 1:
        offs += [(0, 0, -1, 1.0), (0, 0, 1, 1.0)]
    z = sum(o[3] for o in offs)
    n = N * N * Nr
    L = np.zeros((n, n))
    idx = lambda iy, ix, r: (iy * N + ix) * Nr + r
    for iy in range(N):
        for ix in range(N):
            for r in range(Nr):
                for dy, dx, dr, w in offs:
                    yy, xx, rr = iy + dy, ix + dx, r + dr
                    if 0 <= yy < N and 0 <= xx < N and 0 <= rr < Nr:
                        L[idx(iy, ix, r), idx(iy, ix, r)] += w / z
                        L[idx(iy, ix, r), idx(yy, xx, rr)] -= w / z
    return L


def test_quadratic_prior_solves_linear_system(orc):
    # p = q = 2: rho(d) = d^2/(4 sx^2), so Eq. (recon) is quadratic and its minimiser
    # (positivity inactive) solves (A^T A / sv^2 + L / (2 sx^2)) x = A^T V / sv^2
    rng = np.random.default_rng(43)
    N, Nc, Nv, Nr, K = 6, 10, 12, 2, 2
    th = _angles(Nv)
    A = orc.system_matrix(N, Nc, th)
    xt = rng.uniform(0.8, 1.2, size=(N, N, Nr * K))
    V = orc.project(xt, Nc, th) + 0.01 * rng.normal(size=(Nv, Nc, Nr * K))
    sv, sx = np.array([0.1, 0.3]), np.array([0.3, 0.6])
    x = orc.mbir(V, N, Nr, K, th, sv, sx, p=2.0, q=2.0, iters=10000, momentum=True)
    L = _laplacian(N, Nr)
    AtA = np.kron(A.T @ A, np.eye(Nr))          # acts on (pixel, slice) ordering
    for j in range(K):
        rhs = np.kron(A.T, np.eye(Nr)) @ V[:, :, j::K].reshape(-1) / sv[j] ** 2
        H = AtA / sv[j] ** 2 + L / (2 * sx[j] ** 2)
        sol = np.linalg.solve(H, rhs)
        assert sol.min() > 0
        np.testing.assert_allclose(x[:, :, j::K].reshape(-1), sol, atol=1e-7 * np.abs(sol).max())


def test_sqs_cost_monotone_and_nonnegative(orc):
    # plain SQS majorises the cost at every step (qGGMRF with p <= q = 2)
    rng = np.random.default_rng(44)
    N, Nc, Nv, Nr, K = 12, 18, 15, 3, 2
    th = _angles(Nv)
    xt = np.zeros((N, N, Nr * K))
    xt[3:9, 4:8] = rng.uniform(0.5, 1.0, size=(6, 4, Nr * K))
    V = orc.project(xt, Nc, th) + 0.05 * rng.normal(size=(Nv, Nc, Nr * K))
    sv, sx = orc.mbir_sigmas(V.reshape(-1, K), K, Nc)
    x, cost = orc.mbir(V, N, Nr, K, th, sv, sx, p=1.2, iters=40, cost=True)
    c0 = orc.mbir_cost(V, np.zeros_like(x), N, Nr, K, th, sv, sx)
    assert cost[0] <= c0
    assert np.all(np.diff(cost) <= 1e-12 * np.abs(cost[:-1]))
    assert np.all(x >= 0)


def test_noise_free_inverse_crime_recovery(orc):
    # consistent data from the same A ("inverse crime") at high assumed SNR (small
    # sigma_v): the phantom is recovered closely
    from paper_2410_22500_gb300 import synth

    N, Nc, Nv = 16, 24, 40
    ph = synth.Phantom(np.array([[2.0, -1.0, 0.0, 4.5, 3.0, np.inf, 0.3]]))
    xm = synth.volume_fractions(ph, N, 1, sub=4)[0]       # [N][N][1]
    th = _angles(Nv)
    V = orc.project(xm, Nc, th)
    sv, sx = orc.mbir_sigmas(V.reshape(-1, 1), 1, Nc, snr_db=60.0)
    x = orc.mbir(V, N, 1, 1, th, sv, sx, iters=600, momentum=True)
    assert np.linalg.norm(x - xm) / np.linalg.norm(xm) < 0.02


def test_sigma_reading_by_hand(orc):
    # sigma_v = rms(V_j) 10^(-snr/20), sigma_x = 0.2 mean(V_j) / Nc, an all-zero channel 1:
    # channel 0 = [3, 4]: rms^2 = 12.5, so sigma_v = sqrt(12.5e-3) at 30 dB, sigma_x = 0.2 * 3.5 / 10
    V = np.array([[3.0, 0.0], [4.0, 0.0]])
    sv, sx = orc.mbir_sigmas(V, 2, 10, snr_db=30.0)
    np.testing.assert_allclose(sv, [np.sqrt(12.5e-3), 1.0], rtol=1e-14)
    np.testing.assert_allclose(sx, [0.07, 1.0], rtol=1e-14)


def test_momentum_point_clamp_by_hand(orc):
    # The momentum point of the SQS iterations is z = max(0, x' + a (x' - x)) (reading of
    # Eq. (recon) with positivity: the surrogate is built at a feasible point).  Worked by
    # hand on a 2 x 2 image seen at 0 and pi/2 by two unit bins, so each ray sums one
    # column or one row: A^T A 1 = 4 at every pixel, and with beta = 0 one step is
    # x <- max(0, z + A^T (V - A z) / 4).  Data: columns (0.1, 2), rows (0.1, 2).
    #   x1 = A^T V / 4             = [[0.05, 0.525], [0.525, 1.0]]      (a1 = 0, z1 = x1)
    #   A z1: cols = rows = (0.575, 1.525); residual (-0.475, 0.475) on both
    #   x2 = max(0, x1 + A^T r / 4) = [[0, 0.525], [0.525, 1.2375]]     (pixel (0,0): 0.05 - 0.2375 < 0)
    #   a2 = (t1 - 1) / t2, t1 = (1 + sqrt 5) / 2, t2 = (1 + sqrt(1 + 4 t1^2)) / 2
    #   z2 = max(0, x2 + a2 (x2 - x1)): pixel (0,0) gives max(0, -0.05 a2) = 0
    #   A z2: cols = rows = (0.525, 1.7625 + 0.2375 a2); residual (-0.425, 0.2375 (1 - a2))
    #   x3 = [[0, 0.525 + (0.2375 (1 - a2) - 0.425) / 4], [same, 1.35625 + 0.11875 a2]]
    # Without the clamp z2[0,0] = -0.05 a2 and x3[0,1] would be larger by 0.0125 a2 (3.5e-3).
    t1 = 0.5 * (1 + math.sqrt(5.0))
    t2 = 0.5 * (1 + math.sqrt(1 + 4 * t1 * t1))
    a2 = (t1 - 1) / t2
    V = np.array([[0.1, 2.0], [0.1, 2.0]]).reshape(2, 2, 1)     # [view][bin][channel]
    th = np.array([0.0, math.pi / 2])
    one = np.array([1.0])
    x2 = orc.mbir(V, 2, 1, 1, th, one, one, beta=0.0, iters=2, momentum=True)[:, :, 0]
    np.testing.assert_allclose(x2, [[0.0, 0.525], [0.525, 1.2375]], atol=1e-12)
    x3 = orc.mbir(V, 2, 1, 1, th, one, one, beta=0.0, iters=3, momentum=True)[:, :, 0]
    off = 0.525 + (0.2375 * (1 - a2) - 0.425) / 4
    want = np.array([[0.0, off], [off, 1.35625 + 0.11875 * a2]])
    np.testing.assert_allclose(x3, want, atol=1e-12)
    assert abs(0.0125 * a2) > 1e-3     # the unclamped point would miss this pin
