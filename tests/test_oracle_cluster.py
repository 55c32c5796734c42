"""Pins of the oracle's clustering start (k-means++ seeding with splitmix64,
Lloyd iterations, one HALS V step from zero); the library's added init mode."""
import numpy as np
import pytest

import oracle


def test_splitmix64_published_outputs():
    # first outputs of splitmix64 from state 0 (Steele, Lea and Flood 2014; the
    # reference generator's published sequence)
    got = oracle.splitmix64(0, 3)
    assert [int(v) for v in got] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def _blobs(rng, K, per, Nk, spread=0.01):
    centres = rng.uniform(0.5, 2.0, size=(K, Nk)) * (1 + 3 * np.arange(K))[:, None]
    lab = np.repeat(np.arange(K), per)
    X = centres[lab] + spread * rng.normal(size=(K * per, Nk))
    perm = rng.permutation(K * per)
    return X[perm], lab[perm]


@pytest.mark.parametrize("seed", [0, 1, 7])
def test_separated_clusters_reach_label_means(seed):
    rng = np.random.default_rng(40 + seed)
    K, Nk = 4, 12
    X, lab = _blobs(rng, K, 50, Nk)
    C, got, cost, _ = oracle.kmeans(X, len(X), K, 10, seed)
    # the labelling is the true one up to a permutation of the centres
    for m in range(K):
        members = np.unique(lab[got == m])
        assert len(members) == 1
    assert len(np.unique(got)) == K
    # and each centre is the mean of its members (the Lloyd fixed point)
    for m in range(K):
        np.testing.assert_allclose(C[m], X[got == m].mean(axis=0), rtol=1e-13, atol=1e-13)


def test_lloyd_cost_non_increasing():
    rng = np.random.default_rng(3)
    X = rng.gamma(2.0, size=(300, 9))
    _, _, cost, _ = oracle.kmeans(X, 300, 5, 15, 11)
    assert np.all(np.diff(cost) <= 1e-12 * cost[0])
    # the cost is the sum of squared distances to the nearest centre
    C, lab, cost1, _ = oracle.kmeans(X, 300, 5, 0, 11)
    d = ((X[:, None, :] - C[None]) ** 2).sum(-1)
    assert np.isclose(cost1[0], d.min(axis=1).sum(), rtol=1e-13)
    np.testing.assert_array_equal(lab, d.argmin(axis=1))


def test_single_cluster_is_the_sample_mean():
    rng = np.random.default_rng(4)
    P = rng.uniform(size=(103, 6))
    S = 40
    C, _, _, _ = oracle.kmeans(P, S, 1, 3, 5)
    idx = (np.arange(S) * 103) // S
    np.testing.assert_allclose(C[0], P[idx].mean(axis=0), rtol=1e-14)


def test_first_seed_and_subsample():
    rng = np.random.default_rng(5)
    P = rng.uniform(size=(97, 5))
    S = 31
    _, _, _, seeds = oracle.kmeans(P, S, 3, 0, 123)
    u0 = (int(oracle.splitmix64(123, 1)[0]) >> 11) * 2.0 ** -53
    assert seeds[0] == int(u0 * S)
    assert len(set(seeds.tolist())) == 3


def test_zero_distance_samples_are_never_seeded():
    # ten copies of one spectrum and one distinct spectrum: after the first
    # centre, the only sample with positive distance must be the next seed
    X = np.ones((11, 4))
    X[6] = [5.0, 0.0, 1.0, 2.0]
    for seed in range(20):
        _, _, _, seeds = oracle.kmeans(X, 11, 2, 0, seed)
        if seeds[0] != 6:
            assert seeds[1] == 6


def test_cluster_init_w_step_k1_closed_form():
    # K = 1: D0 = the sample mean spectrum d, and one V step from 0 gives
    # w_j = max(0, <p_j, d> / <d, d>)
    rng = np.random.default_rng(6)
    P = rng.uniform(size=(50, 8))
    D0, W0 = oracle.cluster_init(P, 1, S=50, iters=2, seed=9)
    d = P.mean(axis=0)
    np.testing.assert_allclose(D0[:, 0], d, rtol=1e-14)
    np.testing.assert_allclose(W0[:, 0], np.maximum(0, P @ d / (d @ d)), rtol=1e-13)


def test_cluster_init_feeds_nmf():
    # a nonnegative start: D0 >= 0, W0 >= 0, and HALS from it decreases the objective
    rng = np.random.default_rng(8)
    Dt = rng.uniform(size=(20, 3))
    Wt = rng.uniform(size=(200, 3)) ** 3
    P = Wt @ Dt.T
    D0, W0 = oracle.cluster_init(P, 3, S=100, iters=10, seed=2)
    assert np.all(D0 >= 0) and np.all(W0 >= 0)
    f0 = oracle.objective(P, D0, W0)
    _, _, obj = oracle.nmf(P, D0, W0, 20)
    assert obj[-1] < f0 and np.all(np.diff(obj) <= 1e-12 * f0)


def test_kmeanspp_pick_takes_the_first_sample_exceeding_the_target(orc):
    # running sums 1, 2, 4 against u * total: a sum equal to the target does not exceed it
    assert orc.kmpp_pick([1.0, 1.0, 2.0], 0.25) == 1          # target 1: 1 is not > 1, 2 is
    assert orc.kmpp_pick([1.0, 1.0, 2.0], 0.25 - 2.0 ** -54) == 0
    assert orc.kmpp_pick([0.0, 0.0, 3.0, 0.0], 0.0) == 2       # zero-distance samples are never picked
    assert orc.kmpp_pick([1.0, 2.0, 0.0, 0.0], 1.0 - 2.0 ** -53) == 1
    assert orc.kmpp_pick([0.0, 0.0], 0.5) == -1                # every sample on a chosen centre
