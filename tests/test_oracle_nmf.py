"""Pins of the oracle's subspace extraction: fast-HALS NMF and NNDSVD (Sec. III, Eq. sub_extract_solve)."""
import itertools
import os

import numpy as np
import pytest
from scipy.optimize import nnls

HERE = os.path.dirname(os.path.abspath(__file__))


def _rand_problem(seed, Np=40, Nk=30, K=3):
    rng = np.random.default_rng(seed)
    P = rng.uniform(0, 1, size=(Np, Nk))
    D = rng.uniform(0.1, 1, size=(Nk, K))
    W = rng.uniform(0.1, 1, size=(Np, K))
    return P, D, W


def test_w_step_single_coordinate_is_1d_minimiser(orc):
    # K = 1: one HALS step is the exact minimiser of the 1-D nonnegative quadratic
    # ||p_j - w d||^2 over w >= 0; compare with a brute-force scan + refinement.
    rng = np.random.default_rng(10)
    Nk = 17
    d = rng.uniform(0, 1, size=(Nk, 1))
    for trial in range(6):
        p = rng.normal(0.2 if trial % 2 else -0.3, 1.0, size=(1, Nk))
        W = np.array([[rng.uniform(0, 3)]])
        orc.hals_update_W(p, d, W)
        f = lambda w: np.sum((p[0] - w * d[:, 0]) ** 2)
        grid = np.linspace(0, 5, 50001)
        vals = np.array([f(g) for g in grid])
        w0 = grid[np.argmin(vals)]
        lo, hi = max(0.0, w0 - 1e-4), w0 + 1e-4
        for _ in range(200):   # ternary search on the bracket (convex)
            m1, m2 = lo + (hi - lo) / 3, hi - (hi - lo) / 3
            if f(m1) <= f(m2):
                hi = m2
            else:
                lo = m1
        # a scan resolves the minimiser only to ~sqrt(eps * f / d^T d), about 1e-7 here
        assert abs(W[0, 0] - 0.5 * (lo + hi)) < 1e-6


def test_w_steps_converge_to_nnls(orc):
    # repeated V half-steps with D fixed are coordinate descent on a strictly convex
    # NNLS problem per pixel: the limit is scipy's NNLS solution
    P, D, W = _rand_problem(11, Np=12, Nk=25, K=4)
    P[:, :5] *= -1   # make some constraints active
    for _ in range(3000):
        orc.hals_update_W(P, D, W)
    for j in range(P.shape[0]):
        x, _ = nnls(D, P[j])
        np.testing.assert_allclose(W[j], x, atol=1e-9)


def test_d_steps_converge_to_nnls(orc):
    P, D, W = _rand_problem(12, Np=25, Nk=10, K=4)
    P[:5] *= -1
    for _ in range(3000):
        orc.hals_update_D(P, W, D)
    for k in range(P.shape[1]):
        x, _ = nnls(W, P[:, k])
        np.testing.assert_allclose(D[k], x, atol=1e-9)


def test_objective_nonincreasing_every_half_step(orc):
    P, D, W = _rand_problem(13, Np=60, Nk=35, K=5)
    f = orc.objective(P, D, W)
    for _ in range(40):
        orc.hals_update_W(P, D, W)
        f1 = orc.objective(P, D, W)
        assert f1 <= f * (1 + 1e-13)
        orc.hals_update_D(P, W, D)
        f2 = orc.objective(P, D, W)
        assert f2 <= f1 * (1 + 1e-13)
        n = orc.normalise_columns(D, W)
        f3 = orc.objective(P, D, W)
        assert abs(f3 - f2) <= 1e-12 * f2   # scaling leaves W D^T unchanged
        assert np.all(n >= 0)
        f = f3
    assert np.all(W >= 0) and np.all(D >= 0)
    np.testing.assert_allclose(np.linalg.norm(D, axis=0), 1.0, rtol=1e-14)


def test_nmf_history_matches_half_steps(orc):
    P, D0, W0 = _rand_problem(14)
    D, W, obj = orc.nmf(P, D0, W0, 5)
    D1, W1 = D0.copy(), W0.copy()
    for t in range(5):
        orc.hals_update_W(P, D1, W1)
        orc.hals_update_D(P, W1, D1)
        orc.normalise_columns(D1, W1)
        assert abs(obj[t] - orc.objective(P, D1, W1)) <= 1e-12 * obj[t]
    np.testing.assert_array_equal(D, D1)
    np.testing.assert_array_equal(W, W1)


def test_zero_gram_diagonal_leaves_coordinate(orc):
    # a zero column of D gives (D^T D)_ss = 0: that coordinate of V is not touched
    P, D, W = _rand_problem(15, K=3)
    D[:, 1] = 0
    W_before = W.copy()
    orc.hals_update_W(P, D, W)
    np.testing.assert_array_equal(W[:, 1], W_before[:, 1])


def _match(A, B):
    """Best column permutation of B onto A by cosine similarity (K small)."""
    K = A.shape[1]
    An = A / np.linalg.norm(A, axis=0)
    Bn = B / np.linalg.norm(B, axis=0)
    best = max(itertools.permutations(range(K)), key=lambda p: sum(An[:, i] @ Bn[:, p[i]] for i in range(K)))
    return np.array(best)


def test_exact_recovery_rank_k_with_pure_pixels(orc):
    # P = W* D*^T exactly rank K, with one pure pixel per material and one bin per
    # material where only it attenuates (both factors contain a scaled identity, so the
    # factorisation is unique up to scale and order): the objective goes to ~0 and the
    # factors are recovered
    rng = np.random.default_rng(16)
    Np, Nk, K = 80, 40, 3
    Dt = rng.uniform(0, 1, size=(Nk, K))
    Dt[:K] = np.eye(K)
    Wt = rng.uniform(0, 1, size=(Np, K))
    Wt[:K] = np.eye(K)
    P = Wt @ Dt.T
    D0, W0 = orc.nndsvd(P, K)
    D, W, obj = orc.nmf(P, D0, W0, 12000)
    assert obj[-1] / np.sum(P * P) < 1e-20
    perm = _match(Dt, D)
    cos = [Dt[:, i] @ D[:, perm[i]] / np.linalg.norm(Dt[:, i]) / np.linalg.norm(D[:, perm[i]]) for i in range(K)]
    assert min(cos) > 1 - 1e-7


def test_kkt_at_convergence(orc):
    P, D0, W0 = _rand_problem(17, Np=30, Nk=20, K=2)
    D, W, obj = orc.nmf(P, D0, W0, 5000)
    R = W @ D.T - P
    gW = R @ D      # half gradient w.r.t. W
    gD = R.T @ W
    assert np.max(np.abs(np.minimum(W, gW))) < 1e-7 * np.abs(P).max()
    assert np.max(np.abs(np.minimum(D, gD))) < 1e-7 * np.abs(P).max() * np.abs(W).max()


# ------------------------------------------------------------------ NNDSVD
def test_nndsvd_rank_one_exact(orc):
    rng = np.random.default_rng(20)
    w = rng.uniform(0, 1, 30)
    d = rng.uniform(0, 1, 12)
    P = np.outer(w, d)
    D0, W0 = orc.nndsvd(P, 1)
    np.testing.assert_allclose(W0 @ D0.T, P, atol=1e-13)


def test_nndsvd_hand_example(orc):
    W_ref, D_ref = [], []
    with open(os.path.join(HERE, "golden", "nndsvd_2x2.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            tag, *vals = line.split()
            (W_ref if tag == "W" else D_ref).append([float(v) for v in vals])
    s2 = np.sqrt(2.0)
    U = np.array([[1, 1], [1, -1]]) / s2
    P = U @ np.diag([4.0, 1.0])
    D0, W0 = orc.nndsvd(P, 2)
    np.testing.assert_allclose(W0, W_ref, atol=1e-14)
    np.testing.assert_allclose(D0, D_ref, atol=1e-14)


def test_nndsvd_sign_invariant_and_nonnegative(orc):
    rng = np.random.default_rng(21)
    P = rng.uniform(0, 1, size=(50, 20))
    U, S, Vt = np.linalg.svd(P, full_matrices=False)
    K = 5
    D1, W1 = orc.nndsvd_split(U[:, :K], S[:K], Vt[:K], K)
    flip = np.array([1, -1, -1, 1, -1])
    D2, W2 = orc.nndsvd_split(U[:, :K] * flip, S[:K], (Vt[:K].T * flip).T, K)
    np.testing.assert_allclose(D1, D2, atol=1e-14)
    np.testing.assert_allclose(W1, W2, atol=1e-14)
    assert np.all(D1 >= 0) and np.all(W1 >= 0)
    # the first component carries the dominant rank-1 term exactly
    np.testing.assert_allclose(np.outer(W1[:, 0], D1[:, 0]), S[0] * np.outer(np.abs(U[:, 0]), np.abs(Vt[0])), atol=1e-12)


def test_nndsvd_tie_goes_to_the_positive_pair(orc):
    # column 1 has equal positive and negative products (|u+||v+| = |u-||v-|): the reading
    # takes the positive pair, unit-normalised and scaled by sqrt(S_1 * product)
    a, b = 0.6, 0.8
    U = np.array([[1.0, a], [0.0, -a]])
    Vt = np.array([[1.0, 0.0, 0.0], [b, -b, 0.0]])
    S = np.array([4.0, 2.0])
    D, W = orc.nndsvd_split(U, S, Vt, 2)
    lam = np.sqrt(2.0 * a * b)
    np.testing.assert_allclose(W[:, 1], [lam, 0.0], rtol=1e-15)
    np.testing.assert_allclose(D[:, 1], [lam, 0.0, 0.0], rtol=1e-15)


def test_v_half_step_is_gauss_seidel_in_natural_order(orc):
    # one pixel p = (1, 1), D = [[1, 0.5], [0.5, 1]], W = 0: r = D^T p = (1.5, 1.5),
    # G = D^T D = [[1.25, 1], [1, 1.25]]; coordinate 0 first: w0 = 1.5 / 1.25 = 1.2,
    # then w1 = (1.5 - 1 * 1.2) / 1.25 = 0.24 (the reverse order would give (0.24, 1.2))
    P = np.array([[1.0, 1.0]])
    D = np.array([[1.0, 0.5], [0.5, 1.0]])
    W = np.zeros((1, 2))
    orc.hals_update_W(P, D, W)
    np.testing.assert_allclose(W[0], [1.2, 0.24], rtol=1e-15)
