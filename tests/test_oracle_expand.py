"""Pins of the oracle's subspace expansion (Eq. sub_expansion) and of Algorithm 1 end to end."""
import math

import numpy as np


def test_identity_dictionary_is_layout_permutation(orc):
    # D = I (Nk = K): x^h is x^s itself, moved from [iy][ix][r*K+j] to [r][iy][ix][j]
    rng = np.random.default_rng(50)
    N, Nr, K = 5, 3, 4
    xs = rng.normal(size=(N, N, Nr * K))
    xh = orc.expand(xs, np.eye(K), N, Nr)
    np.testing.assert_array_equal(xh, xs.reshape(N, N, Nr, K).transpose(2, 0, 1, 3))


def test_expansion_commutes_with_projection(orc):
    # A (x^s D^T) = (A x^s) D^T  (linearity; App. B uses the same step)
    rng = np.random.default_rng(51)
    N, Nc, Nv, K, Nk = 9, 14, 7, 3, 11
    th = np.arange(Nv) * math.pi / Nv
    xs = rng.uniform(size=(N, N, K))
    D = rng.uniform(size=(Nk, K))
    xh = orc.expand(xs, D, N, 1)[0]                 # [N][N][Nk]
    lhs = orc.project(xh, Nc, th)                   # [Nv][Nc][Nk]
    rhs = orc.project(xs, Nc, th) @ D.T
    np.testing.assert_allclose(lhs, rhs, atol=1e-12)


def test_pipeline_noise_free_reproduces_hyperspectral_volume(orc):
    # Algorithm 1 on noise-free counts (high dose) with K = Nm: the expanded volume is
    # close to x^m (D^m)^T, the hyperspectral ground truth of Eq. (porj_matd_rel).  The
    # data come from analytic line integrals, not from the strip model, so the residual
    # is discretisation and prior smoothing at the material edges (~15% here).
    from paper_2410_22500_gb300 import synth

    pb = synth.make_problem(N=32, Nr=1, Nc=48, Nv=60, Nk=24, Nm=2, I0=60000, seed=52)
    y, y0 = synth.counts_numpy(pb, noise=False)
    g = pb.geom
    out = orc.fhr_pipeline(y, y0, 2, g.N, g.angles(), nmf_iters=300, mbir_iters=300, snr_db=50.0,
                           momentum=True)
    xm = synth.volume_fractions(pb.phantom, g.N, 1, sub=4)        # [1][N][N][Nm]
    truth = xm @ pb.spectra.T                                      # [1][N][N][Nk]
    err = np.linalg.norm(out["xh"] - truth) / np.linalg.norm(truth)
    assert err < 0.2
    assert out["obj"][-1] <= out["obj"][0]
    assert out["obj"][-1] < 1e-8 * np.sum(out["P"] ** 2)      # noise-free P is rank Nm


def test_subspace_reduces_noise_vs_per_bin_reconstruction(orc):
    # the paper's qualitative claim (Sec. V-B): reconstructing through the K-dim subspace
    # is much less noisy than reconstructing every wavelength bin separately
    from paper_2410_22500_gb300 import synth

    pb = synth.make_problem(N=16, Nr=1, Nc=24, Nv=30, Nk=40, Nm=2, I0=200, seed=53)
    y, y0 = synth.counts_numpy(pb, noise=True)
    g = pb.geom
    th = g.angles()
    out = orc.fhr_pipeline(y, y0, 2, g.N, th, nmf_iters=200, mbir_iters=150, momentum=True)
    xm = synth.volume_fractions(pb.phantom, g.N, 1, sub=4)
    truth = (xm @ pb.spectra.T)[0]
    # direct per-bin reconstruction (same solver, every bin its own channel)
    P = out["P"]                                                   # (v, c, r=0) rows
    Vb = P.reshape(g.Nv, g.Nc, pb.Nk)
    sv, sx = orc.mbir_sigmas(P, pb.Nk, g.Nc)
    xd = orc.mbir(Vb, g.N, 1, pb.Nk, th, sv, sx, iters=150, momentum=True)
    e_fhr = np.linalg.norm(out["xh"][0] - truth)
    e_dhr = np.linalg.norm(xd - truth)
    assert e_fhr < 0.8 * e_dhr
