"""Pins of the oracle's semi-supervised material decomposition (Algorithm 2 after
the reconstruction: Eq. trans_mat, Eq. mat_recon_nmf, Eq. sub_mat_rel_basis)."""
import numpy as np

import oracle


def test_region_means_by_hand():
    # 4 voxels, 2 subspace channels, regions {0, 2} -> material 1, {3} -> material 2
    xs = np.array([[1.0, 2.0], [5.0, 5.0], [3.0, 4.0], [7.0, 0.5]])
    labels = np.array([1, 0, 1, 2])
    T = oracle.fmd_transform(xs, labels, 2)
    np.testing.assert_array_equal(T, [[2.0, 3.0], [7.0, 0.5]])


def test_exact_recovery_of_a_nonnegative_mix():
    rng = np.random.default_rng(1)
    Nm, Ns, Nx = 3, 5, 200
    T = rng.uniform(0.1, 1.0, size=(Nm, Ns))
    xm = rng.uniform(size=(Nx, Nm)) * (rng.uniform(size=(Nx, Nm)) > 0.3)
    xs = xm @ T
    np.testing.assert_allclose(oracle.fmd_materials(xs, T), xm, atol=1e-12)


def test_nnls_kkt_on_noisy_data():
    rng = np.random.default_rng(2)
    Nm, Ns, Nx = 4, 6, 300
    T = rng.normal(size=(Nm, Ns))
    xs = rng.normal(size=(Nx, Ns))
    xm = oracle.fmd_materials(xs, T)
    grad = (xm @ T - xs) @ T.T          # gradient of 1/2 ||xs - x T||^2
    assert np.all(xm >= 0)
    assert np.all(grad[xm == 0] >= -1e-10)
    np.testing.assert_allclose(grad[xm > 0], 0.0, atol=1e-10)


def test_appendix_b_identity_recovers_material_spectra():
    # p = x^m D^m^T with pure unit regions; any invertible subspace mixing B gives
    # V^s = x^m B, D^s = D^m B^-T, and FMD maps (x^s, D^s) back to (x^m, D^m)
    rng = np.random.default_rng(3)
    Nm, Nk, Nx = 3, 40, 90
    Dm = rng.uniform(size=(Nk, Nm))
    xm = rng.uniform(size=(Nx, Nm))
    labels = np.zeros(Nx, dtype=np.int32)
    for i in range(Nm):                  # 10 pure voxels of material i at unit concentration
        xm[10 * i:10 * i + 10] = 0.0
        xm[10 * i:10 * i + 10, i] = 1.0
        labels[10 * i:10 * i + 10] = i + 1
    B = rng.normal(size=(Nm, Nm)) + 3 * np.eye(Nm)
    xs = xm @ B
    Ds = Dm @ np.linalg.inv(B).T
    T, xm_est, Dm_est = oracle.fmd(xs, Ds, labels, Nm)
    np.testing.assert_allclose(T, B, atol=1e-12)
    np.testing.assert_allclose(Dm_est, Dm, atol=1e-12)
    np.testing.assert_allclose(xm_est, xm, atol=1e-10)
