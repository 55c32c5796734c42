"""GPU parity of the semi-supervised material decomposition (Algorithm 2 after the
reconstruction: Eq. trans_mat, Eq. mat_recon_nmf, Eq. sub_mat_rel_basis)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _case(seed, Nx, Ns, Nm, Nk, noise=0.05, unlabeled=0.5):
    """Voxels mixing Nm materials (some zero) in an Ns-channel subspace, plus noise;
    a fraction of voxels carries the label of their dominant material."""
    rng = np.random.default_rng(seed)
    B = rng.normal(size=(Nm, Ns)) + np.eye(Nm, Ns) * 3.0
    xm = rng.uniform(size=(Nx, Nm)) * (rng.uniform(size=(Nx, Nm)) > 0.4)
    xs = (xm @ B + noise * rng.normal(size=(Nx, Ns))).astype(np.float32)
    labels = (np.argmax(xm, axis=1) + 1).astype(np.uint8)
    labels[rng.uniform(size=Nx) < unlabeled] = 0
    for i in range(Nm):                  # every region holds at least one voxel
        labels[i] = i + 1
    D = rng.uniform(-1, 1, size=(Nk, Ns)).astype(np.float32)
    return xs, labels, D


def _check(fx, orc, xs, labels, D, Nm, sample=None):
    T, xm, Dm = fx.fmd(_dev(xs), _dev(labels), _dev(D), Nm)
    T, xm, Dm = T.cpu().numpy(), xm.cpu().numpy(), Dm.cpu().numpy()
    T_ref = orc.fmd_transform(xs.astype(np.float64), labels, Nm)
    np.testing.assert_allclose(T, T_ref, rtol=1e-6, atol=1e-7 * np.abs(T_ref).max())
    Dm_ref = orc.fmd_spectra(D.astype(np.float64), T_ref)
    np.testing.assert_allclose(Dm, Dm_ref, rtol=1e-5, atol=1e-6 * np.abs(Dm_ref).max())
    idx = np.arange(xs.shape[0]) if sample is None else sample
    xm_ref = orc.fmd_materials(xs[idx].astype(np.float64), T_ref)
    scale = np.abs(xs).max() / np.linalg.norm(T_ref, 2) + 1e-30
    np.testing.assert_allclose(xm[idx], xm_ref, rtol=0, atol=2e-5 * scale)
    assert (xm >= 0).all()
    return T, xm, Dm


@pytest.mark.parametrize("Nx,Ns,Nm,Nk", [(1000, 5, 3, 300), (4099, 8, 8, 1200), (777, 4, 1, 17), (2053, 6, 6, 64),
                                         (1, 3, 2, 1), (3001, 9, 3, 1500), (1500, 16, 8, 50)])
def test_fmd_matches_oracle(fx, orc, Nx, Ns, Nm, Nk):
    xs, labels, D = _case(900 + Nx, max(Nx, Nm), Ns, Nm, Nk)
    _check(fx, orc, xs, labels, D, Nm)


def test_fmd_appendix_b_recovers_material_spectra(fx):
    # pure unit regions mixed by an invertible B: FMD maps (x^s, D^s) back to (x^m, D^m)
    rng = np.random.default_rng(31)
    Nm, Nk, Nx = 4, 200, 4000
    Dm = rng.uniform(size=(Nk, Nm))
    xm = rng.uniform(size=(Nx, Nm))
    labels = np.zeros(Nx, dtype=np.uint8)
    for i in range(Nm):
        xm[100 * i:100 * i + 100] = 0.0
        xm[100 * i:100 * i + 100, i] = 1.0
        labels[100 * i:100 * i + 100] = i + 1
    B = rng.normal(size=(Nm, Nm)) + 3 * np.eye(Nm)
    xs = (xm @ B).astype(np.float32)
    Ds = (Dm @ np.linalg.inv(B).T).astype(np.float32)
    _, xm_g, Dm_g = fx.fmd(_dev(xs), _dev(labels), _dev(Ds), Nm)
    np.testing.assert_allclose(Dm_g.cpu().numpy(), Dm, atol=2e-5)
    np.testing.assert_allclose(xm_g.cpu().numpy(), xm, atol=2e-5)


def test_fmd_on_the_volume_layout(fx, orc):
    # the 128x128x64 / K=5 reconstruction's [N][N][Nr*K] layout, viewed as [Nr*N*N][K] voxels;
    # T and D^m in full, x^m on a seeded sample of voxels
    N, Nr, K, Nm, Nk = 128, 64, 5, 3, 1200
    xs, labels, D = _case(77, N * N * Nr, K, Nm, Nk, unlabeled=0.9)
    xs3 = xs.reshape(N, N, Nr * K)
    T, xm, _ = fx.fmd(_dev(xs3), _dev(labels), _dev(D), Nm)
    assert xm.shape == (N * N * Nr, Nm)
    sample = np.random.default_rng(5).choice(N * N * Nr, 3000, replace=False)
    sample[:2] = [0, N * N * Nr - 1]
    _check(fx, orc, xs, labels, D, Nm, sample=sample)


def test_fmd_is_deterministic(fx):
    xs, labels, D = _case(8, 50000, 6, 4, 100)
    a = [t.cpu().numpy() for t in fx.fmd(_dev(xs), _dev(labels), _dev(D), 4)]
    b = [t.cpu().numpy() for t in fx.fmd(_dev(xs), _dev(labels), _dev(D), 4)]
    for u, v in zip(a, b):
        np.testing.assert_array_equal(u, v)


def test_fmd_empty_region_reports_and_matches_oracle(fx, orc):
    from paper_2410_22500_gb300 import fhr

    xs, labels, D = _case(12, 600, 5, 3, 40)
    labels[labels == 2] = 0                 # region 2 is empty
    with pytest.raises(fhr.FhrError):
        fx.fmd(_dev(xs), _dev(labels), _dev(D), 3)
    T, xm, _ = fx.fmd(_dev(xs), _dev(labels), _dev(D), 3, check_status=False)
    T_ref = orc.fmd_transform(xs.astype(np.float64), labels, 3)
    np.testing.assert_allclose(T.cpu().numpy(), T_ref, rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(xm.cpu().numpy(), orc.fmd_materials(xs.astype(np.float64), T_ref), atol=1e-4)


def test_fmd_rejects_bad_sizes(fx):
    from paper_2410_22500_gb300 import fhr

    xs, labels, D = _case(3, 100, 3, 3, 10)
    with pytest.raises(fhr.FhrError):
        fx.fmd(_dev(np.zeros((100, 17), np.float32)), _dev(labels), _dev(np.zeros((10, 17), np.float32)), 3)
    with pytest.raises(fhr.FhrError):
        fx.fmd(_dev(xs), _dev(labels), _dev(D), 4)   # Nm > Ns
