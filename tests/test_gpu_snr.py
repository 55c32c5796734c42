"""GPU parity of the signal-to-noise ratios of Sec. V-B, Eq. (snr_fmd) and Eq. (snr_fhr),
against the FP64 oracle on the same inputs."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _rois(rng, Nx, Nm, per=400, bg=400):
    roi = np.zeros(Nx, np.uint8)
    idx = rng.permutation(Nx)
    for m in range(Nm):
        roi[idx[m * per:(m + 1) * per]] = m + 1
    roi[idx[Nm * per:Nm * per + bg]] = 255
    return roi


@pytest.mark.parametrize("Nx,C,Nm", [(5000, 3, 3), (40000, 137, 4), (70001, 1500, 6), (20000, 9, 16)])
def test_snr_matches_oracle(fx, orc, Nx, C, Nm):
    from paper_2410_22500_gb300 import fhr

    rng = np.random.default_rng(Nx + C)
    x = (rng.normal(0, 0.1, size=(Nx, C)) + rng.uniform(0.2, 1.0, size=(1, C))).astype(np.float32)
    roi = _rois(rng, Nx, Nm)
    for mode in (fhr.SNR_FHR, fhr.SNR_FMD):
        if mode == fhr.SNR_FMD and C < Nm:
            continue
        got = float(fx.snr(_dev(x), _dev(roi), Nm, mode).item())
        want = orc.snr(x.astype(np.float64), roi, Nm, mode)
        assert abs(got - want) <= 1e-9 * max(1.0, abs(want)), (mode, got, want)


def test_snr_hand_case_and_empty_region(fx, orc):
    from paper_2410_22500_gb300 import fhr

    x = np.array([[2.0, 0.5], [4.0, 0.5], [0.1, 3.0], [0.1, 5.0], [1.0, -2.0], [-1.0, 2.0], [100.0, 100.0]],
                 np.float32)
    roi = np.array([1, 1, 2, 2, 255, 255, 0], np.uint8)
    got = float(fx.snr(_dev(x), _dev(roi), 2, fhr.SNR_FMD).item())
    assert got == pytest.approx(10 * np.log10(6.5), abs=1e-6)
    with pytest.raises(fhr.FhrError):
        fx.snr(_dev(x), _dev(np.where(roi == 2, 0, roi).astype(np.uint8)), 2, fhr.SNR_FMD)


def test_snr_of_fhr_over_the_volume_is_deterministic(fx):
    # the 3-D layout at size (1,048,576 voxels x 1200 bins would be 5 GB; 262,144 x 600 here):
    # two calls give the same bits
    import torch

    from paper_2410_22500_gb300 import fhr

    g = torch.Generator(device="cuda")
    g.manual_seed(5)
    x = torch.rand((262144, 600), device="cuda", generator=g)
    rng = np.random.default_rng(6)
    roi = _dev(_rois(rng, 262144, 5, per=6400, bg=6400))
    a = fx.snr(x, roi, 5, fhr.SNR_FHR).item()
    b = fx.snr(x, roi, 5, fhr.SNR_FHR).item()
    assert a == b and np.isfinite(a)
