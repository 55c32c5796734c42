"""Pins of the oracle's signal-to-noise ratios, Eq. (snr_fmd) and Eq. (snr_fhr) (Sec. V-B)."""
import math

import numpy as np
import pytest


def _case():
    # 7 voxels, 2 materials, 2 channels; voxel 6 is in no region (its huge value must not count)
    x = np.array([[2.0, 0.5], [4.0, 0.5],      # region of material 0: means (3, 0.5)
                  [0.1, 3.0], [0.1, 5.0],      # region of material 1: means (0.1, 4)
                  [1.0, -2.0], [-1.0, 2.0],    # background: means (0, 0), std (1, 2)
                  [100.0, 100.0]])
    roi = np.array([1, 1, 2, 2, 255, 255, 0], np.uint8)
    return x, roi


def test_snr_fmd_by_hand(orc):
    # Eq. (snr_fmd): channel m over region m: (3/1)^2 = 9, (4/2)^2 = 4 -> 10 log10(6.5)
    x, roi = _case()
    assert orc.snr(x, roi, 2, orc.SNR_FMD) == pytest.approx(10 * math.log10(6.5), abs=1e-12)


def test_snr_fhr_by_hand(orc):
    # Eq. (snr_fhr): every (material, bin): 9, (0.5/2)^2, (0.1/1)^2, (4/2)^2 -> mean 3.268125
    x, roi = _case()
    assert orc.snr(x, roi, 2, orc.SNR_FHR) == pytest.approx(10 * math.log10(13.0725 / 4), abs=1e-12)


def test_snr_scale_invariant_and_known_noise(orc):
    # scaling the image leaves both ratios unchanged; a unit signal over background noise of
    # standard deviation s gives 10 log10(1 / s^2) (population deviation of the drawn noise)
    rng = np.random.default_rng(3)
    n = 4000
    noise = rng.normal(0, 0.25, size=(n, 1))
    x = np.concatenate([np.ones((50, 1)), noise])
    roi = np.concatenate([np.ones(50, np.uint8), np.full(n, 255, np.uint8)])
    s = float(np.std(noise))
    assert orc.snr(x, roi, 1, orc.SNR_FMD) == pytest.approx(-20 * math.log10(s), abs=1e-9)
    assert orc.snr(7.5 * x, roi, 1, orc.SNR_FHR) == pytest.approx(orc.snr(x, roi, 1, orc.SNR_FHR), abs=1e-9)


def test_snr_rejects_empty_regions(orc):
    x, roi = _case()
    with pytest.raises(ValueError):
        orc.snr(x, np.where(roi == 2, 0, roi).astype(np.uint8), 2, orc.SNR_FMD)
    with pytest.raises(ValueError):
        orc.snr(x, np.where(roi == 255, 0, roi).astype(np.uint8), 2, orc.SNR_FHR)
