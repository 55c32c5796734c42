"""Host-side logic on the CPU: the learned start's canonical ordering, the seeded
input generators, the workload shapes of the measured forms, and the bench's
algorithmic-bytes formula."""
import math

import numpy as np
import pytest


def test_match_order_recovers_a_permutation():
    from paper_2410_22500_gb300 import learned, synth

    lib = synth.spectra_library(96, 5, seed=3)
    rng = np.random.default_rng(4)
    perm = rng.permutation(5)
    D = lib[:, perm] * rng.uniform(0.5, 2.0, size=5) + 1e-3 * rng.normal(size=(96, 5))
    r = learned.match_order(D, lib)
    for k in range(5):
        assert r[perm[k]] == k       # library column perm[k] is matched to D's column k


def test_init_params_layout(orc):
    from paper_2410_22500_gb300 import learned

    Nk, H1, H2, K = 40, 16, 8, 3
    p = learned.init_params(np.random.default_rng(0), Nk, H1, H2, K)
    assert p.dtype == np.float32 and p.size == orc.mlp_nparams(Nk, H1, H2, K)
    b3 = p[-K:].astype(np.float64)
    np.testing.assert_allclose(np.log1p(np.exp(b3)), 0.5, rtol=1e-6)   # softplus of the output bias


def test_problem_generation_is_seeded():
    from paper_2410_22500_gb300 import synth

    a = synth.make_problem(N=16, Nr=2, Nc=24, Nv=12, Nk=32, Nm=3, I0=300, seed=11, dead_frac=0.1)
    b = synth.make_problem(N=16, Nr=2, Nc=24, Nv=12, Nk=32, Nm=3, I0=300, seed=11, dead_frac=0.1)
    c = synth.make_problem(N=16, Nr=2, Nc=24, Nv=12, Nk=32, Nm=3, I0=300, seed=12, dead_frac=0.1)
    np.testing.assert_array_equal(a.spectra, b.spectra)
    np.testing.assert_array_equal(a.dead_bins, b.dead_bins)
    ya, y0a = synth.counts_numpy(a)
    yb, y0b = synth.counts_numpy(b)
    np.testing.assert_array_equal(ya, yb)
    np.testing.assert_array_equal(y0a, y0b)
    assert ya.shape == (12, 2, 24, 32) and y0a.shape == (2, 24, 32) and ya.dtype == np.uint16
    assert int(a.dead_bins.sum()) == round(0.1 * 32)
    assert np.all(ya[..., a.dead_bins.astype(bool)] == 0)
    assert not np.array_equal(a.spectra, c.spectra)


def test_batched_form_shapes_are_in_range():
    from paper_2410_22500_gb300 import forms

    shapes = forms._batch_shapes(40)
    assert shapes == forms._batch_shapes(40)
    for N, Nv, K in shapes:
        assert 64 <= N <= 512 and N % 16 == 0
        assert 45 <= Nv <= 180
        assert 3 <= K <= 8


def test_first_within():
    from paper_2410_22500_gb300 import forms

    obj = np.array([5.0, 3.0, 2.0, 1.5, 1.4])
    assert forms._first_within(obj, 2.0) == 3       # 1-based iteration count
    assert forms._first_within(obj, 1.0) is None


def test_bench_algorithmic_pass_bytes():
    import bench

    # the 3-D workload: P (737,280 x 1200 f32) once, W (737,280 x 5 f32) read and written
    assert bench.algorithmic_pass_bytes(737280, 1200, 4, 5) == 737280 * 1200 * 4 + 2 * 737280 * 5 * 4 == 3568435200
    # the 256^3 precision form: the 1500 live bins of P (7,864,320 rows, bf16) once, W (K = 6,
    # f32) read and written; the row padding P is stored with is not counted
    assert bench.algorithmic_pass_bytes(7864320, 1500, 2, 6) == 7864320 * 1500 * 2 + 2 * 7864320 * 6 * 4
    assert bench.whole_job_value(4, 10.0, 1000.0) == pytest.approx(40.0)


def test_preferred_row_stride():
    # host-only entry point: the stride whose 8-row tiles are one contiguous copy when it
    # pads a row by at most 5 %, else Nk rounded up to 8 (bf16) / 4 (f32) values
    from paper_2410_22500_gb300 import build, fhr

    build.build()
    assert fhr.nmf_row_stride(1500, fhr.BF16) == 1544    # 12 x 128 bins staged, 3088-byte rows
    assert fhr.nmf_row_stride(1200, fhr.F32) == 1252     # 13 x 96 bins staged, 5008-byte rows
    assert fhr.nmf_row_stride(96, fhr.BF16) == 96        # the staged row would double it
    assert fhr.nmf_row_stride(37, fhr.F32) == 40
    assert fhr.nmf_row_stride(2000, fhr.BF16) == 2000    # 2120 would pad by 6 %
    L = fhr.load()
    import ctypes
    out = ctypes.c_int()
    assert L.fhr_nmf_row_stride(0, fhr.BF16, ctypes.byref(out)) == fhr.ERR_ARG
    assert L.fhr_nmf_row_stride(100, 7, ctypes.byref(out)) == fhr.ERR_ARG


def test_bench_cpu_info():
    # the CPU baseline reports the cores it may use and the CPU model
    import os

    import bench

    cores, model = bench.cpu_info()
    assert cores == len(os.sched_getaffinity(0)) and model


def test_chords_torch_matches_numpy():
    # the torch evaluation of the analytic chords (used to draw many phantoms) is the numpy one
    from paper_2410_22500_gb300 import synth

    pb = synth.make_problem(N=48, Nr=5, Nc=40, Nv=17, Nk=12, Nm=3, I0=50, seed=11, three_d=True)
    a = synth.chords(pb.phantom, pb.geom)
    b = synth.chords_torch(pb.phantom, pb.geom, "cpu").numpy()
    np.testing.assert_allclose(b, a, rtol=0, atol=1e-12 * np.abs(a).max())
    pb2 = synth.make_problem(N=48, Nr=5, Nc=40, Nv=17, Nk=12, Nm=3, I0=50, seed=11, three_d=True, device="cpu")
    np.testing.assert_allclose(pb2.spectra, pb.spectra, rtol=1e-12)
