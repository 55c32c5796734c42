"""Algorithm 1 end to end on the GPU against the FP64 oracle."""
import numpy as np
import pytest
from _parity import assert_close, rel_l2 as _rel

pytestmark = pytest.mark.gpu


def _run_gpu(fx, pb, K, nmf_iters, mbir_iters, host_io=False, **kw):
    import torch
    from paper_2410_22500_gb300 import synth

    g = pb.geom
    y, y0 = synth.counts_numpy(pb)
    prm = fx.pipeline_params(Nv=g.Nv, Nr=g.Nr, Nc=g.Nc, Nk=pb.Nk, N=g.N, K=K, nmf_iters=nmf_iters,
                             mbir_iters=mbir_iters, host_io=host_io, seed=3, **kw)
    D = torch.empty((pb.Nk, K), dtype=torch.float32, device="cuda")
    obj = torch.empty(nmf_iters, dtype=torch.float64, device="cuda")
    y16, y016 = torch.from_numpy(y.view(np.int16)), torch.from_numpy(y0.view(np.int16))
    if host_io:
        yt = y16.pin_memory()
        y0t = y016.pin_memory()
        xh = torch.empty((g.Nr, g.N, g.N, pb.Nk), dtype=torch.float32).pin_memory()
    else:
        yt, y0t = y16.cuda(), y016.cuda()
        xh = torch.empty((g.Nr, g.N, g.N, pb.Nk), dtype=torch.float32, device="cuda")
    ws = fx.pipeline(prm, yt, y0t, D, xh, obj=obj)
    assert fx.status(ws) == 0
    return y, y0, D.cpu().numpy(), xh.cpu().numpy(), obj.cpu().numpy()


def test_tiny_2d_end_to_end(fx, orc):
    # 32x32, K = 3, 60 views, Nk = 128: end-to-end relative error <= 1e-3 vs FP64
    from paper_2410_22500_gb300 import synth

    pb = synth.tiny_2d()
    g = pb.geom
    y, y0, D, xh, obj = _run_gpu(fx, pb, 3, 200, 30)
    ref = orc.fhr_pipeline(y, y0, 3, g.N, g.angles(), nmf_iters=200, mbir_iters=30)
    assert abs(obj[-1] - ref["obj"][-1]) <= 1e-3 * ref["obj"][-1]
    assert_close(xh, ref["xh"], 1e-3)


def test_host_io_equals_device_io(fx):
    from paper_2410_22500_gb300 import synth

    pb = synth.scaled(synth.tiny_2d, Nk=64, Nv=30)
    a = _run_gpu(fx, pb, 3, 20, 5, host_io=False)
    b = _run_gpu(fx, pb, 3, 20, 5, host_io=True)
    np.testing.assert_array_equal(a[3], b[3])
    np.testing.assert_array_equal(a[2], b[2])


def test_small_3d_end_to_end(fx, orc):
    # a reduced 3-D volume with dead bins: the slice-coupled prior and the (v, c, r) pixel order.
    # The NNDSVD starts (randomised subspace iteration here, exact SVD in the oracle) agree only
    # when the K-th singular gap is clear, so the case has K = Nm = 3 and a high dose
    # (sigma_3 / sigma_4 ~ 7).  At this dose the MBIR is sensitive to rounding: in the FP64
    # oracle alone a 1e-7 relative change of the sinogram moves x^s by 5e-4 (rel-L2) and 3e-3
    # (largest element) after 20 plain SQS iterations, 1e-6 and 7e-6 after 5, so the parity
    # checks run 5 MBIR iterations.
    from paper_2410_22500_gb300 import synth

    pb = synth.scaled(synth.volume_3d_f32, N=32, Nr=8, Nc=48, Nv=30, Nk=64, Nm=3, I0=20000, seed=77)
    g = pb.geom
    y, y0 = synth.counts_numpy(pb)
    import torch

    prm = fx.pipeline_params(Nv=g.Nv, Nr=g.Nr, Nc=g.Nc, Nk=pb.Nk, N=g.N, K=3, nmf_iters=100, mbir_iters=5, seed=3)
    D = torch.empty((pb.Nk, 3), dtype=torch.float32, device="cuda")
    xh = torch.empty((g.Nr, g.N, g.N, pb.Nk), dtype=torch.float32, device="cuda")
    dead = torch.from_numpy(pb.dead_bins).cuda()
    ws = fx.pipeline(prm, torch.from_numpy(y.view(np.int16)).cuda(), torch.from_numpy(y0.view(np.int16)).cuda(), D, xh,
                     dead=dead)
    assert fx.status(ws) == 0
    ref = orc.fhr_pipeline(y, y0, 3, g.N, g.angles(), nmf_iters=100, mbir_iters=5, dead=pb.dead_bins)
    # the two sides start from different NNDSVD factors (the GPU's randomised subspace
    # iteration against the exact SVD), which agree to about 1e-4; the per-element bound
    # carries that difference through 100 NMF and 20 MBIR iterations
    assert_close(xh.cpu().numpy(), ref["xh"], 1e-3, elem_tol=1e-2)
    assert np.all(D.cpu().numpy()[pb.dead_bins.astype(bool)] == 0)
    # the same stages from one shared start (the oracle's NNDSVD factors): arithmetic parity
    Pg = fx.normalise(torch.from_numpy(y.view(np.int16)).cuda(), torch.from_numpy(y0.view(np.int16)).cuda(), dead=dead)
    Dg, Wg, _ = fx.decompose(Pg, pb.Nk, 3, 100, D=torch.from_numpy(ref["D0"].astype(np.float32)).cuda(),
                             W=torch.from_numpy(ref["W0"].astype(np.float32)).cuda(), obj=False)
    xs = fx.reconstruct(Wg.view(g.Nv, g.Nc, g.Nr * 3), g.N, g.Nr, 3, 5)
    xh2 = fx.expand(xs, Dg, g.N, g.Nr).cpu().numpy()
    ref2 = orc.fhr_pipeline(y, y0, 3, g.N, g.angles(), nmf_iters=100, mbir_iters=5, dead=pb.dead_bins,
                            init=(ref["D0"].astype(np.float32).astype(np.float64),
                                  ref["W0"].astype(np.float32).astype(np.float64)))
    assert_close(xh2, ref2["xh"], 1e-3, what="shared start")


def test_host_io_back_to_back_calls(fx):
    # consecutive host-I/O calls on one workspace overlap their copies with each
    # other's compute; each output must still be its own input's result
    import torch

    from paper_2410_22500_gb300 import synth

    pa = synth.scaled(synth.tiny_2d, Nk=64, Nv=30)
    pb = synth.scaled(synth.tiny_2d, Nk=64, Nv=30, seed=1234)
    g = pa.geom
    K = 3
    prm = fx.pipeline_params(Nv=g.Nv, Nr=g.Nr, Nc=g.Nc, Nk=pa.Nk, N=g.N, K=K, nmf_iters=20, mbir_iters=5,
                             host_io=True, seed=3)
    ws, wsb = fx.pipeline_workspace(prm)
    outs, refs = [], []
    D = torch.empty((pa.Nk, K), dtype=torch.float32, device="cuda")
    for pb_ in (pa, pb, pa):
        y, y0 = synth.counts_numpy(pb_)
        yt = torch.from_numpy(y.view(np.int16)).pin_memory()
        y0t = torch.from_numpy(y0.view(np.int16)).pin_memory()
        xh = torch.empty((g.Nr, g.N, g.N, pa.Nk), dtype=torch.float32).pin_memory()
        fx.pipeline(prm, yt, y0t, D, xh, ws=ws, ws_bytes=wsb)
        outs.append((xh, yt, y0t))
    assert fx.status(ws) == 0
    for pb_, (xh, _, _) in zip((pa, pb, pa), outs):
        refs.append(_run_gpu(fx, pb_, K, 20, 5)[3])
        np.testing.assert_array_equal(xh.numpy(), refs[-1])
    assert not np.array_equal(refs[0], refs[1])


def test_learned_start_in_the_pipeline(fx):
    # Algorithm 1 from the learned start on BF16 P: the decomposition inside the pipeline
    # equals fhr_decompose from the same network on the same normalised P
    import ctypes

    import torch
    from paper_2410_22500_gb300 import fhr, learned, synth

    pb = synth.scaled(synth.tiny_2d, Nk=96, Nv=40)
    g = pb.geom
    K, iters = 3, 15
    ldb = (pb.Nk + 7) // 8 * 8
    dims = fx.mlp_dims(pb.Nk, 32, 16, K, ldx=ldb, x_bf16=True, weights_bf16=True)
    params = torch.from_numpy(learned.init_params(np.random.default_rng(4), pb.Nk, 32, 16, K)).cuda()
    y, y0 = synth.counts_numpy(pb)
    yt, y0t = torch.from_numpy(y.view(np.int16)).cuda(), torch.from_numpy(y0.view(np.int16)).cuda()
    prm = fx.pipeline_params(Nv=g.Nv, Nr=g.Nr, Nc=g.Nc, Nk=pb.Nk, N=g.N, K=K, nmf_iters=iters, mbir_iters=3,
                             p_dtype=fhr.BF16, init=fhr.INIT_LEARNED)
    prm.nmf.mlp = ctypes.addressof(dims)
    prm.nmf.mlp_params = params.data_ptr()
    D = torch.empty((pb.Nk, K), dtype=torch.float32, device="cuda")
    obj = torch.empty(iters, dtype=torch.float64, device="cuda")
    xh = torch.empty((g.Nr, g.N, g.N, pb.Nk), dtype=torch.float32, device="cuda")
    ws = fx.pipeline(prm, yt, y0t, D, xh, obj=obj)
    assert fx.status(ws) == 0
    P = fx.normalise(yt, y0t, p_dtype=fhr.BF16)
    D2, _, obj2 = fx.decompose(P, pb.Nk, K, iters, mlp=(dims, params))
    np.testing.assert_array_equal(D.cpu().numpy(), D2.cpu().numpy())
    np.testing.assert_array_equal(obj.cpu().numpy(), obj2.cpu().numpy())
    assert np.isfinite(xh.cpu().numpy()).all()
    prm.nmf.init = fhr.INIT_GIVEN
    with pytest.raises(fhr.FhrError):
        fx.pipeline_workspace(prm)
