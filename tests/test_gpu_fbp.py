"""GPU parity of the FBP variant of the reconstruction step (ramp filter + strip-area back-projection)."""
import math

import numpy as np
import pytest
from _parity import assert_close, rel_l2 as _rel

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("N,Nc,Nv,Wl", [(32, 48, 60, 3), (16, 23, 17, 8), (24, 40, 45, 12), (9, 13, 7, 1),
                                        (40, 64, 90, 33)])
def test_fbp_matches_oracle(fx, orc, N, Nc, Nv, Wl):
    rng = np.random.default_rng(500 + N)
    p = rng.uniform(0, 1, size=(Nv, Nc, Wl)).astype(np.float32)
    th = np.arange(Nv) * (math.pi / Nv)
    got = fx.fbp(_dev(p), N).cpu().numpy()
    ref = orc.fbp(p.astype(np.float64), N, th)
    assert_close(got, ref, 1e-5)


def test_fbp_of_disk_projections(fx, orc):
    # the GPU result inverts a disk's analytic projections like the oracle does
    N, Nc, Nv, R = 64, 96, 180, 20.0
    u = (np.arange(Nc) - (Nc - 1) / 2.0)[:, None] + (np.arange(16) + 0.5)[None, :] / 16 - 0.5
    chord = 2.0 * np.sqrt(np.maximum(R * R - u * u, 0.0)).mean(axis=1)
    p = np.repeat(chord[None, :], Nv, axis=0)[..., None].astype(np.float32)
    x = fx.fbp(_dev(p), N).cpu().numpy()[..., 0]
    c = np.arange(N) - (N - 1) / 2.0
    r = np.sqrt(c[:, None] ** 2 + c[None, :] ** 2)
    assert abs(x[r < 0.8 * R].mean() - 1.0) < 0.02


def test_pipeline_with_fbp_matches_oracle(fx, orc):
    import torch

    from paper_2410_22500_gb300 import fhr, synth

    pb = synth.tiny_2d()
    g = pb.geom
    y, y0 = synth.counts_numpy(pb)
    K, iters = 3, 200
    prm = fx.pipeline_params(Nv=g.Nv, Nr=g.Nr, Nc=g.Nc, Nk=pb.Nk, N=g.N, K=K, nmf_iters=iters, mbir_iters=1,
                             seed=3, recon=fhr.RECON_FBP)
    D = torch.empty((pb.Nk, K), dtype=torch.float32, device="cuda")
    obj = torch.empty(iters, dtype=torch.float64, device="cuda")
    xh = torch.empty((g.Nr, g.N, g.N, pb.Nk), dtype=torch.float32, device="cuda")
    ws = fx.pipeline(prm, torch.from_numpy(y.view(np.int16)).cuda(), torch.from_numpy(y0.view(np.int16)).cuda(),
                     D, xh, obj=obj)
    assert fx.status(ws) == 0
    ref = orc.fhr_pipeline(y, y0, K, g.N, g.angles(), nmf_iters=iters, recon="fbp")
    assert_close(xh.cpu().numpy(), ref["xh"], 1e-3)
