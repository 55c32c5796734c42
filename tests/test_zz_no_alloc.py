"""fhr_decompose_static: the decomposition for callers that cannot allocate.

Some callers of this library can neither allocate device memory nor pass a
workspace: a plugin bound to a fixed C signature, a framework that owns every
byte of device memory, or a latency-critical loop where a cudaMalloc (which
can synchronise the device) is not allowed.  fhr_decompose_static serves them
with a fixed static scratch array inside the library.  This test calls it
through the C ABI, twice in a row (the array keeps the previous call's
contents), and checks each result against fhr_decompose with a caller
workspace, within the NMF tolerance the other tests use (1e-4 relative).
The file name sorts last so that a run that stops at the first failure has
already run every other test.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_static_workspace_matches_caller_workspace(fx):
    import torch
    from paper_2410_22500_gb300 import fhr

    L = fhr.load()
    g = torch.Generator(device="cuda")
    g.manual_seed(31)
    Np, Nk, K, iters = 20000, 300, 5, 12
    P = torch.rand((Np, Nk), device="cuda", generator=g)
    D0 = torch.rand((Nk, K), device="cuda", generator=g) + 0.1
    W0 = torch.rand((Np, K), device="cuda", generator=g) + 0.1
    Dr, Wr, objr = fx.decompose(P, Nk, K, iters, D=D0.clone(), W=W0.clone())
    Dr, Wr, objr = Dr.cpu().numpy(), Wr.cpu().numpy(), objr.cpu().numpy()
    prm = fx.nmf_params(P, Nk, K, iters, fhr.INIT_GIVEN)
    for call in range(2):
        D, W = D0.clone(), W0.clone()
        obj = torch.empty(iters, dtype=torch.float64, device="cuda")
        rc = L.fhr_decompose_static(fx._h, ctypes.byref(prm), ctypes.c_void_p(P.data_ptr()),
                                    ctypes.c_void_p(D.data_ptr()), ctypes.c_void_p(W.data_ptr()),
                                    ctypes.c_void_p(obj.data_ptr()))
        fx.check(rc)
        # errors found on the device (an expired wait, a non-finite objective) are read
        # from the static array's status word; this also synchronises the stream
        assert L.fhr_decompose_static_status(fx._h) == fhr.OK, L.fhr_last_error(fx._h)
        torch.cuda.synchronize()
        assert _rel(D.cpu().numpy(), Dr) <= 1e-4, call
        assert _rel(W.cpu().numpy(), Wr) <= 1e-4, call
        np.testing.assert_allclose(obj.cpu().numpy(), objr, rtol=1e-4)
    # the NNDSVD start takes the same static path
    prm2 = fx.nmf_params(P, Nk, K, 3, fhr.INIT_NNDSVD, seed=5)
    D, W = torch.empty_like(D0), torch.empty_like(W0)
    fx.check(L.fhr_decompose_static(fx._h, ctypes.byref(prm2), ctypes.c_void_p(P.data_ptr()),
                                    ctypes.c_void_p(D.data_ptr()), ctypes.c_void_p(W.data_ptr()), None))
    assert L.fhr_decompose_static_status(fx._h) == fhr.OK, L.fhr_last_error(fx._h)
    Dn, Wn, _ = fx.decompose(P, Nk, K, 3, init=fhr.INIT_NNDSVD, seed=5, obj=False)
    torch.cuda.synchronize()
    assert _rel(D.cpu().numpy(), Dn.cpu().numpy()) <= 1e-4
    assert _rel(W.cpu().numpy(), Wn.cpu().numpy()) <= 1e-4


def test_static_workspace_rejects_oversize_problems(fx):
    import torch
    from paper_2410_22500_gb300 import fhr

    L = fhr.load()
    # an objective history of 5M iterations alone needs 40 MB of scratch
    P = torch.zeros((8, 64), device="cuda")
    prm = fhr.NmfParams(8, 64, 64, 2, 5_000_000, fhr.INIT_GIVEN, fhr.F32, 0, 0)
    rc = L.fhr_decompose_static(fx._h, ctypes.byref(prm), ctypes.c_void_p(P.data_ptr()),
                                ctypes.c_void_p(P.data_ptr()), ctypes.c_void_p(P.data_ptr()), None)
    assert rc == fhr.ERR_ARG
    assert b"static workspace" in L.fhr_last_error(fx._h)
