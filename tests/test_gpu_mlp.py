"""GPU parity of the learned warm start: MLP forward, gradient and AdamW kernels against the
FP64 oracle, and what the trained network gains over the plain start."""
import math

import numpy as np
import pytest
from _parity import assert_close

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def _params(rng, dims, scale=1.0):
    Nk, H1, H2, K = dims
    parts = [rng.normal(0, scale / math.sqrt(Nk), (H1, Nk)), rng.normal(0, 0.1, H1),
             rng.normal(0, scale / math.sqrt(H1), (H2, H1)), rng.normal(0, 0.1, H2),
             rng.normal(0, scale / math.sqrt(H2), (K, H2)), rng.normal(0, 0.1, K)]
    return np.concatenate([p.ravel() for p in parts]).astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("M,dims", [(300, (40, 32, 16, 3)), (70, (128, 256, 128, 6)), (33000, (24, 20, 12, 5))])
def test_forward_f32_matches_oracle(fx, orc, M, dims):
    import torch

    rng = np.random.default_rng(M)
    prm = _params(rng, dims)
    X = rng.uniform(0, 2, size=(M, dims[0])).astype(np.float32)
    d = fx.mlp_dims(*dims)
    Y = fx.mlp_forward(d, torch.from_numpy(prm.astype(np.float32)).cuda(), torch.from_numpy(X).cuda()).cpu().numpy()
    ref = orc.mlp_forward(prm, X.astype(np.float64), dims)
    assert_close(Y, ref, 1e-5)


def test_forward_bf16_weights_and_rows(fx, orc):
    # bf16 weights and bf16 input rows with a padded row stride, FP32 accumulation: the error
    # against FP64 (on the same bf16-rounded inputs) is bounded by bf16 rounding, ~1e-2
    import torch

    rng = np.random.default_rng(5)
    dims = (100, 64, 32, 4)
    prm = _params(rng, dims)
    X = rng.uniform(0, 2, size=(500, 104)).astype(np.float32)
    Xb = torch.from_numpy(X).to(torch.bfloat16)
    d = fx.mlp_dims(*dims, ldx=104, x_bf16=True, weights_bf16=True)
    Y = fx.mlp_forward(d, torch.from_numpy(prm.astype(np.float32)).cuda(), Xb.cuda()).cpu().numpy()
    ref = orc.mlp_forward(prm, Xb.float().numpy()[:, :100].astype(np.float64), dims)
    err = _rel(Y, ref)
    print("bf16-weight forward: relative error %.2e vs FP64" % err)
    assert err <= 2e-2


def test_forward_tensor_core_layers_at_the_volume_shape(fx, orc):
    # the 1500 -> 256 -> 128 -> 6 network on bf16 rows of stride 1504 (the tensor-core layers),
    # two inference chunks with a ragged tail: FP64 oracle on sampled rows, and the CUDA-core
    # layers (taken for a row stride that is not a multiple of 8) on all rows
    import torch

    rng = np.random.default_rng(21)
    dims = (1500, 256, 128, 6)
    prm = _params(rng, dims)
    M = 70001
    X = torch.rand((M, 1504), generator=torch.Generator().manual_seed(3)).mul_(2).to(torch.bfloat16)
    p32 = torch.from_numpy(prm.astype(np.float32)).cuda()
    d = fx.mlp_dims(*dims, ldx=1504, x_bf16=True, weights_bf16=True)
    Y = fx.mlp_forward(d, p32, X.cuda()).cpu().numpy()
    rows = np.sort(rng.choice(M, 600, replace=False))
    rows[-1] = M - 1
    ref = orc.mlp_forward(prm, X[rows, :1500].float().numpy().astype(np.float64), dims)
    err = _rel(Y[rows], ref)
    print("tensor-core forward: relative error %.2e vs FP64" % err)
    assert err <= 2e-2
    X2 = torch.zeros((M, 1502), dtype=torch.bfloat16)
    X2[:, :1500] = X[:, :1500]
    d2 = fx.mlp_dims(*dims, ldx=1502, x_bf16=True, weights_bf16=True)
    Y2 = fx.mlp_forward(d2, p32, X2.cuda()).cpu().numpy()
    assert_close(Y, Y2, 2e-3)


def test_gradient_bf16_rows_and_weights(fx, orc):
    # the training forward on the tensor-core layers (pre-activations kept) and the backward
    import torch

    rng = np.random.default_rng(9)
    dims = (72, 40, 24, 3)
    M = 3000
    prm = _params(rng, dims, scale=1.5)
    X = torch.from_numpy(rng.uniform(0, 1.5, size=(M, 72)).astype(np.float32)).to(torch.bfloat16)
    T = rng.uniform(0.1, 1.0, size=(M, 3)).astype(np.float32)
    d = fx.mlp_dims(*dims, x_bf16=True, weights_bf16=True)
    loss, g = fx.mlp_grad(d, torch.from_numpy(prm.astype(np.float32)).cuda(), X.cuda(), torch.from_numpy(T).cuda())
    lref, gref = orc.mlp_grad(prm, X.float().numpy().astype(np.float64), T.astype(np.float64), dims)
    assert abs(float(loss.item()) - lref) <= 2e-2 * lref
    assert_close(g.cpu().numpy(), gref, 5e-2)


@pytest.mark.parametrize("M,dims", [(200, (30, 24, 12, 3)), (1500, (64, 48, 20, 5))])
def test_gradient_matches_oracle(fx, orc, M, dims):
    import torch

    rng = np.random.default_rng(M + 1)
    prm = _params(rng, dims, scale=1.5)
    X = rng.uniform(0, 1.5, size=(M, dims[0])).astype(np.float32)
    T = rng.uniform(0.1, 1.0, size=(M, dims[3])).astype(np.float32)
    d = fx.mlp_dims(*dims)
    loss, g = fx.mlp_grad(d, torch.from_numpy(prm.astype(np.float32)).cuda(), torch.from_numpy(X).cuda(),
                          torch.from_numpy(T).cuda())
    lref, gref = orc.mlp_grad(prm, X.astype(np.float64), T.astype(np.float64), dims)
    assert abs(float(loss.item()) - lref) <= 1e-5 * lref
    g = g.cpu().numpy()
    assert_close(g, gref, 1e-4)
    # every parameter block separately (a wrong layer hides in a global norm)
    Nk, H1, H2, K = dims
    o = 0
    for n in (H1 * Nk, H1, H2 * H1, H2, K * H2, K):
        assert_close(g[o:o + n], gref[o:o + n], 1e-4)
        o += n


def test_adamw_matches_oracle(fx, orc):
    import torch

    rng = np.random.default_rng(9)
    n = 1000
    w = rng.normal(size=n)
    wt = torch.from_numpy(w.astype(np.float32)).cuda()
    m, v = torch.zeros(n, device="cuda"), torch.zeros(n, device="cuda")
    wr, mr, vr = w.astype(np.float32).astype(np.float64), np.zeros(n), np.zeros(n)
    for t in range(1, 4):
        gr = rng.normal(size=n).astype(np.float32)
        fx.mlp_adamw(wt, torch.from_numpy(gr).cuda(), m, v, t, lr=1e-2, wd=0.01)
        orc.adamw(wr, gr.astype(np.float64), mr, vr, t, lr=1e-2, wd=0.01)
    assert_close(wt.cpu().numpy(), wr, 1e-6)


def test_gpu_training_fits_a_teacher(fx, orc):
    import torch
    from paper_2410_22500_gb300 import learned

    rng = np.random.default_rng(11)
    dims = (16, 32, 16, 3)
    teacher = _params(rng, dims, scale=2.0)
    X = rng.uniform(0, 1, size=(8192, 16)).astype(np.float32)
    T = orc.mlp_forward(teacher, X.astype(np.float64), dims).astype(np.float32)
    d = fx.mlp_dims(*dims)
    Xt, Tt = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    p0 = torch.from_numpy(learned.init_params(np.random.default_rng(0), *dims)).cuda()
    l0, _ = fx.mlp_grad(d, p0, Xt[:4096].contiguous(), Tt[:4096].contiguous())
    prm, hist = learned.train(fx, d, Xt, Tt, steps=600, batch=2048, lr=3e-3, log_every=100, seed=0)
    assert hist[-1][1] < 0.1 * float(l0.item())
    assert hist[-1][1] < hist[0][1]


def test_learned_start_needs_fewer_iterations(fx, orc):
    # train on the plain method's decompositions of phantoms that share one spectra library,
    # then start a held-out phantom from the network: it reaches the plain objective
    # (within 1e-3) in fewer fast-HALS iterations than the NNDSVD start
    import torch
    from paper_2410_22500_gb300 import learned, synth

    K, Nk = 3, 128
    lib = synth.spectra_library(Nk, K, seed=77)
    mk = lambda seed: synth.make_problem(N=32, Nr=2, Nc=48, Nv=40, Nk=Nk, Nm=K, I0=400, seed=seed, spectra=lib)
    train_pbs = [mk(3000 + i) for i in range(8)]
    X, T = learned.make_training_set(fx, lib, train_pbs, K, nmf_iters=300)
    d = fx.mlp_dims(Nk, 64, 32, K)
    prm, hist = learned.train(fx, d, X, T, steps=1500, batch=4096, lr=2e-3, log_every=500)
    held = mk(4000)
    y, y0 = synth.counts_numpy(held)
    P = fx.normalise(torch.from_numpy(y.view(np.int16)).cuda(), torch.from_numpy(y0.view(np.int16)).cuda())
    iters = 300
    _, _, obj_plain = fx.decompose(P, Nk, K, iters, init=1, seed=0)
    _, _, obj_learn = fx.decompose(P, Nk, K, iters, mlp=(d, prm))
    obj_plain, obj_learn = obj_plain.cpu().numpy(), obj_learn.cpu().numpy()
    target = obj_plain[-1] * (1 + 1e-3)
    n_plain = int(np.argmax(obj_plain <= target)) + 1
    n_learn = int(np.argmax(obj_learn <= target)) + 1 if np.any(obj_learn <= target) else iters + 1
    print("iterations to the plain objective (+1e-3): plain %d, learned %d" % (n_plain, n_learn))
    assert n_learn < n_plain
    assert obj_learn[-1] <= obj_plain[-1] * (1 + 1e-3)
