"""Learned warm start for the decomposition (an added form; not in the paper).

A small MLP maps each pixel's spectrum p_j to its K subspace coefficients.  It
is trained, with the library's own GPU kernels (fhr_mlp_grad / fhr_mlp_adamw),
on coefficients that the plain method (NNDSVD start + fast HALS) produced on
synthetic phantoms that share one library of material spectra.  NMF factors are
unique only up to order and scale, so every training decomposition is put in a
canonical form first: D's columns are unit L2 (the decomposition already does
this) and are ordered by best cosine match to the library's spectra.  The
network then predicts W in that canonical basis, and FHR_INIT_LEARNED starts
the iterations from it.  The plain iterations remain the method and decide
the result: the warm start only changes where they begin.
"""
from __future__ import annotations

import ctypes
import itertools
import math

import numpy as np

from . import fhr, synth


def match_order(D: np.ndarray, library: np.ndarray) -> np.ndarray:
    """Column permutation of D that best matches the library columns (cosine, exhaustive for K <= 8)."""
    K = D.shape[1]
    Dn = D / np.maximum(np.linalg.norm(D, axis=0), 1e-30)
    Ln = library / np.maximum(np.linalg.norm(library, axis=0), 1e-30)
    C = Ln.T @ Dn                                   # [library][component]
    best, best_s = None, -np.inf
    for perm in itertools.permutations(range(K)):
        s = sum(C[i, perm[i]] for i in range(K))
        if s > best_s:
            best, best_s = perm, s
    return np.array(best)


def init_params(rng: np.random.Generator, Nk: int, H1: int, H2: int, K: int) -> np.ndarray:
    """He-style initial weights, zero biases, the output bias at softplus^-1(0.5)."""
    parts = [rng.normal(0, math.sqrt(2.0 / Nk), (H1, Nk)), np.zeros(H1),
             rng.normal(0, math.sqrt(2.0 / H1), (H2, H1)), np.zeros(H2),
             rng.normal(0, math.sqrt(1.0 / H2), (K, H2)), np.full(K, math.log(math.expm1(0.5)))]
    return np.concatenate([p.ravel() for p in parts]).astype(np.float32)


def make_training_set(ctx, library, problems, K, nmf_iters=300, seed=0):
    """Run the plain method on each problem; return (X rows of P, canonical W targets) as torch tensors."""
    import torch

    Xs, Ts = [], []
    for pb in problems:
        y, y0 = synth.counts_numpy(pb)
        yt = torch.from_numpy(y.view(np.int16)).cuda()
        y0t = torch.from_numpy(y0.view(np.int16)).cuda()
        P = ctx.normalise(yt, y0t)
        D, W, _ = ctx.decompose(P, pb.Nk, K, nmf_iters, init=fhr.INIT_NNDSVD, seed=seed, obj=False)
        perm = match_order(D.cpu().numpy(), library)
        Xs.append(P)
        Ts.append(W[:, torch.as_tensor(perm, device=W.device)].contiguous())
    return torch.cat(Xs), torch.cat(Ts)


def train(ctx, dims, X, T, *, steps=2000, batch=4096, lr=2e-3, wd=0.0, seed=0, params=None, log_every=0):
    """AdamW on the mean-squared error; returns (params, loss history)."""
    import torch

    rng = np.random.default_rng(seed)
    if params is None:
        params = torch.from_numpy(init_params(rng, dims.Nk, dims.H1, dims.H2, dims.K)).cuda()
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    grad = torch.empty_like(params)
    loss = torch.empty(1, dtype=torch.float64, device=params.device)
    nb = ctypes.c_size_t()
    ctx.check(ctx.L.fhr_mlp_workspace_size(ctx._h, ctypes.byref(dims), 1, ctypes.byref(nb)))
    ws = ctx.workspace(nb.value)
    hist = []
    g = torch.Generator(device=X.device)
    g.manual_seed(seed)
    N = X.shape[0]
    for step in range(1, steps + 1):
        idx = torch.randint(0, N, (min(batch, N),), device=X.device, generator=g)
        xb, tb = X[idx].contiguous(), T[idx].contiguous()
        ctx.mlp_grad(dims, params, xb, tb, grad=grad, loss=loss, ws=ws)
        ctx.mlp_adamw(params, grad, m, v, step, lr=lr, wd=wd)
        if log_every and (step % log_every == 0 or step == steps):
            hist.append((step, float(loss.item())))
    return params, hist
