"""FP64 CPU oracle for the FHR path (arXiv 2410.22500).

TEST INFRASTRUCTURE ONLY: imported by tests/, by __graft_entry__.smoke() and by
bench.py's CPU-baseline / reference leg, never by the library.  It shares no
code with the CUDA path.  The loops live in fhr_oracle.c (plain C, double
precision); this module loads it with ctypes and adds the steps that use a
library primitive (the SVD inside NNDSVD).

Every function cites the passage of the paper it follows.  Parity status:
  normalise        pinned (closed forms, planted offsets, per-bin and per-(pixel,
                   bin) dead masks, hand-worked background with a dead entry)
  HALS / NMF       pinned (NNLS limits, monotone objective, exact recovery)
  NNDSVD           pinned (rank-1 exactness, sign invariance, hand example)
  projector        pinned (polygon clipping, adjointness, mass, disk chords)
  MBIR (SQS)       pinned (dense least squares, quadratic prior solve, monotone)
  expansion        pinned (identity dictionary, commutes with the projector)
  MLP warm start   pinned (closed-form activations, layer-wise numpy, central
                   differences of the loss, AdamW closed form)
  FMD (semi-sup.)  pinned (hand-computed region means, exact recovery of a
                   nonnegative material mix, KKT on noisy data, App. B
                   identity D^m = D^s T^T recovering the material spectra)
  SNR (Sec. V-B)   pinned (both equations worked by hand on a 7-voxel case,
                   scale invariance, Gaussian noise of known sigma)
  FBP variant      pinned (textbook ramp samples, filter = direct convolution
                   with the kernel, disk reconstruction from analytic chords)
  clustering start pinned (published splitmix64 outputs, separated clusters
                   converge to their label means, monotone Lloyd cost, K = 1
                   mean, zero-distance samples never seeded, K = 1 V step)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fhr_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_u16p = ctypes.POINTER(ctypes.c_uint16)
_u8p = ctypes.POINTER(ctypes.c_uint8)


def build(force: bool = False) -> str:
    """Compile fhr_oracle.c into liboracle.so beside it (gcc, -O2, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _MbirParams(ctypes.Structure):
    _fields_ = [("p", ctypes.c_double), ("q", ctypes.c_double), ("T", ctypes.c_double),
                ("beta", ctypes.c_double), ("iters", ctypes.c_int), ("momentum", ctypes.c_int)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            L = _lib
            L.or_set_threads.restype = ctypes.c_int
            L.or_set_threads.argtypes = [ctypes.c_int]
            L.or_set_threads(1)
            L.or_normalise.restype = ctypes.c_int
            L.or_normalise.argtypes = [ctypes.c_int] * 4 + [_u16p, _u16p, _u8p, _u8p, ctypes.c_int, _dp, _dp]
            L.or_hals_update_W.argtypes = [ctypes.c_long, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp]
            L.or_hals_update_D.argtypes = [ctypes.c_long, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp]
            L.or_normalise_columns.argtypes = [ctypes.c_long, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp]
            L.or_objective.restype = ctypes.c_double
            L.or_objective.argtypes = [ctypes.c_long, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp]
            L.or_nmf.argtypes = [ctypes.c_long, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp]
            for f in ("or_strip_area", "or_strip_area_polyclip"):
                getattr(L, f).restype = ctypes.c_double
                getattr(L, f).argtypes = [ctypes.c_double] * 4
            L.or_system_matrix.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int, _dp]
            L.or_project.argtypes = [ctypes.c_int] * 3 + [_dp, ctypes.c_int, _dp, _dp]
            L.or_backproject.argtypes = [ctypes.c_int] * 3 + [_dp, ctypes.c_int, _dp, _dp]
            for f in ("or_qggmrf_rho", "or_qggmrf_influence"):
                getattr(L, f).restype = ctypes.c_double
                getattr(L, f).argtypes = [ctypes.c_double] * 5
            L.or_mbir_cost.restype = ctypes.c_double
            L.or_mbir_cost.argtypes = [ctypes.c_int] * 5 + [_dp, _dp, _dp, _dp, ctypes.POINTER(_MbirParams), _dp]
            L.or_mbir.argtypes = [ctypes.c_int] * 5 + [_dp, _dp, _dp, _dp, ctypes.POINTER(_MbirParams), _dp, _dp]
            L.or_mbir_sigmas.argtypes = [ctypes.c_long, ctypes.c_int, _dp, ctypes.c_double, ctypes.c_int, _dp, _dp]
            L.or_expand.argtypes = [ctypes.c_int] * 4 + [_dp, _dp, _dp]
            L.or_ramp.restype = ctypes.c_double
            L.or_ramp.argtypes = [ctypes.c_int]
            L.or_ramp_filter.argtypes = [ctypes.c_int] * 3 + [_dp, _dp]
            L.or_fbp.argtypes = [ctypes.c_int] * 3 + [_dp, ctypes.c_int, _dp, _dp]
            vp = ctypes.c_void_p
            L.or_snr.argtypes = [ctypes.c_long, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _u8p, _dp]
            L.or_splitmix64.argtypes = [ctypes.c_uint64, ctypes.c_int, vp]
            L.or_splitmix64.restype = None
            L.or_kmeans.argtypes = [ctypes.c_long, ctypes.c_int, _dp, ctypes.c_long, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_uint64, _dp, vp, _dp, vp]
            L.or_cluster_init.argtypes = [ctypes.c_long, ctypes.c_int, _dp, ctypes.c_long, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_uint64, _dp, _dp]
        return _lib


def set_threads(n: int) -> int:
    """Host threads of the oracle's parallel loops (1 = serial, the default).
    Results do not depend on it: every sum is taken in a fixed order."""
    return int(lib().or_set_threads(int(n)))


def _d(a):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------- normalise
def normalise(y, y0, bg=None, dead=None, return_offset=False):
    """Eq. (neglogattenuation) with the offset correction of Appendix A.

    y [Nv][Nr][Nc][Nk] uint16, y0 [Nr][Nc][Nk] uint16 -> P [Nv*Nc*Nr][Nk]
    (pixel order (v, c, r)).  bg: [Nr][Nc] background mask; dead: [Nk] mask of dead
    bins or [Nr][Nc][Nk] mask of dead (detector pixel, bin) entries.  Dead entries give
    p = 0 and are left out of the background mean (a (v, k) with no live background
    entry gets b = 0)."""
    y = np.ascontiguousarray(y, dtype=np.uint16)
    y0 = np.ascontiguousarray(y0, dtype=np.uint16)
    Nv, Nr, Nc, Nk = y.shape
    assert y0.shape == (Nr, Nc, Nk)
    P = np.empty((Nv * Nc * Nr, Nk))
    b = np.empty((Nv, Nk))
    bg_keep = None if bg is None else np.ascontiguousarray(bg, dtype=np.uint8)
    bgp = None if bg_keep is None else bg_keep.ctypes.data_as(_u8p)
    dead_keep = None if dead is None else np.ascontiguousarray(dead, dtype=np.uint8)
    per_pixel = 0
    if dead_keep is not None:
        per_pixel = int(dead_keep.ndim == 3)
        assert dead_keep.shape == ((Nr, Nc, Nk) if per_pixel else (Nk,))
    dp = None if dead_keep is None else dead_keep.ctypes.data_as(_u8p)
    rc = lib().or_normalise(Nv, Nr, Nc, Nk, y.ctypes.data_as(_u16p), y0.ctypes.data_as(_u16p),
                            bgp, dp, per_pixel, _d(P), _d(b))
    if rc:
        raise ValueError("or_normalise failed: %d" % rc)
    return (P, b) if return_offset else P


# ---------------------------------------------------------------- NMF (HALS)
def hals_update_W(P, D, W):
    """One V half-step of fast HALS (Sec. III, Eq. sub_extract_solve); W updated in place."""
    Np, Nk = P.shape
    K = D.shape[1]
    lib().or_hals_update_W(Np, Nk, K, _d(P), _d(D), _d(W))
    return W


def hals_update_D(P, W, D):
    """One D half-step of fast HALS; D updated in place."""
    Np, Nk = P.shape
    K = D.shape[1]
    lib().or_hals_update_D(Np, Nk, K, _d(P), _d(W), _d(D))
    return D


def normalise_columns(D, W):
    """Unit-L2 columns of D, inverse scaling of W's columns (reading: product unchanged)."""
    Nk, K = D.shape
    n = np.empty(K)
    lib().or_normalise_columns(W.shape[0], Nk, K, _d(D), _d(W), _d(n))
    return n


def objective(P, D, W):
    """||P - W D^T||_F^2 evaluated entry by entry (Eq. sub_extract_solve)."""
    Np, Nk = P.shape
    return lib().or_objective(Np, Nk, D.shape[1], _d(_f64(P)), _d(_f64(D)), _d(_f64(W)))


def nmf(P, D0, W0, iters):
    """`iters` iterations of (V step, D step, column scaling); returns D, W, objective history."""
    P = _f64(P)
    D = _f64(D0).copy()
    W = _f64(W0).copy()
    obj = np.empty(max(iters, 1))
    Np, Nk = P.shape
    rc = lib().or_nmf(Np, Nk, D.shape[1], iters, _d(P), _d(D), _d(W), _d(obj))
    if rc:
        raise ValueError("or_nmf failed: %d" % rc)
    return D, W, obj[:iters]


def nndsvd_split(U, S, Vt, K):
    """NNDSVD (Boutsidis & Gallopoulos 2008), the initialisation named in Sec. III.

    Input: the top singular triplets of P = U diag(S) Vt (P is Np x Nk; U holds
    pixel vectors, Vt wavelength vectors).  For j = 0 the factors are
    sqrt(S_0)|u_0| and sqrt(S_0)|v_0|.  For j >= 1 the positive and negative
    parts of (u_j, v_j) are compared by the product of their norms; the larger
    pair (ties to the positive pair), unit-normalised and scaled by
    sqrt(S_j * that product), gives column j.  A zero product gives a zero
    column.  Returns D0 [Nk][K], W0 [Np][K]."""
    Np, Nk = U.shape[0], Vt.shape[1]
    W = np.zeros((Np, K))
    D = np.zeros((Nk, K))
    W[:, 0] = np.sqrt(S[0]) * np.abs(U[:, 0])
    D[:, 0] = np.sqrt(S[0]) * np.abs(Vt[0, :])
    for j in range(1, K):
        x, y = U[:, j], Vt[j, :]
        xp, xn = np.maximum(x, 0), np.maximum(-x, 0)
        yp, yn = np.maximum(y, 0), np.maximum(-y, 0)
        nxp, nxn = np.linalg.norm(xp), np.linalg.norm(xn)
        nyp, nyn = np.linalg.norm(yp), np.linalg.norm(yn)
        mp, mn = nxp * nyp, nxn * nyn
        if mp >= mn:
            u, v, m, nu, nv = xp, yp, mp, nxp, nyp
        else:
            u, v, m, nu, nv = xn, yn, mn, nxn, nyn
        if m > 0:
            lam = np.sqrt(S[j] * m)
            W[:, j] = lam * u / nu
            D[:, j] = lam * v / nv
    return D, W


def nndsvd(P, K):
    """NNDSVD initialisation of P (Np x Nk) from numpy's exact SVD."""
    U, S, Vt = np.linalg.svd(_f64(P), full_matrices=False)
    return nndsvd_split(U[:, :K], S[:K], Vt[:K, :], K)


def splitmix64(seed, n):
    """The first n outputs of splitmix64 started from state `seed`."""
    out = np.zeros(n, dtype=np.uint64)
    lib().or_splitmix64(ctypes.c_uint64(seed), n, out.ctypes.data_as(ctypes.c_void_p))
    return out


def kmpp_pick(d, u):
    """The k-means++ pick: the first sample whose running sum of d exceeds u times the
    total (the last sample with d > 0 if rounding leaves none); -1 for a zero total."""
    L = lib()
    L.or_kmpp_pick.restype = ctypes.c_long
    L.or_kmpp_pick.argtypes = [_dp, ctypes.c_long, ctypes.c_double]
    d = np.ascontiguousarray(d, dtype=np.float64)
    return int(L.or_kmpp_pick(_d(d), d.size, float(u)))


def kmeans(P, S, K, iters, seed):
    """k-means of the sampled rows of P (the clustering start's first three steps).
    Returns (centres [K][Nk], labels [S], cost [iters+1], seeds [K])."""
    P = _f64(P)
    Np, Nk = P.shape
    C = np.zeros((K, Nk))
    lab = np.zeros(S, dtype=np.int32)
    cost = np.zeros(iters + 1)
    seeds = np.zeros(K, dtype=np.int64)
    rc = lib().or_kmeans(Np, Nk, _d(P), S, K, iters, ctypes.c_uint64(seed), _d(C),
                         lab.ctypes.data_as(ctypes.c_void_p), _d(cost), seeds.ctypes.data_as(ctypes.c_void_p))
    if rc:
        raise ValueError("or_kmeans failed: %d" % rc)
    return C, lab, cost, seeds


def cluster_init(P, K, S=None, iters=20, seed=0):
    """Clustering start: D0 [Nk][K] = k-means centres, W0 [Np][K] = one HALS V step from 0."""
    P = _f64(P)
    Np, Nk = P.shape
    S = min(Np, 32768) if S is None else S
    D0 = np.zeros((Nk, K))
    W0 = np.zeros((Np, K))
    rc = lib().or_cluster_init(Np, Nk, _d(P), S, K, iters, ctypes.c_uint64(seed), _d(D0), _d(W0))
    if rc:
        raise ValueError("or_cluster_init failed: %d" % rc)
    return D0, W0


# ---------------------------------------------------------------- projector
def strip_area(theta, px, py, uc):
    return lib().or_strip_area(theta, px, py, uc)


def strip_area_polyclip(theta, px, py, uc):
    return lib().or_strip_area_polyclip(theta, px, py, uc)


def system_matrix(N, Nc, theta, polyclip=False):
    """Dense A, [Nv*Nc][N*N] (tiny cases)."""
    theta = _f64(theta)
    A = np.empty((theta.size * Nc, N * N))
    lib().or_system_matrix(N, Nc, theta.size, _d(theta), int(polyclip), _d(A))
    return A


def project(x, Nc, theta):
    """y = A x.  x [N][N][Wl] -> y [Nv][Nc][Wl]."""
    x = _f64(x)
    N = x.shape[0]
    Wl = x.shape[2] if x.ndim == 3 else 1
    theta = _f64(theta)
    y = np.empty((theta.size, Nc, Wl))
    lib().or_project(N, Nc, theta.size, _d(theta), Wl, _d(x), _d(y))
    return y


def backproject(y, N, theta):
    """x = A^T y.  y [Nv][Nc][Wl] -> x [N][N][Wl]."""
    y = _f64(y)
    Nv, Nc = y.shape[:2]
    Wl = y.shape[2] if y.ndim == 3 else 1
    theta = _f64(theta)
    x = np.empty((N, N, Wl))
    lib().or_backproject(N, Nc, Nv, _d(theta), Wl, _d(y), _d(x))
    return x


def ramp(n):
    """The sampled ramp filter h[n] of the FBP variant (Kak and Slaney, tau = 1)."""
    return lib().or_ramp(int(n))


def ramp_filter(p):
    """q[v][c] = sum_c' h[c - c'] p[v][c'] along the detector, p [Nv][Nc][Wl]."""
    p = _f64(p)
    Nv, Nc = p.shape[:2]
    Wl = p.shape[2] if p.ndim == 3 else 1
    q = np.empty((Nv, Nc, Wl))
    lib().or_ramp_filter(Nv, Nc, Wl, _d(p), _d(q))
    return q


def fbp(p, N, theta):
    """Filtered back-projection x = (pi / Nv) A^T (h * p): p [Nv][Nc][Wl] -> x [N][N][Wl]."""
    p = _f64(p)
    Nv, Nc = p.shape[:2]
    Wl = p.shape[2] if p.ndim == 3 else 1
    theta = _f64(theta)
    x = np.empty((N, N, Wl))
    rc = lib().or_fbp(N, Nc, Nv, _d(theta), Wl, _d(p), _d(x))
    if rc:
        raise ValueError("or_fbp failed: %d" % rc)
    return x


# ---------------------------------------------------------------- MBIR
def qggmrf_rho(d, sx, p=1.2, q=2.0, T=1.0):
    return lib().or_qggmrf_rho(d, sx, p, q, T)


def qggmrf_influence(d, sx, p=1.2, q=2.0, T=1.0):
    return lib().or_qggmrf_influence(d, sx, p, q, T)


def mbir_sigmas(V, K, Nc, snr_db=30.0):
    """Per-channel (sigma_v, sigma_x) from the subspace sinogram (reading, paper silent)."""
    V = _f64(V).reshape(-1, K)
    sv, sx = np.empty(K), np.empty(K)
    lib().or_mbir_sigmas(V.shape[0], K, _d(V), snr_db, Nc, _d(sv), _d(sx))
    return sv, sx


def _params(p, q, T, beta, iters, momentum):
    return _MbirParams(p, q, T, beta, iters, int(momentum))


def mbir(V, N, Nr, K, theta, sv, sx, *, p=1.2, q=2.0, T=1.0, beta=1.0, iters=20, momentum=False,
         x0=None, cost=False):
    """SQS solve of Eq. (recon) for all K channels and Nr slices at once.

    V [Nv][Nc][Nr*K] sinogram -> x [N][N][Nr*K]."""
    V = _f64(V)
    Nv, Nc = V.shape[:2]
    theta = _f64(theta)
    x = np.zeros((N, N, Nr * K)) if x0 is None else _f64(x0).copy()
    hist = np.empty(max(iters, 1))
    prm = _params(p, q, T, beta, iters, momentum)
    rc = lib().or_mbir(N, Nr, K, Nc, Nv, _d(theta), _d(V), _d(_f64(sv)), _d(_f64(sx)),
                       ctypes.byref(prm), _d(x), _d(hist) if cost else None)
    if rc:
        raise ValueError("or_mbir failed: %d" % rc)
    return (x, hist[:iters]) if cost else x


def mbir_cost(V, x, N, Nr, K, theta, sv, sx, *, p=1.2, q=2.0, T=1.0, beta=1.0):
    V = _f64(V)
    Nv, Nc = V.shape[:2]
    prm = _params(p, q, T, beta, 0, False)
    return lib().or_mbir_cost(N, Nr, K, Nc, Nv, _d(_f64(theta)), _d(V), _d(_f64(sv)), _d(_f64(sx)),
                              ctypes.byref(prm), _d(_f64(x)))


# ---------------------------------------------------------------- expansion
def expand(xs, D, N, Nr):
    """Eq. (sub_expansion): x^h = x^s D^T.  xs [N][N][Nr*K] -> xh [Nr][N][N][Nk]."""
    xs = _f64(xs)
    D = _f64(D)
    Nk, K = D.shape
    xh = np.empty((Nr, N, N, Nk))
    lib().or_expand(N, Nr, K, Nk, _d(xs), _d(D), _d(xh))
    return xh


# ---------------------------------------------------------------- SNR (Sec. V-B)
SNR_FMD, SNR_FHR = 0, 1
ROI_BACKGROUND = 255


def snr(x, roi, Nm, mode):
    """Eq. (snr_fmd) (mode SNR_FMD: channel m over region m) or Eq. (snr_fhr) (mode SNR_FHR:
    every channel over every region), in dB.  x [Nx][C]; roi [Nx] u8: 0 none, m + 1 inside
    material m, 255 background."""
    x = _f64(x)
    Nx, C = x.shape
    roi = np.ascontiguousarray(roi, dtype=np.uint8).reshape(-1)
    out = ctypes.c_double()
    rc = lib().or_snr(Nx, C, Nm, mode, _d(x), roi.ctypes.data_as(_u8p), ctypes.byref(out))
    if rc:
        raise ValueError("or_snr failed: %d" % rc)
    return out.value


# ---------------------------------------------------------------- pipeline
def fhr_pipeline(y, y0, K, N, theta, *, nmf_iters=200, mbir_iters=20, dead=None, bg=None,
                 init=None, p=1.2, T=1.0, snr_db=30.0, momentum=False, recon="mbir"):
    """Algorithm 1 end to end: normalise -> NMF -> MBIR (or FBP) per channel -> expansion.

    init: None for NNDSVD, else a (D0, W0) pair.  Returns a dict of every
    intermediate (P, D, W, obj, xs, xh, sigmas)."""
    Nv, Nr, Nc, Nk = y.shape
    P = normalise(y, y0, bg=bg, dead=dead)
    D0, W0 = nndsvd(P, K) if init is None else init
    D, W, obj = nmf(P, D0, W0, nmf_iters)
    V = W.reshape(Nv, Nc, Nr * K)
    sv, sx = mbir_sigmas(W, K, Nc, snr_db)
    if recon == "fbp":
        xs = fbp(V, N, theta)
    else:
        xs = mbir(V, N, Nr, K, theta, sv, sx, p=p, T=T, iters=mbir_iters, momentum=momentum)
    xh = expand(xs, D, N, Nr)
    return dict(P=P, D0=D0, W0=W0, D=D, W=W, obj=obj, sv=sv, sx=sx, xs=xs, xh=xh)


# ---------------------------------------------------------------- FMD, semi-supervised (Algorithm 2)
def fmd_transform(xs, labels, Nm):
    """Eq. trans_mat: T[i][j] = mean of x^s_{n,j} over the voxels n of region i
    (labels[n] = i + 1; 0 = in no region).  xs [Nx][Ns] -> T [Nm][Ns]."""
    xs = _f64(xs)
    labels = np.asarray(labels).reshape(-1)
    T = np.zeros((Nm, xs.shape[1]))
    for i in range(Nm):
        sel = xs[labels == i + 1]
        if len(sel):
            T[i] = sel.mean(axis=0)
    return T


def fmd_materials(xs, T):
    """Eq. mat_recon_nmf: x^m = argmin_{x >= 0} ||x^s - x T||_F^2, one nonnegative
    least-squares problem per voxel (scipy's Lawson-Hanson NNLS as the solver)."""
    from scipy.optimize import nnls

    xs = _f64(xs)
    T = _f64(T)
    xm = np.zeros((xs.shape[0], T.shape[0]))
    A = T.T.copy()
    for n in range(xs.shape[0]):
        xm[n], _ = nnls(A, xs[n])
    return xm


def fmd_spectra(D, T):
    """Eq. sub_mat_rel_basis: D^m = D^s T^T."""
    return _f64(D) @ _f64(T).T


def fmd(xs, D, labels, Nm):
    """Algorithm 2 after the reconstruction, semi-supervised (user regions):
    returns (T, x^m, D^m)."""
    T = fmd_transform(xs, labels, Nm)
    return T, fmd_materials(xs, T), fmd_spectra(D, T)


# ---------------------------------------------------------------- learned warm start (MLP)
def _mlp_lib():
    L = lib()
    if not getattr(L, "_mlp_ready", False):
        L.or_gelu.restype = ctypes.c_double
        L.or_gelu.argtypes = [ctypes.c_double]
        L.or_softplus.restype = ctypes.c_double
        L.or_softplus.argtypes = [ctypes.c_double]
        L.or_mlp_nparams.restype = ctypes.c_long
        L.or_mlp_nparams.argtypes = [ctypes.c_int] * 4
        L.or_mlp_forward.restype = ctypes.c_double
        L.or_mlp_forward.argtypes = [ctypes.c_int] * 5 + [_dp, _dp, _dp, _dp]
        L.or_mlp_grad.restype = ctypes.c_double
        L.or_mlp_grad.argtypes = [ctypes.c_int] * 5 + [_dp, _dp, _dp, _dp]
        L.or_adamw.argtypes = [ctypes.c_long, _dp, _dp, _dp, _dp, ctypes.c_int] + [ctypes.c_double] * 5
        L._mlp_ready = True
    return L


def gelu(x):
    return _mlp_lib().or_gelu(x)


def softplus(z):
    return _mlp_lib().or_softplus(z)


def mlp_nparams(Nk, H1, H2, K):
    return _mlp_lib().or_mlp_nparams(Nk, H1, H2, K)


def mlp_forward(prm, X, dims, T=None):
    """MLP spectrum -> coefficients (the library's learned warm start). Returns Y [M][K] (and the MSE loss)."""
    Nk, H1, H2, K = dims
    X = _f64(X).reshape(-1, Nk)
    Y = np.empty((X.shape[0], K))
    loss = _mlp_lib().or_mlp_forward(X.shape[0], Nk, H1, H2, K, _d(_f64(prm)), _d(X), _d(Y),
                                     None if T is None else _d(_f64(T)))
    return (Y, loss) if T is not None else Y


def mlp_grad(prm, X, T, dims):
    """Mean-squared-error loss and its gradient with respect to the packed parameters."""
    Nk, H1, H2, K = dims
    X = _f64(X).reshape(-1, Nk)
    G = np.empty(mlp_nparams(Nk, H1, H2, K))
    loss = _mlp_lib().or_mlp_grad(X.shape[0], Nk, H1, H2, K, _d(_f64(prm)), _d(X), _d(_f64(T)), _d(G))
    return loss, G


def adamw(w, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8, wd=1e-4):
    """One AdamW step in place (decoupled weight decay)."""
    _mlp_lib().or_adamw(w.size, _d(w), _d(_f64(g)), _d(m), _d(v), t, lr, b1, b2, eps, wd)
    return w
