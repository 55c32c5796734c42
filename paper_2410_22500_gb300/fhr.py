"""ctypes binding of libfhr (include/fhr.h): argument marshalling only.

Every step of the path runs in the library's CUDA kernels; PyTorch is used
here only to own device memory (tensors) and to name the stream.  There is no
CPU fallback: if libfhr.so is missing or no CUDA device is present, calls fail.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfhr.so")

F32, BF16 = 0, 1
INIT_GIVEN, INIT_NNDSVD, INIT_LEARNED, INIT_CLUSTER = 0, 1, 2, 3
RECON_MBIR, RECON_FBP = 0, 1
SNR_FMD, SNR_FHR, ROI_BACKGROUND = 0, 1, 255
OK, ERR_ARG, ERR_CUDA, ERR_TIMEOUT, ERR_NONFINITE, ERR_UNSUPPORTED = 0, -1, -2, -3, -4, -5

# Every entry point declared in include/fhr.h (checked by the ABI test).
ENTRY_POINTS = (
    "fhr_create", "fhr_destroy", "fhr_set_stream", "fhr_last_error", "fhr_version", "fhr_workspace_status",
    "fhr_normalise", "fhr_decompose_workspace_size", "fhr_decompose", "fhr_projector_workspace_size",
    "fhr_project", "fhr_backproject", "fhr_reconstruct_workspace_size", "fhr_reconstruct", "fhr_expand",
    "fhr_pipeline_workspace_size", "fhr_pipeline", "fhr_profile_enable", "fhr_profile_read",
    "fhr_decompose_static", "fhr_decompose_static_status", "fhr_nmf_row_stride", "fhr_mlp_workspace_size", "fhr_mlp_forward", "fhr_mlp_grad", "fhr_mlp_adamw",
    "fhr_reconstruct_batch_workspace_size", "fhr_reconstruct_batch", "fhr_reconstruct_batch_autotune",
    "fhr_fbp_workspace_size", "fhr_fbp", "fhr_io_join", "fhr_fmd_workspace_size", "fhr_fmd",
    "fhr_snr_workspace_size", "fhr_snr",
)


class NormParams(ctypes.Structure):
    _fields_ = [("Nv", ctypes.c_int), ("Nr", ctypes.c_int), ("Nc", ctypes.c_int), ("Nk", ctypes.c_int),
                ("ldP", ctypes.c_int), ("p_dtype", ctypes.c_int), ("dead_per_pixel", ctypes.c_int)]


class NmfParams(ctypes.Structure):
    _fields_ = [("Np", ctypes.c_int64), ("Nk", ctypes.c_int), ("ldP", ctypes.c_int), ("K", ctypes.c_int),
                ("iters", ctypes.c_int), ("init", ctypes.c_int), ("p_dtype", ctypes.c_int),
                ("power_iters", ctypes.c_int), ("seed", ctypes.c_uint64), ("mlp", ctypes.c_void_p),
                ("mlp_params", ctypes.c_void_p), ("kmeans_samples", ctypes.c_int64), ("kmeans_iters", ctypes.c_int)]


class Geom(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("Nr", ctypes.c_int), ("Nc", ctypes.c_int), ("Nv", ctypes.c_int),
                ("angles", ctypes.c_void_p)]


class MbirParams(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int), ("iters", ctypes.c_int), ("p", ctypes.c_float), ("q", ctypes.c_float),
                ("T", ctypes.c_float), ("beta", ctypes.c_float), ("snr_db", ctypes.c_float),
                ("momentum", ctypes.c_int), ("sigma_v", ctypes.POINTER(ctypes.c_float)),
                ("sigma_x", ctypes.POINTER(ctypes.c_float))]


class Problem(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("Nr", ctypes.c_int), ("Nc", ctypes.c_int), ("Nv", ctypes.c_int),
                ("K", ctypes.c_int), ("angles", ctypes.c_void_p), ("sino", ctypes.c_void_p), ("xs", ctypes.c_void_p),
                ("sigma_v", ctypes.c_float * 8), ("sigma_x", ctypes.c_float * 8)]


class BatchParams(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("p", ctypes.c_float), ("q", ctypes.c_float), ("T", ctypes.c_float),
                ("beta", ctypes.c_float), ("snr_db", ctypes.c_float), ("momentum", ctypes.c_int),
                ("tile", ctypes.c_int), ("vw", ctypes.c_int)]


class MlpDims(ctypes.Structure):
    _fields_ = [("Nk", ctypes.c_int), ("H1", ctypes.c_int), ("H2", ctypes.c_int), ("K", ctypes.c_int),
                ("ldx", ctypes.c_int), ("x_dtype", ctypes.c_int), ("weights_bf16", ctypes.c_int)]


def mlp_nparams(Nk, H1, H2, K):
    return H1 * Nk + H1 + H2 * H1 + H2 + K * H2 + K


class PipelineParams(ctypes.Structure):
    _fields_ = [("norm", NormParams), ("nmf", NmfParams), ("geom", Geom), ("mbir", MbirParams),
                ("xh_dtype", ctypes.c_int), ("host_io", ctypes.c_int), ("recon", ctypes.c_int)]


_lib = None
_lock = threading.Lock()


def load():
    """Load libfhr.so from the package directory (build it first with build.build())."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libfhr.so is not built (run paper_2410_22500_gb300.build.build()); "
                               "there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        vp, sz = ctypes.c_void_p, ctypes.c_size_t
        szp = ctypes.POINTER(ctypes.c_size_t)
        L.fhr_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, vp]
        L.fhr_destroy.argtypes = [vp]
        L.fhr_destroy.restype = None
        L.fhr_set_stream.argtypes = [vp, vp]
        L.fhr_last_error.argtypes = [vp]
        L.fhr_last_error.restype = ctypes.c_char_p
        L.fhr_version.restype = ctypes.c_char_p
        L.fhr_workspace_status.argtypes = [vp, vp]
        L.fhr_normalise.argtypes = [vp, ctypes.POINTER(NormParams), vp, vp, vp, vp, vp, vp]
        L.fhr_decompose_workspace_size.argtypes = [vp, ctypes.POINTER(NmfParams), szp]
        L.fhr_decompose.argtypes = [vp, ctypes.POINTER(NmfParams), vp, vp, vp, vp, vp, sz]
        L.fhr_projector_workspace_size.argtypes = [vp, ctypes.POINTER(Geom), szp]
        L.fhr_project.argtypes = [vp, ctypes.POINTER(Geom), ctypes.c_int, vp, vp, vp, sz]
        L.fhr_backproject.argtypes = [vp, ctypes.POINTER(Geom), ctypes.c_int, vp, vp, vp, sz]
        L.fhr_reconstruct_workspace_size.argtypes = [vp, ctypes.POINTER(Geom), ctypes.POINTER(MbirParams), szp]
        L.fhr_reconstruct.argtypes = [vp, ctypes.POINTER(Geom), ctypes.POINTER(MbirParams), vp, vp, vp, sz]
        L.fhr_expand.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                 ctypes.c_int, vp, vp, ctypes.c_int, vp]
        L.fhr_pipeline_workspace_size.argtypes = [vp, ctypes.POINTER(PipelineParams), szp]
        L.fhr_pipeline.argtypes = [vp, ctypes.POINTER(PipelineParams), vp, vp, vp, vp, vp, vp, vp, vp, sz]
        L.fhr_decompose_static.argtypes = [vp, ctypes.POINTER(NmfParams), vp, vp, vp, vp]
        L.fhr_decompose_static_status.argtypes = [vp]
        L.fhr_nmf_row_stride.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
        L.fhr_mlp_workspace_size.argtypes = [vp, ctypes.POINTER(MlpDims), ctypes.c_int, szp]
        L.fhr_mlp_forward.argtypes = [vp, ctypes.POINTER(MlpDims), vp, ctypes.c_int64, vp, vp, vp, sz]
        L.fhr_mlp_grad.argtypes = [vp, ctypes.POINTER(MlpDims), vp, ctypes.c_int64, vp, vp, vp, vp, vp, sz]
        L.fhr_mlp_adamw.argtypes = [vp, ctypes.c_int64, vp, vp, vp, vp, ctypes.c_int] + [ctypes.c_float] * 5
        PP, BP = ctypes.POINTER(Problem), ctypes.POINTER(BatchParams)
        L.fhr_reconstruct_batch_workspace_size.argtypes = [vp, ctypes.c_int, PP, BP, szp]
        L.fhr_reconstruct_batch.argtypes = [vp, ctypes.c_int, PP, BP, vp, sz]
        L.fhr_reconstruct_batch_autotune.argtypes = [vp, ctypes.c_int, PP, BP, vp, sz, ctypes.POINTER(ctypes.c_int),
                                                     ctypes.POINTER(ctypes.c_int)]
        L.fhr_io_join.argtypes = [vp]
        L.fhr_fmd_workspace_size.argtypes = [vp, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int, szp]
        L.fhr_fmd.argtypes = [vp, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int] + [vp] * 7 + [sz]
        L.fhr_snr_workspace_size.argtypes = [vp, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int, szp]
        L.fhr_snr.argtypes = [vp, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp, vp, vp, sz]
        L.fhr_fbp_workspace_size.argtypes = [vp, ctypes.POINTER(Geom), ctypes.c_int, szp]
        L.fhr_fbp.argtypes = [vp, ctypes.POINTER(Geom), ctypes.c_int, vp, vp, vp, sz]
        L.fhr_profile_enable.argtypes = [vp, ctypes.c_int]
        L.fhr_profile_read.argtypes = [vp, ctypes.c_char_p, ctypes.POINTER(ctypes.c_longlong),
                                       ctypes.POINTER(ctypes.c_double)]
        _lib = L
        return L


def nmf_row_stride(Nk, p_dtype=F32):
    """fhr_nmf_row_stride: the row stride of P that the fused NMF pass streams fastest."""
    L = load()
    out = ctypes.c_int()
    rc = L.fhr_nmf_row_stride(int(Nk), int(p_dtype), ctypes.byref(out))
    if rc != OK:
        raise FhrError(rc, "fhr_nmf_row_stride(%d, %d)" % (Nk, p_dtype))
    return out.value


class FhrError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("libfhr error %d: %s" % (code, msg))
        self.code = code


def _torch():
    import torch

    return torch


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class Context:
    """A libfhr context bound to one device and (by default) torch's current stream."""

    def __init__(self, device: int = 0, stream=None):
        torch = _torch()
        self.L = load()
        self.device = device
        self._h = ctypes.c_void_p()
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        rc = self.L.fhr_create(ctypes.byref(self._h), device, ctypes.c_void_p(self.stream.cuda_stream))
        if rc != OK:
            raise FhrError(rc, "fhr_create failed (no CUDA device of compute capability 10.x?)")

    def close(self):
        if self._h:
            self.L.fhr_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, rc):
        if rc != OK:
            raise FhrError(rc, self.L.fhr_last_error(self._h).decode())

    def set_stream(self, stream):
        self.stream = stream
        self.check(self.L.fhr_set_stream(self._h, ctypes.c_void_p(stream.cuda_stream)))

    def profile(self, enable=True):
        """Reset launch counters; with enable, time the kernel families with CUDA events."""
        self.check(self.L.fhr_profile_enable(self._h, int(enable)))

    def profile_read(self, name=None):
        """(launches, total ms) of a kernel family, or (total launches, 0) with name=None."""
        n, ms = ctypes.c_longlong(), ctypes.c_double()
        self.check(self.L.fhr_profile_read(self._h, None if name is None else name.encode(), ctypes.byref(n),
                                           ctypes.byref(ms)))
        return n.value, ms.value

    def workspace(self, nbytes):
        torch = _torch()
        return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device="cuda:%d" % self.device)

    def status(self, ws):
        """Synchronise the stream and return (and clear) the workspace status word."""
        rc = self.L.fhr_workspace_status(self._h, _ptr(ws))
        return rc

    # ------------------------------------------------------------ normalise
    def normalise(self, y, y0, *, ldP=None, p_dtype=F32, bg=None, dead=None, P=None, b=None):
        """Eq. (neglogattenuation) + Appendix A offset: counts -> P [Np][ldP].  dead: [Nk] dead
        bins or [Nr][Nc][Nk] dead detector pixel-bins (uint8)."""
        torch = _torch()
        Nv, Nr, Nc, Nk = y.shape
        mult = 8 if p_dtype == BF16 else 4
        ldP = ldP or (Nk + mult - 1) // mult * mult
        if P is None:
            P = torch.empty((Nv * Nc * Nr, ldP), dtype=torch.bfloat16 if p_dtype == BF16 else torch.float32,
                            device=y.device)
        if bg is not None and b is None:
            b = torch.empty((Nv, Nk), dtype=torch.float32, device=y.device)
        prm = NormParams(Nv, Nr, Nc, Nk, ldP, p_dtype, int(dead is not None and dead.dim() == 3))
        self.check(self.L.fhr_normalise(self._h, ctypes.byref(prm), _ptr(y), _ptr(y0), _ptr(bg), _ptr(dead),
                                        _ptr(b), _ptr(P)))
        return (P, b) if bg is not None else P

    # ------------------------------------------------------------ decompose
    def nmf_params(self, P, Nk, K, iters, init=INIT_GIVEN, power_iters=0, seed=0, mlp=None, kmeans_samples=0,
                   kmeans_iters=0):
        torch = _torch()
        prm = NmfParams(P.shape[0], Nk, P.shape[1], K, iters, init,
                        BF16 if P.dtype == torch.bfloat16 else F32, power_iters, seed)
        prm.kmeans_samples = kmeans_samples
        prm.kmeans_iters = kmeans_iters
        if mlp is not None:
            dims, params = mlp
            prm.mlp = ctypes.addressof(dims)
            prm.mlp_params = params.data_ptr()
            prm._keep = (dims, params)
        return prm

    def decompose(self, P, Nk, K, iters, *, D=None, W=None, init=None, power_iters=0, seed=0, obj=True,
                  check_status=True, mlp=None, kmeans_samples=0, kmeans_iters=0):
        """Fast-HALS NMF of P (Sec. III).  D [Nk][K], W [Np][K] updated in place (GIVEN) or filled
        (NNDSVD, CLUSTER, LEARNED)."""
        torch = _torch()
        dev = P.device
        if init is None:
            init = INIT_GIVEN if D is not None else INIT_NNDSVD
        if D is None:
            D = torch.zeros((Nk, K), dtype=torch.float32, device=dev)
        if W is None:
            W = torch.zeros((P.shape[0], K), dtype=torch.float32, device=dev)
        if mlp is not None:
            init = INIT_LEARNED
        prm = self.nmf_params(P, Nk, K, iters, init, power_iters, seed, mlp, kmeans_samples, kmeans_iters)
        n = ctypes.c_size_t()
        self.check(self.L.fhr_decompose_workspace_size(self._h, ctypes.byref(prm), ctypes.byref(n)))
        ws = self.workspace(n.value)
        ob = torch.empty(max(iters, 1), dtype=torch.float64, device=dev) if obj else None
        self.check(self.L.fhr_decompose(self._h, ctypes.byref(prm), _ptr(P), _ptr(D), _ptr(W), _ptr(ob), _ptr(ws),
                                        n.value))
        if check_status:
            self.check(self.status(ws))
        return D, W, (ob[:iters] if obj else None)

    # ------------------------------------------------------------ projector
    @staticmethod
    def geom(N, Nr, Nc, Nv, angles=None):
        return Geom(N, Nr, Nc, Nv, None if angles is None else angles.data_ptr())

    def project(self, x, Nc, Nv, *, angles=None, y=None):
        """y = A x for x [N][N][Wl] -> y [Nv][Nc][Wl] (strip-area model)."""
        torch = _torch()
        N, Wl = x.shape[0], x.shape[2]
        g = self.geom(N, 1, Nc, Nv, angles)
        n = ctypes.c_size_t()
        self.check(self.L.fhr_projector_workspace_size(self._h, ctypes.byref(g), ctypes.byref(n)))
        ws = self.workspace(n.value)
        if y is None:
            y = torch.empty((Nv, Nc, Wl), dtype=torch.float32, device=x.device)
        self.check(self.L.fhr_project(self._h, ctypes.byref(g), Wl, _ptr(x), _ptr(y), _ptr(ws), n.value))
        return y

    def backproject(self, y, N, *, angles=None, x=None):
        """x = A^T y for y [Nv][Nc][Wl] -> x [N][N][Wl]."""
        torch = _torch()
        Nv, Nc, Wl = y.shape
        g = self.geom(N, 1, Nc, Nv, angles)
        n = ctypes.c_size_t()
        self.check(self.L.fhr_projector_workspace_size(self._h, ctypes.byref(g), ctypes.byref(n)))
        ws = self.workspace(n.value)
        if x is None:
            x = torch.empty((N, N, Wl), dtype=torch.float32, device=y.device)
        self.check(self.L.fhr_backproject(self._h, ctypes.byref(g), Wl, _ptr(y), _ptr(x), _ptr(ws), n.value))
        return x

    # ------------------------------------------------------------ reconstruct
    @staticmethod
    def mbir_params(K, iters, p=1.2, q=2.0, T=1.0, beta=1.0, snr_db=30.0, momentum=False, sigma_v=None,
                    sigma_x=None):
        keep = []
        sv = sx = None
        if sigma_v is not None and sigma_x is not None:
            sv = (ctypes.c_float * K)(*[float(v) for v in sigma_v])
            sx = (ctypes.c_float * K)(*[float(v) for v in sigma_x])
            keep = [sv, sx]
        prm = MbirParams(K, iters, p, q, T, beta, snr_db, int(momentum),
                         ctypes.cast(sv, ctypes.POINTER(ctypes.c_float)) if sv is not None else None,
                         ctypes.cast(sx, ctypes.POINTER(ctypes.c_float)) if sx is not None else None)
        prm._keep = keep
        return prm

    def reconstruct(self, sino, N, Nr, K, iters, *, angles=None, xs=None, check_status=True, **kw):
        """SQS solve of Eq. (recon): sino [Nv][Nc][Nr*K] -> xs [N][N][Nr*K]."""
        torch = _torch()
        Nv, Nc = sino.shape[0], sino.shape[1]
        g = self.geom(N, Nr, Nc, Nv, angles)
        prm = self.mbir_params(K, iters, **kw)
        n = ctypes.c_size_t()
        self.check(self.L.fhr_reconstruct_workspace_size(self._h, ctypes.byref(g), ctypes.byref(prm),
                                                         ctypes.byref(n)))
        ws = self.workspace(n.value)
        if xs is None:
            xs = torch.zeros((N, N, Nr * K), dtype=torch.float32, device=sino.device)
        self.check(self.L.fhr_reconstruct(self._h, ctypes.byref(g), ctypes.byref(prm), _ptr(sino), _ptr(xs),
                                          _ptr(ws), n.value))
        if check_status:
            self.check(self.status(ws))
        return xs

    # ------------------------------------------------------------ FBP variant
    def fbp(self, sino, N, *, angles=None, xs=None):
        """Filtered back-projection: sino [Nv][Nc][Wl] -> xs [N][N][Wl]."""
        torch = _torch()
        Nv, Nc, Wl = sino.shape
        g = self.geom(N, 1, Nc, Nv, angles)
        n = ctypes.c_size_t()
        self.check(self.L.fhr_fbp_workspace_size(self._h, ctypes.byref(g), Wl, ctypes.byref(n)))
        ws = self.workspace(n.value)
        if xs is None:
            xs = torch.empty((N, N, Wl), dtype=torch.float32, device=sino.device)
        self.check(self.L.fhr_fbp(self._h, ctypes.byref(g), Wl, _ptr(sino), _ptr(xs), _ptr(ws), n.value))
        return xs

    # ------------------------------------------------------------ material decomposition (Algorithm 2)
    def fmd(self, xs, labels, D, Nm, *, check_status=True):
        """Semi-supervised FMD: xs [Nx][Ns] (or [N][N][Nr*Ns] viewed so), labels [Nx] u8,
        D [Nk][Ns] -> (T [Nm][Ns], xm [Nx][Nm], Dm [Nk][Nm])."""
        torch = _torch()
        Nk, Ns = D.shape
        xs2 = xs.reshape(-1, Ns)
        Nx = xs2.shape[0]
        n = ctypes.c_size_t()
        self.check(self.L.fhr_fmd_workspace_size(self._h, Nx, Ns, Nm, Nk, ctypes.byref(n)))
        ws = self.workspace(n.value)
        T = torch.empty((Nm, Ns), dtype=torch.float32, device=D.device)
        xm = torch.empty((Nx, Nm), dtype=torch.float32, device=D.device)
        Dm = torch.empty((Nk, Nm), dtype=torch.float32, device=D.device)
        self.check(self.L.fhr_fmd(self._h, Nx, Ns, Nm, Nk, _ptr(xs2), _ptr(labels), _ptr(D), _ptr(T), _ptr(xm),
                                  _ptr(Dm), _ptr(ws), n.value))
        if check_status:
            self.check(self.status(ws))
        return T, xm, Dm

    # ------------------------------------------------------------ SNR (Sec. V-B)
    def snr(self, x, roi, Nm, mode, *, check_status=True):
        """Eq. (snr_fmd) (mode SNR_FMD) or Eq. (snr_fhr) (mode SNR_FHR) in dB, as a device double.
        x [Nx][C] f32 (any shape whose last axis is C), roi [Nx] u8 (0 none, m + 1 material m,
        ROI_BACKGROUND background)."""
        torch = _torch()
        C = x.shape[-1]
        x2 = x.reshape(-1, C)
        Nx = x2.shape[0]
        n = ctypes.c_size_t()
        self.check(self.L.fhr_snr_workspace_size(self._h, Nx, C, Nm, mode, ctypes.byref(n)))
        ws = self.workspace(n.value)
        out = torch.empty(1, dtype=torch.float64, device=x.device)
        self.check(self.L.fhr_snr(self._h, Nx, C, Nm, mode, _ptr(x2), _ptr(roi), _ptr(out), _ptr(ws), n.value))
        if check_status:
            self.check(self.status(ws))
        return out

    # ------------------------------------------------------------ batched MBIR
    @staticmethod
    def batch_problems(sinos, Ns, Ks, xss, *, Nr=1, angles=None, sigmas=None):
        """Problem array for fhr_reconstruct_batch; sinos[i] [Nv][Nc][Nr*K] and
        xss[i] [N][N][Nr*K] are device tensors, Nr an int or one per problem,
        sigmas[i] = (sigma_v, sigma_x) or None."""
        n = len(sinos)
        Nrs = list(Nr) if isinstance(Nr, (list, tuple)) else [Nr] * n
        arr = (Problem * n)()
        for i in range(n):
            s = sinos[i]
            arr[i].N, arr[i].Nr, arr[i].Nc, arr[i].Nv, arr[i].K = Ns[i], Nrs[i], s.shape[1], s.shape[0], Ks[i]
            arr[i].angles = None if angles is None or angles[i] is None else angles[i].data_ptr()
            arr[i].sino = s.data_ptr()
            arr[i].xs = xss[i].data_ptr()
            if sigmas is not None and sigmas[i] is not None:
                for j in range(Ks[i]):
                    arr[i].sigma_v[j] = float(sigmas[i][0][j])
                    arr[i].sigma_x[j] = float(sigmas[i][1][j])
        return arr

    @staticmethod
    def batch_params(iters, p=1.2, q=2.0, T=1.0, beta=1.0, snr_db=30.0, momentum=False, tile=0, vw=0):
        return BatchParams(iters, p, q, T, beta, snr_db, int(momentum), tile, vw)

    def reconstruct_batch(self, sinos, Ns, Ks, iters, *, Nr=1, xss=None, angles=None, sigmas=None, tile=0, vw=0,
                          autotune=False, check_status=True, **kw):
        """Eq. (recon) for every problem of the batch in one persistent launch.
        Returns (xss, tile, vw): the work-item size and the values per thread used
        (vw 0: the widest each problem takes)."""
        torch = _torch()
        Nrs = list(Nr) if isinstance(Nr, (list, tuple)) else [Nr] * len(sinos)
        if xss is None:
            xss = [torch.zeros((N, N, r * K), dtype=torch.float32, device=s.device)
                   for s, N, K, r in zip(sinos, Ns, Ks, Nrs)]
        arr = self.batch_problems(sinos, Ns, Ks, xss, Nr=Nr, angles=angles, sigmas=sigmas)
        prm = self.batch_params(iters, tile=tile, vw=vw, **kw)
        n = ctypes.c_size_t()
        self.check(self.L.fhr_reconstruct_batch_workspace_size(self._h, len(sinos), arr, ctypes.byref(prm),
                                                               ctypes.byref(n)))
        ws = self.workspace(n.value)
        if autotune:
            best, best_vw = ctypes.c_int(), ctypes.c_int()
            self.check(self.L.fhr_reconstruct_batch_autotune(self._h, len(sinos), arr, ctypes.byref(prm), _ptr(ws),
                                                             n.value, ctypes.byref(best), ctypes.byref(best_vw)))
            if check_status:
                self.check(self.status(ws))
            prm.tile, prm.vw = best.value, best_vw.value
        self.check(self.L.fhr_reconstruct_batch(self._h, len(sinos), arr, ctypes.byref(prm), _ptr(ws), n.value))
        if check_status:
            self.check(self.status(ws))
        return xss, (prm.tile or 2), prm.vw

    # ------------------------------------------------------------ expand
    def expand(self, xs, D, N, Nr, *, k0=0, k1=0, xh_dtype=F32, xh=None):
        """Eq. (sub_expansion): xs [N][N][Nr*K], D [Nk][K] -> xh [Nr][N][N][k1-k0]."""
        torch = _torch()
        Nk, K = D.shape
        nk = (k1 - k0) if (k0 or k1) else Nk
        if xh is None:
            xh = torch.empty((Nr, N, N, nk), dtype=torch.bfloat16 if xh_dtype == BF16 else torch.float32,
                             device=xs.device)
        self.check(self.L.fhr_expand(self._h, N, Nr, K, Nk, k0, k1, _ptr(xs), _ptr(D), xh_dtype, _ptr(xh)))
        return xh

    # ------------------------------------------------------------ learned warm start (MLP)
    @staticmethod
    def mlp_dims(Nk, H1, H2, K, *, ldx=None, x_bf16=False, weights_bf16=False):
        return MlpDims(Nk, H1, H2, K, ldx or Nk, BF16 if x_bf16 else F32, int(weights_bf16))

    def mlp_forward(self, dims, params, X, *, Y=None, ws=None):
        """Y [M][K] = MLP(X), X [M][ldx] (f32 or bf16), params packed f32."""
        torch = _torch()
        M = X.shape[0]
        if ws is None:
            n = ctypes.c_size_t()
            self.check(self.L.fhr_mlp_workspace_size(self._h, ctypes.byref(dims), 0, ctypes.byref(n)))
            ws = self.workspace(n.value)
        if Y is None:
            Y = torch.empty((M, dims.K), dtype=torch.float32, device=X.device)
        self.check(self.L.fhr_mlp_forward(self._h, ctypes.byref(dims), _ptr(params), M, _ptr(X), _ptr(Y), _ptr(ws),
                                          ws.numel()))
        return Y

    def mlp_grad(self, dims, params, X, T, *, grad=None, loss=None, ws=None):
        """(loss, grad) of the mean-squared error of MLP(X) against T; up to 32768 rows."""
        torch = _torch()
        if ws is None:
            n = ctypes.c_size_t()
            self.check(self.L.fhr_mlp_workspace_size(self._h, ctypes.byref(dims), 1, ctypes.byref(n)))
            ws = self.workspace(n.value)
        if grad is None:
            grad = torch.empty_like(params)
        if loss is None:
            loss = torch.empty(1, dtype=torch.float64, device=X.device)
        self.check(self.L.fhr_mlp_grad(self._h, ctypes.byref(dims), _ptr(params), X.shape[0], _ptr(X), _ptr(T),
                                       _ptr(grad), _ptr(loss), _ptr(ws), ws.numel()))
        return loss, grad

    def mlp_adamw(self, params, grad, m, v, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8, wd=1e-4):
        self.check(self.L.fhr_mlp_adamw(self._h, params.numel(), _ptr(params), _ptr(grad), _ptr(m), _ptr(v), step,
                                        lr, b1, b2, eps, wd))

    # ------------------------------------------------------------ pipeline
    def pipeline_params(self, *, Nv, Nr, Nc, Nk, N, K, nmf_iters, mbir_iters, p_dtype=F32, xh_dtype=F32,
                        host_io=False, power_iters=0, seed=0, angles=None, init=INIT_NNDSVD, kmeans_samples=0,
                        kmeans_iters=0, recon=RECON_MBIR, dead_per_pixel=False, **mbir_kw):
        ldP = nmf_row_stride(Nk, p_dtype)
        prm = PipelineParams()
        prm.norm = NormParams(Nv, Nr, Nc, Nk, ldP, p_dtype, int(dead_per_pixel))
        prm.nmf = NmfParams(Nv * Nr * Nc, Nk, ldP, K, nmf_iters, init, p_dtype, power_iters, seed, None, None,
                            kmeans_samples, kmeans_iters)
        prm.geom = self.geom(N, Nr, Nc, Nv, angles)
        mp = self.mbir_params(K, mbir_iters, **mbir_kw)
        prm.mbir = mp
        prm._keep = mp._keep
        prm.xh_dtype = xh_dtype
        prm.host_io = int(host_io)
        prm.recon = recon
        return prm

    def io_join(self):
        """Order the context stream after the last host-I/O output copy."""
        self.check(self.L.fhr_io_join(self._h))

    def pipeline_workspace(self, prm):
        n = ctypes.c_size_t()
        self.check(self.L.fhr_pipeline_workspace_size(self._h, ctypes.byref(prm), ctypes.byref(n)))
        return self.workspace(n.value), n.value

    def pipeline(self, prm, y, y0, D, xh, *, obj=None, dead=None, bg=None, ws=None, ws_bytes=None):
        """Algorithm 1: counts -> (D, x^h).  With prm.host_io, y, y0 and xh are pinned host tensors."""
        if ws is None:
            ws, ws_bytes = self.pipeline_workspace(prm)
        self.check(self.L.fhr_pipeline(self._h, ctypes.byref(prm), _ptr(y), _ptr(y0), _ptr(bg), _ptr(dead), _ptr(D),
                                       _ptr(xh), _ptr(obj), _ptr(ws), ws_bytes))
        return ws
