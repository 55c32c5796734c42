"""Seeded synthetic hyperspectral neutron-CT inputs.

This module only *draws inputs*: phantoms, attenuation spectra, analytic line
integrals and Poisson counts.  It holds none of the reconstruction method's
arithmetic (no normalisation, no factorisation, no discrete projector, no
iterative reconstruction), so both the FP64 oracle and the CUDA path can take
their inputs from it without sharing any computation.

Physics it follows (paper Sec. II and Sec. V-A):
  * the object is a set of non-overlapping homogeneous materials (volume
    fraction 1 inside, 0 outside), each with a wavelength-dependent linear
    attenuation spectrum mu_m(lambda) (the dictionary D^m of Eq. porj_matd_rel);
  * the noise-free projection is p = (A x^m)(D^m)^T, where here A x^m is the
    *analytic* parallel-beam line integral of each material's shape (exact
    chord lengths of disks / ellipse slices), not the discrete strip model;
  * counts follow Eq. neutroncounts, y = y^o exp(-p), with y and y^o drawn
    from Poisson distributions (Sec. V-A).

Geometry conventions (shared with the rest of the library, stated here so a
reader can check them): an N x N image with unit pixels centred on the
origin, pixel (iy, ix) centred at (ix - (N-1)/2, iy - (N-1)/2); Nc detector
bins of unit width centred at u_c = c - (Nc-1)/2; view angles
theta_v = v * pi / Nv (parallel beam over 180 degrees); detector row r sees
volume slice r, slice centre z_r = r - (Nr-1)/2.

Layouts: counts y are [Nv][Nr][Nc][Nk] (uint16), the open beam y0 is
[Nr][Nc][Nk] (uint16), chords are [Nv][Nr][Nc][Nm] (detector order).
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

LAMBDA_MIN = 1.5  # Angstrom, Sec. V-A
LAMBDA_MAX = 4.5


@dataclass
class Geometry:
    """Parallel-beam acquisition geometry."""

    N: int          # image side (pixels)
    Nr: int         # detector rows == volume slices
    Nc: int         # detector columns (bins)
    Nv: int         # views over 180 degrees

    def angles(self) -> np.ndarray:
        return np.arange(self.Nv, dtype=np.float64) * (math.pi / self.Nv)

    @property
    def Np(self) -> int:
        return self.Nv * self.Nr * self.Nc

    @property
    def Nx(self) -> int:
        return self.Nr * self.N * self.N


@dataclass
class Phantom:
    """Material shapes: ellipsoids (cx, cy, cz, ax, ay, az, phi), one per material.

    A disk is an ellipsoid with ax == ay and az = inf (2-D problems)."""

    shapes: np.ndarray  # [Nm][7]

    @property
    def Nm(self) -> int:
        return int(self.shapes.shape[0])


@dataclass
class Problem:
    geom: Geometry
    Nk: int
    phantom: Phantom
    spectra: np.ndarray          # [Nk][Nm] attenuation per unit length
    I0: float                    # open-beam mean counts per bin
    dead_bins: np.ndarray        # [Nk] uint8, 1 = dead wavelength bin
    seed: int
    extra: dict = field(default_factory=dict)


def wavelengths(Nk: int) -> np.ndarray:
    """Bin-centre wavelengths, uniform on [1.5, 4.5] Angstrom (Sec. V-A)."""
    edges = np.linspace(LAMBDA_MIN, LAMBDA_MAX, Nk + 1)
    return 0.5 * (edges[:-1] + edges[1:])


def material_spectra(rng: np.random.Generator, Nm: int, lam: np.ndarray) -> np.ndarray:
    """Smooth 1/lambda-like spectra with 2-4 step-down Bragg-like edges each.

    mu_m(lambda) = (a_m + b_m / lambda) * prod_{e: lambda > lambda_e} (1 - delta_e).
    Returned unscaled, shape [Nk][Nm]."""
    out = np.empty((lam.size, Nm), dtype=np.float64)
    for m in range(Nm):
        a = rng.uniform(0.3, 1.0)
        b = rng.uniform(0.5, 2.0)
        ne = int(rng.integers(2, 5))
        edges = rng.uniform(1.7, 4.3, size=ne)
        drops = rng.uniform(0.1, 0.4, size=ne)
        mu = a + b / lam
        for le, de in zip(edges, drops):
            mu = np.where(lam > le, mu * (1.0 - de), mu)
        out[:, m] = mu
    return out


def _nonoverlapping(rng, n_obj, sample, overlaps, tries=20000):
    objs = []
    for _ in range(tries):
        if len(objs) == n_obj:
            break
        cand = sample()
        if all(not overlaps(cand, o) for o in objs):
            objs.append(cand)
    if len(objs) != n_obj:
        raise RuntimeError("could not place non-overlapping shapes; enlarge the image")
    return objs


def disk_phantom(rng: np.random.Generator, N: int, Nm: int) -> Phantom:
    """Nm non-overlapping disks inside the inscribed circle of an N x N image."""
    R = 0.5 * N - 1.0
    rmin, rmax = 0.06 * N, 0.16 * N

    def sample():
        r = rng.uniform(rmin, rmax)
        rho = rng.uniform(0.0, R - r)
        ang = rng.uniform(0, 2 * math.pi)
        return (rho * math.cos(ang), rho * math.sin(ang), r)

    def overlaps(a, b):
        return math.hypot(a[0] - b[0], a[1] - b[1]) < a[2] + b[2] + 1.0

    disks = _nonoverlapping(rng, Nm, sample, overlaps)
    shapes = np.array([[cx, cy, 0.0, r, r, np.inf, 0.0] for cx, cy, r in disks])
    return Phantom(shapes)


def ellipsoid_phantom(rng: np.random.Generator, N: int, Nz: int, Nm: int) -> Phantom:
    """Nm non-overlapping ellipsoids inside the inscribed cylinder of an N x N x Nz volume.

    Overlap is tested conservatively with bounding spheres."""
    R = 0.5 * N - 1.0
    H = 0.5 * Nz - 1.0

    def sample():
        ax = rng.uniform(0.06, 0.16) * N
        ay = rng.uniform(0.06, 0.16) * N
        az = rng.uniform(0.25, 0.45) * Nz
        rb = max(ax, ay)
        rho = rng.uniform(0.0, max(R - rb, 0.0))
        ang = rng.uniform(0, 2 * math.pi)
        cz = rng.uniform(-max(H - az, 0.0), max(H - az, 0.0))
        phi = rng.uniform(0, math.pi)
        return (rho * math.cos(ang), rho * math.sin(ang), cz, ax, ay, az, phi)

    def overlaps(a, b):
        # in-plane bounding circles; slabs overlapping in z
        rin = math.hypot(a[0] - b[0], a[1] - b[1]) < max(a[3], a[4]) + max(b[3], b[4]) + 1.0
        zin = abs(a[2] - b[2]) < a[5] + b[5]
        return rin and zin

    return Phantom(np.array(_nonoverlapping(rng, Nm, sample, overlaps)))


def slice_ellipses(ph: Phantom, z: float):
    """Semi-axes of each material's cross-section at height z: (cx, cy, A, B, phi) or None."""
    out = []
    for cx, cy, cz, ax, ay, az, phi in ph.shapes:
        if np.isinf(az):
            s = 1.0
        else:
            t = 1.0 - ((z - cz) / az) ** 2
            if t <= 0:
                out.append(None)
                continue
            s = math.sqrt(t)
        out.append((cx, cy, ax * s, ay * s, phi))
    return out


def chords(ph: Phantom, g: Geometry, sub: int = 8) -> np.ndarray:
    """Exact line integrals of each material's indicator, [Nv][Nr][Nc][Nm].

    For an ellipse with semi-axes (A, B) rotated by phi and centred at
    (cx, cy), the chord at angle theta and detector offset u is
    2 A B sqrt(s^2 - u'^2) / s^2 with s^2 = A^2 cos^2(theta-phi) + B^2 sin^2(theta-phi)
    and u' = u - (cx cos theta + cy sin theta); zero when |u'| >= s.  Each
    detector bin reports the mean over `sub` equally spaced offsets across its
    unit width (a finite-width bin)."""
    th = g.angles()
    off = (np.arange(sub) + 0.5) / sub - 0.5
    uc = (np.arange(g.Nc, dtype=np.float64) - 0.5 * (g.Nc - 1))[:, None] + off[None, :]   # [Nc][sub]
    out = np.zeros((g.Nv, g.Nr, g.Nc, ph.Nm), dtype=np.float64)
    for r in range(g.Nr):
        z = r - 0.5 * (g.Nr - 1)
        for m, e in enumerate(slice_ellipses(ph, z)):
            if e is None:
                continue
            cx, cy, A, B, phi = e
            al = th - phi
            s2 = ((A * np.cos(al)) ** 2 + (B * np.sin(al)) ** 2)[:, None, None]          # [Nv][1][1]
            up = uc[None] - (cx * np.cos(th) + cy * np.sin(th))[:, None, None]           # [Nv][Nc][sub]
            d = s2 - up * up
            ch = np.where(d > 0, 2.0 * A * B * np.sqrt(np.maximum(d, 0)) / s2, 0.0)
            out[:, r, :, m] = ch.mean(axis=2)
    return out


def chords_torch(ph: Phantom, g: Geometry, device="cuda", sub: int = 8):
    """chords() evaluated with torch on `device` (FP64, the same formula and bin
    averaging), for drawing many phantoms quickly.  Returns [Nv][Nr][Nc][Nm]."""
    import torch

    f64 = torch.float64
    th = torch.from_numpy(g.angles()).to(device, f64)
    off = (torch.arange(sub, device=device, dtype=f64) + 0.5) / sub - 0.5
    uc = (torch.arange(g.Nc, device=device, dtype=f64) - 0.5 * (g.Nc - 1))[:, None] + off[None, :]
    out = torch.zeros((g.Nv, g.Nr, g.Nc, ph.Nm), dtype=f64, device=device)
    cth, sth = torch.cos(th), torch.sin(th)
    for r in range(g.Nr):
        z = r - 0.5 * (g.Nr - 1)
        for m, e in enumerate(slice_ellipses(ph, z)):
            if e is None:
                continue
            cx, cy, A, B, phi = e
            al = th - phi
            s2 = ((A * torch.cos(al)) ** 2 + (B * torch.sin(al)) ** 2)[:, None, None]
            up = uc[None] - (cx * cth + cy * sth)[:, None, None]
            d = s2 - up * up
            ch = torch.where(d > 0, 2.0 * A * B * torch.sqrt(torch.clamp(d, min=0)) / s2, torch.zeros_like(d))
            out[:, r, :, m] = ch.mean(dim=2)
    return out


def volume_fractions(ph: Phantom, N: int, Nr: int, sub: int = 4) -> np.ndarray:
    """Ground-truth volume fractions x^m, [Nr][N][N][Nm], by sub x sub supersampling."""
    o = (np.arange(sub) + 0.5) / sub - 0.5
    pix = np.arange(N) - 0.5 * (N - 1)
    X = (pix[None, :, None, None] + o[None, None, None, :])   # [1][N][1][sub]
    Y = (pix[:, None, None, None] + o[None, None, :, None])   # [N][1][sub][1]
    out = np.zeros((Nr, N, N, ph.Nm))
    for r in range(Nr):
        z = r - 0.5 * (Nr - 1)
        for m, e in enumerate(slice_ellipses(ph, z)):
            if e is None:
                continue
            cx, cy, A, B, phi = e
            dx, dy = X - cx, Y - cy
            xr = dx * math.cos(phi) + dy * math.sin(phi)
            yr = -dx * math.sin(phi) + dy * math.cos(phi)
            inside = (xr / A) ** 2 + (yr / B) ** 2 <= 1.0
            out[r, :, :, m] = inside.mean(axis=(2, 3))
    return out


def make_problem(*, N: int, Nr: int, Nc: int, Nv: int, Nk: int, Nm: int, I0: float,
                 seed: int, dead_frac: float = 0.0, peak_integral: float = 2.0,
                 three_d: bool | None = None, spectra: np.ndarray | None = None,
                 device: str | None = None) -> Problem:
    """Draw phantom, spectra and dead-bin mask; scale spectra so the largest
    noise-free line integral over all pixels and bins is about `peak_integral`.
    `spectra` [Nk][Nm] fixes the materials' spectral shapes (a shared library)."""
    rng = np.random.default_rng(seed)
    g = Geometry(N=N, Nr=Nr, Nc=Nc, Nv=Nv)
    if three_d is None:
        three_d = Nr > 1
    ph = ellipsoid_phantom(rng, N, Nr, Nm) if three_d else disk_phantom(rng, N, Nm)
    lam = wavelengths(Nk)
    mu = material_spectra(rng, Nm, lam) if spectra is None else np.array(spectra, dtype=np.float64, copy=True)
    if device is None:
        C = chords(ph, g).reshape(-1, Nm)
        bound = float((C * mu.max(axis=0)[None, :]).sum(axis=1).max())
    else:   # the same bound from the chords drawn on `device`
        import torch

        Ct = chords_torch(ph, g, device).reshape(-1, Nm)
        bound = float((Ct * torch.from_numpy(mu.max(axis=0)).to(Ct)[None, :]).sum(dim=1).max().item())
    mu *= peak_integral / max(bound, 1e-30)
    dead = np.zeros(Nk, dtype=np.uint8)
    if dead_frac > 0:
        nd = int(round(dead_frac * Nk))
        dead[rng.choice(Nk, size=nd, replace=False)] = 1
    pb = Problem(geom=g, Nk=Nk, phantom=ph, spectra=mu, I0=float(I0), dead_bins=dead, seed=seed)
    if device is not None:
        pb.extra["device"] = device
    return pb


def noise_free_projection(pb: Problem) -> np.ndarray:
    """p = (A x^m)(D^m)^T with the analytic A, [Nv][Nr][Nc][Nk] float64 (small cases)."""
    C = chords(pb.phantom, pb.geom)
    return C @ pb.spectra.T


def counts_numpy(pb: Problem, noise: bool = True):
    """Counts (y, y0) as uint16 numpy arrays, drawn on the host (small cases).

    y0 ~ Poisson(I0) per (r, c, k); y ~ Poisson(I0 exp(-p)) per (v, r, c, k);
    dead bins record zero counts in both.  noise=False gives rounded means."""
    rng = np.random.default_rng(pb.seed + 7919)
    g = pb.geom
    p = noise_free_projection(pb)
    lam_y = pb.I0 * np.exp(-p)
    if noise:
        y0 = rng.poisson(pb.I0, size=(g.Nr, g.Nc, pb.Nk))
        y = rng.poisson(lam_y)
    else:
        y0 = np.full((g.Nr, g.Nc, pb.Nk), round(pb.I0))
        y = np.rint(lam_y)
    y0 = np.minimum(y0, 65535).astype(np.uint16)
    y = np.minimum(y, 65535).astype(np.uint16)
    if pb.dead_bins.any():
        y0[..., pb.dead_bins.astype(bool)] = 0
        y[..., pb.dead_bins.astype(bool)] = 0
    return y, y0


def counts_torch(pb: Problem, device="cuda", chunk_views: int = 8):
    """Counts (y, y0) drawn on `device` (large cases), as int16 tensors holding
    the uint16 bit patterns (torch's uint16 support is partial; the library
    reads the bytes as uint16, and `.cpu().numpy().view(np.uint16)` recovers
    the counts on the host).

    Same distribution as counts_numpy; torch's seeded generator draws the
    Poisson samples view by view so peak memory stays bounded."""
    import torch

    g = pb.geom
    gen = torch.Generator(device=device)
    gen.manual_seed(pb.seed + 7919)
    if pb.extra.get("device") is not None:   # drawn with chords_torch
        C = chords_torch(pb.phantom, g, device).reshape(g.Nv, g.Nr * g.Nc, -1).to(torch.float32)
    else:
        C = torch.from_numpy(chords(pb.phantom, g).reshape(g.Nv, g.Nr * g.Nc, -1)).to(device, torch.float32)
    mu = torch.from_numpy(pb.spectra.T.copy()).to(device, torch.float32)   # [Nm][Nk]
    dead = torch.from_numpy(pb.dead_bins.astype(bool)).to(device)
    y = torch.empty((g.Nv, g.Nr, g.Nc, pb.Nk), dtype=torch.int16, device=device)
    yv = y.view(g.Nv, g.Nr * g.Nc, pb.Nk)
    for v0 in range(0, g.Nv, chunk_views):
        v1 = min(g.Nv, v0 + chunk_views)
        lam = pb.I0 * torch.exp(-(C[v0:v1] @ mu))
        s = torch.poisson(lam, generator=gen).clamp_(max=65535)
        s[..., dead] = 0
        yv[v0:v1] = s.to(torch.int32).to(torch.int16)
        del lam, s
    y0f = torch.poisson(torch.full((g.Nr, g.Nc, pb.Nk), pb.I0, device=device), generator=gen).clamp_(max=65535)
    y0f[..., dead] = 0
    y0 = y0f.to(torch.int32).to(torch.int16)
    return y, y0


# ---------------------------------------------------------------------------
# Named workloads (shapes of the paper's experiments, Table I, and of the five
# configurations this library is measured on).
# ---------------------------------------------------------------------------

def tiny_2d(seed: int = 1000) -> Problem:
    """32x32 image, 3 disks, Nk=128, 60 views over 180 deg, 48 bins, 1000 counts/bin."""
    return make_problem(N=32, Nr=1, Nc=48, Nv=60, Nk=128, Nm=3, I0=1000, seed=seed)


def volume_3d_f32(seed: int = 1001) -> Problem:
    """128x128x64 volume, 5 ellipsoids, Nk=1200, 90 views, 64x128 detector, 200 counts/bin, 4% dead bins."""
    return make_problem(N=128, Nr=64, Nc=128, Nv=90, Nk=1200, Nm=5, I0=200, seed=seed,
                        dead_frac=0.04)


def volume_3d_bf16(seed: int = 1002) -> Problem:
    """256^3 volume, 6 ellipsoids, Nk=1500, 120 views, 256x256 detector, 100 counts/bin."""
    return make_problem(N=256, Nr=256, Nc=256, Nv=120, Nk=1500, Nm=6, I0=100, seed=seed)


def batched_2d(n_problems: int = 40, seed0: int = 2000):
    """Uneven 2-D problems: N in 64..512 (step 16), 45..180 views, Nk 256..2000, K 3..8."""
    out = []
    for i in range(n_problems):
        rng = np.random.default_rng(seed0 + i)
        N = int(rng.integers(4, 33)) * 16
        Nv = int(rng.integers(45, 181))
        Nk = int(rng.integers(256, 2001))
        K = int(rng.integers(3, 9))
        pb = make_problem(N=N, Nr=1, Nc=N, Nv=Nv, Nk=Nk, Nm=K, I0=200, seed=seed0 + i)
        pb.extra["K"] = K
        out.append(pb)
    return out


def scaled(pb_fn, **over) -> Problem:
    """A workload with some sizes overridden (for fast parity cases)."""
    base = pb_fn()
    kw = dict(N=base.geom.N, Nr=base.geom.Nr, Nc=base.geom.Nc, Nv=base.geom.Nv, Nk=base.Nk,
              Nm=base.phantom.Nm, I0=base.I0, seed=base.seed,
              dead_frac=float(base.dead_bins.mean()))
    kw.update(over)
    return make_problem(**kw)


def spectra_library(Nk: int, Nm: int, seed: int = 77) -> np.ndarray:
    """One fixed set of Nm material spectra [Nk][Nm] shared by a family of phantoms."""
    return material_spectra(np.random.default_rng(seed), Nm, wavelengths(Nk))


def random_counts(rng: np.random.Generator, shape, lo=0, hi=2000) -> np.ndarray:
    """Uniform random uint16 counts (edge-case tests: zeros, y > y0, ...)."""
    return rng.integers(lo, hi, size=shape).astype(np.uint16)


def nmf_given_init(rng: np.random.Generator, Np: int, Nk: int, K: int):
    """A strictly positive random (D0, W0) pair for GIVEN-init parity runs."""
    D0 = rng.uniform(0.1, 1.0, size=(Nk, K))
    W0 = rng.uniform(0.1, 1.0, size=(Np, K))
    return D0, W0
