"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws inputs: probe modes, object slices, scan positions
and CBED-like diffraction patterns.  It holds none of the ptychography
method's arithmetic (no shift, no multislice, no loss, no adjoint) and
imports nothing else from this package, so that the FP64 oracle and the
CUDA path can share it without sharing any of the computation under test.

Recipes (arXiv 2505.14372 gives the experiment scale in §4.1 and §6; the
sizes below are the workload table of this library):
  * probe mode 0: P = F^-1[A(q) exp(-i chi(q))], hard aperture
    lambda |q| <= alpha, chi = pi lambda df |q|^2 + pi/2 C3 lambda^3 |q|^4,
    centred in the window, scaled so that sum |P|^2 = weight_0 * dose.
    Modes k >= 1: mode 0 times a smooth random amplitude/phase screen,
    Gram-Schmidt orthogonalised in float64, scaled to weight_k * dose.
  * object: exp(i sigma V) with V a sum of Gaussian atoms (sigma 0.4 A,
    peak 0.3 rad) at uniform random centres; multislice objects draw a
    depth for every atom and keep it in the slice it falls in.
  * scan: raster with a fixed step, uniform jitter of +-0.05 A, centred.
  * patterns: Poisson counts of a CBED-like intensity: the bright-field
    disc of the aperture plus a weak diffuse halo, modulated per position by
    a smooth random screen, at the stated dose.  They have the value
    distribution of measured data; they are not simulated by the forward
    model (tests that need self-consistent data simulate it themselves).
RNG: numpy PCG64 seeded with 1000 * config_id + role.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

ROLE_PROBE, ROLE_OBJECT, ROLE_SCAN, ROLE_NOISE, ROLE_GROUPS, ROLE_PATTERN = range(6)

WAVELENGTH_300KV = 0.0197  # Angstrom (relativistic, 300 kV)


@dataclass
class Workload:
    """One synthetic problem: geometry, scan, optics and data model."""
    cid: int
    name: str
    S: int
    K: int
    N: int            # square window h = w = N
    H: int
    W: int
    scan: tuple       # (ny, nx)
    step_px: float
    B: int            # minibatch size
    loss: int         # 0 amplitude, 1 Poisson
    eps: float
    c: float
    dose: float
    alpha_mrad: float
    defocus_A: float
    C3_A: float
    weights: tuple
    dz_A: float = 10.0
    dx: float = 0.1
    lam: float = WAVELENGTH_300KV
    bandlimit: float = 2.0 / 3.0
    atoms_per_slice: int = 200
    extra: dict = field(default_factory=dict)

    @property
    def P(self) -> int:
        return self.scan[0] * self.scan[1]

    @property
    def dz(self) -> tuple:
        return tuple([self.dz_A] * (self.S - 1))


def _mode_weights_exp(K):
    w = np.exp(-np.arange(K, dtype=np.float64))
    return tuple(w / w.sum())


WORKLOADS = {
    1: Workload(1, "single-slice single-mode 64x64 window, 128x128 object, 16x16 scan",
                S=1, K=1, N=64, H=128, W=128, scan=(16, 16), step_px=4.0, B=256,
                loss=0, eps=1e-3, c=0.0, dose=1e4, alpha_mrad=20.0,
                defocus_A=100.0, C3_A=0.0, weights=(1.0,), atoms_per_slice=200),
    2: Workload(2, "mixed-state single-slice 4 modes, 128x128 window, 512x512 object, 64x64 scan",
                S=1, K=4, N=128, H=512, W=512, scan=(64, 64), step_px=3.0, B=256,
                loss=1, eps=0.8, c=0.0, dose=5e4, alpha_mrad=24.0,
                defocus_A=50.0, C3_A=1e4, weights=(0.7, 0.15, 0.1, 0.05),
                atoms_per_slice=3200),
    3: Workload(3, "mixed-state multislice 20 slices x 8 modes, 192x192 window, 1024x1024 object, 128x128 scan",
                S=20, K=8, N=192, H=1024, W=1024, scan=(128, 128), step_px=6.0, B=512,
                loss=1, eps=0.8, c=0.0, dose=5e4, alpha_mrad=24.0,
                defocus_A=50.0, C3_A=1e4, weights=_mode_weights_exp(8),
                atoms_per_slice=1050),
}


# The multislice case the paper times its iterations on (80 x 80 scan, 20
# slices, 128 x 128 patterns; mode count and step not stated there: one mode,
# the 0.6 A step of workload 3), for quoting seconds per iteration beside the
# paper's own figure.  Not one of the benchmark workloads above.
PAPER_CONTEXT = Workload(6, "paper-shaped multislice: 20 slices, 1 mode, 128x128 window, 80x80 scan",
                         S=20, K=1, N=128, H=640, W=640, scan=(80, 80), step_px=6.0, B=512,
                         loss=1, eps=0.8, c=0.0, dose=5e4, alpha_mrad=24.0,
                         defocus_A=50.0, C3_A=1e4, weights=(1.0,), atoms_per_slice=410)


def rng_for(cid: int, role: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(1000 * int(cid) + int(role)))


def _freq(n):
    u = np.arange(n)
    return np.where(u < (n + 1) // 2, u, u - n)


def _smooth_field(rng, n, corr_px):
    """Zero-mean, unit-rms random field smoothed over ~corr_px pixels."""
    noise = rng.standard_normal((n, n))
    f = _freq(n) / n
    g = np.exp(-2.0 * (np.pi * corr_px) ** 2 * (f[:, None] ** 2 + f[None, :] ** 2))
    x = np.real(np.fft.ifft2(np.fft.fft2(noise) * g))
    x -= x.mean()
    return x / (x.std() + 1e-30)


def aperture_and_aberration(N, dx, lam, alpha_mrad, defocus_A, C3_A):
    q = _freq(N) / (N * dx)
    q2 = q[:, None] ** 2 + q[None, :] ** 2
    A = (lam * np.sqrt(q2) <= alpha_mrad * 1e-3).astype(np.float64)
    chi = np.pi * lam * defocus_A * q2 + 0.5 * np.pi * C3_A * lam ** 3 * q2 * q2
    return A, chi


def probe_modes(wl: Workload) -> np.ndarray:
    """complex64 [K, N, N] probe modes (see module docstring)."""
    rng = rng_for(wl.cid, ROLE_PROBE)
    N = wl.N
    A, chi = aperture_and_aberration(N, wl.dx, wl.lam, wl.alpha_mrad, wl.defocus_A, wl.C3_A)
    f = _freq(N)
    centre = np.exp(-1j * np.pi * (f[:, None] + f[None, :]))  # move to N/2, N/2
    p0 = np.fft.ifft2(A * np.exp(-1j * chi) * centre)
    modes = [p0]
    for _ in range(1, wl.K):
        amp = 1.0 + 0.3 * _smooth_field(rng, N, N / 16)
        ph = 0.8 * _smooth_field(rng, N, N / 16)
        modes.append(p0 * amp * np.exp(1j * ph))
    basis = []
    for m in modes:
        v = m.astype(np.complex128).copy()
        for b in basis:
            v -= np.vdot(b, v) * b
        v /= np.sqrt(np.vdot(v, v).real)
        basis.append(v)
    out = np.stack([b * math.sqrt(wk * wl.dose) for b, wk in zip(basis, wl.weights)])
    return out.astype(np.complex64)


def _atoms(rng, V, cy, cx, sigma_px, peak):
    H, W = V.shape
    r = int(math.ceil(4 * sigma_px))
    for y, x in zip(cy, cx):
        y0, x0 = int(math.floor(y)) - r, int(math.floor(x)) - r
        yy = np.arange(y0, y0 + 2 * r + 2)
        xx = np.arange(x0, x0 + 2 * r + 2)
        g = peak * np.exp(-((yy[:, None] - y) ** 2 + (xx[None, :] - x) ** 2) / (2 * sigma_px ** 2))
        V[np.ix_(yy % H, xx % W)] += g


def phase_object(wl: Workload, slices=None) -> np.ndarray:
    """complex64 [S, H, W] transmission exp(i sigma V) of Gaussian atoms."""
    rng = rng_for(wl.cid, ROLE_OBJECT)
    sigma_px = 0.4 / wl.dx
    S = wl.S
    n_total = wl.atoms_per_slice * S
    cy = rng.uniform(0, wl.H, n_total)
    cx = rng.uniform(0, wl.W, n_total)
    sl = rng.integers(0, S, n_total) if S > 1 else np.zeros(n_total, dtype=np.int64)
    want = range(S) if slices is None else slices
    out = np.empty((len(want), wl.H, wl.W), dtype=np.complex64)
    for i, s in enumerate(want):
        V = np.zeros((wl.H, wl.W))
        sel = sl == s
        _atoms(rng, V, cy[sel], cx[sel], sigma_px, 0.3)
        out[i] = np.exp(1j * V)
    return out


def raster_positions(wl: Workload) -> np.ndarray:
    """float32 [P, 2] (y, x) window top-left corners in object pixels."""
    rng = rng_for(wl.cid, ROLE_SCAN)
    ny, nx = wl.scan
    ext_y = (ny - 1) * wl.step_px + wl.N
    ext_x = (nx - 1) * wl.step_px + wl.N
    oy = (wl.H - ext_y) / 2.0
    ox = (wl.W - ext_x) / 2.0
    jit = 0.05 / wl.dx
    yy, xx = np.meshgrid(np.arange(ny) * wl.step_px + oy, np.arange(nx) * wl.step_px + ox, indexing="ij")
    pos = np.stack([yy.ravel(), xx.ravel()], axis=1)
    pos += rng.uniform(-jit, jit, pos.shape)
    lo = 0.5
    pos[:, 0] = np.clip(pos[:, 0], lo, wl.H - wl.N - lo)
    pos[:, 1] = np.clip(pos[:, 1], lo, wl.W - wl.N - lo)
    return pos.astype(np.float32)


def cbed_like_rate(wl: Workload) -> np.ndarray:
    """float64 [N, N] mean pattern (DC at [0, 0]) summing to the dose."""
    A, _ = aperture_and_aberration(wl.N, wl.dx, wl.lam, wl.alpha_mrad, wl.defocus_A, wl.C3_A)
    q = _freq(wl.N) / (wl.N * wl.dx)
    qa = np.sqrt(q[:, None] ** 2 + q[None, :] ** 2)
    halo = np.exp(-qa / (0.5 * wl.alpha_mrad * 1e-3 / wl.lam))
    rate = A + 0.05 * halo
    return rate * (wl.dose / rate.sum())


def cbed_like_patterns(wl: Workload, count: int, first: int = 0) -> np.ndarray:
    """float32 [count, N, N] Poisson patterns for positions first..first+count."""
    base = cbed_like_rate(wl)
    out = np.empty((count, wl.N, wl.N), dtype=np.float32)
    for i in range(count):
        r = np.random.Generator(np.random.PCG64([1000 * wl.cid + ROLE_PATTERN, first + i]))
        mod = 1.0 + 0.25 * _smooth_field(r, wl.N, wl.N / 12)
        out[i] = r.poisson(np.clip(base * mod, 0.0, None))
    return out


def poisson_counts(I: np.ndarray, cid: int) -> np.ndarray:
    """Poisson noise on a given mean intensity (for self-consistent data)."""
    return rng_for(cid, ROLE_NOISE).poisson(np.clip(np.asarray(I, np.float64), 0, None)).astype(np.float32)


def small_workload(cid=101, S=2, K=2, N=8, H=12, W=12, scan=(2, 2), step_px=2.0,
                   loss=0, eps=1e-3, c=0.0, dose=100.0, bandlimit=2.0 / 3.0,
                   dz_A=10.0, atoms=4) -> Workload:
    """A tiny problem for brute-force checks."""
    return Workload(cid, f"tiny S{S} K{K} N{N}", S=S, K=K, N=N, H=H, W=W, scan=scan,
                    step_px=step_px, B=scan[0] * scan[1], loss=loss, eps=eps, c=c,
                    dose=dose, alpha_mrad=400.0, defocus_A=5.0, C3_A=0.0,
                    weights=tuple([1.0 / K] * K), dz_A=dz_A, dx=0.1,
                    bandlimit=bandlimit, atoms_per_slice=atoms)


def cbed_like_patterns_device(wl: Workload, count: int, device="cuda", chunk=1024):
    """float32 [count, N, N] Poisson patterns drawn on a CUDA device with torch
    (same recipe as cbed_like_patterns; used for full-size workloads, where
    drawing millions of counts on the host would take minutes)."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(1000 * wl.cid + ROLE_PATTERN)
    base = torch.from_numpy(cbed_like_rate(wl)).to(device=device, dtype=torch.float32)
    f = torch.from_numpy(_freq(wl.N) / wl.N).to(device=device, dtype=torch.float32)
    corr = wl.N / 12
    g = torch.exp(-2.0 * (math.pi * corr) ** 2 * (f[:, None] ** 2 + f[None, :] ** 2))
    out = torch.empty((count, wl.N, wl.N), dtype=torch.float32, device=device)
    for i0 in range(0, count, chunk):
        n = min(chunk, count - i0)
        noise = torch.randn((n, wl.N, wl.N), generator=gen, device=device)
        x = torch.fft.ifft2(torch.fft.fft2(noise) * g).real
        x = x - x.mean(dim=(1, 2), keepdim=True)
        x = x / (x.std(dim=(1, 2), keepdim=True) + 1e-30)
        rate = torch.clamp(base * (1.0 + 0.25 * x), min=0.0)
        out[i0:i0 + n] = torch.poisson(rate, generator=gen)
    return out
