"""FP64 reference of the gradient-descent multislice ptychography path.

TEST INFRASTRUCTURE ONLY (see the package docstring): plain, slow and
obviously correct; complex128 throughout; every transform is a dense DFT
written out as two matrix products.

What it computes (arXiv 2505.14372):
  * §3, multislice recurrence: the entry wave is the probe mode shifted to the
    scan position; each slice multiplies by the object slice and, between
    slices, convolves with the Fresnel kernel p(dz) (done as DFT, product with
    the propagator, inverse DFT) under an anti-aliasing band limit.
  * §3, far field: I(k) = sum over incoherent modes of |F(exit wave)|^2.
  * §3.1, noise models: amplitude / Anscombe least squares on sqrt(I + c) and
    the Poisson negative log-likelihood in Stirling form with an epsilon
    inside the logarithms; the analytic detector-plane gradients of §3.1 are
    what the seed of the adjoint reduces to.
  * §3.2, gradient of the real loss with respect to every complex variable
    (Wirtinger calculus), for all slices and modes at once, and the Adam
    update applied to it.

Readings taken where the paper is silent or ambiguous (numbered as in the
repository's list of readings):
  R1  S slices take S-1 propagations; nothing is propagated after the last.
  R2  F is the unnormalised DFT with kernel exp(-2 pi i k x / N); F^-1 carries
      1/N; the far field uses the orthonormal F/sqrt(N); no fftshift: the
      zero frequency sits at pixel [0, 0] of every pattern.
  R3  Fresnel propagator H(q) = B(q) exp(-i pi lambda dz |q|^2), with
      q = f / (N dx) and f the integer DFT frequency in numpy fftfreq order
      (the Nyquist bin of an even size is -N/2).  B is a circular band limit
      at beta times the Nyquist frequency 1/(2 dx): on the discrete grid it
      keeps (f_u w)^2 + (f_v h)^2 <= floor(x*x) with x = beta*h*w*0.5
      evaluated left to right in IEEE double, so that the boundary decision
      is an exact integer comparison.  beta <= 0 switches the band limit off.
      The band limit acts in every propagation, not in the shift or far field.
  R4  A scan position r = (y, x) is in object pixels and locates the window's
      top-left corner.  n = floor(r + 1/2) picks the object patch and
      delta = r - n in [-1/2, 1/2) is applied as the Fourier phase ramp
      exp(-2 pi i (f_u delta_y / h + f_v delta_x / w)), i.e. P(r - delta).
  R5/R6 Amplitude (c = 0) / Anscombe (c = 3/8) loss per pixel:
      l = 1/2 (sqrt(I + c + eps) - sqrt(I_exp + c + eps))^2.
      Poisson loss per pixel: l = I - I_exp - I_exp (log(I+eps) - log(I_exp+eps)),
      whose derivative 1 - I_exp/(I + eps) is exactly the paper's Poisson
      detector gradient factor.
  R7  Gradient of a real L with respect to complex z is
      dL/dRe z + i dL/dIm z (= 2 dL/d conj(z)), twice the paper's
      conj(dL/dz); it matches finite differences on Re and Im directly.
  R8  Complex Adam: m <- b1 m + (1-b1) g, v <- b2 v + (1-b2)|g|^2 (real),
      z <- z - lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps_adam).
  R9  Incoherent mode weights are carried by the mode amplitudes.
  R10 The loss is the plain sum over pixels and positions.
  R13 Gaussian noise model (§3.1): l = (I - I_exp)^2 / (2 sigma^2), the
      normalisation constant dropped; sigma is passed in the c field.
  R14 Cost regularisers (§3.4) act on the complex transmission and the probe
      (the paper names the phase; for weak phase objects |grad O|^2 is
      |grad phase|^2): object L2 lambda sum |O - 1|^2 (vacuum is O = 1),
      probe L2 lambda sum |P|^2, in-plane Tikhonov lambda sum of squared
      forward differences along y and x inside each slice, and Tikhonov
      across layers lambda sum_s |O_{s+1} - O_s|^2.
      TV regularisers (§3.4, in-plane and across layers) act on the complex
      transmission like the Tikhonov ones, with the absolute value of each
      forward difference d smoothed to sqrt(|d|^2 + eta^2) - eta (eta > 0,
      the paper gives no smoothing; without one the gradient is undefined
      at d = 0).
  R15 Reduced-precision wavefields (§2.2 names 16-bit formats as future
      work): the entry waves that the backward pass reads for the object
      gradient may be stored as binary16 or bfloat16, rounded to nearest
      even from their binary32 values; nothing else is rounded.
  R16 ePIE / 3PIE (§3.3.1): the group's positions are updated together
      from the same O and P; the object normaliser max|O_s|^2 is taken over
      the whole slice and the wave normaliser max|psi_s|^2 per position and
      mode (the paper writes both per slice); between slices the update of
      the incident wave is carried back to the previous exit plane by the
      adjoint propagator conj(H); the probe update of each mode is the
      group mean of the unshifted entry-plane updates (the paper's mean is
      over the group); c and eps are the noise model's.
  R17 LSQML (§3.3.2): the detector update is ePIE's; the object direction
      is summed over the group and the modes; the step sizes alpha are
      least-squares steps per position (and per slice for the object), with
      the object direction restricted to the position's window in them; the
      probe update follows the object's at the entry plane (the paper says
      only that it is computed similarly): direction conj(O_0) chi_0 moved
      to the probe frame by the inverse sub-pixel shift, normaliser the
      transmission prod_s |O_s|^2 summed over the group's positions, step
      sizes from the exit-wave change O_0 S_j dP; the normalising sums are the
      group's own unless running sums of a previous iteration are passed in
      (the paper keeps them from the previous iteration); delta_O, delta_P
      and gamma are absolute.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from functools import lru_cache

import numpy as np

AMPLITUDE = 0
POISSON = 1
GAUSSIAN = 2

__all__ = [
    "AMPLITUDE", "POISSON", "Geom", "freq_index", "dft_matrix", "dft2",
    "idft2", "dft2_ortho", "idft2_ortho", "split_positions", "shift_ramp",
    "shift_probe", "bandlimit_mask", "propagator", "propagate",
    "forward", "forward_waves", "loss_terms", "loss_value", "gradient",
    "adam_update", "step", "position_gradient", "vjp", "GAUSSIAN", "regularizers",
    "round_storage", "epie_update", "lsqml_update", "lsqml_directions", "transmission",
]


@dataclass
class Geom:
    """Problem geometry (§3): S slices, K probe modes, h x w window,
    H x W object, pixel size dx [A], wavelength lam [A], S-1 gaps dz [A]."""
    S: int
    K: int
    h: int
    w: int
    H: int
    W: int
    dx: float = 0.1
    lam: float = 0.0197
    dz: tuple = field(default_factory=tuple)
    bandlimit: float = 2.0 / 3.0
    loss: int = AMPLITUDE
    eps: float = 0.0
    c: float = 0.0

    def __post_init__(self):
        self.dz = tuple(float(z) for z in self.dz)
        if len(self.dz) != max(self.S - 1, 0):
            raise ValueError("need S-1 slice gaps")


# ---------------------------------------------------------------- DFT (R2)

def freq_index(n: int) -> np.ndarray:
    """Integer DFT frequency of each bin in fftfreq order (R3)."""
    u = np.arange(n)
    return np.where(u < (n + 1) // 2, u, u - n)


@lru_cache(maxsize=None)
def dft_matrix(n: int) -> np.ndarray:
    """Dense F[k, x] = exp(-2 pi i (k x mod n) / n), angles from exact
    integer products."""
    idx = np.arange(n, dtype=np.int64)
    m = np.outer(idx, idx) % n
    ang = 2.0 * np.pi * m.astype(np.float64) / n
    F = np.cos(ang) - 1j * np.sin(ang)
    F.setflags(write=False)
    return F


def dft2(x: np.ndarray) -> np.ndarray:
    """Unnormalised 2-D DFT over the last two axes: F_h x F_w^T."""
    h, w = x.shape[-2:]
    return dft_matrix(h) @ x @ dft_matrix(w).T


def idft2(X: np.ndarray) -> np.ndarray:
    """Inverse of dft2 (carries 1/(h w))."""
    h, w = X.shape[-2:]
    return (np.conj(dft_matrix(h)) @ X @ np.conj(dft_matrix(w)).T) / (h * w)


def dft2_ortho(x: np.ndarray) -> np.ndarray:
    h, w = x.shape[-2:]
    return dft2(x) / math.sqrt(h * w)


def idft2_ortho(X: np.ndarray) -> np.ndarray:
    h, w = X.shape[-2:]
    return idft2(X) * math.sqrt(h * w)


# ------------------------------------------------------ shift & gather (R4)

def split_positions(pos) -> tuple[np.ndarray, np.ndarray]:
    """Integer patch origin n = floor(r + 1/2) and subpixel part r - n."""
    r = np.asarray(pos, dtype=np.float64).reshape(-1, 2)
    n = np.floor(r + 0.5)
    return n.astype(np.int64), r - n


def shift_ramp(dy: float, dx_: float, h: int, w: int) -> np.ndarray:
    """exp(-2 pi i (f_u dy / h + f_v dx / w)); the phase is formed in turns
    and reduced to [-1/2, 1/2] before the exponential."""
    t = (freq_index(h)[:, None] * float(dy) / h
         + freq_index(w)[None, :] * float(dx_) / w)
    t = t - np.round(t)
    return np.exp(-2j * np.pi * t)


def shift_probe(P: np.ndarray, dy: float, dx_: float) -> np.ndarray:
    """P(r - delta) for every mode: F^-1[ramp * F P] (§3, first equation)."""
    h, w = P.shape[-2:]
    return idft2(shift_ramp(dy, dx_, h, w) * dft2(P))


def _patch(O, s, n, h, w):
    """Object sub-region of slice s under the window at origin n (§2.2: the
    object is sampled around each probe position to form the transmission
    functions)."""
    return O[s, n[0]:n[0] + h, n[1]:n[1] + w]


# ------------------------------------------------------- propagator (R3)

def bandlimit_mask(h: int, w: int, beta: float) -> np.ndarray:
    """Circular anti-alias band limit on the DFT grid (R3)."""
    if beta <= 0.0:
        return np.ones((h, w), dtype=bool)
    x = float(beta) * float(h) * float(w) * 0.5
    T = math.floor(x * x)
    fu = freq_index(h).astype(np.int64)[:, None]
    fv = freq_index(w).astype(np.int64)[None, :]
    lhs = (fu * w) ** 2 + (fv * h) ** 2
    return lhs <= T


def propagator(h: int, w: int, dx: float, lam: float, dz: float,
               beta: float) -> np.ndarray:
    """Band-limited Fresnel propagator over gap dz (§3 and R3)."""
    qu = freq_index(h)[:, None] / (h * dx)
    qv = freq_index(w)[None, :] / (w * dx)
    chirp = np.exp(-1j * np.pi * lam * dz * (qu * qu + qv * qv))
    return chirp * bandlimit_mask(h, w, beta)


def propagate(phi: np.ndarray, Hs: np.ndarray) -> np.ndarray:
    """Convolution with p(dz) as F^-1[H F phi]."""
    return idft2(Hs * dft2(phi))


# ------------------------------------------------------- forward (§3)

def _check(O, P, pos, g: Geom):
    O = np.asarray(O, dtype=np.complex128)
    P = np.asarray(P, dtype=np.complex128)
    if O.shape != (g.S, g.H, g.W) or P.shape != (g.K, g.h, g.w):
        raise ValueError("shape mismatch")
    n, d = split_positions(pos)
    if (n[:, 0] < 0).any() or (n[:, 1] < 0).any() or \
       (n[:, 0] + g.h > g.H).any() or (n[:, 1] + g.w > g.W).any():
        raise ValueError("scan position outside the object")
    return O, P, n, d


def _props(g: Geom):
    return [propagator(g.h, g.w, g.dx, g.lam, dz, g.bandlimit) for dz in g.dz]


def forward_waves(O, P, pos, g: Geom):
    """Per position: entry waves psi[s] of every slice (K modes each) and the
    orthonormal far field A of the exit wave.  Returns (psis, A, n, d) with
    psis [B, S, K, h, w] and A [B, K, h, w]."""
    O, P, n, d = _check(O, P, pos, g)
    Hs = _props(g)
    B = n.shape[0]
    psis = np.zeros((B, g.S, g.K, g.h, g.w), dtype=np.complex128)
    A = np.zeros((B, g.K, g.h, g.w), dtype=np.complex128)
    for j in range(B):
        psi = shift_probe(P, d[j, 0], d[j, 1])
        for s in range(g.S):
            psis[j, s] = psi
            phi = psi * _patch(O, s, n[j], g.h, g.w)
            if s < g.S - 1:
                psi = propagate(phi, Hs[s])
        A[j] = dft2_ortho(phi)
    return psis, A, n, d


def forward(O, P, pos, g: Geom) -> np.ndarray:
    """Simulated patterns I [B, h, w] = sum_k |F_o exit_k|^2, DC at [0, 0]."""
    _, A, _, _ = forward_waves(O, P, pos, g)
    return np.sum(np.abs(A) ** 2, axis=1)


# ----------------------------------------------------------- loss (§3.1)

def loss_terms(I, I_exp, g: Geom):
    """Per-pixel loss l(I) and its derivative dl/dI (R5/R6, R13)."""
    I = np.asarray(I, dtype=np.float64)
    E = np.asarray(I_exp, dtype=np.float64)
    if g.loss == AMPLITUDE:
        a = np.sqrt(I + g.c + g.eps)
        b = np.sqrt(E + g.c + g.eps)
        return 0.5 * (a - b) ** 2, 0.5 * (1.0 - b / a)
    if g.loss == POISSON:
        l = I - E - E * (np.log(I + g.eps) - np.log(E + g.eps))
        return l, 1.0 - E / (I + g.eps)
    if g.loss == GAUSSIAN:
        s2 = g.c * g.c
        return (I - E) ** 2 / (2.0 * s2), (I - E) / s2
    raise ValueError("unknown loss")


def loss_value(I, I_exp, g: Geom) -> float:
    return float(np.sum(loss_terms(I, I_exp, g)[0]))


# ------------------------------------------------------- gradient (§3.2)

def _backprop(O, psis, A, n, d, seeds, g: Geom):
    """Cotangents of O and P from detector-plane seeds g_A [B, K, h, w]
    (R7 convention) by the exact chain rule: for each linear map y = M x the
    cotangent is M^H g_y; the transmission product gives
    g_O += conj(psi) g_phi and g_psi = conj(O) g_phi."""
    Hs = _props(g)
    gO = np.zeros_like(O)
    gPhat = np.zeros((g.K, g.h, g.w), dtype=np.complex128)
    for j in range(n.shape[0]):
        g_phi = idft2_ortho(seeds[j])
        for s in range(g.S - 1, -1, -1):
            patch = _patch(O, s, n[j], g.h, g.w)
            y0, x0 = n[j]
            gO[s, y0:y0 + g.h, x0:x0 + g.w] += np.sum(np.conj(psis[j, s]) * g_phi, axis=0)
            g_psi = np.conj(patch) * g_phi
            if s > 0:
                g_phi = idft2(np.conj(Hs[s - 1]) * dft2(g_psi))
        gPhat += np.conj(shift_ramp(d[j, 0], d[j, 1], g.h, g.w)) * dft2(g_psi)
    return gO, idft2(gPhat)


def round_storage(z, fmt):
    """Complex array as held in a reduced storage format (R15), real and
    imaginary parts separately: first rounded to binary32 (the precision the
    kernels compute in), then to nearest with ties to even on
    'f16' - IEEE binary16 (11 significant bits, subnormals below 2^-14),
    'bf16' - bfloat16 (the upper 16 bits of binary32: 8 significant bits).
    None or 'f32' keeps binary32."""
    z = np.asarray(z, dtype=np.complex128)

    def part(x):
        x32 = np.asarray(x, dtype=np.float32)
        if fmt in (None, "f32"):
            return x32.astype(np.float64)
        if fmt == "f16":
            return x32.astype(np.float16).astype(np.float64)
        if fmt == "bf16":
            u = x32.view(np.uint32).astype(np.uint64)
            # add half of the dropped 16 bits, plus one when the kept part is
            # odd (ties to even), then drop them
            u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
            return u.astype(np.uint32).view(np.float32).astype(np.float64)
        raise ValueError("unknown storage format")

    return part(z.real) + 1j * part(z.imag)


def gradient(O, P, pos, I_exp, g: Geom, wave_fmt=None):
    """Loss and its gradients (R7 convention) with respect to every object
    slice and every probe mode; the detector seed is 2 l'(I) A.
    wave_fmt: storage format of the entry waves that the object-gradient
    term g_O += conj(psi) g_phi reads (R15, see round_storage); the
    propagated wavefield itself is never rounded.
    Returns (loss, gO [S,H,W], gP [K,h,w])."""
    psis, A, n, d = forward_waves(O, P, pos, g)
    if wave_fmt is not None:
        psis = round_storage(psis, wave_fmt)
    O = np.asarray(O, dtype=np.complex128)
    E = np.asarray(I_exp, dtype=np.float64).reshape(-1, g.h, g.w)
    seeds = np.zeros_like(A)
    loss = 0.0
    for j in range(n.shape[0]):
        I = np.sum(np.abs(A[j]) ** 2, axis=0)
        l, dl = loss_terms(I, E[j], g)
        loss += float(np.sum(l))
        seeds[j] = 2.0 * dl * A[j]
    gO, gP = _backprop(O, psis, A, n, d, seeds, g)
    return loss, gO, gP


def vjp(O, P, pos, gI, g: Geom):
    """Vector-Jacobian product of the forward model for a cotangent
    gI = dL/dI [B, h, w]: seed 2 gI A.  Returns (gO, gP)."""
    psis, A, n, d = forward_waves(O, P, pos, g)
    O = np.asarray(O, dtype=np.complex128)
    G = np.asarray(gI, dtype=np.float64).reshape(-1, 1, g.h, g.w)
    return _backprop(O, psis, A, n, d, 2.0 * G * A, g)


def position_gradient(O, P, pos, I_exp, g: Geom) -> np.ndarray:
    """dL/d(r_y, r_x) per position [B, 2] through the Fourier ramp only (the
    integer patch origin is piecewise constant).  With psi0 = F^-1[R F P],
    R = exp(-2 pi i (f_u dy/h + f_v dx/w)): dpsi0/ddy = F^-1[-2 pi i f_u/h R F P],
    and dL/ddy = Re sum conj(g_psi0) dpsi0/ddy under the R7 convention."""
    psis, A, n, d = forward_waves(O, P, pos, g)
    O = np.asarray(O, dtype=np.complex128)
    P = np.asarray(P, dtype=np.complex128)
    E = np.asarray(I_exp, dtype=np.float64).reshape(-1, g.h, g.w)
    Hs = _props(g)
    FP = dft2(P)
    fu = freq_index(g.h)[:, None] / g.h
    fv = freq_index(g.w)[None, :] / g.w
    out = np.zeros((n.shape[0], 2))
    for j in range(n.shape[0]):
        I = np.sum(np.abs(A[j]) ** 2, axis=0)
        _, dl = loss_terms(I, E[j], g)
        g_phi = idft2_ortho(2.0 * dl * A[j])
        for s in range(g.S - 1, -1, -1):
            g_psi = np.conj(_patch(O, s, n[j], g.h, g.w)) * g_phi
            if s > 0:
                g_phi = idft2(np.conj(Hs[s - 1]) * dft2(g_psi))
        R = shift_ramp(d[j, 0], d[j, 1], g.h, g.w)
        dpsi_y = idft2(-2j * np.pi * fu * R * FP)
        dpsi_x = idft2(-2j * np.pi * fv * R * FP)
        out[j, 0] = float(np.real(np.sum(np.conj(g_psi) * dpsi_y)))
        out[j, 1] = float(np.real(np.sum(np.conj(g_psi) * dpsi_x)))
    return out


# ---------------------------------------------------- ePIE / 3PIE (§3.3.1)

def epie_update(O, P, pos, I_exp, g: Geom, beta_O=1.0, beta_P=1.0, tiny=1e-30):
    """One ePIE (multislice: 3PIE) update of O and P from one group of
    positions, all of which see the same O and P (R16).  The steps, in the
    order of §3.3.1:
      1. detector-plane update of each mode from the generalised modulus
         constraint of §3.1: chi(k) = (sqrt(I_exp + c) / (eps + sqrt(I + c)) - 1) A_k,
         I the mode sum; carried to the exit plane with the inverse
         orthonormal DFT;
      2. for slices s = S-1 .. 0: the object update
         dO_s = conj(psi_s) chi_s / max_r |psi_s|^2 (psi_s the incident
         wave of this position and mode), then the incident-wave update
         conj(O_s) chi_s / max_r |O_s|^2 (maximum over the whole slice),
         propagated back to the exit plane of slice s-1 with conj(H);
      3. the probe-plane update is unshifted (conjugate Fourier ramp);
         object updates are summed over modes and positions, probe updates
         averaged over the positions:
         O += beta_O sum dO, P_k += beta_P mean_j unshift(chi_0).
    The noise model must be the amplitude one (c = 0 ePIE, c = 3/8
    Anscombe).  Returns (O_new, P_new, loss) with the group's amplitude loss
    before the update."""
    if g.loss != AMPLITUDE:
        raise ValueError("ePIE uses the amplitude / Anscombe modulus update")
    psis, A, n, d = forward_waves(O, P, pos, g)
    O = np.asarray(O, dtype=np.complex128)
    P = np.asarray(P, dtype=np.complex128)
    E = np.asarray(I_exp, dtype=np.float64).reshape(-1, g.h, g.w)
    Hs = _props(g)
    B = n.shape[0]
    inv_omax = [1.0 / max(float(np.max(np.abs(O[s]) ** 2)), tiny) for s in range(g.S)]
    dO = np.zeros_like(O)
    dPhat = np.zeros((g.K, g.h, g.w), dtype=np.complex128)
    loss = 0.0
    for j in range(B):
        I = np.sum(np.abs(A[j]) ** 2, axis=0)
        loss += float(np.sum(loss_terms(I, E[j], g)[0]))
        m = np.sqrt(E[j] + g.c) / (g.eps + np.sqrt(I + g.c)) - 1.0
        y0, x0 = n[j]
        for k in range(g.K):
            chi = idft2_ortho(m * A[j, k])
            for s in range(g.S - 1, -1, -1):
                psi = psis[j, s, k]
                pmax = max(float(np.max(np.abs(psi) ** 2)), tiny)
                dO[s, y0:y0 + g.h, x0:x0 + g.w] += np.conj(psi) * chi / pmax
                chi = inv_omax[s] * np.conj(_patch(O, s, n[j], g.h, g.w)) * chi
                if s > 0:
                    chi = idft2(np.conj(Hs[s - 1]) * dft2(chi))
            dPhat[k] += np.conj(shift_ramp(d[j, 0], d[j, 1], g.h, g.w)) * dft2(chi)
    O_new = O + beta_O * dO
    P_new = P + beta_P * idft2(dPhat) / max(B, 1)
    return O_new, P_new, loss


# ------------------------------------------------------------ LSQML (§3.3.2)

def transmission(O, n, h, w):
    """Product over slices of |O_s|^2 on the window at integer origin n: how
    transparent the object is to each pixel of the probe (R17)."""
    t = np.ones((h, w))
    for s in range(O.shape[0]):
        t *= np.abs(_patch(O, s, n, h, w)) ** 2
    return t


def lsqml_directions(O, P, pos, I_exp, g: Geom):
    """Step 1 of the LSQML update (R17): for one group, the object and probe
    update directions summed over positions and modes (NO [S,H,W], NP [K,h,w],
    probe frame), the group's illumination W [S,H,W] and transmission
    T [h,w], the exit-plane updates chi [B,S,K,h,w] of every slice, and the
    forward pass (psis, n, d) and loss they came from."""
    if g.loss != AMPLITUDE:
        raise ValueError("LSQML uses the amplitude / Anscombe modulus update")
    psis, A, n, d = forward_waves(O, P, pos, g)
    O = np.asarray(O, dtype=np.complex128)
    E = np.asarray(I_exp, dtype=np.float64).reshape(-1, g.h, g.w)
    Hs = _props(g)
    B = n.shape[0]
    S, K, h, w = g.S, g.K, g.h, g.w
    NO = np.zeros_like(O)                       # object directions, summed
    NP_ = np.zeros((K, h, w), np.complex128)    # probe directions, summed (probe frame)
    W = np.zeros(O.shape)                       # illumination of this group
    T = np.zeros((h, w))                        # transmission of this group
    chis = np.zeros((B, S, K, h, w), np.complex128)  # exit-plane updates per slice
    loss = 0.0
    for j in range(B):
        I = np.sum(np.abs(A[j]) ** 2, axis=0)
        loss += float(np.sum(loss_terms(I, E[j], g)[0]))
        m = np.sqrt(E[j] + g.c) / (g.eps + np.sqrt(I + g.c)) - 1.0
        y0, x0 = n[j]
        T += transmission(O, n[j], h, w)
        for k in range(K):
            chi = idft2_ortho(m * A[j, k])
            for s in range(S - 1, -1, -1):
                chis[j, s, k] = chi
                NO[s, y0:y0 + h, x0:x0 + w] += np.conj(psis[j, s, k]) * chi
                W[s, y0:y0 + h, x0:x0 + w] += np.abs(psis[j, s, k]) ** 2
                chi = np.conj(_patch(O, s, n[j], h, w)) * chi
                if s > 0:
                    chi = idft2(np.conj(Hs[s - 1]) * dft2(chi))
            NP_[k] += idft2(np.conj(shift_ramp(d[j, 0], d[j, 1], h, w)) * dft2(chi))
    return NO, NP_, W, T, chis, psis, n, d, loss


def lsqml_update(O, P, pos, I_exp, g: Geom, beta_O=1.0, beta_P=1.0, delta_O=0.0, delta_P=0.0, gamma=0.0,
                 illum=None, trans=None):
    """One LSQML update of O and P from one group of positions (R17), in the
    order of §3.3.2:
      1. exit-plane updates chi of every position and mode from the
         generalised modulus constraint (as ePIE), carried back through the
         slices: at slice s the object direction conj(psi_s) chi_s and the
         illumination direction conj(O_s) chi_s, the latter propagated back
         (conj(H)) to become chi_{s-1}; at the entry plane it is unshifted
         into the probe frame;
      2. the object direction summed over the group and modes, divided by the
         illumination sum_{j,k} |psi_s|^2 + delta_O (object frame); the probe
         direction summed over the group, divided by the transmission
         sum_j prod_s |O_s|^2 + delta_P (probe frame); `illum` [S,H,W] and
         `trans` [h,w] replace these sums when given (the running sums of a
         previous iteration);
      3. per position j, least-squares step sizes
         alpha_{s,j} = sum_{r,k} Re[chi_s conj(dO_s psi_s)] / (sum |dO_s psi_s|^2 + gamma)
         alpha_{P,j} = sum_{r,k} Re[chi_0 conj(O_0 S_j dP_k)] / (sum |O_0 S_j dP_k|^2 + gamma),
         S_j the position's sub-pixel shift;
      4. O_s += beta_O dO_s sum_j alpha_{s,j} w_{s,j} / sum_j w_{s,j}, with
         w_{s,j} = sum_k |psi_{s,k,j}|^2; P_k += beta_P dP_k sum_j alpha_{P,j} t_j /
         sum_j t_j, with t_j the transmission of position j (zero weight sums
         leave the pixel unchanged).
    The noise model must be the amplitude one.  Returns
    (O_new, P_new, loss, illum_group [S,H,W], trans_group [h,w])."""
    NO, NP_, W, T, chis, psis, n, d, loss = lsqml_directions(O, P, pos, I_exp, g)
    O = np.asarray(O, dtype=np.complex128)
    P = np.asarray(P, dtype=np.complex128)
    B = n.shape[0]
    S, K, h, w = g.S, g.K, g.h, g.w
    Wd = W if illum is None else np.asarray(illum, dtype=np.float64)
    Td = T if trans is None else np.asarray(trans, dtype=np.float64)
    # pixels no position of the group reaches keep a zero direction
    dO = np.divide(NO, Wd + delta_O, out=np.zeros_like(NO), where=(Wd + delta_O) > 0)
    dP = np.divide(NP_, (Td + delta_P)[None], out=np.zeros_like(NP_), where=((Td + delta_P) > 0)[None])
    AW = np.zeros(O.shape)
    AT = np.zeros((h, w))
    for j in range(B):
        y0, x0 = n[j]
        for s in range(S):
            dOs = dO[s, y0:y0 + h, x0:x0 + w]
            num = den = 0.0
            for k in range(K):
                q = dOs * psis[j, s, k]
                num += float(np.sum(np.real(chis[j, s, k] * np.conj(q))))
                den += float(np.sum(np.abs(q) ** 2))
            a = num / (den + gamma) if den + gamma > 0 else 0.0
            AW[s, y0:y0 + h, x0:x0 + w] += a * np.sum(np.abs(psis[j, s]) ** 2, axis=0)
        O0 = _patch(O, 0, n[j], h, w)
        num = den = 0.0
        for k in range(K):
            q = O0 * shift_probe(dP[k:k + 1], d[j, 0], d[j, 1])[0]
            num += float(np.sum(np.real(chis[j, 0, k] * np.conj(q))))
            den += float(np.sum(np.abs(q) ** 2))
        aP = num / (den + gamma) if den + gamma > 0 else 0.0
        AT += aP * transmission(O, n[j], h, w)
    O_new = O + beta_O * dO * np.divide(AW, W, out=np.zeros_like(AW), where=W > 0)
    P_new = P + beta_P * dP * np.divide(AT, T, out=np.zeros_like(AT), where=T > 0)[None]
    return O_new, P_new, loss, W, T


# ---------------------------------------------------- regularisers (§3.4)

def regularizers(O, P, l2_obj=0.0, tikhonov=0.0, layers=0.0, l2_probe=0.0, tv=0.0, tv_layers=0.0,
                 tv_eps=1e-3):
    """Cost-regulariser value and gradients (R7 convention) (R14)."""
    O = np.asarray(O, dtype=np.complex128)
    P = np.asarray(P, dtype=np.complex128)
    val = 0.0
    gO = np.zeros_like(O)
    gP = np.zeros_like(P)
    if l2_obj:
        val += l2_obj * float(np.sum(np.abs(O - 1.0) ** 2))
        gO += 2.0 * l2_obj * (O - 1.0)
    if l2_probe:
        val += l2_probe * float(np.sum(np.abs(P) ** 2))
        gP += 2.0 * l2_probe * P
    if tikhonov:
        dy = O[:, 1:, :] - O[:, :-1, :]
        dx = O[:, :, 1:] - O[:, :, :-1]
        val += tikhonov * float(np.sum(np.abs(dy) ** 2) + np.sum(np.abs(dx) ** 2))
        gO[:, 1:, :] += 2.0 * tikhonov * dy
        gO[:, :-1, :] -= 2.0 * tikhonov * dy
        gO[:, :, 1:] += 2.0 * tikhonov * dx
        gO[:, :, :-1] -= 2.0 * tikhonov * dx
    if layers and O.shape[0] > 1:
        dz = O[1:] - O[:-1]
        val += layers * float(np.sum(np.abs(dz) ** 2))
        gO[1:] += 2.0 * layers * dz
        gO[:-1] -= 2.0 * layers * dz

    def tv_term(lam, d):
        # lam sum (sqrt(|d|^2 + eta^2) - eta); its R7 gradient with respect to
        # the minuend of d is lam d / sqrt(|d|^2 + eta^2)
        r = np.sqrt(np.abs(d) ** 2 + tv_eps ** 2)
        return lam * float(np.sum(r - tv_eps)), lam * d / r

    if tv:
        v1, t1 = tv_term(tv, O[:, 1:, :] - O[:, :-1, :])
        v2, t2 = tv_term(tv, O[:, :, 1:] - O[:, :, :-1])
        val += v1 + v2
        gO[:, 1:, :] += t1
        gO[:, :-1, :] -= t1
        gO[:, :, 1:] += t2
        gO[:, :, :-1] -= t2
    if tv_layers and O.shape[0] > 1:
        v3, t3 = tv_term(tv_layers, O[1:] - O[:-1])
        val += v3
        gO[1:] += t3
        gO[:-1] -= t3
    return val, gO, gP


# ----------------------------------------------------------- Adam (§3.2)

def adam_update(z, m, v, gz, t: int, lr: float, b1=0.9, b2=0.999, eps=1e-8):
    """One complex Adam step (R8); t counts steps from 1.  Returns new
    (z, m, v)."""
    m = b1 * m + (1.0 - b1) * gz
    v = b2 * v + (1.0 - b2) * (np.abs(gz) ** 2)
    mhat = m / (1.0 - b1 ** t)
    vhat = v / (1.0 - b2 ** t)
    return z - lr * mhat / (np.sqrt(vhat) + eps), m, v


def step(O, P, mO, vO, mP, vP, t, pos_all, I_exp_all, idx, g: Geom,
         lr_O, lr_P, b1=0.9, b2=0.999, eps_adam=1e-8, update_probe=True, reg=None):
    """One gradient-descent iteration on the minibatch idx (§2.2 grouping,
    §3.2 solver, optional §3.4 cost regularisers `reg`, a dict of
    regularizers() weights).  t is the Adam step count AFTER this step.  Returns
    (O, P, mO, vO, mP, vP, loss, gnorm) where gnorm = sqrt(sum |g|^2) over
    the object and probe gradients."""
    idx = np.asarray(idx, dtype=np.int64)
    pos = np.asarray(pos_all, dtype=np.float64).reshape(-1, 2)[idx]
    E = np.asarray(I_exp_all, dtype=np.float64).reshape(-1, g.h, g.w)[idx]
    loss, gO, gP = gradient(O, P, pos, E, g)
    if reg:
        rv, rO, rP = regularizers(O, P, **reg)
        loss, gO, gP = loss + rv, gO + rO, gP + rP
    gnorm = math.sqrt(float(np.sum(np.abs(gO) ** 2) + np.sum(np.abs(gP) ** 2)))
    O2, mO, vO = adam_update(np.asarray(O, np.complex128), mO, vO, gO, t, lr_O, b1, b2, eps_adam)
    if update_probe:
        P2, mP, vP = adam_update(np.asarray(P, np.complex128), mP, vP, gP, t, lr_P, b1, b2, eps_adam)
    else:
        P2 = np.asarray(P, np.complex128)
    return O2, P2, mO, vO, mP, vP, loss, gnorm
