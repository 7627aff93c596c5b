"""Pins of the oracle's DFT, subpixel shift and propagator against closed
forms, invariants and a library routine (arXiv 2505.14372 §3)."""
import math

import numpy as np
import pytest

import oracle as orc

RNG = np.random.default_rng(7)


def crand(*shape):
    return RNG.standard_normal(shape) + 1j * RNG.standard_normal(shape)


# ------------------------------------------------------------------ DFT

@pytest.mark.parametrize("h,w", [(8, 8), (12, 16), (64, 64), (7, 9), (192, 192)])
def test_dft_roundtrip_and_parseval(h, w):
    x = crand(3, h, w)
    assert np.max(np.abs(orc.idft2(orc.dft2(x)) - x)) < 1e-12 * np.max(np.abs(x)) * max(h, w)
    X = orc.dft2_ortho(x)
    assert abs(np.sum(np.abs(X) ** 2) - np.sum(np.abs(x) ** 2)) < 1e-11 * np.sum(np.abs(x) ** 2)


@pytest.mark.parametrize("n", [8, 12, 64, 128, 192, 256])
def test_dft_matches_library_fft(n):
    # special case that reduces to a library routine (test-only use of numpy.fft)
    x = crand(n, n)
    assert np.max(np.abs(orc.dft2(x) - np.fft.fft2(x))) < 1e-11 * n * n
    assert np.max(np.abs(orc.idft2(x) - np.fft.ifft2(x))) < 1e-11


def test_dft_of_delta_and_plane_wave():
    n = 16
    d = np.zeros((n, n), complex)
    d[0, 0] = 1.0
    assert np.allclose(orc.dft2(d), 1.0, atol=1e-14)
    # a delta at (a, b) has spectrum exp(-2 pi i (u a + v b)/n)
    d2 = np.zeros((n, n), complex)
    d2[3, 5] = 1.0
    u = np.arange(n)
    ref = np.exp(-2j * np.pi * (u[:, None] * 3 + u[None, :] * 5) / n)
    assert np.allclose(orc.dft2(d2), ref, atol=1e-13)
    # a plane wave exp(+2 pi i (m x + p y)/n) is n^2 delta at (m, p)
    pw = np.exp(2j * np.pi * (2 * u[:, None] + 7 * u[None, :]) / n)
    X = orc.dft2(pw)
    ref = np.zeros((n, n), complex)
    ref[2, 7] = n * n
    assert np.allclose(X, ref, atol=1e-10)


def test_freq_index_is_fftfreq_order():
    for n in (7, 8, 64, 192):
        assert np.array_equal(orc.freq_index(n), np.rint(np.fft.fftfreq(n) * n).astype(int))


# ---------------------------------------------------------------- shift

def test_split_positions_rounding():
    n, d = orc.split_positions([[2.5, 3.49999], [0.0, 7.25], [4.75, 1.5]])
    assert n.tolist() == [[3, 3], [0, 7], [5, 2]]
    assert np.all(d >= -0.5) and np.all(d < 0.5)
    assert np.allclose(d, [[-0.5, 0.49999], [0.0, 0.25], [-0.25, -0.5]])


def test_shift_identity_and_integer_roll():
    P = crand(2, 12, 10)
    assert np.allclose(orc.shift_probe(P, 0.0, 0.0), P, atol=1e-13)
    for a, b in [(1, 0), (0, 3), (-2, 4), (5, -1)]:
        assert np.allclose(orc.shift_probe(P, a, b), np.roll(P, (a, b), axis=(1, 2)), atol=1e-12)


def test_shift_sign_on_plane_wave():
    # P(r - delta) for a single Fourier component is the component times
    # exp(-2 pi i f delta / n): fixes sign and direction of the shift
    n = 16
    x = np.arange(n)
    f = 3
    P = np.exp(2j * np.pi * f * x[:, None] / n) * np.ones((1, n))
    out = orc.shift_probe(P[None], 0.3, 0.0)[0]
    ref = np.exp(2j * np.pi * f * (x[:, None] - 0.3) / n) * np.ones((1, n))
    assert np.allclose(out, ref, atol=1e-12)


def test_shift_modulus_invariance_and_composition():
    P = crand(3, 16, 16)
    a, b = (0.3, -0.45), (-0.2, 0.1)
    Sa = orc.shift_probe(P, *a)
    assert np.allclose(np.abs(orc.dft2(Sa)), np.abs(orc.dft2(P)), atol=1e-10)
    Sab = orc.shift_probe(Sa, *b)
    assert np.allclose(Sab, orc.shift_probe(P, a[0] + b[0], a[1] + b[1]), atol=1e-12)


# ------------------------------------------------------------ propagator

def test_bandlimit_mask_geometry():
    for n, beta in [(64, 2 / 3), (192, 2 / 3), (128, 0.5), (12, 0.9)]:
        m = orc.bandlimit_mask(n, n, beta)
        f = orc.freq_index(n)
        r = np.sqrt(f[:, None] ** 2 + f[None, :] ** 2) / n   # |q| dx
        away = np.abs(r - beta / 2) > 1e-9
        assert np.array_equal(m[away], (r <= beta / 2)[away])
        assert m[0, 0]
        assert np.array_equal(m, m.T)
    assert orc.bandlimit_mask(16, 16, 0.0).all()
    assert orc.bandlimit_mask(16, 16, -1.0).all()


def test_propagator_unitary_and_semigroup():
    n = 32
    x = crand(2, n, n)
    H0 = orc.propagator(n, n, 0.1, 0.0197, 10.0, 0.0)
    assert np.allclose(np.abs(H0), 1.0)
    y = orc.propagate(x, H0)
    assert abs(np.sum(np.abs(y) ** 2) - np.sum(np.abs(x) ** 2)) < 1e-10 * np.sum(np.abs(x) ** 2)
    Hz = orc.propagator(n, n, 0.1, 0.0197, 0.0, 2 / 3)
    assert np.array_equal(Hz, orc.bandlimit_mask(n, n, 2 / 3).astype(complex))
    H1 = orc.propagator(n, n, 0.1, 0.0197, 7.0, 2 / 3)
    H2 = orc.propagator(n, n, 0.1, 0.0197, 5.0, 2 / 3)
    H12 = orc.propagator(n, n, 0.1, 0.0197, 12.0, 2 / 3)
    assert np.allclose(H1 * H2, H12, atol=1e-12)


@pytest.mark.parametrize("beta", [0.0, 2 / 3])
def test_fresnel_gaussian_beam_closed_form(beta):
    """A Gaussian exp(-r^2/(2 s^2)) propagated over z by the Fresnel kernel
    exp(-i pi lam z q^2) is (2 pi^2 s^2/a) exp(-pi^2 r^2/a) with
    a = 2 pi^2 s^2 + i pi lam z (paraxial propagation of a Gaussian beam)."""
    n, dx, lam, z, s = 64, 0.1, 0.0197, 25.0, 0.4
    c = np.arange(n) - n // 2
    r2 = (c[:, None] ** 2 + c[None, :] ** 2) * dx * dx
    g = np.exp(-r2 / (2 * s * s)).astype(complex)
    a = 2 * np.pi ** 2 * s * s + 1j * np.pi * lam * z
    ref = (2 * np.pi ** 2 * s * s / a) * np.exp(-np.pi ** 2 * r2 / a)
    out = orc.propagate(g, orc.propagator(n, n, dx, lam, z, beta))
    assert np.max(np.abs(out - ref)) < 1e-10
