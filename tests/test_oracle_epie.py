"""Pins of the oracle's ePIE / 3PIE update (arXiv 2505.14372 §3.3.1): the
single-slice, single-mode case against the textbook ePIE iteration written
out here, the fixed point on consistent data, and the multislice update
against the amplitude-loss gradient (already pinned by finite differences)
with the per-slice normalisers that ePIE adds."""
import numpy as np
import pytest

import oracle as orc

RNG = np.random.default_rng(31)


def crand(*shape, scale=1.0):
    return scale * (RNG.standard_normal(shape) + 1j * RNG.standard_normal(shape))


def geom(S, K, c=0.0, eps=0.0, beta=2 / 3):
    return orc.Geom(S=S, K=K, h=8, w=8, H=14, W=14, dx=0.1, lam=0.0197, dz=(10.0,) * (S - 1),
                    bandlimit=beta, loss=orc.AMPLITUDE, eps=eps, c=c)


def test_single_slice_single_mode_is_textbook_epie():
    # ePIE (one position at an integer offset): exit wave psi = P O_patch,
    # replace the Fourier modulus by the measured one, then
    # O_patch += bO conj(P) / max|P|^2 (psi' - psi),
    # P      += bP conj(O_patch) / max|O|^2 (psi' - psi)
    g = geom(1, 1)
    O = np.exp(1j * 0.5 * RNG.standard_normal((1, 14, 14))) * (0.7 + 0.3 * RNG.random((1, 14, 14)))
    P = crand(1, 8, 8, scale=2.0)
    y0, x0 = 3, 5
    E = RNG.random((1, 8, 8)) * 20 + 1
    bO, bP = 0.7, 0.4
    O_new, P_new, _ = orc.epie_update(O, P, np.array([[y0, x0]], float), E, g, beta_O=bO, beta_P=bP)
    patch = O[0, y0:y0 + 8, x0:x0 + 8]
    psi = P[0] * patch
    Psi = np.fft.fft2(psi, norm="ortho")
    psi2 = np.fft.ifft2(np.sqrt(E[0]) * Psi / np.abs(Psi), norm="ortho")
    want_O = O.copy()
    want_O[0, y0:y0 + 8, x0:x0 + 8] += bO * np.conj(P[0]) / np.max(np.abs(P[0]) ** 2) * (psi2 - psi)
    want_P = P[0] + bP * np.conj(patch) / np.max(np.abs(O[0]) ** 2) * (psi2 - psi)
    assert np.allclose(O_new, want_O, rtol=1e-11, atol=1e-12)
    assert np.allclose(P_new[0], want_P, rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("S,K", [(1, 2), (3, 2)])
def test_consistent_data_is_a_fixed_point(S, K):
    g = geom(S, K)
    O = np.exp(1j * 0.4 * RNG.standard_normal((S, 14, 14)))
    P = crand(K, 8, 8)
    pos = np.array([[0.3, 1.2], [4.6, 2.2], [2.0, 5.9]])
    E = orc.forward(O, P, pos, g)
    O_new, P_new, loss = orc.epie_update(O, P, pos, E, g)
    assert loss < 1e-20
    assert np.allclose(O_new, O, rtol=0, atol=1e-12) and np.allclose(P_new, P, rtol=0, atol=1e-12)


@pytest.mark.parametrize("c", [0.0, 0.375])
def test_multislice_update_is_normalised_negative_gradient(c):
    # one position, one mode, eps = 0: the detector update is minus the
    # amplitude-loss seed, so slice s receives -b_s prod_{l>s} a_l g_O[s]
    # (b_s = 1/max|psi_s|^2, a_l = 1/max|O_l|^2) and the probe
    # -prod_l a_l g_P
    S = 3
    g = geom(S, 1, c=c)
    O = np.exp(1j * 0.4 * RNG.standard_normal((S, 14, 14))) * (0.8 + 0.2 * RNG.random((S, 14, 14)))
    P = crand(1, 8, 8, scale=2.0)
    pos = np.array([[2.3, 3.6]])
    E = RNG.random((1, 8, 8)) * 10 + 0.5
    O_new, P_new, _ = orc.epie_update(O, P, pos, E, g, beta_O=1.0, beta_P=1.0)
    _, gO, gP = orc.gradient(O, P, pos, E, g)
    psis, _, n, _ = orc.forward_waves(O, P, pos, g)
    a = [1.0 / np.max(np.abs(O[s]) ** 2) for s in range(S)]
    y0, x0 = n[0]
    for s in range(S):
        b = 1.0 / np.max(np.abs(psis[0, s, 0]) ** 2)
        want = -b * np.prod(a[s + 1:]) * gO[s]
        assert np.allclose(O_new[s] - O[s], want, rtol=1e-9, atol=1e-12 * np.abs(want).max())
        outside = np.ones((14, 14), bool)
        outside[y0:y0 + 8, x0:x0 + 8] = False
        assert np.all(O_new[s][outside] == O[s][outside])
    assert np.allclose(P_new - P, -np.prod(a) * gP, rtol=1e-9, atol=1e-12 * np.abs(gP).max())


def test_probe_update_is_group_mean_and_steps_scale():
    g = geom(2, 2, c=0.375, eps=1e-3)
    O = np.exp(1j * 0.3 * RNG.standard_normal((2, 14, 14)))
    P = crand(2, 8, 8)
    pos = np.array([[0.4, 0.1], [5.2, 4.9]])
    E = RNG.random((2, 8, 8)) * 5
    O1, P1, _ = orc.epie_update(O, P, pos, E, g, beta_O=1.0, beta_P=1.0)
    O2, P2, _ = orc.epie_update(O, P, pos, E, g, beta_O=0.25, beta_P=0.5)
    assert np.allclose(O2 - O, 0.25 * (O1 - O), rtol=1e-12, atol=1e-14)
    assert np.allclose(P2 - P, 0.5 * (P1 - P), rtol=1e-12, atol=1e-14)
    # the group update is the sum (object) and mean (probe) of the
    # one-position updates, since every position sees the same O and P
    parts = [orc.epie_update(O, P, pos[j:j + 1], E[j:j + 1], g) for j in range(2)]
    assert np.allclose(O1 - O, sum(p[0] - O for p in parts), rtol=1e-11, atol=1e-13)
    assert np.allclose(P1 - P, sum(p[1] - P for p in parts) / 2, rtol=1e-11, atol=1e-13)


def test_epie_needs_the_amplitude_model():
    g = orc.Geom(S=1, K=1, h=8, w=8, H=14, W=14, loss=orc.POISSON, eps=1.0)
    with pytest.raises(ValueError):
        orc.epie_update(np.ones((1, 14, 14)), np.ones((1, 8, 8)), np.zeros((1, 2)), np.ones((1, 8, 8)), g)
