"""Pins of the oracle's LSQML update (arXiv 2505.14372 §3.3.2): with one
position, one mode and one slice, a full object step (or a full probe step on
a phase object) moves the model's exit wave onto the modulus-constrained one,
so the simulated pattern equals the data; the update directions are minus
the amplitude-loss gradient (already pinned by finite differences);
consistent data is a fixed point; the running sums replace the group's."""
import numpy as np
import pytest

import oracle as orc

RNG = np.random.default_rng(41)


def crand(*shape, scale=1.0):
    return scale * (RNG.standard_normal(shape) + 1j * RNG.standard_normal(shape))


def geom(S, K, c=0.0, eps=0.0):
    return orc.Geom(S=S, K=K, h=8, w=8, H=14, W=14, dx=0.1, lam=0.0197, dz=(10.0,) * (S - 1),
                    bandlimit=2 / 3, loss=orc.AMPLITUDE, eps=eps, c=c)


def test_object_step_projects_onto_the_data():
    g = geom(1, 1)
    O = np.exp(1j * 0.4 * RNG.standard_normal((1, 14, 14))) * (0.7 + 0.3 * RNG.random((1, 14, 14)))
    P = crand(1, 8, 8, scale=2.0)
    pos = np.array([[2.3, 4.6]])
    E = RNG.random((1, 8, 8)) * 30 + 1
    O2, P2, _, W, T = orc.lsqml_update(O, P, pos, E, g, beta_O=1.0, beta_P=0.0)
    assert np.allclose(P2, P)
    assert np.allclose(orc.forward(O2, P, pos, g), E, rtol=1e-9)


def test_probe_step_projects_onto_the_data_for_a_phase_object():
    g = geom(1, 1)
    O = np.exp(1j * 0.4 * RNG.standard_normal((1, 14, 14)))       # |O| = 1
    P = crand(1, 8, 8, scale=2.0)
    pos = np.array([[3.4, 1.8]])                                   # sub-pixel
    E = RNG.random((1, 8, 8)) * 30 + 1
    O2, P2, _, _, _ = orc.lsqml_update(O, P, pos, E, g, beta_O=0.0, beta_P=1.0)
    assert np.allclose(O2, O)
    assert np.allclose(orc.forward(O, P2, pos, g), E, rtol=1e-9)


@pytest.mark.parametrize("S,K", [(1, 2), (3, 2)])
def test_directions_are_minus_the_amplitude_gradient(S, K):
    g = geom(S, K)
    O = np.exp(1j * 0.3 * RNG.standard_normal((S, 14, 14))) * (0.8 + 0.2 * RNG.random((S, 14, 14)))
    P = crand(K, 8, 8)
    pos = np.array([[0.3, 1.2], [4.6, 2.2], [2.0, 5.9]])
    E = RNG.random((3, 8, 8)) * 10 + 0.5
    NO, NP, W, T, chis, psis, n, d, loss = orc.lsqml_directions(O, P, pos, E, g)
    L, gO, gP = orc.gradient(O, P, pos, E, g)
    assert np.isclose(loss, L)
    assert np.allclose(NO, -gO, rtol=1e-10, atol=1e-12 * np.abs(gO).max())
    assert np.allclose(NP, -gP, rtol=1e-10, atol=1e-12 * np.abs(gP).max())
    # illumination and transmission of the group
    Wr = np.zeros(W.shape)
    Tr = np.zeros(T.shape)
    for j in range(3):
        y0, x0 = n[j]
        Wr[:, y0:y0 + 8, x0:x0 + 8] += np.sum(np.abs(psis[j]) ** 2, axis=1)
        Tr += np.prod(np.abs(O[:, y0:y0 + 8, x0:x0 + 8]) ** 2, axis=0)
    assert np.allclose(W, Wr) and np.allclose(T, Tr)


def test_consistent_data_is_a_fixed_point_and_running_sums_replace_the_groups():
    g = geom(2, 2)
    O = np.exp(1j * 0.4 * RNG.standard_normal((2, 14, 14)))
    P = crand(2, 8, 8)
    pos = np.array([[0.3, 1.2], [4.6, 2.2], [2.0, 5.9]])
    E = orc.forward(O, P, pos, g)
    O2, P2, loss, W, T = orc.lsqml_update(O, P, pos, E, g, delta_O=1e-3, delta_P=1e-3, gamma=1e-9)
    assert loss < 1e-20
    assert np.allclose(O2, O, atol=1e-12) and np.allclose(P2, P, atol=1e-12)
    E2 = E * (0.8 + 0.4 * RNG.random(E.shape))
    a = orc.lsqml_update(O, P, pos, E2, g, delta_O=1e-3, delta_P=1e-3, gamma=1e-9)
    b = orc.lsqml_update(O, P, pos, E2, g, delta_O=1e-3, delta_P=1e-3, gamma=1e-9, illum=a[3], trans=a[4])
    assert np.allclose(a[0], b[0]) and np.allclose(a[1], b[1])


def test_lsqml_needs_the_amplitude_model():
    g = orc.Geom(S=1, K=1, h=8, w=8, H=14, W=14, loss=orc.POISSON, eps=1.0)
    with pytest.raises(ValueError):
        orc.lsqml_update(np.ones((1, 14, 14)), np.ones((1, 8, 8)), np.zeros((1, 2)), np.ones((1, 8, 8)), g)
