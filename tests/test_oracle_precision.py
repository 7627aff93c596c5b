"""Pins of the oracle's reduced-precision storage of entry waves (the 16-bit
wavefields that arXiv 2505.14372 §2.2 names as future work): rounding rule
cases worked by hand, the rounding-error bounds of each format, and the
invariants of the gradient when only the stored entry waves are rounded."""
import numpy as np
import pytest

import oracle as orc

RNG = np.random.default_rng(23)


def r(x, fmt):
    return orc.round_storage(np.asarray(x, dtype=np.float64) + 0j, fmt).real


# values worked out by hand: (input, f16 result, bf16 result)
CASES = [
    (1.5, 1.5, 1.5),                                  # exact in both
    (-0.375, -0.375, -0.375),
    (1 + 2.0**-11, 1.0, 1.0),                         # f16 tie -> even (1.0)
    (1 + 3 * 2.0**-11, 1 + 2.0**-9, 1.0),             # f16 tie -> even (1 + 2^-9)
    (1 + 2.0**-8, 1 + 2.0**-8, 1.0),                  # bf16 tie -> even (1.0)
    (1 + 3 * 2.0**-8, 1 + 3 * 2.0**-8, 1 + 2.0**-6),  # bf16 tie -> even
    (1 + 2.0**-8 + 2.0**-20, 1 + 2.0**-8, 1 + 2.0**-7),  # bf16 above the tie
    (65504.0, 65504.0, 65536.0),                      # f16 max; bf16 rounds up
    (2.0**-14, 2.0**-14, 2.0**-14),                   # f16 smallest normal
    (3 * 2.0**-25, 2.0**-23, 3 * 2.0**-25),           # f16 subnormal spacing 2^-24: tie -> even
    (2.0**100 * 1.25, np.inf, 2.0**100 * 1.25),       # beyond f16's range
]
pytestmark = pytest.mark.filterwarnings("ignore:overflow encountered in cast")


@pytest.mark.parametrize("x,f16,bf16", CASES)
def test_rounding_cases_by_hand(x, f16, bf16):
    assert r(x, "f16") == f16
    assert r(x, "bf16") == bf16
    assert r(-x, "bf16") == -bf16  # symmetric
    assert r(x, "f32") == np.float32(x)


def test_rounding_error_bounds_and_idempotence():
    x = RNG.standard_normal(20000) * 10.0 ** RNG.uniform(-3, 3, 20000)
    for fmt, u in (("f16", 2.0**-11), ("bf16", 2.0**-8)):
        y = r(x, fmt)
        normal = np.abs(x) >= (2.0**-14 if fmt == "f16" else 2.0**-126)
        assert np.all(np.abs(y - x)[normal] <= u * np.abs(x[normal]) * (1 + 1e-6))
        # below binary16's normal range the absolute spacing is 2^-24
        assert np.all(np.abs(y - x)[~normal] <= 2.0**-25 * (1 + 1e-6))
        assert np.array_equal(r(y, fmt), y)                  # idempotent
        # round to nearest: no representable neighbour is closer
        assert np.mean(np.abs(y - x)[normal] / (u * np.abs(x[normal]))) < 0.6
    # bf16 keeps every value with at most 8 significant bits exactly
    m = RNG.integers(128, 256, 1000) * 2.0 ** RNG.integers(-20, 20, 1000)
    assert np.array_equal(r(m, "bf16"), m)


def test_gradient_with_rounded_waves():
    g = orc.Geom(S=3, K=2, h=8, w=8, H=12, W=12, dx=0.1, lam=0.0197, dz=(10.0, 10.0),
                 bandlimit=2 / 3, loss=orc.POISSON, eps=0.5)
    O = np.exp(1j * 0.4 * RNG.standard_normal((3, 12, 12)))
    P = 3.0 * (RNG.standard_normal((2, 8, 8)) + 1j * RNG.standard_normal((2, 8, 8)))
    pos = np.array([[0.2, 0.4], [1.7, 3.1], [3.6, 0.9], [2.9, 3.3]])
    E = RNG.poisson(orc.forward(O, P, pos, g) * 0.9).astype(np.float64)
    l0, gO0, gP0 = orc.gradient(O, P, pos, E, g)
    for fmt, u in (("f16", 2.0**-11), ("bf16", 2.0**-8)):
        l1, gO1, gP1 = orc.gradient(O, P, pos, E, g, wave_fmt=fmt)
        # only the object-gradient term reads the stored waves
        assert l1 == l0
        assert np.array_equal(gP1, gP0)
        # g_O = sum conj(psi) g_phi and each stored psi moves by at most u |psi|:
        # the relative change is of order u (not zero, not much larger)
        rel = np.linalg.norm(gO1 - gO0) / np.linalg.norm(gO0)
        assert u / 50 < rel < 2 * u
