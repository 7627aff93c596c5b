"""Writes tests/golden/oracle_tiny.json: the FP64 oracle's outputs on one
fixed tiny multislice mixed-state problem (two slices, two modes, 8x8 window,
12x12 object, four positions, amplitude / Poisson / Gaussian noise models,
the ePIE update).  It calls only oracle/ and the fixed inputs below.  The
fixture freezes the oracle: a later change to its arithmetic shows up as a
failing comparison and has to be regenerated with this script, naming in
its commit the passage of the paper (or the reading of it) that justifies
the change.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
import oracle as orc  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def inputs():
    rng = np.random.default_rng(20250514)
    O = np.exp(1j * 0.5 * rng.standard_normal((2, 12, 12))) * (0.8 + 0.2 * rng.random((2, 12, 12)))
    P = 2.0 * (rng.standard_normal((2, 8, 8)) + 1j * rng.standard_normal((2, 8, 8)))
    pos = np.array([[0.2, 0.4], [1.7, 3.1], [3.6, 0.9], [2.9, 3.3]])
    E = np.round(rng.random((4, 8, 8)) * 40.0)
    return O, P, pos, E


def geom(loss, eps, c):
    return orc.Geom(S=2, K=2, h=8, w=8, H=12, W=12, dx=0.1, lam=0.0197, dz=(10.0,), bandlimit=2 / 3,
                    loss=loss, eps=eps, c=c)


def cplx(z):
    z = np.asarray(z).ravel()
    return [[float(v.real), float(v.imag)] for v in z]


def compute():
    O, P, pos, E = inputs()
    out = {"_note": "written by tests/golden/make_golden.py from oracle/ only; see its docstring"}
    out["I"] = np.asarray(orc.forward(O, P, pos, geom(orc.AMPLITUDE, 1e-3, 0.0))).ravel().tolist()
    for name, (loss, eps, c) in {"amplitude": (orc.AMPLITUDE, 1e-3, 0.0), "anscombe": (orc.AMPLITUDE, 1e-3, 0.375),
                                 "poisson": (orc.POISSON, 0.8, 0.0), "gaussian": (orc.GAUSSIAN, 0.0, 3.0)}.items():
        L, gO, gP = orc.gradient(O, P, pos, E, geom(loss, eps, c))
        out[name] = {"loss": float(L), "gO_sample": cplx(gO[:, ::5, ::5]), "gP_sample": cplx(gP[:, ::3, ::3])}
    O2, P2, L = orc.epie_update(O, P, pos, E, geom(orc.AMPLITUDE, 1e-3, 0.0), beta_O=0.7, beta_P=0.4)
    out["epie"] = {"loss": float(L), "O_sample": cplx(O2[:, ::5, ::5]), "P_sample": cplx(P2[:, ::3, ::3])}
    return out


if __name__ == "__main__":
    with open(os.path.join(HERE, "oracle_tiny.json"), "w") as f:
        json.dump(compute(), f, indent=0)
    print("wrote", os.path.join(HERE, "oracle_tiny.json"))
