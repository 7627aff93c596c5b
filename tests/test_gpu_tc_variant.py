"""Tensor-core DFT variant of the 192x192 tile (DFT-matrix products with
split tf32 / bf16 operands) against the FP64 oracle: each mode's error is
bounded by what its arithmetic allows (arXiv 2505.14372 §2.3 reduced-precision
outlook; the forward model and gradient of §3, §3.2)."""
import numpy as np
import pytest

import oracle as orc
from gpu_util import dev, host, problem, rel_l2
from paper_2505_14372_b300 import Context, PtychoError

pytestmark = pytest.mark.gpu

# mode: (intensity bound, gradient bound) for a 3-slice, 2-mode problem
BOUNDS = {"fft": (1e-4, 1e-4), "tf32x3": (1e-4, 1e-4), "bf16x3": (1e-3, 1e-3), "tf32": (2e-2, 5e-2)}


@pytest.mark.parametrize("dft", ["tf32x3", "bf16x3", "tf32"])
def test_tensor_core_variant_error_vs_oracle(dft):
    geom, og, P, O, pos = problem(91, 3, 2, 192, 200, 204, 4, loss="poisson", eps=0.8, edge=True)
    I_exp = np.random.default_rng(3).poisson(orc.forward(O, P, pos, og) + 0.4).astype(np.float32)
    L, rO, rP = orc.gradient(O, P, pos, I_exp, og)
    rI = orc.forward(O, P, pos, og)
    errs = {}
    for mode in ("fft", dft):
        geom.dft = mode
        ctx = Context(geom, max_batch=4)
        I = host(ctx.forward(dev(O), dev(P), dev(pos)))
        loss, gO, gP = ctx.adjoint(dev(O), dev(P), dev(pos), dev(I_exp))
        ctx.check_status()
        errs[mode] = (rel_l2(I, rI), abs(float(loss.item()) - L) / abs(L), rel_l2(host(gO), rO), rel_l2(host(gP), rP))
    bI, bG = BOUNDS[dft]
    eI, eL, eO, eP = errs[dft]
    assert eI < bI and eL < bI and eO < bG and eP < bG, errs
    print(dft, "rel-L2 (I, loss, gO, gP):", errs[dft], "fft:", errs["fft"])
    # split tf32 recovers fp32-level accuracy: within a small factor of the FFT path
    if dft == "tf32x3":
        assert eI < max(50 * errs["fft"][0], 1e-6), errs


def test_tensor_core_variant_only_for_192():
    geom, og, P, O, pos = problem(92, 1, 1, 64, 80, 80, 2)
    geom.dft = "tf32x3"
    with pytest.raises(PtychoError):
        Context(geom, max_batch=2)
