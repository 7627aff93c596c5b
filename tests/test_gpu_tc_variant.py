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

# mode: (intensity bound, gradient bound) for a 3-slice, 2-mode problem.
# TF32x3 keeps 22 significand bits of each operand and BF16x6 all 24, and
# both sum the leading products with round-to-nearest fp32 adds, so they
# stay within a small factor of the FFT path; BF16x3 keeps 16 bits (2^-16 =
# 1.5e-5 per operand, grown over the chain's ~30 one-dimensional passes);
# TF32 alone keeps 11.
BOUNDS = {"fft": (1e-4, 1e-4), "tf32x3": (1e-5, 2e-5), "bf16x3": (1e-3, 1e-3), "tf32": (2e-2, 5e-2),
          "bf16x6": (1e-5, 2e-5)}


@pytest.mark.parametrize("dft", ["tf32x3", "bf16x3", "tf32", "bf16x6"])
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
    # the near-fp32 splits stay within a small factor of the FFT path
    if dft in ("tf32x3", "bf16x6"):
        assert eI < 4 * errs["fft"][0] and eO < 4 * errs["fft"][2] and eP < 4 * errs["fft"][3], errs


@pytest.mark.parametrize("dft", ["tf32x3", "bf16x6"])
def test_split_modes_meet_the_multislice_bound_at_full_depth(dft):
    """20 slices, 8 modes, 192 x 192 windows (the multislice workload's
    depth), 4 positions: the near-fp32 splits keep intensities, loss and
    both gradients within 1e-5 of the FP64 oracle (the multislice bound is
    1e-4; two bf16 parts, 16 significand bits, reach 2e-4 here)."""
    geom, og, P, O, pos = problem(93, 20, 8, 192, 230, 230, 4, loss="poisson", eps=0.8)
    I_exp = np.random.default_rng(4).poisson(orc.forward(O, P, pos, og) + 0.4).astype(np.float32)
    L, rO, rP = orc.gradient(O, P, pos, I_exp, og)
    rI = orc.forward(O, P, pos, og)
    geom.dft = dft
    ctx = Context(geom, max_batch=4)
    I = host(ctx.forward(dev(O), dev(P), dev(pos)))
    loss, gO, gP = ctx.adjoint(dev(O), dev(P), dev(pos), dev(I_exp))
    ctx.check_status()
    errs = (rel_l2(I, rI), abs(float(loss.item()) - L) / abs(L), rel_l2(host(gO), rO), rel_l2(host(gP), rP))
    print(dft, "at 20 slices, 8 modes, rel-L2 (I, loss, gO, gP):", errs)
    assert max(errs) < 1e-5, errs


# one forward and one inverse 2-D transform of the 192 x 192 tile: FFT
# (radix stages, FP32 rounding ~2^-24 per stage), TF32x3 and BF16x6
# (near-fp32 operands, leading sums rounded to nearest), BF16x3 (2^-16
# operands), TF32 (2^-11 operands)
DFT2_TOL = {"fft": 5e-7, "tf32x3": 5e-7, "bf16x6": 5e-7, "bf16x3": 3e-5, "tf32": 2e-3}


@pytest.mark.parametrize("dft", ["fft", "tf32x3", "bf16x3", "tf32", "bf16x6"])
def test_tile_dft_modes_match_the_oracle_dft(dft):
    from paper_2505_14372_b300.api import fft2_dft
    rng = np.random.default_rng(77)
    x = (rng.standard_normal((3, 192, 192)) + 1j * rng.standard_normal((3, 192, 192))).astype(np.complex64)
    X = host(fft2_dft(dev(x), dft))
    ef = rel_l2(X, orc.dft2(x.astype(np.complex128)))
    y = host(fft2_dft(dev(x), dft, inverse=True))
    ei = rel_l2(y, orc.idft2(x.astype(np.complex128)) * 192 * 192)
    print(dft, "2-D DFT rel-L2 forward / inverse:", ef, ei)
    assert ef < DFT2_TOL[dft] and ei < DFT2_TOL[dft]


def test_tensor_core_variant_only_for_192():
    geom, og, P, O, pos = problem(92, 1, 1, 64, 80, 80, 2)
    geom.dft = "tf32x3"
    with pytest.raises(PtychoError):
        Context(geom, max_batch=2)
