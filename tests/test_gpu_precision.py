"""Reduced-precision storage of the entry waves (binary16 / bfloat16 copies
read by the object-gradient term, the 16-bit wavefields of arXiv 2505.14372
§2.2) against the oracle that rounds the same copies, through the C-ABI.

Tolerances: the kernels' FP32 entry waves differ from the oracle's by a
relative e ~ 1e-5 (20 slices), so a fraction ~ e/u of the stored parts round
to the other neighbour, each off by ~u relative (u = 2^-11 binary16,
2^-8 bfloat16): relative L2 ~ sqrt(e/u) u on top of the FP32 path's 1e-4,
i.e. 2e-4 (binary16) and 4e-4 (bfloat16).  Everything that does not read the
stored copies (loss, probe gradient) keeps the FP32 tolerances."""
import numpy as np
import pytest

import oracle as orc
from gpu_util import dev, host, problem, rel_l2
from paper_2505_14372_b300 import Context

pytestmark = pytest.mark.gpu

TOL = {"f16": 2e-4, "bf16": 4e-4}


@pytest.mark.parametrize("fmt", ["f16", "bf16"])
@pytest.mark.parametrize("N,S,K,H,W,B,waves", [
    (64, 3, 2, 100, 100, 7, "store"),
    (64, 3, 2, 100, 100, 7, "recompute"),
    (192, 4, 3, 230, 230, 3, "recompute"),
    (128, 2, 2, 160, 160, 5, "store"),
])
def test_reduced_precision_waves_match_rounding_oracle(fmt, N, S, K, H, W, B, waves):
    geom, og, P, O, pos = problem(N + 7 * S, S, K, N, H, W, B, loss="poisson", eps=0.8, edge=True)
    geom.waves = waves
    geom.wave_prec = fmt
    I_exp = np.random.default_rng(9).poisson(orc.forward(O, P, pos, og)).astype(np.float32)
    ctx = Context(geom, max_batch=B)
    loss_d, gO, gP = ctx.adjoint(dev(O), dev(P), dev(pos), dev(I_exp))
    ctx.check_status()
    L, rO, rP = orc.gradient(O, P, pos, I_exp, og, wave_fmt=fmt)
    assert abs(float(loss_d.item()) - L) <= 1e-4 * abs(L)
    assert rel_l2(host(gP), rP) < 1e-4
    e_round = rel_l2(host(gO), rO)
    assert e_round < TOL[fmt]
    if fmt == "bf16":
        # the copies really are bfloat16: the unrounded oracle is much further
        _, rO32, _ = orc.gradient(O, P, pos, I_exp, og)
        assert rel_l2(host(gO), rO32) > 4 * e_round

