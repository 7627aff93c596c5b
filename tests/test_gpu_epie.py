"""ePIE / 3PIE group update (arXiv 2505.14372 §3.3.1) through the C-ABI
against the FP64 oracle: the object and probe updates (new minus old),
element by element, for single- and multi-slice, mixed-state problems, with
stored and recomputed entry waves (the recompute path at 192x192 runs the
position-major loss + adjoint kernel).  Tolerance: relative L2 <= 1e-4, the gradient's
(the update is the adjoint chain with per-slice scalar normalisers)."""
import numpy as np
import pytest
import torch

import oracle as orc
from gpu_util import dev, host, problem, rel_l2
from paper_2505_14372_b300 import Context, PtychoError

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N,S,K,H,W,n_pos,B,c,waves", [
    (64, 1, 1, 90, 90, 9, 6, 0.0, "store"),
    (64, 3, 2, 100, 100, 9, 7, 0.375, "recompute"),
    (128, 2, 3, 170, 170, 5, 4, 0.0, "store"),
    (192, 3, 2, 230, 230, 4, 3, 0.375, "recompute"),
])
def test_epie_update_parity(N, S, K, H, W, n_pos, B, c, waves):
    geom, og, P, O, pos = problem(5 * N + S, S, K, N, H, W, n_pos, loss="amplitude", eps=1e-3, c=c, edge=True)
    geom.waves = waves
    rng = np.random.default_rng(17)
    I_exp = rng.poisson(orc.forward(O, P, pos, og) * 0.8 + 0.5).astype(np.float32)
    idx = rng.permutation(n_pos)[:B].astype(np.int32)
    bO, bP = 0.8, 0.6
    ctx = Context(geom, max_batch=B)
    Od, Pd = dev(O), dev(P)
    loss = ctx.epie_step(Od, Pd, dev(pos), dev(I_exp), dev(idx), beta_O=bO, beta_P=bP)
    ctx.check_status()
    rO, rP, rl = orc.epie_update(O, P, pos[idx], I_exp[idx], og, beta_O=bO, beta_P=bP)
    assert abs(float(loss.item()) - rl) <= 1e-4 * abs(rl)
    assert rel_l2(host(Od) - O, rO - O) < 1e-4
    assert rel_l2(host(Pd) - P, rP - P) < 1e-4


def test_epie_held_probe_and_model_check():
    geom, og, P, O, pos = problem(3, 2, 2, 64, 80, 80, 4)
    I_exp = np.ones((4, 64, 64), np.float32)
    idx = np.arange(4, dtype=np.int32)
    ctx = Context(geom, max_batch=4)
    Pd = dev(P)
    ctx.epie_step(dev(O), Pd, dev(pos), dev(I_exp), dev(idx), beta_O=1.0, beta_P=0.0)
    assert torch.equal(Pd, dev(P))
    geom.loss, geom.eps = "poisson", 0.8
    ctxp = Context(geom, max_batch=4)
    with pytest.raises(PtychoError):
        ctxp.epie_step(dev(O), dev(P), dev(pos), dev(I_exp), dev(idx))
