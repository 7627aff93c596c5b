"""LSQML group update (arXiv 2505.14372 §3.3.2) through the C-ABI against the
FP64 oracle: the object and probe updates (new minus old) element by
element, the group's illumination and transmission sums, and the one-position
projection onto the data.  Tolerance: relative L2 <= 1e-4 (the update is a
ratio of sums of the gradient chain's FP32 terms; the regularisers delta and
gamma are set to a few per cent of the sums they guard, so no pixel divides
two near-zero FP32 sums)."""
import numpy as np
import pytest
import torch

import oracle as orc
from gpu_util import dev, host, problem, rel_l2
from paper_2505_14372_b300 import Context, PtychoError

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N,S,K,H,W,n_pos,B,c", [
    (64, 1, 1, 90, 90, 9, 6, 0.0),
    (64, 3, 2, 100, 100, 9, 7, 0.375),
    (192, 2, 2, 230, 230, 4, 3, 0.0),
])
def test_lsqml_update_parity(N, S, K, H, W, n_pos, B, c):
    geom, og, P, O, pos = problem(7 * N + S, S, K, N, H, W, n_pos, loss="amplitude", eps=1e-3, c=c, edge=True)
    geom.waves = "recompute"
    rng = np.random.default_rng(19)
    I_exp = rng.poisson(orc.forward(O, P, pos, og) * 0.8 + 0.5).astype(np.float32)
    idx = rng.permutation(n_pos)[:B].astype(np.int32)
    # regularisers: a few per cent of the group's largest sums
    _, _, Wg, Tg = orc.lsqml_directions(O, P, pos[idx], I_exp[idx], og)[:4]
    dO_, dP_, gam = 0.05 * Wg.max(), 0.05 * Tg.max(), 1e-3
    kw = dict(beta_O=0.9, beta_P=0.7, delta_O=dO_, delta_P=dP_, gamma=gam)
    ctx = Context(geom, max_batch=B)
    Od, Pd = dev(O), dev(P)
    il = torch.zeros((S, H, W), dtype=torch.float32, device="cuda")
    tr = torch.zeros((N, N), dtype=torch.float32, device="cuda")
    loss = ctx.lsqml_step(Od, Pd, dev(pos), dev(I_exp), dev(idx), illum_acc=il, trans_acc=tr, **kw)
    ctx.check_status()
    rO, rP, rl, rW, rT = orc.lsqml_update(O, P, pos[idx], I_exp[idx], og, **kw)
    assert abs(float(loss.item()) - rl) <= 1e-4 * abs(rl)
    assert rel_l2(host(il), rW) < 1e-5 and rel_l2(host(tr), rT) < 1e-5
    assert rel_l2(host(Od) - O, rO - O) < 1e-4
    assert rel_l2(host(Pd) - P, rP - P) < 1e-4
    # the running sums replace the group's own
    Od2, Pd2 = dev(O), dev(P)
    ctx.lsqml_step(Od2, Pd2, dev(pos), dev(I_exp), dev(idx), illum_prev=2 * il, trans_prev=2 * tr, **kw)
    sO, sP, *_ = orc.lsqml_update(O, P, pos[idx], I_exp[idx], og, illum=2 * rW, trans=2 * rT, **kw)
    assert rel_l2(host(Od2) - O, sO - O) < 1e-4 and rel_l2(host(Pd2) - P, sP - P) < 1e-4


def test_one_position_object_step_projects_onto_the_data():
    geom, og, P, O, pos = problem(5, 1, 1, 64, 80, 80, 1, loss="amplitude", eps=1e-6)
    geom.waves = "recompute"
    I_exp = (orc.forward(O, P, pos, og) * 1.3).astype(np.float32)
    ctx = Context(geom, max_batch=1)
    Od = dev(O)
    ctx.lsqml_step(Od, dev(P), dev(pos), dev(I_exp), dev(np.zeros(1, np.int32)), beta_O=1.0, beta_P=0.0)
    I_new = orc.forward(host(Od), P, pos, og)
    assert rel_l2(I_new, I_exp) < 1e-4


def test_lsqml_argument_checks():
    geom, og, P, O, pos = problem(3, 2, 2, 64, 80, 80, 4)
    I_exp = np.ones((4, 64, 64), np.float32)
    idx = np.arange(4, dtype=np.int32)
    geom.waves = "store"
    with pytest.raises(PtychoError):
        Context(geom, max_batch=4).lsqml_step(dev(O), dev(P), dev(pos), dev(I_exp), dev(idx))
    geom.waves, geom.loss, geom.eps = "recompute", "poisson", 0.8
    with pytest.raises(PtychoError):
        Context(geom, max_batch=4).lsqml_step(dev(O), dev(P), dev(pos), dev(I_exp), dev(idx))
