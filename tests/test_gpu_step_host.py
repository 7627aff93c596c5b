"""The host-buffer step (ptycho_step_host, §3.2 solver step on one group,
§2.2) equals the device-buffer step on the same group.  With more positions
than one round of clusters it copies the later positions' patterns on its
own stream while the first round computes, and runs the position-major
kernel as two launches; the result must not change."""
import numpy as np
import pytest
import torch

from gpu_util import dev, host, problem, rel_l2
from paper_2505_14372_b300 import AdamState, Context, PtychoError, adam_opt

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("B", [40, 200])
def test_step_host_equals_device_step(B):
    N = 192
    geom, og, P, O, pos = problem(51, 2, 2, N, 300, 296, B, loss="poisson", eps=0.8)
    geom.waves = "recompute"
    I_exp = np.random.default_rng(52).poisson(3.0, size=(B, N, N)).astype(np.float32)
    ctx = Context(geom, max_batch=B)
    opt = adam_opt(1e-2, 1e-3)

    O1, P1, st1 = dev(O), dev(P), AdamState(geom)
    stats = ctx.step(O1, P1, st1, opt, dev(pos), dev(I_exp), dev(np.arange(B, dtype=np.int32)))
    loss1 = float(stats[0].item())

    O2, P2, st2 = dev(O), dev(P), AdamState(geom)
    pos_h = torch.from_numpy(pos).pin_memory()
    I_h = torch.from_numpy(I_exp).pin_memory()
    loss2, _ = ctx.step_host(O2, P2, st2, opt, pos_h, I_h)
    torch.cuda.synchronize()
    ctx.check_status()
    assert abs(loss2 - loss1) <= 1e-6 * abs(loss1)
    # gradients are scattered with float atomics: equal up to summation order
    assert rel_l2(host(O2), host(O1)) < 1e-6 and rel_l2(host(P2), host(P1)) < 1e-6


def test_step_host_rejects_a_window_outside_the_object():
    N, B = 64, 4
    geom, og, P, O, pos = problem(53, 1, 1, N, 96, 96, B)
    geom.waves = "recompute"
    ctx = Context(geom, max_batch=B)
    bad = pos.copy()
    bad[2] = [96 - N + 1.0, 3.0]  # the window's last row leaves the object
    I_exp = np.ones((B, N, N), np.float32)
    with pytest.raises(PtychoError) as e:
        ctx.step_host(dev(O), dev(P), AdamState(geom), adam_opt(1e-3, 1e-4), bad, I_exp)
    assert e.value.code == -2
