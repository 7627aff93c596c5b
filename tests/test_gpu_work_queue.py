"""Work queue of the position-major loss + adjoint launch.

Once a launch holds more scan positions than it runs clusters, each cluster
takes its first position directly and then claims the next entry of the
processing order from the launch's queue whenever it finishes one; the last
cluster to leave resets the queue for the next launch.  The cases below
hold more positions than a B300 runs clusters at once, so the queue is in
use: the loss and gradients of §3.1 / §3.2 against the FP64 oracle with
out-of-object positions skipped in between, against launches small enough
to need no queue, two launches back to back, and a captured launch
replayed."""
import numpy as np
import pytest
import torch

import oracle as orc
from gpu_util import dev, host, problem, rel_l2
from paper_2505_14372_b300 import Context, PtychoError

pytestmark = pytest.mark.gpu

TOL = 1e-4  # multislice loss and gradients against the oracle


def _sms():
    return torch.cuda.get_device_properties(0).multi_processor_count


def test_queued_launch_matches_oracle_with_skipped_positions():
    # 192 x 192 windows run one 2-CTA cluster per two SMs at most
    N, S, K, H, W = 192, 2, 1, 400, 380
    B = _sms() // 2 + 50
    geom, og, P, O, pos = problem(601, S, K, N, H, W, B, loss="poisson", eps=0.8)
    geom.waves = "recompute"
    skipped = [10, B // 2, B - 3]
    for j in skipped:
        pos[j] = [H - N + 5.0, 10.0]  # the window leaves the object
    keep = np.array([j not in skipped for j in range(B)])
    I_exp = np.random.default_rng(17).poisson(
        orc.forward(O, P, pos[keep], og) * 1.1 + 0.2).astype(np.float32)
    I_all = np.zeros((B, N, N), np.float32)
    I_all[keep] = I_exp
    ctx = Context(geom, max_batch=B)
    loss, gO, gP = ctx.adjoint(dev(O), dev(P), dev(pos), dev(I_all))
    with pytest.raises(PtychoError) as e:
        ctx.check_status()
    assert e.value.code == -2
    L, rO, rP = orc.gradient(O, P, pos[keep], I_exp, og)
    assert abs(float(loss.item()) - L) <= TOL * abs(L)
    assert rel_l2(host(gO), rO) < TOL
    assert rel_l2(host(gP), rP) < TOL


def test_queued_launch_equals_unqueued_chunks_and_repeats():
    # 64 x 64 windows: a few hundred resident CTAs; 1024 positions exceed them
    N, S, K, H, W, B = 64, 2, 2, 200, 190, 1024
    geom, og, P, O, pos = problem(602, S, K, N, H, W, B, loss="amplitude")
    geom.waves = "recompute"
    I_exp = np.random.default_rng(18).poisson(3.0, size=(B, N, N)).astype(np.float32)
    ctx = Context(geom, max_batch=B)
    Od, Pd, posd, Id = dev(O), dev(P), dev(pos), dev(I_exp)
    l1, gO1, gP1 = ctx.adjoint(Od, Pd, posd, Id)
    l1, gO1, gP1 = float(l1.item()), host(gO1), host(gP1)
    # the second launch finds the queue reset by the first
    l2, gO2, gP2 = ctx.adjoint(Od, Pd, posd, Id)
    assert abs(float(l2.item()) - l1) <= 1e-6 * abs(l1)
    assert rel_l2(host(gO2), gO1) < 1e-5 and rel_l2(host(gP2), gP1) < 1e-5
    # chunks of 32 positions: no launch needs the queue
    small = Context(geom, max_batch=32)
    lc = 0.0
    gOc = gPc = None
    for c0 in range(0, B, 32):
        l, gOc, gPc = small.adjoint(Od, Pd, posd[c0:c0 + 32], Id[c0:c0 + 32], gO=gOc, gP=gPc,
                                    accumulate=c0 > 0)
        lc += float(l.item())
    ctx.check_status()
    small.check_status()
    assert abs(lc - l1) <= 1e-5 * abs(l1)
    assert rel_l2(host(gOc), gO1) < 1e-5 and rel_l2(host(gPc), gP1) < 1e-5


def test_queued_launch_capture_and_replay():
    N, S, K, H, W = 192, 2, 1, 300, 310
    B = _sms() // 2 + 20
    geom, og, P, O, pos = problem(603, S, K, N, H, W, B, loss="poisson", eps=0.8)
    geom.waves = "recompute"
    I_exp = np.random.default_rng(19).poisson(3.0, size=(B, N, N)).astype(np.float32)
    ctx = Context(geom, max_batch=B)
    Od, Pd, posd, Id = dev(O), dev(P), dev(pos), dev(I_exp)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        ctx.adjoint(Od, Pd, posd, Id)
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        out = ctx.adjoint(Od, Pd, posd, Id)
    eager = [host(t) for t in ctx.adjoint(Od, Pd, posd, Id)]
    for _ in range(3):  # every replay starts from a reset queue
        graph.replay()
        torch.cuda.synchronize()
        rep = [host(t) for t in out]
        assert abs(float(rep[0]) - float(eager[0])) <= 1e-6 * abs(float(eager[0]))
        assert rel_l2(rep[1], eager[1]) < 1e-5 and rel_l2(rep[2], eager[2]) < 1e-5
    ctx.check_status()
