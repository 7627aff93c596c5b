"""Calls that take a stream only enqueue work, so they can be captured in a
CUDA graph and replayed on new inputs (the launch-overhead-free way to run a
reconstruction loop): forward and adjoint of the multislice model (§3,
§3.1, §3.2) captured once, replayed after the inputs changed in place, and
compared with eager calls on the same inputs."""
import numpy as np
import pytest
import torch

from gpu_util import dev, host, problem, rel_l2
from paper_2505_14372_b300 import AdamState, Context, adam_opt

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N,S,K", [(64, 2, 2), (192, 2, 2)])
def test_forward_adjoint_capture_and_replay(N, S, K):
    B = 5
    geom, og, P, O, pos = problem(41, S, K, N, N + 40, N + 36, B, loss="poisson", eps=0.8)
    geom.waves = "recompute"
    rng = np.random.default_rng(42)
    I_exp = rng.poisson(3.0, size=(B, N, N)).astype(np.float32)
    ctx = Context(geom, max_batch=B)
    Od, Pd, posd, Id = dev(O), dev(P), dev(pos), dev(I_exp)

    def calls():
        I = ctx.forward(Od, Pd, posd)
        loss, gO, gP = ctx.adjoint(Od, Pd, posd, Id)
        return I, loss, gO, gP

    # warm-up outside the capture (torch's recipe: on a side stream)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        calls()
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        out = calls()
    ctx.check_status()

    # new inputs, written in place into the captured tensors
    geom2, _, P2, O2, pos2 = problem(43, S, K, N, N + 40, N + 36, B, loss="poisson", eps=0.8)
    Od.copy_(dev(O2))
    Pd.copy_(dev(P2))
    posd.copy_(dev(pos2))
    graph.replay()
    torch.cuda.synchronize()
    replayed = [host(t) for t in out]
    eager = [host(t) for t in calls()]
    torch.cuda.synchronize()
    ctx.check_status()
    assert rel_l2(replayed[0], eager[0]) < 1e-6  # intensities: the same kernels on the same inputs
    assert abs(float(replayed[1]) - float(eager[1])) <= 1e-6 * abs(float(eager[1]))
    # gradients are scattered with float atomics: equal up to summation order
    assert rel_l2(replayed[2], eager[2]) < 1e-5 and rel_l2(replayed[3], eager[3]) < 1e-5
    # and the replay really used the new inputs
    first = host(ctx.forward(dev(O), dev(P), dev(pos)))
    assert rel_l2(replayed[0], first) > 1e-2


def test_captured_step_replays_with_a_device_step_count():
    """A whole Adam step (§3.2) captured once and replayed on successive
    groups equals the same steps run eagerly, with the step count kept in
    device memory (ptycho_set_step_counter)."""
    N, S, K, B, n_pos = 64, 2, 2, 8, 24
    geom, og, P, O, pos = problem(61, S, K, N, 112, 108, n_pos, loss="poisson", eps=0.8)
    geom.waves = "recompute"
    I_exp = np.random.default_rng(62).poisson(3.0, size=(n_pos, N, N)).astype(np.float32)
    ctx = Context(geom, max_batch=B)
    posd, Id = dev(pos), dev(I_exp)
    opt = adam_opt(1e-2, 1e-3)
    groups = [np.roll(np.arange(n_pos, dtype=np.int32), -5 * i)[:B].copy() for i in range(6)]

    Oe, Pe, ste = dev(O), dev(P), AdamState(geom)
    eager_loss = []
    for gidx in groups:
        eager_loss.append(float(ctx.step(Oe, Pe, ste, opt, posd, Id, dev(gidx))[0].item()))

    t = torch.zeros(1, dtype=torch.int64, device="cuda")
    ctx.set_step_counter(t)
    Og, Pg, stg = dev(O), dev(P), AdamState(geom)
    idx = torch.empty(B, dtype=torch.int32, device="cuda")
    stats = torch.zeros(2, dtype=torch.float64, device="cuda")
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        ctx.step(Og, Pg, stg, opt, posd, Id, idx, stats=stats)
    replay_loss = []
    for gidx in groups:
        idx.copy_(dev(gidx))
        graph.replay()
        replay_loss.append(float(stats[0].item()))
    torch.cuda.synchronize()
    ctx.set_step_counter(None)
    ctx.check_status()
    assert int(t.item()) == len(groups)
    assert np.allclose(replay_loss, eager_loss, rtol=1e-5)
    assert rel_l2(host(Og), host(Oe)) < 1e-5 and rel_l2(host(Pg), host(Pe)) < 1e-5
