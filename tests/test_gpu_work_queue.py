"""Launches with more scan positions than clusters.

A launch of one problem (all positions cost the same) hands cluster c the
entries c, c + clusters, ... of its processing order; a launch that mixes
problems of one window size (served requests: positions cost S slices times
K modes of their own problem) hands each cluster its first entry and then
lets it claim the next one from the launch's work queue whenever it
finishes a position, the last cluster out resetting the queue.  Cases: one
problem against the FP64 oracle with out-of-object positions skipped in
between (§3.1, §3.2), against launches too small to need a second round,
two launches back to back, a captured launch replayed; and served mixes
whose every launch holds more positions than clusters, each request's
result equal to the same request served alone (one problem per launch), and
one of them to the oracle's trajectory."""
import numpy as np
import pytest
import torch

import oracle as orc
from gpu_util import dev, host, problem, rel_l2
from paper_2505_14372_b300 import Context, PtychoError, Server, adam_opt

pytestmark = pytest.mark.gpu

TOL = 1e-4  # multislice loss and gradients against the oracle


def _sms():
    return torch.cuda.get_device_properties(0).multi_processor_count


def test_multi_round_launch_matches_oracle_with_skipped_positions():
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


def test_multi_round_launch_equals_single_round_chunks_and_repeats():
    # 64 x 64 windows: a few hundred resident CTAs; 1024 positions take several rounds
    N, S, K, H, W, B = 64, 2, 2, 200, 190, 1024
    geom, og, P, O, pos = problem(602, S, K, N, H, W, B, loss="amplitude")
    geom.waves = "recompute"
    I_exp = np.random.default_rng(18).poisson(3.0, size=(B, N, N)).astype(np.float32)
    ctx = Context(geom, max_batch=B)
    Od, Pd, posd, Id = dev(O), dev(P), dev(pos), dev(I_exp)
    l1, gO1, gP1 = ctx.adjoint(Od, Pd, posd, Id)
    l1, gO1, gP1 = float(l1.item()), host(gO1), host(gP1)
    # the same launch again
    l2, gO2, gP2 = ctx.adjoint(Od, Pd, posd, Id)
    assert abs(float(l2.item()) - l1) <= 1e-6 * abs(l1)
    assert rel_l2(host(gO2), gO1) < 1e-5 and rel_l2(host(gP2), gP1) < 1e-5
    # chunks of 32 positions: every launch in one round of clusters
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


def test_multi_round_launch_capture_and_replay():
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
    for _ in range(3):
        graph.replay()
        torch.cuda.synchronize()
        rep = [host(t) for t in out]
        assert abs(float(rep[0]) - float(eager[0])) <= 1e-6 * abs(float(eager[0]))
        assert rel_l2(rep[1], eager[1]) < 1e-5 and rel_l2(rep[2], eager[2]) < 1e-5
    ctx.check_status()


GB = 1 << 30


def _served(reqs, iters=3, budget=16 * GB):
    """Serves the requests together (all resident, one launch per tick) and
    returns their results and the server's statistics."""
    srv = Server(budget, len(reqs))
    # hold the worker until every request is in, so that all are admitted
    # before the first tick and share every launch
    srv.inject_stall(500.0)
    ts = [srv.submit(g, pos, I, P, iterations=iters, batch=pos.shape[0], seed=5 + k, opt=adam_opt(1e-2, 1e-3))
          for k, (g, P, pos, I) in enumerate(reqs)]
    for t in ts:
        srv.wait(t)
    out = [srv.poll(t, r[0]) for t, r in zip(ts, reqs)]
    st = srv.stats()
    srv.close()
    return out, st


def _request(seed, S, K, n_pos, N=192, H=330, W=320):
    geom, og, P, O, pos = problem(seed, S, K, N, H, W, n_pos, loss="poisson", eps=0.8)
    geom.waves = "recompute"
    I_exp = np.random.default_rng(seed).poisson(orc.forward(O, P, pos, og) + 0.3).astype(np.float32)
    return geom, P, pos, I_exp


def test_served_mix_through_the_queue_equals_each_request_alone():
    # 192 x 192 windows: at most 74 clusters; every tick's launch holds the
    # one group of each request: 60 + 50 = 110 positions of different cost
    reqs = [_request(611, 2, 2, 60), _request(612, 1, 1, 50)]
    mix, st = _served(reqs)
    assert st["launches"] == 3  # one position-major launch per tick, three ticks
    for k, r in enumerate(reqs):
        alone, _ = _served([r])
        a, m = alone[0], mix[k]
        assert m["state"] == "done" and a["state"] == "done"
        assert np.allclose(m["loss"], a["loss"], rtol=1e-4), (k, m["loss"], a["loss"])
        assert rel_l2(m["O"], a["O"]) < 1e-4 and rel_l2(m["P"], a["P"]) < 1e-4


def test_served_mix_through_the_queue_follows_the_oracle():
    from test_gpu_serving import oracle_trajectory
    reqs = [_request(613, 1, 1, 40, H=260, W=250), _request(614, 2, 1, 45, H=260, W=250)]
    mix, _ = _served(reqs, iters=2)
    g, P, pos, I = reqs[1]
    O_ref, P_ref, L_ref = oracle_trajectory(g, P, pos, I, 2, pos.shape[0], 6, 1e-2, 1e-3)
    m = mix[1]
    assert len(m["loss"]) == len(L_ref)
    assert np.allclose(m["loss"], L_ref, rtol=1e-4)
    assert rel_l2(m["O"], O_ref) < 1e-4 and rel_l2(m["P"], P_ref) < 1e-4
