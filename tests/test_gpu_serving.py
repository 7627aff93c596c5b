"""Serving runtime (ptycho_submit / ptycho_poll): continuous batching of
requests with different shapes, HBM admission, results equal alone and in
the mix, and equal to the plain step path (arXiv 2505.14372 §2.3 job model,
§3.2 solver)."""
import numpy as np
import pytest
import torch

import oracle as orc
from gpu_util import dev, host, problem, rel_l2
from paper_2505_14372_b300 import AdamState, Context, PtychoError, Server, adam_opt, make_groups

pytestmark = pytest.mark.gpu

GB = 1 << 30


def request(seed, S, K, N, H, W, n_pos, loss="poisson"):
    geom, og, P, O, pos = problem(seed, S, K, N, H, W, n_pos, loss=loss, eps=0.8 if loss == "poisson" else 1e-3)
    geom.waves = "recompute"
    I_exp = np.random.default_rng(seed).poisson(orc.forward(O, P, pos, og) + 0.3).astype(np.float32)
    return geom, P, pos, I_exp


REQS = [
    dict(seed=1, S=2, K=2, N=64, H=80, W=84, n_pos=30),
    dict(seed=2, S=1, K=1, N=64, H=90, W=72, n_pos=21),
    dict(seed=3, S=3, K=2, N=128, H=150, W=144, n_pos=10),
    dict(seed=4, S=2, K=1, N=192, H=200, W=200, n_pos=6),
]


def run_alone(i, iters=3, batch=8, budget=8 * GB):
    r = request(**REQS[i])
    srv = Server(budget, 4)
    t = srv.submit(r[0], r[2], r[3], r[1], iterations=iters, batch=batch, seed=11, opt=adam_opt(1e-2, 1e-3))
    srv.wait(t)
    out = srv.poll(t, r[0])
    st = srv.stats()
    srv.close()
    return out, st


@pytest.mark.parametrize("budget,launches_per_step", [(8 * GB, 1), (2 * GB, 2)])
def test_served_result_equals_plain_step_path(budget, launches_per_step):
    geom, P, pos, I_exp = request(**REQS[0])
    out, st = run_alone(0, budget=budget)
    assert out["state"] == "done" and out["iterations_done"] == 3
    # 8 GB holds the position-major scratch of the 64 x 64 class (one tile
    # launch per step); 2 GB does not (a forward + recomputing adjoint pair);
    # 3 iterations of 4 groups, one request per tick
    assert st["launches"] == 12 * launches_per_step
    # plain path: same groups, same Adam steps, one ptycho_step per group
    ctx = Context(geom, max_batch=8)
    Od = torch.ones((geom.S, geom.H, geom.W), dtype=torch.complex64, device="cuda")
    Pd = dev(P)
    st = AdamState(geom)
    opt = adam_opt(1e-2, 1e-3)
    losses = []
    for it in range(3):
        perm = make_groups(len(pos), 8, seed=11, iteration=it, mode="sparse")
        for g0 in range(0, len(pos), 8):
            idx = dev(perm[g0:g0 + 8].astype(np.int32))
            losses.append(float(ctx.step(Od, Pd, st, opt, dev(pos), dev(I_exp), idx)[0].item()))
    assert rel_l2(out["O"], host(Od)) < 1e-4 and rel_l2(out["P"], host(Pd)) < 1e-4
    assert np.allclose(out["loss"], losses, rtol=1e-4)


def test_results_equal_alone_and_in_the_mix():
    alone = [run_alone(i)[0] for i in range(len(REQS))]
    srv = Server(16 * GB, 8)
    reqs = [request(**q) for q in REQS]
    tickets = [srv.submit(r[0], r[2], r[3], r[1], iterations=3, batch=8, seed=11, opt=adam_opt(1e-2, 1e-3))
               for r in reqs]
    for t in tickets:
        srv.wait(t)
    st = srv.stats()
    assert st["finished"] == len(REQS) and st["failed"] == 0
    assert st["p50_iter_ms"] > 0 and st["p99_iter_ms"] >= st["p50_iter_ms"] and st["positions_per_s"] > 0
    for r, t, a in zip(reqs, tickets, alone):
        o = srv.poll(t, r[0])
        assert o["state"] == "done"
        assert rel_l2(o["O"], a["O"]) < 1e-4 and rel_l2(o["P"], a["P"]) < 1e-4
        assert np.allclose(o["loss"], a["loss"], rtol=1e-4)
        srv.release(t)
    with pytest.raises(PtychoError):
        srv.poll(tickets[0])
    srv.close()


def oracle_trajectory(geom, P, pos, I_exp, iters, batch, seed, lr_O, lr_P):
    """The FP64 oracle's steps over the groups the server forms (the same
    seeded grouping), from a vacuum object and the request's probe."""
    og = orc.Geom(S=geom.S, K=geom.K, h=geom.N, w=geom.N, H=geom.H, W=geom.W, dx=geom.dx, lam=geom.lam,
                  dz=geom.dz, bandlimit=geom.bandlimit, loss={"amplitude": 0, "poisson": 1}[geom.loss],
                  eps=geom.eps, c=geom.c)
    O = np.ones((geom.S, geom.H, geom.W), np.complex128)
    Pc = P.astype(np.complex128)
    mO, vO, mP, vP = np.zeros_like(O), np.zeros(O.shape), np.zeros_like(Pc), np.zeros(Pc.shape)
    t, losses = 0, []
    for it in range(iters):
        perm = make_groups(len(pos), batch, seed=seed, iteration=it, mode="sparse")
        for g0 in range(0, len(pos), batch):
            t += 1
            O, Pc, mO, vO, mP, vP, L, _ = orc.step(O, Pc, mO, vO, mP, vP, t, pos, I_exp, perm[g0:g0 + batch], og,
                                                   lr_O, lr_P)
            losses.append(L)
    return O, Pc, np.array(losses)


def test_served_results_match_the_oracle_in_the_mix():
    """Two requests of different window sizes served together (their steps
    share launches): each result follows the FP64 oracle's trajectory over
    the same groups (loss of every step, final object and probe)."""
    picks = [0, 3]
    reqs = [request(**REQS[i]) for i in picks]
    srv = Server(16 * GB, 4)
    tickets = [srv.submit(r[0], r[2], r[3], r[1], iterations=2, batch=8, seed=13, opt=adam_opt(1e-2, 1e-3))
               for r in reqs]
    for t in tickets:
        srv.wait(t)
    for r, t in zip(reqs, tickets):
        o = srv.poll(t, r[0])
        assert o["state"] == "done"
        O, P, L = oracle_trajectory(r[0], r[1], r[2], r[3], 2, 8, 13, 1e-2, 1e-3)
        assert len(o["loss"]) == len(L)
        assert np.allclose(o["loss"], L, rtol=1e-4)
        assert rel_l2(o["O"], O) < 1e-4 and rel_l2(o["P"], P) < 1e-4
    srv.close()


def test_admission_by_budget_and_rejection():
    r = request(**REQS[2])
    big = request(seed=9, S=2, K=1, N=128, H=140, W=140, n_pos=4)
    tiny = Server(1 << 20, 2)   # 1 MiB cannot hold even the recompute scratch
    with pytest.raises(PtychoError) as e:
        tiny.submit(big[0], big[2], np.zeros((4, 128, 128), np.float32), big[1], iterations=1, batch=4)
    assert e.value.code == -3
    tiny.close()
    # more requests than active slots: queued, admitted as slots free up
    budget = 2 * GB
    srv = Server(budget, 2)
    tickets = [srv.submit(r[0], r[2], r[3], r[1], iterations=2, batch=5, seed=k) for k in range(5)]
    peak = 0
    while srv.stats()["finished"] < 5:
        st = srv.stats()
        peak = max(peak, st["admitted_bytes"])
        assert st["admitted_bytes"] <= budget
    for t in tickets:
        srv.wait(t)
    st = srv.stats()
    assert st["finished"] == 5 and st["admitted"] == 5 and st["queue_depth"] == 0 and st["failed"] == 0
    srv.close()
