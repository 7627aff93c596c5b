"""Deterministic gradient sums (geometry flag `deterministic`): every
position's object-patch and probe-spectrum gradient is kept apart and the
sums over the group run in position order, so the gradients of §3.2 (and a
step's Adam update) are bit-identical from run to run, while the default
path adds them with float atomics in whatever order the clusters finish.
Both agree with the FP64 oracle and with each other within the multislice
tolerance."""
import dataclasses

import numpy as np
import pytest
import torch

import oracle as orc
from gpu_util import dev, host, problem, rel_l2
from paper_2505_14372_b300 import AdamState, Context, PtychoError, adam_opt

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N,S,K,H,W,B", [(64, 2, 2, 96, 90, 37), (192, 3, 2, 230, 240, 9)])
def test_deterministic_gradients_bitwise_repeatable(N, S, K, H, W, B):
    geom, og, P, O, pos = problem(90 + N, S, K, N, H, W, B, loss="poisson", eps=0.8, edge=True)
    I_exp = np.random.default_rng(3).poisson(orc.forward(O, P, pos, og) + 0.4).astype(np.float32)
    Od, Pd, pd, Ed = dev(O), dev(P), dev(pos), dev(I_exp)
    det = Context(dataclasses.replace(geom, waves="recompute", deterministic=True), max_batch=B)
    runs = [det.adjoint(Od, Pd, pd, Ed) for _ in range(3)]
    det.check_status()
    g0 = [host(t) for t in runs[0][1:]]
    for r in runs[1:]:
        assert np.array_equal(host(r[1]), g0[0]) and np.array_equal(host(r[2]), g0[1])
    atomic = Context(dataclasses.replace(geom, waves="recompute"), max_batch=B)
    la, gOa, gPa = atomic.adjoint(Od, Pd, pd, Ed)
    assert rel_l2(g0[0], host(gOa)) < 1e-5 and rel_l2(g0[1], host(gPa)) < 1e-5
    L, rO, rP = orc.gradient(O, P, pos, I_exp, og)
    assert rel_l2(g0[0], rO) < 1e-4 and rel_l2(g0[1], rP) < 1e-4
    assert abs(float(runs[0][0].item()) - L) < 1e-4 * abs(L)


def test_deterministic_steps_bitwise_repeatable():
    """Three Adam steps over groups in a fixed order, twice from the same
    start: identical objects, probes and moments bit for bit."""
    geom, og, P, O, pos = problem(95, 2, 2, 128, 150, 156, 24, loss="poisson", eps=0.8)
    geom = dataclasses.replace(geom, waves="recompute", deterministic=True)
    I_exp = np.random.default_rng(4).poisson(orc.forward(O, P, pos, og) + 0.4).astype(np.float32)
    groups = [np.array(g, np.int32) for g in ([3, 7, 1, 20, 11, 5, 0, 9], [2, 4, 6, 8, 10, 12, 14, 16],
                                              [23, 22, 21, 19, 18, 17, 15, 13])]
    outs = []
    for _ in range(2):
        ctx = Context(geom, max_batch=8)
        Od, Pd = dev(O), dev(P)
        st = AdamState(geom)
        for g in groups:
            ctx.step(Od, Pd, st, adam_opt(1e-2, 1e-3), dev(pos), dev(I_exp), dev(g))
        ctx.check_status()
        outs.append([host(t) for t in (Od, Pd, st.mO, st.vO, st.mP, st.vP)])
        ctx.close()
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


def test_deterministic_needs_the_recomputed_fft_path():
    geom, og, P, O, pos = problem(96, 1, 1, 64, 80, 80, 2)
    with pytest.raises(PtychoError):
        Context(dataclasses.replace(geom, waves="store", deterministic=True), max_batch=2)
    with pytest.raises(PtychoError):
        Context(dataclasses.replace(geom, wave_prec="f16", deterministic=True), max_batch=2)
