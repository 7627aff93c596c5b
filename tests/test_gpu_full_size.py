"""Parity at the full workload sizes, in the launch configuration bench.py
times (one group of B positions per call, the workload's object, window,
slices and modes, recomputed entry waves), on outputs the FP64 oracle can
compute one position at a time:

* intensities of sampled positions of the group, element by element;
* the loss and object gradient of one sampled position j, recovered from
  the full-size calls by linearity in the positions: (call on the whole
  group) minus (call on the group without j).  The other positions'
  contributions cancel up to FP32 summation order: with ~d positions
  overlapping a pixel the difference carries about d * 2^-24 relative error,
  far inside the tolerance; the probe gradient sums all B positions, so its
  difference carries ~B * 2^-24 (3e-5 at B = 512) on top of 1e-4.

Tolerances as in the parity tests: 1e-5 single slice, 1e-4 multislice and
gradients."""
import numpy as np
import pytest
import torch

import oracle as orc
from gpu_util import dev, host, rel_l2
from paper_2505_14372_b300 import Context, Geometry, synth
from paper_2505_14372_b300.api import make_groups

pytestmark = pytest.mark.gpu


def setup(w):
    wl = synth.WORKLOADS[w]
    rng = np.random.default_rng(100 + w)
    # a seeded weak phase object at the workload's full size (phase_object at
    # 1024 x 1024 x 20 would take minutes on the host)
    O = np.exp(1j * 0.25 * rng.standard_normal((wl.S, wl.H, wl.W))).astype(np.complex64)
    P = synth.probe_modes(wl)
    pos_all = synth.raster_positions(wl)
    idx = make_groups(wl.P, wl.B, seed=5, iteration=0, mode="sparse")[:wl.B]
    loss = {0: "amplitude", 1: "poisson"}[wl.loss]
    geom = Geometry(S=wl.S, K=wl.K, N=wl.N, H=wl.H, W=wl.W, dx=wl.dx, lam=wl.lam, dz=wl.dz,
                    bandlimit=wl.bandlimit, loss=loss, eps=wl.eps, c=wl.c, waves="recompute")
    og = orc.Geom(S=wl.S, K=wl.K, h=wl.N, w=wl.N, H=wl.H, W=wl.W, dx=wl.dx, lam=wl.lam, dz=wl.dz,
                  bandlimit=wl.bandlimit, loss=wl.loss, eps=wl.eps, c=wl.c)
    return wl, geom, og, O, P, pos_all[idx]


@pytest.mark.parametrize("w", [1, 2, 3])
def test_full_size_forward_sampled(w):
    wl, geom, og, O, P, pos = setup(w)
    ctx = Context(geom, max_batch=wl.B)
    I = host(ctx.forward(dev(O), dev(P), dev(pos)))
    ctx.check_status()
    tol = 1e-5 if wl.S == 1 else 1e-4
    for j in (0, wl.B // 2, wl.B - 1):
        ref = orc.forward(O, P, pos[j:j + 1].astype(np.float64), og)[0]
        assert rel_l2(I[j], ref) < tol, j


@pytest.mark.parametrize("w", [1, 2, 3])
def test_full_size_gradient_of_one_position_by_linearity(w):
    wl, geom, og, O, P, pos = setup(w)
    j = wl.B // 3
    E = synth.cbed_like_patterns(wl, wl.B).astype(np.float32)
    ctx = Context(geom, max_batch=wl.B)
    Od, Pd = dev(O), dev(P)
    L_all, gO_all, gP_all = ctx.adjoint(Od, Pd, dev(pos), dev(E))
    rest = np.r_[0:j, j + 1:wl.B]
    L_rest, gO_rest, gP_rest = ctx.adjoint(Od, Pd, dev(pos[rest]), dev(E[rest]))
    ctx.check_status()
    Lj, rO, rP = orc.gradient(O, P, pos[j:j + 1].astype(np.float64), E[j:j + 1], og)
    assert abs(float(L_all.item()) - float(L_rest.item()) - Lj) <= 1e-4 * abs(Lj)
    n = np.floor(pos[j].astype(np.float64) + 0.5).astype(int)
    win = (slice(None), slice(n[0], n[0] + wl.N), slice(n[1], n[1] + wl.N))
    gO_j = host(gO_all)[win] - host(gO_rest)[win]
    assert rel_l2(gO_j, rO[win]) < 1e-4
    gP_j = host(gP_all) - host(gP_rest)
    assert rel_l2(gP_j, rP) < 1e-4 + 4 * wl.B * 2.0**-24
