"""Ten full-batch gradient-descent iterations of the single-slice,
single-mode workload (64 x 64 window, 128 x 128 phase object of Gaussian
atoms, 16 x 16 raster, amplitude loss, data simulated from the ground truth
with Poisson noise at 1e4 counts per pattern; arXiv 2505.14372 §3, §3.1,
§3.2): ptycho_step (FP32) against oracle.step (FP64) from the same start,
every iteration.  Checks that FP32 rounding does not drift the trajectory:
the loss of every iteration within 1e-5 (single slice) and the final object
and probe within 1e-4."""
import numpy as np
import pytest

import oracle as orc
from gpu_util import dev, host, rel_l2
from paper_2505_14372_b300 import AdamState, Context, Geometry, adam_opt, synth

pytestmark = pytest.mark.gpu


def test_single_slice_ten_full_batch_iterations_track_the_oracle():
    wl = synth.WORKLOADS[1]
    P0 = synth.probe_modes(wl)
    pos = synth.raster_positions(wl)
    O_true = synth.phase_object(wl)
    og = orc.Geom(S=1, K=1, h=wl.N, w=wl.N, H=wl.H, W=wl.W, dx=wl.dx, lam=wl.lam, dz=(), bandlimit=wl.bandlimit,
                  loss=orc.AMPLITUDE, eps=wl.eps, c=0.0)
    I_exp = synth.poisson_counts(orc.forward(O_true, P0, pos, og), wl.cid)
    geom = Geometry(S=1, K=1, N=wl.N, H=wl.H, W=wl.W, dx=wl.dx, lam=wl.lam, bandlimit=wl.bandlimit,
                    loss="amplitude", eps=wl.eps, c=0.0)
    lr_O, lr_P = 1e-2, 1e-2
    ctx = Context(geom, max_batch=wl.P)
    O = np.ones((1, wl.H, wl.W), np.complex64)
    Od, Pd = dev(O), dev(P0)
    st = AdamState(geom)
    opt = adam_opt(lr_O=lr_O, lr_P=lr_P)
    idx = np.arange(wl.P, dtype=np.int32)          # full batch, scan order
    posd, Id, idxd = dev(pos), dev(I_exp), dev(idx)
    rO, rP = O.astype(np.complex128), P0.astype(np.complex128)
    mO, vO = np.zeros_like(rO), np.zeros(rO.shape)
    mP, vP = np.zeros_like(rP), np.zeros(rP.shape)
    losses = []
    for t in range(1, 11):
        stats = host(ctx.step(Od, Pd, st, opt, posd, Id, idxd))
        rO, rP, mO, vO, mP, vP, L, gn = orc.step(rO, rP, mO, vO, mP, vP, t, pos, I_exp, idx, og, lr_O, lr_P)
        losses.append(L)
        assert abs(stats[0] - L) <= 1e-5 * abs(L), (t, stats[0], L)
        assert abs(stats[1] - gn) <= 1e-4 * gn, (t, stats[1], gn)
    ctx.check_status()
    assert st.t == 10
    assert rel_l2(host(Od), rO) < 1e-4
    assert rel_l2(host(Pd), rP) < 1e-4
    # the iterations make progress on consistent data
    assert losses[-1] < 0.9 * losses[0]
