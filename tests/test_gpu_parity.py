"""GPU path (through the C-ABI) against the FP64 oracle, element by element,
on seeded inputs spanning several tiles, ragged batches and the edge cases
(arXiv 2505.14372 §3, §3.1, §3.2)."""
import numpy as np
import pytest
import torch

import oracle as orc
from gpu_util import dev, host, problem, rel_l2
from paper_2505_14372_b300 import AdamState, Context, PtychoError, adam_opt, fft2

pytestmark = pytest.mark.gpu

TOL_S1 = 1e-5    # single slice intensities and loss
TOL_MS = 1e-4    # multislice and all gradients


@pytest.mark.parametrize("N", [64, 128, 192, 256])
def test_fft2_tile_matches_dft(N):
    rng = np.random.default_rng(N)
    x = (rng.standard_normal((3, N, N)) + 1j * rng.standard_normal((3, N, N))).astype(np.complex64)
    X = host(fft2(dev(x)))
    assert rel_l2(X, orc.dft2(x.astype(np.complex128))) < 2e-6
    y = host(fft2(dev(x), inverse=True))
    assert rel_l2(y, orc.idft2(x.astype(np.complex128)) * N * N) < 2e-6


CASES = [
    # (N, S, K, H, W, B, loss)
    (64, 1, 1, 100, 90, 37, "amplitude"),
    (64, 3, 2, 80, 80, 11, "poisson"),
    (128, 1, 3, 150, 140, 9, "poisson"),
    (128, 2, 2, 140, 140, 5, "amplitude"),
    (192, 1, 2, 200, 210, 5, "amplitude"),
    (192, 3, 2, 200, 200, 3, "poisson"),
    (256, 2, 1, 260, 270, 3, "amplitude"),
    # the multislice workload's depth and modes (20 slices, 8 modes, 192 x 192)
    # on a reduced object, element by element
    (192, 20, 8, 230, 230, 4, "poisson"),
]


def _tol(S):
    return TOL_S1 if S == 1 else TOL_MS


@pytest.mark.parametrize("N,S,K,H,W,B,loss", CASES)
def test_forward_parity(N, S, K, H, W, B, loss):
    geom, og, P, O, pos = problem(N * 7 + S, S, K, N, H, W, B, loss=loss, eps=0.8 if loss == "poisson" else 1e-3,
                                  edge=True)
    ctx = Context(geom, max_batch=B)
    I = host(ctx.forward(dev(O), dev(P), dev(pos)))
    ctx.check_status()
    ref = orc.forward(O, P, pos, og)
    assert rel_l2(I, ref) < _tol(S)


@pytest.mark.parametrize("waves", ["store", "recompute"])
@pytest.mark.parametrize("N,S,K,H,W,B,loss", CASES)
def test_adjoint_parity(N, S, K, H, W, B, loss, waves):
    geom, og, P, O, pos = problem(N * 11 + S, S, K, N, H, W, B, loss=loss, eps=0.8 if loss == "poisson" else 1e-3,
                                  edge=True)
    geom.waves = waves
    rng = np.random.default_rng(5)
    I_exp = rng.poisson(orc.forward(O, P, pos, og) * 1.1 + 0.2).astype(np.float32)
    ctx = Context(geom, max_batch=B)
    loss_d, gO, gP = ctx.adjoint(dev(O), dev(P), dev(pos), dev(I_exp))
    ctx.check_status()
    L, rO, rP = orc.gradient(O, P, pos, I_exp, og)
    assert abs(float(loss_d.item()) - L) <= _tol(S) * abs(L)
    assert rel_l2(host(gO), rO) < TOL_MS
    assert rel_l2(host(gP), rP) < TOL_MS


@pytest.mark.parametrize("waves", ["store", "recompute"])
@pytest.mark.parametrize("N,S,K,H,W,B", [(64, 2, 2, 90, 84, 9), (192, 2, 2, 200, 206, 3)])
def test_adjoint_parity_anscombe(N, S, K, H, W, B, waves):
    """The Anscombe noise model (§3.1: least squares on sqrt(I + 3/8)),
    loss and gradients against the oracle."""
    geom, og, P, O, pos = problem(N * 13 + S, S, K, N, H, W, B, loss="anscombe", eps=1e-3, c=0.375, edge=True)
    geom.waves = waves
    I_exp = np.random.default_rng(15).poisson(orc.forward(O, P, pos, og) * 1.1 + 0.2).astype(np.float32)
    ctx = Context(geom, max_batch=B)
    loss_d, gO, gP = ctx.adjoint(dev(O), dev(P), dev(pos), dev(I_exp))
    ctx.check_status()
    L, rO, rP = orc.gradient(O, P, pos, I_exp, og)
    assert abs(float(loss_d.item()) - L) <= TOL_MS * abs(L)
    assert rel_l2(host(gO), rO) < TOL_MS
    assert rel_l2(host(gP), rP) < TOL_MS


def test_adjoint_accumulate_and_empty_batch():
    geom, og, P, O, pos = problem(3, 2, 2, 64, 90, 90, 6)
    I_exp = np.full((6, 64, 64), 2.0, np.float32)
    ctx = Context(geom, max_batch=6)
    Od, Pd = dev(O), dev(P)
    _, gO1, gP1 = ctx.adjoint(Od, Pd, dev(pos[:3]), dev(I_exp[:3]))
    _, gO2, gP2 = ctx.adjoint(Od, Pd, dev(pos[3:]), dev(I_exp[3:]), gO=gO1.clone(), gP=gP1.clone(), accumulate=True)
    _, gOa, gPa = ctx.adjoint(Od, Pd, dev(pos), dev(I_exp))
    assert rel_l2(host(gO2), host(gOa)) < 1e-5 and rel_l2(host(gP2), host(gPa)) < 1e-5
    # B = 0: zero gradients and zero loss
    l0, g0, p0 = ctx.adjoint(Od, Pd, dev(pos[:0]), dev(I_exp[:0]))
    assert float(l0.item()) == 0.0 and float(g0.abs().max()) == 0.0 and float(p0.abs().max()) == 0.0


def test_vjp_parity():
    geom, og, P, O, pos = problem(21, 3, 2, 128, 150, 150, 4)
    gI = np.random.default_rng(2).standard_normal((4, 128, 128)).astype(np.float32)
    ctx = Context(geom, max_batch=4)
    gO, gP = ctx.vjp(dev(O), dev(P), dev(pos), dev(gI))
    rO, rP = orc.vjp(O, P, pos, gI, og)
    assert rel_l2(host(gO), rO) < TOL_MS and rel_l2(host(gP), rP) < TOL_MS


def test_autograd_function_matches_oracle_vjp():
    from paper_2505_14372_b300 import simulate
    geom, og, P, O, pos = problem(23, 2, 2, 64, 80, 80, 5)
    ctx = Context(geom, max_batch=5)
    Ot = dev(O).requires_grad_(True)
    Pt = dev(P).requires_grad_(True)
    I = simulate(ctx, Ot, Pt, dev(pos))
    wts = torch.linspace(0.5, 1.5, 64 * 64, device="cuda").reshape(64, 64)
    (I * wts).sum().backward()
    rO, rP = orc.vjp(O, P, pos, np.broadcast_to(host(wts), (5, 64, 64)), og)
    assert rel_l2(host(Ot.grad), rO) < TOL_MS and rel_l2(host(Pt.grad), rP) < TOL_MS


@pytest.mark.parametrize("waves", ["store", "recompute"])
def test_step_parity(waves):
    geom, og, P, O, pos = problem(31, 2, 2, 64, 96, 96, 12, loss="poisson", eps=0.8)
    geom.waves = waves
    I_exp = np.random.default_rng(9).poisson(orc.forward(O, P, pos, og) * 0.9 + 0.5).astype(np.float32)
    idx = np.array([5, 0, 7, 3, 11, 2], np.int32)
    ctx = Context(geom, max_batch=6)
    Od, Pd = dev(O), dev(P)
    st = AdamState(geom)
    opt = adam_opt(lr_O=1e-2, lr_P=1e-3)
    stats = host(ctx.step(Od, Pd, st, opt, dev(pos), dev(I_exp), dev(idx)))
    z = np.zeros
    O2, P2, mO, vO, mP, vP, L, gn = orc.step(O, P, z(O.shape, complex), z(O.shape), z(P.shape, complex), z(P.shape),
                                             1, pos, I_exp, idx, og, 1e-2, 1e-3)
    assert st.t == 1
    assert abs(stats[0] - L) < TOL_S1 * 10 * abs(L) and abs(stats[1] - gn) < TOL_MS * gn
    assert rel_l2(host(Od), O2) < 1e-5 and rel_l2(host(Pd), P2) < 1e-5
    assert rel_l2(host(st.mO), mO) < TOL_MS and rel_l2(host(st.vO), vO) < TOL_MS


def test_out_of_bounds_position_is_flagged():
    geom, og, P, O, pos = problem(41, 1, 1, 64, 80, 80, 3)
    pos[1] = [16.6, 0.0]   # rounds to 17: 17 + 64 > 80
    ctx = Context(geom, max_batch=3)
    ctx.forward(dev(O), dev(P), dev(pos))
    with pytest.raises(PtychoError) as e:
        ctx.check_status()
    assert e.value.code == -2
    ctx.check_status()  # cleared


def test_invalid_arguments():
    geom, og, P, O, pos = problem(43, 1, 1, 64, 80, 80, 3)
    geom.N = 96
    with pytest.raises(PtychoError):
        Context(geom, max_batch=3)
    geom.N = 64
    ctx = Context(geom, max_batch=2)
    with pytest.raises(PtychoError):
        ctx.forward(dev(O), dev(P), dev(pos))   # B = 3 > max_batch


@pytest.mark.parametrize("N,S,K,H,W", [(64, 2, 2, 80, 84), (192, 2, 2, 200, 200)])
def test_position_gradient_parity(N, S, K, H, W):
    geom, og, P, O, pos = problem(61 + N, S, K, N, H, W, 5, loss="poisson", eps=0.8)
    I_exp = np.random.default_rng(8).poisson(orc.forward(O, P, pos, og) * 1.2 + 0.3).astype(np.float32)
    ctx = Context(geom, max_batch=5)
    loss, gO, gP, gpos = ctx.adjoint_positions(dev(O), dev(P), dev(pos), dev(I_exp))
    ref = orc.position_gradient(O, P, pos, I_exp, og)
    assert rel_l2(host(gpos), ref) < TOL_MS
    # the other outputs are those of ptycho_adjoint
    L, rO, rP = orc.gradient(O, P, pos, I_exp, og)
    assert rel_l2(host(gO), rO) < TOL_MS and rel_l2(host(gP), rP) < TOL_MS


def test_gaussian_noise_model_parity():
    geom, og, P, O, pos = problem(71, 2, 2, 64, 84, 80, 7, loss="amplitude")
    geom.loss, geom.c, geom.eps = "gaussian", 4.0, 0.0
    og.loss, og.c, og.eps = orc.GAUSSIAN, 4.0, 0.0
    I_exp = np.random.default_rng(4).poisson(orc.forward(O, P, pos, og) * 1.1 + 0.5).astype(np.float32)
    ctx = Context(geom, max_batch=7)
    loss, gO, gP = ctx.adjoint(dev(O), dev(P), dev(pos), dev(I_exp))
    L, rO, rP = orc.gradient(O, P, pos, I_exp, og)
    assert abs(float(loss.item()) - L) < TOL_MS * abs(L)
    assert rel_l2(host(gO), rO) < TOL_MS and rel_l2(host(gP), rP) < TOL_MS


@pytest.mark.parametrize("reg", [dict(l2_obj=0.05, tikhonov=0.05, layers=0.5, l2_probe=1e-3),
                                 dict(tv=0.5, tv_layers=2.0, tv_eps=0.02, l2_probe=1e-3)])
def test_step_with_regularizers_parity(reg):
    geom, og, P, O, pos = problem(73, 3, 2, 64, 90, 90, 10, loss="poisson", eps=0.8)
    I_exp = np.random.default_rng(6).poisson(orc.forward(O, P, pos, og) + 0.5).astype(np.float32)
    idx = np.array([1, 4, 7, 9, 0], np.int32)
    ctx = Context(geom, max_batch=5)
    Od, Pd = dev(O), dev(P)
    st = AdamState(geom)
    opt = adam_opt(lr_O=1e-2, lr_P=1e-3, reg_obj_l2=reg.get("l2_obj", 0.0), reg_obj_tikhonov=reg.get("tikhonov", 0.0),
                   reg_obj_layers=reg.get("layers", 0.0), reg_probe_l2=reg.get("l2_probe", 0.0),
                   reg_obj_tv=reg.get("tv", 0.0), reg_obj_layers_tv=reg.get("tv_layers", 0.0),
                   reg_tv_eps=reg.get("tv_eps", 1e-3))
    stats = host(ctx.step(Od, Pd, st, opt, dev(pos), dev(I_exp), dev(idx)))
    z = np.zeros
    O2, P2, *_, L, gn = orc.step(O, P, z(O.shape, complex), z(O.shape), z(P.shape, complex), z(P.shape), 1, pos,
                                 I_exp, idx, og, 1e-2, 1e-3, reg=reg)
    assert abs(stats[0] - L) < TOL_MS * abs(L) and abs(stats[1] - gn) < TOL_MS * gn
    assert rel_l2(host(Od), O2) < 1e-5 and rel_l2(host(Pd), P2) < 1e-5


@pytest.mark.parametrize("N,S,K,H,W", [(64, 2, 2, 84, 84), (192, 2, 2, 200, 200)])
def test_step_with_fixed_probe_parity(N, S, K, H, W):
    """A step that keeps the probe fixed (§3.2 with only the object among the
    optimised variables): the object moves as the oracle's, the probe does
    not, and the reported gradient norm still covers the probe gradient."""
    geom, og, P, O, pos = problem(75 + N, S, K, N, H, W, 6, loss="poisson", eps=0.8)
    I_exp = np.random.default_rng(9).poisson(orc.forward(O, P, pos, og) + 0.5).astype(np.float32)
    idx = np.array([5, 2, 0, 3], np.int32)
    ctx = Context(geom, max_batch=4)
    Od, Pd = dev(O), dev(P)
    st = AdamState(geom)
    stats = host(ctx.step(Od, Pd, st, adam_opt(lr_O=1e-2, lr_P=1e-2, update_probe=False), dev(pos), dev(I_exp),
                          dev(idx)))
    z = np.zeros
    O2, P2, *_, L, gn = orc.step(O, P, z(O.shape, complex), z(O.shape), z(P.shape, complex), z(P.shape), 1, pos,
                                 I_exp, idx, og, 1e-2, 1e-2, update_probe=False)
    assert np.array_equal(host(Pd), P.astype(np.complex64))
    assert abs(stats[0] - L) < TOL_MS * abs(L) and abs(stats[1] - gn) < TOL_MS * gn
    assert rel_l2(host(Od), O2) < 1e-5


def test_fused_step_end_between_other_calls():
    """The 64 x 64 step ends in one fused launch that also clears the
    gradient accumulators for the next call (which then skips its memsets).
    Steps interleaved with adjoint and VJP calls on the same context must
    each still match the oracle (§3.2)."""
    geom, og, P, O, pos = problem(97, 1, 2, 64, 96, 92, 10, loss="poisson", eps=0.8)
    geom.waves = "recompute"
    I_exp = np.random.default_rng(98).poisson(orc.forward(O, P, pos, og) + 0.5).astype(np.float32)
    ctx = Context(geom, max_batch=10)
    Od, Pd = dev(O), dev(P)
    st = AdamState(geom)
    opt = adam_opt(lr_O=1e-2, lr_P=1e-3)
    z = np.zeros
    rO, rP = O.astype(np.complex128), P.astype(np.complex128)
    mO, vO, mP, vP = z(O.shape, complex), z(O.shape), z(P.shape, complex), z(P.shape)
    groups = [np.array(g, np.int32) for g in ([0, 3, 6, 9], [1, 4, 7], [2, 5, 8, 0, 1], [9, 8, 7, 6, 5, 4])]
    for t, g in enumerate(groups, start=1):
        stats = host(ctx.step(Od, Pd, st, opt, dev(pos), dev(I_exp), dev(g)))
        rO, rP, mO, vO, mP, vP, L, gn = orc.step(rO, rP, mO, vO, mP, vP, t, pos, I_exp, g, og, 1e-2, 1e-3)
        assert abs(stats[0] - L) < TOL_S1 * 10 * abs(L) and abs(stats[1] - gn) < TOL_MS * gn, t
        assert rel_l2(host(Od), rO) < 1e-5 and rel_l2(host(Pd), rP) < 1e-5, t
        # a different call right after the step, on the updated state
        Oc, Pc = host(Od).astype(np.complex128), host(Pd).astype(np.complex128)
        if t % 2:
            loss, gO, gP = ctx.adjoint(Od, Pd, dev(pos[:7]), dev(I_exp[:7]))
            L2, eO, eP = orc.gradient(Oc, Pc, pos[:7], I_exp[:7], og)
            assert abs(float(loss.item()) - L2) < TOL_S1 * 10 * abs(L2)
            assert rel_l2(host(gO), eO) < TOL_MS and rel_l2(host(gP), eP) < TOL_MS
        else:
            gI = np.random.default_rng(t).standard_normal((5, 64, 64)).astype(np.float32)
            gO, gP = ctx.vjp(Od, Pd, dev(pos[:5]), dev(gI))
            eO, eP = orc.vjp(Oc, Pc, pos[:5], gI, og)
            assert rel_l2(host(gO), eO) < TOL_MS and rel_l2(host(gP), eP) < TOL_MS
    ctx.check_status()
