"""Pins of the oracle's multislice forward model, noise models, gradient and
Adam step (arXiv 2505.14372 §3, §3.1, §3.2) against invariants, closed forms
and brute-force finite differences."""
import math

import numpy as np
import pytest

import oracle as orc

RNG = np.random.default_rng(11)


def crand(*shape, scale=1.0):
    return scale * (RNG.standard_normal(shape) + 1j * RNG.standard_normal(shape))


def phase_obj(S, H, W, amp=0.5):
    return np.exp(1j * amp * RNG.standard_normal((S, H, W)))


def tiny(S=2, K=2, h=8, w=8, H=12, W=12, loss=orc.AMPLITUDE, eps=1e-3, c=0.0,
         beta=2 / 3, dz=10.0):
    return orc.Geom(S=S, K=K, h=h, w=w, H=H, W=W, dx=0.1, lam=0.0197,
                    dz=tuple([dz] * (S - 1)), bandlimit=beta, loss=loss, eps=eps, c=c)


POS4 = np.array([[0.2, 0.4], [1.7, 3.1], [3.6, 0.9], [2.9, 3.3]])


# ------------------------------------------------------------- forward

def test_zero_thickness_multislice_is_projection():
    # dz = 0 and no band limit: the multislice product collapses to a single
    # slice with the product of all transmissions (projection approximation)
    g = tiny(S=3, K=2, dz=0.0, beta=0.0)
    O = phase_obj(3, 12, 12) * (0.8 + 0.2 * RNG.random((3, 12, 12)))
    P = crand(2, 8, 8)
    I3 = orc.forward(O, P, POS4, g)
    g1 = tiny(S=1, K=2, beta=0.0)
    I1 = orc.forward(np.prod(O, axis=0, keepdims=True), P, POS4, g1)
    assert np.allclose(I3, I1, rtol=1e-11, atol=1e-12 * I1.max())


def test_single_slice_integer_position_is_library_fft():
    g = tiny(S=1, K=3)
    O = crand(1, 12, 12)
    P = crand(3, 8, 8)
    pos = np.array([[2.0, 3.0], [0.0, 4.0]])
    I = orc.forward(O, P, pos, g)
    for j, (y, x) in enumerate(pos.astype(int)):
        ref = np.sum(np.abs(np.fft.fft2(P * O[0, y:y + 8, x:x + 8], norm="ortho")) ** 2, axis=0)
        assert np.allclose(I[j], ref, rtol=1e-11, atol=1e-12 * ref.max())


@pytest.mark.parametrize("S", [1, 3])
def test_vacuum_object_gives_probe_pattern(S):
    # O = 1: every position gives sum_k |B F_o P_k|^2 (band limit only when a
    # propagation happens), whatever the subpixel shift
    g = tiny(S=S, K=2)
    P = crand(2, 8, 8)
    I = orc.forward(np.ones((S, 12, 12), complex), P, POS4, g)
    mask = orc.bandlimit_mask(8, 8, g.bandlimit) if S > 1 else np.ones((8, 8), bool)
    ref = np.sum(np.abs(mask * np.fft.fft2(P, norm="ortho")) ** 2, axis=0)
    for j in range(len(POS4)):
        assert np.allclose(I[j], ref, rtol=1e-10, atol=1e-12 * ref.max())


def test_mode_sum_is_incoherent():
    g = tiny(S=2, K=3)
    O = phase_obj(2, 12, 12)
    P = crand(3, 8, 8)
    I = orc.forward(O, P, POS4, g)
    g1 = tiny(S=2, K=1)
    parts = sum(orc.forward(O, P[k:k + 1], POS4, g1) for k in range(3))
    assert np.allclose(I, parts, rtol=1e-12, atol=1e-13 * I.max())


def test_energy_conservation_for_phase_object():
    g = tiny(S=3, K=2, beta=0.0)
    P = crand(2, 8, 8)
    I = orc.forward(phase_obj(3, 12, 12), P, POS4, g)
    assert np.allclose(I.sum(axis=(1, 2)), np.sum(np.abs(P) ** 2), rtol=1e-11)


def test_translation_covariance():
    g = tiny(S=2, K=2, H=16, W=16)
    O = phase_obj(2, 16, 16)
    P = crand(2, 8, 8)
    pos = np.array([[1.3, 2.2], [0.6, 0.7]])
    Oshift = np.roll(O, (2, 3), axis=(1, 2))
    assert np.allclose(orc.forward(O, P, pos, g), orc.forward(Oshift, P, pos + [2, 3], g), rtol=1e-11)


def test_multislice_waves_follow_gaussian_beam():
    # vacuum object and a Gaussian entry wave: the entry wave of slice s is
    # the beam propagated over the sum of the first s gaps (closed form)
    n, dx, lam, s0 = 64, 0.1, 0.0197, 0.4
    dz = (8.0, 12.0, 5.0)
    g = orc.Geom(S=4, K=1, h=n, w=n, H=n, W=n, dx=dx, lam=lam, dz=dz, bandlimit=2 / 3)
    c = np.arange(n) - n // 2
    r2 = (c[:, None] ** 2 + c[None, :] ** 2) * dx * dx
    P = np.exp(-r2 / (2 * s0 * s0))[None].astype(complex)
    psis, _, _, _ = orc.forward_waves(np.ones((4, n, n), complex), P, [[0.0, 0.0]], g)
    z = 0.0
    for s in range(4):
        a = 2 * np.pi ** 2 * s0 * s0 + 1j * np.pi * lam * z
        ref = (2 * np.pi ** 2 * s0 * s0 / a) * np.exp(-np.pi ** 2 * r2 / a)
        assert np.max(np.abs(psis[0, s, 0] - ref)) < 1e-10
        if s < 3:
            z += dz[s]


def test_out_of_bounds_positions_rejected():
    g = tiny()
    with pytest.raises(ValueError):
        orc.forward(np.ones((2, 12, 12)), crand(2, 8, 8), [[4.6, 0.0]], g)
    with pytest.raises(ValueError):
        orc.forward(np.ones((2, 12, 12)), crand(2, 8, 8), [[-0.6, 0.0]], g)


# ---------------------------------------------------------------- loss

def test_loss_zero_at_data_and_derivative_by_fd():
    for loss, eps, c in [(orc.AMPLITUDE, 1e-3, 0.0), (orc.AMPLITUDE, 0.0, 3 / 8), (orc.POISSON, 0.8, 0.0)]:
        g = tiny(loss=loss, eps=eps, c=c)
        I = RNG.random((5, 5)) * 50 + 0.5
        l, dl = orc.loss_terms(I, I, g)
        assert np.allclose(l, 0.0, atol=1e-12)
        # the amplitude models are stationary at the data; the Poisson model
        # with its epsilon inside the logarithms is not: l'(E) = eps/(E + eps)
        want = 0.0 if loss == orc.AMPLITUDE else eps / (I + eps)
        assert np.allclose(dl, want, atol=1e-12)
        E = RNG.poisson(I).astype(float)
        h = 1e-6
        lp, _ = orc.loss_terms(I + h, E, g)
        lm, _ = orc.loss_terms(I - h, E, g)
        _, dl = orc.loss_terms(I, E, g)
        assert np.allclose((lp - lm) / (2 * h), dl, rtol=1e-6, atol=1e-8)


def test_detector_gradient_matches_paper_forms():
    """The seed 2 l'(I) A equals the paper's analytic detector-plane gradient
    for the amplitude model (eps = 0) and twice the Poisson one (§3.1)."""
    A = crand(6, 6, scale=3.0)
    I = np.abs(A) ** 2
    E = RNG.poisson(I).astype(float)
    g = tiny(loss=orc.AMPLITUDE, eps=0.0, c=3 / 8)
    _, dl = orc.loss_terms(I, E, g)
    paper_a = (1 - np.sqrt(E + 3 / 8) / (0.0 + np.sqrt(I + 3 / 8))) * A
    assert np.allclose(2 * dl * A, paper_a, rtol=1e-12)
    g = tiny(loss=orc.POISSON, eps=0.8)
    _, dl = orc.loss_terms(I, E, g)
    paper_p = (1 - E / (0.8 + I)) * A
    assert np.allclose(2 * dl * A, 2 * paper_p, rtol=1e-12)


def test_poisson_loss_is_stirling_nll_up_to_constant():
    # without eps the per-pixel loss differs from the exact negative
    # log-likelihood I - E log I + log E! by a term that does not depend on I
    g = tiny(loss=orc.POISSON, eps=0.0)
    E = np.array([3.0, 7.0, 12.0])
    for I in (np.array([2.0, 5.0, 9.0]), np.array([4.5, 8.0, 20.0])):
        l, _ = orc.loss_terms(I, E, g)
        nll = I - E * np.log(I) + np.array([math.lgamma(e + 1) for e in E])
        diff = nll - l
        stirling = np.array([math.lgamma(e + 1) for e in E]) - (E * np.log(E) - E)
        assert np.allclose(diff, stirling, rtol=1e-12)


# ------------------------------------------------------------ gradient

def _fd_check(g, O, P, pos, E, n_check=None):
    loss, gO, gP = orc.gradient(O, P, pos, E, g)
    h = 1e-6

    def L(O_, P_):
        return orc.loss_value(orc.forward(O_, P_, pos, g), E, g)

    idxO = list(np.ndindex(O.shape))
    idxP = list(np.ndindex(P.shape))
    if n_check is not None:
        sel = RNG.choice(len(idxO), n_check, replace=False)
        idxO = [idxO[i] for i in sel]
    errs = []
    for ix in idxO:
        for unit in (1.0, 1j):
            Op, Om = O.copy(), O.copy()
            Op[ix] += h * unit
            Om[ix] -= h * unit
            fd = (L(Op, P) - L(Om, P)) / (2 * h)
            an = gO[ix].real if unit == 1.0 else gO[ix].imag
            errs.append((fd, an))
    for ix in idxP:
        for unit in (1.0, 1j):
            Pp, Pm = P.copy(), P.copy()
            Pp[ix] += h * unit
            Pm[ix] -= h * unit
            fd = (L(O, Pp) - L(O, Pm)) / (2 * h)
            an = gP[ix].real if unit == 1.0 else gP[ix].imag
            errs.append((fd, an))
    fd, an = np.array(errs).T
    scale = np.max(np.abs(an))
    assert scale > 0
    assert np.max(np.abs(fd - an)) < 2e-6 * max(scale, 1.0), np.max(np.abs(fd - an))
    return loss


@pytest.mark.parametrize("loss,eps,c", [(orc.AMPLITUDE, 1e-3, 0.0), (orc.POISSON, 0.8, 0.0),
                                        (orc.AMPLITUDE, 1e-3, 3 / 8)])
def test_gradient_matches_finite_differences(loss, eps, c):
    g = tiny(S=2, K=2, loss=loss, eps=eps, c=c)
    O = phase_obj(2, 12, 12) * (0.9 + 0.1 * RNG.random((2, 12, 12)))
    P = crand(2, 8, 8, scale=2.0)
    I = orc.forward(O, P, POS4, g)
    E = RNG.poisson(I * 1.3 + 0.5).astype(float)
    _fd_check(g, O, P, POS4, E)


def test_gradient_three_slices_no_bandlimit_fd():
    g = tiny(S=3, K=1, beta=0.0, loss=orc.POISSON, eps=0.5)
    O = phase_obj(3, 12, 12)
    P = crand(1, 8, 8, scale=2.0)
    E = RNG.poisson(orc.forward(O, P, POS4, g) + 1.0).astype(float)
    _fd_check(g, O, P, POS4, E, n_check=60)


def test_gradient_zero_at_data_amplitude():
    g = tiny(S=2, K=2, loss=orc.AMPLITUDE, eps=1e-3)
    O = phase_obj(2, 12, 12)
    P = crand(2, 8, 8)
    I = orc.forward(O, P, POS4, g)
    loss, gO, gP = orc.gradient(O, P, POS4, I, g)
    assert abs(loss) < 1e-20 and np.abs(gO).max() < 1e-12 and np.abs(gP).max() < 1e-12


def test_adjoint_dot_products():
    # <M x, y> = <x, M^H y> for the linear maps the gradient goes through
    n = 12
    x, y = crand(n, n), crand(n, n)
    H = orc.propagator(n, n, 0.1, 0.0197, 9.0, 2 / 3)
    lhs = np.vdot(y, orc.propagate(x, H))
    rhs = np.vdot(orc.propagate(y, np.conj(H)), x)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    R = orc.shift_ramp(0.3, -0.2, n, n)
    lhs = np.vdot(y, orc.idft2(R * orc.dft2(x)))
    rhs = np.vdot(orc.idft2(np.conj(R) * orc.dft2(y)), x)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    lhs = np.vdot(y, orc.dft2_ortho(x))
    rhs = np.vdot(orc.idft2_ortho(y), x)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_position_gradient_fd():
    g = tiny(S=2, K=2, loss=orc.POISSON, eps=0.8)
    O = phase_obj(2, 12, 12)
    P = crand(2, 8, 8, scale=2.0)
    pos = np.array([[1.2, 2.3], [2.1, 0.8]])
    E = RNG.poisson(orc.forward(O, P, pos, g) * 1.2 + 0.3).astype(float)
    gp = orc.position_gradient(O, P, pos, E, g)
    h = 1e-6
    for j in range(2):
        for a in range(2):
            pp, pm = pos.copy(), pos.copy()
            pp[j, a] += h
            pm[j, a] -= h
            fd = (orc.loss_value(orc.forward(O, P, pp, g), E, g)
                  - orc.loss_value(orc.forward(O, P, pm, g), E, g)) / (2 * h)
            assert abs(fd - gp[j, a]) < 1e-5 * max(1.0, abs(fd))


# ---------------------------------------------------------------- Adam

def test_adam_closed_forms():
    z = crand(20)
    g = crand(20)
    m = np.zeros(20, complex)
    v = np.zeros(20)
    lr = 0.01
    # constant gradient: m_hat = g, v_hat = |g|^2 at every t
    zz, mm, vv = z, m, v
    for t in range(1, 5):
        zn, mm, vv = orc.adam_update(zz, mm, vv, g, t, lr)
        assert np.allclose(zz - zn, lr * g / (np.abs(g) + 1e-8), rtol=1e-10)
        zz = zn
    # alternating sign: second step moves by -(1-b1)/(1+b1) * lr g/|g|
    z1, m1, v1 = orc.adam_update(z, m, v, g, 1, lr)
    z2, _, _ = orc.adam_update(z1, m1, v1, -g, 2, lr)
    assert np.allclose(z1 - z2, -(0.1 / 1.9) * lr * g / (np.abs(g) + 1e-8), rtol=1e-8)
    # zero gradient: no move
    z0, _, _ = orc.adam_update(z, m, v, np.zeros(20, complex), 1, lr)
    assert np.allclose(z0, z)


def test_step_reduces_loss_on_consistent_data():
    g = tiny(S=2, K=1, loss=orc.AMPLITUDE, eps=1e-3, H=16, W=16)
    Otrue = phase_obj(2, 16, 16, amp=0.3)
    P = crand(1, 8, 8, scale=3.0)
    pos = np.array([[y + 0.3, x - 0.2] for y in (1, 3, 5, 7) for x in (1, 3, 5, 7)])
    E = orc.forward(Otrue, P, pos, g)
    O = np.ones_like(Otrue)
    mO, vO = np.zeros_like(O), np.zeros(O.shape)
    mP, vP = np.zeros_like(P), np.zeros(P.shape)
    losses = []
    for t in range(1, 16):
        O, P2, mO, vO, mP, vP, loss, gn = orc.step(O, P, mO, vO, mP, vP, t, pos, E,
                                                    np.arange(len(pos)), g, 0.02, 0.0,
                                                    update_probe=False)
        losses.append(loss)
        assert gn > 0
    assert losses[-1] < 0.5 * losses[0]


def _adam_closed(z, m, v, g, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    # Adam's moment recursion and bias corrections written out per element
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * (g.real ** 2 + g.imag ** 2)
    return z - lr * (m / (1.0 - b1 ** t)) / (np.sqrt(v / (1.0 - b2 ** t)) + eps), m, v


def test_step_gnorm_holds_regularizer_gradient_and_step_count():
    """The step's gradient norm, loss and Adam step count (§3.2, §3.4), on a
    case whose gradient is known in closed form: with a zero probe the
    wavefield, the patterns and the data term's gradient vanish for ANY
    object (amplitude loss, I = I_exp = 0), so the whole gradient is the
    object-L2 regulariser's 2 lam (O - 1) and the loss its lam sum |O - 1|^2.
    Two steps at t = 1, 2 must reproduce Adam written out by hand: the first
    moves every element by exactly lr along (O - 1) / |O - 1| (bias
    correction of t = 1); the second sees the new gradient 2 lam (O1 - 1).
    Fails if the regulariser is left out of the norm or of the update, or if
    the step count is passed off by one."""
    g = tiny(S=2, K=2, loss=orc.AMPLITUDE, eps=1e-3)
    O = phase_obj(2, 12, 12) * (0.7 + 0.6 * RNG.random((2, 12, 12)))
    P = np.zeros((2, 8, 8), complex)
    E = np.zeros((4, 8, 8))
    lam, lr = 0.05, 0.01
    zO, zP = np.zeros_like(O), np.zeros(O.shape)
    mP, vP = np.zeros_like(P), np.zeros(P.shape)
    O1, P1, mO, vO, mP1, vP1, loss, gn = orc.step(O, P, zO, zP, mP, vP, 1, POS4, E, np.arange(4), g,
                                                   lr, 0.02, reg={"l2_obj": lam})
    d = O - 1.0
    assert math.isclose(loss, lam * float(np.sum(np.abs(d) ** 2)), rel_tol=1e-12)
    assert math.isclose(gn, 2 * lam * float(np.sqrt(np.sum(np.abs(d) ** 2))), rel_tol=1e-12)
    # first step: m_hat = g, v_hat = |g|^2, so the move is lr g / (|g| + eps)
    gO0 = 2 * lam * d
    assert np.allclose(O - O1, lr * gO0 / (np.abs(gO0) + 1e-8), rtol=1e-12, atol=1e-15)
    assert np.array_equal(P1, P)  # zero probe gradient: no move
    O2, _, _, _, _, _, loss2, gn2 = orc.step(O1, P1, mO, vO, mP1, vP1, 2, POS4, E, np.arange(4), g,
                                             lr, 0.02, reg={"l2_obj": lam})
    gO1 = 2 * lam * (O1 - 1.0)
    assert math.isclose(gn2, float(np.sqrt(np.sum(np.abs(gO1) ** 2))), rel_tol=1e-12)
    assert math.isclose(loss2, lam * float(np.sum(np.abs(O1 - 1.0) ** 2)), rel_tol=1e-12)
    zc, mc, vc = _adam_closed(O, np.zeros_like(O), np.zeros(O.shape), gO0, 1, lr)
    zc, mc, vc = _adam_closed(zc, mc, vc, gO1, 2, lr)
    assert np.allclose(O2, zc, rtol=1e-12, atol=1e-15)
    # an off-by-one step count moves the second step measurably
    zw, _, _ = _adam_closed(O1, mc * 0 + (1 - 0.9) * gO0, (1 - 0.999) * np.abs(gO0) ** 2, gO1, 3, lr)
    assert np.max(np.abs(zw - zc)) > 1e-4 * lr


def test_step_gnorm_holds_probe_gradient():
    """At data simulated from the current object and probe, the amplitude
    loss and its gradient vanish (§3.1), so with the probe-L2 regulariser
    alone the step's gradient is g_P = 2 lam P (closed form) and g_O = 0:
    the norm is 2 lam |P|, the loss lam |P|^2, the object stays put and the
    probe takes Adam's first step lr g / |g|.  With the probe held fixed the
    norm still counts g_P.  Fails if g_P is dropped from the norm."""
    g = tiny(S=2, K=2, loss=orc.AMPLITUDE, eps=1e-3)
    O = phase_obj(2, 12, 12)
    P = crand(2, 8, 8, scale=2.0)
    E = orc.forward(O, P, POS4, g)
    lam, lr = 0.03, 0.02
    for upd in (True, False):
        O1, P1, *_, loss, gn = orc.step(O, P, np.zeros_like(O), np.zeros(O.shape), np.zeros_like(P),
                                       np.zeros(P.shape), 1, POS4, E, np.arange(4), g, 0.01, lr,
                                       update_probe=upd, reg={"l2_probe": lam})
        nP = float(np.sqrt(np.sum(np.abs(P) ** 2)))
        assert math.isclose(gn, 2 * lam * nP, rel_tol=1e-9)
        assert math.isclose(loss, lam * nP ** 2, rel_tol=1e-9)
        assert np.allclose(O1, O, rtol=0, atol=1e-12)
        if upd:
            gP = 2 * lam * P
            assert np.allclose(P - P1, lr * gP / (np.abs(gP) + 1e-8), rtol=1e-8, atol=1e-12)
        else:
            assert np.array_equal(P1, P)


def test_gradient_fd_on_four_position_multislice_subproblem():
    """Directional finite differences of the full 20-slice, 8-mode, 192x192
    problem on four neighbouring scan positions (the workload's gradient
    check), on random directions in the object and in the probe."""
    from paper_2505_14372_b300 import synth
    wl = synth.WORKLOADS[3]
    P = synth.probe_modes(wl).astype(np.complex128)
    pos = synth.raster_positions(wl)[[0, 1, 128, 129]].astype(np.float64)
    org = np.floor(pos.min(0)).astype(int) - 1
    pos = pos - org
    H = W = 200
    small = synth.Workload(**{**wl.__dict__, "H": H, "W": W, "atoms_per_slice": 40})
    O = synth.phase_object(small).astype(np.complex128)
    g = orc.Geom(S=20, K=8, h=192, w=192, H=H, W=W, dx=wl.dx, lam=wl.lam, dz=wl.dz,
                 bandlimit=wl.bandlimit, loss=orc.POISSON, eps=0.8)
    E = synth.cbed_like_patterns(wl, 4).astype(np.float64)
    loss, gO, gP = orc.gradient(O, P, pos, E, g)
    rng = np.random.default_rng(5)
    h = 1e-5
    for which in ("O", "P"):
        if which == "O":
            d = rng.standard_normal(O.shape) + 1j * rng.standard_normal(O.shape)
            Lp = orc.loss_value(orc.forward(O + h * d, P, pos, g), E, g)
            Lm = orc.loss_value(orc.forward(O - h * d, P, pos, g), E, g)
            an = np.real(np.vdot(gO, d))
        else:
            d = (rng.standard_normal(P.shape) + 1j * rng.standard_normal(P.shape)) * 0.01
            Lp = orc.loss_value(orc.forward(O, P + h * d, pos, g), E, g)
            Lm = orc.loss_value(orc.forward(O, P - h * d, pos, g), E, g)
            an = np.real(np.vdot(gP, d))
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - an) < 1e-6 * abs(an), (which, fd, an)


def test_vjp_is_gradient_of_linearised_loss():
    # for L = sum c * I the VJP with gI = c equals the FD derivative of L
    g = tiny(S=2, K=2)
    O = phase_obj(2, 12, 12)
    P = crand(2, 8, 8)
    cI = RNG.standard_normal((4, 8, 8))
    gO, gP = orc.vjp(O, P, POS4, cI, g)
    d = crand(2, 12, 12)
    h = 1e-6
    fd = (np.sum(cI * orc.forward(O + h * d, P, POS4, g)) - np.sum(cI * orc.forward(O - h * d, P, POS4, g))) / (2 * h)
    assert abs(fd - np.real(np.vdot(gO, d))) < 1e-6 * max(1.0, abs(fd))
    d = crand(2, 8, 8)
    fd = (np.sum(cI * orc.forward(O, P + h * d, POS4, g)) - np.sum(cI * orc.forward(O, P - h * d, POS4, g))) / (2 * h)
    assert abs(fd - np.real(np.vdot(gP, d))) < 1e-6 * max(1.0, abs(fd))


def test_gaussian_model_and_fd():
    g = tiny(loss=orc.GAUSSIAN, c=3.0, eps=0.0)
    I = RNG.random((6, 6)) * 40
    E = RNG.poisson(I).astype(float)
    l, dl = orc.loss_terms(I, E, g)
    # negative log-likelihood of N(I, sigma^2) up to its constant
    nll = -np.log(np.exp(-(I - E) ** 2 / (2 * 9.0)) / (3.0 * np.sqrt(2 * np.pi)))
    assert np.allclose(nll - l, np.log(3.0 * np.sqrt(2 * np.pi)))
    h = 1e-6
    assert np.allclose((orc.loss_terms(I + h, E, g)[0] - orc.loss_terms(I - h, E, g)[0]) / (2 * h), dl, rtol=1e-6,
                       atol=1e-9)


@pytest.mark.parametrize("kw", [dict(l2_obj=0.3), dict(l2_probe=0.2), dict(tikhonov=0.4), dict(layers=0.5),
                                dict(l2_obj=0.1, tikhonov=0.2, layers=0.3, l2_probe=0.05),
                                dict(tv=0.3, tv_eps=0.05), dict(tv_layers=0.4, tv_eps=0.02),
                                dict(tv=0.2, tv_layers=0.1, tikhonov=0.1, tv_eps=0.1)])
def test_regularizer_gradients_by_fd(kw):
    O = crand(3, 5, 6)
    P = crand(2, 4, 4)
    val, gO, gP = orc.regularizers(O, P, **kw)
    h = 1e-6
    for arr, grad, which in ((O, gO, "O"), (P, gP, "P")):
        for ix in list(np.ndindex(arr.shape))[::7]:
            for unit in (1.0, 1j):
                a1, a2 = arr.copy(), arr.copy()
                a1[ix] += h * unit
                a2[ix] -= h * unit
                args1 = (a1, P) if which == "O" else (O, a1)
                args2 = (a2, P) if which == "O" else (O, a2)
                fd = (orc.regularizers(*args1, **kw)[0] - orc.regularizers(*args2, **kw)[0]) / (2 * h)
                an = grad[ix].real if unit == 1.0 else grad[ix].imag
                assert abs(fd - an) < 1e-6 * max(1.0, abs(fd))


def test_regularizers_vanish_on_their_null_space():
    O = np.ones((3, 5, 5), complex) * np.exp(0.3j)    # constant in plane and depth
    P = crand(1, 4, 4)
    assert orc.regularizers(O, P, tikhonov=1.0, layers=1.0)[0] < 1e-24
    assert orc.regularizers(np.ones((2, 3, 3), complex), P, l2_obj=1.0)[0] == 0.0
    assert orc.regularizers(O, P, tv=1.0, tv_layers=1.0, tv_eps=1e-3)[0] == 0.0


def test_tv_of_a_phase_step_is_closed_form():
    # one slice, O = 1 on the left half and exp(i phi) on the right: only the
    # H horizontal differences across the step are non-zero, each of modulus
    # |exp(i phi) - 1| = 2 sin(phi / 2)
    H, W, phi, lam, eta = 6, 8, 0.7, 0.25, 1e-3
    O = np.ones((1, H, W), complex)
    O[:, :, W // 2:] = np.exp(1j * phi)
    val, gO, _ = orc.regularizers(O, np.zeros((1, 2, 2), complex), tv=lam, tv_eps=eta)
    d = 2 * np.sin(phi / 2)
    assert np.isclose(val, lam * H * (np.sqrt(d * d + eta * eta) - eta), rtol=1e-12)
    # the gradient pulls the two sides of the step towards each other
    unit = (np.exp(1j * phi) - 1) / abs(np.exp(1j * phi) - 1)
    assert np.allclose(gO[0, :, W // 2], lam * unit * d / np.sqrt(d * d + eta * eta))
    assert np.allclose(gO[0, :, W // 2 - 1], -lam * unit * d / np.sqrt(d * d + eta * eta))
