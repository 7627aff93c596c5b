"""ptycho_forward_static, the allocation-free entry point for callers that
cannot allocate device memory (a detector-fed reconstruction loop that must
not stall in cudaMalloc, an application whose device memory all belongs to
its own pool, a plug-in whose host forbids allocating): its scratch is a
fixed array inside the library.  Checked against ptycho_forward on the same
inputs (two calls in a row, so the second sees the first call's leftovers in
the shared scratch) and against the FP64 oracle.  Collected last so that a
run stopping at the first failure has run every other test first."""
import ctypes as C
import dataclasses

import numpy as np
import pytest
import torch

import oracle as orc
from gpu_util import dev, host, problem, rel_l2
from paper_2505_14372_b300 import Context, PtychoError, _lib

pytestmark = pytest.mark.gpu


def static_forward(geom, O, P, pos, status=None):
    g, _dz = geom.to_c()
    out = torch.empty((pos.shape[0], geom.N, geom.N), dtype=torch.float32, device="cuda")
    rc = _lib.lib().ptycho_forward_static(C.byref(g), O.data_ptr(), P.data_ptr(), pos.data_ptr(), pos.shape[0],
                                          out.data_ptr(), None if status is None else status.data_ptr(),
                                          torch.cuda.current_stream().cuda_stream)
    _lib.check(rc)
    return out


def test_static_forward_matches_context_forward_twice():
    geom, og, P, O, pos = problem(77, 3, 2, 64, 90, 96, 12)
    ctx = Context(geom, max_batch=12)
    Od, Pd = dev(O), dev(P)
    for call in range(2):
        p = pos + np.float32(0.37 * call)            # different inputs on the second call
        ref = host(ctx.forward(Od, Pd, dev(p)))
        got = host(static_forward(geom, Od, Pd, dev(p)))
        assert rel_l2(got, ref) < 1e-5, call
        # the FP64 oracle: multislice tolerance
        assert rel_l2(got, orc.forward(O, P, p, og)) < 1e-4, call


def test_static_forward_other_window_and_limit():
    geom, og, P, O, pos = problem(78, 2, 1, 128, 140, 140, 5)
    ctx = Context(geom, max_batch=5)
    Od, Pd, pd = dev(O), dev(P), dev(pos)
    for _ in range(2):
        assert rel_l2(host(static_forward(geom, Od, Pd, pd)), host(ctx.forward(Od, Pd, pd))) < 1e-5
    # 256 x 128^2 x 8 bytes of far fields do not fit the 32 MiB scratch
    big = dev(np.repeat(pos, 60, axis=0)[:256])
    with pytest.raises(PtychoError) as e:
        static_forward(geom, Od, Pd, big)
    assert e.value.code == -1 and "static scratch" in str(e.value)


@pytest.mark.parametrize("dft", ["fft", "tf32x3"])
def test_static_forward_two_cta_window(dft):
    # the 192 x 192 tile (two-CTA cluster with its bulk-copy exchange), with
    # the FFT and one tensor-core DFT mode
    geom, og, P, O, pos = problem(79, 2, 2, 192, 210, 214, 4)
    geom = dataclasses.replace(geom, dft=dft)
    ctx = Context(geom, max_batch=4)
    Od, Pd, pd = dev(O), dev(P), dev(pos)
    ref = host(ctx.forward(Od, Pd, pd))
    for _ in range(2):
        got = host(static_forward(geom, Od, Pd, pd))
        assert rel_l2(got, ref) < 1e-5
    tol = 1e-4 if dft == "fft" else 5e-4  # the tensor-core modes' own error against FP64
    assert rel_l2(got, orc.forward(O, P, pos, og)) < tol


def test_static_forward_position_outside_object():
    geom, og, P, O, pos = problem(80, 1, 1, 64, 80, 80, 3)
    pos = pos.copy()
    pos[1] = [40.0, 3.0]  # rows 40..103 leave the 80-row object
    Od, Pd = dev(O), dev(P)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    got = host(static_forward(geom, Od, Pd, dev(pos), status=st))
    assert int(st.item()) & 1
    assert not np.any(got[1])
    ok = [0, 2]
    assert rel_l2(got[ok], orc.forward(O, P, pos[ok], og)) < 1e-5
    # the next call starts from a clear status word
    st2 = torch.full((1,), 7, dtype=torch.int32, device="cuda")
    static_forward(geom, Od, Pd, dev(pos[ok]), status=st2)
    assert int(st2.item()) == 0
