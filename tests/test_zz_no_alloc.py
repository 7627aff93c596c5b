"""ptycho_forward_static, the allocation-free entry point for callers that
cannot allocate device memory (its scratch is a fixed array inside the
library), against ptycho_forward on the same inputs, two calls in a row.
Collected last so that a run stopping at the first failure has run every
other test first."""
import ctypes as C

import numpy as np
import pytest
import torch

from gpu_util import dev, host, problem, rel_l2
from paper_2505_14372_b300 import Context, PtychoError, _lib

pytestmark = pytest.mark.gpu


def static_forward(geom, O, P, pos):
    g, _dz = geom.to_c()
    out = torch.empty((pos.shape[0], geom.N, geom.N), dtype=torch.float32, device="cuda")
    rc = _lib.lib().ptycho_forward_static(C.byref(g), O.data_ptr(), P.data_ptr(), pos.data_ptr(), pos.shape[0],
                                          out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    _lib.check(rc)
    return out


def test_static_forward_matches_context_forward_twice():
    geom, og, P, O, pos = problem(77, 3, 2, 64, 90, 96, 12)
    ctx = Context(geom, max_batch=12)
    Od, Pd = dev(O), dev(P)
    for call in range(2):
        p = dev(pos + np.float32(0.37 * call))       # different inputs on the second call
        ref = host(ctx.forward(Od, Pd, p))
        got = host(static_forward(geom, Od, Pd, p))
        assert rel_l2(got, ref) < 1e-5, call


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
