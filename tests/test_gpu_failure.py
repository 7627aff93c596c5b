"""Failure detection on the device without a fault: the 192 x 192 tile's
layout-switch waits are bounded, and a self-test kernel whose waits receive
nothing must give up, flag the time-out (ETIMEDOUT to the host) and leave the
GPU usable, as the next computation, checked against the oracle, shows."""
import numpy as np
import pytest

import oracle as orc
from gpu_util import dev, host, problem, rel_l2
from paper_2505_14372_b300 import Context, _lib

pytestmark = pytest.mark.gpu


def test_bounded_exchange_wait_times_out_and_the_gpu_stays_usable():
    lib = _lib.lib()
    assert lib.ptycho_exchange_selftest(192) == _lib.ETIMEDOUT
    assert lib.ptycho_exchange_selftest(64) == _lib.EINVAL  # no mbarrier exchange there
    geom, og, P, O, pos = problem(31, 2, 2, 192, 210, 210, 2)
    ctx = Context(geom, max_batch=2)
    I = host(ctx.forward(dev(O), dev(P), dev(pos)))
    ctx.check_status()  # the self-test's flag was read and cleared: no stale time-out
    assert rel_l2(I, orc.forward(O, P, pos, og)) < 1e-4
