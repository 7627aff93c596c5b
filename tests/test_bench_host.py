"""Host-side logic of bench.py's end-to-end leg (no GPU): every timed step
through host buffers carries a full group of positions, also when a group
is the whole scan (P = B, the 64x64 workload), so the leg never times
steps without work."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


@pytest.mark.parametrize("P,B,used,steps", [(256, 256, 23, 10), (4096, 256, 23, 10), (16384, 512, 23, 10),
                                            (1000, 300, 5, 7)])
def test_host_buffer_groups_are_full(P, B, used, steps):
    import bench
    order = np.arange(P, dtype=np.int32)  # one pass of the device-timed leg
    h = bench.host_buffer_order(order, used, steps, P, B)
    assert len(h) == steps * B
    groups = h.reshape(steps, B)
    assert groups.min() >= 0 and groups.max() < P
    if P % B == 0:  # whole groups of one pass: distinct positions
        for g in groups:
            assert len(np.unique(g)) == B
