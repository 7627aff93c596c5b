"""Child process of tests/test_gpu_checked_build.py: runs the cases below
through the library named by PTYCHO_LIBRARY (the checked build when it is
"checked"), checks each context's status (PTYCHO_ECHECK would raise), and
writes the outputs to the .npz file given as the only argument.

Cases (seeded problems of gpu_util.problem): forward and adjoint of every
window size (64, 128: one CTA per wavefield; 192: the two-CTA cluster;
256: the four-CTA cluster), the 192 x 192 tensor-core tile (BF16x6), an
out-of-object position, more positions than clusters (the work queue) and
a fused 64 x 64 gradient step."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import numpy as np  # noqa: E402

from gpu_util import dev, host, problem  # noqa: E402
from paper_2505_14372_b300 import AdamState, Context, PtychoError, adam_opt  # noqa: E402
from paper_2505_14372_b300._lib import lib  # noqa: E402

CASES = [
    # name, seed, S, K, N, H, W, B, dft
    ("n64", 701, 2, 2, 64, 90, 84, 9, "fft"),
    ("n128", 702, 2, 2, 128, 150, 140, 5, "fft"),
    ("n192", 703, 3, 2, 192, 200, 206, 3, "fft"),
    ("n256", 704, 2, 1, 256, 270, 260, 3, "fft"),
    ("n192_bf16x6", 705, 2, 2, 192, 200, 200, 3, "bf16x6"),
    ("n192_queued", 706, 1, 1, 192, 300, 310, 100, "fft"),
]


def run(out_path):
    res = {"checked": np.array(int(lib().ptycho_build_checked()))}
    for name, seed, S, K, N, H, W, B, dft in CASES:
        geom, og, P, O, pos = problem(seed, S, K, N, H, W, B, loss="poisson", eps=0.8)
        geom.dft = dft
        geom.waves = "recompute"
        I_exp = np.random.default_rng(seed).poisson(2.0, size=(B, N, N)).astype(np.float32)
        ctx = Context(geom, max_batch=B)
        I = ctx.forward(dev(O), dev(P), dev(pos))
        loss, gO, gP = ctx.adjoint(dev(O), dev(P), dev(pos), dev(I_exp))
        ctx.check_status()
        res[name + "_I"], res[name + "_loss"] = host(I), np.array(float(loss.item()))
        res[name + "_gO"], res[name + "_gP"] = host(gO), host(gP)
        ctx.close()
    # an out-of-object position: skipped and flagged, not an index error
    geom, og, P, O, pos = problem(707, 1, 1, 64, 80, 80, 3)
    pos[1] = [16.6, 0.0]
    ctx = Context(geom, max_batch=3)
    res["oob_I"] = host(ctx.forward(dev(O), dev(P), dev(pos)))
    try:
        ctx.check_status()
        res["oob_code"] = np.array(0)
    except PtychoError as e:
        res["oob_code"] = np.array(e.code)
    ctx.close()
    # two fused 64 x 64 gradient steps (probe spectrum, tile, fused step end)
    geom, og, P, O, pos = problem(708, 1, 1, 64, 96, 96, 12, loss="poisson", eps=0.8)
    I_exp = np.random.default_rng(9).poisson(3.0, size=(12, 64, 64)).astype(np.float32)
    idx = np.arange(12, dtype=np.int32)
    ctx = Context(geom, max_batch=12)
    Od, Pd = dev(O), dev(P)
    st = AdamState(geom)
    for _ in range(2):
        stats = ctx.step(Od, Pd, st, adam_opt(lr_O=1e-2, lr_P=1e-3), dev(pos), dev(I_exp), dev(idx))
    ctx.check_status()
    res["step_O"], res["step_P"], res["step_stats"] = host(Od), host(Pd), host(stats)
    np.savez(out_path, **res)


if __name__ == "__main__":
    run(sys.argv[1])
