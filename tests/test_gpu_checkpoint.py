"""Checkpoint / resume: a reconstruction's whole state is the caller's object,
probe and Adam moments plus the step count (the context keeps only scratch),
so copying them to the host and back into a new context resumes it: the next
step equals the uninterrupted run's next step (up to the FP32 summation order
of the gradient scatter)."""
import numpy as np
import pytest
import torch

import oracle as orc
from gpu_util import dev, host, problem, rel_l2
from paper_2505_14372_b300 import AdamState, Context, adam_opt

pytestmark = pytest.mark.gpu


def test_resume_from_host_copies_gives_the_same_next_step():
    geom, og, P, O, pos = problem(61, 3, 2, 64, 96, 96, 12, loss="poisson", eps=0.8)
    I_exp = np.random.default_rng(3).poisson(orc.forward(O, P, pos, og) + 0.5).astype(np.float32)
    opt = adam_opt(lr_O=1e-2, lr_P=1e-3)
    groups = [np.array(g, np.int32) for g in ([0, 3, 6, 9], [1, 4, 7, 10], [2, 5, 8, 11])]
    ctx = Context(geom, max_batch=4)
    Od, Pd, st = dev(O), dev(P), AdamState(geom)
    posd, Id = dev(pos), dev(I_exp)
    for g in groups[:2]:
        ctx.step(Od, Pd, st, opt, posd, Id, dev(g))
    saved = {k: host(v).copy() for k, v in dict(O=Od, P=Pd, mO=st.mO, vO=st.vO, mP=st.mP, vP=st.vP).items()}
    t = st.t
    ctx.step(Od, Pd, st, opt, posd, Id, dev(groups[2]))
    # resume in a fresh context from the host copies
    ctx2 = Context(geom, max_batch=4)
    st2 = AdamState(geom)
    for name in ("mO", "vO", "mP", "vP"):
        getattr(st2, name).copy_(torch.from_numpy(saved[name]))
    st2.c.t = t
    O2, P2 = dev(saved["O"]), dev(saved["P"])
    ctx2.step(O2, P2, st2, opt, posd, Id, dev(groups[2]))
    assert st2.t == st.t == 3
    assert rel_l2(host(O2), host(Od)) < 1e-6 and rel_l2(host(P2), host(Pd)) < 1e-6
    assert rel_l2(host(st2.mO), host(st.mO)) < 1e-5 and rel_l2(host(st2.vP), host(st.vP)) < 1e-5
