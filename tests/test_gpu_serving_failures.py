"""Failure detection of the serving runtime, injected on the host (nothing
faults, traps or hangs the GPU): non-finite data refused at submit, a
request whose loss turns non-finite ended with ENONFINITE, cancelled
requests (queued and running) ended with ECANCELED while the others finish
with their usual results, and a stalled worker seen by a client's time-out
and then recovered from."""
import numpy as np
import pytest

from gpu_util import rel_l2
from paper_2505_14372_b300 import PtychoError, Server, adam_opt
from test_gpu_serving import REQS, request

pytestmark = pytest.mark.gpu

GB = 1 << 30
EINVAL, ETIMEDOUT, ECANCELED, ENONFINITE = -1, -5, -9, -10


def _submit(srv, r, iters=2, batch=8, seed=11, opt=None):
    return srv.submit(r[0], r[2], r[3], r[1], iterations=iters, batch=batch, seed=seed,
                      opt=opt if opt is not None else adam_opt(1e-2, 1e-3))


def test_non_finite_data_is_refused_at_submit():
    geom, P, pos, I_exp = request(**REQS[0])
    srv = Server(8 * GB, 4)
    bad = [("patterns", dict(I=I_exp.copy())), ("positions", dict(pos=pos.copy())),
           ("probe", dict(P=P.copy()))]
    bad[0][1]["I"][3, 5, 7] = np.nan
    bad[1][1]["pos"][2, 1] = np.inf
    bad[2][1]["P"][0, 1, 1] = complex(np.nan, 0.0)
    for what, b in bad:
        with pytest.raises(PtychoError) as e:
            srv.submit(geom, b.get("pos", pos), b.get("I", I_exp), b.get("P", P), iterations=1, batch=8)
        assert e.value.code == EINVAL, what
    assert srv.stats()["submitted"] == 0
    srv.close()


def test_diverging_request_ends_with_nonfinite_and_spares_the_others():
    good, bad = request(**REQS[0]), request(**REQS[1])
    srv = Server(8 * GB, 4)
    t_good = _submit(srv, good)
    # an object step of 1e30: the object overflows after the first step
    t_bad = _submit(srv, bad, iters=20, opt=adam_opt(1e30, 1e-3))
    with pytest.raises(PtychoError) as e:
        srv.wait(t_bad)
    assert e.value.code == ENONFINITE
    st = srv.poll(t_bad)
    assert st["state"] == "failed" and st["error"] == ENONFINITE and st["iterations_done"] < 20
    srv.wait(t_good)
    out = srv.poll(t_good, good[0])
    assert out["state"] == "done" and np.all(np.isfinite(out["loss"]))
    s = srv.stats()
    assert s["failed"] == 1 and s["finished"] == 1
    srv.close()


def _alone(r, iters=2):
    srv = Server(8 * GB, 4)
    t = _submit(srv, r, iters=iters)
    srv.wait(t)
    out = srv.poll(t, r[0])
    srv.close()
    return out


def test_cancel_queued_and_running_requests():
    a, b, c = request(**REQS[0]), request(**REQS[2]), request(**REQS[1])
    ref = _alone(a)
    srv = Server(8 * GB, 1)  # one resident request: the others queue
    t_long = _submit(srv, b, iters=400, batch=5)
    t_queued = _submit(srv, c)
    t_a = _submit(srv, a)
    srv.cancel(t_queued)  # still queued behind t_long
    st = srv.poll(t_queued)
    assert st["state"] == "failed" and st["error"] == ECANCELED
    # t_long runs; cancel it once it has done an iteration
    for _ in range(200000):
        if srv.poll(t_long)["iterations_done"] >= 1:
            break
    srv.cancel(t_long)
    with pytest.raises(PtychoError) as e:
        srv.wait(t_long)
    assert e.value.code == ECANCELED
    st = srv.poll(t_long)
    assert st["state"] == "failed" and st["iterations_done"] < 400
    # the request behind them runs as it would alone
    srv.wait(t_a)
    out = srv.poll(t_a, a[0])
    assert out["state"] == "done"
    assert np.allclose(out["loss"], ref["loss"], rtol=1e-4)
    assert rel_l2(out["O"], ref["O"]) < 1e-4 and rel_l2(out["P"], ref["P"]) < 1e-4
    srv.cancel(t_a)  # no effect on a finished request
    assert srv.poll(t_a)["state"] == "done"
    s = srv.stats()
    assert s["failed"] == 2 and s["finished"] == 1 and s["queue_depth"] == 0
    for t in (t_long, t_queued, t_a):
        srv.release(t)
    srv.close()


def test_stalled_worker_times_out_a_client_then_recovers():
    r = request(**REQS[0])
    ref = _alone(r)
    srv = Server(8 * GB, 4)
    srv.inject_stall(1500.0)
    t = _submit(srv, r)
    with pytest.raises(PtychoError) as e:
        srv.wait(t, timeout_ms=300.0)
    assert e.value.code == ETIMEDOUT
    srv.wait(t, timeout_ms=120e3)
    out = srv.poll(t, r[0])
    assert out["state"] == "done"
    assert np.allclose(out["loss"], ref["loss"], rtol=1e-4) and rel_l2(out["O"], ref["O"]) < 1e-4
    srv.close()
