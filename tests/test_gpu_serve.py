"""Serving form (hybrid_server_*): continuous batching of independent requests.

A request's result must not depend on the requests it shared batches with:
bitwise in the FP64 form, to FP32 summation order in the FP32 form. The
reference for a request is the same server driving that request alone; each
request of a mix is also held to the FP64 oracle run on it alone.
"""
import numpy as np
import pytest

import oracle
from paper_1406_6158_gb300 import ics

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

FIELDS = ("x", "y", "z", "vx", "vy", "vz", "m")


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1406_6158_gb300 import build, hybrid
    build.build()
    hybrid.load()
    return hybrid


def req_params(H, n, prec):
    eps = 1.0 / (4.0 * n ** (1.0 / 3.0))
    return H.Params(eps=eps, theta=0.5, R1=4 * eps, R2=8 * eps, dt_soft=1.0 / 128, n_hard=2, precision=prec)


REQS = [(0, 3000, 3), (1, 5000, 5), (2, 2000, 2), (3, 4100, 1)]   # tag, n, soft steps


def drive(H, prec, reqs, budget=4e9, arrivals=None):
    """Submits request k before server step arrivals[k]; returns {tag: state} and the step log."""
    srv = H.Server(H.Params(n_hard=2, precision=prec), budget)
    arrivals = arrivals or [0] * len(reqs)
    states = {t: ics.plummer(n, 100 + t) for t, n, _ in reqs}
    out, log, k, step = {}, [], 0, 0
    while len(out) < len(reqs):
        while k < len(reqs) and arrivals[k] <= step:
            t, n, ns = reqs[k]
            srv.submit(t, states[t], req_params(H, n, prec), ns)
            k += 1
        log.append(srv.step() + (srv.used_bytes(),))
        while True:
            r = srv.next()
            if r is None:
                break
            out[r[0]] = r[1]
        step += 1
        assert step < 100
    srv.close()
    return out, log


@pytest.mark.parametrize("prec", [0, 1])
def test_served_equals_alone(H, prec):
    mix, log = drive(H, prec, REQS, arrivals=[0, 1, 1, 3])
    assert max(a for a, _, _, _ in log) >= 2          # requests did share batches
    for t, n, ns in REQS:
        alone, _ = drive(H, prec, [(t, n, ns)])
        a, b = alone[t], mix[t]
        for k in FIELDS:
            if prec == 0:
                assert np.array_equal(a[k], b[k]), (t, k)
            else:
                assert np.max(np.abs(a[k] - b[k])) <= 1e-7 * max(1.0, np.max(np.abs(a[k]))), (t, k)
        ic = ics.plummer(n, 100 + t)
        assert np.array_equal(b["m"], ic["m"])         # returned in input order
        assert not np.array_equal(b["x"], ic["x"])     # and advanced


@pytest.mark.parametrize("prec", [0, 1])
def test_served_follow_the_oracle(H, prec):
    # each request of a mix whose members join at different server steps, against the oracle on that request
    # alone: two soft steps each (n_hard = 2); FP64 within 1e-9, FP32 pairs positions within 1e-8 and
    # velocities within 1e-6 (a 1e-5 force error kicked over 2 dt_s)
    reqs = [(0, 3000, 2), (1, 5000, 2), (2, 2000, 2), (3, 4100, 2)]
    mix, log = drive(H, prec, reqs, arrivals=[0, 1, 1, 2])
    assert max(a for a, _, _, _ in log) >= 2
    tol_x, tol_v = (1e-9, 1e-9) if prec == 0 else (1e-8, 1e-6)
    for t, n, ns in reqs:
        p = req_params(H, n, prec)
        ost = ics.plummer(n, 100 + t)
        ost["id"] = np.arange(n, dtype=np.int64)
        oracle.hybrid_steps(ost, oracle.Params(G=p.G, eps=p.eps, theta=p.theta, R1=p.R1, R2=p.R2,
                                               dt_soft=p.dt_soft, a_err=p.a_err, n_hard=p.n_hard, n_leaf=p.n_leaf,
                                               n_crit=p.n_crit, mac=p.mac), ns)
        q = np.argsort(ost["id"])
        for k in ("x", "y", "z", "vx", "vy", "vz"):
            tol = tol_v if k.startswith("v") else tol_x
            assert np.max(np.abs(mix[t][k] - ost[k][q])) <= tol, (t, k)


def test_admission_by_bytes(H):
    per = H.SERVER_BYTES_PER_PARTICLE
    budget = per * 5500.0                              # room for one of the larger requests at a time
    reqs = [(0, 3000, 2), (1, 5000, 2), (2, 2000, 2)]
    out, log = drive(H, 0, reqs, budget=budget)
    assert sorted(out) == [0, 1, 2]
    for active, queued, finished, used in log:
        assert used <= budget
    # 3000 and 5000 cannot be resident together, 3000 and 2000 can
    assert all(u <= budget for *_, u in log)
    for t, n, ns in reqs:
        alone, _ = drive(H, 0, [(t, n, ns)])
        for k in FIELDS:
            assert np.array_equal(alone[t][k], out[t][k])


def test_too_large_request_and_bad_tag(H):
    srv = H.Server(H.Params(precision=1), 1e6)
    st = ics.plummer(2000, 1)
    with pytest.raises(H.HybridError, match="ETOOLARGE"):
        srv.submit(0, st, None, 1)
    with pytest.raises(H.HybridError, match="EINVAL"):   # tags are >= 0: -1 means "none finished"
        srv.submit(-1, ics.plummer(100, 1), None, 1)
    assert srv.next() is None
    srv.close()
