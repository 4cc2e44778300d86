"""Continuous batching through the C ABI: requests on many plans (new systems
and repeat right-hand sides on resident factors) queued while others run;
each result must equal the same request solved alone (direct dm_factor +
dm_solve), within the precision's tolerance."""
import time

import numpy as np
import pytest

from paper_1505_06864_gb300 import workloads as w

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1505_06864_gb300 import build
    build.build()
    from paper_1505_06864_gb300 import dm as D
    return D


def alone(dm, s, b, prec):
    P, lv, _ = dm.dm_plan_tune(s.N, s.m, s.nrhs)
    plan = dm.dm_plan(s.N, s.m, s.nrhs, P, lv, prec)
    try:
        dm.dm_factor(plan, s.A, s.B, s.C)
        x = np.zeros_like(b)
        dm.dm_solve(plan, b, x)
    finally:
        dm.dm_destroy(plan)
    return x


def wait_all(dm, tickets, timeout=120.0):
    out, t0 = {}, time.time()
    while len(out) < len(tickets):
        for t in tickets:
            if t in out:
                continue
            st, rel = dm.dm_poll(t)
            if st != dm.DM_PENDING:
                out[t] = (st, rel)
        assert time.time() - t0 < timeout, "serving requests did not finish"
        time.sleep(0.001)
    return out


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("bf16x3", 1e-10)])
def test_mix_equals_alone(dm, prec, tol):
    shapes = w.batch_shapes(10, 9, n_lo=20, n_hi=400, ms=(32, 64, 96, 128), r_lo=1, r_hi=8)
    systems = [w.dominant_system(N, m, r, 500 + i) for i, (N, m, r) in enumerate(shapes)]
    plans, jobs = [], []
    try:
        for s in systems:
            P, lv, _ = dm.dm_plan_tune(s.N, s.m, s.nrhs)
            plans.append(dm.dm_plan(s.N, s.m, s.nrhs, P, lv, prec))
        # new systems first, then repeat right-hand sides on the same plans, interleaved
        for i, s in enumerate(systems):
            x = np.zeros_like(s.b)
            jobs.append((dm.dm_submit_system(plans[i], s.A, s.B, s.C, s.b, x), i, s.b, x))
        for k in range(2):
            for i, s in enumerate(systems):
                b = w.random_rhs(s.N, s.m, s.nrhs, 900 + 10 * i + k)
                x = np.zeros_like(b)
                jobs.append((dm.dm_submit(plans[i], b, x), i, b, x))
        res = wait_all(dm, [j[0] for j in jobs])
    finally:
        for p in plans:
            dm.dm_destroy(p)
    for t, i, b, x in jobs:
        st, rel = res[t]
        assert st == dm.DM_OK and rel < 1e-13
        xa = alone(dm, systems[i], b, prec)
        scale = np.max(np.abs(xa), axis=(0, 1))
        assert np.all(np.max(np.abs(x - xa), axis=(0, 1)) <= tol * scale)


def test_tickets_and_destroy_waits(dm):
    s = w.dominant_system(300, 64, 2, 77)
    plan = dm.dm_plan(300, 64, 2, 0, 0, "fp64")
    x = np.zeros_like(s.b)
    t = dm.dm_submit_system(plan, s.A, s.B, s.C, s.b, x)
    dm.dm_destroy(plan)            # waits for the queued request
    st, rel = dm.dm_poll(t)
    assert st == dm.DM_OK and rel < 1e-13
    with pytest.raises(dm.DMError) as e:
        dm.dm_poll(t)              # a finished ticket is forgotten after reporting
    assert e.value.code == dm.DM_EINVAL
    assert np.max(np.abs(x - s.x_true)) < 1e-10 * np.max(np.abs(s.x_true))


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("bf16x3", 1e-10)])
def test_narrow_requests_merged(dm, prec, tol):
    """Narrow repeat right-hand sides queued behind a factorisation on one plan
    are packed into one solve of the plan's nrhs columns; every request's
    columns equal the oracle's solution for its own right-hand side."""
    from oracle import dm_oracle as o
    N, m, R = 300, 32, 8
    s = w.dominant_system(N, m, R, 811)
    P, lv, _ = dm.dm_plan_tune(N, m, R)
    widths = [1, 2, 1, 3, 1]                     # 8 columns: one merged solve
    before = dm.dm_serve_stats()
    plan = dm.dm_plan(N, m, R, P, lv, prec)
    try:
        x0 = np.zeros_like(s.b)
        jobs = [(dm.dm_submit_system(plan, s.A, s.B, s.C, s.b, x0), s.b, x0)]
        for k, c in enumerate(widths):
            b = w.random_rhs(N, m, c, 820 + k)
            x = np.zeros_like(b)
            jobs.append((dm.dm_submit_cols(plan, b, x, c), b, x))
        res = wait_all(dm, [j[0] for j in jobs])
        P2 = dm.dm_plan_query(plan)["P2"]
    finally:
        dm.dm_destroy(plan)
    after = dm.dm_serve_stats()
    assert after["merged"] - before["merged"] >= 2
    assert after["admitted"] - before["admitted"] == len(jobs)
    for t, b, x in jobs:
        st, rel = res[t]
        assert st == dm.DM_OK and rel < 1e-13
        xo = o.dm(s.A, s.B, s.C, b, P, levels=lv, P2=P2 if P2 > 1 else None)
        scale = np.max(np.abs(xo), axis=(0, 1))
        assert np.all(np.max(np.abs(x - xo), axis=(0, 1)) <= tol * scale)


def test_latency_budget_refuses(dm):
    """Once a plan's service time is measured, a budget below it refuses the
    next submit with DM_EAGAIN (nothing queued); without a budget it is
    admitted again."""
    import torch
    N, m, r = 400, 64, 2
    s = w.dominant_system(N, m, r, 833)
    P, lv, _ = dm.dm_plan_tune(N, m, r)
    plan = dm.dm_plan(N, m, r, P, lv, "fp64")
    try:
        x = np.zeros_like(s.b)
        wait_all(dm, [dm.dm_submit_system(plan, s.A, s.B, s.C, s.b, x)])
        wait_all(dm, [dm.dm_submit(plan, s.b, x)])
        before = dm.dm_serve_stats()
        dm.dm_serve_budget(1e-9)
        with pytest.raises(dm.DMError) as e:
            dm.dm_submit(plan, s.b, x)
        assert e.value.code == dm.DM_EAGAIN and "budget" in dm.dm_last_error()
        with pytest.raises(dm.DMError):
            dm.dm_submit_system(plan, s.A, s.B, s.C, s.b, x)
        dm.dm_serve_budget(60.0)
        t = dm.dm_submit(plan, s.b, x)
        assert wait_all(dm, [t])[t][0] == dm.DM_OK
    finally:
        dm.dm_serve_budget(0.0)
        dm.dm_destroy(plan)
    after = dm.dm_serve_stats()
    assert after["refused"] - before["refused"] == 2
    assert after["admitted"] - before["admitted"] == 1
