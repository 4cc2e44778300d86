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
