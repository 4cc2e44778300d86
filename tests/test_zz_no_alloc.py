"""The allocation-free entry point dm_solve_noalloc, through the C ABI.

It exists for callers that cannot call cudaMalloc (another component owns the
device memory pool, or the solve path must never enter the allocator); its
workspace is the library's static device array.  Its x must equal what the
allocating entry points (dm_plan + dm_factor + dm_solve, float64, levels=1)
give for the same system, within the float64 parity tolerance, on calls made
one after another (the static array keeps the previous call's contents).
This file sorts last so that a run stopping at the first failure has run
every other test before it.
"""
import numpy as np
import pytest

from paper_1505_06864_gb300 import workloads as w

pytestmark = pytest.mark.gpu
TOL64 = 1e-12


@pytest.fixture(scope="module")
def dm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1505_06864_gb300 import build
    build.build()
    from paper_1505_06864_gb300 import dm as D
    return D


def allocating(dm, s, P):
    plan = dm.dm_plan(s.N, s.m, s.nrhs, P, 1, dm.DM_FP64)
    try:
        dm.dm_factor(plan, s.A, s.B, s.C)
        x = np.zeros_like(s.b)
        dm.dm_solve(plan, s.b, x)
    finally:
        dm.dm_destroy(plan)
    return x


def no_alloc(dm, s, P):
    import torch
    T = lambda a: torch.from_numpy(a).cuda()
    A, B, C, b = T(s.A), T(s.B), T(s.C), T(s.b)
    x = torch.full_like(b, float("nan"))
    dm.dm_solve_noalloc(s.N, s.m, s.nrhs, P, A, B, C, b, x)
    return x.cpu().numpy()


def close(x, xref):
    assert np.all(np.isfinite(x))
    scale = np.max(np.abs(xref), axis=(0, 1))
    assert np.all(np.max(np.abs(x - xref), axis=(0, 1)) <= TOL64 * scale)



def test_no_alloc_two_calls_in_a_row(dm):
    s1 = w.dominant_system(64, 16, 1, 1)       # larger P first, then a different shape
    s2 = w.dominant_system(41, 24, 3, 2)
    x1 = no_alloc(dm, s1, 4)
    x2 = no_alloc(dm, s2, 5)
    close(x1, allocating(dm, s1, 4))
    close(x2, allocating(dm, s2, 5))
    # again with the first system: the leftovers of call two must not leak in
    close(no_alloc(dm, s1, 4), x1)


def test_no_alloc_single_subsystem_and_limits(dm):
    import torch
    s = w.dominant_system(9, 8, 2, 3)
    close(no_alloc(dm, s, 1), allocating(dm, s, 1))
    big = torch.zeros((70, 128, 128), dtype=torch.float64, device="cuda")
    v = torch.zeros((70, 128, 1), dtype=torch.float64, device="cuda")
    with pytest.raises(dm.DMError) as e:
        dm.dm_solve_noalloc(70, 128, 1, 4, big, big, big, v, v.clone())
    assert e.value.code == dm.DM_EINVAL and "static" in str(e.value)
