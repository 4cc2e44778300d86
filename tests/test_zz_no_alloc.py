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


def test_no_alloc_rejects_host_memory_and_overlap(dm):
    """The library itself checks every pointer before it launches anything:
    host memory (given through the raw C entry point, past the binding's own
    check) and an x that overlaps b are DM_EINVAL."""
    import ctypes
    import torch
    s = w.dominant_system(9, 8, 2, 3)
    T = lambda a: torch.from_numpy(a).cuda()
    A, B, C, b = T(s.A), T(s.B), T(s.C), T(s.b)
    L = dm.lib()
    P = lambda t: ctypes.c_void_p(t.data_ptr())
    host = np.ascontiguousarray(s.b)
    rc = L.dm_solve_noalloc(9, 8, 2, 1, P(A), P(B), P(C), ctypes.c_void_p(host.ctypes.data), P(b.clone()), None)
    assert rc == dm.DM_EINVAL and "device memory" in dm.dm_last_error()
    rc = L.dm_solve_noalloc(9, 8, 2, 1, P(A), P(B), P(C), P(b), P(b), None)
    assert rc == dm.DM_EINVAL and "overlap" in dm.dm_last_error()
    # the refused calls left nothing behind: the next call is still exact
    close(no_alloc(dm, s, 1), allocating(dm, s, 1))
