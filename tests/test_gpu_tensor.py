"""Parity of the tcgen05 mixed-precision factor paths (DM_TF32, DM_BF16X3)
with the float64 oracle after float64 iterative refinement (tolerance 1e-10,
the mixed-precision target)."""
import numpy as np
import pytest

from oracle import dm_oracle as o
from paper_1505_06864_gb300 import workloads as w

pytestmark = pytest.mark.gpu
TOLMIX = 1e-10


@pytest.fixture(scope="module")
def dm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1505_06864_gb300 import build
    build.build()
    from paper_1505_06864_gb300 import dm as D
    return D


def run(dm, s, P, levels, prec):
    plan = dm.dm_plan(s.N, s.m, s.nrhs, P, levels, prec)
    try:
        dm.dm_factor(plan, s.A, s.B, s.C)
        x = np.zeros_like(s.b)
        rel = dm.dm_solve(plan, s.b, x)
        info = dm.dm_plan_query(plan)
    finally:
        dm.dm_destroy(plan)
    return x, rel, info


def check(x, xref, tol):
    assert np.all(np.isfinite(x))
    scale = np.max(np.abs(xref), axis=(0, 1))
    assert np.all(np.max(np.abs(x - xref), axis=(0, 1)) <= tol * scale)
    assert o.rel_err(x, xref) <= tol


@pytest.mark.parametrize("prec", ["tf32", "bf16x3"])
@pytest.mark.parametrize("N,m,r,P,levels", [(64, 16, 1, 4, 1), (40, 128, 2, 6, 1), (97, 40, 3, 7, 2),
                                            (9, 256, 2, 2, 1), (30, 100, 1, 5, 1), (33, 64, 17, 4, 1)])
def test_tensor_precisions_dominant(dm, prec, N, m, r, P, levels):
    s = w.dominant_system(N, m, r, 300 + N + m)
    x, rel, info = run(dm, s, P, levels, prec)
    P2 = info["P2"] if info["P2"] > 1 else None
    check(x, o.dm(s.A, s.B, s.C, s.b, P, levels=levels, P2=P2), TOLMIX)
    assert info["last_iters"] >= 2 and rel < 1e-13


def test_bf16x3_conditioned(dm):
    s = w.conditioned_system(48, 64, 4, 5, cond=1e4)
    xt = o.refine_truth(s.A, s.B, s.C, s.b)
    x, rel, info = run(dm, s, 6, 1, "bf16x3")
    check(x, xt, TOLMIX)


def test_tensor_rejects_large_blocks(dm):
    with pytest.raises(dm.DMError) as e:
        dm.dm_plan(10, 300, 1, 2, 1, "tf32")
    assert e.value.code == dm.DM_EINVAL
