"""Parity of the tcgen05 mixed-precision factor paths (DM_TF32, DM_BF16X3)
with the float64 oracle: after float64 iterative refinement (tolerance 1e-10,
the mixed-precision target), and before it -- one pass x = M^-1 b through the
low-precision factors alone, where refinement cannot hide a wrong product.

First-pass bound: |x - x_oracle| <= C_FIRST * kappa * U[prec] * max|x_oracle|
per right-hand-side column, U the relative error of one block product in
that precision -- float32 CUDA cores 2^-24; TF32 operands read with 10
explicit mantissa bits, 2^-10; split bf16 hi + lo with the lo*lo term dropped,
about 3 * 2^-18 per product plus float32 accumulation, 2^-16 -- and
C_FIRST = 16 for the growth over m-term dot products and a sweep.  A bf16x3
product that lost its hi*lo or lo*hi terms is bf16-accurate (2^-9) and
breaks this bound by a factor 8; its first-pass error also stops being ten
times below TF32's, which the tests assert as well."""
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


U = {"fp32": 2.0 ** -24, "tf32": 2.0 ** -10, "bf16x3": 2.0 ** -16}
C_FIRST = 16.0
MAX_ITERS = {"fp32": 3, "tf32": 6, "bf16x3": 4}   # refinement to 1e-12 on these well-conditioned systems


def kappa_inf_bound(A, B, C):
    """cond_inf(T) <= ||T||_inf / min_i (|t_ii| - sum_{j != i} |t_ij|) (Varah's
    bound on ||T^-1||_inf) for a strictly row-dominant T, from the blocks."""
    d = np.abs(np.diagonal(B, axis1=1, axis2=2))
    s = np.abs(A).sum(axis=2) + np.abs(B).sum(axis=2) + np.abs(C).sum(axis=2)
    margin = 2 * d - s
    assert np.min(margin) > 0
    return float(np.max(s) / np.min(margin))


def first_pass(dm, s, P, levels, prec):
    """x = M^-1 b: one pass through the precision's factors, no refinement."""
    plan = dm.dm_plan(s.N, s.m, s.nrhs, P, levels, prec)
    try:
        dm.dm_set_refinement(plan, 1e-12, 1)
        dm.dm_factor(plan, s.A, s.B, s.C)
        x = np.zeros_like(s.b)
        dm.dm_solve(plan, s.b, x, allow_notconv=True)
        assert dm.dm_plan_query(plan)["last_iters"] == 1
    finally:
        dm.dm_destroy(plan)
    return x


def check(x, xref, tol):
    assert np.all(np.isfinite(x))
    scale = np.max(np.abs(xref), axis=(0, 1))
    assert np.all(np.max(np.abs(x - xref), axis=(0, 1)) <= tol * scale)
    assert o.rel_err(x, xref) <= tol


@pytest.mark.parametrize("step_kernels", ["1", "0"])
@pytest.mark.parametrize("prec", ["tf32", "bf16x3"])
@pytest.mark.parametrize("N,m,r,P,levels", [(64, 16, 1, 4, 1), (40, 128, 2, 6, 1), (97, 40, 3, 7, 2),
                                            (9, 256, 2, 2, 1), (30, 100, 1, 5, 1), (33, 64, 17, 4, 1),
                                            (5, 8, 1, 2, 1), (2, 24, 1, 1, 1)])
def test_tensor_precisions_dominant(dm, monkeypatch, prec, N, m, r, P, levels, step_kernels):
    monkeypatch.setenv("DM_TC_STEP", step_kernels)
    s = w.dominant_system(N, m, r, 300 + N + m)
    x, rel, info = run(dm, s, P, levels, prec)
    P2 = info["P2"] if info["P2"] > 1 else None
    check(x, o.dm(s.A, s.B, s.C, s.b, P, levels=levels, P2=P2), TOLMIX)
    assert 2 <= info["last_iters"] <= MAX_ITERS[prec] and rel < 1e-13


@pytest.mark.parametrize("step_kernels", ["1", "0"])
@pytest.mark.parametrize("N,m,r,P,levels", [(64, 16, 1, 4, 1), (40, 64, 2, 6, 1), (24, 128, 2, 4, 1),
                                            (12, 256, 1, 3, 1), (97, 40, 3, 7, 2)])
def test_first_pass_before_refinement(dm, monkeypatch, N, m, r, P, levels, step_kernels):
    """One pass through the low-precision factors against the float64 oracle,
    element by element, at the bound derived from each precision's product
    error and cond_2(T) of the assembled matrix; and bf16x3 at least ten
    times more accurate than TF32.  Both tensor-core factor paths: the step
    kernels with TMA-fed operand copies (DM_TC_STEP=1, the default for
    m % 8 == 0) and the per-panel kernels (DM_TC_STEP=0)."""
    monkeypatch.setenv("DM_TC_STEP", step_kernels)
    s = w.dominant_system(N, m, r, 500 + N + m)
    kappa = float(np.linalg.cond(o.dense_from_blocks(s.A, s.B, s.C)))
    P2 = dm.dm_plan_tune(N, m, r, P, levels)[2]
    xo = o.dm(s.A, s.B, s.C, s.b, P, levels=levels, P2=P2 if P2 > 1 else None)
    err = {}
    for prec in ("fp32", "tf32", "bf16x3"):
        x = first_pass(dm, s, P, levels, prec)
        check(x, xo, C_FIRST * kappa * U[prec])
        err[prec] = o.rel_err(x, xo)
    assert err["bf16x3"] * 10 <= err["tf32"], err


def test_first_pass_config2_full_size(dm):
    """The same at the benchmark's size (N=2048 grid points x m=256 banded
    blocks, P=64, three levels), where cond_inf(T) is bounded from the blocks."""
    s = w.pde_banded_system(2048, 256, 1, 2)
    kappa = kappa_inf_bound(s.A, s.B, s.C)
    xo = o.dm(s.A, s.B, s.C, s.b, 64, levels=3, P2=dm.dm_plan_tune(2048, 256, 1, 64, 3)[2])
    err = {}
    for prec in ("tf32", "bf16x3"):
        x = first_pass(dm, s, 64, 3, prec)
        check(x, xo, C_FIRST * kappa * U[prec])
        err[prec] = o.rel_err(x, xo)
        assert err[prec] < 2.0 ** -6
    assert err["bf16x3"] * 10 <= err["tf32"], err


def test_bf16x3_conditioned(dm):
    s = w.conditioned_system(48, 64, 4, 5, cond=1e4)
    xt = o.refine_truth(s.A, s.B, s.C, s.b)
    x, rel, info = run(dm, s, 6, 1, "bf16x3")
    check(x, xt, TOLMIX)


def test_tensor_rejects_large_blocks(dm):
    with pytest.raises(dm.DMError) as e:
        dm.dm_plan(10, 300, 1, 2, 1, "tf32")
    assert e.value.code == dm.DM_EINVAL
