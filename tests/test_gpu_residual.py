"""The two residual methods (float64 CUDA cores; exact digit products on the
tensor cores) against r = b - T x in extended precision, through dm_residual.

Bound per entry (both methods): 3m * 2^-50 * max|row of [A_i B_i C_i]| *
max|column of [x_{i-1}; x_i; x_{i+1}]| -- the sliced method's digit
truncation and dropped digit pairs, and at least the float64 dot product's
own worst case.  Cases: random x (residual of the order of |T||x|), x close
to the solution (massive cancellation, the refinement's situation), block
rows at the ends (A_1, C_N absent), ragged sizes, nrhs 1..16, m up to the
128 limit, a batch that mixes systems inside and outside the sliced limits,
and a NaN in x."""
import numpy as np
import pytest

from oracle import dm_oracle as o
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


def exact_residual(A, B, C, x, b):
    """b - T x accumulated in numpy's long double (quad on aarch64)."""
    L = np.longdouble
    N = A.shape[0]
    r = b.astype(L).copy()
    for i in range(N):
        r[i] -= B[i].astype(L) @ x[i].astype(L)
        if i > 0:
            r[i] -= A[i].astype(L) @ x[i - 1].astype(L)
        if i < N - 1:
            r[i] -= C[i].astype(L) @ x[i + 1].astype(L)
    return r


def bound(A, B, C, x):
    N, m, _ = B.shape
    out = np.zeros(x.shape)
    for i in range(N):
        rowmax = np.abs(B[i]).max(axis=1)
        cols = [x[i]]
        if i > 0:
            rowmax = np.maximum(rowmax, np.abs(A[i]).max(axis=1))
            cols.append(x[i - 1])
        if i < N - 1:
            rowmax = np.maximum(rowmax, np.abs(C[i]).max(axis=1))
            cols.append(x[i + 1])
        colmax = np.abs(np.concatenate(cols, axis=0)).max(axis=0)
        out[i] = 3 * m * 2.0 ** -50 * np.outer(rowmax, colmax)
    return out


def residual_both(dm, s, x, b, P=1):
    plan = dm.dm_plan(s.N, s.m, s.nrhs, P, 1, "fp32")
    try:
        dm.dm_factor(plan, s.A, s.B, s.C)
        out = {}
        for mode in ("fp64", "sliced"):
            dm.dm_set_residual(plan, mode)
            r = np.zeros_like(b)
            rel = dm.dm_residual(plan, x, b, r)
            out[mode] = (r, rel, dm.dm_plan_query(plan)["residual_tc_systems"])
    finally:
        dm.dm_destroy(plan)
    return out


@pytest.mark.parametrize("N,m,r", [(2, 5, 1), (7, 32, 3), (9, 100, 8), (5, 128, 16), (3, 17, 2), (1, 64, 4)])
@pytest.mark.parametrize("near", [False, True])
def test_residual_methods_against_extended_precision(dm, N, m, r, near):
    s = w.dominant_system(N, m, r, 31 + m + r)
    rng = np.random.default_rng(N * m + r)
    if near:  # a float64 solution: the residual is pure cancellation
        x = o.dm(s.A, s.B, s.C, s.b, 1)
    else:
        x = rng.standard_normal(s.b.shape) * np.exp(rng.uniform(-3, 3, size=(1, 1, r)))
    out = residual_both(dm, s, x, s.b)
    rex = exact_residual(s.A, s.B, s.C, x, s.b)
    bd = bound(s.A, s.B, s.C, x)
    for mode, (rv, rel, ntc) in out.items():
        err = np.abs(rv.astype(np.longdouble) - rex).astype(np.float64)
        assert np.all(err <= bd), (mode, float((err / bd).max()))
        assert ntc == (1 if mode == "sliced" else 0)
        num = np.sqrt(((rex.astype(np.float64)) ** 2).sum(axis=(0, 1)))
        den = np.sqrt((s.b ** 2).sum(axis=(0, 1)))
        assert abs(rel - (num / den).max()) <= 1e-6 * (num / den).max() + 1e-300 or near


def test_batch_mixes_both_methods(dm):
    """Systems outside the sliced limits (m = 200, nrhs = 20) keep the float64
    kernel inside the same plan; every system's residual meets the bound."""
    shapes = [(6, 40, 3), (4, 200, 2), (5, 64, 20), (8, 128, 16)]
    systems = [w.dominant_system(n, m, r, 50 + k) for k, (n, m, r) in enumerate(shapes)]
    Ns, ms, rs = zip(*shapes)
    plan = dm.dm_plan_batch(list(Ns), list(ms), list(rs), "fp32")
    try:
        cat = lambda f: np.concatenate([f(s).ravel() for s in systems])
        dm.dm_factor(plan, cat(lambda s: s.A), cat(lambda s: s.B), cat(lambda s: s.C))
        rng = np.random.default_rng(5)
        xs = [rng.standard_normal(s.b.shape) for s in systems]
        x = np.concatenate([v.ravel() for v in xs])
        b = cat(lambda s: s.b)
        dm.dm_set_residual(plan, "sliced")
        assert dm.dm_plan_query(plan)["residual_tc_systems"] == 2
        r = np.zeros_like(b)
        dm.dm_residual(plan, x, b, r)
    finally:
        dm.dm_destroy(plan)
    off = 0
    for s, xv in zip(systems, xs):
        n = s.b.size
        rv = r[off:off + n].reshape(s.b.shape)
        off += n
        err = np.abs(rv.astype(np.longdouble) - exact_residual(s.A, s.B, s.C, xv, s.b)).astype(np.float64)
        assert np.all(err <= bound(s.A, s.B, s.C, xv))


def test_sliced_residual_propagates_nan(dm):
    s = w.dominant_system(4, 32, 2, 9)
    x = np.ones_like(s.b)
    x[2, 5, 1] = np.nan
    out = residual_both(dm, s, x, s.b)
    for mode, (rv, _, _) in out.items():
        assert np.all(np.isnan(rv[1:4, :, 1])), mode      # rows coupled to x_2
        assert np.all(np.isfinite(rv[:, :, 0])), mode      # the other column is unaffected
        assert np.all(np.isfinite(rv[0, :, 1])), mode


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_refinement_with_each_residual(dm, monkeypatch, prec):
    """Mixed precision reaches the oracle within 1e-10 with either residual,
    in the same number of iterations (give or take one)."""
    s = w.conditioned_system(60, 64, 4, 3, cond=1e4)
    xt = o.refine_truth(s.A, s.B, s.C, s.b)
    iters = {}
    for mode in ("fp64", "sliced"):
        monkeypatch.setenv("DM_RESIDUAL", mode)
        plan = dm.dm_plan(s.N, s.m, s.nrhs, 6, 1, prec)
        try:
            dm.dm_factor(plan, s.A, s.B, s.C)
            x = np.zeros_like(s.b)
            dm.dm_solve(plan, s.b, x)
            q = dm.dm_plan_query(plan)
        finally:
            dm.dm_destroy(plan)
        assert q["residual_mode"] == (1 if mode == "sliced" else 0)
        assert q["residual_tc_systems"] == (1 if mode == "sliced" else 0)
        assert o.rel_err(x, xt) <= 1e-10
        iters[mode] = q["last_iters"]
    assert abs(iters["fp64"] - iters["sliced"]) <= 1


def test_auto_mode_picks_by_size(dm):
    """AUTO: tensor cores for m^2 nrhs >= 2^17 (here m = 128, nrhs = 8), float64
    for the rest; mixed plans default to AUTO, float64 plans to FP64."""
    plan = dm.dm_plan_batch([4, 4, 4], [128, 128, 64], [8, 4, 16], "bf16x3")
    try:
        q = dm.dm_plan_query(plan)
        assert q["residual_mode"] == 2 and q["residual_tc_systems"] == 1
        dm.dm_set_residual(plan, "sliced")
        assert dm.dm_plan_query(plan)["residual_tc_systems"] == 3
    finally:
        dm.dm_destroy(plan)
    plan = dm.dm_plan(8, 128, 8, 2, 1, "fp64")
    try:
        assert dm.dm_plan_query(plan)["residual_mode"] == 0
    finally:
        dm.dm_destroy(plan)
