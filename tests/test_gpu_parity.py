"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances (the accuracy targets of this solver): plain float64 GPU DM within 1e-12 relative
of the float64 oracle; mixed precision with float64 iterative refinement
within 1e-10.  Every comparison is element by element (|x - x_ref| <= tol *
max|x_ref| per right-hand-side column) and normwise (max over columns of
||x - x_ref||_2 / ||x_ref||_2).
"""
import numpy as np
import pytest

from oracle import dm_oracle as o
from paper_1505_06864_gb300 import workloads as w

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOLMIX = 1e-10


@pytest.fixture(scope="module")
def dm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1505_06864_gb300 import build
    build.build()
    from paper_1505_06864_gb300 import dm as D
    return D


def solve(dm, s, P, levels, prec="fp64", b=None):
    plan = dm.dm_plan(s.N, s.m, s.nrhs, P, levels, prec)
    try:
        dm.dm_factor(plan, s.A, s.B, s.C)
        b = s.b if b is None else b
        x = np.zeros_like(b)
        rel = dm.dm_solve(plan, b, x)
        info = dm.dm_plan_query(plan)
    finally:
        dm.dm_destroy(plan)
    return x, rel, info


def check(x, xref, tol):
    assert np.all(np.isfinite(x))
    scale = np.max(np.abs(xref), axis=(0, 1))
    err = np.max(np.abs(x - xref), axis=(0, 1))
    assert np.all(err <= tol * scale), (err / scale, tol)
    assert o.rel_err(x, xref) <= tol


def test_config1_exact_shape(dm):
    """N=64, m=16, P=4, 1 right-hand side, dominant generator, seed 1."""
    s = w.dominant_system(64, 16, 1, 1)
    x, rel, info = solve(dm, s, 4, 1)
    check(x, o.dm(s.A, s.B, s.C, s.b, 4), TOL64)
    assert rel < 1e-14
    assert info["P"] == 4 and info["levels"] == 1 and info["max_rows"] == 16


CASES = [
    # N, m, nrhs, P, levels
    (1, 1, 1, 1, 1), (2, 3, 1, 1, 1), (3, 2, 1, 2, 1), (10, 5, 3, 3, 1), (33, 17, 2, 4, 1),
    (50, 33, 20, 5, 2), (97, 40, 3, 7, 2), (200, 8, 1, 30, 2), (200, 8, 1, 30, 3),
    (40, 64, 4, 6, 1), (12, 200, 2, 3, 1), (7, 300, 1, 2, 1), (5, 512, 1, 2, 1),
    (65, 48, 16, 32, 2), (31, 24, 17, 16, 1),
]


@pytest.mark.parametrize("N,m,r,P,levels", CASES)
def test_fp64_matches_oracle(dm, N, m, r, P, levels):
    s = w.dominant_system(N, m, r, 100 + N + m)
    x, rel, info = solve(dm, s, P, levels)
    check(x, o.dm(s.A, s.B, s.C, s.b, P, levels=levels, P2=info["P2"] if info["P2"] > 1 else None), TOL64)
    check(x, s.x_true, 1e-11)


def test_fp64_pivoting_conditioned_blocks(dm):
    s = w.conditioned_system(40, 32, 2, 7, cond=1e4)
    xt = o.refine_truth(s.A, s.B, s.C, s.b)
    for P in (1, 4, 13):
        x, rel, _ = solve(dm, s, P, 1)
        check(x, xt, 1e-11)


def test_pde_banded_shape(dm):
    s = w.pde_banded_system(130, 64, 1, 2)
    for P, lv in ((4, 1), (16, 2), (64, 2)):
        x, rel, info = solve(dm, s, P, lv)
        check(x, o.dm(s.A, s.B, s.C, s.b, P, levels=lv, P2=info["P2"] if info["P2"] > 1 else None), TOL64)


@pytest.mark.parametrize("N,m,r,P,levels", [(64, 16, 1, 4, 1), (97, 40, 3, 7, 2), (40, 128, 8, 8, 1),
                                            (9, 256, 2, 2, 1)])
def test_fp32_refined_matches_oracle(dm, N, m, r, P, levels):
    s = w.dominant_system(N, m, r, 7 + N)
    x, rel, info = solve(dm, s, P, levels, "fp32")
    check(x, o.dm(s.A, s.B, s.C, s.b, P, levels=levels, P2=info["P2"] if info["P2"] > 1 else None), TOLMIX)
    assert info["last_iters"] >= 2 and info["last_correction"] <= 1e-12


def test_fp32_refined_conditioned(dm):
    s = w.conditioned_system(64, 32, 4, 3, cond=1e4)
    xt = o.refine_truth(s.A, s.B, s.C, s.b)
    x, rel, info = solve(dm, s, 8, 1, "fp32")
    check(x, xt, TOLMIX)


def test_repeat_rhs_on_resident_factors(dm):
    s = w.dominant_system(80, 24, 3, 11)
    plan = dm.dm_plan(80, 24, 3, 6, 2, "fp64")
    try:
        dm.dm_factor(plan, s.A, s.B, s.C)
        for k in range(3):
            b = w.random_rhs(80, 24, 3, 50 + k)
            x = np.zeros_like(b)
            dm.dm_solve(plan, b, x)
            check(x, o.dm(s.A, s.B, s.C, b, 6, levels=2, P2=dm.dm_plan_query(plan)["P2"]), TOL64)
    finally:
        dm.dm_destroy(plan)


def test_device_pointers_and_alias(dm):
    import torch
    s = w.dominant_system(50, 20, 2, 5)
    T = lambda a: torch.from_numpy(a).cuda()
    plan = dm.dm_plan(50, 20, 2, 5, 1, "fp64")
    try:
        dm.dm_factor(plan, T(s.A), T(s.B), T(s.C))
        bx = T(s.b)
        dm.dm_solve(plan, bx, bx)   # x aliases b
        torch.cuda.synchronize()
        check(bx.cpu().numpy(), o.dm(s.A, s.B, s.C, s.b, 5), TOL64)
    finally:
        dm.dm_destroy(plan)


def test_singular_block_reported(dm):
    s = w.dominant_system(6, 4, 1, 1)
    s.B[3] = 0.0
    s.A[3] = 0.0
    s.C[2] = 0.0   # row 3 decoupled from row 2: its Schur complement is exactly zero
    plan = dm.dm_plan(6, 4, 1, 1, 1, "fp64")
    try:
        with pytest.raises(dm.DMError) as e:
            dm.dm_factor(plan, s.A, s.B, s.C)
        assert e.value.code == dm.DM_ESINGULAR
        assert "block row 3" in str(e.value)
    finally:
        dm.dm_destroy(plan)


def test_solve_before_factor(dm):
    plan = dm.dm_plan(8, 4, 1, 2, 1, "fp64")
    try:
        b = np.ones((8, 4, 1))
        with pytest.raises(dm.DMError) as e:
            dm.dm_solve(plan, b, np.zeros_like(b))
        assert e.value.code == dm.DM_ESTATE
    finally:
        dm.dm_destroy(plan)


@pytest.mark.parametrize("P,levels", [(64, 1), (64, 2), (64, 3), (16, 2), (4, 1)])
def test_config2_full_size(dm, P, levels):
    """N=2048 grid points x m=256 spline block, banded blocks, 1 right-hand side,
    float64 (the benchmarked workload), compared in full with the oracle."""
    s = _config2()
    x, rel, info = solve(dm, s, P, levels)
    xo = o.dm(s.A, s.B, s.C, s.b, P, levels=levels, P2=info["P2"] if info["P2"] > 1 else None)
    check(x, xo, TOL64)
    assert rel < 1e-14


_C2 = {}


def _config2():
    if "s" not in _C2:
        _C2["s"] = w.pde_banded_system(2048, 256, 1, 2)
    return _C2["s"]


def test_config3_fp32_refined_full_size(dm):
    """N=4096, m=128 dense blocks with cond(B_i)=1e4, 8 right-hand sides, float32
    factors refined in float64 to the mixed-precision tolerance."""
    s = w.conditioned_system(4096, 128, 8, 3, cond=1e4)
    x, rel, info = solve(dm, s, 0, 0, "fp32")
    xo = o.dm(s.A, s.B, s.C, s.b, info["P"], levels=info["levels"], P2=info["P2"] if info["P2"] > 1 else None)
    check(x, xo, TOLMIX)


def _batch(shapes, seed0):
    systems = [w.dominant_system(N, m, r, seed0 + i) for i, (N, m, r) in enumerate(shapes)]
    cat = lambda k: np.concatenate([getattr(s, k).reshape(-1) for s in systems])
    return systems, cat("A"), cat("B"), cat("C"), cat("b")


@pytest.mark.parametrize("prec,tol", [("fp64", TOL64), ("fp32", TOLMIX)])
def test_batch_uneven_systems(dm, prec, tol):
    """Independent systems of uneven N, m, nrhs (the batching workload's shape
    distribution, with N capped) factored and solved in the same launches;
    every system compared with the oracle at the decomposition the tuner gives it."""
    shapes = w.batch_shapes(24, 4, n_lo=5, n_hi=300, ms=(8, 16, 24, 32), r_lo=1, r_hi=6)
    shapes += [(1, 4, 1), (2, 3, 2), (300, 40, 3)]
    systems, A, B, C, b = _batch(shapes, 40)
    Ns, ms, rs = zip(*shapes)
    plan = dm.dm_plan_batch(Ns, ms, rs, prec)
    try:
        dm.dm_factor(plan, A, B, C)
        x = np.zeros_like(b)
        rel = dm.dm_solve(plan, b, x, count=len(shapes))
    finally:
        dm.dm_destroy(plan)
    off = 0
    for s, (N, m, r) in zip(systems, shapes):
        xs = x[off:off + N * m * r].reshape(N, m, r)
        off += N * m * r
        P, lv, P2 = dm.dm_plan_tune(N, m, r)
        check(xs, o.dm(s.A, s.B, s.C, s.b, P, levels=lv, P2=P2 if P2 > 1 else None), tol)
    assert max(rel) < 1e-13


_B4 = {}


def _config4_batch():
    """Uneven systems drawn like the batching workload (N ~ U{32..2048},
    m in {32, 64, 96, 128}, nrhs ~ U{1..16}), the four corners of that
    distribution forced in, the total kept small enough for the oracle."""
    if "b" not in _B4:
        shapes = [(2048, 128, 3), (1400, 96, 16), (700, 64, 1), (1200, 32, 8), (33, 128, 2), (32, 32, 16)]
        shapes += w.batch_shapes(8, 44, n_hi=600)
        systems, A, B, C, b = _batch(shapes, 80)
        ref = []
        for s, (N, m, r) in zip(systems, shapes):
            P, lv, P2 = dm_tune_host(N, m, r)
            ref.append(o.dm(s.A, s.B, s.C, s.b, P, levels=lv, P2=P2 if P2 > 1 else None))
        _B4["b"] = (shapes, systems, A, B, C, b, ref)
    return _B4["b"]


def dm_tune_host(N, m, r):
    from paper_1505_06864_gb300 import dm as D
    return D.dm_plan_tune(N, m, r)


@pytest.mark.parametrize("prec", ["tf32", "bf16x3"])
def test_batch_mixed_precision_config4_shapes(dm, prec):
    """The batching workload's launch shape on the tensor cores: m in
    {32, 64, 96, 128} mixed in one grid (shared memory sized per launch), N up
    to 2048, 1..16 right-hand sides -- refined x against the oracle per system,
    and the first pass (no refinement) within its product-error bound."""
    shapes, systems, A, B, C, b, ref = _config4_batch()
    Ns, ms, rs = zip(*shapes)
    out = {}
    for iters in (30, 1):
        plan = dm.dm_plan_batch(Ns, ms, rs, prec)
        try:
            dm.dm_set_refinement(plan, 1e-12, iters)
            dm.dm_factor(plan, A, B, C)
            x = np.zeros_like(b)
            rel = dm.dm_solve(plan, b, x, count=len(shapes), allow_notconv=(iters == 1))
            info = dm.dm_plan_query(plan)
        finally:
            dm.dm_destroy(plan)
        out[iters] = (x, rel, info)
    x, rel, info = out[30]
    assert max(rel) < 1e-13 and info["last_iters"] <= {"tf32": 6, "bf16x3": 4}[prec]
    x1 = out[1][0]
    u = {"tf32": 2.0 ** -10, "bf16x3": 2.0 ** -16}[prec]
    off = 0
    for s, (N, m, r), xo in zip(systems, shapes, ref):
        n = N * m * r
        check(x[off:off + n].reshape(N, m, r), xo, TOLMIX)
        d = np.abs(s.B.diagonal(axis1=1, axis2=2))
        rs_ = np.abs(s.A).sum(2) + np.abs(s.B).sum(2) + np.abs(s.C).sum(2)
        kappa = float(rs_.max() / (2 * d - rs_).min())
        check(x1[off:off + n].reshape(N, m, r), xo, 16.0 * kappa * u)
        off += n


def test_batch_same_as_alone(dm):
    """A system's x from a batch equals (within tolerance) its x solved alone."""
    shapes = [(120, 16, 2), (37, 24, 1), (200, 8, 3)]
    systems, A, B, C, b = _batch(shapes, 70)
    plan = dm.dm_plan_batch(*zip(*shapes), "fp64")
    try:
        dm.dm_factor(plan, A, B, C)
        x = np.zeros_like(b)
        dm.dm_solve(plan, b, x, count=3)
    finally:
        dm.dm_destroy(plan)
    off = 0
    for s, (N, m, r) in zip(systems, shapes):
        P, lv, _ = dm.dm_plan_tune(N, m, r)
        xa, _, _ = solve(dm, s, P, lv)
        check(x[off:off + N * m * r].reshape(N, m, r), xa, TOL64)
        off += N * m * r


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_graph_replay_repeats(dm, prec):
    """Repeated factor + solve on one plan: the first call runs eagerly, the
    second captures CUDA graphs, later calls replay them; all results agree
    and the launch counter advances by the same amount each time."""
    s = w.dominant_system(70, 24, 2, 21)
    plan = dm.dm_plan(70, 24, 2, 6, 2, prec)
    try:
        xs, counts = [], []
        for _ in range(4):
            c0 = dm.dm_launch_count(plan)
            dm.dm_factor(plan, s.A, s.B, s.C)
            x = np.zeros_like(s.b)
            dm.dm_solve(plan, s.b, x)
            counts.append(dm.dm_launch_count(plan) - c0)
            xs.append(x)
    finally:
        dm.dm_destroy(plan)
    tol = TOL64 if prec == "fp64" else TOLMIX
    ref = o.dm(s.A, s.B, s.C, s.b, 6, levels=2, P2=dm.dm_plan_tune(70, 24, 2, 6, 2)[2])
    for x in xs:
        check(x, ref, tol)
    assert len(set(counts)) == 1 and counts[0] > 0


def test_borrowed_inputs(dm):
    """A plan that borrows device inputs gives the copy path's x, also when the
    borrowed arrays change between calls (captured graphs are rebuilt)."""
    import torch
    s1 = w.dominant_system(60, 32, 2, 31)
    s2 = w.dominant_system(60, 32, 2, 32)
    T = lambda a: torch.from_numpy(a).cuda()
    plan = dm.dm_plan(60, 32, 2, 5, 1, "fp64")
    try:
        dm.dm_set_borrow_inputs(plan)
        with pytest.raises(dm.DMError):
            dm.dm_factor(plan, s1.A, s1.B, s1.C)        # host arrays are refused
        for s in (s1, s1, s2, s2, s1):
            A, B, C = T(s.A), T(s.B), T(s.C)
            dm.dm_factor(plan, A, B, C)
            x = np.zeros_like(s.b)
            dm.dm_solve(plan, s.b, x)
            check(x, o.dm(s.A, s.B, s.C, s.b, 5), TOL64)
    finally:
        dm.dm_destroy(plan)


def test_residual_wide_rhs_m128(dm):
    """m = 128 with 9..16 right-hand sides: the float64 residual kernel's shared
    memory (dynamic + static) goes past the default 48 KB."""
    s = w.dominant_system(20, 128, 16, 41)
    x, rel, _ = solve(dm, s, 3, 1, "fp32")
    check(x, o.dm(s.A, s.B, s.C, s.b, 3), TOLMIX)


def test_autotune_choice_used_by_plan(dm):
    P, lv, ms = dm.dm_autotune(300, 32, 2, "fp64")
    assert P >= 1 and lv >= 1 and ms > 0
    assert dm.dm_autotune(300, 32, 2, "fp64")[:2] == (P, lv)      # remembered
    s = w.dominant_system(300, 32, 2, 61)
    plan = dm.dm_plan(300, 32, 2, 0, 0, "fp64")
    try:
        q = dm.dm_plan_query(plan)
        assert (q["P"], q["levels"]) == (P, lv)
        dm.dm_factor(plan, s.A, s.B, s.C)
        x = np.zeros_like(s.b)
        dm.dm_solve(plan, s.b, x)
        check(x, o.dm(s.A, s.B, s.C, s.b, P, levels=lv, P2=q["P2"] if q["P2"] > 1 else None), TOL64)
    finally:
        dm.dm_destroy(plan)


def test_equal_time_partitions(dm):
    s = w.dominant_system(200, 24, 2, 71)
    L = o.partition_lengths_equal_time(200, 9, 24, 2)
    assert L[0] > L[1]
    plan = dm.dm_plan_ex(200, 24, 2, 9, 1, "fp64", dm.DM_PLAN_EQUAL_TIME)
    try:
        dm.dm_factor(plan, s.A, s.B, s.C)
        x = np.zeros_like(s.b)
        dm.dm_solve(plan, s.b, x)
        assert dm.dm_plan_query(plan)["max_rows"] == max(L)
    finally:
        dm.dm_destroy(plan)
    check(x, o.dm(s.A, s.B, s.C, s.b, 9, lengths=L), TOL64)


def test_laplace_fill_paper_shape_small(dm):
    """The paper's validation matrices (2-D Laplace blocks with small random
    fill), m above the tensor-core limit, float64."""
    s = w.laplace_fill_system(40, 300, 1, 3)
    x, rel, _ = solve(dm, s, 6, 1)
    check(x, o.dm(s.A, s.B, s.C, s.b, 6), TOL64)


@pytest.mark.parametrize("N,m,r,P,levels", [(64, 16, 1, 4, 1), (97, 40, 3, 7, 2), (30, 8, 2, 1, 1), (3, 5, 1, 2, 1),
                                            (200, 24, 2, 30, 2)])
def test_solve_last_row_only(dm, N, m, r, P, levels):
    """b zero except its last block row; only x_N is computed (the paper's
    application case)."""
    s = w.dominant_system(N, m, r, 90 + N)
    b = np.zeros_like(s.b)
    b[-1] = w.random_rhs(1, m, r, 5)[0]
    plan = dm.dm_plan(N, m, r, P, levels, "fp64")
    try:
        dm.dm_factor(plan, s.A, s.B, s.C)
        xl = np.zeros((m, r))
        dm.dm_solve_last(plan, np.ascontiguousarray(b[-1]), xl)
        P2 = dm.dm_plan_query(plan)["P2"]
        with pytest.raises(dm.DMError):
            q = dm.dm_plan(N, m, r, P, levels, "fp32")
            try:
                dm.dm_factor(q, s.A, s.B, s.C)
                dm.dm_solve_last(q, np.ascontiguousarray(b[-1]), xl.copy())
            finally:
                dm.dm_destroy(q)
    finally:
        dm.dm_destroy(plan)
    xo = o.dm(s.A, s.B, s.C, b, P, levels=levels, P2=P2 if P2 > 1 else None)
    check(xl[None], xo[-1:], TOL64)


@pytest.mark.parametrize("N,m,r,P,levels,prec", [(64, 16, 1, 4, 1, "fp64"), (97, 40, 3, 7, 2, "fp64"),
                                                 (130, 100, 5, 9, 2, "fp64"), (40, 200, 16, 6, 1, "fp64"),
                                                 (33, 512, 2, 4, 1, "fp64"), (97, 40, 9, 7, 2, "fp32"),
                                                 (70, 128, 8, 8, 2, "fp32"), (3, 5, 1, 2, 1, "fp64")])
def test_solve_sweep_and_per_step_kernels(dm, monkeypatch, N, m, r, P, levels, prec):
    """The persistent cluster sweep (default for <= 16 right-hand sides) and
    the per-step solve kernels (DM_SOLVE_SWEEP=0) against the oracle, on
    ragged rows per CTA (m = 5, 40, 100, 200), the largest block (m = 512)
    and the column buckets 1..16."""
    s = w.dominant_system(N, m, r, 11)
    tol = TOL64 if prec == "fp64" else TOLMIX
    out, xref = {}, None
    for flag in ("1", "0"):
        monkeypatch.setenv("DM_SOLVE_SWEEP", flag)
        x, rel, info = solve(dm, s, P, levels, prec)
        if xref is None:
            xref = o.dm(s.A, s.B, s.C, s.b, P, levels=levels, P2=info["P2"] if info["P2"] > 1 else None)
        check(x, xref, tol)
        assert rel < (1e-13 if prec == "fp64" else 1e-12)
        out[flag] = x
    monkeypatch.delenv("DM_SOLVE_SWEEP")
    check(out["1"], out["0"], tol)


@pytest.mark.parametrize("N,m,r,M,J,outer,prec", [(200, 8, 2, 4, 3, 1, "fp64"), (130, 24, 1, 3, 4, 1, "fp64"),
                                                  (301, 16, 3, 9, 3, 2, "fp64"), (512, 128, 1, 8, 4, 1, "fp64"),
                                                  (41, 6, 1, 1, 4, 1, "fp64"), (150, 32, 2, 3, 3, 1, "bf16x3"),
                                                  (150, 32, 2, 3, 3, 1, "tf32"), (97, 40, 2, 4, 2, 1, "fp32")])
def test_dm_inside_subsystems(dm, N, m, r, M, J, outer, prec):
    """DM inside the subsystems (Section 4.2.2): M subsystems, each split into
    J sub-subsystems, the outer supplementary system by block Thomas or by DM
    (outer = 2, both levels recursive) -- against the oracle's construction in
    the paper's order (every subsystem's Eq. e231 solved by DM)."""
    s = w.dominant_system(N, m, r, 1000 + N + m)
    plan = dm.dm_plan_inside(N, m, r, M, J, outer, prec)
    try:
        q = dm.dm_plan_query(plan)
        dm.dm_factor(plan, s.A, s.B, s.C)
        x = np.zeros_like(s.b)
        rel = dm.dm_solve(plan, s.b, x)
    finally:
        dm.dm_destroy(plan)
    assert q["J"] == J and q["P"] == M * J and (q["P2"] == M or M == 1)
    _, Lk, _ = o.partition_plan(N, M)
    assert q["max_rows"] == max(Li for L in Lk for Li in o.partition_plan(L, J)[1])
    xo = o.dm(s.A, s.B, s.C, s.b, M, levels=outer, J=J)
    check(x, xo, TOL64 if prec == "fp64" else TOLMIX)
    assert rel < 1e-13


@pytest.mark.parametrize("gen,N,m,r,P,levels,prec", [("dominant", 64, 16, 1, 4, 1, "fp64"),
                                                     ("dominant", 97, 20, 3, 7, 2, "fp64"),
                                                     ("pde", 130, 64, 1, 16, 2, "fp64"),
                                                     ("pde", 257, 128, 2, 32, 3, "fp64"),
                                                     ("dominant", 60, 32, 2, 6, 1, "bf16x3"),
                                                     ("pde", 130, 64, 1, 16, 2, "tf32"),
                                                     ("dominant", 41, 8, 4, 5, 1, "fp32")])
def test_complex_systems(dm, gen, N, m, r, P, levels, prec):
    """Complex systems (the paper's application has complex boundary
    conditions) through the real embedding of block size 2m, against the
    complex128 oracle: host arrays, and device tensors for the right-hand side."""
    import torch
    s = (w.dominant_system_complex(N, m, r, 300 + N) if gen == "dominant"
         else w.pde_banded_system_complex(N, m, r, 301 + N))
    plan = dm.dm_plan_complex(N, m, r, P, levels, prec)
    try:
        dm.dm_factor_complex(plan, s.A, s.B, s.C)
        x = np.zeros_like(s.b)
        rel = dm.dm_solve_complex(plan, s.b, x)
        bd = torch.from_numpy(s.b).cuda()
        xd = torch.zeros_like(bd)
        dm.dm_solve_complex(plan, bd, xd)
        torch.cuda.synchronize()
        q = dm.dm_plan_query(plan)
    finally:
        dm.dm_destroy(plan)
    xo = o.dm(s.A, s.B, s.C, s.b, P, levels=levels, P2=q["P2"] if q["P2"] > 1 else None)
    tol = TOL64 if prec == "fp64" else TOLMIX
    assert o.rel_err(x, xo) <= tol and o.rel_err(xd.cpu().numpy(), xo) <= tol
    scale = np.max(np.abs(xo), axis=(0, 1))
    assert np.all(np.max(np.abs(x - xo), axis=(0, 1)) <= tol * scale)
    assert rel < 1e-13 and q["m"] == 2 * m


def test_pinned_host_inputs(dm):
    """Page-locked host arrays are copied by a kernel through their device
    mapping (and outputs written back the same way): the same x as with
    pageable host arrays and with device arrays, also for a length that is
    not a multiple of 16 bytes."""
    import torch
    s = w.dominant_system(37, 9, 3, 17)
    pin = lambda a: torch.from_numpy(a).pin_memory()
    plan = dm.dm_plan(37, 9, 3, 4, 1, "fp64")
    try:
        dm.dm_factor(plan, pin(s.A), pin(s.B), pin(s.C))
        xp = torch.zeros(s.b.shape, dtype=torch.float64).pin_memory()
        dm.dm_solve(plan, pin(s.b), xp)
        x = np.zeros_like(s.b)
        dm.dm_factor(plan, s.A, s.B, s.C)
        dm.dm_solve(plan, s.b, x)
    finally:
        dm.dm_destroy(plan)
    assert (37 * 9 * 3 * 8) % 16 != 0
    np.testing.assert_array_equal(xp.numpy(), x)
    check(x, o.dm(s.A, s.B, s.C, s.b, 4), TOL64)


@pytest.mark.parametrize("N,m,r,P,levels", [(64, 16, 1, 4, 1), (97, 40, 3, 7, 2), (40, 64, 4, 6, 1),
                                            (12, 256, 2, 3, 1), (200, 8, 1, 30, 3), (33, 128, 16, 4, 2)])
def test_fp64_products_sliced_and_fma(dm, N, m, r, P, levels):
    """Float64 block products on the tensor cores by exact digit slicing (the
    default where a level has one block size m % 8 == 0) and on the FP64 pipe
    (DM_PLAN_FP64_FMA): both against the oracle at the float64 tolerance and
    against each other."""
    s = w.dominant_system(N, m, r, 700 + N + m)
    out = {}
    for flags in (0, dm.DM_PLAN_FP64_FMA):
        plan = dm.dm_plan_ex(N, m, r, P, levels, "fp64", flags)
        try:
            dm.dm_factor(plan, s.A, s.B, s.C)
            x = np.zeros_like(s.b)
            rel = dm.dm_solve(plan, s.b, x)
            P2 = dm.dm_plan_query(plan)["P2"]
        finally:
            dm.dm_destroy(plan)
        assert rel < 1e-14
        out[flags] = x
    xo = o.dm(s.A, s.B, s.C, s.b, P, levels=levels, P2=P2 if P2 > 1 else None)
    check(out[0], xo, TOL64)
    check(out[dm.DM_PLAN_FP64_FMA], xo, TOL64)
    check(out[0], out[dm.DM_PLAN_FP64_FMA], TOL64)


def test_autotune_variants_and_column_inverse(dm):
    """dm_autotune_ex picks (P, levels) and then the fastest kernel variant of
    the float64 sliced levels; dm_plan with P = levels = 0 applies all three.
    The column-by-column inverse (DM_PLAN_FP64_INV_COLUMN) launches no panel
    kernel and agrees with the oracle and with the blocked inverse."""
    N, m, r = 260, 64, 2
    P, lv, fl, ms = dm.dm_autotune_ex(N, m, r, "fp64")
    assert P >= 1 and lv >= 1 and ms > 0
    assert fl in (0, dm.DM_PLAN_FP64_FMA, dm.DM_PLAN_FP64_INV_COLUMN)
    assert dm.dm_autotune_ex(N, m, r, "fp64")[:3] == (P, lv, fl)   # remembered
    assert dm.dm_autotune(N, m, r, "fp64")[:2] == (P, lv)
    s = w.dominant_system(N, m, r, 67)
    plan = dm.dm_plan(N, m, r, 0, 0, "fp64")
    try:
        q = dm.dm_plan_query(plan)
        assert (q["P"], q["levels"]) == (P, lv)
        dm.dm_factor(plan, s.A, s.B, s.C)
        x = np.zeros_like(s.b)
        dm.dm_solve(plan, s.b, x)
        check(x, o.dm(s.A, s.B, s.C, s.b, P, levels=lv, P2=q["P2"] if q["P2"] > 1 else None), TOL64)
    finally:
        dm.dm_destroy(plan)
    out = {}
    for flags in (0, dm.DM_PLAN_FP64_INV_COLUMN):
        plan = dm.dm_plan_ex(N, m, r, 8, 2, "fp64", flags)
        try:
            dm.dm_factor(plan, s.A, s.B, s.C)
            dm.dm_profile(plan, True)
            dm.dm_factor(plan, s.A, s.B, s.C)
            prof = dm.dm_profile(plan, False)
            x = np.zeros_like(s.b)
            assert dm.dm_solve(plan, s.b, x) < 1e-14
            P2 = dm.dm_plan_query(plan)["P2"]
        finally:
            dm.dm_destroy(plan)
        panel = sum(v["launches"] for k, v in prof.items() if k.split("@")[0] == "inv_panel")
        assert (panel > 0) == (flags == 0), (flags, panel)
        out[flags] = x
    xo = o.dm(s.A, s.B, s.C, s.b, 8, levels=2, P2=P2 if P2 > 1 else None)
    check(out[0], xo, TOL64)
    check(out[dm.DM_PLAN_FP64_INV_COLUMN], xo, TOL64)
    check(out[0], out[dm.DM_PLAN_FP64_INV_COLUMN], TOL64)


def test_fp64_sliced_products_conditioned_blocks(dm):
    """Dense nonsymmetric blocks with cond(B_i) = 1e4 (pivoting inside the
    blocks, entries of widely different size in G_i): the digit-sliced
    products against the extended-precision truth."""
    s = w.conditioned_system(60, 64, 3, 19, cond=1e4)
    xt = o.refine_truth(s.A, s.B, s.C, s.b)
    for P, lv in ((1, 1), (6, 1), (15, 2)):
        x, rel, _ = solve(dm, s, P, lv)
        check(x, xt, 1e-11)


@pytest.mark.parametrize("N,m,r,P,levels", [(64, 16, 1, 4, 1), (40, 64, 2, 6, 2), (12, 256, 2, 3, 1),
                                            (30, 40, 3, 5, 1), (20, 200, 1, 4, 1)])
def test_fp64_blocked_inverse(dm, monkeypatch, N, m, r, P, levels):
    """The float64 block inverse by panels of 32 columns whose rank-32 updates
    run as digit-sliced tensor-core products (the default on sliced levels)
    and the column-by-column cluster inverse (DM_FP64_INVERSE=cluster): both
    against the oracle and against each other, on dominant and conditioned
    blocks (partial pivoting exercised), m not a multiple of 32 included."""
    for gen in ("dominant", "conditioned"):
        s = (w.dominant_system(N, m, r, 900 + N) if gen == "dominant"
             else w.conditioned_system(N, m, r, 901 + N, cond=1e3))
        xs = {}
        for mode in ("blocked", "cluster"):
            monkeypatch.setenv("DM_FP64_INVERSE", mode)
            x, rel, info = solve(dm, s, P, levels)
            assert rel < 1e-13
            xs[mode] = x
        monkeypatch.delenv("DM_FP64_INVERSE")
        xo = o.dm(s.A, s.B, s.C, s.b, P, levels=levels, P2=info["P2"] if info["P2"] > 1 else None)
        tol = TOL64 if gen == "dominant" else 1e-10
        check(xs["blocked"], xo, tol)
        check(xs["cluster"], xo, tol)


@pytest.mark.parametrize("N,m,r,P,levels", [(64, 16, 1, 4, 1), (40, 64, 2, 6, 2), (30, 40, 3, 5, 1),
                                            (24, 256, 1, 5, 1), (60, 32, 2, 12, 3)])
def test_fp64_sliced_assembly(dm, monkeypatch, N, m, r, P, levels):
    """The supplementary blocks (Eq. e2311) as digit-sliced tensor-core
    products (the default on sliced levels) and by the float64 kernel
    (DM_FP64_ASSEMBLY=fma): both against the oracle and against each other;
    separators with and without both off-diagonal blocks, recursion levels
    whose own supplementary blocks are sliced too, m not a multiple of 32."""
    for gen in ("dominant", "conditioned"):
        s = (w.dominant_system(N, m, r, 700 + N) if gen == "dominant"
             else w.conditioned_system(N, m, r, 701 + N, cond=1e3))
        xs = {}
        for mode in ("sliced", "fma"):
            if mode == "fma":
                monkeypatch.setenv("DM_FP64_ASSEMBLY", "fma")
            x, rel, info = solve(dm, s, P, levels)
            assert rel < 1e-13
            xs[mode] = x
        monkeypatch.delenv("DM_FP64_ASSEMBLY")
        xo = o.dm(s.A, s.B, s.C, s.b, P, levels=levels, P2=info["P2"] if info["P2"] > 1 else None)
        tol = TOL64 if gen == "dominant" else 1e-10
        check(xs["sliced"], xo, tol)
        check(xs["fma"], xo, tol)
        check(xs["sliced"], xs["fma"], tol)


@pytest.mark.parametrize("N,m,r,P,levels,hb,spike", [(48, 64, 1, 6, 2, 3, False), (40, 40, 2, 5, 1, 6, False),
                                                     (40, 40, 2, 5, 1, 7, False), (30, 256, 1, 4, 1, 3, False),
                                                     (64, 16, 2, 8, 2, 2, False), (40, 40, 2, 5, 1, 3, True)])
def test_banded_products(dm, monkeypatch, N, m, r, P, levels, hb, spike):
    """Banded off-diagonal blocks (half-bandwidth hb): with hb <= 6 the
    products with A or C as an operand run over the band in float64 (found on
    the device before each factorisation), with hb = 7 -- or one entry far from
    the diagonal in a single C block (spike) -- the tensor-core products run;
    both against the oracle and against the path with the detection off
    (DM_BANDED=0), also on recursion levels whose own blocks are dense."""
    s = w.pde_banded_system(N, m, r, 500 + N + hb, hb=hb)
    if spike:  # one off-band entry in one block; b re-manufactured for x_true
        s.C[N // 2][0][m - 1] = 0.25
        s.b[:] = w.manufacture_rhs(s.A, s.B, s.C, s.x_true)
    xs = {}
    for mode in ("auto", "off"):
        if mode == "off":
            monkeypatch.setenv("DM_BANDED", "0")
        x, rel, info = solve(dm, s, P, levels)
        assert rel < 1e-13
        xs[mode] = x
    monkeypatch.delenv("DM_BANDED")
    # the path taken: a second factorisation's profile counts banded flops
    # exactly when the first one found a band of at most 6
    plan = dm.dm_plan(N, m, r, P, levels, "fp64")
    try:
        dm.dm_factor(plan, s.A, s.B, s.C)
        dm.dm_profile(plan, True)
        dm.dm_factor(plan, s.A, s.B, s.C)
        prof = dm.dm_profile(plan, False)
    finally:
        dm.dm_destroy(plan)
    banded_flops = prof.get("banded", {}).get("flops", 0.0)
    assert (banded_flops > 0) == (hb <= 6 and not spike)
    xo = o.dm(s.A, s.B, s.C, s.b, P, levels=levels, P2=info["P2"] if info["P2"] > 1 else None)
    check(xs["auto"], xo, TOL64)
    check(xs["off"], xo, TOL64)
    check(xs["auto"], xs["off"], TOL64)


def test_singular_block_reported_blocked_inverse(dm):
    """A zero Schur complement on a sliced level (m = 16): the blocked
    inversion reports DM_ESINGULAR with the block row, like the cluster one."""
    s = w.dominant_system(6, 16, 1, 1)
    s.B[3] = 0.0
    s.A[3] = 0.0
    s.C[2] = 0.0
    plan = dm.dm_plan(6, 16, 1, 1, 1, "fp64")
    try:
        with pytest.raises(dm.DMError) as e:
            dm.dm_factor(plan, s.A, s.B, s.C)
        assert e.value.code == dm.DM_ESINGULAR
        assert "block row 3" in str(e.value)
    finally:
        dm.dm_destroy(plan)
