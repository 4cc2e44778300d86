"""Pins for the CPU oracle (oracle/dm_oracle.py) against facts fixed by the
paper and by mathematics, not against the oracle itself.

* dense Gaussian elimination (itself pinned to LAPACK) on tiny systems,
* manufactured solutions x_true with b = T x_true,
* exact multiplicative-operation counts of Table 1, Table 2, Eq. (DMtotal) and
  Eq. (DMrec1) under the paper's cost model (Section 4),
* the optimum parameters the paper prints (Section 5),
* planted mistakes in a copy of the oracle must fail at least one pin.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import dm_oracle as o
from paper_1505_06864_gb300 import workloads as w

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _tiny_cases():
    for (N, m, l, seed) in [(1, 1, 1, 1), (1, 3, 2, 2), (2, 2, 1, 3), (3, 1, 1, 4),
                            (5, 3, 2, 5), (7, 2, 3, 6), (9, 4, 1, 7), (12, 3, 2, 8)]:
        yield N, m, l, seed


# ---------------------------------------------------------------- dense GE
def test_dense_ge_matches_lapack():
    rng = np.random.default_rng(0)
    for n in (1, 2, 5, 17):
        T = rng.standard_normal((n, n)) + n * np.eye(n)
        b = rng.standard_normal((n, 3))
        np.testing.assert_allclose(o.dense_ge(T, b), np.linalg.solve(T, b), rtol=1e-12, atol=1e-12)


def test_dense_ge_needs_pivoting():
    # a zero leading pivot: elimination without row exchange would divide by 0
    T = np.array([[0.0, 1.0, 2.0], [3.0, 1.0, 0.0], [1.0, 4.0, 1.0]])
    b = np.array([[1.0], [2.0], [3.0]])
    np.testing.assert_allclose(o.dense_ge(T, b), np.linalg.solve(T, b), rtol=1e-13)


def test_dense_from_blocks_layout():
    s = w.dominant_system(3, 2, 1, 9)
    T = o.dense_from_blocks(s.A, s.B, s.C)
    np.testing.assert_array_equal(T[2:4, 0:2], s.A[1])
    np.testing.assert_array_equal(T[2:4, 2:4], s.B[1])
    np.testing.assert_array_equal(T[2:4, 4:6], s.C[1])
    np.testing.assert_array_equal(T[0:2, 4:6], 0.0)
    # b = T x_true, built by the generator, agrees with the dense product
    np.testing.assert_allclose(T @ s.x_true.reshape(-1, 1), s.b.reshape(-1, 1), rtol=1e-14)


# ---------------------------------------------------------------- TA and DM vs dense GE
@pytest.mark.parametrize("N,m,l,seed", list(_tiny_cases()))
def test_thomas_matches_dense_ge(N, m, l, seed):
    s = w.dominant_system(N, m, l, seed)
    xd = o.dense_ge(o.dense_from_blocks(s.A, s.B, s.C), s.b.reshape(-1, l)).reshape(N, m, l)
    assert o.rel_err(o.thomas(s.A, s.B, s.C, s.b), xd) < 1e-13


@pytest.mark.parametrize("N,m,l,seed", [c for c in _tiny_cases() if c[0] >= 3])
def test_dm_matches_dense_ge_all_partitions(N, m, l, seed):
    s = w.dominant_system(N, m, l, seed)
    xd = o.dense_ge(o.dense_from_blocks(s.A, s.B, s.C), s.b.reshape(-1, l)).reshape(N, m, l)
    for P in range(1, (N + 1) // 2 + 1):
        for levels in (1, 2, 3):
            x = o.dm(s.A, s.B, s.C, s.b, P, levels=levels)
            assert o.rel_err(x, xd) < 1e-13, (P, levels)


def test_dm_general_nonsymmetric_blocks():
    # pivoting inside a block: conditioned blocks, not point-wise dominant
    s = w.conditioned_system(6, 4, 2, 11, cond=1e3)
    xd = o.dense_ge(o.dense_from_blocks(s.A, s.B, s.C), s.b.reshape(-1, 2)).reshape(6, 4, 2)
    for P in (1, 2, 3):
        assert o.rel_err(o.dm(s.A, s.B, s.C, s.b, P), xd) < 1e-11


def test_p1_is_thomas_bitwise():
    s = w.dominant_system(20, 5, 2, 3)
    np.testing.assert_array_equal(o.dm(s.A, s.B, s.C, s.b, 1), o.thomas(s.A, s.B, s.C, s.b))


def test_separator_rows_equal_h():
    s = w.dominant_system(30, 4, 2, 4)
    x, parts = o.dm(s.A, s.B, s.C, s.b, 5, return_parts=True)
    for j, q in enumerate(parts["seps"]):
        np.testing.assert_array_equal(x[q], parts["h"][j])
    # the supplementary system is block-tridiagonal with zero corner blocks
    assert np.all(parts["HA"][0] == 0) and np.all(parts["HC"][-1] == 0)


def test_manufactured_solution_and_residual():
    for gen, tol in ((w.dominant_system, 1e-13), (w.pde_banded_system, 1e-13)):
        s = gen(96, 12, 3, 21)
        for P in (1, 4, 16):
            x = o.dm(s.A, s.B, s.C, s.b, P)
            assert o.rel_err(x, s.x_true) < tol
            r = o.residual(s.A, s.B, s.C, x, s.b)
            assert np.linalg.norm(r) / np.linalg.norm(s.b) < 1e-15


def _dyadic_ill_conditioned(N=4, eps_pow=22, seed=3):
    """A block-tridiagonal system (m = 3, two right-hand sides) whose entries
    are dyadic rationals with few bits, an integer solution x and b = T x
    formed exactly (checked with Fractions), so x is known without rounding.
    Every B_i has rows [1, 1, 0], [1, 1 + 2^-eps_pow, 0] and every A_i, C_i has
    equal columns 0 and 1, so (1, -1, 0) placed in any block row is nearly a
    null vector of T: cond(T) ~ 2^eps_pow."""
    from fractions import Fraction as Fr
    m = 3
    rng = np.random.default_rng(seed)
    A, B, C = (np.zeros((N, m, m)) for _ in range(3))
    for i in range(N):
        a = rng.integers(-4, 5) / 8.0
        B[i] = [[1, 1, 0], [1, 1 + 2.0 ** -eps_pow, 0], [a, a, 2]]
        for M_, on in ((A, i > 0), (C, i < N - 1)):
            if on:
                Mi = rng.integers(-2, 3, (m, m)) / 16.0
                Mi[:, 1] = Mi[:, 0]
                M_[i] = Mi
    x = rng.integers(-8, 9, (N, m, 2)).astype(np.float64)
    b = np.zeros((N, m, 2))
    for i in range(N):
        for r in range(m):
            for c in range(2):
                acc = Fr(0)
                for k in range(m):
                    acc += Fr(B[i, r, k]) * Fr(x[i, k, c])
                    if i > 0:
                        acc += Fr(A[i, r, k]) * Fr(x[i - 1, k, c])
                    if i < N - 1:
                        acc += Fr(C[i, r, k]) * Fr(x[i + 1, k, c])
                b[i, r, c] = float(acc)
                assert Fr(b[i, r, c]) == acc          # b is exact in float64
    return A, B, C, x, b


def test_refine_truth_reaches_exact_solution():
    """refine_truth against an exactly known x on a system with cond(T) ~ 2e7:
    the plain float64 solve is off by ~1e-5 and refinement with float64
    residuals stalls near cond * 2^-53 (here 2.5e-10); refine_truth's
    extended-precision residuals must get within 1e-12 (on x86 long double,
    u = 2^-64; binary128 elsewhere)."""
    A, B, C, x, b = _dyadic_ill_conditioned()
    assert np.linalg.cond(o.dense_from_blocks(A, B, C)) > 1e7
    assert o.rel_err(o.thomas(A, B, C, b), x) > 1e-7
    xt = o.refine_truth(A, B, C, b)
    assert o.rel_err(xt, x) < 1e-12
    # the same loop with float64 residuals cannot pass this pin
    xf = o.thomas(A, B, C, b)
    for _ in range(6):
        xf = xf + o.thomas(A, B, C, o.residual(A, B, C, xf, b))
    assert o.rel_err(xf, x) > 1e-11


def test_refine_truth_reduces_extended_residual():
    s = w.conditioned_system(10, 8, 1, 5, cond=1e4)
    x0 = o.thomas(s.A, s.B, s.C, s.b)
    xt = o.refine_truth(s.A, s.B, s.C, s.b)
    r0 = o.residual(s.A, s.B, s.C, x0.astype(np.longdouble), s.b, np.longdouble)
    r1 = o.residual(s.A, s.B, s.C, xt.astype(np.longdouble), s.b, np.longdouble)
    assert float(np.linalg.norm(r1.astype(np.float64))) <= float(np.linalg.norm(r0.astype(np.float64)))
    assert o.rel_err(xt, x0) < 1e-10


# ---------------------------------------------------------------- partition plan
@pytest.mark.parametrize("N,P", [(3, 2), (64, 4), (65, 4), (2048, 64), (9, 5), (100, 1), (1, 1)])
def test_partition_plan(N, P):
    st, L, seps = o.partition_plan(N, P)
    assert len(L) == P and len(seps) == P - 1
    assert sum(L) == N - (P - 1)          # sum N_k = N - (M - 1), Section 4.1
    assert min(L) >= 1 and max(L) - min(L) <= 1
    assert L == sorted(L, reverse=True)   # remainder on the lowest subsystems
    covered = sorted([st[k] + t for k in range(P) for t in range(L[k])] + seps)
    assert covered == list(range(N))
    assert all(1 <= q <= N - 2 for q in seps)  # rows 2..N-1 in 1-based counting


def test_partition_plan_rejects():
    for N, P in ((4, 3), (1, 2), (10, 0)):
        with pytest.raises(ValueError):
            o.partition_plan(N, P)


# ---------------------------------------------------------------- operation counts (Section 4)
@pytest.mark.parametrize("N,n,l", [(1, 3, 1), (2, 4, 2), (17, 5, 3), (40, 2, 7)])
def test_ta_counts_table1(N, n, l):
    s = w.dominant_system(N, n, l, 2)
    ctr = o.OpCounter()
    o.thomas(s.A, s.B, s.C, s.b, ctr)
    parts = o.mo_ta_parts(N, n, l)
    for k, v in parts.items():
        assert ctr.total(k) == v, k
    assert ctr.total() == o.mo_ta(N, n, l) == sum(parts.values())


@pytest.mark.parametrize("N,P,n,l", [(40, 5, 5, 2), (41, 4, 3, 1), (64, 4, 16, 1), (23, 11, 2, 3),
                                     (9, 2, 4, 4), (30, 3, 6, 9)])
def test_dm_counts_table2_and_dmtotal(N, P, n, l):
    s = w.dominant_system(N, n, l, 3)
    ctr = o.OpCounter()
    o.dm(s.A, s.B, s.C, s.b, P, ctr=ctr)
    _, Ls, _ = o.partition_plan(N, P)
    for k in range(P):
        assert ctr.total(f"solve/{k}") == o.mo_dm_solve(k + 1, P, Ls[k], n, l)
        assert ctr.total(f"wing/{k}") == o.mo_dm_wing(k + 1, P, n, l)
        assert ctr.total(f"back/{k}") == o.mo_dm_back(k + 1, P, Ls[k], n, l)
    assert ctr.total("supp") == o.mo_dm_supp(P, n, l)
    assert ctr.total() == o.mo_dm_total(Ls, n, l)


@pytest.mark.parametrize("N,P,n,l", [(40, 13, 3, 2), (101, 21, 2, 1), (60, 9, 4, 3)])
def test_dm_counts_dmrec1(N, P, n, l):
    s = w.dominant_system(N, n, l, 4)
    ctr = o.OpCounter()
    o.dm(s.A, s.B, s.C, s.b, P, levels=2, ctr=ctr)
    _, Ls, _ = o.partition_plan(N, P)
    p2 = o.supp_partitions(P - 1, P, l, n)
    assert p2 >= 2
    _, Ms, _ = o.partition_plan(P - 1, p2)
    assert sum(Ms) == P - p2            # M_j sum to (M - m), Section 4.2.1
    assert ctr.total() == o.mo_dm_rec1(Ls, Ms, n, l)


def test_table2_totals_are_sums_of_rows():
    # Eq. (DMtotal) is the sum of Table 2's rows for every k plus the supplementary term
    for Ns in ([5, 4, 4, 4], [3, 3], [7, 6, 6, 6, 6, 6, 6]):
        M, n, l = len(Ns), 6, 2
        rows = sum(o.mo_dm_solve(k + 1, M, Ns[k], n, l) + o.mo_dm_wing(k + 1, M, n, l)
                   + o.mo_dm_back(k + 1, M, Ns[k], n, l) for k in range(M))
        assert rows + o.mo_dm_supp(M, n, l) == o.mo_dm_total(Ns, n, l)


# ---------------------------------------------------------------- DM inside subsystems (Section 4.2.2)
@pytest.mark.parametrize("N,m,l,P,J,seed", [(40, 3, 2, 2, 2, 5), (40, 3, 2, 3, 3, 6), (31, 2, 1, 3, 2, 7),
                                            (57, 4, 3, 4, 3, 8), (25, 2, 2, 2, 5, 9)])
def test_dm_inside_matches_dense_ge(N, m, l, P, J, seed):
    s = w.dominant_system(N, m, l, seed)
    xd = o.dense_ge(o.dense_from_blocks(s.A, s.B, s.C), s.b.reshape(-1, l)).reshape(N, m, l)
    for levels in (1, 2):
        assert o.rel_err(o.dm(s.A, s.B, s.C, s.b, P, levels=levels, J=J), xd) < 1e-13


def test_dm_inside_conditioned_blocks_matches_dense_ge():
    s = w.conditioned_system(23, 4, 2, 12, cond=1e3)
    xd = o.dense_ge(o.dense_from_blocks(s.A, s.B, s.C), s.b.reshape(-1, 2)).reshape(23, 4, 2)
    assert o.rel_err(o.dm(s.A, s.B, s.C, s.b, 3, J=3), xd) < 1e-11


@pytest.mark.parametrize("N,P,J,n,l", [(40, 2, 2, 3, 2), (40, 3, 3, 3, 2), (61, 4, 3, 2, 5), (52, 3, 4, 4, 1),
                                       (33, 5, 2, 3, 3)])
def test_dm_inside_counts_dmrec121_1212_122(N, P, J, n, l):
    """The instrumented count of each subsystem's Eq. (e231) solved by DM with
    J sub-subsystems equals Eq. (DMrec121) for k = 1, Eq. (DMrec1212) for
    k = M and Eq. (DMrec122) in between, exactly, for the sub-subsystem sizes
    the partition produces (unequal ones included)."""
    s = w.dominant_system(N, n, l, 13)
    ctr = o.OpCounter()
    o.dm(s.A, s.B, s.C, s.b, P, J=J, ctr=ctr)
    _, Ls, _ = o.partition_plan(N, P)
    for k in range(P):
        _, Lk, _ = o.partition_plan(Ls[k], J)
        f = o.mo_dm_sub_first if k == 0 else (o.mo_dm_sub_last if k == P - 1 else o.mo_dm_sub_mid)
        assert ctr.total(f"solve/{k}") == f(Lk, n, l), k
        # the inner supplementary system's share is the formulas' last term
        inner = {0: (4 * J - 6), P - 1: (6 * J - 10)}.get(k, 7 * J - 11)
        assert ctr.total(f"solve/{k}/supp") == inner * n ** 3 + (3 * J - 5) * n ** 2 * l
        # the rest of Eq. (DMtotal) is unchanged (Table 2 wings, Eq. endSolution)
        assert ctr.total(f"wing/{k}") == o.mo_dm_wing(k + 1, P, n, l)
        assert ctr.total(f"back/{k}") == o.mo_dm_back(k + 1, P, Ls[k], n, l)
    assert ctr.total("supp") == o.mo_dm_supp(P, n, l)


def test_dm_inside_serial_count_dmrec3():
    """Eq. (DMrec3) is the serial count with P = M J processors: one middle
    sub-subsystem of a middle subsystem (N_2 rows), that subsystem's inner
    supplementary system, its wing products, the supplementary system of
    Eq. (e232) and its rows of Eq. (endSolution) -- read off the counter."""
    n, l, M, J, N2 = 3, 2, 3, 3, 2
    N1 = J * N2 + J - 1
    N = M * N1 + M - 1
    s = w.dominant_system(N, n, l, 14)
    ctr = o.OpCounter()
    o.dm(s.A, s.B, s.C, s.b, M, J=J, ctr=ctr)
    k, i = 1, 1
    serial = (ctr.total(f"solve/{k}/sub/{i}") + ctr.total(f"solve/{k}/supp") + ctr.total(f"wing/{k}")
              + ctr.total("supp") + ctr.total(f"back/{k}"))
    assert ctr.total(f"solve/{k}/sub/{i}") == N2 * (11 * n ** 3 + 5 * n ** 2 * l)
    assert serial == o.mo_dm_rec3(N, M, J, n, l)


def test_dm_both_levels_serial_count_dmrec4():
    """Eq. (DMrec4): Eq. (DMrec3) with the supplementary system solved by DM
    with m subsystems of M_j = (M - m)/m rows: its serial part is one middle
    subsystem of that DM plus its own supplementary system."""
    n, l, msub, Mj, J, N2 = 3, 2, 3, 1, 3, 1
    M = msub * (Mj + 1)
    N1 = J * N2 + J - 1
    N = M * N1 + M - 1
    s = w.dominant_system(N, n, l, 15)
    ctr = o.OpCounter()
    o.dm(s.A, s.B, s.C, s.b, M, levels=2, P2=msub, J=J, ctr=ctr)
    k, i, j = 1, 1, 1
    supp_serial = (ctr.total(f"supp/solve/{j}") + ctr.total(f"supp/wing/{j}") + ctr.total(f"supp/back/{j}")
                   + ctr.total("supp/supp"))
    serial = (ctr.total(f"solve/{k}/sub/{i}") + ctr.total(f"solve/{k}/supp") + ctr.total(f"wing/{k}")
              + supp_serial + ctr.total(f"back/{k}"))
    assert serial == o.mo_dm_rec4(N, M, J, msub, n, l)


@pytest.mark.parametrize("N,m,l,M,J,outer,seed", [(60, 3, 2, 3, 3, 1, 18), (101, 2, 1, 4, 4, 1, 19),
                                                  (130, 3, 2, 7, 3, 2, 20), (41, 2, 3, 1, 4, 1, 21)])
def test_dm_inside_equals_aligned_form(N, m, l, M, J, outer, seed):
    """DM inside the subsystems (the paper's construction, Section 4.2.2) and
    the form the library executes -- DM with the M J sub-subsystems whose
    supplementary system is split into M parts at the outer separators, so
    that part k is subsystem k's inner supplementary system -- give the same
    x; the executed form never forms the subsystem spikes over all rows and
    so counts fewer multiplicative operations."""
    s = w.dominant_system(N, m, l, seed)
    c1, c2 = o.OpCounter(), o.OpCounter()
    x1 = o.dm(s.A, s.B, s.C, s.b, M, levels=outer, J=J, ctr=c1)
    _, Lk, _ = o.partition_plan(N, M)
    nested = [Li for L in Lk for Li in o.partition_plan(L, J)[1]]
    x2 = o.dm(s.A, s.B, s.C, s.b, M * J, levels=outer + 1, P2=M, lengths=nested, ctr=c2)
    assert o.rel_err(x1, x2) < 1e-13
    # the supplementary partition of the executed form falls on the outer separators
    assert o.partition_plan(M * J - 1, M)[1] == [J - 1] * M
    # (with M = 1 there are no subsystem spikes and the two forms coincide)
    assert c2.total() < c1.total() if M > 1 else c2.total() == c1.total()


# ---------------------------------------------------------------- complex systems (Section 7's boundary conditions)
def test_complex_dense_ge_matches_lapack():
    rng = np.random.default_rng(3)
    for n in (1, 3, 8):
        T = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)) + n * np.eye(n)
        b = rng.standard_normal((n, 2)) + 1j * rng.standard_normal((n, 2))
        np.testing.assert_allclose(o.dense_ge(T, b), np.linalg.solve(T, b), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("gen", ["dominant", "pde"])
def test_complex_dm_matches_dense_ge(gen):
    N, m, l = 13, 3, 2
    s = (w.dominant_system_complex(N, m, l, 22) if gen == "dominant" else w.pde_banded_system_complex(N, m, l, 23))
    assert np.iscomplexobj(s.A) and np.abs(s.B[-1].imag).max() > 0
    xd = o.dense_ge(o.dense_from_blocks(s.A, s.B, s.C), s.b.reshape(-1, l)).reshape(N, m, l)
    assert o.rel_err(xd, s.x_true) < 1e-13
    for P, lv, J in ((1, 1, None), (3, 1, None), (4, 2, None), (2, 1, 2), (3, 2, 2)):
        x = o.dm(s.A, s.B, s.C, s.b, P, levels=lv, J=J)
        assert np.iscomplexobj(x) and o.rel_err(x, xd) < 1e-13, (P, lv, J)
    xt = o.refine_truth(s.A, s.B, s.C, s.b)
    assert o.rel_err(xt, s.x_true) < 1e-14


def test_real_embedding_identity():
    """The identity the complex path of the library relies on: with
    X + iY -> [[X, -Y], [Y, X]] for every block and u + iv -> [u; v] for every
    right-hand-side block, the real system's solution is [Re x; Im x] of the
    complex system's (written out here, independently of the library)."""
    s = w.dominant_system_complex(11, 4, 3, 24)
    emb = lambda M: np.block([[M.real, -M.imag], [M.imag, M.real]])
    E = lambda Ms: np.stack([emb(M) for M in Ms])
    bR = np.concatenate([s.b.real, s.b.imag], axis=1)
    xR = o.dm(E(s.A), E(s.B), E(s.C), bR, 3)
    xc = o.dm(s.A, s.B, s.C, s.b, 3)
    np.testing.assert_allclose(xR[:, :4] + 1j * xR[:, 4:], xc, rtol=0, atol=1e-13 * np.abs(xc).max())


# ---------------------------------------------------------------- Section 5.1 speedups from counted runs
def _serial_count(ctr, ks):
    return sum(ctr.total(f"{st}/{k}") for k in ks for st in ("solve", "wing", "back")) + ctr.total("supp")


def test_speedup_unequal_from_counted_run():
    """Eq. (SpeedupMPNk) is Mo_TA over the serial count of a run whose first
    and last subsystems are alpha and beta times a middle one (the middle
    subsystems take the longest): both counts come from the instrumented
    solvers, not from the formulas."""
    n, l = 4, 2
    Nk, a, b, P = 4, 6, 5, 5
    lengths = [a] + [Nk] * (P - 2) + [b]
    N = sum(lengths) + P - 1
    s = w.dominant_system(N, n, l, 16)
    cta, ctr = o.OpCounter(), o.OpCounter()
    o.thomas(s.A, s.B, s.C, s.b, cta)
    o.dm(s.A, s.B, s.C, s.b, P, lengths=lengths, ctr=ctr)
    per = [_serial_count(ctr, [k]) - ctr.total("supp") for k in range(P)]
    assert max(per) == per[1]                       # a middle subsystem sets the time
    S = cta.total() / _serial_count(ctr, [1])
    assert o.speedup_mp_unequal(N, P, n, l, a / Nk, b / Nk) == pytest.approx(S, rel=1e-13)
    # alpha = beta = 1 is Eq. (SpeedupMP)
    assert o.speedup_mp_unequal(61, 6, n, l, 1.0, 1.0) == pytest.approx(o.speedup_mp(61, 6, n, l), rel=1e-15)


@pytest.mark.parametrize("i", [1, 2, 3])
def test_speedup_queue_from_counted_run(i):
    """Eq. (SpeedupMiPNk): M = iP subsystems, a processor runs i middle
    subsystems one after another, then the supplementary system."""
    n, l, P = 3, 1, 3
    Nk, a, b = 4, 7, 5
    M = i * P
    lengths = [a] + [Nk] * (M - 2) + [b]
    N = sum(lengths) + M - 1
    s = w.dominant_system(N, n, l, 17)
    cta, ctr = o.OpCounter(), o.OpCounter()
    o.thomas(s.A, s.B, s.C, s.b, cta)
    o.dm(s.A, s.B, s.C, s.b, M, lengths=lengths, ctr=ctr)
    S = cta.total() / _serial_count(ctr, list(range(1, i + 1)))
    assert o.speedup_queue(N, P, i, n, l, a / Nk, b / Nk) == pytest.approx(S, rel=1e-13)


# ---------------------------------------------------------------- Section 5 formulas
def test_printed_optimum_both_levels():
    g = GOLD["optimum_both_levels"]
    M, msub, J = o.mmj_opt_rec4_free(g["N"], g["n"], g["l"])
    assert round(M) == g["M"] and round(J) == g["J"] and round(msub) == g["m"]


def test_maxspeed_p_and_linear_slope():
    n, l, N = 400, 1, 3071
    P = o.p_opt_mp(N, n, l)
    assert abs(P - math.sqrt(7 * (N + 1) / 3)) / P < 0.01         # "close to sqrt(7(N+1)/3)"
    s = [o.speedup_mp(N, p, n, l) for p in range(2, 200)]
    assert abs((2 + int(np.argmax(s))) - P) <= 1                   # the maximum of Eq. (SpeedupMP)
    # S ~ 3P/7 for P << N: the slope of the l << n model at small P
    slope = o.speedup_mp(10 ** 9, 8, 10 ** 6, 1) / 8
    assert abs(slope - GOLD["linear_speedup_slopes"]["nonrecursive"]) < 1e-3
    for p in (4, 16, 64):
        assert o.speedup_mp(N, p, n, l) > o.speedup_mp_bound(N, p)


def test_supp_dm_optimum():
    n, l = 10 ** 6, 1                   # l << n
    assert o.m_opt_supp(20, n, l) == pytest.approx(20 / 3)          # boundary m = P/3 below P = 21
    msub = o.m_opt_supp(GOLD["supp_dm_condition"]["P_min"], n, l)
    assert (21 - msub) / msub >= 2.0
    assert (20 - math.sqrt(20 * 7 / 3)) / math.sqrt(20 * 7 / 3) < 2.0
    # Eq. (Speedup521) is Eq. (DMrec2) at m = sqrt(7P/3), l -> 0
    N, P = 3071, 64
    msub = math.sqrt(7 * P / 3)
    s_rec2 = (3 * N - 2) * n ** 3 / o.mo_dm_rec2((N - P + 1) / P, (P - msub) / msub, msub, n, 0)
    assert s_rec2 == pytest.approx(o.speedup_rec_supp_small_l(N, P), rel=1e-12)
    # Eq. (SuppMatrM) minimises Eq. (DMrec2) over m for fixed P
    ms = np.linspace(2, 20, 20001)
    N1 = (N - P + 1) / P
    f = [o.mo_dm_rec2(N1, (P - v) / v, v, 400, 1) for v in ms]
    assert abs(ms[int(np.argmin(f))] - o.m_opt_supp(P, 400, 1)) < 0.01


def test_supp_free_optimum_is_minimum():
    N, n, l = 3071, 400, 1
    P, msub = o.p_m_opt_supp_free(N, n, l)
    f0 = o.mo_dm_rec2((N - P + 1) / P, (P - msub) / msub, msub, n, l)
    for dP, dm_ in ((3, 0), (-3, 0), (0, 1), (0, -1), (2, 1)):
        P1, m1 = P + dP, msub + dm_
        assert o.mo_dm_rec2((N - P1 + 1) / P1, (P1 - m1) / m1, m1, n, l) > f0


def test_inside_subsystems_optimum():
    N, n, l = 3071, 400, 1
    M, J = o.mj_opt_rec3_free(N, n, l)
    f0 = o.mo_dm_rec3(N, M, J, n, l)
    for dM, dJ in ((5, 0), (-5, 0), (0, 0.5), (0, -0.5)):
        assert o.mo_dm_rec3(N, M + dM, J + dJ, n, l) > f0
    # fixed P: Eq. (ParamDMrec3) minimises Eq. (DMrec3) along M J = P
    P = 400
    Mf, Jf = o.mj_opt_rec3_fixed_p(N, P, n, l)
    f1 = o.mo_dm_rec3(N, Mf, Jf, n, l)
    for Mv in (Mf * 0.9, Mf * 1.1):
        assert o.mo_dm_rec3(N, Mv, P / Mv, n, l) > f1
    # "S ~ 3P/11" for small P
    Nb, nb = 10 ** 9, 10 ** 6
    Mf, Jf = o.mj_opt_rec3_fixed_p(Nb, 12, nb, 1)
    s = o.mo_ta(Nb, nb, 1) / o.mo_dm_rec3(Nb, Mf, Jf, nb, 1)
    assert abs(s / 12 - GOLD["linear_speedup_slopes"]["inside_subsystems"]) < 0.01


def test_both_levels_fixed_p_optimum():
    N, n, l, P = 3071, 400, 1, 600
    M, msub, J = o.mmj_opt_rec4_fixed_p(N, P, n, l)
    f0 = o.mo_dm_rec4(N, M, J, msub, n, l)
    for fM in (0.9, 1.1):
        Mv = M * fM
        mv = math.sqrt(Mv * (7 * n ** 3 + 5 * n ** 2 * l) / (3 * (n ** 3 + n ** 2 * l)))
        assert o.mo_dm_rec4(N, Mv, P / Mv, mv, n, l) > f0


def test_equal_time_sizes():
    g = GOLD["equal_time_ratios"]
    n = 10 ** 6
    Nk = 10 ** 6
    N1, NM = o.first_last_sizes(Nk, n, 1)
    assert N1 / Nk == pytest.approx(g["alpha"], rel=1e-5)
    assert NM / Nk == pytest.approx(g["beta"], rel=1e-5)
    # interval endpoints printed after Eq. (SpeedupMPNk), read as l << n and l = n
    Nk = 40
    assert o.first_last_sizes(Nk, n, 1)[0] == pytest.approx((7 * Nk + 1) / 4, rel=1e-5)
    assert o.first_last_sizes(Nk, 8, 8)[0] == pytest.approx((6 * Nk + 1) / 4)
    assert o.first_last_sizes(Nk, n, 1)[1] == pytest.approx((7 * Nk + 3) / 6, rel=1e-5)
    assert o.first_last_sizes(Nk, 8, 8)[1] == pytest.approx((12 * Nk + 4) / 10)


# ---------------------------------------------------------------- generator
def test_splitmix64_reference_value():
    v = w._mix64(np.array([0x9E3779B97F4A7C15], dtype=np.uint64))[0]
    assert hex(int(v)) == GOLD["splitmix64_first_output"]["value"]


def test_generators_deterministic_and_dominant():
    a = w.dominant_system(6, 4, 2, 5)
    b = w.dominant_system(6, 4, 2, 5)
    for u, v in zip((a.A, a.B, a.C, a.b), (b.A, b.B, b.C, b.b)):
        np.testing.assert_array_equal(u, v)
    T = o.dense_from_blocks(a.A, a.B, a.C)
    d = np.abs(np.diag(T))
    off = np.sum(np.abs(T), axis=1) - d
    assert np.all(d - off >= 1.0 - 1e-12)
    assert np.all(a.A[0] == 0) and np.all(a.C[-1] == 0)
    p = w.pde_banded_system(4, 10, 1, 2)
    r, c = np.nonzero(p.B[1])
    assert np.max(np.abs(r - c)) == 3
    q = w.conditioned_system(3, 16, 1, 3, cond=1e4)
    assert np.linalg.cond(q.B[1]) == pytest.approx(1e4, rel=1e-6)
    sh = w.batch_shapes(200, 4)
    assert all(32 <= n <= 2048 and m in (32, 64, 96, 128) and 1 <= r <= 16 for n, m, r in sh)


# ---------------------------------------------------------------- planted mistakes
def _mutated_dm(monkeypatch, kind):
    """Run DM with a mistake planted in the oracle's block operations."""
    real_mul = o._mul
    if kind == "transpose":
        def mul(X, Y, ctr):
            if X is None or Y is None:
                return None
            return X.T @ Y if X.shape[0] == X.shape[1] and X.shape[0] > 1 else X @ Y
        monkeypatch.setattr(o, "_mul", mul)
    elif kind == "sign":
        def sub(X, Y):
            if Y is None:
                return X
            if X is None:
                return Y          # wrong sign
            return X - Y
        monkeypatch.setattr(o, "_sub", sub)
    elif kind == "drop_left":
        orig = o.dm

        def dm_drop(*a, **k):
            x, parts = orig(*a, return_parts=True, **{kk: v for kk, v in k.items() if kk != "return_parts"})
            st, L = parts["starts"], parts["lengths"]
            for kk in range(1, len(L)):
                for t in range(L[kk]):
                    x[st[kk] + t] += parts["ZL"][kk][t] @ parts["h"][kk - 1]
            return x
        return dm_drop
    return o.dm


@pytest.mark.parametrize("kind", ["transpose", "sign", "drop_left"])
def test_planted_mistakes_are_caught(monkeypatch, kind):
    s = w.dominant_system(9, 3, 2, 12)
    xd = o.dense_ge(o.dense_from_blocks(s.A, s.B, s.C), s.b.reshape(-1, 2)).reshape(9, 3, 2)
    f = _mutated_dm(monkeypatch, kind)
    x = f(s.A, s.B, s.C, s.b, 3)
    assert o.rel_err(x, xd) > 1e-6


def test_device_generator_bit_identical_uniforms():
    torch = pytest.importorskip("torch")
    a = w.uniform(7, 3, 1000, -1.0, 1.0, offset=12345)
    b = w.uniform_t(7, 3, 1000, -1.0, 1.0, offset=12345, device="cpu").numpy()
    np.testing.assert_array_equal(a, b)
    s = w.dominant_system(5, 4, 2, 9)
    A, B, C, bb, x = w.dominant_system_t(5, 4, 2, 9, device="cpu")
    np.testing.assert_array_equal(s.A, A.numpy())
    np.testing.assert_array_equal(s.B, B.numpy())     # same draws and same shift summation order
    np.testing.assert_allclose(s.x_true, x.numpy(), rtol=1e-13)


# ---------------------------------------------------------------- equal-time subsystems (Section 5.1)
def _per_subsystem_counts(Ls, n, l):
    M = len(Ls)
    return [o.mo_dm_solve(k + 1, M, Ls[k], n, l) + o.mo_dm_wing(k + 1, M, n, l) + o.mo_dm_back(k + 1, M, Ls[k], n, l)
            for k in range(M)]


@pytest.mark.parametrize("N,P,n,l", [(2048, 64, 256, 1), (3071, 64, 400, 1), (3071, 16, 100, 1), (500, 7, 50, 50)])
def test_equal_time_sizes_balance_table2(N, P, n, l):
    L = o.partition_lengths_equal_time(N, P, n, l)
    assert len(L) == P and sum(L) == N - P + 1 and min(L) >= 1
    c = _per_subsystem_counts(L, n, l)
    ce = _per_subsystem_counts(o.partition_plan(N, P)[1], n, l)
    row = 7 * n ** 3 + 5 * n ** 2 * l          # one middle row's count
    assert max(c) - min(c) <= 2 * row           # balanced to within rounding of a row or two
    assert max(ce) - min(ce) > max(c) - min(c)  # better balanced than equal sizes
    # the enlargement of the first and last subsystems approaches 7/4 and 7/6 (Section 5.1)
    if l * 100 < n:
        mid = L[P // 2]
        assert abs(L[0] / mid - 7 / 4) < 0.15 and abs(L[-1] / mid - 7 / 6) < 0.15


def test_dm_with_equal_time_sizes_matches_dense():
    s = w.dominant_system(40, 3, 2, 31)
    L = o.partition_lengths_equal_time(40, 5, 3, 2)
    xd = o.dense_ge(o.dense_from_blocks(s.A, s.B, s.C), s.b.reshape(-1, 2)).reshape(40, 3, 2)
    assert o.rel_err(o.dm(s.A, s.B, s.C, s.b, 5, lengths=L), xd) < 1e-13
    ctr = o.OpCounter()
    o.dm(s.A, s.B, s.C, s.b, 5, lengths=L, ctr=ctr)
    assert ctr.total() == o.mo_dm_total(L, 3, 2)
