"""CPU oracle for the decomposition method (DM) for block-tridiagonal systems.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
CPU-baseline leg may import this module.  It shares no code with the CUDA path
and must never serve as a fallback for it.

Source: P. A. Belov, E. R. Nugumanov, S. L. Yakovlev, "Decomposition method for
block-tridiagonal matrix systems", arXiv:1505.06864.

Notation.  The paper writes the system as A_i X_{i-1} + C_i X_i + B_i X_{i+1}
= F_i with blocks n x n (Eq. 1).  Here, as in the rest of this library, the
diagonal block is B_i, the super-diagonal block C_i and the block size m:
    A_i X_{i-1} + B_i X_i + C_i X_{i+1} = F_i,   A_1 = C_N = 0.
Indices below are 0-based (row 0 .. N-1) while the paper counts from 1.

Everything is float64 and written for readability, not speed: one library
routine per block operation (``numpy.linalg.inv`` = LAPACK LU followed by a
solve against the identity, which is how the paper inverts blocks in
Section 4; ``@`` for block products).  A right-hand-side block that is
structurally zero is carried as ``None`` and no product is formed with it;
this is the sparse right-hand side rule the paper's operation counts rely on
(Section 4.1, Table 2), so an ``OpCounter`` attached to a run reproduces the
paper's multiplicative-operation counts exactly.

Functions and the passages they follow:
    partition_plan   Section 2 (choice of the M-1 separator block-rows)
    partition_lengths_equal_time   Section 5.1 (equal execution time, Table 2)
    ta_factor/ta_solve/thomas   Section 3 (Thomas algorithm, forward and backward sweeps)
    dm               Section 2, Eqs. (e220)-(endSolution); recursion on the
                     supplementary system as in Section 4.2.1; with J >= 2 every
                     subsystem solved by DM with J sub-subsystems (Section
                     4.2.2, ``_dm_groups``)
    dense_ge         textbook Gaussian elimination with partial pivoting on the
                     assembled dense matrix (independent check, tiny systems)
    residual, refine_truth   r = b - T x in float64 / extended precision
    mo_* and the optimum functions   Section 4 (Table 1, Table 2, Eq. DMtotal,
                     Eq. DMrec1, Eqs. DMrec121/DMrec1212/DMrec122) and
                     Section 5 (Eqs. SpeedupMP, MAXSpeedP, SpeedupMPNk,
                     SuppMatrM, SuppMatrPM, DMrec2-P3DMrec4)
Parity pins: every function above is pinned in tests/test_oracle_pins.py by
dense Gaussian elimination, manufactured solutions, an exactly known solution
(``refine_truth``), exact operation counts of instrumented runs (Table 1,
Table 2, Eqs. DMtotal, DMrec1, DMrec121/DMrec1212/DMrec122, DMrec3, DMrec4,
SpeedupMPNk, SpeedupMiPNk) and the paper's printed optimum values.  No
function here is "parity unpinned".
"""
from __future__ import annotations

import math
from contextlib import contextmanager

import numpy as np

__all__ = [
    "OpCounter", "partition_plan", "ta_factor", "ta_solve", "thomas", "dm",
    "dense_from_blocks", "dense_ge", "residual", "rel_err", "refine_truth",
]


# --------------------------------------------------------------------------
# Multiplicative-operation counter (Section 4 cost model)
# --------------------------------------------------------------------------
class OpCounter:
    """Counts multiplicative operations with the paper's cost model
    (Section 4): inverting an m x m block costs m^3, a product of an
    (a x b) block by a (b x c) block costs a*b*c; additions are free.
    Counts go to the bucket named by ``stage`` (nested stages join with '/')."""

    def __init__(self):
        self.buckets = {}
        self._stack = []

    @contextmanager
    def stage(self, name):
        self._stack.append(str(name))
        try:
            yield self
        finally:
            self._stack.pop()

    def _add(self, v):
        key = "/".join(self._stack)
        self.buckets[key] = self.buckets.get(key, 0) + int(v)

    def inv(self, X):
        self._add(X.shape[0] ** 3)

    def mul(self, X, Y):
        self._add(X.shape[0] * X.shape[1] * Y.shape[1])

    def total(self, stage=""):
        """Sum of the bucket ``stage`` and every bucket nested under it."""
        if not stage:
            return sum(self.buckets.values())
        return sum(v for k, v in self.buckets.items()
                   if k == stage or k.startswith(stage + "/"))


class _NoCount:
    def inv(self, X):
        pass

    def mul(self, X, Y):
        pass

    @contextmanager
    def stage(self, name):
        yield self


def _inv(X, ctr):
    ctr.inv(X)
    return np.linalg.inv(X)


def _mul(X, Y, ctr):
    """X @ Y, or None when either operand is structurally zero."""
    if X is None or Y is None:
        return None
    ctr.mul(X, Y)
    return X @ Y


def _sub(X, Y):
    """X - Y where None stands for a zero block."""
    if Y is None:
        return X
    if X is None:
        return -Y
    return X - Y


# --------------------------------------------------------------------------
# Partition plan (Section 2)
# --------------------------------------------------------------------------
def partition_plan(N: int, P: int):
    """Separator rows and subsystem ranges for P subsystems (the paper's M).

    The paper lets the M-1 separator block-rows be any rows from the second to
    the last-but-one.  Reading used here: equal subsystem sizes
    L_k = floor((N-P+1)/P), the remainder given one extra row each to the
    lowest-numbered subsystems, and separator k placed right after subsystem k.
    Requires every L_k >= 1, i.e. 1 <= P <= (N+1)/2.

    Returns (starts, lengths, seps): subsystem k owns rows
    starts[k] .. starts[k]+lengths[k]-1 and seps[k] (k < P-1) is the separator
    row between subsystems k and k+1.
    """
    if P < 1 or N < 1 or (P > 1 and 2 * P - 1 > N):
        raise ValueError(f"invalid partition: N={N}, P={P}")
    rows = N - (P - 1)
    base, extra = divmod(rows, P)
    starts, lengths, seps = [], [], []
    r = 0
    for k in range(P):
        L = base + (1 if k < extra else 0)
        starts.append(r)
        lengths.append(L)
        r += L
        if k < P - 1:
            seps.append(r)
            r += 1
    assert r == N
    return starts, lengths, seps


def partition_lengths_equal_time(N: int, P: int, n: int, l: int):
    """Subsystem sizes with equal operation counts (Section 5.1, second case):
    from Table 2, a middle subsystem of N_k rows costs N_k (7n^3 + 5n^2 l), the
    first (4N_1 - 1)(n^3 + n^2 l) and the last (6N_M - 3)n^3 + (4N_M - 1)n^2 l.
    Equating them gives N_1 = a1 N_k + b1 and N_M = a2 N_k + b2; the size
    constraint N_1 + N_M + (P - 2) N_k = N - P + 1 fixes N_k.  Rounding
    (reading): N_1 and N_M to the nearest integer (halves up), the middle
    subsystems share the remaining rows equally, remainder to the lowest ones;
    equal sizes when a subsystem would be left empty."""
    if P < 1 or (P > 1 and 2 * P - 1 > N):
        raise ValueError(f"invalid partition: N={N}, P={P}")
    if P == 1:
        return [N]
    rows = N - P + 1
    c = 7.0 * n ** 3 + 5.0 * n ** 2 * l
    a1, b1 = c / (4.0 * n ** 3 + 4.0 * n ** 2 * l), 0.25
    a2 = c / (6.0 * n ** 3 + 4.0 * n ** 2 * l)
    b2 = (3.0 * n ** 3 + n ** 2 * l) / (6.0 * n ** 3 + 4.0 * n ** 2 * l)
    nk = (rows - b1 - b2) / (a1 + a2 + P - 2)
    n1 = int(math.floor(a1 * nk + b1 + 0.5))
    nm = int(math.floor(a2 * nk + b2 + 0.5))
    mid = rows - n1 - nm
    if n1 < 1 or nm < 1 or (P > 2 and mid < P - 2) or (P == 2 and mid != 0):
        if P == 2 and n1 >= 1 and rows - n1 >= 1:
            return [n1, rows - n1]
        _, L, _ = partition_plan(N, P)
        return L
    if P == 2:
        return [n1, nm]
    base, extra = divmod(mid, P - 2)
    return [n1] + [base + (1 if k < extra else 0) for k in range(P - 2)] + [nm]


def plan_from_lengths(lengths):
    """(starts, lengths, seps) for subsystems of the given sizes, separator k
    right after subsystem k."""
    starts, seps, r = [], [], 0
    for k, L in enumerate(lengths):
        starts.append(r)
        r += L
        if k < len(lengths) - 1:
            seps.append(r)
            r += 1
    return starts, list(lengths), seps


# --------------------------------------------------------------------------
# Thomas algorithm (Section 3)
# --------------------------------------------------------------------------
def ta_factor(A, B, C, ctr=None):
    """Forward-stage blocks that do not depend on the right-hand side:
    G_1 = B_1^{-1}, G_i = (B_i - A_i Acal_{i-1})^{-1}, Acal_i = G_i C_i
    (i = 1..N-1).  A, B, C are sequences of N blocks (A[0], C[N-1] unused)."""
    ctr = ctr or _NoCount()
    N = len(B)
    G, Acal = [None] * N, [None] * N
    with ctr.stage("G"):
        G[0] = _inv(B[0], ctr)
    for i in range(N):
        if i > 0:
            with ctr.stage("G"):
                G[i] = _inv(B[i] - _mul(A[i], Acal[i - 1], ctr), ctr)
        if i < N - 1:
            with ctr.stage("Acal"):
                Acal[i] = _mul(G[i], C[i], ctr)
    return G, Acal


def ta_solve(G, Acal, A, F, ctr=None):
    """Right-hand-side stages of the Thomas algorithm for one supervector F
    (a sequence of N blocks, None = structurally zero block):
    forward  Bcal_1 = G_1 F_1,  Bcal_i = G_i (F_i - A_i Bcal_{i-1});
    backward X_N = Bcal_N,      X_i = Bcal_i - Acal_i X_{i+1}."""
    ctr = ctr or _NoCount()
    N = len(G)
    Bcal = [None] * N
    with ctr.stage("Bcal"):
        Bcal[0] = _mul(G[0], F[0], ctr)
        for i in range(1, N):
            Bcal[i] = _mul(G[i], _sub(F[i], _mul(A[i], Bcal[i - 1], ctr)), ctr)
    X = [None] * N
    with ctr.stage("X"):
        X[N - 1] = Bcal[N - 1]
        for i in range(N - 2, -1, -1):
            X[i] = _sub(Bcal[i], _mul(Acal[i], X[i + 1], ctr))
    return X


def thomas(A, B, C, F, ctr=None):
    """Solve the block-tridiagonal system by the Thomas algorithm (Section 3).
    A, B, C: [N, m, m]; F: [N, m, l].  Returns X: [N, m, l]."""
    G, Acal = ta_factor(list(A), list(B), list(C), ctr)
    X = ta_solve(G, Acal, list(A), list(F), ctr)
    return np.stack(X)


# --------------------------------------------------------------------------
# Decomposition method (Section 2)
# --------------------------------------------------------------------------
def supp_partitions(Ms: int, P: int, l: int, m: int):
    """Number of subsystems for DM applied to a supplementary system of Ms
    blocks that came from P subsystems (Eq. SuppMatrM, with its boundary case
    m = P/3 when P < 21), rounded and clamped so every sub-subsystem keeps at
    least one row.  Returns 1 when DM cannot be applied."""
    c = 5.0 + 2.0 / (1.0 + l / m)
    p2 = math.sqrt(P / 3.0 * c)
    if (P - p2) / p2 < 2.0:
        p2 = P / 3.0
    p2 = int(round(p2))
    p2 = min(p2, (Ms + 1) // 2)
    return max(p2, 1)


def _dm_groups(Ak, Bk, Ck, groups, J, ctr):
    """DM applied to one subsystem of Eq. (e231) (Section 4.2.2): the
    subsystem's block-tridiagonal matrix (Ak[0] and Ck[-1] unused) is split
    into J sub-subsystems by J-1 inner separator rows (placement as in
    partition_plan), each sub-subsystem is solved by the Thomas algorithm for
    every right-hand-side group and for its own two spikes, the inner
    supplementary system (J-1 blocks, Eq. e2311) is assembled and solved by
    the Thomas algorithm, and Eq. (endSolution) gives every group's solution.

    ``groups`` is a list of right-hand-side groups, each a list of one block
    per row (None = structurally zero block) or None for an absent group;
    the result has the same structure.  Operation counts go to the stages
    "sub/<i>" (sub-subsystem i: its Thomas solves, its products with the
    inner separators' blocks, its rows of Eq. endSolution) and "supp" (the
    inner supplementary system), the split the paper's Eqs. (DMrec121),
    (DMrec1212), (DMrec122) use."""
    L = len(Bk)
    starts, lens, seps = partition_plan(L, J)
    ng = len(groups)
    Y = [[None] * J for _ in range(ng)]       # Y[g][i]: group g on sub-subsystem i
    SL, SR = [None] * J, [None] * J            # inner spikes of sub-subsystem i
    for i in range(J):
        s, Li = starts[i], lens[i]
        Ai = [None] + [Ak[s + t] for t in range(1, Li)]
        Bi = [Bk[s + t] for t in range(Li)]
        Ci = [Ck[s + t] for t in range(Li - 1)] + [None]
        with ctr.stage(f"sub/{i}"):
            G, Acal = ta_factor(Ai, Bi, Ci, ctr)
            for g, grp in enumerate(groups):
                if grp is not None:
                    Y[g][i] = ta_solve(G, Acal, Ai, [grp[s + t] for t in range(Li)], ctr)
            if i > 0:
                SL[i] = ta_solve(G, Acal, Ai, [Ak[s]] + [None] * (Li - 1), ctr)
            if i < J - 1:
                SR[i] = ta_solve(G, Acal, Ai, [None] * (Li - 1) + [Ck[s + Li - 1]], ctr)
    # inner supplementary system on the separators q_0..q_{J-2}
    Ms = J - 1
    HA, HB, HC = [None] * Ms, [Bk[q] for q in seps], [None] * Ms
    fh = [None if grp is None else [grp[q] for q in seps] for grp in groups]
    for i in range(J):
        with ctr.stage(f"sub/{i}"):
            if i > 0:            # separator i-1 above: its C meets row 0 of sub-subsystem i
                j = i - 1
                Cq = Ck[seps[j]]
                HB[j] = _sub(HB[j], _mul(Cq, SL[i][0], ctr))
                if i < J - 1:
                    HC[j] = _sub(None, _mul(Cq, SR[i][0], ctr))
                for g in range(ng):
                    if fh[g] is not None:
                        fh[g][j] = _sub(fh[g][j], _mul(Cq, Y[g][i][0], ctr))
            if i < J - 1:        # separator i below: its A meets the last row of sub-subsystem i
                j = i
                Aq = Ak[seps[j]]
                if i > 0:
                    HA[j] = _sub(None, _mul(Aq, SL[i][-1], ctr))
                HB[j] = _sub(HB[j], _mul(Aq, SR[i][-1], ctr))
                for g in range(ng):
                    if fh[g] is not None:
                        fh[g][j] = _sub(fh[g][j], _mul(Aq, Y[g][i][-1], ctr))
    with ctr.stage("supp"):
        G, Acal = ta_factor(HA, HB, HC, ctr)
        h = [None if f is None else ta_solve(G, Acal, HA, f, ctr) for f in fh]
    # Eq. (endSolution) inside the subsystem, for every group
    out = []
    for g in range(ng):
        if groups[g] is None:
            out.append(None)
            continue
        x = [None] * L
        for i in range(J):
            s, Li = starts[i], lens[i]
            with ctr.stage(f"sub/{i}"):
                for t in range(Li):
                    v = Y[g][i][t]
                    if i > 0:
                        v = _sub(v, _mul(SL[i][t], h[g][i - 1], ctr))
                    if i < J - 1:
                        v = _sub(v, _mul(SR[i][t], h[g][i], ctr))
                    x[s + t] = v
        for j, q in enumerate(seps):
            x[q] = h[g][j]
        out.append(x)
    return out


def dm(A, B, C, F, P, levels=1, P2=None, ctr=None, return_parts=False, lengths=None, J=None):
    """Solve A_i X_{i-1} + B_i X_i + C_i X_{i+1} = F_i by the decomposition
    method with P subsystems (Section 2).

    levels = 1 solves the supplementary system (Eq. e232) by the Thomas
    algorithm; levels = L > 1 solves it by DM with P2 subsystems and
    levels = L - 1 (Section 4.2.1).  P = 1 is the Thomas algorithm itself.
    J >= 2 solves every subsystem's Eq. (e231) by DM with J sub-subsystems
    (Section 4.2.2): the right-hand sides F^k and the two columns of W_R^k
    are carried as separate groups, so the structurally zero blocks of W_R^k
    cost nothing.
    """
    ctr = ctr or _NoCount()
    A, B, C, F = np.asarray(A), np.asarray(B), np.asarray(C), np.asarray(F)
    N, m, l = B.shape[0], B.shape[1], F.shape[2]
    dt = np.result_type(A, B, C, F, np.float64)   # float64, or complex128 for complex systems
    if P == 1 and J is not None and J >= 2:
        # the whole system is the one subsystem: Eq. (e231) without spikes, by DM
        with ctr.stage("solve/0"):
            x = _dm_groups([None] + list(A[1:]), list(B), list(C[:-1]) + [None], [list(F)], J, ctr)[0]
        return np.stack(x)
    if P == 1:
        with ctr.stage("ta"):
            return thomas(A, B, C, F, ctr)
    if lengths is None:
        starts, lengths, seps = partition_plan(N, P)
    else:
        assert len(lengths) == P and sum(lengths) == N - P + 1 and min(lengths) >= 1
        starts, lengths, seps = plan_from_lengths(lengths)

    # Eq. (e231): S^k Z^k = W_R^k and S^k z^k = F_s^k for every subsystem.
    # S^k is the block-tridiagonal matrix of subsystem k's rows with the
    # couplings to the separators removed.  W_R^k has two non-zero blocks:
    # column h^{k-1} holds A of the subsystem's first row (top block only),
    # column h^k holds C of its last row (bottom block only).
    z, ZL, ZR = [], [], []
    for k in range(P):
        s, L = starts[k], lengths[k]
        Ak = [None] + [A[s + t] for t in range(1, L)]
        Bk = [B[s + t] for t in range(L)]
        Ck = [C[s + t] for t in range(L - 1)] + [None]
        with ctr.stage(f"solve/{k}"):
            if J is not None and J >= 2:
                grp = [[F[s + t] for t in range(L)],
                       [A[s]] + [None] * (L - 1) if k > 0 else None,
                       [None] * (L - 1) + [C[s + L - 1]] if k < P - 1 else None]
                zk, zl, zr = _dm_groups(Ak, Bk, Ck, grp, J, ctr)
                z.append(zk)
                ZL.append(zl)
                ZR.append(zr)
                continue
            G, Acal = ta_factor(Ak, Bk, Ck, ctr)
            z.append(ta_solve(G, Acal, Ak, [F[s + t] for t in range(L)], ctr))
            ZL.append(ta_solve(G, Acal, Ak, [A[s]] + [None] * (L - 1), ctr) if k > 0 else None)
            ZR.append(ta_solve(G, Acal, Ak, [None] * (L - 1) + [C[s + L - 1]], ctr)
                      if k < P - 1 else None)

    # Eq. (e2311): H - sum_k W_L^k Z^k and F_h - sum_k W_L^k z^k.  W_L^k has
    # two non-zero blocks: separator k-1's C (against subsystem k's first row)
    # and separator k's A (against its last row).  The result is the
    # block-tridiagonal supplementary system of Eq. (e232) on h_0..h_{P-2}.
    Ms = P - 1
    HA = np.zeros((Ms, m, m), dtype=dt)
    HB = np.zeros((Ms, m, m), dtype=dt)
    HC = np.zeros((Ms, m, m), dtype=dt)
    fh = np.zeros((Ms, m, l), dtype=dt)
    for j in range(Ms):
        q = seps[j]
        HB[j] = B[q]
        fh[j] = F[q]
    for k in range(P):
        with ctr.stage(f"wing/{k}"):
            if k > 0:   # separator k-1 sits above subsystem k: its C meets row first
                j = k - 1
                q = seps[j]
                HB[j] -= _mul(C[q], ZL[k][0], ctr)
                if k < P - 1:
                    HC[j] -= _mul(C[q], ZR[k][0], ctr)
                fh[j] -= _mul(C[q], z[k][0], ctr)
            if k < P - 1:   # separator k sits below subsystem k: its A meets row last
                j = k
                q = seps[j]
                if k > 0:
                    HA[j] -= _mul(A[q], ZL[k][-1], ctr)
                HB[j] -= _mul(A[q], ZR[k][-1], ctr)
                fh[j] -= _mul(A[q], z[k][-1], ctr)

    # Eq. (e232): the supplementary system, by TA or recursively by DM.
    with ctr.stage("supp"):
        if levels > 1:
            p2 = P2 if P2 is not None else supp_partitions(Ms, P, l, m)
            h = dm(HA, HB, HC, fh, max(1, min(p2, (Ms + 1) // 2)), levels - 1, None, ctr)
        else:
            h = thomas(HA, HB, HC, fh, ctr)

    # Eq. (endSolution): s^k = z^k - Z^k_(left) h^{k-1} - Z^k_(right) h^k,
    # with h^0 = h^M = 0 (here: no left term for k = 0, no right term for k = P-1).
    X = np.zeros((N, m, l), dtype=dt)
    for k in range(P):
        s, L = starts[k], lengths[k]
        with ctr.stage(f"back/{k}"):
            for t in range(L):
                v = z[k][t]
                if k > 0:
                    v = v - _mul(ZL[k][t], h[k - 1], ctr)
                if k < P - 1:
                    v = v - _mul(ZR[k][t], h[k], ctr)
                X[s + t] = v
    for j in range(Ms):
        X[seps[j]] = h[j]
    if return_parts:
        return X, dict(z=z, ZL=ZL, ZR=ZR, HA=HA, HB=HB, HC=HC, fh=fh, h=h,
                       starts=starts, lengths=lengths, seps=seps)
    return X


# --------------------------------------------------------------------------
# Independent checks
# --------------------------------------------------------------------------
def dense_from_blocks(A, B, C):
    """The (Nm) x (Nm) matrix T of Eq. (1)."""
    N, m = B.shape[0], B.shape[1]
    T = np.zeros((N * m, N * m), dtype=np.result_type(A, B, C, np.float64))
    for i in range(N):
        T[i * m:(i + 1) * m, i * m:(i + 1) * m] = B[i]
        if i > 0:
            T[i * m:(i + 1) * m, (i - 1) * m:i * m] = A[i]
        if i < N - 1:
            T[i * m:(i + 1) * m, (i + 1) * m:(i + 2) * m] = C[i]
    return T


def dense_ge(T, b):
    """Textbook Gaussian elimination with partial pivoting and back
    substitution on a dense n x n matrix (n small); b is n x l.  Real or
    complex (pivot by largest modulus)."""
    dt = np.result_type(T, b, np.float64)
    T = np.array(T, dtype=dt)
    b = np.array(b, dtype=dt)
    n = T.shape[0]
    for k in range(n):
        p = k + int(np.argmax(np.abs(T[k:, k])))
        if T[p, k] == 0.0:
            raise ZeroDivisionError("singular matrix")
        if p != k:
            T[[k, p]] = T[[p, k]]
            b[[k, p]] = b[[p, k]]
        for i in range(k + 1, n):
            f = T[i, k] / T[k, k]
            T[i, k:] -= f * T[k, k:]
            b[i] -= f * b[k]
    x = np.zeros_like(b)
    for i in range(n - 1, -1, -1):
        x[i] = (b[i] - T[i, i + 1:] @ x[i + 1:]) / T[i, i]
    return x


def residual(A, B, C, x, b, dtype=np.float64):
    """r = b - T x evaluated in ``dtype`` (float64 or np.longdouble; for
    complex systems the complex type of that precision)."""
    if any(np.iscomplexobj(v) for v in (A, B, C, x, b)):
        dtype = np.clongdouble if dtype == np.longdouble else np.complex128
    A, B, C, x, b = (np.asarray(v, dtype=dtype) for v in (A, B, C, x, b))
    r = b - np.matmul(B, x)
    r[1:] -= np.matmul(A[1:], x[:-1])
    r[:-1] -= np.matmul(C[:-1], x[1:])
    return r


def rel_err(x, xref):
    """max over right-hand-side columns of ||x - xref||_2 / ||xref||_2."""
    dt = np.result_type(x, xref, np.float64)
    x = np.asarray(x, dtype=dt).reshape(-1, x.shape[-1])
    xref = np.asarray(xref, dtype=dt).reshape(-1, xref.shape[-1])
    num = np.linalg.norm(x - xref, axis=0)
    den = np.linalg.norm(xref, axis=0)
    den[den == 0] = 1.0
    return float(np.max(num / den))


def refine_truth(A, B, C, b, x0=None, iters=6):
    """Near-exact solution of T x = b: float64 Thomas solves corrected with
    residuals evaluated in extended precision (np.longdouble)."""
    cplx = any(np.iscomplexobj(v) for v in (A, B, C, b))
    lo, hi = (np.complex128, np.clongdouble) if cplx else (np.float64, np.longdouble)
    x = thomas(A, B, C, b) if x0 is None else np.array(x0, dtype=lo)
    xl = x.astype(hi)
    for _ in range(iters):
        r = residual(A, B, C, xl, b, dtype=np.longdouble)
        d = thomas(A, B, C, r.astype(lo))
        xl = xl + d.astype(hi)
        if np.max(np.abs(d)) <= 1e-18 * max(1.0, float(np.max(np.abs(xl)))):
            break
    return xl.astype(lo)


# --------------------------------------------------------------------------
# Section 4: multiplicative-operation counts (paper letters n = m, l = nrhs)
# --------------------------------------------------------------------------
def mo_ta(N, n, l):
    """Table 1 total: (3N - 2)(n^3 + n^2 l)."""
    return (3 * N - 2) * (n ** 3 + n ** 2 * l)


def mo_ta_parts(N, n, l):
    """Table 1 rows: G, Acal, Bcal, X."""
    return {"G": (2 * N - 1) * n ** 3, "Acal": (N - 1) * n ** 3,
            "Bcal": (2 * N - 1) * n ** 2 * l, "X": (N - 1) * n ** 2 * l}


def mo_dm_solve(k, M, Nk, n, l):
    """Table 2, solution of Eq. (e231) for subsystem k (1-based)."""
    if k == 1:
        return (4 * Nk - 2) * n ** 3 + (3 * Nk - 2) * n ** 2 * l
    if k == M:
        return (6 * Nk - 4) * n ** 3 + (3 * Nk - 2) * n ** 2 * l
    return (7 * Nk - 4) * n ** 3 + (3 * Nk - 2) * n ** 2 * l


def mo_dm_wing(k, M, n, l):
    """Table 2, products W_L^k Z^k and W_L^k z^k."""
    if k in (1, M):
        return n ** 3 + n ** 2 * l
    return 4 * n ** 3 + 2 * n ** 2 * l


def mo_dm_supp(M, n, l):
    """Table 2, supplementary system (Eq. e232) by the Thomas algorithm."""
    return (3 * M - 5) * (n ** 3 + n ** 2 * l)


def mo_dm_back(k, M, Nk, n, l):
    """Table 2, products of Eq. (endSolution)."""
    return (Nk if k in (1, M) else 2 * Nk) * n ** 2 * l


def mo_dm_total(Ns, n, l):
    """Eq. (DMtotal) for subsystem sizes Ns = [N_1, ..., N_M], M >= 2."""
    M = len(Ns)
    t = ((4 * Ns[0] - 1) * n ** 3 + (4 * Ns[0] - 1) * n ** 2 * l)
    t += ((6 * Ns[-1] - 3) * n ** 3 + (4 * Ns[-1] - 1) * n ** 2 * l)
    t += sum(7 * Nk * n ** 3 + 5 * Nk * n ** 2 * l for Nk in Ns[1:-1])
    return t + (3 * M - 5) * (n ** 3 + n ** 2 * l)


def mo_dm_rec1(Ns, Ms, n, l):
    """Eq. (DMtotal) with its last term replaced by Eq. (DMrec1): DM with
    len(Ms) subsystems of sizes Ms applied to the supplementary system."""
    M = len(Ns)
    return mo_dm_total(Ns, n, l) - (3 * M - 5) * (n ** 3 + n ** 2 * l) + mo_dm_total(Ms, n, l)


def mo_dm_sub_first(L, n, l):
    """Eq. (DMrec121): subsystem k = 1 solved by DM with sub-subsystems L."""
    J = len(L)
    return ((5 * L[0] - 1) * n ** 3 + (4 * L[0] - 1) * n ** 2 * l
            + (8 * L[-1] - 2) * n ** 3 + (4 * L[-1] - 1) * n ** 2 * l
            + sum(Li * (9 * n ** 3 + 5 * n ** 2 * l) for Li in L[1:-1])
            + (4 * J - 6) * n ** 3 + (3 * J - 5) * n ** 2 * l)


def mo_dm_sub_last(L, n, l):
    """Eq. (DMrec1212): subsystem k = M solved by DM with sub-subsystems L."""
    J = len(L)
    return ((8 * L[0] - 2) * n ** 3 + (4 * L[0] - 1) * n ** 2 * l
            + (7 * L[-1] - 3) * n ** 3 + (4 * L[-1] - 1) * n ** 2 * l
            + sum(Li * (9 * n ** 3 + 5 * n ** 2 * l) for Li in L[1:-1])
            + (6 * J - 10) * n ** 3 + (3 * J - 5) * n ** 2 * l)


def mo_dm_sub_mid(L, n, l):
    """Eq. (DMrec122): subsystem 1 < k < M solved by DM with sub-subsystems L."""
    J = len(L)
    return ((9 * L[0] - 2) * n ** 3 + (4 * L[0] - 1) * n ** 2 * l
            + (9 * L[-1] - 2) * n ** 3 + (4 * L[-1] - 1) * n ** 2 * l
            + sum(Li * (11 * n ** 3 + 5 * n ** 2 * l) for Li in L[1:-1])
            + (7 * J - 11) * n ** 3 + (3 * J - 5) * n ** 2 * l)


# --------------------------------------------------------------------------
# Section 5: speedup model and optimum parameters
# --------------------------------------------------------------------------
def _c(n, l):
    return 5.0 + 2.0 / (1.0 + l / n)


def speedup_mp(N, P, n, l):
    """Eq. (SpeedupMP): equal subsystems, M = P."""
    return (3 * N - 2) / (3 * P - 5 + _c(n, l) * (N - P + 1) / P)


def speedup_mp_bound(N, P):
    """Lower bound printed with Eq. (SpeedupMP): 1 / (7/(3P) + P/N)."""
    return 1.0 / (7.0 / (3.0 * P) + P / N)


def p_opt_mp(N, n, l):
    """Eq. (MAXSpeedP): P maximising Eq. (SpeedupMP)."""
    return math.sqrt((N + 1) / 3.0 * _c(n, l))


def speedup_mp_unequal(N, P, n, l, alpha, beta):
    """Eq. (SpeedupMPNk): first/last subsystems alpha, beta times larger."""
    return (3 * N - 2) / (3 * P - 5 + _c(n, l) * (N - P + 1) / (P - 2 + alpha + beta))


def speedup_queue(N, P, i, n, l, alpha, beta):
    """Eq. (SpeedupMiPNk): M = iP subsystems, a queue of i per processor."""
    return (3 * N - 2) / (3 * i * P - 5 + i * _c(n, l) * (N - i * P + 1) / (i * P - 2 + alpha + beta))


def mo_dm_rec2(N1, M1, m_sub, n, l):
    """Eq. (DMrec2): serial count with DM on the supplementary system."""
    return ((7 * N1 * n ** 3 + 5 * N1 * n ** 2 * l) + (7 * M1 * n ** 3 + 5 * M1 * n ** 2 * l)
            + (3 * m_sub - 5) * (n ** 3 + n ** 2 * l))


def m_opt_supp(P, n, l):
    """Eq. (SuppMatrM): subsystems of the supplementary system for fixed P;
    the boundary value P/3 when (P - m)/m >= 2 fails."""
    msub = math.sqrt(P / 3.0 * _c(n, l))
    return msub if (P - msub) / msub >= 2.0 else P / 3.0


def speedup_rec_supp_small_l(N, P):
    """Eq. (Speedup521): S for l << n with m = sqrt(7P/3)."""
    return (3 * N - 2) / (7 * (N + 1) / P + 2 * math.sqrt(21 * P) - 19)


def p_m_opt_supp_free(N, n, l):
    """Eq. (SuppMatrPM): optimum (P, m) when P is free."""
    P = ((N + 1) ** 2 / 3.0 * _c(n, l)) ** (1.0 / 3.0)
    return P, P ** 2 / (N + 1)


def mo_dm_rec3(N, M, J, n, l):
    """Eq. (DMrec3): serial count with DM inside each subsystem (P = MJ)."""
    N1 = (N - M + 1) / M
    N2 = (N1 - J + 1) / J
    return ((11 * n ** 3 + 5 * n ** 2 * l) * N2 + (n ** 3 * (7 * J - 11) + n ** 2 * l * (3 * J - 5))
            + 4 * n ** 3 + 2 * n ** 2 * l + (n ** 3 + n ** 2 * l) * (3 * M - 5) + 2 * n ** 2 * l * N1)


def mj_opt_rec3_fixed_p(N, P, n, l):
    """Eq. (ParamDMrec3): M and J = P/M for fixed P."""
    M = math.sqrt(((7 * n ** 3 + 3 * n ** 2 * l) * P + 2 * n ** 2 * l * (N + 1))
                  / (3 * (n ** 3 + n ** 2 * l)))
    return M, P / M


def _positive_root(coeffs):
    r = np.roots(coeffs)
    r = [float(v.real) for v in r if abs(v.imag) < 1e-9 * max(1.0, abs(v)) and v.real > 0]
    assert len(r) == 1, r
    return r[0]


def mj_opt_rec3_free(N, n, l):
    """Eqs. (P2DMrec3), (P3DMrec3): free P; J from the quartic, then M."""
    a = (11 * n ** 3 + 5 * n ** 2 * l) / (2 * n ** 2 * l)
    c0 = (N + 1) * 3 * (n ** 3 + n ** 2 * l) * (11 * n ** 3 + 5 * n ** 2 * l) ** 2 / (
        (7 * n ** 3 + 3 * n ** 2 * l) ** 2 * 2 * n ** 2 * l)
    J = _positive_root([1.0, a, 0.0, 0.0, -c0])
    M = (N + 1) / J ** 2 * (11 * n ** 3 + 5 * n ** 2 * l) / (7 * n ** 3 + 3 * n ** 2 * l)
    return M, J


def mo_dm_rec4(N, M, J, m_sub, n, l):
    """Eq. (DMrec4): DM inside subsystems and on the supplementary system."""
    N1 = (N - M + 1) / M
    N2 = (N1 - J + 1) / J
    return ((11 * n ** 3 + 5 * n ** 2 * l) * N2 + (n ** 3 * (7 * J - 11) + n ** 2 * l * (3 * J - 5))
            + 4 * n ** 3 + 2 * n ** 2 * l + (7 * n ** 3 + 5 * n ** 2 * l) * ((M - m_sub) / m_sub)
            + (n ** 3 + n ** 2 * l) * (3 * m_sub - 5) + 2 * n ** 2 * l * N1)


def mmj_opt_rec4_fixed_p(N, P, n, l):
    """Eq. (P1DMrec4): M, m and J = P/M for fixed P."""
    q = 3 * P + 4 * P / (1 + l / n) + 2 * l * (N + 1) / (n + l)
    M = q ** (2.0 / 3.0) / (3 * _c(n, l)) ** (1.0 / 3.0)
    msub = math.sqrt(M * (7 * n ** 3 + 5 * n ** 2 * l) / (3 * (n ** 3 + n ** 2 * l)))
    return M, msub, P / M


def mmj_opt_rec4_free(N, n, l):
    """Eqs. (P2DMrec4), (P3DMrec4): free P; J from the cubic, then M and m."""
    a = (11 * n ** 3 + 5 * n ** 2 * l) / (2 * n ** 2 * l)
    r = (11 * n ** 3 + 5 * n ** 2 * l) / (7 * n ** 3 + 3 * n ** 2 * l)
    c0 = math.sqrt(N + 1) / (2 * n ** 2 * l) * r ** 1.5 * math.sqrt(
        3 * (7 * n ** 3 + 5 * n ** 2 * l) * (n ** 3 + n ** 2 * l))
    J = _positive_root([1.0, a, 0.0, -c0])
    M = (N + 1) / J ** 2 * r
    msub = math.sqrt(M * (7 * n ** 3 + 5 * n ** 2 * l) / (3 * (n ** 3 + n ** 2 * l)))
    return M, msub, J


def first_last_sizes(Nk, n, l):
    """Equal-time sizes of the first and last subsystems from Table 2: the
    first subsystem's count (4N_1-1)n^3 + (4N_1-1)n^2 l and the last one's
    (6N_M-3)n^3 + (4N_M-1)n^2 l set equal to a middle one's 7N_k n^3 + 5N_k n^2 l."""
    mid = 7 * Nk * n ** 3 + 5 * Nk * n ** 2 * l
    N1 = (mid + n ** 3 + n ** 2 * l) / (4 * n ** 3 + 4 * n ** 2 * l)
    NM = (mid + 3 * n ** 3 + n ** 2 * l) / (6 * n ** 3 + 4 * n ** 2 * l)
    return N1, NM
