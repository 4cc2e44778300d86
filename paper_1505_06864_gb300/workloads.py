"""Seeded synthetic block-tridiagonal systems.

This module only draws random numbers and shapes them into the blocks of
``A_i X_{i-1} + B_i X_i + C_i X_{i+1} = b_i`` (blocks m x m, right-hand sides
m x nrhs, A_1 = C_N = 0).  It holds none of the decomposition method's
arithmetic and is the one module that both the CPU oracle and the CUDA path's
tests and benchmark use, so that both sides see identical inputs.

Letters: the paper (arXiv:1505.06864, Eq. 1) writes the diagonal block as C and
the super-diagonal block as B; this library writes the diagonal block as B and
the super-diagonal block as C, and the block size as m (the paper's n).

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based
generator: draw k of stream s under seed S is ``mix64(key(S, s) + (k + 1) * G)``
with G = 0x9E3779B97F4A7C15 and mix64 the SplitMix64 output function.  Uniform
doubles take the top 53 bits; normals use the Box-Muller transform.  Every
quantity (A, B, C, x, ...) has its own stream, so the draws for one quantity
never depend on the sizes of another.

Workload recipes (one function each):

* ``dominant_system`` -- entries of A_i, B_i, C_i uniform in [-1, 1]; A_1 and
  C_N zeroed; then B_i[r, r] += sum_j(|A_i[r, j]| + |B_i[r, j]| + |C_i[r, j]|) + 1,
  so every point row of T is strictly diagonally dominant with margin >= 1.
  x_true ~ N(0, 1) and b = T x_true.
* ``pde_banded_system`` -- second-order finite differences in one coordinate
  times cubic-spline collocation in the other: every block is banded with
  half-bandwidth 3 (stored dense), band entries uniform in [0.5, 2];
  A_i = -band, C_i = -band, B_i = band plus the same per-row dominance shift.
* ``conditioned_system`` -- dense nonsymmetric diagonal blocks
  B_i = U_i diag(sigma) V_i^T with U_i, V_i orthogonal (QR of Gaussian
  matrices) and sigma log-spaced in [1, cond]; A_i, C_i uniform in [-1, 1],
  each scaled to Frobenius norm 0.25 so ||A_i||_2 + ||C_i||_2 <= 0.5 sigma_min.
* ``laplace_fill_system`` -- the 5-point 2-D Laplace operator (blocks
  tridiag(-1, 4, -1) and -I) with its zero entries filled by small uniform
  values, the shape of the paper's validation matrices.
* ``batch_shapes`` -- shapes of a batch of independent systems: N uniform in
  [n_lo, n_hi], m drawn from a set, nrhs uniform in [r_lo, r_hi].
* ``dominant_system_complex`` -- the dominant recipe with complex entries:
  real and imaginary parts uniform in [-1, 1] from separate streams, the
  diagonal shift summing complex moduli; x_true with N(0, 1) real and
  imaginary parts.
* ``pde_banded_system_complex`` -- the PDE-shaped recipe whose last block row
  (A_N, B_N) is complex, as where the paper's application imposes its
  asymptotic boundary condition with complex (Hankel-function) coefficients
  (Section 7): the band entries of that row get imaginary parts uniform in
  [0.5, 2]; the dominance shift uses complex moduli.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "uniform", "normal", "dominant_system", "pde_banded_system",
    "conditioned_system", "batch_shapes", "manufacture_rhs", "System",
    "dominant_system_complex", "pde_banded_system_complex",
]

_G = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# One stream id per drawn quantity.
STREAM_A, STREAM_B, STREAM_C, STREAM_X = 1, 2, 3, 4
STREAM_X2, STREAM_U, STREAM_V, STREAM_SHAPE = 5, 6, 7, 8
STREAM_RHS, STREAM_RHS2 = 9, 10
STREAM_IM = 100  # added to a quantity's stream for its imaginary part


def _mix64(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _key(seed: int, stream: int) -> np.uint64:
    s = np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
    t = np.array([stream & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix64(s ^ (t * _M2 + _G))[0]


def _u64(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    k = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix64(_key(seed, stream) + k * _G)


def uniform(seed: int, stream: int, count: int, lo: float = 0.0, hi: float = 1.0,
            offset: int = 0) -> np.ndarray:
    """``count`` doubles uniform in [lo, hi) from draws offset.. of (seed, stream)."""
    u = (_u64(seed, stream, count, offset) >> np.uint64(11)).astype(np.float64)
    u *= 2.0 ** -53
    return lo + (hi - lo) * u


def normal(seed: int, stream: int, count: int) -> np.ndarray:
    """``count`` standard normals by Box-Muller from two uniform draws per value."""
    u1 = uniform(seed, stream, count)
    u2 = uniform(seed, stream + 1000, count)
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)


class System:
    """One block-tridiagonal system: A, B, C of shape [N, m, m], b and x_true of
    shape [N, m, nrhs], all float64 and C-contiguous (row-major blocks)."""

    def __init__(self, A, B, C, b, x_true, name=""):
        self.A, self.B, self.C, self.b, self.x_true = A, B, C, b, x_true
        self.name = name

    @property
    def N(self):
        return self.B.shape[0]

    @property
    def m(self):
        return self.B.shape[1]

    @property
    def nrhs(self):
        return self.b.shape[2]


def manufacture_rhs(A, B, C, x):
    """b = T x for the manufactured solution x (input preparation only)."""
    b = np.matmul(B, x)
    b[1:] += np.matmul(A[1:], x[:-1])
    b[:-1] += np.matmul(C[:-1], x[1:])
    return b


def _dominance_shift(A, B, C):
    """B[i, r, r] += sum_j |A[i,r,j]| + |B[i,r,j]| + |C[i,r,j]| + 1, summed in a
    fixed order (all of A's row, then B's, then C's, left to right)."""
    N, m, _ = B.shape
    s = np.zeros((N, m))
    for M in (A, B, C):
        for j in range(m):
            s += np.abs(M[:, :, j])
    idx = np.arange(m)
    B[:, idx, idx] += s + 1.0


def dominant_system(N: int, m: int, nrhs: int, seed: int) -> System:
    """Diagonally dominant random system (uniform [-1, 1] blocks plus a per-row
    diagonal shift); x_true ~ N(0, 1), b = T x_true."""
    A = uniform(seed, STREAM_A, N * m * m, -1.0, 1.0).reshape(N, m, m)
    B = uniform(seed, STREAM_B, N * m * m, -1.0, 1.0).reshape(N, m, m)
    C = uniform(seed, STREAM_C, N * m * m, -1.0, 1.0).reshape(N, m, m)
    A[0] = 0.0
    C[N - 1] = 0.0
    _dominance_shift(A, B, C)
    x = normal(seed, STREAM_X, N * m * nrhs).reshape(N, m, nrhs)
    return System(A, B, C, manufacture_rhs(A, B, C, x), x,
                  f"dominant N={N} m={m} nrhs={nrhs} seed={seed}")


def dominant_system_complex(N: int, m: int, nrhs: int, seed: int) -> System:
    """Complex diagonally dominant system (real and imaginary parts uniform in
    [-1, 1], per-row shift by the sum of complex moduli plus one); x_true with
    N(0, 1) real and imaginary parts, b = T x_true (complex128 arrays)."""
    draw = lambda st: (uniform(seed, st, N * m * m, -1.0, 1.0)
                       + 1j * uniform(seed, st + STREAM_IM, N * m * m, -1.0, 1.0)).reshape(N, m, m)
    A, B, C = draw(STREAM_A), draw(STREAM_B), draw(STREAM_C)
    A[0] = 0.0
    C[N - 1] = 0.0
    _dominance_shift(A, B, C)
    x = (normal(seed, STREAM_X, N * m * nrhs) + 1j * normal(seed, STREAM_X + STREAM_IM, N * m * nrhs)).reshape(N, m, nrhs)
    return System(A, B, C, manufacture_rhs(A, B, C, x), x,
                  f"dominant-complex N={N} m={m} nrhs={nrhs} seed={seed}")


def _band(seed: int, stream: int, N: int, m: int, hb: int, lo: float, hi: float):
    """Dense [N, m, m] blocks whose entries with |r - c| <= hb are uniform in
    [lo, hi) (draw (i, r, d) fills column r + d - hb) and zero elsewhere."""
    w = 2 * hb + 1
    v = uniform(seed, stream, N * m * w, lo, hi).reshape(N, m, w)
    M = np.zeros((N, m, m))
    for d in range(w):
        off = d - hb
        r0, r1 = max(0, -off), min(m, m - off)
        if r1 <= r0:
            continue
        r = np.arange(r0, r1)
        M[:, r, r + off] = v[:, r0:r1, d]
    return M


def pde_banded_system(N: int, m: int, nrhs: int, seed: int, hb: int = 3) -> System:
    """Finite differences (first coordinate) x cubic-spline collocation (second
    coordinate): banded blocks (half-bandwidth ``hb``) stored dense, band
    entries uniform in [0.5, 2], A_i = -band, C_i = -band, B_i = band + shift."""
    A = -_band(seed, STREAM_A, N, m, hb, 0.5, 2.0)
    B = _band(seed, STREAM_B, N, m, hb, 0.5, 2.0)
    C = -_band(seed, STREAM_C, N, m, hb, 0.5, 2.0)
    A[0] = 0.0
    C[N - 1] = 0.0
    _dominance_shift(A, B, C)
    x = normal(seed, STREAM_X, N * m * nrhs).reshape(N, m, nrhs)
    return System(A, B, C, manufacture_rhs(A, B, C, x), x,
                  f"pde-banded N={N} m={m} nrhs={nrhs} hb={hb} seed={seed}")


def pde_banded_system_complex(N: int, m: int, nrhs: int, seed: int, hb: int = 3) -> System:
    """pde_banded_system with a complex last block row: the band entries of
    A_N and B_N get imaginary parts uniform in [0.5, 2] (drawn from their own
    streams), then the dominance shift with complex moduli; x_true with N(0, 1)
    real and imaginary parts, b = T x_true (complex128 arrays)."""
    A = -_band(seed, STREAM_A, N, m, hb, 0.5, 2.0).astype(np.complex128)
    B = _band(seed, STREAM_B, N, m, hb, 0.5, 2.0).astype(np.complex128)
    C = -_band(seed, STREAM_C, N, m, hb, 0.5, 2.0)
    C = C.astype(np.complex128)
    A[-1] -= 1j * _band(seed, STREAM_A + STREAM_IM, 1, m, hb, 0.5, 2.0)[0]
    B[-1] += 1j * _band(seed, STREAM_B + STREAM_IM, 1, m, hb, 0.5, 2.0)[0]
    A[0] = 0.0
    C[N - 1] = 0.0
    _dominance_shift(A, B, C)
    x = (normal(seed, STREAM_X, N * m * nrhs) + 1j * normal(seed, STREAM_X + STREAM_IM, N * m * nrhs)).reshape(N, m, nrhs)
    return System(A, B, C, manufacture_rhs(A, B, C, x), x,
                  f"pde-banded-complex N={N} m={m} nrhs={nrhs} hb={hb} seed={seed}")


def laplace_fill_system(N: int, m: int, nrhs: int, seed: int, eps: float = 1e-2) -> System:
    """Five-point 2-D Laplace operator on an N x m grid (blocks: B_i =
    tridiag(-1, 4, -1), A_i = C_i = -I), every block's zero entries filled
    with uniform [-eps, eps] values -- the shape of the paper's validation
    matrices (Laplace discretisation with small random fill)."""
    A = eps * uniform(seed, STREAM_A, N * m * m, -1.0, 1.0).reshape(N, m, m)
    B = eps * uniform(seed, STREAM_B, N * m * m, -1.0, 1.0).reshape(N, m, m)
    C = eps * uniform(seed, STREAM_C, N * m * m, -1.0, 1.0).reshape(N, m, m)
    idx = np.arange(m)
    A[:, idx, idx] = -1.0
    C[:, idx, idx] = -1.0
    B[:, idx, idx] = 4.0
    B[:, idx[1:], idx[:-1]] = -1.0
    B[:, idx[:-1], idx[1:]] = -1.0
    A[0] = 0.0
    C[N - 1] = 0.0
    x = normal(seed, STREAM_X, N * m * nrhs).reshape(N, m, nrhs)
    return System(A, B, C, manufacture_rhs(A, B, C, x), x,
                  f"laplace-fill N={N} m={m} nrhs={nrhs} eps={eps:g} seed={seed}")


def conditioned_system(N: int, m: int, nrhs: int, seed: int, cond: float = 1e4) -> System:
    """Dense nonsymmetric diagonal blocks with cond_2(B_i) = ``cond`` and
    off-diagonal blocks small enough for block diagonal dominance."""
    gu = normal(seed, STREAM_U, N * m * m).reshape(N, m, m)
    gv = normal(seed, STREAM_V, N * m * m).reshape(N, m, m)
    U, _ = np.linalg.qr(gu)
    V, _ = np.linalg.qr(gv)
    sigma = np.logspace(np.log10(cond), 0.0, m) if m > 1 else np.ones(1)
    B = np.ascontiguousarray(np.matmul(U * sigma[None, None, :], np.swapaxes(V, 1, 2)))
    A = uniform(seed, STREAM_A, N * m * m, -1.0, 1.0).reshape(N, m, m)
    C = uniform(seed, STREAM_C, N * m * m, -1.0, 1.0).reshape(N, m, m)
    A[0] = 0.0
    C[N - 1] = 0.0
    for M in (A, C):
        f = np.sqrt(np.sum(M * M, axis=(1, 2)))
        f[f == 0] = 1.0
        M *= (0.25 / f)[:, None, None]
    x = normal(seed, STREAM_X, N * m * nrhs).reshape(N, m, nrhs)
    return System(A, B, C, manufacture_rhs(A, B, C, x), x,
                  f"conditioned N={N} m={m} nrhs={nrhs} cond={cond:g} seed={seed}")


def batch_shapes(count: int, seed: int, n_lo=32, n_hi=2048, ms=(32, 64, 96, 128),
                 r_lo=1, r_hi=16):
    """Shapes (N, m, nrhs) of ``count`` independent systems: N uniform in
    [n_lo, n_hi], m uniform over ``ms``, nrhs uniform in [r_lo, r_hi]."""
    u = uniform(seed, STREAM_SHAPE, 3 * count).reshape(count, 3)
    Ns = n_lo + np.minimum((u[:, 0] * (n_hi - n_lo + 1)).astype(np.int64), n_hi - n_lo)
    mi = np.minimum((u[:, 1] * len(ms)).astype(np.int64), len(ms) - 1)
    rs = r_lo + np.minimum((u[:, 2] * (r_hi - r_lo + 1)).astype(np.int64), r_hi - r_lo)
    return [(int(n), int(ms[j]), int(r)) for n, j, r in zip(Ns, mi, rs)]


# ---------------------------------------------------------------- device copies
# The same generator written with torch int64 tensors, so that large inputs
# can be drawn directly in device memory.  Uniform draws are bit-identical to
# the numpy version (wrapping int64 arithmetic, logical shifts by masking);
# the dominance shift uses the same summation order; normals and b = T x may
# differ from the numpy version in the last bits (different log/cos/matmul).
def _t_u64(torch, seed, stream, count, offset, device):
    I64 = torch.int64
    sgn = lambda v: v - (1 << 64) if v >= (1 << 63) else v
    key = int(_key(seed, stream))
    k = torch.arange(offset + 1, offset + count + 1, dtype=I64, device=device)
    z = sgn(key) + k * sgn(int(_G))
    z = (z ^ ((z >> 30) & ((1 << 34) - 1))) * sgn(int(_M1))
    z = (z ^ ((z >> 27) & ((1 << 37) - 1))) * sgn(int(_M2))
    return z ^ ((z >> 31) & ((1 << 33) - 1))


def uniform_t(seed, stream, count, lo=0.0, hi=1.0, offset=0, device="cuda"):
    """torch version of ``uniform`` (bit-identical draws)."""
    import torch
    z = _t_u64(torch, seed, stream, count, offset, device)
    u = ((z >> 11) & ((1 << 53) - 1)).to(torch.float64) * (2.0 ** -53)
    return lo + (hi - lo) * u


def normal_t(seed, stream, count, device="cuda"):
    import torch
    u1 = uniform_t(seed, stream, count, device=device)
    u2 = uniform_t(seed, stream + 1000, count, device=device)
    return torch.sqrt(-2.0 * torch.log1p(-u1)) * torch.cos(2.0 * np.pi * u2)


def dominant_system_t(N, m, nrhs, seed, device="cuda"):
    """``dominant_system`` drawn in device memory: returns torch tensors
    (A, B, C, b, x_true) with the numpy version's shapes."""
    import torch
    A = uniform_t(seed, STREAM_A, N * m * m, -1.0, 1.0, device=device).reshape(N, m, m)
    B = uniform_t(seed, STREAM_B, N * m * m, -1.0, 1.0, device=device).reshape(N, m, m)
    C = uniform_t(seed, STREAM_C, N * m * m, -1.0, 1.0, device=device).reshape(N, m, m)
    A[0] = 0.0
    C[N - 1] = 0.0
    sh = torch.zeros((N, m), dtype=torch.float64, device=device)
    for M in (A, B, C):
        for j in range(m):
            sh += torch.abs(M[:, :, j])
    idx = torch.arange(m, device=device)
    B[:, idx, idx] += sh + 1.0
    x = normal_t(seed, STREAM_X, N * m * nrhs, device=device).reshape(N, m, nrhs)
    b = torch.matmul(B, x)
    b[1:] += torch.matmul(A[1:], x[:-1])
    b[:-1] += torch.matmul(C[:-1], x[1:])
    return A, B, C, b, x


def random_rhs(N: int, m: int, nrhs: int, seed: int) -> np.ndarray:
    """A fresh right-hand side ~ N(0, 1) for repeat solves on resident factors."""
    return normal(seed, STREAM_RHS, N * m * nrhs).reshape(N, m, nrhs)
