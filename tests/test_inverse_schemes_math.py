"""CPU check (no GPU) of the algebra behind the two float32 block inverses,
emulated in numpy on small blocks and compared with numpy.linalg.inv.

* Implicit pivoting (k_inv_reg): rows are never exchanged; step k takes the
  unused row p_k with the largest |w[i][k]| as its pivot row.  The working
  matrix then ends as W[p_r][c] = inv(D)[r][p_c].
* Panel-blocked Gauss-Jordan (k_inv_blocked): a panel of NB columns is
  eliminated alone (its row exchanges and eliminations restricted to the
  panel), which leaves the panel holding the NB non-trivial columns of the
  composed elimination M = I + X; every other column then takes the panel's
  row exchanges and the rank-NB update a[i][j] <- [i not a pivot row] a[i][j]
  + sum_l M[i][k0+l] a[k0+l][j]; the exchanges are undone on the columns at
  the end."""
import numpy as np
import pytest


def inv_implicit(D):
    m = D.shape[0]
    W = D.copy()
    used = np.zeros(m, bool)
    piv = []
    for k in range(m):
        cand = [i for i in range(m) if not used[i]]
        p = max(cand, key=lambda i: (abs(W[i, k]), -i))
        used[p] = True
        piv.append(p)
        inv = 1.0 / W[p, k]
        rs = W[p, :] * inv
        col = W[:, k].copy()
        W = W - np.outer(col, rs)
        W[p, :] = rs
        W[:, k] = -col * inv
        W[p, k] = inv
    G = np.empty_like(W)
    for r in range(m):
        for c in range(m):
            G[r, piv[c]] = W[piv[r], c]
    return G


def inv_panels(D, nb):
    m = D.shape[0]
    a = D.copy()
    perm = np.zeros(m, int)
    for k0 in range(0, m, nb):
        nbk = min(nb, m - k0)
        P = slice(k0, k0 + nbk)
        for j in range(nbk):
            k = k0 + j
            bi = k + int(np.argmax(np.abs(a[k:, k])))
            a[[k, bi], P] = a[[bi, k], P]
            perm[k] = bi
            inv = 1.0 / a[k, k]
            rk = a[k, P] * inv
            ck = a[:, k].copy()
            a[:, P] = a[:, P] - np.outer(ck, rk)
            a[k, P] = rk
            a[:, k] = -ck * inv
            a[k, k] = inv
        pan = a[:, P].copy()
        other = [j for j in range(m) if not (k0 <= j < k0 + nbk)]
        for l in range(nbk):
            k, pr = k0 + l, perm[k0 + l]
            if pr != k:
                tmp = a[k, other].copy()
                a[k, other] = a[pr, other]
                a[pr, other] = tmp
        Y = a[P][:, other].copy()
        base = a[:, other].copy()
        base[P, :] = 0.0
        a[:, other] = base + pan @ Y
    idx = list(range(m))
    for k in range(m - 1, -1, -1):
        q = perm[k]
        idx[k], idx[q] = idx[q], idx[k]
    G = np.empty_like(a)
    for c in range(m):
        G[:, idx.index(c)] = a[:, c]
    return G


@pytest.mark.parametrize("m", [1, 2, 5, 16, 40])
def test_implicit_pivoting_relabels_rows_and_columns(m):
    D = np.random.default_rng(m).standard_normal((m, m))
    assert np.allclose(inv_implicit(D), np.linalg.inv(D), rtol=1e-9, atol=1e-9 * np.abs(np.linalg.inv(D)).max())


@pytest.mark.parametrize("m,nb", [(5, 8), (16, 8), (40, 8), (33, 4), (64, 16)])
def test_panel_update_composes_the_eliminations(m, nb):
    D = np.random.default_rng(100 + m).standard_normal((m, m))
    Ginv = np.linalg.inv(D)
    assert np.allclose(inv_panels(D, nb), Ginv, rtol=1e-9, atol=1e-9 * np.abs(Ginv).max())


def test_pivots_match_explicit_exchanges():
    """Implicit pivoting chooses the same pivot rows as explicit exchanges
    (away from ties): compare the sequences on a random block."""
    m = 24
    D = np.random.default_rng(7).standard_normal((m, m))
    # explicit partial pivoting with exchanges: record the original row of each pivot
    a, rows, expl = D.copy(), list(range(m)), []
    for k in range(m):
        p = k + int(np.argmax(np.abs(a[k:, k])))
        a[[k, p]] = a[[p, k]]
        rows[k], rows[p] = rows[p], rows[k]
        expl.append(rows[k])
        a[k + 1:] -= np.outer(a[k + 1:, k] / a[k, k], a[k])
    W, used, impl = D.copy(), np.zeros(m, bool), []
    for k in range(m):
        p = max((i for i in range(m) if not used[i]), key=lambda i: abs(W[i, k]))
        used[p] = True
        impl.append(p)
        W[~used] -= np.outer(W[~used, k] / W[p, k], W[p])
    assert impl == expl
