"""Two product decompositions the GPU path uses, checked on the CPU with exact
(integer-valued) matrices so that equality is exact.

* Presplit Z products (double-blocked SBR, Sec. 4.1): the product of a principal
  submatrix A2[off:, off:] with W equals the product started at the row tile below
  off (off0 = 128 floor(off / 128), e = off - off0) against W with e zero rows in
  front, with the first e rows of the result dropped.
* D&C merge by halves: with the merged block's columns grouped as [top only | both
  | bottom only] (a column is "both" once a deflation rotation mixes a top and a
  bottom column) and U's rows permuted the same way, X = Qn U equals
  [Qn_top[:, :c1+c2] U[:c1+c2]; Qn_bot[:, c1:] U[c1:]]; a control that ignores the
  mixing gets a different product.
"""
import numpy as np
import pytest


@pytest.mark.parametrize("m_block,b,q", [(1000, 64, 1), (1000, 64, 2), (1000, 64, 3), (700, 32, 5), (513, 16, 9)])
def test_presplit_offset_product(m_block, b, q):
    rng = np.random.default_rng(100 + q)
    A2 = rng.integers(-5, 6, (m_block, m_block)).astype(np.float64)
    A2 = np.tril(A2) + np.tril(A2, -1).T  # symmetric, as the presplit mirrors the lower triangle
    off = q * b
    m = m_block - off
    W = rng.integers(-5, 6, (m, b)).astype(np.float64)
    direct = A2[off:, off:] @ W
    off0 = off // 128 * 128
    e = off - off0
    Wpad = np.vstack([np.zeros((e, b)), W])  # K-elements 0 .. e-1 read as zero
    prod = A2[off0:, off0:] @ Wpad  # rows and K from the tile boundary
    assert np.array_equal(prod[e:], direct)  # the first e rows are not stored


def deflation_groups(is_top, rotations):
    """Group of each column after the rotations (1 top, 2 bottom, 3 both): a rotation
    (p, j) leaves j holding a combination of p and j."""
    g = np.where(is_top, 1, 2)
    for p, j in rotations:
        g[j] |= g[p]
    return g


@pytest.mark.parametrize("seed", range(6))
def test_merge_by_halves(seed):
    rng = np.random.default_rng(seed)
    n1, n2 = 37 + seed, 41
    m = n1 + n2
    Q1 = rng.integers(-3, 4, (n1, n1)).astype(np.float64)
    Q2 = rng.integers(-3, 4, (n2, n2)).astype(np.float64)
    Qb = np.zeros((m, m))
    Qb[:n1, :n1] = Q1
    Qb[n1:, n1:] = Q2
    # columns in sorted (pole) order: a random interleaving of the two halves
    perm = rng.permutation(m)
    Qt = Qb[:, perm]
    is_top = perm < n1
    # deflation rotations between neighbours (p, j), p < j, applied in order; p is deflated
    rots, deflated = [], set()
    j = 0
    while j < m - 1:
        if rng.random() < 0.25:
            rots.append((j, j + 1))
            deflated.add(j)
        j += 1
    for p, jj in rots:  # integer-valued "rotation" that mixes the two columns
        qp, qj = Qt[:, p].copy(), Qt[:, jj].copy()
        Qt[:, p] = qp - qj
        Qt[:, jj] = qp + qj
    groups = deflation_groups(is_top, rots)
    nd = [c for c in range(m) if c not in deflated]
    k = len(nd)
    U = rng.integers(-3, 4, (k, k)).astype(np.float64)
    dense = Qt[:, nd] @ U
    # grouped order, ascending within a group
    g = groups[nd]
    order = [i for i in range(k) if g[i] == 1] + [i for i in range(k) if g[i] == 3] + \
            [i for i in range(k) if g[i] == 2]
    c1, c2 = int(np.sum(g == 1)), int(np.sum(g == 3))
    Qn = Qt[:, nd][:, order]
    Ug = U[order, :]
    # top-only columns vanish below n1, bottom-only ones above n1
    assert not np.any(Qn[n1:, :c1]) and not np.any(Qn[:n1, c1 + c2:])
    X = np.vstack([Qn[:n1, :c1 + c2] @ Ug[:c1 + c2], Qn[n1:, c1:] @ Ug[c1:]])
    assert np.array_equal(X, dense)
    # control: leaving the mixed columns out of the bottom product loses their share
    if c2 > 0:
        X_wrong = np.vstack([Qn[:n1, :c1 + c2] @ Ug[:c1 + c2], Qn[n1:, c1 + c2:] @ Ug[c1 + c2:]])
        assert not np.array_equal(X_wrong, dense)
