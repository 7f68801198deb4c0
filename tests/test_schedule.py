"""Host-side schedule rules of the CUDA path, checked by brute force on the CPU.

1. Bulge chasing (Sec. 4.2): sweep j step k may start once sweep j-1 has completed
   step k+1, provided sweep j-1 publishes the beta entry of its step k+2 during step
   k+1.  Checked on the entry sets every step touches (lower triangle): sweep j step k
   shares no entry with any later step of an earlier sweep except that one beta
   entry.  Lag 1 (no look-ahead) must fail the same check.
2. BC back-transformation (Sec. 2.1.2): applying the reflector groups G(J, k) by waves
   t = k + (nJ - 1 - J), groups of a wave in any order, gives the same product as
   applying every reflector in generation order.  A wrong wave formula must fail.
"""
import numpy as np
import pytest


def sweep_steps(n, b, j):
    return 0 if j + 3 > n else (n - 3 - j) // b + 1


def touch(n, b, j, k):
    """Lower-triangle entries step k of sweep j reads or writes."""
    r0 = j + 1 + k * b
    r1 = min(r0 + b - 1, n - 1)
    c = j if k == 0 else r0 - b
    S = set()
    for r in range(r0, r1 + 1):
        S.update((r, cc) for cc in range(c, r0))      # left block (bulge) incl. annihilated column
        S.update((r, q) for q in range(r0, r + 1))    # diagonal block
    for r in range(r1 + 1, min(r1 + b, n - 1) + 1):
        S.update((r, q) for q in range(r0, r1 + 1))   # block below (next bulge)
    return S


def beta_entry(n, b, j, k):
    r0 = j + 1 + k * b
    return (r0, j if k == 0 else r0 - b)


def lag_violations(n, b, lag, early_beta):
    T = {(j, k): touch(n, b, j, k) for j in range(n - 2) for k in range(sweep_steps(n, b, j))}
    bad = []
    for (j, k), S in T.items():
        for d in range(1, 4):
            jj = j - d
            if jj < 0:
                continue
            done = k + (lag - 1) * d  # steps of sweep j-d complete when (j, k) starts
            for kk in range(sweep_steps(n, b, jj)):
                if kk <= done:
                    continue
                inter = S & T[(jj, kk)]
                if early_beta and d == 1 and kk == done + 1:
                    inter -= {beta_entry(n, b, jj, kk)}
                if inter:
                    bad.append((j, k, jj, kk))
    return bad


@pytest.mark.parametrize("n,b", [(20, 2), (37, 3), (64, 4), (70, 5), (100, 8), (41, 16)])
def test_bc_lag2_with_early_beta_is_race_free(n, b):
    assert lag_violations(n, b, lag=2, early_beta=True) == []


@pytest.mark.parametrize("n,b", [(37, 3), (64, 4)])
def test_bc_lag3_is_race_free_and_lag2_needs_early_beta(n, b):
    assert lag_violations(n, b, lag=3, early_beta=False) == []
    assert lag_violations(n, b, lag=2, early_beta=False) != []
    assert lag_violations(n, b, lag=1, early_beta=True) != []


def _reflectors(n, b, rng):
    """Random Householder reflectors H_{j,k} = I - tau v v^T on rows r0 .. r0+m-1."""
    H = {}
    for j in range(n - 2):
        for k in range(sweep_steps(n, b, j)):
            r0 = j + 1 + k * b
            m = min(b, n - r0)
            v = rng.standard_normal(m)
            v[0] = 1.0
            H[(j, k)] = (r0, v, 2.0 / (v @ v))
    return H


def _apply(X, r0, v, tau):
    rows = slice(r0, r0 + len(v))
    X[rows] -= tau * np.outer(v, v @ X[rows])


def _waves(n, b, g, formula):
    nJ = -(-(n - 2) // g)
    groups = [(J, k) for J in range(nJ) for k in range(sweep_steps(n, b, J * g))]
    out = {}
    for (J, k) in groups:
        out.setdefault(formula(J, k, nJ), []).append((J, k))
    return [out[t] for t in sorted(out)]


def _apply_group(X, H, n, b, g, J, k):
    # G(J, k) = H_{Jg,k} H_{Jg+1,k} ... H_{Jg+g-1,k}; X <- G X applies j descending
    for j in range(min(J * g + g, n - 2) - 1, J * g - 1, -1):
        if (j, k) in H:
            _apply(X, *H[(j, k)])


@pytest.mark.parametrize("n,b", [(40, 3), (57, 4), (66, 5), (30, 2)])
def test_bc_back_waves_equal_sequential_product(n, b):
    rng = np.random.default_rng(16174 + n + b)
    H = _reflectors(n, b, rng)
    X0 = rng.standard_normal((n, n))
    # sequential: Q_b = prod over (j, k) in generation order; X <- Q_b X applies reverse order
    Xs = X0.copy()
    for key in sorted(H, reverse=True):
        _apply(Xs, *H[key])
    g = b
    waves = _waves(n, b, g, lambda J, k, nJ: k + (nJ - 1 - J))
    Xw = X0.copy()
    for wave in waves:
        # groups of one wave are row-disjoint
        rows = [set(range(J * g + 1 + k * b, min(J * g + k * b + g + b, n))) for (J, k) in wave]
        for a in range(len(rows)):
            for c in range(a + 1, len(rows)):
                assert not (rows[a] & rows[c])
        for (J, k) in reversed(wave):  # any order inside a wave
            _apply_group(Xw, H, n, b, g, J, k)
    assert np.max(np.abs(Xw - Xs)) <= 1e-12 * np.max(np.abs(Xs))
    # a plausible mistake -- waves by k - (nJ - 1 - J) -- must not reproduce it
    bad = _waves(n, b, g, lambda J, k, nJ: k - (nJ - 1 - J))
    Xb = X0.copy()
    for wave in bad:
        for (J, k) in wave:
            _apply_group(Xb, H, n, b, g, J, k)
    assert np.max(np.abs(Xb - Xs)) > 1e-6
