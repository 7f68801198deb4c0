"""Reference error-free splitting of FP64 rows into small integer slices
(test infrastructure).

This is the splitting definition the tensor-core product uses, written out with
exact integer arithmetic (the Ozaki scheme: Ozaki, Ogita, Oishi & Rump, "Error-free
transformations of matrix multiplication by using fast routines of matrix
multiplication and its applications", Numer. Algorithms 59 (2012); here with
balanced base-2^w digits so each digit fits a bfloat16 exactly):

For a row a (length K) of the left operand (or a column of the right operand):

* e = the binary exponent with max_k |a_k| < 2^e <= 2 max_k |a_k| (frexp's
  exponent of the row maximum); e = 0 for an all-zero row.
* T_k = round_half_away(a_k * 2^(w s - e)), an integer with |T_k| <= 2^(w s).
* balanced digits: T_k = sum_{t<s} sigma_{t,k} 2^(w (s-1-t)) with
  sigma_t in [-2^(w-1), 2^(w-1)) for t >= 1 and |sigma_0| <= 2^w.

so that a_k ~= 2^e sum_t sigma_t 2^(-w (t+1)) with error <= 2^(e - w s - 1).

``ozaki_split`` returns (sigma[s, rows, K] int64, e[rows] int64).
``ozaki_exact_products`` returns the exact integer products sum_k sigma^A_t sigma^B_u
for every slice pair, and ``ozaki_value`` the FP64 value the truncated pair sum
represents.
"""
from __future__ import annotations

import numpy as np


def _row_exponents(X):
    amax = np.max(np.abs(X), axis=1) if X.shape[1] > 0 else np.zeros(X.shape[0])
    _, E = np.frexp(amax)
    E = E.astype(np.int64)
    E[amax == 0] = 0
    return E


def ozaki_split(X, s=8, w=7):
    """Split each ROW of X (rows x K float64) into s balanced base-2^w digits."""
    X = np.asarray(X, dtype=np.float64)
    rows, K = X.shape
    e = _row_exponents(X)
    f, E = np.frexp(X)                       # X = f 2^E, 0.5 <= |f| < 1
    M = np.round(f * 2.0 ** 53).astype(np.int64)   # exact: |M| < 2^53 integer
    sh = E.astype(np.int64) - 53 + w * s - e[:, None]  # T = M * 2^sh
    T = np.zeros_like(M)
    pos = sh >= 0
    T[pos] = M[pos] << sh[pos]
    neg = ~pos
    rsh = np.minimum(-sh[neg], 62)
    mag = np.abs(M[neg])
    half = np.where(rsh > 0, np.left_shift(np.int64(1), np.maximum(rsh - 1, 0)), 0)
    q = (mag + half) >> rsh
    T[neg] = np.where(M[neg] < 0, -q, q)
    T[X == 0] = 0
    base = 1 << w
    halfb = base >> 1
    sig = np.zeros((s, rows, K), dtype=np.int64)
    for t in range(s - 1, 0, -1):
        r = ((T + halfb) % base) - halfb
        sig[t] = r
        T = (T - r) >> w
    sig[0] = T
    return sig, e


def ozaki_exact_products(sa, sb):
    """sa: [s, M, K], sb: [s, N, K] integer slices.  Returns P[t, u] = sa_t sb_u^T
    as exact int64 (|entries| stay far below 2^63 for K < 2^40)."""
    s = sa.shape[0]
    P = np.zeros((s, s, sa.shape[1], sb.shape[1]), dtype=np.int64)
    for t in range(s):
        for u in range(s):
            P[t, u] = sa[t] @ sb[u].T
    return P


def ozaki_value(sa, ea, sb, eb, w=7, max_weight=None):
    """FP64 value of the truncated Ozaki product sum over pairs with t + u <= L,
    C = 2^(ea + eb) sum 2^(-w (t + u + 2)) P_tu, evaluated in exact rationals via
    Python integers per weight then rounded once."""
    s = sa.shape[0]
    L = s - 1 if max_weight is None else max_weight
    P = ozaki_exact_products(sa, sb)
    M, N = sa.shape[1], sb.shape[1]
    out = np.zeros((M, N))
    for i in range(M):
        for j in range(N):
            tot = 0
            for k in range(L + 1):
                Sk = sum(int(P[t, k - t, i, j]) for t in range(k + 1) if k - t < s)
                tot += Sk << (w * (L - k))
            # value = tot * 2^(ea+eb - w (L + 2))
            out[i, j] = float(tot) * 2.0 ** (int(ea[i]) + int(eb[j]) - w * (L + 2)) if tot != 0 else 0.0
    return out
