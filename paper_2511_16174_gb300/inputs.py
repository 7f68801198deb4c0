"""Seeded synthetic inputs shared by the tests, the oracle checks and the benchmark.

This module holds none of the eigensolver's arithmetic: it only draws random
matrices and spectra.  Every generator is deterministic in its seed (numpy PCG64 on
the host; a torch generator on the device for the large cases).

Workloads (the paper measures only synthetic matrices, Sec. 5 and Table 2):

* ``goe(n, seed)``             A = (G + G^T)/2 with G i.i.d. N(0, 1).
* ``qlq(lam, seed, k)``        A = H_k ... H_1 diag(lam) H_1 ... H_k, H_i = I - 2 v v^T / v^T v
                               with v ~ N(0, 1)^n: a dense matrix with a known spectrum.
* ``spectrum_geometric``       lam_i = +-10^(-8 i/(n-1)) with random signs (cond 1e8, ||A||_2 = 1).
* ``spectrum_uniform``         lam ~ U[-1, 1].
* ``spectrum_clustered``       5% of lam in clusters of 8 spaced 1e-6 (centres in [-1, 1]),
                               the rest U[-1, 1].
* ``batch_sizes``              n = round(exp(U[ln 64, ln 2048])) per matrix.
* ``laplacian(n)``             tridiag(-1, 2, -1).
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 16174


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def goe(n, seed):
    g = rng(seed).standard_normal((n, n))
    return np.asfortranarray((g + g.T) * 0.5)


def spectrum_uniform(n, seed):
    return np.sort(rng(seed).uniform(-1.0, 1.0, n))


def spectrum_geometric(n, seed):
    r = rng(seed)
    i = np.arange(n)
    mag = 10.0 ** (-8.0 * i / max(n - 1, 1))
    sgn = np.where(r.random(n) < 0.5, -1.0, 1.0)
    return np.sort(mag * sgn)


def spectrum_clustered(n, seed, frac=0.05, size=8, gap=1e-6):
    r = rng(seed)
    nclust = int(round(frac * n / size))
    lam = []
    for _ in range(nclust):
        c = r.uniform(-1.0 + size * gap, 1.0 - size * gap)
        lam.extend(c + gap * np.arange(size))
    rest = n - len(lam)
    lam.extend(r.uniform(-1.0, 1.0, rest))
    return np.sort(np.asarray(lam[:n]))


def reflector_vectors(n, seed, k=32):
    return rng(seed + 7919).standard_normal((k, n))


def qlq(lam, seed, k=32):
    """Dense symmetric matrix with eigenvalues lam (host, O(k n^2))."""
    lam = np.asarray(lam, dtype=np.float64)
    n = lam.shape[0]
    A = np.diag(lam)
    for v in reflector_vectors(n, seed, k):
        v = v / np.linalg.norm(v)
        # A <- H A H, H = I - 2 v v^T
        Av = A @ v
        vAv = v @ Av
        A = A - 2.0 * np.outer(v, Av) - 2.0 * np.outer(Av, v) + 4.0 * vAv * np.outer(v, v)
    A = 0.5 * (A + A.T)
    return np.asfortranarray(A)


def qlq_device(lam, seed, k=32, device="cuda"):
    """Same construction as ``qlq`` on the device with torch (for n >= 16384).
    Returns a column-major float64 tensor (as the transpose view of a contiguous
    tensor; A is symmetric so the values are the same)."""
    import torch
    lam_t = torch.as_tensor(np.asarray(lam, dtype=np.float64), device=device)
    n = lam_t.shape[0]
    A = torch.diag(lam_t)
    V = torch.as_tensor(reflector_vectors(n, seed, k), device=device)
    for v in V:
        v = v / torch.linalg.vector_norm(v)
        Av = A @ v
        vAv = torch.dot(v, Av)
        A.addr_(v, Av, alpha=-2.0)
        A.addr_(Av, v, alpha=-2.0)
        A.addr_(v, v, alpha=4.0 * float(vAv))
    A = 0.5 * (A + A.T)
    return A.contiguous()


def goe_device(n, seed, device="cuda"):
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    G = torch.randn((n, n), generator=g, device=device, dtype=torch.float64)
    A = G + G.T
    A.mul_(0.5)
    return A


def batch_sizes(count, seed, lo=64, hi=2048):
    r = rng(seed)
    return np.rint(np.exp(r.uniform(np.log(lo), np.log(hi), count))).astype(np.int64)


def laplacian(n):
    return np.asfortranarray(2.0 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1))
