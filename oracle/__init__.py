"""Plain FP64 CPU oracle for A = Q Lambda Q^T (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA product path never does, and it
shares no code with it.  The arithmetic lives in ``evd_oracle.c`` (built by
``oracle/build.py``); this module only marshals numpy arrays.

Functions (each restates the passage cited in the C source):

* ``sytrd(A, want_q)``     one-stage Householder tridiagonalization (Sec. 1)
* ``steql(d, e, Z)``       implicit QL with Wilkinson shift (Sec. 1, QR-algorithm family)
* ``bisect(d, e)``         Sturm bisection
* ``jacobi(A)``            cyclic Jacobi (brute force, tiny n)
* ``sbr(A, b)``            successive band reduction, panel QR + Eq. 1 (Sec. 2.1.1)
* ``sbr_q(Ys, taus)``      Q_s from the SBR reflectors
* ``bc(B, b, want_q)``     bulge chasing band -> tridiagonal (Sec. 2.1.1, Sec. 4.2)
* ``eigh(A, want_vectors)`` the oracle EVD: sytrd + steql
* ``metrics(...)``         the error measures of Sec. 3.3.1 / Table 2 and the
                           acceptance bounds
* ``refine(...)``          one Ogita-Aishima eigenpair refinement step
* ``refine_steps(...)``    several steps, the cluster threshold held
* ``ozaki_split(...)``     reference error-free splitting of FP64 rows into
                           integer slices (definition written out)

Numbers are column-major float64 (``order='F'``).
"""
from __future__ import annotations

import ctypes
import os
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_LIB = None

_dp = ctypes.POINTER(ctypes.c_double)


def _lib():
    global _LIB
    if _LIB is None:
        path = _HERE / "libevd_oracle.so"
        if not path.exists():
            from . import build as _b
            _b.build()
        lib = ctypes.CDLL(str(path))
        for name, args in {
            "orc_sytrd_lower": [ctypes.c_int, _dp, ctypes.c_int, _dp, _dp, _dp, ctypes.c_int],
            "orc_steql": [ctypes.c_int, _dp, _dp, _dp, ctypes.c_int],
            "orc_bisect": [ctypes.c_int, _dp, _dp, _dp],
            "orc_jacobi": [ctypes.c_int, _dp, ctypes.c_int, _dp, _dp, ctypes.c_int],
            "orc_sbr": [ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int, _dp, ctypes.c_int, _dp],
            "orc_sbr_q": [ctypes.c_int, _dp, ctypes.c_int, _dp, _dp, ctypes.c_int],
            "orc_bc": [ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int, _dp, _dp, _dp, ctypes.c_int],
            "orc_house": [ctypes.c_int, _dp, _dp],
        }.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int if name != "orc_house" else None
        lib.orc_num_threads.restype = ctypes.c_int
        _LIB = lib
    return _LIB


def _p(a):
    if a is None:
        return None
    return a.ctypes.data_as(_dp)


def _fmat(A):
    return np.array(A, dtype=np.float64, order="F", copy=True)


def num_threads() -> int:
    return int(_lib().orc_num_threads())


def house(x):
    """Householder reflector of x: returns (beta, v, tau), v[0] = 1."""
    x = np.array(x, dtype=np.float64)
    tau = ctypes.c_double(0.0)
    _lib().orc_house(len(x), _p(x), ctypes.byref(tau))
    beta = x[0]
    v = x.copy()
    v[0] = 1.0
    return beta, v, tau.value


def sytrd(A, want_q=False):
    """One-stage tridiagonalization of the lower triangle of A -> (d, e, Q|None)."""
    A = _fmat(A)
    n = A.shape[0]
    d = np.zeros(n)
    e = np.zeros(max(n, 1))
    Q = np.zeros((n, n), order="F") if want_q else None
    rc = _lib().orc_sytrd_lower(n, _p(A), max(n, 1), _p(d), _p(e), _p(Q), max(n, 1))
    if rc != 0:
        raise RuntimeError(f"orc_sytrd_lower failed: {rc}")
    return d, e[: max(n - 1, 0)], Q


def steql(d, e, Z=None):
    """Implicit QL on (d, e); rotations accumulated into Z (None: values only,
    'I': identity).  Returns (w ascending, Z|None)."""
    n = len(d)
    d = np.array(d, dtype=np.float64)
    ee = np.zeros(max(n, 1))
    ee[: max(n - 1, 0)] = np.asarray(e, dtype=np.float64)[: max(n - 1, 0)]
    if isinstance(Z, str) and Z == "I":
        Z = np.eye(n, order="F")
    elif Z is not None:
        Z = _fmat(Z)
    rc = _lib().orc_steql(n, _p(d), _p(ee), _p(Z), max(n, 1))
    if rc != 0:
        raise RuntimeError(f"orc_steql did not converge: {rc}")
    return d, Z


def bisect(d, e):
    n = len(d)
    d = np.array(d, dtype=np.float64)
    ee = np.zeros(max(n, 1))
    ee[: max(n - 1, 0)] = np.asarray(e, dtype=np.float64)[: max(n - 1, 0)]
    w = np.zeros(n)
    _lib().orc_bisect(n, _p(d), _p(ee), _p(w))
    return w


def jacobi(A, want_vectors=True):
    A = _fmat(A)
    n = A.shape[0]
    w = np.zeros(n)
    V = np.zeros((n, n), order="F") if want_vectors else None
    rc = _lib().orc_jacobi(n, _p(A), max(n, 1), _p(w), _p(V), max(n, 1))
    if rc < 0:
        raise RuntimeError(f"orc_jacobi failed: {rc}")
    return w, V


def sbr(A, b, keep_reflectors=False):
    """Successive band reduction of the lower triangle of A with half-width b.
    Returns (B full symmetric, Ys|None, taus|None)."""
    A = _fmat(A)
    n = A.shape[0]
    Ys = np.zeros((n, n), order="F") if keep_reflectors else None
    taus = np.zeros(max(n, 1)) if keep_reflectors else None
    rc = _lib().orc_sbr(n, int(b), _p(A), max(n, 1), _p(Ys), max(n, 1), _p(taus))
    if rc != 0:
        raise RuntimeError(f"orc_sbr failed: {rc}")
    return A, Ys, (taus[:n] if taus is not None else None)


def sbr_q(Ys, taus):
    n = Ys.shape[0]
    Q = np.zeros((n, n), order="F")
    Ys = _fmat(Ys)
    t = np.array(taus, dtype=np.float64)
    _lib().orc_sbr_q(n, _p(Ys), max(n, 1), _p(t), _p(Q), max(n, 1))
    return Q


def bc(B, b, want_q=False):
    """Bulge chasing of the band (half-width b) in the lower triangle of B.
    Returns (d, e, Qb|None) with B = Qb T Qb^T."""
    B = _fmat(B)
    n = B.shape[0]
    d = np.zeros(n)
    e = np.zeros(max(n, 1))
    Q = np.zeros((n, n), order="F") if want_q else None
    rc = _lib().orc_bc(n, int(b), _p(B), max(n, 1), _p(d), _p(e), _p(Q), max(n, 1))
    if rc != 0:
        raise RuntimeError(f"orc_bc failed: {rc}")
    return d, e[: max(n - 1, 0)], Q


def eigh(A, want_vectors=True):
    """Oracle EVD: one-stage tridiagonalization + implicit QL.
    Returns (w ascending, Q|None) with A = Q diag(w) Q^T."""
    d, e, Q = sytrd(A, want_q=want_vectors)
    w, Z = steql(d, e, Q if want_vectors else None)
    return w, Z


from .metrics import metrics, acceptance  # noqa: E402,F401
from .refine import refine, refine_steps  # noqa: E402,F401
from .ozaki import ozaki_split, ozaki_exact_products, ozaki_value  # noqa: E402,F401
