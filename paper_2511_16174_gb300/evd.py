"""Python binding of libevd (argument marshalling only).

Every name mirrors a C entry point of ``include/evd.h``; all arithmetic runs in the
CUDA library.  Matrices are column-major float64 CUDA tensors: a tensor ``X`` of shape
(n, n) is passed with leading dimension ``X.stride(1)`` and must have ``X.stride(0) ==
1`` (create one with :func:`empty_colmajor`).  The library is loaded from this
package's folder; if it is missing, importing this module raises -- there is no
fallback.
"""
from __future__ import annotations

import ctypes
from pathlib import Path

import torch

_HERE = Path(__file__).resolve().parent
_LIBPATH = _HERE / "libevd.so"
if not _LIBPATH.exists():
    raise ImportError(f"libevd.so not built ({_LIBPATH}); run __graft_entry__.build()")
_lib = ctypes.CDLL(str(_LIBPATH))

_i64 = ctypes.c_int64
_vp = ctypes.c_void_p
_int = ctypes.c_int
_dbl = ctypes.c_double
_sz = ctypes.c_size_t

EVD_VALUES, EVD_VECTORS = 0, 1
EVD_FP64, EVD_SPLIT_INT8, EVD_SPLIT_BF16 = 0, 1, 2
OPTIONS = {"slices": 0, "refine_iters": 1, "bcback_fused": 2, "bc_kernel": 3, "panel_ctas": 4, "xe_slices": 5,
           "bc_ctas_per_sm": 6, "order": 7, "sbr_slices": 8}
STATUS = ["EVD_OK", "EVD_ERR_INVALID_ARG", "EVD_ERR_WORKSPACE", "EVD_ERR_OOM", "EVD_ERR_CUDA",
          "EVD_ERR_NONFINITE", "EVD_ERR_NO_CONVERGENCE", "EVD_ERR_TIMEOUT", "EVD_ERR_NOT_SUPPORTED"]

_SIGS = {
    "evd_plan_create": ([ctypes.POINTER(_vp), _i64, _i64, _int, _int, _int, _int, _vp], _int),
    "evd_plan_workspace_size": ([_vp, ctypes.POINTER(_sz)], _int),
    "evd_plan_get_blocking": ([_vp, ctypes.POINTER(_int), ctypes.POINTER(_int)], _int),
    "evd_plan_set_option": ([_vp, _int, _int], _int),
    "evd_plan_get_option": ([_vp, _int, ctypes.POINTER(_int)], _int),
    "evd_sbr": ([_vp, _vp, _vp], _int),
    "evd_bulge_chase": ([_vp, _vp, _vp, _vp], _int),
    "evd_tridiag_solve": ([_vp, _vp, _vp, _vp, _i64, _vp], _int),
    "evd_back_transform": ([_vp, _vp, _vp, _vp, _i64], _int),
    "evd_syevd": ([_vp, _vp, _vp, _vp, _i64, _vp], _int),
    "evd_refine": ([_vp, _vp, _vp, _vp, _i64, _int, _vp], _int),
    "evd_plan_status": ([_vp, ctypes.POINTER(_int)], _int),
    "evd_wait_selftest": ([_vp, _int], _int),
    "evd_plan_destroy": ([_vp], None),
    "evd_status_string": ([_int], ctypes.c_char_p),
    "evd_batched_workspace_size": ([_int, ctypes.POINTER(_i64), _int, ctypes.POINTER(_sz)], _int),
    "evd_syevd_batched": ([_int, ctypes.POINTER(_i64), ctypes.POINTER(_vp), ctypes.POINTER(_i64),
                           ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_i64), _int, _vp, _sz, _vp], _int),
    "evd_gemm_workspace_size": ([_i64, _i64, _i64, _int, ctypes.POINTER(_sz)], _int),
    "evd_dgemm": ([ctypes.c_char, ctypes.c_char, _i64, _i64, _i64, _dbl, _vp, _i64, _vp, _i64, _dbl, _vp, _i64,
                   _int, _vp, _sz, _vp], _int),
    "evd_dgemm_status": ([_vp, ctypes.POINTER(_int)], _int),
    "evd_dgemm_static": ([ctypes.c_char, ctypes.c_char, _i64, _i64, _i64, _dbl, _vp, _i64, _vp, _i64, _dbl, _vp,
                          _i64, _int, _vp], _int),
    "evd_batched_last_graph": ([], _int),
    "evd_autotune": ([_i64, _int, _int, ctypes.c_char_p, ctypes.POINTER(_int), ctypes.POINTER(_int)], _int),
    "evd_stats_enable": ([_int], None),
    "evd_stats_reset": ([], None),
    "evd_launch_count": ([], _i64),
    "evd_stats_categories": ([ctypes.c_char_p, _int], _int),
    "evd_stats_query": ([ctypes.c_char_p, ctypes.POINTER(_dbl), ctypes.POINTER(_dbl), ctypes.POINTER(_dbl),
                         ctypes.POINTER(_i64)], _int),
}
for _name, (_args, _res) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _res


class EvdError(RuntimeError):
    def __init__(self, code, where=""):
        self.code = code
        name = STATUS[code] if 0 <= code < len(STATUS) else f"status {code}"
        super().__init__(f"{where}: {name}" if where else name)


def _check(code, where):
    if code != 0:
        raise EvdError(code, where)


def library_path() -> str:
    return str(_LIBPATH)


def empty_colmajor(m, n, device="cuda", dtype=torch.float64):
    """An (m, n) tensor with column-major strides (1, m)."""
    return torch.empty((n, m), device=device, dtype=dtype).t()


def as_colmajor(X):
    if X.dim() != 2 or X.stride(0) != 1:
        Y = empty_colmajor(X.shape[0], X.shape[1], device=X.device, dtype=X.dtype)
        Y.copy_(X)
        return Y
    return X


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _ld(X):
    return max(1, X.stride(1)) if X.dim() == 2 else 1


def _stream_ptr(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def status_string(code):
    return _lib.evd_status_string(code).decode()


class Plan:
    """Mirror of evd_plan_t.  job: 'N' (values) or 'V' (vectors); prec: 'fp64' or
    'split_bf16' ('split_int8' is rejected with EVD_ERR_NOT_SUPPORTED)."""

    def __init__(self, n, lda=None, job="V", prec="fp64", b=0, nb=0, stream=None, options=None):
        self.n = int(n)
        self.lda = int(lda if lda is not None else max(1, n))
        self.job = EVD_VECTORS if job in ("V", EVD_VECTORS, True) else EVD_VALUES
        self.prec = {"fp64": EVD_FP64, "split_int8": EVD_SPLIT_INT8, "split_bf16": EVD_SPLIT_BF16}.get(prec, prec)
        self.stream = stream
        h = _vp()
        _check(_lib.evd_plan_create(ctypes.byref(h), self.n, self.lda, self.job, self.prec, int(b), int(nb),
                                    _stream_ptr(stream)), "evd_plan_create")
        self._h = h
        for key, value in (options or {}).items():
            _check(_lib.evd_plan_set_option(h, OPTIONS[key], int(value)), f"evd_plan_set_option({key})")
        bb, nbb = _int(), _int()
        _lib.evd_plan_get_blocking(h, ctypes.byref(bb), ctypes.byref(nbb))
        self.b, self.nb = bb.value, nbb.value
        sz = _sz()
        _check(_lib.evd_plan_workspace_size(h, ctypes.byref(sz)), "evd_plan_workspace_size")
        self.workspace_bytes = sz.value

    def option(self, key):
        v = _int()
        _check(_lib.evd_plan_get_option(self._h, OPTIONS[key], ctypes.byref(v)), "evd_plan_get_option")
        return v.value

    def workspace(self, device="cuda"):
        return torch.empty(max(self.workspace_bytes, 256), dtype=torch.uint8, device=device)

    def close(self):
        if getattr(self, "_h", None):
            _lib.evd_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- stage calls (names follow include/evd.h)
    def sbr(self, A, ws):
        _check(_lib.evd_sbr(self._h, _ptr(A), _ptr(ws)), "evd_sbr")

    def bulge_chase(self, ws, d, e):
        _check(_lib.evd_bulge_chase(self._h, _ptr(ws), _ptr(d), _ptr(e)), "evd_bulge_chase")

    def tridiag_solve(self, d, e, Qd, ws):
        _check(_lib.evd_tridiag_solve(self._h, _ptr(d), _ptr(e), _ptr(Qd), _ld(Qd) if Qd is not None else 1,
                                      _ptr(ws)), "evd_tridiag_solve")

    def back_transform(self, A_reduced, ws, Q):
        _check(_lib.evd_back_transform(self._h, _ptr(A_reduced), _ptr(ws), _ptr(Q), _ld(Q)), "evd_back_transform")

    def syevd(self, A, w, Q, ws):
        _check(_lib.evd_syevd(self._h, _ptr(A), _ptr(w), _ptr(Q), _ld(Q) if Q is not None else 1, _ptr(ws)),
               "evd_syevd")

    def refine(self, A0, w, Q, iterations, ws):
        _check(_lib.evd_refine(self._h, _ptr(A0), _ptr(w), _ptr(Q), _ld(Q), int(iterations), _ptr(ws)),
               "evd_refine")

    def wait_selftest(self, kind):
        _check(_lib.evd_wait_selftest(self._h, int(kind)), "evd_wait_selftest")

    def status(self):
        info = _int()
        code = _lib.evd_plan_status(self._h, ctypes.byref(info))
        return code, info.value

    def check(self, where="device"):
        code, info = self.status()
        if code != 0:
            raise EvdError(code, f"{where} (info {info})")


def syevd(A, job="V", prec="fp64", b=0, nb=0, stream=None, overwrite=False, options=None):
    """Eigen-decomposition of the symmetric float64 CUDA matrix A (lower triangle
    read).  Returns (w ascending, Q column-major) or (w, None) for job='N'."""
    n = A.shape[0]
    Awork = as_colmajor(A) if overwrite else as_colmajor(A).clone(memory_format=torch.preserve_format)
    if Awork.stride(0) != 1:
        Awork = as_colmajor(Awork)
    plan = Plan(n, lda=_ld(Awork), job=job, prec=prec, b=b, nb=nb, stream=stream, options=options)
    ws = plan.workspace(A.device)
    w = torch.empty(n, dtype=torch.float64, device=A.device)
    Q = empty_colmajor(n, n, device=A.device) if plan.job == EVD_VECTORS else None
    plan.syevd(Awork, w, Q, ws)
    plan.check("evd_syevd")
    plan.close()
    return w, Q


def dgemm(transa, transb, alpha, A, B, beta, C, slices=8, stream=None):
    """C = alpha op(A) op(B) + beta C through evd_dgemm (column-major tensors)."""
    m, n = C.shape
    k = A.shape[1] if transa == "N" else A.shape[0]
    sz = _sz()
    _check(_lib.evd_gemm_workspace_size(m, n, k, int(slices), ctypes.byref(sz)), "evd_gemm_workspace_size")
    ws = torch.empty(max(sz.value, 256), dtype=torch.uint8, device=C.device)
    _check(_lib.evd_dgemm(transa.encode(), transb.encode(), m, n, k, float(alpha), _ptr(A), _ld(A), _ptr(B), _ld(B),
                          float(beta), _ptr(C), _ld(C), int(slices), _ptr(ws), sz.value, _stream_ptr(stream)),
           "evd_dgemm")
    return C


def dgemm_static(transa, transb, alpha, A, B, beta, C, slices=8, stream=None):
    """C = alpha op(A) op(B) + beta C through evd_dgemm_static (library-owned scratch,
    no workspace argument; see include/evd.h for its size limit and ordering rule)."""
    m, n = C.shape
    k = A.shape[1] if transa == "N" else A.shape[0]
    _check(_lib.evd_dgemm_static(transa.encode(), transb.encode(), m, n, k, float(alpha), _ptr(A), _ld(A), _ptr(B),
                                 _ld(B), float(beta), _ptr(C), _ld(C), int(slices), _stream_ptr(stream)),
           "evd_dgemm_static")
    return C


def dgemm_status(stream=None):
    """(code, info) of the stand-alone products' device status (evd_dgemm_status)."""
    info = _int()
    code = _lib.evd_dgemm_status(_stream_ptr(stream), ctypes.byref(info))
    return code, info.value


def syevd_batched(As, job="V", stream=None):
    """Batched solve of a list of symmetric float64 CUDA matrices (each overwritten).
    Returns lists (ws, Qs)."""
    count = len(As)
    ns = (_i64 * count)(*[a.shape[0] for a in As])
    Acm = [as_colmajor(a) for a in As]
    lds = (_i64 * count)(*[_ld(a) for a in Acm])
    ws_list = [torch.empty(a.shape[0], dtype=torch.float64, device=a.device) for a in Acm]
    Qs = [empty_colmajor(a.shape[0], a.shape[0], device=a.device) for a in Acm] if job == "V" else [None] * count
    ldq = (_i64 * count)(*[max(1, a.shape[0]) for a in Acm])
    jb = EVD_VECTORS if job == "V" else EVD_VALUES
    sz = _sz()
    _check(_lib.evd_batched_workspace_size(count, ns, jb, ctypes.byref(sz)), "evd_batched_workspace_size")
    ws = torch.empty(max(sz.value, 256), dtype=torch.uint8, device=As[0].device)
    Ap = (_vp * count)(*[a.data_ptr() for a in Acm])
    wp = (_vp * count)(*[w.data_ptr() for w in ws_list])
    Qp = (_vp * count)(*[(q.data_ptr() if q is not None else 0) for q in Qs])
    _check(_lib.evd_syevd_batched(count, ns, Ap, lds, wp, Qp, ldq, jb, _ptr(ws), sz.value, _stream_ptr(stream)),
           "evd_syevd_batched")
    return ws_list, Qs


class Batch:
    """Fixed buffers for repeated batched solves of the same sizes: inputs A[i]
    (column-major, overwritten by each run), outputs w[i], Q[i], one workspace.  A
    run with the same buffers replays the library's captured graph."""

    def __init__(self, sizes, job="V", device="cuda"):
        self.sizes = [int(n) for n in sizes]
        self.job = EVD_VECTORS if job == "V" else EVD_VALUES
        cnt = len(self.sizes)
        self.A = [empty_colmajor(n, n, device=device) for n in self.sizes]
        self.w = [torch.empty(n, dtype=torch.float64, device=device) for n in self.sizes]
        self.Q = [empty_colmajor(n, n, device=device) for n in self.sizes] if self.job == EVD_VECTORS else [None] * cnt
        self._n = (_i64 * cnt)(*self.sizes)
        self._ld = (_i64 * cnt)(*[max(1, n) for n in self.sizes])
        sz = _sz()
        _check(_lib.evd_batched_workspace_size(cnt, self._n, self.job, ctypes.byref(sz)), "evd_batched_workspace_size")
        self.ws_bytes = sz.value
        self.ws = torch.empty(max(sz.value, 256), dtype=torch.uint8, device=device)
        self._Ap = (_vp * cnt)(*[a.data_ptr() for a in self.A])
        self._wp = (_vp * cnt)(*[w.data_ptr() for w in self.w])
        self._Qp = (_vp * cnt)(*[(q.data_ptr() if q is not None else 0) for q in self.Q])

    def run(self, stream=None):
        _check(_lib.evd_syevd_batched(len(self.sizes), self._n, self._Ap, self._ld, self._wp, self._Qp, self._ld,
                                      self.job, _ptr(self.ws), self.ws_bytes, _stream_ptr(stream)),
               "evd_syevd_batched")


def batched_last_graph():
    return bool(_lib.evd_batched_last_graph())


def autotune(n, job="V", prec="fp64", cache_path=None):
    b, nb = _int(), _int()
    jb = EVD_VECTORS if job == "V" else EVD_VALUES
    pr = {"fp64": EVD_FP64, "split_bf16": EVD_SPLIT_BF16}.get(prec, prec)
    _check(_lib.evd_autotune(int(n), jb, pr, cache_path.encode() if cache_path else None, ctypes.byref(b),
                             ctypes.byref(nb)), "evd_autotune")
    return b.value, nb.value


# ---------------------------------------------------------------- instrumentation
def stats_enable(on=True):
    _lib.evd_stats_enable(1 if on else 0)


def stats_reset():
    _lib.evd_stats_reset()


def launch_count():
    return int(_lib.evd_launch_count())


def stats():
    """{category: (ms, flops, bytes, calls)} of everything recorded since the reset."""
    buf = ctypes.create_string_buffer(8192)
    _lib.evd_stats_categories(buf, 8192)
    out = {}
    for name in [c for c in buf.value.decode().split("\n") if c]:
        ms, fl, by, ca = _dbl(), _dbl(), _dbl(), _i64()
        _check(_lib.evd_stats_query(name.encode(), ctypes.byref(ms), ctypes.byref(fl), ctypes.byref(by),
                                    ctypes.byref(ca)), "evd_stats_query")
        out[name] = (ms.value, fl.value, by.value, ca.value)
    return out
