"""Python binding of libdpt (C ABI declared in include/dpt.h).

Argument marshalling only: every step of a solve runs in the CUDA library.
Inputs may be torch tensors (CUDA or CPU) or NumPy arrays; matrices follow the
mathematical indexing Delta[j, k] and are handed to the library in column-major
order (a tensor whose strides are already (1, ld) is passed without a copy).
Outputs are returned as column-major views: A[:, i] is eigenvector i.

There is no CPU fallback: if libdpt.so is missing or the GPU is absent the
calls raise.
"""
from __future__ import annotations

import ctypes
from collections.abc import Sequence
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libdpt.so")

OK, PENDING = 0, 1
STATUS = {0: "OK", 1: "PENDING", -1: "ERR_ARG", -2: "ERR_DEGENERATE", -3: "ERR_MAXITER",
          -4: "ERR_DIVERGED", -5: "ERR_NOMEM", -6: "ERR_CUDA", -7: "ERR_TIMEOUT",
          -8: "ERR_UNSUPPORTED", -9: "ERR_TOO_LARGE", -10: "ERR_BUSY", -11: "ERR_CANCELLED"}
R64, C128 = 0, 1
PREC = {"fp64": 0, "mixed": 1, "bf16": 1}


class Options(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int32),
                ("prec", ctypes.c_int32), ("epstein_nesbet", ctypes.c_int32),
                ("graph_iters", ctypes.c_int32), ("max_slices", ctypes.c_int32),
                ("profile", ctypes.c_int32), ("slice_tol", ctypes.c_double),
                ("cta_pair", ctypes.c_int32), ("grouped_form", ctypes.c_int32),
                ("ramp_alpha", ctypes.c_double), ("start", ctypes.c_void_p),
                ("ld_start", ctypes.c_int64), ("certify", ctypes.c_int32),
                ("refine_tol", ctypes.c_double), ("pair_clusters", ctypes.c_int32)]


class Info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("slice_gemms", ctypes.c_int32),
                ("residual", ctypes.c_double), ("status", ctypes.c_int32),
                ("nstar", ctypes.c_int32), ("seconds", ctypes.c_double),
                ("launches", ctypes.c_int32), ("product_launches", ctypes.c_int32),
                ("product_ms", ctypes.c_double), ("cta_pair", ctypes.c_int32),
                ("grouped_form", ctypes.c_int32), ("fp64_iters", ctypes.c_int32),
                ("refined_cols", ctypes.c_int32)]

    def as_dict(self):
        return {"iters": self.iters, "slice_gemms": self.slice_gemms,
                "residual": self.residual, "status": STATUS.get(self.status, str(self.status)),
                "code": self.status, "nstar": self.nstar, "seconds": self.seconds,
                "launches": self.launches, "product_launches": self.product_launches,
                "product_ms": self.product_ms, "cta_pair": self.cta_pair,
                "grouped_form": self.grouped_form, "fp64_iters": self.fp64_iters,
                "refined_cols": self.refined_cols}


class InfoList(Sequence):
    """The per-problem dpt_info of a grouped solve as a read-only sequence of dicts,
    converted on access (building 20,000 dicts on every call would cost the host more
    than some solves take on the device)."""

    def __init__(self, arr):
        self._arr = arr

    def __len__(self):
        return len(self._arr)

    def __getitem__(self, k):
        if isinstance(k, slice):
            return [self._arr[q].as_dict() for q in range(*k.indices(len(self._arr)))]
        return self._arr[k].as_dict()


class ServerCfg(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_uint64), ("max_active", ctypes.c_int32),
                ("max_queue", ctypes.c_int32), ("opt", Options)]


class Problem(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("dtype", ctypes.c_int32),
                ("theta", ctypes.c_void_p), ("delta", ctypes.c_void_p),
                ("ld_delta", ctypes.c_int64), ("lam", ctypes.c_double),
                ("tol", ctypes.c_double), ("max_iter", ctypes.c_int32),
                ("A_out", ctypes.c_void_p), ("ld_a", ctypes.c_int64),
                ("E_out", ctypes.c_void_p)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("failed", ctypes.c_int64), ("cancelled", ctypes.c_int64),
                ("rejected", ctypes.c_int64), ("queued", ctypes.c_int32),
                ("active", ctypes.c_int32), ("max_queued", ctypes.c_int32),
                ("steps", ctypes.c_int64), ("hbm_budget", ctypes.c_uint64),
                ("hbm_in_use", ctypes.c_uint64), ("hbm_peak", ctypes.c_uint64),
                ("p50_s", ctypes.c_double), ("p99_s", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def lib() -> ctypes.CDLL:
    """Load libdpt.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build it with "
                "`python -m paper_2002_12872_gb300.build` (needs nvcc)")
        L = ctypes.CDLL(LIB_PATH)
        P, i64, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double
        L.dpt_options_default.argtypes = [ctypes.POINTER(Options)]
        L.dpt_options_default.restype = None
        L.dpt_status_string.argtypes = [ctypes.c_int]
        L.dpt_status_string.restype = ctypes.c_char_p
        L.dpt_solve_full.argtypes = [i64, ctypes.c_int, P, P, i64, dbl,
                                     ctypes.POINTER(Options), P, i64, P,
                                     ctypes.POINTER(Info), P]
        L.dpt_solve_full.restype = ctypes.c_int
        L.dpt_solve_dominant.argtypes = [i64, P, P, P, P, i64, dbl, ctypes.POINTER(Options),
                                         P, P, ctypes.POINTER(Info), P]
        L.dpt_solve_dominant.restype = ctypes.c_int
        L.dpt_solve_homotopy.argtypes = [i64, P, P, i64, dbl, ctypes.c_int32,
                                         ctypes.POINTER(Options), P, i64, P,
                                         ctypes.POINTER(Info), P]
        L.dpt_solve_homotopy.restype = ctypes.c_int
        L.dpt_rs_series.argtypes = [i64, P, P, i64, dbl, ctypes.c_int32, P, i64, P, P]
        L.dpt_rs_series.restype = ctypes.c_int
        L.dpt_solve_dominant_dense.argtypes = [i64, P, P, i64, i64, dbl,
                                               ctypes.POINTER(Options), P, P,
                                               ctypes.POINTER(Info), P]
        L.dpt_solve_dominant_dense.restype = ctypes.c_int
        L.dpt_solve_dominant_noalloc.argtypes = [i64, P, P, P, P, i64, dbl, dbl,
                                                 ctypes.c_int32, P, P, ctypes.POINTER(Info), P]
        L.dpt_solve_dominant_noalloc.restype = ctypes.c_int
        L.dpt_probe_gather.argtypes = [i64, P, P, P, P, ctypes.c_int32,
                                       ctypes.POINTER(ctypes.c_double), P]
        L.dpt_probe_gather.restype = ctypes.c_int
        L.dpt_solve_batched.argtypes = [i64, ctypes.c_int, P, P, P, P, P,
                                        ctypes.POINTER(Options), P, P, P, P, P]
        L.dpt_solve_batched.restype = ctypes.c_int
        L.dpt_tune_batched.argtypes = [i64, ctypes.c_int, P, P, P, P, P,
                                       ctypes.POINTER(Options), P, P, P, P, P, P]
        L.dpt_tune_batched.restype = ctypes.c_int
        L.dpt_server_cfg_default.argtypes = [ctypes.POINTER(ServerCfg)]
        L.dpt_server_cfg_default.restype = None
        L.dpt_server_create.argtypes = [ctypes.POINTER(ServerCfg), ctypes.POINTER(P)]
        L.dpt_server_create.restype = ctypes.c_int
        L.dpt_submit.argtypes = [P, ctypes.POINTER(Problem), ctypes.POINTER(i64)]
        L.dpt_submit.restype = ctypes.c_int
        L.dpt_poll.argtypes = [P, i64, ctypes.POINTER(Info)]
        L.dpt_poll.restype = ctypes.c_int
        L.dpt_wait.argtypes = [P, i64, dbl, ctypes.POINTER(Info)]
        L.dpt_wait.restype = ctypes.c_int
        L.dpt_cancel.argtypes = [P, i64]
        L.dpt_cancel.restype = ctypes.c_int
        L.dpt_server_stats_get.argtypes = [P, ctypes.POINTER(ServerStats)]
        L.dpt_server_stats_get.restype = ctypes.c_int
        L.dpt_server_destroy.argtypes = [P]
        L.dpt_server_destroy.restype = ctypes.c_int
        L.dpt_selftest_bounded_wait.argtypes = [dbl, P]
        L.dpt_selftest_bounded_wait.restype = ctypes.c_int
        L.dpt_workspace_bytes.argtypes = [i64, ctypes.c_int, ctypes.c_int]
        L.dpt_workspace_bytes.restype = i64
        L.dpt_release_workspace.argtypes = []
        L.dpt_release_workspace.restype = None
        _lib = L
    return _lib


def options(**kw) -> Options:
    o = Options()
    lib().dpt_options_default(ctypes.byref(o))
    for k, v in kw.items():
        if k == "prec" and isinstance(v, str):
            v = PREC[v]
        if v is not None:
            setattr(o, k, v)
    return o


def status_string(code: int) -> str:
    return lib().dpt_status_string(int(code)).decode()


# ---------------------------------------------------------------------------
# tensor helpers
# ---------------------------------------------------------------------------
def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _vec_ptr(x, dtype):
    """(pointer, keepalive) of a contiguous 1-D buffer."""
    if _is_torch(x):
        import torch
        t = x.to(dtype=getattr(torch, dtype)).contiguous()
        return t.data_ptr(), t
    a = np.ascontiguousarray(x, dtype=dtype)
    return a.ctypes.data, a


def _colmajor(x, cplx):
    """(pointer, ld, keepalive) of a matrix in column-major memory."""
    if _is_torch(x):
        import torch
        t = x.to(dtype=torch.complex128 if cplx else torch.float64)
        n0, n1 = t.shape
        if t.stride(0) == 1 and t.stride(1) >= n0:
            return t.data_ptr(), t.stride(1), t
        c = t.t().contiguous()           # memory = columns of t
        return c.data_ptr(), n0, c
    a = np.asfortranarray(x, dtype=np.complex128 if cplx else np.float64)
    return a.ctypes.data, a.shape[0], a


def _empty_colmajor(n, like, cplx):
    if _is_torch(like):
        import torch
        dt = torch.complex128 if cplx else torch.float64
        return torch.empty((n, n), dtype=dt, device=like.device).t()
    return np.empty((n, n), dtype=np.complex128 if cplx else np.float64, order="F")


def _empty_vec(n, like, cplx):
    if _is_torch(like):
        import torch
        dt = torch.complex128 if cplx else torch.float64
        return torch.empty((n,), dtype=dt, device=like.device)
    return np.empty(n, dtype=np.complex128 if cplx else np.float64)


def colmajor_tensor(a, device="cuda", pin=False):
    """Torch tensor with the values of the 2-D array `a` stored column-major
    (strides (1, n0)), the layout the library reads without a copy."""
    import torch
    t = torch.from_numpy(np.ascontiguousarray(np.asarray(a).T))   # rows = columns of a
    if pin:
        t = t.pin_memory()
    elif device is not None and str(device) != "cpu":
        t = t.to(device)
    return t.t()


def _ptr(x):
    return x.data_ptr() if _is_torch(x) else x.ctypes.data


def _stream_of(x, stream):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    if _is_torch(x) and x.is_cuda:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream(x.device).cuda_stream)
    return ctypes.c_void_p(0)


def _iscomplex(x) -> bool:
    if _is_torch(x):
        return x.is_complex()
    return np.iscomplexobj(x)


# ---------------------------------------------------------------------------
# entry points
# ---------------------------------------------------------------------------
def solve_full(theta, delta, lam, *, prec="mixed", tol=1e-12, max_iter=200,
               epstein_nesbet=False, graph_iters=None, max_slices=None, slice_tol=None,
               profile=False, cta_pair=None, ramp_alpha=None, start=None, certify=None,
               refine_tol=None, pair_clusters=None, A_out=None, E_out=None, stream=None,
               check=True):
    """All eigenpairs of M = diag(theta) + lam * Delta by the DPT map (dpt_solve_full).

    Returns (A, E, info): A[:, i] is eigenvector i with A[i, i] = 1 and
    E[i] = theta[i] + lam * (Delta A)[i, i].  With check=True a status other than
    OK raises RuntimeError (the outputs are still returned via the exception's
    ``result`` attribute)."""
    cplx = _iscomplex(delta)
    n = int(theta.shape[0])
    th_ptr, th_keep = _vec_ptr(theta, "float64")
    d_ptr, ldd, d_keep = _colmajor(delta, cplx)
    A = _empty_colmajor(n, delta, cplx) if A_out is None else A_out
    E = _empty_vec(n, delta, cplx) if E_out is None else E_out
    lda = A.stride(1) if _is_torch(A) else A.strides[1] // A.itemsize
    o = options(tol=tol, max_iter=max_iter, prec=prec, epstein_nesbet=int(bool(epstein_nesbet)),
                graph_iters=graph_iters, max_slices=max_slices, slice_tol=slice_tol,
                profile=int(bool(profile)), cta_pair=None if cta_pair is None else int(cta_pair),
                ramp_alpha=ramp_alpha, certify=None if certify is None else int(bool(certify)),
                refine_tol=refine_tol,
                pair_clusters=None if pair_clusters is None else int(pair_clusters))
    s_keep = None
    if start is not None:
        s_ptr, s_ld, s_keep = _colmajor(start, cplx)
        o.start, o.ld_start = s_ptr, s_ld
    info = Info()
    st = lib().dpt_solve_full(n, C128 if cplx else R64, th_ptr, d_ptr, ldd, float(lam),
                              ctypes.byref(o), _ptr(A), lda, _ptr(E), ctypes.byref(info),
                              _stream_of(delta, stream))
    res = (A, E, info.as_dict())
    if check and st != OK:
        err = RuntimeError(f"dpt_solve_full: {status_string(st)}")
        err.result = res
        raise err
    return res


class FullSolve:
    """dpt_solve_full with its arguments marshalled once, for repeated solves of the
    same buffers (the library reads theta and Delta and writes A and E in place on
    every call).  Keyword options are those of solve_full; the stream is fixed here
    (`stream`, else the current stream of Delta's device at construction).  solve()
    returns the info dict and raises RuntimeError on a status other than OK unless
    check=False."""

    def __init__(self, theta, delta, lam, *, A_out=None, E_out=None, stream=None, **opts):
        cplx = _iscomplex(delta)
        n = int(theta.shape[0])
        th_ptr, self._th_keep = _vec_ptr(theta, "float64")
        d_ptr, ldd, self._d_keep = _colmajor(delta, cplx)
        self.A = _empty_colmajor(n, delta, cplx) if A_out is None else A_out
        self.E = _empty_vec(n, delta, cplx) if E_out is None else E_out
        lda = self.A.stride(1) if _is_torch(self.A) else self.A.strides[1] // self.A.itemsize
        for k in ("epstein_nesbet", "profile", "certify"):
            if opts.get(k) is not None:
                opts[k] = int(bool(opts[k]))
        if opts.get("cta_pair") is not None:
            opts["cta_pair"] = int(opts["cta_pair"])
        self.opts = options(**opts)
        self._info = Info()
        self._fn = lib().dpt_solve_full
        self._args = (n, C128 if cplx else R64, th_ptr, d_ptr, ldd, float(lam),
                      ctypes.byref(self.opts), _ptr(self.A), lda, _ptr(self.E),
                      ctypes.byref(self._info), _stream_of(delta, stream))

    def solve(self, check=True):
        st = self._fn(*self._args)
        info = self._info.as_dict()
        if check and st != OK:
            raise RuntimeError(f"dpt_solve_full: {status_string(st)}")
        return info


def solve_homotopy(theta, delta, lam, stages, *, prec="mixed", tol=1e-12, max_iter=200,
                   graph_iters=None, max_slices=None, A_out=None, E_out=None, stream=None,
                   check=True):
    """Homotopy continuation (dpt_solve_homotopy): lambda in `stages` steps, each
    solved in the eigenbasis of the previous one.  Real CUDA tensors only.  Returns
    (A, E, info) as solve_full."""
    n = int(theta.shape[0])
    th_ptr, th_keep = _vec_ptr(theta, "float64")
    d_ptr, ldd, d_keep = _colmajor(delta, False)
    A = _empty_colmajor(n, delta, False) if A_out is None else A_out
    E = _empty_vec(n, delta, False) if E_out is None else E_out
    lda = A.stride(1) if _is_torch(A) else A.strides[1] // A.itemsize
    o = options(tol=tol, max_iter=max_iter, prec=prec, graph_iters=graph_iters,
                max_slices=max_slices)
    info = Info()
    st = lib().dpt_solve_homotopy(n, th_ptr, d_ptr, ldd, float(lam), int(stages),
                                  ctypes.byref(o), _ptr(A), lda, _ptr(E), ctypes.byref(info),
                                  _stream_of(delta, stream))
    res = (A, E, info.as_dict())
    if check and st != OK:
        err = RuntimeError(f"dpt_solve_homotopy: {status_string(st)}")
        err.result = res
        raise err
    return res


def rs_series(theta, delta, lam, order, *, A_out=None, E_out=None, stream=None, check=True):
    """Rayleigh-Schroedinger partial sums of the given order (dpt_rs_series, FP64):
    (A, E) with A = sum_l lam^l C^(l), E = theta + sum_l lam^l eps^(l).  Real CUDA
    tensors."""
    n = int(theta.shape[0])
    th_ptr, th_keep = _vec_ptr(theta, "float64")
    d_ptr, ldd, d_keep = _colmajor(delta, False)
    A = _empty_colmajor(n, delta, False) if A_out is None else A_out
    E = _empty_vec(n, delta, False) if E_out is None else E_out
    lda = A.stride(1) if _is_torch(A) else A.strides[1] // A.itemsize
    st = lib().dpt_rs_series(n, th_ptr, d_ptr, ldd, float(lam), int(order), _ptr(A), lda,
                             _ptr(E), _stream_of(delta, stream))
    if check and st != OK:
        raise RuntimeError(f"dpt_rs_series: {status_string(st)}")
    return A, E, STATUS.get(st, str(st))


class Batch:
    """A grouped solve (dpt_solve_batched) with its argument arrays built once.

    thetas / deltas: sequences of CUDA tensors, deltas column-major (e.g. from
    colmajor_tensor), all real or all complex128 (theta and lambda real).  The
    outputs A_outs / E_outs are allocated here unless given.  solve() can be called
    repeatedly; it writes the outputs in place."""

    def __init__(self, thetas, deltas, lams, *, A_outs=None, E_outs=None):
        import torch
        count = len(thetas)
        cplx = deltas[0].is_complex()
        want = torch.complex128 if cplx else torch.float64
        self.count, self.cplx = count, cplx
        ns, th, ds, ldd, keep = [], [], [], [], []
        for t, d in zip(thetas, deltas):
            if t.dtype != torch.float64:
                t = t.to(torch.float64)
            if d.dtype != want:
                d = d.to(want)
            n0 = d.shape[0]
            if not (d.stride(0) == 1 and d.stride(1) >= n0):
                d = d.t().contiguous().t()
            ns.append(int(t.shape[0]))
            th.append(t.data_ptr())
            ds.append(d.data_ptr())
            ldd.append(d.stride(1))
            keep.append((t, d))
        if A_outs is None:
            A_outs = [torch.empty((n, n), dtype=want, device=thetas[0].device).t() for n in ns]
        if E_outs is None:
            E_outs = [torch.empty(n, dtype=want, device=thetas[0].device) for n in ns]
        self.A_outs, self.E_outs, self._keep = A_outs, E_outs, keep
        P = ctypes.c_void_p
        self._n = (ctypes.c_int64 * count)(*ns)
        self._th = (P * count)(*th)
        self._d = (P * count)(*ds)
        self._ldd = (ctypes.c_int64 * count)(*ldd)
        self._lam = (ctypes.c_double * count)(*[float(x) for x in lams])
        self._a = (P * count)(*[a.data_ptr() for a in A_outs])
        self._lda = (ctypes.c_int64 * count)(*[a.stride(1) for a in A_outs])
        self._e = (P * count)(*[e.data_ptr() for e in E_outs])
        self._dev = thetas[0]
        self.form = None      # the tile shape tune() chose, used by solve() by default

    def tune(self, *, tol=1e-12, max_iter=200, graph_iters=None, max_slices=None,
             slice_tol=None, stream=None):
        """dpt_tune_batched: runs this group with each grouped product form and keeps
        the one with the least product time for later solve() calls.  Returns
        (best_form, {form: summed product ms, or -1})."""
        o = options(tol=tol, max_iter=max_iter, prec="mixed", graph_iters=graph_iters,
                    max_slices=max_slices, slice_tol=slice_tol)
        best = ctypes.c_int32(0)
        ms = (ctypes.c_double * 3)()
        st = lib().dpt_tune_batched(self.count, C128 if self.cplx else R64, self._n, self._th,
                                    self._d, self._ldd, self._lam, ctypes.byref(o), self._a,
                                    self._lda, self._e, ctypes.byref(best), ms,
                                    _stream_of(self._dev, stream))
        if st != OK:
            raise RuntimeError(f"dpt_tune_batched: {status_string(st)}")
        self.form = int(best.value)
        return self.form, {f: float(ms[f - 1]) for f in (1, 2, 3)}

    def solve(self, *, tol=1e-12, max_iter=200, graph_iters=None, max_slices=None,
              slice_tol=None, profile=False, form=None, stream=None, check=True):
        """Returns (A_outs, E_outs, infos).  form: the product form (grouped_form);
        by default the one tune() chose, if it ran."""
        if form is None:
            form = self.form
        infos = (Info * self.count)()
        o = options(tol=tol, max_iter=max_iter, prec="mixed", graph_iters=graph_iters,
                    max_slices=max_slices, slice_tol=slice_tol, profile=int(bool(profile)),
                    grouped_form=None if form is None else int(form))
        st = lib().dpt_solve_batched(self.count, C128 if self.cplx else R64, self._n, self._th,
                                     self._d, self._ldd, self._lam, ctypes.byref(o), self._a,
                                     self._lda, self._e, infos, _stream_of(self._dev, stream))
        res = (self.A_outs, self.E_outs, InfoList(infos))
        if check and st != OK:
            err = RuntimeError(f"dpt_solve_batched: {status_string(st)}")
            err.result = res
            raise err
        return res


def solve_batched(thetas, deltas, lams, *, tol=1e-12, max_iter=200, graph_iters=None,
                  max_slices=None, slice_tol=None, profile=False, form=None, A_outs=None,
                  E_outs=None, stream=None, check=True):
    """Grouped solve of independent problems (dpt_solve_batched), all real or all
    complex (complex128 deltas; theta and lambda real).

    thetas / deltas: sequences of CUDA tensors (deltas column-major, e.g. from
    colmajor_tensor).  Returns (As, Es, infos).  For repeated solves of the same
    problems build a Batch once and call its solve()."""
    return Batch(thetas, deltas, lams, A_outs=A_outs, E_outs=E_outs).solve(
        tol=tol, max_iter=max_iter, graph_iters=graph_iters, max_slices=max_slices,
        slice_tol=slice_tol, profile=profile, form=form, stream=stream, check=check)


def solve_dominant(theta, row_ptr, col_idx, vals, lam, *, nstar=-1, prec="mixed", tol=1e-12,
                   max_iter=200, graph_iters=None, profile=False, ramp_alpha=None, start=None,
                   z_out=None, stream=None, check=True):
    """Dominant eigenpair by the single-vector map (dpt_solve_dominant) for a CSR
    perturbation (int32 row_ptr / col_idx, FP32 values).  Returns (z, E, info)
    with z[n*] = 1."""
    n = int(theta.shape[0])
    th_ptr, k1 = _vec_ptr(theta, "float64")
    rp_ptr, k2 = _vec_ptr(row_ptr, "int32")
    ci_ptr, k3 = _vec_ptr(col_idx, "int32")
    va_ptr, k4 = _vec_ptr(vals, "float32")
    if z_out is None:
        z_out = _empty_vec(n, theta, False)
    E = np.zeros(1)
    o = options(tol=tol, max_iter=max_iter, prec=prec, graph_iters=graph_iters,
                profile=int(bool(profile)), ramp_alpha=ramp_alpha)
    s_keep = None
    if start is not None:
        o.start, s_keep = _vec_ptr(start, "float64")
    info = Info()
    st = lib().dpt_solve_dominant(n, th_ptr, rp_ptr, ci_ptr, va_ptr, int(nstar), float(lam),
                                  ctypes.byref(o), _ptr(z_out), E.ctypes.data,
                                  ctypes.byref(info), _stream_of(theta, stream))
    res = (z_out, float(E[0]), info.as_dict())
    if check and st != OK:
        err = RuntimeError(f"dpt_solve_dominant: {status_string(st)}")
        err.result = res
        raise err
    return res


def solve_dominant_dense(theta, delta, lam, *, nstar=-1, prec="mixed", tol=1e-12, max_iter=200,
                         graph_iters=None, profile=False, ramp_alpha=None, start=None,
                         z_out=None, stream=None, check=True):
    """Dominant eigenpair by the single-vector map with a dense FP64 perturbation
    (dpt_solve_dominant_dense, a GEMV per iteration).  Returns (z, E, info) with
    z[n*] = 1."""
    n = int(theta.shape[0])
    th_ptr, k1 = _vec_ptr(theta, "float64")
    d_ptr, ldd, k2 = _colmajor(delta, False)
    if z_out is None:
        z_out = _empty_vec(n, theta, False)
    E = np.zeros(1)
    o = options(tol=tol, max_iter=max_iter, prec=prec, graph_iters=graph_iters,
                profile=int(bool(profile)), ramp_alpha=ramp_alpha)
    s_keep = None
    if start is not None:
        o.start, s_keep = _vec_ptr(start, "float64")
    info = Info()
    st = lib().dpt_solve_dominant_dense(n, th_ptr, d_ptr, ldd, int(nstar), float(lam),
                                        ctypes.byref(o), _ptr(z_out), E.ctypes.data,
                                        ctypes.byref(info), _stream_of(theta, stream))
    res = (z_out, float(E[0]), info.as_dict())
    if check and st != OK:
        err = RuntimeError(f"dpt_solve_dominant_dense: {status_string(st)}")
        err.result = res
        raise err
    return res


def solve_dominant_noalloc(theta, row_ptr, col_idx, vals, lam, *, nstar=-1, tol=1e-12,
                           max_iter=200, z_out=None, stream=None, check=True):
    """dpt_solve_dominant_noalloc: the dominant solve for callers that cannot allocate
    device memory (fixed built-in scratch, n <= 262144, device inputs only)."""
    n = int(theta.shape[0])
    if z_out is None:
        z_out = _empty_vec(n, theta, False)
    E = np.zeros(1)
    info = Info()
    st = lib().dpt_solve_dominant_noalloc(n, _ptr(theta), _ptr(row_ptr), _ptr(col_idx),
                                          _ptr(vals), int(nstar), float(lam), float(tol),
                                          int(max_iter), _ptr(z_out), E.ctypes.data,
                                          ctypes.byref(info), _stream_of(theta, stream))
    res = (z_out, float(E[0]), info.as_dict())
    if check and st != OK:
        err = RuntimeError(f"dpt_solve_dominant_noalloc: {status_string(st)}")
        err.result = res
        raise err
    return res


def probe_gather(row_ptr, col_idx, z, reps=20, stream=None):
    """dpt_probe_gather: mean device time (ms) of one pass of the CSR form's access
    pattern without its arithmetic (index stream and 8-byte gathers of z), the
    ceiling of a pass on this GPU.  row_ptr / col_idx: int32 CUDA tensors; z: n
    float pairs (an (n, 2) float32 CUDA tensor)."""
    import torch
    n = int(row_ptr.shape[0]) - 1
    y = torch.empty(n, dtype=torch.float32, device=row_ptr.device)
    ms = ctypes.c_double(0.0)
    st = lib().dpt_probe_gather(n, _ptr(row_ptr), _ptr(col_idx), _ptr(z), _ptr(y), int(reps),
                                ctypes.byref(ms), _stream_of(row_ptr, stream))
    if st != OK:
        raise RuntimeError(f"dpt_probe_gather: {status_string(st)}")
    return float(ms.value)


def selftest_bounded_wait(seconds=0.5, stream=None):
    """dpt_selftest_bounded_wait: status name of a bounded device wait that is made to
    expire ('ERR_TIMEOUT' is the expected outcome)."""
    s = ctypes.c_void_p(0) if stream is None else ctypes.c_void_p(int(stream))
    return STATUS.get(lib().dpt_selftest_bounded_wait(float(seconds), s))


def workspace_bytes(n, complex_=False, prec="mixed"):
    """dpt_workspace_bytes: device workspace of one dpt_solve_full of size n (device
    inputs and outputs, default options); -1 for invalid arguments."""
    return int(lib().dpt_workspace_bytes(int(n), C128 if complex_ else R64, PREC[prec]))


def release_workspace():
    lib().dpt_release_workspace()


# ---------------------------------------------------------------------------
# solve server (continuous batching)
# ---------------------------------------------------------------------------
class ServerError(RuntimeError):
    def __init__(self, where, code):
        super().__init__(f"{where}: {status_string(code)}")
        self.code = code
        self.status = STATUS.get(code, str(code))


class Server:
    """dpt_server_*: requests of mixed sizes admitted against a device-memory
    budget, advanced together one map application per step, each retired at its
    own convergence.  Buffers handed to submit() are kept referenced here until
    the request's final status has been collected."""

    def __init__(self, *, hbm_budget=0, max_active=64, max_queue=65536, tol=None,
                 max_iter=None, max_slices=None, slice_tol=None, form=None):
        cfg = ServerCfg()
        lib().dpt_server_cfg_default(ctypes.byref(cfg))
        cfg.hbm_budget = int(hbm_budget)
        cfg.max_active = int(max_active)
        cfg.max_queue = int(max_queue)
        for k, v in (("tol", tol), ("max_iter", max_iter), ("max_slices", max_slices),
                     ("slice_tol", slice_tol), ("grouped_form", form)):
            if v is not None:
                setattr(cfg.opt, k, v)
        h = ctypes.c_void_p()
        st = lib().dpt_server_create(ctypes.byref(cfg), ctypes.byref(h))
        if st != OK:
            raise ServerError("dpt_server_create", st)
        self._h = h
        self._keep = {}

    def submit(self, theta, delta, lam, *, tol=0.0, max_iter=0, A_out=None, E_out=None):
        """Queue one problem; returns its request id.  Raises ServerError when the
        request is refused (ERR_ARG, ERR_TOO_LARGE, ERR_BUSY)."""
        cplx = _iscomplex(delta)
        n = int(theta.shape[0])
        th_ptr, th_keep = _vec_ptr(theta, "float64")
        d_ptr, ldd, d_keep = _colmajor(delta, cplx)
        A = _empty_colmajor(n, delta, cplx) if A_out is None else A_out
        E = _empty_vec(n, delta, cplx) if E_out is None else E_out
        lda = A.stride(1) if _is_torch(A) else A.strides[1] // A.itemsize
        p = Problem(n=n, dtype=C128 if cplx else R64, theta=th_ptr, delta=d_ptr, ld_delta=ldd,
                    lam=float(lam), tol=float(tol), max_iter=int(max_iter), A_out=_ptr(A),
                    ld_a=lda, E_out=_ptr(E))
        rid = ctypes.c_int64()
        st = lib().dpt_submit(self._h, ctypes.byref(p), ctypes.byref(rid))
        if st != OK:
            raise ServerError("dpt_submit", st)
        self._keep[rid.value] = (th_keep, d_keep, A, E)
        return rid.value

    def _final(self, rid, st, info):
        A, E = self._keep.pop(rid, (None, None, None, None))[2:]
        return A, E, info.as_dict()

    def poll(self, rid):
        """None while pending, else (A, E, info); info['status'] is the outcome."""
        info = Info()
        st = lib().dpt_poll(self._h, int(rid), ctypes.byref(info))
        if st == PENDING:
            return None
        if st == -1 and rid not in self._keep:
            raise ServerError("dpt_poll", st)
        return self._final(rid, st, info)

    def wait(self, rid, timeout=-1.0):
        """(A, E, info) once finished; None if the timeout expired first."""
        info = Info()
        st = lib().dpt_wait(self._h, int(rid), float(timeout), ctypes.byref(info))
        if st == PENDING:
            return None
        if st == -1 and rid not in self._keep:
            raise ServerError("dpt_wait", st)
        return self._final(rid, st, info)

    def cancel(self, rid):
        return STATUS.get(lib().dpt_cancel(self._h, int(rid)))

    def stats(self):
        s = ServerStats()
        lib().dpt_server_stats_get(self._h, ctypes.byref(s))
        return s.as_dict()

    def close(self):
        if self._h:
            lib().dpt_server_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
