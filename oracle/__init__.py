"""CPU oracle for dynamical perturbation theory (arXiv:2002.12872).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The CUDA
product path never imports it; the two share no code.

The arithmetic lives in plain C (``dpt_oracle.c``: FP64 / complex128, plain
loops, built with gcc); this module only builds the shared library and marshals
NumPy arrays.  All matrices cross the boundary in column-major order.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_SOURCES = ("dpt_oracle.c", "dpt_oracle_body.inc", "dpt_oracle.h")

OK, ERR_ARG, ERR_DEGENERATE, ERR_MAXITER, ERR_DIVERGED = 0, -1, -2, -3, -4
STATUS_NAMES = {0: "OK", -1: "ARG", -2: "DEGENERATE", -3: "MAXITER", -4: "DIVERGED"}


class _Info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int64), ("residual", ctypes.c_double),
                ("status", ctypes.c_int64)]


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (OpenMP when available)."""
    src = os.path.join(_HERE, "dpt_oracle.c")
    newest = max(os.path.getmtime(os.path.join(_HERE, s)) for s in _SOURCES)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
        return _LIB
    os.makedirs(_LIBDIR, exist_ok=True)
    tmp = _LIB + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, src, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i64, dbl, cint = ctypes.c_int64, ctypes.c_double, ctypes.c_int
        _lib.ora_step_r.argtypes = [i64, P, P, dbl, P, P, P]
        _lib.ora_residual_r.argtypes = [i64, P, P, dbl, P, P, P]
        _lib.ora_residual_r.restype = dbl
        _lib.ora_solve_full_r.argtypes = [i64, P, P, dbl, i64, P, dbl, i64, cint, dbl, P,
                                          P, P, ctypes.POINTER(_Info)]
        # complex lambda crosses the boundary as (re, im)
        _lib.ora_step_c.argtypes = [i64, P, P, dbl, dbl, P, P, P]
        _lib.ora_residual_c.argtypes = [i64, P, P, dbl, dbl, P, P, P]
        _lib.ora_residual_c.restype = dbl
        _lib.ora_solve_full_c.argtypes = [i64, P, P, dbl, dbl, i64, P, dbl, i64, cint, dbl, P,
                                          P, P, ctypes.POINTER(_Info)]
        _lib.ora_solve_dominant_csr.argtypes = [i64, P, P, P, P, i64, dbl, dbl, i64, dbl, P,
                                                P, P, ctypes.POINTER(_Info)]
        _lib.ora_rs_series_r.argtypes = [i64, P, P, dbl, i64, P, P]
        _lib.ora_jacobi_sym.argtypes = [i64, P, P, P]
    return _lib


def _c128(z):
    z = complex(z)
    return (z.real, z.imag)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _is_complex(*xs) -> bool:
    return any(np.iscomplexobj(x) for x in xs)


def _prep(theta, delta, lam):
    cplx = _is_complex(theta, delta, lam)
    dt = np.complex128 if cplx else np.float64
    theta = np.ascontiguousarray(theta, dtype=dt)
    delta = np.asfortranarray(delta, dtype=dt)
    n = theta.shape[0]
    if delta.shape != (n, n):
        raise ValueError("delta must be n x n")
    return cplx, dt, n, theta, delta


def step(theta, delta, lam, A):
    """One application of the map F of Eq. (dyn) (column form) to all columns.

    Returns (F(A), E) where E_i = theta_i + lam * (Delta A)_ii of the input A."""
    cplx, dt, n, theta, delta = _prep(theta, delta, lam)
    A = np.asfortranarray(A, dtype=dt)
    An = np.zeros((n, n), dtype=dt, order="F")
    E = np.zeros(n, dtype=dt)
    if cplx:
        st = lib().ora_step_c(n, _ptr(theta), _ptr(delta), *_c128(lam), _ptr(A),
                              _ptr(An), _ptr(E))
    else:
        st = lib().ora_step_r(n, _ptr(theta), _ptr(delta), float(lam), _ptr(A),
                              _ptr(An), _ptr(E))
    if st != OK:
        raise RuntimeError(f"ora_step failed: {STATUS_NAMES.get(st, st)}")
    return An, E


def iterate(theta, delta, lam, k):
    """A^(k) = F^k(I) and the read-out E of A^(k) (Sec. II.B)."""
    cplx, dt, n, theta, delta = _prep(theta, delta, lam)
    A = np.eye(n, dtype=dt, order="F")
    E = None
    for _ in range(k):
        A, E = step(theta, delta, lam, A)
    _, E = step(theta, delta, lam, A)
    return A, E


def residual(theta, delta, lam, A, E):
    """Explicit normalised residual ||M a_i - E_i a_i|| / (s ||a_i||) per column."""
    cplx, dt, n, theta, delta = _prep(theta, delta, lam)
    A = np.asfortranarray(A, dtype=dt)
    E = np.ascontiguousarray(E, dtype=dt)
    rho = np.zeros(n)
    if cplx:
        m = lib().ora_residual_c(n, _ptr(theta), _ptr(delta), *_c128(lam), _ptr(A),
                                 _ptr(E), _ptr(rho))
    else:
        m = lib().ora_residual_r(n, _ptr(theta), _ptr(delta), float(lam), _ptr(A),
                                 _ptr(E), _ptr(rho))
    return m, rho


def set_threads(n: int = 0) -> int:
    """Threads of the oracle's column-parallel loops (n <= 0: unchanged); returns
    the count in effect."""
    f = lib().ora_set_threads
    f.argtypes = [ctypes.c_int]
    f.restype = ctypes.c_int
    return int(f(int(n)))


def solve_full(theta, delta, lam, tol=1e-12, max_iter=1000, cols=None,
               epstein_nesbet=False, ramp_alpha=0.0, start=None):
    """Full-spectrum DPT solve from A_0 = I (Sec. II.B) on the listed columns.
    ramp_alpha in (0, 1) runs the non-autonomous iteration of the Supplement's 3x3
    example (step k at lambda (1 - alpha^k)); 0 is the autonomous map.  start
    (n x len(cols)) replaces A_0, each column scaled to its chart entry 1.

    Returns (A, E, info): A is n x len(cols), E has len(cols) entries, info is a
    dict with 'iters', 'residual', 'status' (name) and 'code'."""
    cplx, dt, n, theta, delta = _prep(theta, delta, lam)
    if cols is None:
        ncols, cptr = n, None
        colarr = None
    else:
        colarr = np.ascontiguousarray(cols, dtype=np.int64)
        ncols, cptr = colarr.shape[0], _ptr(colarr)
    A = np.zeros((n, ncols), dtype=dt, order="F")
    E = np.zeros(ncols, dtype=dt)
    info = _Info()
    args = (n, _ptr(theta), _ptr(delta))
    st_arr = None if start is None else np.asfortranarray(start, dtype=dt).reshape(n, ncols,
                                                                                 order="F")
    tail = (ncols, cptr, float(tol), int(max_iter), int(bool(epstein_nesbet)),
            float(ramp_alpha), None if st_arr is None else _ptr(st_arr), _ptr(A), _ptr(E),
            ctypes.byref(info))
    if cplx:
        st = lib().ora_solve_full_c(*args, *_c128(lam), *tail)
    else:
        st = lib().ora_solve_full_r(*args, float(lam), *tail)
    return A, E, {"iters": int(info.iters), "residual": float(info.residual),
                  "status": STATUS_NAMES.get(st, str(st)), "code": int(st)}


def solve_dominant_csr(theta, row_ptr, col_idx, vals, lam, nstar=-1, tol=1e-12,
                       max_iter=1000, ramp_alpha=0.0, start=None):
    """Dominant eigenvector by the single-vector map F_{n*} (Sec. II.H); ramp_alpha
    and start (n values) as for solve_full."""
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
    vals = np.ascontiguousarray(vals, dtype=np.float32)
    n = theta.shape[0]
    st_arr = None if start is None else np.ascontiguousarray(start, dtype=np.float64)
    z = np.zeros(n)
    E = np.zeros(1)
    info = _Info()
    st = lib().ora_solve_dominant_csr(n, _ptr(theta), _ptr(row_ptr), _ptr(col_idx),
                                      _ptr(vals), int(nstar), float(lam), float(tol),
                                      int(max_iter), float(ramp_alpha),
                                      None if start is None else _ptr(st_arr), _ptr(z), _ptr(E),
                                      ctypes.byref(info))
    return z, float(E[0]), {"iters": int(info.iters), "residual": float(info.residual),
                            "status": STATUS_NAMES.get(st, str(st)), "code": int(st)}


def homotopy(theta, delta, lam, stages, tol=1e-12, max_iter=1000):
    """Homotopy continuation of the Discussion (Sec. III): lambda is split into
    `stages` equal steps; after each step the problem is re-expressed in the
    eigenbasis just computed (the diagonal matrix of its eigenvalues becomes the
    next unperturbed matrix) and the map is iterated again from the identity.

    Reading of the basis change (the paper gives none): with V the accumulated
    right eigenvectors and W^T = V^{-1}, step q + 1 solves the matrix
        S = W^T M_{q+1} V = diag(E_q) + (lam/Q) Delta_q,
        Delta_q = (W^T (diag(theta) V + lambda_{q+1} Delta V) - diag(E_q)) Q / lam,
    i.e. the exact similarity transform of M_{q+1} = diag(theta) + lambda_{q+1}
    Delta, lambda_{q+1} = (q + 1) lam / Q, so errors of earlier stages are carried
    into the next stage's perturbation instead of being dropped.  Each stage solves
    S for its right eigenvectors A' (A'_ii = 1) and, except in the last stage, its
    transpose for the left ones B' (scaled so that B'^T A' = I); then V <- V A',
    W <- W B', followed by one Newton-Schulz step W <- W (2 I - V^T W) that
    restores W^T V = I to working precision.  Stage solves are solve_full (FP64,
    from the identity); the basis changes are plain matrix products.  Real only.

    Returns (A, E, info): A = V with each column scaled to its chart entry
    A[i, i] = 1 (the chart of the original problem), E the eigenvalues, info with
    'status' (of the first failing stage, else 'OK'), 'stages', 'iters' (summed)."""
    theta = np.asarray(theta, dtype=np.float64)
    D = np.asarray(delta, dtype=np.float64)
    n = theta.shape[0]
    Q = int(stages)
    if Q < 1:
        raise ValueError("stages must be >= 1")
    step_lam = float(lam) / Q
    V = np.eye(n)
    W = np.eye(n)
    Eq = theta.copy()
    iters = 0
    for q in range(Q):
        lam_next = (q + 1) * step_lam
        S = W.T @ (theta[:, None] * V + lam_next * (D @ V))
        Dq = (S - np.diag(Eq)) / step_lam
        Ar, E, ir = solve_full(Eq, Dq, step_lam, tol=tol, max_iter=max_iter)
        iters += ir["iters"]
        if ir["status"] != "OK":
            return V, Eq, {"status": ir["status"], "stages": q, "iters": iters}
        V = V @ Ar
        if q + 1 < Q:
            Bl, _, il = solve_full(Eq, Dq.T, step_lam, tol=tol, max_iter=max_iter)
            iters += il["iters"]
            if il["status"] != "OK":
                return V, Eq, {"status": il["status"], "stages": q, "iters": iters}
            Bl = Bl / np.sum(Bl * Ar, axis=0)[None, :]      # b_i^T a_i = 1
            W = W @ Bl
            W = W @ (2.0 * np.eye(n) - V.T @ W)             # Newton-Schulz: W^T V -> I
        Eq = np.real(E).astype(np.float64)
    V = V / np.diag(V)[None, :]
    return V, Eq, {"status": "OK", "stages": Q, "iters": iters}


def rs_series(theta, delta, lam, k):
    """Rayleigh-Schroedinger partial sums A_RS^(k), E_RS^(k) of Eq. (ARS-alpha)."""
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    delta = np.asfortranarray(delta, dtype=np.float64)
    n = theta.shape[0]
    A = np.zeros((n, n), order="F")
    E = np.zeros(n)
    st = lib().ora_rs_series_r(n, _ptr(theta), _ptr(delta), float(lam), int(k),
                               _ptr(A), _ptr(E))
    if st != OK:
        raise RuntimeError(f"ora_rs_series failed: {STATUS_NAMES.get(st, st)}")
    return A, E


def jacobi_sym(S):
    """Cyclic Jacobi eigen-decomposition of a real symmetric matrix: (w, V)."""
    S = np.asfortranarray(S, dtype=np.float64)
    n = S.shape[0]
    w = np.zeros(n)
    V = np.zeros((n, n), order="F")
    st = lib().ora_jacobi_sym(n, _ptr(S), _ptr(w), _ptr(V))
    if st != OK:
        raise RuntimeError(f"ora_jacobi_sym failed: {STATUS_NAMES.get(st, st)}")
    return w, V


def jacobi_herm(H):
    """Eigen-decomposition of a complex Hermitian matrix through the real
    symmetric embedding [[X, -Y], [Y, X]] of H = X + iY, whose spectrum is that of
    H with every eigenvalue doubled; each real eigenvector [u; v] maps to the
    eigenvector u + i v of H.  Returns (w, V) with n eigenpairs, one per doubled
    pair (the embedding vector with the larger norm of u + i v is kept)."""
    H = np.asarray(H, dtype=np.complex128)
    n = H.shape[0]
    X, Y = H.real, H.imag
    S = np.block([[X, -Y], [Y, X]])
    w2, V2 = jacobi_sym(S)
    order = np.argsort(w2)
    w2, V2 = w2[order], V2[:, order]
    w = w2[0::2].copy()
    V = np.zeros((n, n), dtype=np.complex128)
    for p in range(n):
        best = None
        for q in (2 * p, 2 * p + 1):
            u = V2[:n, q] + 1j * V2[n:, q]
            if best is None or np.linalg.norm(u) > np.linalg.norm(best):
                best = u
        V[:, p] = best / np.linalg.norm(best)
    return w, V
