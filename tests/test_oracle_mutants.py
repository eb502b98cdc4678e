"""The oracle's pins must catch plausible mistakes.  Each mutant below is a copy
of the oracle's C source with one planted error (a dropped term, a flipped sign,
a transposed operand, a missing factor), compiled on the CPU into a temporary
library.  Every mutant must fail at least one of the pins that the real oracle
passes: the exact 2x2 iterates (Sec. II.E), the printed 3x3 polynomials
(Supplement E), the trace and right-eigenvector residual of an unsymmetric
problem (M a = E a, Sec. II.A), and the hand-computed normalised residuals of
tests/test_oracle_residual.py (full and single-vector forms)."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ORA = os.path.join(os.path.dirname(HERE), "oracle")

MUTANTS = {
    "drop_d_a_term": ("an[j] = lam_map * g * (p[j] - d * a[j]);", "an[j] = lam_map * g * (p[j]);"),
    "flip_gap_sign": ("const T g = 1.0 / (theta[i] - theta[j]);",
                      "const T g = 1.0 / (theta[j] - theta[i]);"),
    "transpose_delta": ("for (int64_t j = 0; j < n; ++j) p[j] += dk[j] * akc;",
                        "for (int64_t j = 0; j < n; ++j) p[j] += delta[k + j * n] * akc;"),
    "eigenvalue_without_lambda": ("E[c] = theta[i] + lambda * d;", "E[c] = theta[i] + d;"),
    "diagonal_not_pinned": ("an[j] = 1;  ", "an[j] = a[j] + lambda * d;  "),
    "ramp_exponent_off_by_one": (
        "const T lam_map = ramp_alpha > 0.0 ? lambda * (1.0 - pw) : lambda;\n      pw *= ramp_alpha;",
        "pw *= ramp_alpha;\n      const T lam_map = ramp_alpha > 0.0 ? lambda * (1.0 - pw) : lambda;"),
    "ramp_in_eigenvalue": ("E[c] = theta[i] + lambda * d;", "E[c] = theta[i] + lam_map * d;"),
    # the normalisation of the residual (the stopping rule and the metric's bar)
    "residual_without_scale": ("const double v = sqrt(rr) / (s * sqrt(aa));",
                               "const double v = sqrt(rr) / sqrt(aa);"),
    "residual_without_norm_a": ("const double v = sqrt(rr) / (s * sqrt(aa));",
                                "const double v = sqrt(rr) / s;"),
    "scale_column_sums": ("for (int64_t k = 0; k < n; ++k) row += ABS(delta[j + k * n]);",
                          "for (int64_t k = 0; k < n; ++k) row += ABS(delta[k + j * n]);"),
    "scale_without_lambda": ("return tmax + ABS(lambda) * rmax;", "return tmax + rmax;"),
    "scale_signed_lambda": ("return tmax + ABS(lambda) * rmax;",
                            "return tmax + creal(lambda) * rmax;"),
    "scale_signed_theta": ("if (ABS(theta[j]) > tmax) tmax = ABS(theta[j]);",
                           "if (creal(theta[j]) > tmax) tmax = creal(theta[j]);"),
    "dominant_scale_without_lambda": ("const double s = tmax + fabs(lambda) * rmax;",
                                      "const double s = tmax + rmax;", "dpt_oracle.c"),
    "dominant_residual_without_scale": ("rho = sqrt(rr) / (s * sqrt(zz));",
                                        "rho = sqrt(rr) / sqrt(zz);", "dpt_oracle.c"),
}


def _build(tmp, name, old, new, target="dpt_oracle_body.inc"):
    d = os.path.join(tmp, name)
    os.makedirs(d)
    for f in ("dpt_oracle.c", "dpt_oracle_body.inc", "dpt_oracle.h"):
        shutil.copy(os.path.join(ORA, f), d)
    body = open(os.path.join(d, target)).read()
    assert old in body, name
    open(os.path.join(d, target), "w").write(body.replace(old, new))
    so = os.path.join(d, "lib.so")
    subprocess.run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", so,
                    os.path.join(d, "dpt_oracle.c"), "-lm"], check=True,
                   capture_output=True)
    lib = ctypes.CDLL(so)
    P, i64, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double
    lib.ora_step_r.argtypes = [i64, P, P, dbl, P, P, P]
    lib.ora_solve_full_r.argtypes = [i64, P, P, dbl, i64, P, dbl, i64, ctypes.c_int, dbl,
                                     P, P, P, P]
    lib.ora_residual_r.argtypes = [i64, P, P, dbl, P, P, P]
    lib.ora_residual_r.restype = dbl
    lib.ora_solve_dominant_csr.argtypes = [i64, P, P, P, P, i64, dbl, dbl, i64, dbl, P, P,
                                           P, P]
    return lib


class _Info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int64), ("residual", ctypes.c_double),
                ("status", ctypes.c_int64)]


def _residual_pins_pass(lib):
    """The hand-computed residuals of tests/test_oracle_residual.py: the 3 x 3 at
    A = I (s = 3 + 0.1 * 4.25 from the largest row sum, |theta| and |lambda|) and
    with a non-unit column, and the single-vector oracle at its start."""
    p = lambda x: x.ctypes.data_as(ctypes.c_void_p)
    th = np.ascontiguousarray([0.0, 1.0, -3.0])
    D = np.asfortranarray([[0.0, 2.0, -1.0], [0.5, 1.0, 0.0], [-4.0, 0.0, 0.25]])
    s3 = 3.0 + 0.1 * 4.25
    for A, E, want in (
            (np.eye(3), [0.0, 0.9, -3.025], [0.1 * np.sqrt(16.25), 0.2, 0.1]),
            ([[1.0, 0.0, 0.0], [2.0, 1.0, 0.0], [0.0, 0.0, 1.0]], [1.0, 0.9, -3.025],
             [np.sqrt(1.4**2 + 0.25**2 + 0.4**2) / np.sqrt(5.0), 0.2, 0.1])):
        A = np.asfortranarray(A, float)
        E = np.ascontiguousarray(E, float)
        rho = np.zeros(3)
        lib.ora_residual_r(3, p(th), p(D), -0.1, p(A), p(E), p(rho))
        if not np.allclose(rho, np.array(want) / s3, rtol=1e-13, atol=0):
            return False
    row_ptr = np.array([0, 2, 4, 6], dtype=np.int32)
    col_idx = np.array([1, 2, 0, 1, 0, 2], dtype=np.int32)
    vals = np.array([2.0, -1.0, 0.5, 1.0, -4.0, 0.25], dtype=np.float32)
    z, Eo, info = np.zeros(3), np.zeros(1), _Info()
    lib.ora_solve_dominant_csr(3, p(th), p(row_ptr), p(col_idx), p(vals), -1, -0.1, 1e-300, 0,
                               0.0, None, p(z), p(Eo), ctypes.cast(ctypes.pointer(info),
                                                                   ctypes.c_void_p))
    return bool(abs(info.residual - 0.2 / s3) <= 1e-14 * (0.2 / s3))


def _solve_ramp(lib, th, D, lam, alpha, max_iter):
    """(A_k, E) returned by the ramped full solve after max_iter map applications."""
    n = len(th)
    th = np.ascontiguousarray(th, float)
    D = np.asfortranarray(D, float)
    A = np.zeros((n, n), order="F")
    E = np.zeros(n)
    info = ctypes.create_string_buffer(64)   # iterations, residual, status (unused here)
    p = lambda x: x.ctypes.data_as(ctypes.c_void_p)
    lib.ora_solve_full_r(n, p(th), p(D), lam, n, None, 1e-300, max_iter, 0, alpha, None,
                         p(A), p(E), ctypes.cast(info, ctypes.c_void_p))
    return A, E


def _step(lib, th, D, lam, A):
    n = len(th)
    th = np.ascontiguousarray(th, float)
    D = np.asfortranarray(D, float)
    A = np.asfortranarray(A, float)
    An = np.zeros((n, n), order="F")
    E = np.zeros(n)
    p = lambda x: x.ctypes.data_as(ctypes.c_void_p)
    lib.ora_step_r(n, p(th), p(D), lam, p(A), p(An), p(E))
    return An, E


def _pins_pass(lib):
    if not _residual_pins_pass(lib):
        return False
    # 0. the non-autonomous iteration's A_2 in closed form: I + lam (1 - alpha) G o Delta
    #    (zero-diagonal Delta), and E of the iterate read out at the full lambda
    th0 = np.array([0.0, 1.0, 3.0])
    D0 = np.array([[0.0, 1.0, 2.0], [1.0, 0.0, 3.0], [2.0, 3.0, 0.0]])
    G0 = np.array([[0.0 if i == j else 1.0 / (th0[i] - th0[j]) for i in range(3)]
                   for j in range(3)])
    A2, E2 = _solve_ramp(lib, th0, D0, 0.1, 0.5, 2)
    if not np.allclose(A2, np.eye(3) + 0.1 * 0.5 * G0 * D0, atol=1e-15, rtol=0):
        return False
    if not np.allclose(E2, th0 + 0.1 * np.diag(D0 @ A2), atol=1e-15, rtol=0):
        return False
    # 1. exact 2x2 iterates, column form [[1, -x], [x, 1]]
    th2, D2 = np.array([0.0, 1.0]), np.array([[0.0, 1.0], [1.0, 0.0]])
    A, x, lam = np.eye(2), 0.0, 0.3
    for _ in range(10):
        if not np.allclose(A, [[1.0, -x], [x, 1.0]], atol=1e-13):
            return False
        A, _ = _step(lib, th2, D2, lam, A)
        x = lam * (x * x - 1.0)
    # 2. trace invariant on a random unsymmetric 6x6 at the fixed point
    rng = np.random.Generator(np.random.PCG64(1))
    th = np.arange(6.0) + rng.uniform(-0.2, 0.2, 6)
    D = rng.uniform(-1, 1, (6, 6))
    A = np.eye(6)
    for _ in range(200):
        A, E = _step(lib, th, D, 0.05, A)
    _, E = _step(lib, th, D, 0.05, A)
    if not abs(E.sum() - (th.sum() + 0.05 * np.trace(D))) < 1e-10:
        return False
    # 2b. the columns are right eigenvectors: M A = A diag(E), M = diag(theta) + lam Delta
    M = np.diag(th) + 0.05 * D
    if not np.abs(M @ A - A * E[None, :]).max() < 1e-10:
        return False
    # 3. printed 3x3 polynomial P_1 at the multipliers of line 1
    terms = []
    for line in open(os.path.join(HERE, "golden", "poly_3x3.txt")):
        if not line.startswith("#") and line.strip():
            n, a, b, c = map(int, line.split())
            if n == 1:
                terms.append((a, b, c))
    th3 = np.array([0.0, 1.0, 3.0])
    D3 = np.array([[0.0, 1.0, 2.0], [1.0, 0.0, 3.0], [2.0, 3.0, 0.0]])
    lam = 0.2
    A = np.eye(3)
    for _ in range(300):
        A, _ = _step(lib, th3, D3, lam, A)
    if not np.all(np.isfinite(A)):
        return False
    J = np.zeros((2, 2))
    for q, k in enumerate((1, 2)):
        Ap, Am = A.copy(), A.copy()
        Ap[k, 0] += 1e-6
        Am[k, 0] -= 1e-6
        J[:, q] = (_step(lib, th3, D3, lam, Ap)[0][[1, 2], 0]
                   - _step(lib, th3, D3, lam, Am)[0][[1, 2], 0]) / 2e-6
    for mu in np.linalg.eigvals(J):
        v = sum(c * lam**a * mu**b for a, b, c in terms)
        s = sum(abs(c * lam**a * mu**b) for a, b, c in terms)
        if abs(v) / s > 1e-8:
            return False
    return True


def test_unmutated_copy_passes(tmp_path):
    lib = _build(str(tmp_path), "original", "an[j] = 1;", "an[j] = 1;")
    assert _pins_pass(lib)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    lib = _build(str(tmp_path), name, *MUTANTS[name])
    assert not _pins_pass(lib), name
