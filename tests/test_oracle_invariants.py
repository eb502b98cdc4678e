"""Pins of the oracle against invariants of the eigenproblem M a = E a with
M = diag(theta) + lam Delta (Sec. II.A-B), brute-force diagonalisation on tiny n,
the Banach bound of Sec. II.C, and the residual identity of the column update."""
import numpy as np
import pytest

from paper_2002_12872_gb300 import inputs


def _match_columns(theta, lam, D, w, V):
    """Assign each eigenpair (w_p, V[:, p]) to the chart index i where |v_i|/||v||
    is largest (greedy on the overlap with e_i), then rescale so v_i = 1."""
    n = len(theta)
    order = np.argsort(-np.abs(V).max(axis=0))
    taken, Wm, Vm = set(), np.zeros(n, dtype=w.dtype), np.zeros((n, n), dtype=V.dtype)
    for p in order:
        v = V[:, p]
        cand = [i for i in np.argsort(-np.abs(v)) if i not in taken]
        i = cand[0]
        taken.add(i)
        Wm[i] = w[p]
        Vm[:, i] = v / v[i]
    return Wm, Vm


def _unit_cols(A):
    return A / np.linalg.norm(A, axis=0)


@pytest.mark.parametrize("n", [3, 5, 8, 12])
def test_symmetric_vs_jacobi(ora, n):
    cfg = inputs.full_symmetric(n=n, lam=0.05)
    th, D, lam = cfg["theta"], cfg["delta"], cfg["lam"]
    A, E, info = ora.solve_full(th, D, lam, tol=1e-14)
    assert info["status"] == "OK"
    M = np.diag(th) + lam * D
    w, V = ora.jacobi_sym(M)
    Wm, Vm = _match_columns(th, lam, D, w, V)
    assert np.abs(E - Wm).max() < 1e-12
    assert np.abs(_unit_cols(A) - _unit_cols(Vm)).max() < 1e-10


def test_jacobi_against_library(ora):
    rng = np.random.Generator(np.random.PCG64(4))
    S = rng.standard_normal((9, 9))
    S = S + S.T
    w, V = ora.jacobi_sym(S)
    assert np.allclose(np.sort(w), np.linalg.eigvalsh(S), atol=1e-12)
    assert np.allclose(V @ np.diag(w) @ V.T, S, atol=1e-12)
    assert np.allclose(V.T @ V, np.eye(9), atol=1e-13)


@pytest.mark.parametrize("n", [4, 7])
def test_hermitian_vs_jacobi(ora, n):
    rng = inputs.rng_for(5, 99)
    th = np.arange(n, dtype=float)
    D = inputs.hermitian_gaussian(n, 1.0 / n, rng)
    lam = 0.06
    A, E, info = ora.solve_full(th.astype(complex), D, lam, tol=1e-14)
    assert info["status"] == "OK"
    M = np.diag(th) + lam * D
    w, V = ora.jacobi_herm(M)
    Wm, Vm = _match_columns(th, lam, D, w.astype(complex), V)
    assert np.abs(E - Wm).max() < 1e-12
    assert np.abs(_unit_cols(A) - _unit_cols(Vm)).max() < 1e-10
    # Hermitian M: normalised eigenvectors are orthonormal
    Q = _unit_cols(A)
    assert np.abs(Q.conj().T @ Q - np.eye(n)).max() < 1e-10


def test_unsymmetric_vs_library_eig(ora):
    cfg = inputs.full_unsymmetric(n=10)
    th, D, lam = cfg["theta"], cfg["delta"], cfg["lam"]
    A, E, info = ora.solve_full(th, D, lam, tol=1e-14)
    assert info["status"] == "OK"
    w, V = np.linalg.eig(np.diag(th) + lam * D)   # test-only library cross-check
    Wm, Vm = _match_columns(th, lam, D, w, V)
    assert np.abs(E - Wm.real).max() < 1e-12
    assert np.abs(_unit_cols(A) - _unit_cols(Vm.real)).max() < 1e-10


@pytest.mark.parametrize("which", ["sym", "unsym"])
def test_trace_and_residual(ora, which):
    cfg = inputs.full_symmetric(n=64) if which == "sym" else inputs.full_unsymmetric(n=64)
    th, D, lam = cfg["theta"], cfg["delta"], cfg["lam"]
    A, E, info = ora.solve_full(th, D, lam, tol=1e-13)
    assert info["status"] == "OK"
    tr = th.sum() + lam * np.trace(D)
    assert abs(E.sum() - tr) <= 1e-12 * abs(tr)
    rmax, rho = ora.residual(th, D, lam, A, E)
    assert rmax <= 1e-13
    if which == "sym":
        Q = _unit_cols(A)
        assert np.abs(Q.T @ Q - np.eye(64)).max() < 1e-10


def test_residual_identity(ora):
    """For any iterate A with E_i = theta_i + lam (Delta A)_ii, the explicit residual
    M A - A diag(E) equals (theta_i - theta_j)(F(A) - A) entrywise (and is 0 on the
    diagonal): the update of Eq. (dyn) moves a_i by the residual divided by the gap."""
    cfg = inputs.full_unsymmetric(n=20)
    th, D, lam = cfg["theta"], cfg["delta"], cfg["lam"]
    A, _ = ora.iterate(th, D, lam, 2)
    An, E = ora.step(th, D, lam, A)
    R = (np.diag(th) + lam * D) @ A - A * E[None, :]
    gap = th[None, :] - th[:, None]
    assert np.abs(R - gap * (An - A)).max() < 1e-14


def test_epstein_nesbet_same_fixed_point(ora):
    cfg = inputs.full_unsymmetric(n=40)
    th, D, lam = cfg["theta"], cfg["delta"], cfg["lam"]
    A1, E1, i1 = ora.solve_full(th, D, lam, tol=1e-14)
    A2, E2, i2 = ora.solve_full(th, D, lam, tol=1e-14, epstein_nesbet=True)
    assert i1["status"] == "OK" and i2["status"] == "OK"
    assert np.abs(E1 - E2).max() < 1e-12
    assert np.abs(A1 - A2).max() < 1e-11


def test_degenerate_theta_rejected(ora):
    th = np.array([0.0, 1.0, 1.0])
    D = np.ones((3, 3))
    _, _, info = ora.solve_full(th, D, 0.01)
    assert info["status"] == "DEGENERATE"


def test_column_subset_equals_bundle(ora):
    cfg = inputs.full_unsymmetric(n=50)
    th, D, lam = cfg["theta"], cfg["delta"], cfg["lam"]
    A, E, _ = ora.solve_full(th, D, lam, tol=1e-14)
    cols = [3, 17, 49]
    As, Es, info = ora.solve_full(th, D, lam, tol=1e-14, cols=cols)
    assert np.abs(As - A[:, cols]).max() < 1e-13 and np.abs(Es - E[cols]).max() < 1e-13


def test_banach_ball(ora):
    """Sec. II.C: with ||Delta|| = 1 and |lam| ||theta|| <= 3 - 2 sqrt(2) (~0.17), F maps
    the ball ||A - I|| <= sqrt(2) into itself and contracts: the iterates stay in it
    and converge."""
    rng = np.random.Generator(np.random.PCG64(77))
    n = 12
    th = np.sort(rng.uniform(0, 6, n))
    D = rng.standard_normal((n, n))
    D /= np.linalg.norm(D, 2)
    gap = th[:, None] - th[None, :]           # paper theta_n^m = 1/(eps_n - eps_m)
    Th = np.zeros((n, n))
    off = ~np.eye(n, dtype=bool)
    Th[off] = 1.0 / gap[off]
    lam = 0.99 * (3 - 2 * np.sqrt(2)) / np.linalg.norm(Th, 2)
    A = np.eye(n)
    for k in range(60):
        assert np.linalg.norm(A - np.eye(n), 2) <= np.sqrt(2)
        A, _ = ora.step(th, D, lam, A)
    _, _, info = ora.solve_full(th, D, lam, tol=1e-13)
    assert info["status"] == "OK"
