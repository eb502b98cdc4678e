"""Pins of the oracle's homotopy continuation (the Discussion's extension: lambda in
Q steps, each step re-expressed in the eigenbasis of the previous one) against the
mathematics:

- one stage is the plain solve;
- where the direct iteration from the identity fails (lambda beyond its convergence
  domain), two and four stages reach the eigen-decomposition: every column is an
  eigenvector (explicit residual), the eigenvalues are numpy's, and each pair is the
  one continued from e_i along [0, lambda] (numpy's eigen-decomposition followed in
  small steps), for a symmetric and an unsymmetric Delta;
- different stage counts reach the same eigenpairs."""
import numpy as np
import pytest

from test_oracle_ramp import _continued_eigvecs


def _sym_case(n=64, seed=1):
    rng = np.random.Generator(np.random.PCG64(seed))
    th = np.arange(n, dtype=float)
    S = rng.standard_normal((n, n)) / np.sqrt(n)
    return th, (S + S.T) / np.sqrt(2)


def test_one_stage_is_the_plain_solve(ora):
    th, D = _sym_case(24, 3)
    A, E, info = ora.homotopy(th, D, 0.3, 1, tol=1e-13)
    A0, E0, i0 = ora.solve_full(th, D, 0.3, tol=1e-13)
    assert info["status"] == "OK" and i0["status"] == "OK"
    # one stage solves (diag(theta) + lam Delta - diag(theta)) / lam = Delta up to rounding
    assert np.max(np.abs(E - E0)) < 1e-13 and np.max(np.abs(A - A0)) < 1e-13


@pytest.mark.parametrize("kind", ["sym", "unsym"])
def test_stages_reach_what_the_direct_iteration_misses(ora, kind):
    if kind == "sym":
        th, D = _sym_case()
        lam = 1.2
    else:
        # symmetric part plus a small antisymmetric one: unsymmetric, real spectrum
        rng = np.random.Generator(np.random.PCG64(4))
        n = 40
        th = np.arange(n, dtype=float)
        S = rng.standard_normal((n, n)) / np.sqrt(n)
        K = rng.standard_normal((n, n)) / np.sqrt(n)
        D = (S + S.T) / np.sqrt(2) + 0.2 * (K - K.T) / np.sqrt(2)
        lam = 1.5
    _, _, i0 = ora.solve_full(th, D, lam, tol=1e-12, max_iter=2000)
    assert i0["status"] != "OK"
    M = np.diag(th) + lam * D
    V, w = _continued_eigvecs(th, D, lam, steps=3000)
    res = {}
    for Q in (2, 4):
        A, E, info = ora.homotopy(th, D, lam, Q, tol=1e-13, max_iter=2000)
        assert info["status"] == "OK", (Q, info)
        assert np.allclose(np.diag(A), 1.0, atol=1e-15)
        R = M @ A - A * E[None, :]
        assert np.max(np.linalg.norm(R, axis=0) / np.linalg.norm(A, axis=0)) < 1e-10
        assert np.max(np.abs(E - w)) < 1e-9
        assert np.max(np.linalg.norm(A - V, axis=0) / np.linalg.norm(V, axis=0)) < 1e-8
        ev = np.sort(np.linalg.eigvals(M).real)
        assert np.max(np.abs(np.sort(E) - ev)) < 1e-9
        res[Q] = (A, E)
    assert np.max(np.abs(res[2][1] - res[4][1])) < 1e-10
