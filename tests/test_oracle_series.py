"""Pins of the oracle against the Rayleigh-Schroedinger series (Sec. II.D,
Supplements B and C): D-PT contains the RS series, A_D^(k) = A_RS^(k) + O(lam^(k+1)),
the closed second-order forms, and the second-order eigenvalue correction."""
import numpy as np
import pytest


def _problem(n=8, seed=5, zero_diag=False):
    rng = np.random.Generator(np.random.PCG64(seed))
    theta = np.arange(n, dtype=float) + rng.uniform(-0.2, 0.2, n)
    D = rng.uniform(-1, 1, (n, n))
    if zero_diag:
        np.fill_diagonal(D, 0.0)
    return theta, D


def _G(theta):
    n = len(theta)
    gap = theta[None, :] - theta[:, None]  # theta_i - theta_j at (j, i)
    G = np.zeros((n, n))
    off = ~np.eye(n, dtype=bool)
    G[off] = 1.0 / gap[off]
    return G


def test_first_order_identical(ora):
    """F(I) = I + lam G o Delta is exactly the first-order RS partial sum."""
    theta, D = _problem()
    AD, _ = ora.iterate(theta, D, 0.1, 1)
    AR, _ = ora.rs_series(theta, D, 0.1, 1)
    assert np.abs(AD - AR).max() < 1e-16


@pytest.mark.parametrize("k", [2, 3, 4])
def test_dpt_contains_rs_series(ora, k):
    """||A_D^(k) - A_RS^(k)|| = O(lam^(k+1)): halving lam divides it by ~2^(k+1)."""
    theta, D = _problem()
    errs = []
    for lam in (0.02, 0.01, 0.005):
        AD, _ = ora.iterate(theta, D, lam, k)
        AR, _ = ora.rs_series(theta, D, lam, k)
        errs.append(np.linalg.norm(AD - AR))
    for a, b in zip(errs, errs[1:]):
        assert abs(np.log2(a / b) - (k + 1)) < 0.15, errs


def test_second_order_closed_forms(ora):
    """With diag(Delta) = 0 the map gives, in column form with B = G o Delta,
        A_RS^(2) = I + lam B + lam^2 G o (Delta B)
        A_D^(2)  = A_RS^(2) - lam^3 G o ( B diag(Delta B) ).
    The printed Sec. II.D form carries '+' on the lam^3 term; expanding Eq. (dyn)
    twice gives '-' (checked below: the '+' reading misses by 2 lam^3 |...|)."""
    theta, D = _problem(zero_diag=True)
    G = _G(theta)
    B = G * D
    DB = D @ B
    lam = 0.3
    ARS2 = np.eye(len(theta)) + lam * B + lam**2 * (G * DB)
    third = lam**3 * (G * (B * np.diag(DB)[None, :]))
    AD, _ = ora.iterate(theta, D, lam, 2)
    AR, _ = ora.rs_series(theta, D, lam, 2)
    assert np.allclose(AR, ARS2, rtol=0, atol=1e-14)
    assert np.allclose(AD, ARS2 - third, rtol=0, atol=1e-14)
    assert np.linalg.norm(AD - (ARS2 + third)) > 1e3 * 1e-14


def test_second_order_eigenvalues(ora):
    """E_i = theta_i + lam Delta_ii + lam^2 sum_{j!=i} Delta_ij Delta_ji/(theta_i - theta_j)
    + O(lam^3) (Supplement B: eps^(l) = (a^(l-1) Delta')_nn)."""
    theta, D = _problem(n=10, seed=9)
    G = _G(theta)
    second = np.einsum("ij,ji->i", D, G * D)   # sum_j Delta_ij G_ji Delta_ji
    errs_d, errs_r = [], []
    for lam in (0.02, 0.01, 0.005):
        _, E, info = ora.solve_full(theta, D, lam, tol=1e-15, max_iter=200)
        ref = theta + lam * np.diag(D) + lam**2 * second
        errs_d.append(np.abs(E - ref).max())
        _, ER = ora.rs_series(theta, D, lam, 2)
        errs_r.append(np.abs(ER - ref).max())
    for a, b in zip(errs_d, errs_d[1:]):
        assert abs(np.log2(a / b) - 3) < 0.2, errs_d
    assert max(errs_r) < 1e-13


def test_rs_partial_sums_converge_to_dpt_limit(ora):
    theta, D = _problem(n=6, seed=3)
    lam = 0.05
    A, E, info = ora.solve_full(theta, D, lam, tol=1e-15)
    AR, ER = ora.rs_series(theta, D, lam, 30)
    assert np.abs(AR - A).max() < 1e-12 and np.abs(ER - E).max() < 1e-12
