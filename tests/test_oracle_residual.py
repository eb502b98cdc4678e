"""Pins of the oracle's residual and its normalisation.

The stopping rule of every solve, and the "residual <= 1e-10" of the metric, is the
normalised eigen-residual of the plain eigen-equation M a = E a (Sec. II.A):

    rho_i = ||M a_i - E_i a_i||_2 / (s ||a_i||_2),
    s     = max_j |theta_j| + |lambda| max_j sum_k |Delta_jk|   (a bound of ||M||_inf).

None of the expected values below is computed by retyping that formula on matrices:
they are closed forms of the 2 x 2 example of Sec. II.E (the residual of the k-th
iterate follows from the scalar map x -> lambda (x^2 - 1)) and 3 x 3 cases worked
out by hand, each written as the arithmetic of the hand calculation.  The 3 x 3
perturbation is unsymmetric with different largest row and column sums, the
largest |theta| belongs to a negative theta and lambda is negative, so a residual
that drops s, sums columns instead of rows, drops |lambda|, takes the largest
signed theta or forgets ||a_i|| fails one of them (tests/test_oracle_mutants.py
plants each of these mistakes)."""
import numpy as np
import pytest

TH3 = np.array([0.0, 1.0, -3.0])
D3 = np.array([[0.0, 2.0, -1.0],
               [0.5, 1.0, 0.0],
               [-4.0, 0.0, 0.25]])
LAM3 = -0.1
# row sums of |Delta|: 3, 1.5, 4.25 (column sums 4.5, 3, 1.25); max |theta| = 3
S3 = 3.0 + 0.1 * 4.25


@pytest.mark.parametrize("lam", [0.3, -0.45, 0.8])
def test_two_by_two_at_identity(ora, lam):
    """A = I: E = theta (diag Delta = 0) and R = lambda Delta, so each column has
    ||R|| = |lambda|, ||a|| = 1 and s = max|theta| + |lambda| * 1 = 1 + |lambda|."""
    th = np.array([0.0, 1.0])
    D = np.array([[0.0, 1.0], [1.0, 0.0]])
    rmax, rho = ora.residual(th, D, lam, np.eye(2), th)
    want = abs(lam) / (1.0 + abs(lam))
    assert np.allclose(rho, [want, want], rtol=1e-14, atol=0)
    assert rmax == pytest.approx(want, rel=1e-14)


@pytest.mark.parametrize("lam", [0.3, -0.6])
def test_two_by_two_iterates(ora, lam):
    """The k-th iterate of Sec. II.E is [[1, -x_k], [x_k, 1]] (column form) with
    x_{k+1} = lambda (x_k^2 - 1), x_0 = 0, and E = (lambda x_k, 1 - lambda x_k).
    Working M A - A diag(E) out by hand leaves one nonzero entry per column, both
    equal to lambda + x_k - lambda x_k^2 = x_k - x_{k+1}; ||a_i|| = sqrt(1 + x_k^2)."""
    th = np.array([0.0, 1.0])
    D = np.array([[0.0, 1.0], [1.0, 0.0]])
    x = 0.0
    for _ in range(8):
        xn = lam * (x * x - 1.0)
        A = np.array([[1.0, -x], [x, 1.0]])
        E = np.array([lam * x, 1.0 - lam * x])
        _, rho = ora.residual(th, D, lam, A, E)
        want = abs(x - xn) / ((1.0 + abs(lam)) * np.sqrt(1.0 + x * x))
        # x_k - x_{k+1} cancels as the orbit converges: an absolute floor of FP64 rounding
        assert np.allclose(rho, [want, want], rtol=1e-12, atol=1e-15), (x, rho, want)
        x = xn


def test_three_by_three_at_identity(ora):
    """A = I, E = theta + lambda diag(Delta) = (0, 0.9, -3.025): R is lambda times
    the off-diagonal part of Delta, column norms 0.1 sqrt(0.5^2 + 4^2), 0.1 * 2,
    0.1 * 1, divided by s = 3 + 0.1 * 4.25 (the largest ROW sum of |Delta|)."""
    E = np.array([0.0, 0.9, -3.025])
    rmax, rho = ora.residual(TH3, D3, LAM3, np.eye(3), E)
    want = np.array([0.1 * np.sqrt(0.25 + 16.0), 0.2, 0.1]) / S3
    assert np.allclose(rho, want, rtol=1e-13, atol=0)
    assert rmax == pytest.approx(want[0], rel=1e-13)


def test_three_by_three_general_iterate(ora):
    """A non-unit column and an arbitrary E.  M = [[0, -0.2, 0.1], [-0.05, 0.9, 0],
    [0.4, 0, -3.025]]; column 0 of A is (1, 2, 0): M a = (-0.4, 1.75, 0.4), and with
    E_0 = 1, R_0 = (-1.4, -0.25, 0.4), ||a|| = sqrt(5).  Columns 1, 2 are e_1, e_2
    with E = 0.9, -3.025: R = (-0.2, 0, 0) and (0.1, 0, 0)."""
    A = np.array([[1.0, 0.0, 0.0], [2.0, 1.0, 0.0], [0.0, 0.0, 1.0]])
    E = np.array([1.0, 0.9, -3.025])
    _, rho = ora.residual(TH3, D3, LAM3, A, E)
    want = np.array([np.sqrt(1.4**2 + 0.25**2 + 0.4**2) / np.sqrt(5.0), 0.2, 0.1]) / S3
    assert np.allclose(rho, want, rtol=1e-13, atol=0)
    # the normalisation makes rho blind to the scale of a column (E fixed)
    A2 = A.copy()
    A2[:, 0] *= -3.5
    _, rho2 = ora.residual(TH3, D3, LAM3, A2, E)
    assert np.allclose(rho2, rho, rtol=1e-14, atol=0)


def test_complex_two_by_two(ora):
    """Hermitian Delta = [[0, i], [-i, 0]] with complex lambda = 0.3i: s uses |lambda|
    = 0.3, so s = 1.3.  At A = I, R = lambda Delta: ||R_i|| = 0.3.  With column 0 of
    A = (1, i) and E_0 = 0: M = [[0, -0.3], [0.3, 1]], R_0 = M a = (-0.3i, 0.3 + i),
    ||R_0||^2 = 0.09 + 0.09 + 1, ||a||^2 = 2."""
    th = np.array([0.0, 1.0], dtype=complex)
    D = np.array([[0.0, 1j], [-1j, 0.0]])
    lam = 0.3j
    _, rho = ora.residual(th, D, lam, np.eye(2, dtype=complex), th)
    assert np.allclose(rho, [0.3 / 1.3, 0.3 / 1.3], rtol=1e-14, atol=0)
    A = np.array([[1.0, 0.0], [1j, 1.0]])
    E = np.array([0.0, 1.0], dtype=complex)
    _, rho = ora.residual(th, D, lam, A, E)
    assert rho[0] == pytest.approx(np.sqrt(1.18) / (1.3 * np.sqrt(2.0)), rel=1e-13)


def test_solve_reports_the_same_residual(ora):
    """The full solve stops on this residual: with no map application allowed it
    returns A_0 = I of the 2 x 2 and the residual |lambda| / (1 + |lambda|)."""
    th = np.array([0.0, 1.0])
    D = np.array([[0.0, 1.0], [1.0, 0.0]])
    A, E, info = ora.solve_full(th, D, 0.4, tol=1e-300, max_iter=0)
    assert info["status"] == "MAXITER"
    assert np.array_equal(A, np.eye(2))
    assert info["residual"] == pytest.approx(0.4 / 1.4, rel=1e-14)


def test_dominant_residual_at_start(ora):
    """The CSR single-vector oracle at z = e_{n*} (no map application): n* = 1 (the
    largest theta), y = Delta e_1 = (2, 1, 0), E = 1 + lambda * 1 = 0.9 and the
    residual (lambda * 2, 0, 0) has norm 0.2; s = 3.425 as above."""
    row_ptr = np.array([0, 2, 4, 6], dtype=np.int32)
    col_idx = np.array([1, 2, 0, 1, 0, 2], dtype=np.int32)
    vals = np.array([2.0, -1.0, 0.5, 1.0, -4.0, 0.25], dtype=np.float32)
    z, E, info = ora.solve_dominant_csr(TH3, row_ptr, col_idx, vals, LAM3, tol=1e-300,
                                        max_iter=0)
    assert info["status"] == "MAXITER"
    assert E == pytest.approx(0.9, rel=1e-15)
    assert np.array_equal(z, [0.0, 1.0, 0.0])
    assert info["residual"] == pytest.approx(0.2 / S3, rel=1e-14)
