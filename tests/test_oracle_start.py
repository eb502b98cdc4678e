"""Pins of the oracle's generalised start (the closing remark of Sec. II.H: approximate
eigenvectors from another method, refined by the map's final convergent steps):

- a start at the fixed point stops at once (k = 0) with that fixed point;
- a start is rescaled to the chart a_i = 1, so any nonzero multiple gives the same
  iteration;
- on the Supplement's 3x3 example at lambda = -0.48 the second line, which the
  autonomous iteration from e_2 does not reach, is reached from the continued
  eigenvector perturbed by 1 % (numpy's eigen-decomposition followed along
  [0, lambda]); full form and CSR single-vector form;
- a start whose chart entry is zero is rejected."""
import numpy as np

from test_oracle_ramp import D3, TH3, _continued_eigvecs


def test_start_at_fixed_point_stops_at_once(ora):
    rng = np.random.Generator(np.random.PCG64(21))
    n = 30
    th = np.arange(n, dtype=float)
    D = rng.standard_normal((n, n)) / np.sqrt(n)
    A, E, info = ora.solve_full(th, D, 0.1, tol=1e-14)
    assert info["status"] == "OK" and info["iters"] > 3
    A2, E2, i2 = ora.solve_full(th, D, 0.1, tol=1e-13, start=A)
    assert i2["status"] == "OK" and i2["iters"] == 0
    assert np.array_equal(A2, A) and np.array_equal(E2, E)


def test_start_is_rescaled_to_the_chart(ora):
    rng = np.random.Generator(np.random.PCG64(22))
    n = 12
    th = np.arange(n, dtype=float)
    D = rng.standard_normal((n, n)) / np.sqrt(n)
    S = np.eye(n) + 0.01 * rng.standard_normal((n, n))
    A1, E1, _ = ora.solve_full(th, D, 0.1, tol=1e-14, start=S)
    A2, E2, _ = ora.solve_full(th, D, 0.1, tol=1e-14, start=S * 4.0)   # exact scaling
    assert np.array_equal(A1, A2) and np.array_equal(E1, E2)
    bad = S.copy()
    bad[3, 3] = 0.0
    _, _, info = ora.solve_full(th, D, 0.1, start=bad)
    assert info["status"] == "ARG"


def test_start_reaches_second_line_of_the_3x3_example(ora):
    lam = -0.48
    V, w = _continued_eigvecs(TH3, D3, lam)
    rng = np.random.Generator(np.random.PCG64(5))
    s = V[:, 1] * (1.0 + 0.01 * rng.standard_normal(3))
    _, _, i0 = ora.solve_full(TH3, D3, lam, tol=1e-12, max_iter=3000, cols=[1])
    assert i0["status"] != "OK"
    A, E, info = ora.solve_full(TH3, D3, lam, tol=1e-13, max_iter=3000, cols=[1],
                                start=s[:, None])
    assert info["status"] == "OK"
    assert np.max(np.abs(A[:, 0] - V[:, 1])) < 1e-9 and abs(E[0] - w[1]) < 1e-10
    rp = np.array([0, 2, 4, 6], dtype=np.int32)
    ci = np.array([1, 2, 0, 2, 0, 1], dtype=np.int32)
    va = np.array([1, 2, 1, 3, 2, 3], dtype=np.float32)
    z, Ez, iz = ora.solve_dominant_csr(TH3, rp, ci, va, lam, nstar=1, tol=1e-13,
                                       max_iter=3000, start=s)
    assert iz["status"] == "OK"
    assert np.max(np.abs(z - V[:, 1])) < 1e-9 and abs(Ez - w[1]) < 1e-10
    zero = s.copy()
    zero[1] = 0.0
    _, _, ib = ora.solve_dominant_csr(TH3, rp, ci, va, lam, nstar=1, start=zero)
    assert ib["status"] == "ARG"
