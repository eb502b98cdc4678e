"""Pins of the oracle's non-autonomous iteration (the Supplement's explicit 3x3
example: step k applies the map at lambda (1 - alpha^k), starting from the
unperturbed vector) against what the paper states and what the mathematics fixes:

- the early iterates in closed form (step 0 is the identity map, step 1 the map at
  lambda (1 - alpha)), which catches an off-by-one in the exponent;
- on the printed 3x3 example at lambda = -0.48 the autonomous iteration of the second
  line diverges while the ramped one converges (the effect the Supplement reports),
  to the eigenvector continued from e_2 along [0, lambda] (computed by numpy's
  eigen-decomposition in small steps, matched by overlap), both in the full form and
  in the single-vector CSR form;
- where the autonomous iteration converges, the ramp reaches the same fixed point."""
import numpy as np
import pytest

TH3 = np.array([0.0, 1.0, 3.0])
D3 = np.array([[0.0, 1.0, 2.0], [1.0, 0.0, 3.0], [2.0, 3.0, 0.0]])


def _continued_eigvecs(th, D, lam, steps=4000):
    """Eigenvectors continued from e_i at lambda = 0 by small steps along the real
    segment [0, lam], each matched to the previous one by overlap; unit-diagonal
    chart (a_i[i] = 1).  Returns (V, w)."""
    n = len(th)
    V = np.eye(n)
    w = np.array(th, dtype=float)
    for t in np.linspace(0.0, lam, steps)[1:]:
        ev, U = np.linalg.eig(np.diag(th) + t * D)
        Un = U / np.linalg.norm(U, axis=0)
        Vn = np.zeros_like(V)
        wn = np.zeros(n)
        for i in range(n):
            j = int(np.argmax(np.abs(Un.T @ (V[:, i] / np.linalg.norm(V[:, i])))))
            Vn[:, i] = np.real(U[:, j] / U[i, j])
            wn[i] = np.real(ev[j])
        V, w = Vn, wn
    return V, w


def test_ramp_early_iterates_closed_form(ora):
    """max_iter = k returns the iterate A_k: with the ramp A_1 = I (step 0 applies
    strength 0) and A_2 = I + lambda (1 - alpha) G o offdiag(Delta)."""
    rng = np.random.Generator(np.random.PCG64(3))
    n, lam, alpha = 7, 0.07, 0.6
    th = np.arange(n, dtype=float) + rng.uniform(-0.2, 0.2, n)
    D = rng.standard_normal((n, n))
    A1, _, i1 = ora.solve_full(th, D, lam, tol=1e-300, max_iter=1, ramp_alpha=alpha)
    assert i1["iters"] == 1
    assert np.array_equal(A1, np.eye(n))
    A2, _, _ = ora.solve_full(th, D, lam, tol=1e-300, max_iter=2, ramp_alpha=alpha)
    G = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if i != j:
                G[j, i] = 1.0 / (th[i] - th[j])
    want = np.eye(n) + lam * (1 - alpha) * G * (D - np.diag(np.diag(D)))
    assert np.max(np.abs(A2 - want)) < 1e-15
    # the autonomous iteration's A_1 is already the map at full strength
    Aa, _, _ = ora.solve_full(th, D, lam, tol=1e-300, max_iter=1)
    assert np.max(np.abs(Aa - (np.eye(n) + lam * G * (D - np.diag(np.diag(D)))))) < 1e-15


def test_ramp_rescues_second_line_of_the_3x3_example(ora):
    lam = -0.48
    V, w = _continued_eigvecs(TH3, D3, lam)
    # autonomous: the second line does not converge from e_2
    _, _, io = ora.solve_full(TH3, D3, lam, tol=1e-12, max_iter=3000, cols=[1])
    assert io["status"] != "OK"
    for alpha in (0.9, 0.95):
        A, E, ir = ora.solve_full(TH3, D3, lam, tol=1e-13, max_iter=3000, cols=[1],
                                  ramp_alpha=alpha)
        assert ir["status"] == "OK", ir
        assert np.max(np.abs(A[:, 0] - V[:, 1])) < 1e-9
        assert abs(E[0] - w[1]) < 1e-10
        # E is an eigenvalue of M and A[:, 0] its eigenvector
        M = np.diag(TH3) + lam * D3
        assert np.linalg.norm(M @ A[:, 0] - E[0] * A[:, 0]) < 1e-11
    # the single-vector CSR form agrees
    rp = np.array([0, 2, 4, 6], dtype=np.int32)
    ci = np.array([1, 2, 0, 2, 0, 1], dtype=np.int32)
    va = np.array([1, 2, 1, 3, 2, 3], dtype=np.float32)
    z, Ez, iz = ora.solve_dominant_csr(TH3, rp, ci, va, lam, nstar=1, tol=1e-13,
                                       max_iter=3000, ramp_alpha=0.9)
    assert iz["status"] == "OK"
    assert np.max(np.abs(z - V[:, 1])) < 1e-9 and abs(Ez - w[1]) < 1e-10
    _, _, iz0 = ora.solve_dominant_csr(TH3, rp, ci, va, lam, nstar=1, tol=1e-12,
                                       max_iter=3000)
    assert iz0["status"] != "OK"


def test_ramp_reaches_the_autonomous_fixed_point(ora):
    rng = np.random.Generator(np.random.PCG64(9))
    n = 40
    th = np.arange(n, dtype=float)
    S = rng.standard_normal((n, n)) / np.sqrt(n)
    D = (S + S.T) / 2
    A0, E0, i0 = ora.solve_full(th, D, 0.2, tol=1e-14)
    A1, E1, i1 = ora.solve_full(th, D, 0.2, tol=1e-14, ramp_alpha=0.7)
    assert i0["status"] == "OK" and i1["status"] == "OK"
    assert i1["iters"] > i0["iters"]
    assert np.max(np.abs(E1 - E0)) < 1e-12 and np.max(np.abs(A1 - A0)) < 1e-11


def test_ramp_alpha_out_of_range_rejected(ora):
    for a in (-0.1, 1.0, 2.0):
        _, _, info = ora.solve_full(TH3, D3, 0.1, ramp_alpha=a)
        assert info["status"] == "ARG"
