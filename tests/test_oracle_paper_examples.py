"""Pins of the oracle against worked examples printed in the paper:
the 3x3 example and its polynomials P_n(lam, mu) (Supplement E), and the
delta-potential oscillator of Sec. II.F (qualitative claims)."""
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "poly_3x3.txt")
TH3 = np.array([0.0, 1.0, 3.0])
D3 = np.array([[0.0, 1.0, 2.0], [1.0, 0.0, 3.0], [2.0, 3.0, 0.0]])


def _poly():
    terms = {1: [], 2: [], 3: []}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        n, a, b, c = map(int, line.split())
        terms[n].append((a, b, c))
    return terms


def _jacobian(ora, th, D, lam, A, i, h=1e-6):
    """Jacobian of the single-vector map F_i on its free coordinates (m != i),
    by central differences of the oracle's map at the fixed point A[:, i]."""
    n = len(th)
    free = [m for m in range(n) if m != i]
    J = np.zeros((n - 1, n - 1))
    for q, k in enumerate(free):
        Ap, Am = A.copy(), A.copy()
        Ap[k, i] += h
        Am[k, i] -= h
        Fp, _ = ora.step(th, D, lam, Ap)
        Fm, _ = ora.step(th, D, lam, Am)
        J[:, q] = (Fp[free, i] - Fm[free, i]) / (2 * h)
    return J


@pytest.mark.parametrize("lam", [0.1, 0.2, -0.2, 0.3])
def test_3x3_multipliers_are_roots_of_printed_polynomials(ora, lam):
    terms = _poly()
    assert all(len(t) == 31 for t in terms.values())
    A, E, info = ora.solve_full(TH3, D3, lam, tol=1e-14, max_iter=5000)
    assert info["status"] == "OK"
    for n in (1, 2, 3):
        mus = np.linalg.eigvals(_jacobian(ora, TH3, D3, lam, A, n - 1))
        for mu in mus:
            v = sum(c * lam**a * mu**b for a, b, c in terms[n])
            s = sum(abs(c * lam**a * mu**b) for a, b, c in terms[n])
            assert abs(v) / s < 1e-8, (n, mu, abs(v) / s)
        # a point that is not a multiplier does not solve P_n
        mu = mus[0] + 0.05
        v = sum(c * lam**a * mu**b for a, b, c in terms[n])
        s = sum(abs(c * lam**a * mu**b) for a, b, c in terms[n])
        assert abs(v) / s > 1e-4


def _delta_potential(N=100):
    """The workload of Sec. II.F (paper_2002_12872_gb300.inputs.delta_oscillator)."""
    from paper_2002_12872_gb300 import inputs
    w = inputs.delta_oscillator(N)
    return w["theta"], w["delta"]


def test_delta_potential_lambda_1p5(ora):
    """Sec. II.F: at lam = 1.5 D-PT reaches in ~40 iterations a precision that the
    RS series needs over 70 orders for."""
    th, D = _delta_potential()
    lam = 1.5
    A, E, info = ora.solve_full(th, D, lam, tol=1e-14, max_iter=500)
    assert info["status"] == "OK" and info["iters"] <= 50
    target = 1e-12
    Ak = np.eye(len(th))
    kd = None
    for k in range(60):
        if np.linalg.norm(Ak - A) < target:
            kd = k
            break
        Ak, _ = ora.step(th, D, lam, Ak)
    kr = None
    for k in range(30, 100, 5):
        AR, _ = ora.rs_series(th, D, lam, k)
        if np.linalg.norm(AR - A) < target:
            kr = k
            break
    assert kd is not None and kd <= 45
    assert kr is None or kr >= kd + 10


def test_delta_potential_lambda_2p5(ora):
    """Sec. II.F: at lam = 2.5 the RS series diverges while D-PT still converges."""
    th, D = _delta_potential()
    lam = 2.5
    A, E, info = ora.solve_full(th, D, lam, tol=1e-13, max_iter=3000)
    assert info["status"] == "OK"
    errs = [np.linalg.norm(ora.rs_series(th, D, lam, k)[0] - A) for k in (20, 40, 60)]
    assert errs[0] < errs[1] < errs[2] and errs[2] > 1.0


def test_delta_oscillator_hermite_values():
    """phi_2n(0) of the workload against the closed form
    (-1)^n sqrt((2n)!) / (2^n n!) / pi^(1/4) (H_2n(0) = (-1)^n (2n)!/n!)."""
    import math
    from paper_2002_12872_gb300 import inputs
    w = inputs.delta_oscillator(12)
    phi = np.sqrt(np.diag(w["delta"])) * np.sign(w["delta"][0])
    for n in range(12):
        want = (-1) ** n * math.sqrt(math.factorial(2 * n)) / (2**n * math.factorial(n)) / np.pi**0.25
        assert abs(phi[n] - want) < 1e-14 * abs(want)
    assert np.array_equal(w["theta"], 2 * np.arange(12) + 0.5)
