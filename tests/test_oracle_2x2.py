"""Pins of the oracle against the explicit 2x2 example of Sec. II.E (Eq. (2by2))
and the general 2x2 structure of Supplement E.

M = [[0, 0], [0, 1]] + lam [[0, 1], [1, 0]].  The paper prints the iterates in its
row convention as A^(k) = [[1, f^k(0)], [-f^k(0), 1]] with f(x) = lam (x^2 - 1);
in the column convention used here that is [[1, -x_k], [x_k, 1]].  The stable fixed
point is x* = eps_-/lam with eps_+- = (1 +- sqrt(1 + 4 lam^2))/2; it is attracting
for real lam in (-sqrt(3)/2, sqrt(3)/2) and for lam = i t with |t| < 1/2, and the
error decays like |1 - sqrt(1 + 4 lam^2)|^k.
"""
import numpy as np
import pytest

TH = np.array([0.0, 1.0])
DL = np.array([[0.0, 1.0], [1.0, 0.0]])


def eps(lam):
    r = np.sqrt(1 + 4 * lam * lam + 0j)
    return (1 - r) / 2, (1 + r) / 2


@pytest.mark.parametrize("lam", [0.3, -0.6, 0.8, 0.9, 1.3])
def test_iterates_follow_scalar_map(ora, lam):
    A = np.eye(2)
    x = 0.0
    for k in range(40):
        expect = np.array([[1.0, -x], [x, 1.0]])
        assert np.allclose(A, expect, rtol=0, atol=1e-14 * (1 + abs(x)) * (k + 1)), k
        A, E = ora.step(TH, DL, lam, A)
        x = lam * (x * x - 1.0)
        if abs(x) > 1e6:
            break


@pytest.mark.parametrize("lam", [0.05, 0.3, 0.5, -0.7, 0.8])
def test_fixed_point_and_eigenvalues(ora, lam):
    A, E, info = ora.solve_full(TH, DL, lam, tol=1e-14, max_iter=5000)
    assert info["status"] == "OK"
    em, ep = eps(lam)
    assert abs(E[0] - em.real) < 1e-13 and abs(E[1] - ep.real) < 1e-13
    xs = em.real / lam
    assert np.allclose(A, [[1.0, -xs], [xs, 1.0]], atol=1e-12)


@pytest.mark.parametrize("lam", [0.9, -0.9, 1.2])
def test_flip_bifurcation_outside_domain(ora, lam):
    # beyond sqrt(3)/2 the fixed point is repelling: no false convergence
    A, E, info = ora.solve_full(TH, DL, lam, tol=1e-12, max_iter=3000)
    assert info["status"] in ("MAXITER", "DIVERGED")


def test_just_inside_flip_boundary(ora):
    A, E, info = ora.solve_full(TH, DL, 0.84, tol=1e-12, max_iter=20000)
    assert info["status"] == "OK"


@pytest.mark.parametrize("t,ok", [(0.3, True), (0.45, True), (0.55, False), (0.8, False)])
def test_imaginary_axis(ora, t, ok):
    lam = 1j * t
    A, E, info = ora.solve_full(TH.astype(complex), DL.astype(complex), lam, tol=1e-14,
                                max_iter=20000)
    assert (info["status"] == "OK") == ok
    if ok:
        em, ep = eps(lam)
        assert abs(E[0] - em) < 1e-11 and abs(E[1] - ep) < 1e-11


@pytest.mark.parametrize("lam", [0.3, 0.5])
def test_convergence_rate(ora, lam):
    em, _ = eps(lam)
    xs = em.real / lam
    A = np.eye(2)
    errs = []
    for k in range(22):
        errs.append(abs(A[1, 0] - xs))
        A, _ = ora.step(TH, DL, lam, A)
    # asymptotic ratio; the sub-leading term decays like the square of the rate
    ratios = [errs[k + 1] / errs[k] for k in range(4, 21) if errs[k + 1] > 1e-10]
    expect = abs(1 - np.sqrt(1 + 4 * lam * lam))
    assert np.allclose(ratios[-3:], expect, rtol=1e-4)


def test_general_2x2_lines_share_domain(ora):
    """Supplement E: for any 2x2 D and Delta, both lines of A converge or fail
    together (their multipliers at the two eigenvector fixed points coincide)."""
    rng = np.random.Generator(np.random.PCG64(12872))
    agree = 0
    for trial in range(30):
        th = np.sort(rng.uniform(-1, 1, 2))
        if th[1] - th[0] < 0.2:
            continue
        D = rng.uniform(-1, 1, (2, 2))
        for lam in np.linspace(0.1, 2.0, 12):
            st = []
            for c in (0, 1):
                _, _, info = ora.solve_full(th, D, lam, tol=1e-11, max_iter=4000, cols=[c])
                st.append((info["status"] == "OK", info["iters"]))
            # exclude runs whose convergence was too slow to classify
            if any(ok and it > 3000 for ok, it in st):
                continue
            assert st[0][0] == st[1][0], (th, D, lam, st)
            agree += 1
    assert agree > 100
