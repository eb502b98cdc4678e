"""GPU parity of dpt_solve_homotopy (the Discussion's homotopy continuation: lambda
in Q steps, each solved in the eigenbasis of the previous one) against the
oracle's homotopy, through the C ABI: symmetric and unsymmetric problems where the
direct iteration from the identity fails, mixed and plain-FP64 stage solves,
several stage counts, a size with ragged 128-wide tiles, one stage equal to the
direct solve, and the argument errors."""
import numpy as np
import pytest

from gpu_util import EIG_RTOL, VEC_TOL, eig_err, to_np, vec_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dpt():
    from paper_2002_12872_gb300 import build, dpt
    build.build()
    return dpt


def _sym(n, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    th = np.arange(n, dtype=float)
    S = rng.standard_normal((n, n)) / np.sqrt(n)
    return th, (S + S.T) / np.sqrt(2)


def _unsym(n, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    th = np.arange(n, dtype=float)
    S = rng.standard_normal((n, n)) / np.sqrt(n)
    K = rng.standard_normal((n, n)) / np.sqrt(n)
    return th, (S + S.T) / np.sqrt(2) + 0.2 * (K - K.T) / np.sqrt(2)


def _dev(th, D):
    from paper_2002_12872_gb300 import dpt as d
    return torch.tensor(th, device="cuda"), d.colmajor_tensor(D, "cuda")


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
@pytest.mark.parametrize("case", [("sym", 64, 1, 1.2, 2, True), ("sym", 64, 1, 1.2, 4, True),
                                  ("unsym", 40, 4, 1.5, 2, True),
                                  ("sym", 300, 7, 2.5, 3, False)])
def test_homotopy_parity(ora, dpt, prec, case):
    kind, n, seed, lam, Q, direct_fails = case
    th, D = (_sym if kind == "sym" else _unsym)(n, seed)
    Ao, Eo, io = ora.homotopy(th, D, lam, Q, tol=1e-13, max_iter=2000)
    assert io["status"] == "OK"
    thd, Dd = _dev(th, D)
    if direct_fails:   # the direct iteration from the identity does not reach it
        _, _, i0 = dpt.solve_full(thd, Dd, lam, prec=prec, max_iter=2000, check=False)
        assert i0["status"] != "OK"
    A, E, info = dpt.solve_homotopy(thd, Dd, lam, Q, prec=prec, tol=1e-13, max_iter=2000)
    assert info["status"] == "OK"
    assert eig_err(to_np(E), Eo) <= EIG_RTOL
    assert vec_err(to_np(A), Ao) <= VEC_TOL
    assert np.array_equal(np.diag(to_np(A)), np.ones(n))


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_one_stage_is_the_direct_solve(ora, dpt, prec):
    th, D = _sym(200, 3)
    thd, Dd = _dev(th, D)
    A1, E1, i1 = dpt.solve_homotopy(thd, Dd, 0.3, 1, prec=prec, tol=1e-13)
    Ao, Eo, io = ora.solve_full(th, D, 0.3, tol=1e-14)
    assert i1["status"] == "OK" and io["status"] == "OK"
    assert eig_err(to_np(E1), Eo) <= EIG_RTOL and vec_err(to_np(A1), Ao) <= VEC_TOL


def test_homotopy_argument_errors(dpt):
    th, D = _sym(32, 2)
    thd, Dd = _dev(th, D)
    for Q in (0, 2000):
        _, _, info = dpt.solve_homotopy(thd, Dd, 0.5, Q, check=False)
        assert info["status"] == "ERR_ARG"
    _, _, info = dpt.solve_homotopy(th, D, 0.5, 2, check=False)      # host arrays
    assert info["status"] == "ERR_UNSUPPORTED"
