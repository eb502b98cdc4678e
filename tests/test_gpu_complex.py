"""GPU parity of the complex mixed path against the complex128 oracle.

The complex product runs as the real GEMM of the interleaved 2n x 2n embedding of
Delta on the tensor cores; the control, iteration 0 and output stages carry the
complex diagonal and eigenvalues (Sec. II.B applies unchanged to complex M)."""
import numpy as np
import pytest

from gpu_util import EIG_RTOL, VEC_TOL, eig_err, to_np, vec_err
from paper_2002_12872_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dpt():
    from paper_2002_12872_gb300 import build, dpt
    build.build()
    return dpt


def _hermitian(n, seed, lam=0.05):
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.arange(n, dtype=float), inputs.hermitian_gaussian(n, 1.0 / n, rng), lam


def _general(n, seed, lam=0.05):
    rng = np.random.Generator(np.random.PCG64(seed))
    th = inputs.spaced_uniform(n, 0.5, rng)
    D = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(2.0 * n)
    return th, np.asfortranarray(D), lam


@pytest.mark.parametrize("n", [1, 2, 3, 31, 64, 65, 100, 129, 200, 300])
def test_complex_hermitian_full_parity(ora, dpt, n):
    th, D, lam = _hermitian(n, 900 + n)
    Ao, Eo, io = ora.solve_full(th, D, lam, tol=1e-13)
    assert io["status"] == "OK"
    A, E, info = dpt.solve_full(torch.tensor(th, device="cuda"), dpt.colmajor_tensor(D, "cuda"),
                                lam, prec="mixed")
    A, E = to_np(A), to_np(E)
    assert A.dtype == np.complex128 and E.dtype == np.complex128
    assert eig_err(E, Eo) <= EIG_RTOL, (n, info)
    assert vec_err(A, Ao) <= VEC_TOL, (n, info)
    assert np.allclose(np.diag(A), 1.0, rtol=0, atol=1e-12)
    # Hermitian M: real spectrum up to the iteration's own residual
    assert np.max(np.abs(E.imag)) <= 1e-10 * max(1.0, np.max(np.abs(E.real)))


@pytest.mark.parametrize("n", [5, 96, 257])
def test_complex_general_full_parity(ora, dpt, n):
    th, D, lam = _general(n, 1900 + n)
    Ao, Eo, io = ora.solve_full(th, D, lam, tol=1e-13)
    assert io["status"] == "OK"
    A, E, info = dpt.solve_full(torch.tensor(th, device="cuda"), dpt.colmajor_tensor(D, "cuda"),
                                lam, prec="mixed")
    assert eig_err(to_np(E), Eo) <= EIG_RTOL, (n, info)
    assert vec_err(to_np(A), Ao) <= VEC_TOL, (n, info)


def test_complex_host_buffers_match_device(dpt):
    th, D, lam = _hermitian(150, 77)
    A1, E1, _ = dpt.solve_full(th, D, lam, prec="mixed")            # numpy in, numpy out
    A2, E2, _ = dpt.solve_full(torch.tensor(th, device="cuda"), dpt.colmajor_tensor(D, "cuda"),
                               lam, prec="mixed")
    assert np.array_equal(A1, to_np(A2)) and np.array_equal(E1, to_np(E2))


def test_complex_mixed_agrees_with_fp64_path(dpt):
    th, D, lam = _hermitian(180, 91)
    Am, Em, _ = dpt.solve_full(th, D, lam, prec="mixed")
    Af, Ef, _ = dpt.solve_full(th, D, lam, prec="fp64")
    assert eig_err(Em, Ef) <= EIG_RTOL and vec_err(Am, Af) <= VEC_TOL


def test_complex_batched_uneven_parity(ora, dpt):
    sizes = [1, 2, 17, 64, 100, 129, 200, 333]
    probs = [_hermitian(n, 3000 + n, lam=0.02 + 0.01 * (q % 6)) for q, n in enumerate(sizes)]
    th = [torch.tensor(p[0], device="cuda") for p in probs]
    D = [dpt.colmajor_tensor(p[1], "cuda") for p in probs]
    As, Es, infos = dpt.solve_batched(th, D, [p[2] for p in probs])
    for (t, d, lam), A, E, inf in zip(probs, As, Es, infos):
        Ao, Eo, io = ora.solve_full(t, d, lam, tol=1e-13)
        assert inf["status"] == "OK" and io["status"] == "OK"
        assert eig_err(to_np(E), Eo) <= EIG_RTOL, (len(t), inf)
        assert vec_err(to_np(A), Ao) <= VEC_TOL, (len(t), inf)


def test_complex_served_size_sampled(ora, dpt):
    """A 2048-level problem of the served stream's recipe (theta equally spaced,
    Hermitian Delta of variance 1/n); sampled columns checked against the oracle."""
    th, D, lam = _hermitian(2048, 4096, lam=0.08)
    A, E, info = dpt.solve_full(torch.tensor(th, device="cuda"), dpt.colmajor_tensor(D, "cuda"),
                                lam, prec="mixed")
    A, E = to_np(A), to_np(E)
    cols = np.array([0, 1, 511, 1024, 1500, 2046, 2047])
    Ao, Eo, io = ora.solve_full(th, D, lam, tol=1e-13, cols=cols)
    assert io["status"] == "OK"
    assert eig_err(E[cols], Eo) <= EIG_RTOL, info
    assert vec_err(A[:, cols], Ao) <= VEC_TOL, info


@pytest.mark.parametrize("form", [2, 3])
def test_complex_other_product_forms(ora, dpt, form):
    sizes = [2, 64, 130, 300]
    probs = [_hermitian(n, 5000 + n, lam=0.04) for n in sizes]
    th = [torch.tensor(p[0], device="cuda") for p in probs]
    D = [dpt.colmajor_tensor(p[1], "cuda") for p in probs]
    As, Es, infos = dpt.solve_batched(th, D, [p[2] for p in probs], form=form)
    for (t, d, lam), A, E, inf in zip(probs, As, Es, infos):
        Ao, Eo, io = ora.solve_full(t, d, lam, tol=1e-13)
        assert inf["status"] == "OK"
        assert eig_err(to_np(E), Eo) <= EIG_RTOL, (len(t), inf)
        assert vec_err(to_np(A), Ao) <= VEC_TOL, (len(t), inf)
