"""The FP16 operands of the mixed solves (single and grouped) and the FP64 finish of
strongly coupled single solves (through the C ABI).

Delta enters the tensor cores as FP16 slices of Delta 2^sig and each increment as
FP16 with its own power-of-two scale.  Replacing (Delta, lambda) by
(2^p Delta, 2^-p lambda) leaves M = diag(theta) + lambda Delta unchanged (Sec. II.B)
and shifts every scale by an exact power of two, so the solve must return the same
bits, far outside FP16's own range (|p| up to 60).  A problem whose float recursion
carried large residuals (the 2 x 2 of Sec. II.E at lambda = 0.3) is finished by the
plain FP64 map; a weakly coupled one is not."""
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
    assert torch.cuda.is_available()
    return dpt


@pytest.mark.parametrize("p", [-60, -20, 24, 60])
@pytest.mark.parametrize("pair", [True, False])
def test_power_of_two_rescaling_is_exact(dpt, p, pair):
    cfg = inputs.full_unsymmetric(n=300)
    th = torch.tensor(cfg["theta"], device="cuda")
    D = dpt.colmajor_tensor(cfg["delta"], "cuda")
    A0, E0, i0 = dpt.solve_full(th, D, cfg["lam"], cta_pair=pair)
    Ds = dpt.colmajor_tensor(np.ldexp(cfg["delta"], p), "cuda")
    A1, E1, i1 = dpt.solve_full(th, Ds, np.ldexp(cfg["lam"], -p), cta_pair=pair)
    assert i0["status"] == "OK" and i1["status"] == "OK"
    assert i1["iters"] == i0["iters"] and i1["slice_gemms"] == i0["slice_gemms"]
    assert torch.equal(A0, A1) and torch.equal(E0, E1)


@pytest.mark.parametrize("p", [-40, 30])
@pytest.mark.parametrize("form", [1, 2, 3])
@pytest.mark.parametrize("cplx", [False, True])
def test_grouped_power_of_two_rescaling_is_exact(dpt, p, form, cplx):
    """The grouped solves (batched, served, complex) carry each problem's own FP16
    scales (sig from its Delta, the increments' from its iteration): rescaling one
    problem of a group leaves its result, and every other problem's, bit for bit."""
    rng = np.random.Generator(np.random.PCG64(77 + form))
    sizes = [40, 130, 257]
    ths, Ds, Dss, lams = [], [], [], []
    for q, n in enumerate(sizes):
        th = np.arange(n, dtype=np.float64) + rng.uniform(-0.2, 0.2, n)
        D = rng.standard_normal((n, n)) / np.sqrt(n)
        if cplx:
            D = (D + 1j * rng.standard_normal((n, n)) / np.sqrt(n)) / np.sqrt(2)
            D = (D + D.conj().T) / 2
        else:
            D = (D + D.T) / 2
        ths.append(torch.tensor(th, device="cuda"))
        Ds.append(dpt.colmajor_tensor(D, "cuda"))
        Dss.append(dpt.colmajor_tensor(D * 2.0 ** p if q == 1 else D, "cuda"))
        lams.append(0.05)
    lams_s = [lams[0], np.ldexp(lams[1], -p), lams[2]]
    A0, E0, i0 = dpt.solve_batched(ths, Ds, lams, form=form)
    A1, E1, i1 = dpt.solve_batched(ths, Dss, lams_s, form=form)
    for q in range(len(sizes)):
        assert i0[q]["status"] == "OK" and i1[q]["status"] == "OK", (q, i0[q], i1[q])
        assert i1[q]["iters"] == i0[q]["iters"]
        assert i1[q]["slice_gemms"] == i0[q]["slice_gemms"]
        assert torch.equal(A0[q], A1[q]) and torch.equal(E0[q], E1[q]), q


def test_weakly_coupled_solve_needs_no_fp64_finish(ora, dpt):
    """A weakly coupled problem is not finished by the plain FP64 map on all columns;
    at most a few of its columns, whose estimated error exceeds refine_tol, get FP64
    steps of their own (none with that finish switched off)."""
    cfg = inputs.full_unsymmetric(n=513)
    th = torch.tensor(cfg["theta"], device="cuda")
    D = dpt.colmajor_tensor(cfg["delta"], "cuda")
    _, _, off = dpt.solve_full(th, D, cfg["lam"], refine_tol=0.0)
    assert off["status"] == "OK" and off["fp64_iters"] == 0 and off["refined_cols"] == 0
    A, E, info = dpt.solve_full(th, D, cfg["lam"])
    # the estimate is conservative (two to four times the error measured on
    # near-degenerate pairs), so a minority of columns gets a few FP64 steps
    assert info["status"] == "OK" and info["refined_cols"] <= 513 // 8
    assert info["fp64_iters"] <= 6
    # two FP16 slices for the first product, one once the increments are small
    assert info["slice_gemms"] <= 2 * (info["iters"] - info["fp64_iters"])
    Ao, Eo, io = ora.solve_full(cfg["theta"], cfg["delta"], cfg["lam"], tol=1e-13,
                                cols=np.array([0, 256, 512]))
    assert eig_err(to_np(E)[[0, 256, 512]], Eo) <= EIG_RTOL
    assert vec_err(to_np(A)[:, [0, 256, 512]], Ao) <= VEC_TOL


@pytest.mark.parametrize("host", [False, True])
def test_strongly_coupled_solve_is_finished_in_fp64(dpt, host):
    lam = 0.3
    th = np.array([0.0, 1.0])
    D = np.array([[0.0, 1.0], [1.0, 0.0]], order="F")
    if not host:
        th, D = torch.tensor(th, device="cuda"), torch.tensor(D, device="cuda")
    A, E, info = dpt.solve_full(th, D, lam)
    assert info["status"] == "OK" and info["fp64_iters"] > 0
    assert info["iters"] > info["fp64_iters"]
    r = np.sqrt(1 + 4 * lam * lam)
    E = to_np(E)
    # the plain FP64 map's bar (its residual at tol 1e-12)
    assert abs(E[0] - (1 - r) / 2) < 1e-12 and abs(E[1] - (1 + r) / 2) < 1e-12


@pytest.mark.parametrize("pair", [True, False])
def test_solve_returning_the_first_iterate(ora, dpt, pair):
    """Iteration 0 stores only dt_0 (A_1 = I + dt_0 is formed where it is read): at
    lambda = 1e-7 the first product already certifies A_1, which the output kernel
    then builds from dt_0."""
    cfg = inputs.full_unsymmetric(n=300)
    lam = 1e-7
    th = torch.tensor(cfg["theta"], device="cuda")
    D = dpt.colmajor_tensor(cfg["delta"], "cuda")
    A, E, info = dpt.solve_full(th, D, lam, cta_pair=pair)
    assert info["status"] == "OK" and info["iters"] == 1, info
    Ao, Eo, io = ora.solve_full(cfg["theta"], cfg["delta"], lam, tol=1e-13)
    assert io["status"] == "OK"
    assert eig_err(to_np(E), Eo) <= EIG_RTOL
    assert vec_err(to_np(A), Ao) <= VEC_TOL
    assert np.all(np.diag(to_np(A)) == 1.0)
