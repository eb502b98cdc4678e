"""GPU parity of the generalised start (option start: the polisher use of the closing
remark of Sec. II.H, approximate eigenvectors refined by the map's last steps)
against the oracle iterating from the same start, through the C ABI:

- both dominant forms and precisions on the Supplement's 3x3 example at
  lambda = -0.48, second line: unreachable from e_2, reached from the continued
  eigenvector perturbed by 1 %;
- a seeded n = 3000 dense problem from its solution perturbed by 1e-4: fewer steps
  than from e_{n*}, same eigenpair; a host-resident start;
- the plain-FP64 full solve (real and complex Hermitian) from a perturbed solution,
  invariant under scaling of the start, and its argument errors;
- the mixed real full solve, whose first increment is the start's offset from I:
  parity from a perturbed solution (device, host and scaled starts), fewer products
  from the solution itself than from I, a zero chart entry refused; the complex mixed
  solve refuses the option."""
import numpy as np
import pytest

from gpu_util import EIG_RTOL, VEC_TOL, eig_err, to_np, vec_err
from paper_2002_12872_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TH3 = np.array([0.0, 1.0, 3.0])
D3 = np.array([[0.0, 1.0, 2.0], [1.0, 0.0, 3.0], [2.0, 3.0, 0.0]])
RP3 = np.array([0, 2, 4, 6], dtype=np.int32)
CI3 = np.array([1, 2, 0, 2, 0, 1], dtype=np.int32)
VA3 = np.array([1, 2, 1, 3, 2, 3], dtype=np.float32)


@pytest.fixture(scope="module")
def dpt():
    from paper_2002_12872_gb300 import build, dpt
    build.build()
    return dpt


def _unit(v):
    v = np.asarray(v)
    return v / np.linalg.norm(v)


def _t(a):
    return torch.tensor(np.ascontiguousarray(a), device="cuda")


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_start_reaches_3x3_second_line(ora, dpt, prec):
    lam = -0.48
    # a start near the fixed point: the ramped oracle's solution perturbed by 1 %
    Ar, _, _ = ora.solve_full(TH3, D3, lam, tol=1e-14, max_iter=5000, cols=[1],
                              ramp_alpha=0.9)
    rng = np.random.Generator(np.random.PCG64(5))
    s = Ar[:, 0] * (1.0 + 0.01 * rng.standard_normal(3))
    A, Eo, io = ora.solve_full(TH3, D3, lam, tol=1e-14, max_iter=3000, cols=[1],
                               start=s[:, None])
    assert io["status"] == "OK"
    zo = A[:, 0]
    z, E, info = dpt.solve_dominant_dense(_t(TH3), _t(D3), lam, nstar=1, prec=prec, tol=1e-13,
                                          max_iter=3000, start=_t(s))
    assert info["status"] == "OK"
    assert abs(E - Eo[0]) <= EIG_RTOL * max(1.0, abs(Eo[0]))
    assert np.linalg.norm(_unit(to_np(z)) - _unit(zo)) <= VEC_TOL
    z, E, info = dpt.solve_dominant(_t(TH3), _t(RP3), _t(CI3), _t(VA3), lam, nstar=1, prec=prec,
                                    tol=1e-13, max_iter=3000, start=_t(s))
    assert info["status"] == "OK"
    assert abs(E - Eo[0]) <= EIG_RTOL * max(1.0, abs(Eo[0]))
    assert np.linalg.norm(_unit(to_np(z)) - _unit(zo)) <= VEC_TOL


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_start_dense_polisher(ora, dpt, prec):
    cfg = inputs.dominant_dense(n=3000, rep=5)
    A, Eo, io = ora.solve_full(cfg["theta"], cfg["delta"], cfg["lam"], tol=1e-14, cols=[0])
    assert io["status"] == "OK"
    rng = np.random.Generator(np.random.PCG64(8))
    s = A[:, 0] * (1.0 + 1e-4 * rng.standard_normal(cfg["n"]))
    th, D = _t(cfg["theta"]), _t(cfg["delta"])
    _, _, i0 = dpt.solve_dominant_dense(th, D, cfg["lam"], prec=prec, tol=1e-13)
    for start in (_t(s), s, 2.5 * s):      # device, host, and a scaled start
        z, E, info = dpt.solve_dominant_dense(th, D, cfg["lam"], prec=prec, tol=1e-13,
                                              start=start)
        assert info["status"] == "OK" and info["iters"] < i0["iters"]
        assert abs(E - Eo[0]) <= EIG_RTOL * max(1.0, abs(Eo[0]))
        assert np.linalg.norm(_unit(to_np(z)) - _unit(A[:, 0])) <= VEC_TOL
    bad = s.copy()
    bad[0] = 0.0
    _, _, info = dpt.solve_dominant_dense(th, D, cfg["lam"], prec=prec, start=_t(bad),
                                          check=False)
    assert info["status"] == "ERR_ARG"
    bad = s.copy()
    bad[7] = np.nan
    _, _, info = dpt.solve_dominant_dense(th, D, cfg["lam"], prec=prec, start=_t(bad),
                                          check=False)
    assert info["status"] == "ERR_ARG"


@pytest.mark.parametrize("cplx", [False, True])
def test_start_full_fp64(ora, dpt, cplx):
    from paper_2002_12872_gb300 import dpt as d
    if cplx:
        rng = np.random.Generator(np.random.PCG64(12))
        n = 96
        th = np.arange(n, dtype=float)
        delta = inputs.hermitian_gaussian(n, 1.0 / n, rng)
        lam = 0.1
    else:
        cfg = inputs.full_unsymmetric(n=160)
        th, delta, lam, n = cfg["theta"], cfg["delta"], cfg["lam"], cfg["n"]
    Aref, _, _ = ora.solve_full(th, delta, lam, tol=1e-14)
    rng = np.random.Generator(np.random.PCG64(13))
    S = Aref * (1.0 + 1e-3 * rng.standard_normal(Aref.shape))
    Ao, Eo, io = ora.solve_full(th, delta, lam, tol=1e-14, start=S)
    assert io["status"] == "OK"
    D = d.colmajor_tensor(delta, "cuda")
    thd = _t(th)
    for start in (d.colmajor_tensor(S, "cuda"), np.asfortranarray(S * 3.0)):
        A, E, info = dpt.solve_full(thd, D, lam, prec="fp64", tol=1e-13, start=start)
        assert info["status"] == "OK"
        assert eig_err(to_np(E), Eo) <= EIG_RTOL and vec_err(to_np(A), Ao) <= VEC_TOL
    bad = S.copy()
    bad[5, 5] = 0.0
    _, _, info = dpt.solve_full(thd, D, lam, prec="fp64", start=np.asfortranarray(bad),
                                check=False)
    assert info["status"] == "ERR_ARG"
    if cplx:
        _, _, info = dpt.solve_full(thd, D, lam, start=d.colmajor_tensor(S, "cuda"),
                                    check=False)
        assert info["status"] == "ERR_UNSUPPORTED"


def test_start_full_mixed(ora, dpt):
    from paper_2002_12872_gb300 import dpt as d
    cfg = inputs.full_unsymmetric(n=300)
    th, delta, lam = cfg["theta"], cfg["delta"], cfg["lam"]
    Aref, _, _ = ora.solve_full(th, delta, lam, tol=1e-14)
    rng = np.random.Generator(np.random.PCG64(14))
    S = Aref * (1.0 + 1e-3 * rng.standard_normal(Aref.shape))
    Ao, Eo, io = ora.solve_full(th, delta, lam, tol=1e-14, start=S)
    assert io["status"] == "OK"
    D = d.colmajor_tensor(delta, "cuda")
    thd = _t(th)
    for start in (d.colmajor_tensor(S, "cuda"), np.asfortranarray(S * 3.0)):
        A, E, info = dpt.solve_full(thd, D, lam, prec="mixed", tol=1e-13, start=start)
        assert info["status"] == "OK", info
        assert eig_err(to_np(E), Eo) <= EIG_RTOL and vec_err(to_np(A), Ao) <= VEC_TOL, info
    # from the solution itself (its FP16 rounding is all that is left to remove)
    _, _, i0 = dpt.solve_full(thd, D, lam, prec="mixed", tol=1e-13)
    _, _, i1 = dpt.solve_full(thd, D, lam, prec="mixed", tol=1e-13,
                              start=d.colmajor_tensor(Aref, "cuda"))
    assert i1["status"] == "OK" and i1["iters"] <= i0["iters"], (i0, i1)
    bad = S.copy()
    bad[7, 7] = 0.0
    _, _, info = dpt.solve_full(thd, D, lam, prec="mixed", start=d.colmajor_tensor(bad, "cuda"),
                                check=False)
    assert info["status"] == "ERR_ARG"
