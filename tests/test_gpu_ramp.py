"""GPU parity of the non-autonomous iteration (option ramp_alpha: step k applies the
map at lambda (1 - alpha^k), the continuation the Supplement applies to its explicit
3x3 example) against the oracle's ramped iteration, through the C ABI:

- the dense and CSR dominant forms, both arithmetic variants, on the printed 3x3
  example at lambda = -0.48 for its second line, where the autonomous iteration
  from e_2 does not converge and the ramped one does;
- the same forms on a seeded n = 3000 problem (the ramp changes the path, not the
  fixed point), against the oracle's ramped single-vector map;
- the plain-FP64 full solve against the oracle's ramped full solve, and its first
  iterates in closed form (step 0 applies strength 0, so A_1 = I exactly);
- the forms that carry the residual across steps at one lambda refuse the option."""
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
def test_ramp_rescues_3x3_second_line(ora, dpt, prec):
    lam = -0.48
    A, Eo, io = ora.solve_full(TH3, D3, lam, tol=1e-14, max_iter=5000, cols=[1],
                               ramp_alpha=0.9)
    assert io["status"] == "OK"
    zo = A[:, 0]
    # dense form: autonomous fails, ramped converges to the oracle's vector
    _, _, i0 = dpt.solve_dominant_dense(_t(TH3), _t(D3), lam, nstar=1, prec=prec,
                                        max_iter=3000, check=False)
    assert i0["status"] != "OK"
    z, E, info = dpt.solve_dominant_dense(_t(TH3), _t(D3), lam, nstar=1, prec=prec,
                                          max_iter=3000, tol=1e-13, ramp_alpha=0.9)
    assert info["status"] == "OK"
    assert abs(E - Eo[0]) <= EIG_RTOL * max(1.0, abs(Eo[0]))
    assert np.linalg.norm(_unit(to_np(z)) - _unit(zo)) <= VEC_TOL
    # CSR form
    _, _, i1 = dpt.solve_dominant(_t(TH3), _t(RP3), _t(CI3), _t(VA3), lam, nstar=1, prec=prec,
                                  max_iter=3000, check=False)
    assert i1["status"] != "OK"
    z, E, info = dpt.solve_dominant(_t(TH3), _t(RP3), _t(CI3), _t(VA3), lam, nstar=1,
                                    prec=prec, max_iter=3000, tol=1e-13, ramp_alpha=0.9)
    assert info["status"] == "OK"
    assert abs(E - Eo[0]) <= EIG_RTOL * max(1.0, abs(Eo[0]))
    assert np.linalg.norm(_unit(to_np(z)) - _unit(zo)) <= VEC_TOL


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_ramp_dominant_forms_larger(ora, dpt, prec):
    cfg = inputs.dominant_dense(n=3000, rep=4)
    A, Eo, io = ora.solve_full(cfg["theta"], cfg["delta"], cfg["lam"], tol=1e-14, cols=[0],
                               ramp_alpha=0.5)
    assert io["status"] == "OK"
    z, E, info = dpt.solve_dominant_dense(_t(cfg["theta"]), _t(cfg["delta"]), cfg["lam"],
                                          prec=prec, tol=1e-13, ramp_alpha=0.5)
    assert info["status"] == "OK"
    assert abs(E - Eo[0]) <= EIG_RTOL * max(1.0, abs(Eo[0]))
    assert np.linalg.norm(_unit(to_np(z)) - _unit(A[:, 0])) <= VEC_TOL
    # the autonomous solve reaches the same point in fewer steps
    z0, E0, i0 = dpt.solve_dominant_dense(_t(cfg["theta"]), _t(cfg["delta"]), cfg["lam"],
                                          prec=prec, tol=1e-13)
    assert i0["iters"] < info["iters"]
    assert abs(E0 - E) <= EIG_RTOL * max(1.0, abs(E))
    c = inputs.dominant_csr(n=3000, nnz_per_row=16, rep=4)
    zc, Ec, ic = ora.solve_dominant_csr(c["theta"], c["row_ptr"], c["col_idx"], c["vals"],
                                        c["lam"], tol=1e-14, ramp_alpha=0.5)
    assert ic["status"] == "OK"
    z, E, info = dpt.solve_dominant(_t(c["theta"]), _t(c["row_ptr"]), _t(c["col_idx"]),
                                    _t(c["vals"]), c["lam"], prec=prec, tol=1e-13,
                                    ramp_alpha=0.5)
    assert info["status"] == "OK"
    assert abs(E - Ec) <= EIG_RTOL * max(1.0, abs(Ec))
    assert np.linalg.norm(_unit(to_np(z)) - _unit(zc)) <= VEC_TOL


def test_ramp_full_fp64(ora, dpt):
    cfg = inputs.full_symmetric(n=200, lam=0.05)
    Ao, Eo, io = ora.solve_full(cfg["theta"], cfg["delta"], cfg["lam"], tol=1e-14,
                                ramp_alpha=0.6)
    assert io["status"] == "OK"
    th = _t(cfg["theta"])
    from paper_2002_12872_gb300 import dpt as d
    D = d.colmajor_tensor(cfg["delta"], "cuda")
    A, E, info = dpt.solve_full(th, D, cfg["lam"], prec="fp64", tol=1e-13, ramp_alpha=0.6)
    assert info["status"] == "OK"
    assert eig_err(to_np(E), Eo) <= EIG_RTOL and vec_err(to_np(A), Ao) <= VEC_TOL
    # one step of the ramp applies strength 0: A_1 = I exactly
    A1, _, i1 = dpt.solve_full(th, D, cfg["lam"], prec="fp64", max_iter=1, ramp_alpha=0.6,
                               check=False)
    assert i1["status"] == "ERR_MAXITER" and i1["iters"] == 1
    assert np.array_equal(to_np(A1), np.eye(cfg["n"]))


@pytest.mark.parametrize("which,alpha", [("sym", 0.6), ("unsym", 0.5)])
def test_ramp_full_mixed(ora, dpt, which, alpha):
    """The mixed full solve with the non-autonomous iteration: each step's increment
    is r G o R - (1 - r)(A - I), r = 1 - alpha^(k+1) (the ramp's identity step 0 is not
    run, so its iterate A_k is the ramped map's A_{k+1}); the carried residual stays
    the one at lambda, so the limit is the autonomous fixed point, to the bar."""
    cfg = (inputs.full_symmetric(n=200, lam=0.05) if which == "sym"
           else inputs.full_unsymmetric(n=300))
    Ao, Eo, io = ora.solve_full(cfg["theta"], cfg["delta"], cfg["lam"], tol=1e-14,
                                ramp_alpha=alpha)
    assert io["status"] == "OK"
    th = _t(cfg["theta"])
    from paper_2002_12872_gb300 import dpt as d
    D = d.colmajor_tensor(cfg["delta"], "cuda")
    A, E, info = dpt.solve_full(th, D, cfg["lam"], prec="mixed", tol=1e-13, ramp_alpha=alpha)
    assert info["status"] == "OK", info
    assert eig_err(to_np(E), Eo) <= EIG_RTOL and vec_err(to_np(A), Ao) <= VEC_TOL, info
    # the schedule: the mixed A_3 follows the ramped map's A_4 (to the FP16 rounding of
    # the increments, which the carried remainder corrects in later steps)
    A3, _, i3 = dpt.solve_full(th, D, cfg["lam"], prec="mixed", max_iter=3, ramp_alpha=alpha,
                               check=False)
    assert i3["status"] == "ERR_MAXITER"
    A4o, _, _ = ora.solve_full(cfg["theta"], cfg["delta"], cfg["lam"], tol=1e-300, max_iter=4,
                               ramp_alpha=alpha)
    X = A4o - np.eye(cfg["n"])
    assert np.abs(to_np(A3) - A4o).max() <= 1e-3 * np.abs(X).max()


def test_ramp_refused_where_unsupported(dpt):
    """The grouped mixed path (complex mixed full solves, batches, the server) runs no
    ramp; invalid ramp factors are refused everywhere."""
    cfg = inputs.full_symmetric(n=64)
    th = _t(cfg["theta"])
    from paper_2002_12872_gb300 import dpt as d
    D = d.colmajor_tensor(cfg["delta"], "cuda")
    rng = np.random.Generator(np.random.PCG64(3))
    Dc = d.colmajor_tensor(inputs.hermitian_gaussian(64, 1.0 / 64, rng), "cuda")
    _, _, info = dpt.solve_full(th, Dc, cfg["lam"], ramp_alpha=0.5, check=False)
    assert info["status"] == "ERR_UNSUPPORTED"
    for bad in (-0.5, 1.0):
        _, _, info = dpt.solve_full(th, D, cfg["lam"], prec="fp64", ramp_alpha=bad, check=False)
        assert info["status"] == "ERR_ARG"
        _, _, info = dpt.solve_dominant_dense(th, D, cfg["lam"], ramp_alpha=bad, check=False)
        assert info["status"] == "ERR_ARG"
