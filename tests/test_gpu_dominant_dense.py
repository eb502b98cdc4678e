"""GPU parity of dpt_solve_dominant_dense (dense Delta, a GEMV per iteration,
through the C ABI) against the FP64 oracle: the single-vector map of Sec. II.H is
the full-form map restricted to column n* (Eq. (single_line_dyn)), so the oracle's
full solve on that one column is the reference.  Sizes span several row blocks
and column slices with ragged tails, odd n (one row per thread), a leading
dimension larger than n, host-resident Delta, both arithmetic variants, an
interior n*, and the full n = 32768 workload checked through properties that hold
at any size; degenerate and non-finite inputs return their statuses."""
import numpy as np
import pytest

from gpu_util import EIG_RTOL, VEC_TOL, to_np
from paper_2002_12872_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dpt():
    from paper_2002_12872_gb300 import build, dpt
    build.build()
    return dpt


def _unit(v):
    v = np.asarray(v)
    return v / np.linalg.norm(v)


def _check(z, E, zo, Eo):
    z = to_np(z)
    assert abs(E - Eo) <= EIG_RTOL * max(1.0, abs(Eo)), (E, Eo)
    assert np.linalg.norm(_unit(z) - _unit(zo)) <= VEC_TOL


def _oracle(ora, cfg, nstar=0):
    A, E, io = ora.solve_full(cfg["theta"], cfg["delta"], cfg["lam"], tol=1e-14,
                              cols=[nstar])
    assert io["status"] == "OK", io
    return A[:, 0], float(E[0])


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
@pytest.mark.parametrize("n", [1, 2, 40, 1000, 3001, 4096])
def test_dense_dominant_parity(ora, dpt, prec, n):
    cfg = inputs.dominant_dense(n=n)
    zo, Eo = _oracle(ora, cfg)
    th = torch.tensor(cfg["theta"], device="cuda")
    D = torch.tensor(cfg["delta"], device="cuda")
    z, E, info = dpt.solve_dominant_dense(th, D, cfg["lam"], prec=prec, tol=1e-13)
    assert info["status"] == "OK" and info["nstar"] == 0
    assert to_np(z)[0] == 1.0
    _check(z, E, zo, Eo)


def test_dense_dominant_padded_ld_and_interior_nstar(ora, dpt):
    """Delta as a view with leading dimension n + 13 (odd: one row per thread) and
    an eigenvector from the middle of the spectrum, n* given explicitly."""
    n, nstar = 1500, 611
    rng = np.random.Generator(np.random.PCG64(7))
    theta = np.arange(n, dtype=np.float64) + rng.uniform(-0.2, 0.2, n)
    big = rng.standard_normal((n + 13, n)) / np.sqrt(n)
    delta = np.asfortranarray(big)[:n, :]
    cfg = {"theta": theta, "delta": np.asfortranarray(delta), "lam": 0.05}
    zo, Eo = _oracle(ora, cfg, nstar)
    Dt = torch.tensor(np.ascontiguousarray(big.T), device="cuda")   # memory = columns
    view = Dt.t()[:n, :]
    assert view.stride(0) == 1 and view.stride(1) == n + 13
    z, E, info = dpt.solve_dominant_dense(torch.tensor(theta, device="cuda"), view, 0.05,
                                          nstar=nstar, tol=1e-13)
    assert info["nstar"] == nstar and to_np(z)[nstar] == 1.0
    _check(z, E, zo, Eo)


def test_dense_dominant_host_inputs(ora, dpt):
    """Host theta / Delta / z: the library stages them through its workspace."""
    cfg = inputs.dominant_dense(n=777, rep=2)
    zo, Eo = _oracle(ora, cfg)
    z, E, info = dpt.solve_dominant_dense(cfg["theta"], cfg["delta"], cfg["lam"], tol=1e-13)
    assert isinstance(z, np.ndarray)
    _check(z, E, zo, Eo)


def test_dense_dominant_matches_csr_form(dpt):
    """The dense and CSR forms of one sparse Delta reach the same eigenpair."""
    cfg = inputs.dominant_csr(n=2000, nnz_per_row=16, lam=0.01)
    D = inputs.csr_to_dense(cfg["row_ptr"], cfg["col_idx"], cfg["vals"], cfg["n"])
    t = lambda a: torch.tensor(np.ascontiguousarray(a), device="cuda")
    zs, Es, _ = dpt.solve_dominant(t(cfg["theta"]), t(cfg["row_ptr"]), t(cfg["col_idx"]),
                                   t(cfg["vals"]), cfg["lam"], tol=1e-13)
    zd, Ed, _ = dpt.solve_dominant_dense(t(cfg["theta"]), torch.tensor(D, device="cuda"),
                                         cfg["lam"], tol=1e-13)
    assert abs(Es - Ed) <= EIG_RTOL * max(1.0, abs(Es))
    assert np.linalg.norm(_unit(to_np(zs)) - _unit(to_np(zd))) <= VEC_TOL


def test_dense_dominant_wide_exponent_range(ora, dpt):
    """Entries spread over 2^-140 .. 2^6 in magnitude (below the float range, where
    the float-float split flushes, through its lower-part cut-off near 2^-103) give
    the oracle's eigenpair."""
    n = 900
    rng = np.random.Generator(np.random.PCG64(11))
    theta = rng.uniform(0, 1, n)
    theta[0] = 2.0
    scale = 2.0 ** rng.integers(-140, 7, size=(n, n))
    delta = np.asfortranarray(rng.standard_normal((n, n)) * scale / n)
    cfg = {"theta": theta, "delta": delta, "lam": 0.01}
    zo, Eo = _oracle(ora, cfg)
    z, E, info = dpt.solve_dominant_dense(torch.tensor(theta, device="cuda"),
                                          torch.tensor(delta, device="cuda"), 0.01, tol=1e-13)
    assert info["status"] == "OK"
    _check(z, E, zo, Eo)


def test_dense_dominant_deterministic(dpt):
    cfg = inputs.dominant_dense(n=2048, rep=1)
    th = torch.tensor(cfg["theta"], device="cuda")
    D = torch.tensor(cfg["delta"], device="cuda")
    z1, E1, _ = dpt.solve_dominant_dense(th, D, cfg["lam"])
    z2, E2, _ = dpt.solve_dominant_dense(th, D, cfg["lam"], graph_iters=0)
    assert E1 == E2 and torch.equal(z1, z2)


def test_dense_dominant_statuses(dpt):
    n = 300
    cfg = inputs.dominant_dense(n=n)
    th = torch.tensor(cfg["theta"], device="cuda")
    D = torch.tensor(cfg["delta"], device="cuda")
    # degenerate: theta_{n*} repeated
    th2 = th.clone()
    th2[5] = th2[0]
    _, _, info = dpt.solve_dominant_dense(th2, D, cfg["lam"], check=False)
    assert info["status"] == "ERR_DEGENERATE"
    # non-finite Delta entry (found by the first pass)
    for bad in (float("nan"), float("inf")):
        D2 = D.clone()
        D2[17, 211] = bad
        _, _, info = dpt.solve_dominant_dense(th, D2, cfg["lam"], check=False)
        assert info["status"] == "ERR_ARG"
    # an entry beyond the float range: rejected by the float-float form only
    D2 = D.clone()
    D2[3, 4] = 1e39
    _, _, info = dpt.solve_dominant_dense(th, D2, cfg["lam"], check=False)
    assert info["status"] == "ERR_ARG"
    _, _, info = dpt.solve_dominant_dense(th, D2, cfg["lam"], prec="fp64", check=False)
    assert info["status"] != "ERR_ARG"
    # non-finite theta
    th3 = th.clone()
    th3[9] = float("nan")
    _, _, info = dpt.solve_dominant_dense(th3, D, cfg["lam"], check=False)
    assert info["status"] == "ERR_ARG"
    # iteration budget: one iteration is not enough
    _, _, info = dpt.solve_dominant_dense(th, D, cfg["lam"], max_iter=1, check=False)
    assert info["status"] == "ERR_MAXITER"


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_dense_dominant_full_size(dpt, prec):
    """n = 32768 (8.6 GB of Delta), the launch configuration the benchmark times.
    Checked by properties that hold at any size: the eigen-residual of (E, z)
    against M = diag(theta) + lam Delta in FP64 (plain torch matrix-vector
    product), z[n*] = 1, and E beside the Rayleigh quotient e_{n*}^T M z."""
    cfg = inputs.dominant_dense_device(n=32768)
    th, D, lam = cfg["theta"], cfg["delta"], cfg["lam"]
    z, E, info = dpt.solve_dominant_dense(th, D, lam, prec=prec, tol=1e-12)
    assert info["status"] == "OK" and info["nstar"] == 0
    assert float(z[0]) == 1.0
    Mz = th * z + lam * (D @ z)
    r = torch.linalg.vector_norm(Mz - E * z).item()
    s = th.abs().max().item() + abs(lam) * D.abs().sum(dim=1).max().item()
    assert r / (s * torch.linalg.vector_norm(z).item()) <= 1e-11
    assert abs(E - Mz[0].item()) <= 1e-12 * abs(E)
    del D, cfg
    torch.cuda.empty_cache()
