"""GPU parity of dpt_solve_dominant (CSR, through the C ABI) against the FP64
oracle's single-vector map (Sec. II.H), on the seeded sparse workload: small and
medium sizes with a ragged row structure, the full n = 2e6 / nnz = 3.2e7 case,
both arithmetic variants, and the degenerate / malformed cases."""
import numpy as np
import pytest

from gpu_util import to_np
from paper_2002_12872_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dpt():
    from paper_2002_12872_gb300 import build, dpt
    build.build()
    return dpt


def _dev(cfg):
    t = lambda a: torch.tensor(np.ascontiguousarray(a), device="cuda")
    return t(cfg["theta"]), t(cfg["row_ptr"]), t(cfg["col_idx"]), t(cfg["vals"])


def _check(z, E, zo, Eo):
    z = to_np(z)
    un = lambda v: v / np.linalg.norm(v)
    assert abs(E - Eo) <= 1e-10 * max(1.0, abs(Eo)), (E, Eo)
    assert np.linalg.norm(un(z) - un(zo)) <= 1e-9


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
@pytest.mark.parametrize("n,k", [(40, 3), (1000, 16), (20000, 16), (5000, 70)])
def test_dominant_parity(ora, dpt, prec, n, k):
    cfg = inputs.dominant_csr(n=n, nnz_per_row=k)
    zo, Eo, io = ora.solve_dominant_csr(cfg["theta"], cfg["row_ptr"], cfg["col_idx"],
                                        cfg["vals"], cfg["lam"], tol=1e-14)
    assert io["status"] == "OK"
    z, E, info = dpt.solve_dominant(*_dev(cfg), cfg["lam"], prec=prec, tol=1e-13)
    assert info["nstar"] == 0 and to_np(z)[0] == 1.0
    _check(z, E, zo, Eo)


def test_dominant_ragged_rows(ora, dpt):
    """Rows of very different length (0 to 200 nonzeros), explicit n*."""
    rng = np.random.Generator(np.random.PCG64(5))
    n = 3000
    lens = rng.integers(0, 200, size=n)
    lens[::7] = 0
    row_ptr = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    col_idx = np.concatenate([np.sort(rng.choice(n, l, replace=False)) for l in lens]).astype(np.int32)
    vals = (rng.standard_normal(row_ptr[-1]) * 0.05).astype(np.float32)
    theta = rng.uniform(0, 1, n)
    theta[17] = 3.0
    zo, Eo, io = ora.solve_dominant_csr(theta, row_ptr, col_idx, vals, 0.02, nstar=17, tol=1e-14)
    z, E, info = dpt.solve_dominant(torch.tensor(theta, device="cuda"),
                                    torch.tensor(row_ptr, device="cuda"),
                                    torch.tensor(col_idx, device="cuda"),
                                    torch.tensor(vals, device="cuda"), 0.02, nstar=17, tol=1e-13)
    assert info["nstar"] == 17
    _check(z, E, zo, Eo)


def test_dominant_host_buffers(ora, dpt):
    cfg = inputs.dominant_csr(n=3000, nnz_per_row=16)
    zo, Eo, io = ora.solve_dominant_csr(cfg["theta"], cfg["row_ptr"], cfg["col_idx"],
                                        cfg["vals"], cfg["lam"], tol=1e-14)
    z, E, info = dpt.solve_dominant(cfg["theta"], cfg["row_ptr"], cfg["col_idx"], cfg["vals"],
                                    cfg["lam"], tol=1e-13)
    assert isinstance(z, np.ndarray)
    _check(z, E, zo, Eo)


def test_dominant_degenerate_and_malformed(dpt):
    cfg = inputs.dominant_csr(n=100, nnz_per_row=4)
    th, rp, ci, va = _dev(cfg)
    th2 = th.clone()
    th2[5] = th2[0]            # ties with the largest theta
    _, _, info = dpt.solve_dominant(th2, rp, ci, va, 0.01, check=False)
    assert info["status"] == "ERR_DEGENERATE"
    ci2 = ci.clone()
    ci2[10] = 100              # column out of range
    _, _, info = dpt.solve_dominant(th, rp, ci2, va, 0.01, check=False)
    assert info["status"] == "ERR_ARG"
    rp2 = rp.clone()
    rp2[50] = rp2[49] - 1      # decreasing row pointer
    _, _, info = dpt.solve_dominant(th, rp2, ci, va, 0.01, check=False)
    assert info["status"] == "ERR_ARG"


def test_dominant_full_size(ora, dpt):
    """The full n = 2,000,000 / 16 nonzeros per row workload, in the configuration
    bench.py times, against the oracle's full solve."""
    cfg = inputs.dominant_csr()
    zo, Eo, io = ora.solve_dominant_csr(cfg["theta"], cfg["row_ptr"], cfg["col_idx"],
                                        cfg["vals"], cfg["lam"], tol=1e-13)
    assert io["status"] == "OK"
    z, E, info = dpt.solve_dominant(*_dev(cfg), cfg["lam"], tol=1e-12)
    _check(z, E, zo, Eo)


def test_gather_probe(dpt):
    """dpt_probe_gather (a calibration of the CSR form's roofline): it gathers exactly
    what a pass gathers, so its per-row sums of the gathered high parts equal a plain
    reference, and it reports a positive time per pass."""
    cfg = inputs.dominant_csr(n=50_000, nnz_per_row=16, rep=2)
    _, rp, ci, _ = _dev(cfg)
    g = torch.Generator(device="cuda")
    g.manual_seed(3)
    z = torch.rand((50_000, 2), generator=g, device="cuda", dtype=torch.float32)
    from paper_2002_12872_gb300 import dpt as d
    n = 50_000
    y = torch.empty(n, dtype=torch.float32, device="cuda")
    import ctypes
    ms = ctypes.c_double(0.0)
    st = d.lib().dpt_probe_gather(n, rp.data_ptr(), ci.data_ptr(), z.data_ptr(), y.data_ptr(), 3,
                                  ctypes.byref(ms), None)
    assert st == 0 and ms.value > 0
    rows = torch.repeat_interleave(torch.arange(n, device="cuda"), rp[1:] - rp[:-1])
    ref = torch.zeros(n, dtype=torch.float64, device="cuda").index_add_(
        0, rows, z[ci.long(), 0].double())
    assert torch.allclose(y.double(), ref, rtol=1e-5, atol=1e-5)
    assert dpt.probe_gather(rp, ci, z, reps=2) > 0
