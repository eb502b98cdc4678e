"""GPU parity of the two forms of the mixed full solve's first step (Sec. II.B:
iteration 0 from A_0 = I, plus the FP16 slicing of Delta).

The library takes the pass over pairs of mirrored 64 x 64 tiles (Delta read once, by
TMA) when Delta's base is 16-byte aligned and its column pitch is even; any other
layout (or a start matrix) runs the slicing pass and then iteration 0.  Both must meet
the oracle's parity bar and agree with each other: the same problem is solved from an
even and from an odd column pitch, at sizes that leave ragged 64- and 128-wide tiles
(and n below one tile)."""
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


def _pitched(delta, ld):
    """Delta on the device, column-major with column pitch ld >= n."""
    n = delta.shape[0]
    store = torch.zeros((n, ld), dtype=torch.float64, device="cuda")   # row c = column c
    store[:, :n] = torch.tensor(np.asarray(delta).T, device="cuda")
    D = store[:, :n].t()
    assert D.stride(0) == 1 and D.stride(1) == ld
    return D


def _pitches(n):
    even = n if n % 2 == 0 else n + 1
    odd = n if n % 2 == 1 else n + 1
    return even, odd


@pytest.mark.parametrize("n", [2, 3, 17, 64, 65, 127, 129, 200, 257, 300])
def test_both_forms_meet_the_oracle_and_agree(ora, dpt, n):
    cfg = inputs.full_unsymmetric(n=n)
    Ao, Eo, io = ora.solve_full(cfg["theta"], cfg["delta"], cfg["lam"], tol=1e-13)
    assert io["status"] == "OK"
    th = torch.tensor(cfg["theta"], device="cuda")
    res = {}
    for name, ld in zip(("fused", "two-pass"), _pitches(n)):
        A, E, info = dpt.solve_full(th, _pitched(cfg["delta"], ld), cfg["lam"], prec="mixed",
                                    tol=1e-12)
        ee, ve = eig_err(to_np(E), Eo), vec_err(to_np(A), Ao)
        assert ee <= EIG_RTOL and ve <= VEC_TOL, (name, n, ee, ve, info)
        assert info["residual"] <= 1e-12
        res[name] = (to_np(A), to_np(E), info)
    (Af, Ef, inf_f), (At, Et, inf_t) = res["fused"], res["two-pass"]
    # the two forms differ only in the order of the float-float column sums
    assert np.max(np.abs(Ef - Et) / np.maximum(1.0, np.abs(Et))) <= 1e-11
    assert vec_err(Af, At) <= 1e-10
    if inf_f["iters"] == inf_t["iters"]:
        # the fused form is one kernel fewer (no separate slicing pass)
        assert inf_f["launches"] == inf_t["launches"] - 1, (inf_f, inf_t)


@pytest.mark.parametrize("n", [65, 200])
def test_fused_form_epstein_nesbet(ora, dpt, n):
    cfg = inputs.full_symmetric(n=n)
    Ao, Eo, io = ora.solve_full(cfg["theta"], cfg["delta"], cfg["lam"], tol=1e-13)
    th = torch.tensor(cfg["theta"], device="cuda")
    ld = _pitches(n)[0]
    A, E, info = dpt.solve_full(th, _pitched(cfg["delta"], ld), cfg["lam"], prec="mixed",
                                epstein_nesbet=True)
    ee, ve = eig_err(to_np(E), Eo), vec_err(to_np(A), Ao)
    assert ee <= EIG_RTOL and ve <= VEC_TOL, (ee, ve, info)


@pytest.mark.parametrize("where", [(0, 0), (5, 130), (130, 5), (199, 198)])
def test_fused_form_rejects_nonfinite_entries(dpt, where):
    n = 200
    cfg = inputs.full_unsymmetric(n=n)
    th = torch.tensor(cfg["theta"], device="cuda")
    D = _pitched(cfg["delta"], n)
    D[where] = float("inf")
    _, _, info = dpt.solve_full(th, D, cfg["lam"], prec="mixed", check=False)
    assert info["status"] == "ERR_ARG"


def test_forms_agree_at_bench_size(dpt):
    """n = 4096, the bench's workload: the fused form (even pitch, as the bench runs
    it) is checked against the oracle on sampled columns in test_gpu_full.py; here it
    must agree with the two-pass form on every eigenpair."""
    n = 4096
    cfg = inputs.full_unsymmetric(n=n)
    th = torch.tensor(cfg["theta"], device="cuda")
    out = []
    for ld in (n, n + 1):
        A, E, info = dpt.solve_full(th, _pitched(cfg["delta"], ld), cfg["lam"], prec="mixed",
                                    tol=1e-12)
        assert info["status"] == "OK"
        out.append((to_np(A), to_np(E)))
    (Af, Ef), (At, Et) = out
    assert np.max(np.abs(Ef - Et) / np.maximum(1.0, np.abs(Et))) <= 1e-11
    assert vec_err(Af, At) <= 1e-10
