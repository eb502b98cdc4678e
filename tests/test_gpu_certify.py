"""The certifying pass of the mixed full solve (option certify, default on): a
product whose iterate is predicted to pass the tolerance forms only that iterate's
residual; if it does not pass, the iteration runs again in full.  The results and
iteration counts must be those of the plain iteration (certify = 0) bit for bit: for
the headline workload, parity sizes with ragged tiles, both product forms, and
tolerances near the mixed path's precision floor (where a predicted pass can fail
and the iteration is repeated)."""
import numpy as np
import pytest

from paper_2002_12872_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dpt():
    from paper_2002_12872_gb300 import build, dpt
    build.build()
    return dpt


def _pair(dpt, cfg, **kw):
    th = torch.tensor(cfg["theta"], device="cuda")
    D = dpt.colmajor_tensor(cfg["delta"], "cuda")
    out = []
    for cert in (True, False):
        A, E, info = dpt.solve_full(th, D, cfg["lam"], certify=cert, check=False, **kw)
        out.append((A.clone(), E.clone(), info))
    return out


@pytest.mark.parametrize("cta_pair", [2, 1, 0])
@pytest.mark.parametrize("case", [("unsym", 4096, 1e-12), ("sym", 256, 1e-12), ("unsym", 513, 1e-13),
                                  ("unsym", 1000, 1e-14), ("sym", 300, 3e-15)])
def test_certify_matches_plain_iteration(dpt, cta_pair, case):
    kind, n, tol = case
    cfg = inputs.full_unsymmetric(n=n) if kind == "unsym" else inputs.full_symmetric(n=n)
    (A1, E1, i1), (A0, E0, i0) = _pair(dpt, cfg, tol=tol, max_iter=40, cta_pair=cta_pair)
    assert i1["status"] == i0["status"]
    assert i1["iters"] == i0["iters"]
    assert i1["residual"] == i0["residual"]
    assert torch.equal(E1, E0) and torch.equal(A1, A0)
