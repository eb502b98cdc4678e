"""dpt_solve_dominant_noalloc, the entry point for callers that cannot allocate
device memory (it runs from a fixed scratch block built into the library).

Checked through the C ABI against the regular dpt_solve_dominant and against the
CPU oracle's single-vector map (Eq. (single_line_dyn), Sec. II.H) on the same
inputs, twice in a row (the second call finds the block holding the first call's
data), with the tolerances of the other GPU parity tests.  This file is collected
last so that a run stopping at the first failure has already run every other
test; it passes on its own in a fresh process as well."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dpt():
    from paper_2002_12872_gb300 import build, dpt
    build.build()
    assert torch.cuda.is_available()
    return dpt


def _dev(cfg):
    t = lambda a: torch.tensor(np.ascontiguousarray(a), device="cuda")
    return t(cfg["theta"]), t(cfg["row_ptr"]), t(cfg["col_idx"]), t(cfg["vals"])


def _close(z, E, zr, Er):
    z = z.cpu().numpy()
    zr = zr.cpu().numpy() if hasattr(zr, "cpu") else np.asarray(zr)
    un = lambda v: v / np.linalg.norm(v)
    assert abs(E - Er) <= 1e-10 * max(1.0, abs(Er))
    assert np.linalg.norm(un(z) - un(zr)) <= 1e-9


def test_noalloc_matches_pooled_entry_point_twice(ora, dpt):
    from paper_2002_12872_gb300 import inputs
    cfgs = [inputs.dominant_csr(n=200_000, nnz_per_row=16),
            inputs.dominant_csr(n=50_000, nnz_per_row=9, rep=1)]
    for cfg in cfgs:
        args = _dev(cfg)
        zr, Er, ir = dpt.solve_dominant(*args, cfg["lam"], tol=1e-13)
        zo, Eo, io = ora.solve_dominant_csr(cfg["theta"], cfg["row_ptr"], cfg["col_idx"],
                                            cfg["vals"], cfg["lam"], tol=1e-13)
        assert io["status"] == "OK"
        for _ in range(2):
            z, E, info = dpt.solve_dominant_noalloc(*args, cfg["lam"], tol=1e-13)
            assert info["status"] == "OK" and info["nstar"] == ir["nstar"]
            _close(z, E, zr, Er)
            _close(z, E, zo, Eo)


def test_noalloc_rejects_oversized_problem(dpt):
    from paper_2002_12872_gb300 import inputs
    cfg = inputs.dominant_csr(n=(1 << 18) + 1, nnz_per_row=2)
    _, _, info = dpt.solve_dominant_noalloc(*_dev(cfg), cfg["lam"], check=False)
    assert info["status"] == "ERR_TOO_LARGE"
