"""The bounded device waits: a wait that nothing completes gives up after its limit,
the kernel returns, and the host reads DPT_ERR_TIMEOUT -- no fault, no hang, and
the device context stays usable for the next solve."""
import time

import numpy as np
import pytest

from gpu_util import EIG_RTOL, eig_err, to_np
from paper_2002_12872_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dpt():
    from paper_2002_12872_gb300 import build, dpt
    build.build()
    return dpt


def test_expired_wait_returns_timeout_and_context_survives(ora, dpt):
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    assert dpt.selftest_bounded_wait(0.3) == "ERR_TIMEOUT"
    dt = time.perf_counter() - t0
    assert 0.3 <= dt < 5.0
    cfg = inputs.full_symmetric(n=64)
    A, E, info = dpt.solve_full(torch.tensor(cfg["theta"], device="cuda"),
                                dpt.colmajor_tensor(cfg["delta"], "cuda"), cfg["lam"])
    Ao, Eo, _ = ora.solve_full(cfg["theta"], cfg["delta"], cfg["lam"], tol=1e-13)
    assert info["status"] == "OK" and eig_err(to_np(E), Eo) <= EIG_RTOL
