"""The solve server (dpt_server_create / dpt_submit / dpt_poll / dpt_wait /
dpt_cancel) on the GPU: continuous batching of problems of different n, kind and
lambda, each retired at its own convergence.

Checked here: every result equals the same problem solved alone, bit for bit,
whatever else shares its steps; results match the oracle; host and device
buffers; admission against a small memory budget; and failures made on the host
side -- malformed requests, non-finite or degenerate inputs, queue overflow,
cancellation of queued and running requests -- end only the request concerned."""
import time

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


def _problem(n, seed, cplx, lam):
    rng = np.random.Generator(np.random.PCG64(seed))
    if cplx:
        return np.arange(n, dtype=float), inputs.hermitian_gaussian(n, 1.0 / n, rng), lam
    th = np.arange(n, dtype=float) + rng.uniform(-0.2, 0.2, n)
    return th, inputs.symmetric_gaussian(n, 1.0 / n, rng), lam


def _mix():
    specs = [(37, 0, 0.05), (300, 1, 0.08), (129, 0, 0.02), (64, 1, 0.03), (513, 0, 0.06),
             (200, 1, 0.05), (1, 0, 0.1), (2, 1, 0.1), (700, 1, 0.04), (96, 0, 0.09)]
    return [_problem(n, 7000 + q, c, lam) for q, (n, c, lam) in enumerate(specs)]


def _dev(p, dpt):
    return torch.tensor(p[0], device="cuda"), dpt.colmajor_tensor(p[1], "cuda")


def test_results_identical_alone_and_in_the_mix(ora, dpt):
    probs = _mix()
    alone = []
    with dpt.Server(max_active=16) as srv:
        for p in probs:
            th, D = _dev(p, dpt)
            A, E, info = srv.wait(srv.submit(th, D, p[2]))
            assert info["status"] == "OK", info
            alone.append((to_np(A).copy(), to_np(E).copy(), info["iters"]))
    with dpt.Server(max_active=16) as srv:
        ids = []
        # staggered arrivals: later requests join while earlier ones are iterating
        for q, p in enumerate(probs):
            th, D = _dev(p, dpt)
            ids.append(srv.submit(th, D, p[2]))
            if q % 3 == 2:
                time.sleep(0.002)
        mixed = [srv.wait(i) for i in ids]
        st = srv.stats()
    assert st["completed"] == len(probs) and st["failed"] == 0
    for p, (A1, E1, it1), (A2, E2, info) in zip(probs, alone, mixed):
        assert info["status"] == "OK"
        assert info["iters"] == it1
        assert np.array_equal(A1, to_np(A2)) and np.array_equal(E1, to_np(E2)), len(p[0])
    for q in (0, 1, 4, 8):
        th, D, lam = probs[q]
        Ao, Eo, io = ora.solve_full(th, D, lam, tol=1e-13)
        assert eig_err(alone[q][1], Eo) <= EIG_RTOL and vec_err(alone[q][0], Ao) <= VEC_TOL


def test_server_matches_batched_solve(dpt):
    probs = [_problem(n, 8100 + n, 1, 0.05) for n in (64, 150, 333)]
    th = [torch.tensor(p[0], device="cuda") for p in probs]
    D = [dpt.colmajor_tensor(p[1], "cuda") for p in probs]
    As, Es, _ = dpt.solve_batched(th, D, [p[2] for p in probs])
    with dpt.Server() as srv:
        ids = [srv.submit(t, d, p[2]) for t, d, p in zip(th, D, probs)]
        res = [srv.wait(i) for i in ids]
    for (A, E, info), A0, E0 in zip(res, As, Es):
        assert info["status"] == "OK"
        assert torch.equal(A, A0) and torch.equal(E, E0)


def test_host_buffers(ora, dpt):
    th, D, lam = _problem(180, 8200, 1, 0.07)
    with dpt.Server() as srv:
        A, E, info = srv.wait(srv.submit(th, D, lam))          # numpy in and out
        A2, E2, _ = srv.wait(srv.submit(*_dev((th, D), dpt), lam))
    assert isinstance(A, np.ndarray) and info["status"] == "OK"
    assert np.array_equal(A, to_np(A2)) and np.array_equal(E, to_np(E2))
    Ao, Eo, _ = ora.solve_full(th, D, lam, tol=1e-13)
    assert eig_err(E, Eo) <= EIG_RTOL and vec_err(A, Ao) <= VEC_TOL


def test_admission_against_a_small_budget(dpt):
    probs = [_problem(600, 8300 + q, 1, 0.05) for q in range(6)]
    # one complex n = 600 problem holds about 28 MB on the device (float-float A
    # and its ping-pong, the remainder, two FP16 increments, three FP16 slice places
    # of the 1200 x 1200 real embedding), so 70 MB admits two at a time
    budget = 70 << 20
    with dpt.Server(hbm_budget=budget, max_active=8) as srv:
        ids = [srv.submit(*_dev(p, dpt), p[2]) for p in probs]
        res = [srv.wait(i) for i in ids]
        st = srv.stats()
    assert all(r[2]["status"] == "OK" for r in res)
    assert st["hbm_budget"] == budget and 0 < st["hbm_peak"] <= budget
    assert st["hbm_in_use"] == 0 and st["completed"] == 6


def test_malformed_requests_rejected_on_submit(dpt):
    th, D, lam = _problem(50, 8400, 0, 0.05)
    thd, Dd = _dev((th, D), dpt)
    with dpt.Server(hbm_budget=32 << 20) as srv:
        with pytest.raises(dpt.ServerError) as e:
            srv.submit(thd, Dd, float("nan"))
        assert e.value.status == "ERR_ARG"
        with pytest.raises(dpt.ServerError) as e:
            srv.submit(thd[:0], Dd[:0, :0], 0.1)
        assert e.value.status == "ERR_ARG"
        big = _problem(1500, 8401, 1, 0.05)
        with pytest.raises(dpt.ServerError) as e:
            srv.submit(*_dev(big, dpt), 0.05)
        assert e.value.status == "ERR_TOO_LARGE"
        A, E, info = srv.wait(srv.submit(thd, Dd, lam))      # still serving
        assert info["status"] == "OK"
        st = srv.stats()
    assert st["rejected"] == 3 and st["completed"] == 1


def test_bad_inputs_end_only_their_request(dpt):
    good = [_problem(n, 8500 + n, 1, 0.05) for n in (90, 210)]
    nan = _problem(120, 8510, 1, 0.05)
    Dn = nan[1].copy()
    Dn[5, 7] = np.nan
    deg = _problem(100, 8511, 1, 0.05)
    thg = deg[0].copy()
    thg[10] = thg[40]
    with dpt.Server() as srv:
        ids = [srv.submit(*_dev(good[0], dpt), 0.05),
               srv.submit(torch.tensor(nan[0], device="cuda"), dpt.colmajor_tensor(Dn, "cuda"), 0.05),
               srv.submit(torch.tensor(thg, device="cuda"), dpt.colmajor_tensor(deg[1], "cuda"), 0.05),
               srv.submit(*_dev(good[1], dpt), 0.05)]
        res = [srv.wait(i)[2]["status"] for i in ids]
    assert res == ["OK", "ERR_ARG", "ERR_DEGENERATE", "OK"]


def test_queue_overflow_refuses_without_losing_work(dpt):
    p = _problem(700, 8600, 1, 0.05)
    th, D = _dev(p, dpt)
    accepted, busy = [], 0
    with dpt.Server(max_active=1, max_queue=2) as srv:
        for _ in range(12):
            try:
                accepted.append(srv.submit(th, D, p[2]))
            except dpt.ServerError as e:
                assert e.status == "ERR_BUSY"
                busy += 1
        res = [srv.wait(i) for i in accepted]
        st = srv.stats()
    assert busy >= 1 and st["rejected"] == busy
    assert all(r[2]["status"] == "OK" for r in res)
    E0 = to_np(res[0][1])
    assert all(np.array_equal(E0, to_np(r[1])) for r in res)


def test_cancel_queued_and_running(dpt):
    # 2 x 2 at lambda = 0.9 cycles with period two (outside the convergence
    # domain), so it runs until cancelled
    th = torch.tensor([0.0, 1.0], device="cuda")
    D = dpt.colmajor_tensor(np.array([[0.0, 1.0], [1.0, 0.0]]), "cuda")
    p = _problem(300, 8700, 1, 0.05)
    with dpt.Server(max_active=1) as srv:
        spin = srv.submit(th, D, 0.9, max_iter=10**8)
        queued = srv.submit(*_dev(p, dpt), 0.05)
        later = srv.submit(*_dev(p, dpt), 0.05)
        assert srv.cancel(queued) == "OK"
        assert srv.wait(queued)[2]["status"] == "ERR_CANCELLED"
        time.sleep(0.2)
        assert srv.poll(spin) is None                         # still running
        assert srv.cancel(spin) == "OK"
        info = srv.wait(spin, timeout=30)[2]
        assert info["status"] == "ERR_CANCELLED"
        A, E, info = srv.wait(later, timeout=60)
        assert info["status"] == "OK"
        st = srv.stats()
    assert st["cancelled"] == 2 and st["completed"] == 1


def test_poisson_stream_sampled(ora, dpt):
    """A short Poisson stream (2000 req/s) of the served recipe -- complex
    Hermitian, theta_i = i, Delta variance 1/n, lambda in [0.02, 0.08] -- with n
    log-uniform in [64, 1024]; sampled columns of some results vs the oracle."""
    reqs = inputs.served_hermitian(count=32, rep=9, lo=64, hi=1024)
    dev = [(torch.tensor(r["theta"], device="cuda"), dpt.colmajor_tensor(r["delta"], "cuda"))
           for r in reqs]
    torch.cuda.synchronize()
    with dpt.Server() as srv:
        t0 = time.perf_counter()
        ids = []
        for r, (th, D) in zip(reqs, dev):
            while time.perf_counter() - t0 < r["arrival_s"]:
                pass
            ids.append(srv.submit(th, D, r["lam"]))
        res = [srv.wait(i) for i in ids]
        st = srv.stats()
    assert st["completed"] == len(reqs)
    for q in (0, 5, 11, 31):
        r = reqs[q]
        n = r["n"]
        cols = np.unique(np.array([0, n // 3, n - 1]))
        Ao, Eo, io = ora.solve_full(r["theta"], r["delta"], r["lam"], tol=1e-13, cols=cols)
        A, E = to_np(res[q][0]), to_np(res[q][1])
        assert eig_err(E[cols], Eo) <= EIG_RTOL and vec_err(A[:, cols], Ao) <= VEC_TOL
