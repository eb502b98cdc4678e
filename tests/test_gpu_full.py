"""GPU parity of dpt_solve_full (through the C ABI) against the FP64 oracle.

Bar (per eigenpair): |E - E_ora| <= 1e-10 max(1, |E_ora|) and
|| a/||a|| - a_ora/||a_ora|| ||_2 <= 1e-9; inputs are the seeded workloads of
paper_2002_12872_gb300.inputs at sizes that span several 128-wide tiles and a
ragged tail, plus the degenerate and edge cases of the method."""
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


def _dev(cfg):
    from paper_2002_12872_gb300 import dpt
    th = torch.tensor(cfg["theta"], device="cuda")
    D = dpt.colmajor_tensor(cfg["delta"], "cuda")
    return th, D


def _parity(A, E, Ao, Eo):
    A, E = to_np(A), to_np(E)
    return eig_err(E, Eo), vec_err(A, Ao)


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
@pytest.mark.parametrize("which,n", [("sym", 256), ("unsym", 300), ("unsym", 130),
                                     ("sym", 64), ("unsym", 513)])
def test_full_parity(ora, dpt, prec, which, n):
    cfg = inputs.full_symmetric(n=n) if which == "sym" else inputs.full_unsymmetric(n=n)
    Ao, Eo, io = ora.solve_full(cfg["theta"], cfg["delta"], cfg["lam"], tol=1e-13)
    assert io["status"] == "OK"
    th, D = _dev(cfg)
    A, E, info = dpt.solve_full(th, D, cfg["lam"], prec=prec, tol=1e-12)
    ee, ve = _parity(A, E, Ao, Eo)
    assert ee <= EIG_RTOL and ve <= VEC_TOL, (ee, ve, info)
    Ad = to_np(A)
    assert np.all(np.diag(Ad) == 1.0)
    assert info["residual"] <= 1e-12


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_two_by_two_closed_form(dpt, prec):
    lam = 0.3
    th = torch.tensor([0.0, 1.0], device="cuda", dtype=torch.float64)
    D = torch.tensor([[0.0, 1.0], [1.0, 0.0]], device="cuda", dtype=torch.float64)
    A, E, info = dpt.solve_full(th, D, lam, prec=prec)
    r = np.sqrt(1 + 4 * lam * lam)
    em, ep = (1 - r) / 2, (1 + r) / 2
    E = to_np(E)
    # FP64 path: to rounding; mixed path: the parity bar (diagonal increments of
    # the product are carried in FP32)
    etol = 1e-12 if prec == "fp64" else EIG_RTOL
    assert abs(E[0] - em) < etol and abs(E[1] - ep) < etol
    x = em / lam
    assert np.allclose(to_np(A), [[1.0, -x], [x, 1.0]], atol=1e-11)


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_n_equals_one(dpt, prec):
    th = torch.tensor([3.0], device="cuda", dtype=torch.float64)
    D = torch.tensor([[0.5]], device="cuda", dtype=torch.float64)
    A, E, info = dpt.solve_full(th, D, 0.2, prec=prec)
    assert to_np(A)[0, 0] == 1.0 and abs(to_np(E)[0] - 3.1) < 1e-15


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_outside_domain_reports_failure(dpt, prec):
    th = torch.tensor([0.0, 1.0], device="cuda", dtype=torch.float64)
    D = torch.tensor([[0.0, 1.0], [1.0, 0.0]], device="cuda", dtype=torch.float64)
    A, E, info = dpt.solve_full(th, D, 0.9, prec=prec, max_iter=300, check=False)
    assert info["status"] in ("ERR_MAXITER", "ERR_DIVERGED")


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_degenerate_theta(dpt, prec):
    th = torch.tensor([0.0, 1.0, 1.0], device="cuda", dtype=torch.float64)
    D = torch.ones(3, 3, device="cuda", dtype=torch.float64)
    A, E, info = dpt.solve_full(th, D, 0.1, prec=prec, check=False)
    assert info["status"] == "ERR_DEGENERATE"


# a device theta is checked on the device over 256-index blocks of i and 32-index chunks
# of j: pairs within a chunk, across chunk and block boundaries, and in the ragged end
@pytest.mark.parametrize("pair", [(5, 6), (40, 300), (255, 256), (31, 32), (600, 699),
                                  (0, 699), (287, 288)])
def test_device_theta_duplicates_found_anywhere(dpt, pair):
    n = 700
    cfg = inputs.full_unsymmetric(n=n)
    th, D = _dev(cfg)
    a, b = pair
    th[b] = th[a]
    _, _, info = dpt.solve_full(th, D, cfg["lam"], prec="mixed", check=False)
    assert info["status"] == "ERR_DEGENERATE", (pair, info)


@pytest.mark.parametrize("where,value", [(0, float("nan")), (257, float("inf")),
                                         (699, float("-inf")), (32, float("nan"))])
def test_device_theta_nonfinite_rejected(dpt, where, value):
    n = 700
    cfg = inputs.full_unsymmetric(n=n)
    th, D = _dev(cfg)
    th[where] = value
    _, _, info = dpt.solve_full(th, D, cfg["lam"], prec="mixed", check=False)
    assert info["status"] == "ERR_ARG", (where, info)


def test_device_theta_signed_zeros_are_equal(dpt):
    n = 300
    cfg = inputs.full_unsymmetric(n=n)
    th, D = _dev(cfg)
    th[10], th[270] = 0.0, -0.0
    _, _, info = dpt.solve_full(th, D, cfg["lam"], prec="mixed", check=False)
    assert info["status"] == "ERR_DEGENERATE"


def test_device_theta_adjacent_doubles_are_distinct(dpt):
    """theta_j one ulp above theta_i is a distinct level: the check must not flag it
    (the solve itself may then fail to converge, with the gap at rounding level)."""
    n = 300
    cfg = inputs.full_unsymmetric(n=n)
    th, D = _dev(cfg)
    th[200] = float(np.nextafter(float(th[40]), np.inf))
    _, _, info = dpt.solve_full(th, D, cfg["lam"], prec="mixed", check=False, max_iter=3)
    assert info["status"] not in ("ERR_DEGENERATE", "ERR_ARG"), info


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_nonfinite_delta_rejected(dpt, prec):
    cfg = inputs.full_unsymmetric(n=40)
    th, D = _dev(cfg)
    D[3, 5] = float("nan")
    A, E, info = dpt.solve_full(th, D, cfg["lam"], prec=prec, check=False)
    assert info["status"] == "ERR_ARG"


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_epstein_nesbet_same_result(ora, dpt, prec):
    cfg = inputs.full_unsymmetric(n=200)
    Ao, Eo, _ = ora.solve_full(cfg["theta"], cfg["delta"], cfg["lam"], tol=1e-13)
    th, D = _dev(cfg)
    A, E, info = dpt.solve_full(th, D, cfg["lam"], prec=prec, epstein_nesbet=True)
    ee, ve = _parity(A, E, Ao, Eo)
    assert ee <= EIG_RTOL and ve <= VEC_TOL, (ee, ve)


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_host_buffers(ora, dpt, prec):
    """Host (numpy) inputs and outputs: the library stages them itself."""
    cfg = inputs.full_symmetric(n=150)
    Ao, Eo, _ = ora.solve_full(cfg["theta"], cfg["delta"], cfg["lam"], tol=1e-13)
    A, E, info = dpt.solve_full(cfg["theta"], np.asfortranarray(cfg["delta"]), cfg["lam"],
                                prec=prec)
    assert isinstance(A, np.ndarray)
    ee, ve = _parity(A, E, Ao, Eo)
    assert ee <= EIG_RTOL and ve <= VEC_TOL


def test_graph_and_plain_loop_agree(dpt):
    cfg = inputs.full_unsymmetric(n=260)
    th, D = _dev(cfg)
    A1, E1, i1 = dpt.solve_full(th, D, cfg["lam"], graph_iters=4)
    A2, E2, i2 = dpt.solve_full(th, D, cfg["lam"], graph_iters=0)
    assert i1["iters"] == i2["iters"]
    assert np.abs(to_np(A1) - to_np(A2)).max() < 1e-13


def test_complex_hermitian_fp64(ora, dpt):
    rng = inputs.rng_for(5, 7)
    n = 96
    th = np.arange(n, dtype=float)
    D = inputs.hermitian_gaussian(n, 1.0 / n, rng)
    lam = 0.05
    Ao, Eo, io = ora.solve_full(th.astype(complex), D, lam, tol=1e-13)
    A, E, info = dpt.solve_full(torch.tensor(th, device="cuda"),
                                torch.tensor(D, device="cuda"), lam, prec="fp64")
    ee, ve = _parity(A, E, Ao, Eo)
    assert ee <= EIG_RTOL and ve <= VEC_TOL, (ee, ve)


def test_full_size_unsymmetric_sampled_columns(ora, dpt):
    """The full n = 4096 unsymmetric workload in the bench's configuration (mixed
    path, default options); the oracle solves a seeded sample of columns (each
    column is its own map, Sec. II.B) together with the eight columns whose nearest
    level is closest (the smallest gaps theta_i - theta_j the map divides by), and
    the explicit residual M a - E a of the sample is recomputed in FP64.  The error
    bound of the mixed arithmetic holds for every column of this workload, so no
    column needs the FP64 finish."""
    cfg = inputs.full_unsymmetric(n=4096)
    th, D = _dev(cfg)
    A, E, info = dpt.solve_full(th, D, cfg["lam"])
    assert info["status"] == "OK"
    assert info["refined_cols"] == 0 and info["fp64_iters"] == 0
    rng = np.random.Generator(np.random.PCG64(4096))
    cols = np.sort(rng.choice(4096, size=6, replace=False))
    t = cfg["theta"]
    gap = np.abs(t[:, None] - t[None, :])
    np.fill_diagonal(gap, np.inf)
    tight = np.argsort(gap.min(axis=0), kind="stable")[:8]
    cols = np.unique(np.concatenate([[0, 4095], cols, tight]))
    Ao, Eo, io = ora.solve_full(cfg["theta"], cfg["delta"], cfg["lam"], tol=1e-13,
                                cols=cols)
    assert io["status"] == "OK"
    An, En = to_np(A)[:, cols], to_np(E)[cols]
    assert eig_err(En, Eo) <= EIG_RTOL
    assert vec_err(An, Ao) <= VEC_TOL
    M = np.diag(cfg["theta"]) + cfg["lam"] * cfg["delta"]
    R = M @ An - An * En[None, :]
    s = np.abs(cfg["theta"]).max() + cfg["lam"] * np.abs(cfg["delta"]).sum(1).max()
    rho = np.linalg.norm(R, axis=0) / (s * np.linalg.norm(An, axis=0))
    assert rho.max() <= 1e-10


def test_full_max_size_sampled_columns(ora, dpt):
    """n = 32768, the largest size whose full mixed solve fits comfortably in device
    memory beside its input and output (32 GB of workspace, 8.6 GB each for Delta
    and A): every 64-bit offset of the slices (3 n^2 elements), partials and tiles is
    exercised.  Checked on sampled columns: the explicit FP64 residual M a - E a of
    16 seeded columns, and the oracle's solution of two of them (each column is its
    own map, Sec. II.B)."""
    n = 32768
    cfg = inputs.full_unsymmetric_device(n=n)
    th = torch.tensor(cfg["theta"], device="cuda")
    D, lam = cfg["delta"], cfg["lam"]
    A = torch.empty((n, n), dtype=torch.float64, device="cuda").t()
    E = torch.empty(n, dtype=torch.float64, device="cuda")
    _, _, info = dpt.solve_full(th, D, lam, A_out=A, E_out=E)
    assert info["status"] == "OK"
    rng = np.random.Generator(np.random.PCG64(n))
    cols = np.sort(np.concatenate([[0, n - 1], rng.choice(np.arange(1, n - 1), 14, replace=False)]))
    ct = torch.tensor(cols, device="cuda")
    Ac = A[:, ct]
    R = th[:, None] * Ac + lam * (D @ Ac) - Ac * E[ct][None, :]
    s = th.abs().max().item() + lam * D.abs().sum(1).max().item()
    rho = (torch.linalg.vector_norm(R, dim=0) / (s * torch.linalg.vector_norm(Ac, dim=0))).max()
    assert rho.item() <= 1e-10
    assert torch.all(A[ct, ct] == 1.0)
    Dh = D.t().contiguous().cpu().numpy().T          # column-major host copy
    two = np.array([0, n - 1])
    Ao, Eo, io = ora.solve_full(cfg["theta"], Dh, lam, tol=1e-13, cols=two)
    assert io["status"] == "OK"
    assert eig_err(to_np(E)[two], Eo) <= EIG_RTOL
    assert vec_err(to_np(A[:, torch.tensor(two, device="cuda")]), Ao) <= VEC_TOL
    del A, D, cfg, Dh
    dpt.release_workspace()
    torch.cuda.empty_cache()


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_profiled_solve_reports_product_time(dpt, prec):
    cfg = inputs.full_unsymmetric(n=300)
    th, D = _dev(cfg)
    A1, E1, i1 = dpt.solve_full(th, D, cfg["lam"], prec=prec, profile=True)
    A2, E2, i2 = dpt.solve_full(th, D, cfg["lam"], prec=prec, profile=False)
    # mixed: one product per mixed iteration (FP64 steps that finish columns are counted
    # in iters and fp64_iters, not as tensor-core products)
    mixed_iters = i1["iters"] - i1["fp64_iters"]
    assert i1["product_launches"] == mixed_iters + (1 if prec == "fp64" else 0) or \
        i1["product_launches"] >= mixed_iters
    assert i1["product_ms"] > 0 and i2["product_ms"] == 0
    assert i1["launches"] > i1["product_launches"]
    assert np.abs(to_np(A1) - to_np(A2)).max() == 0.0


@pytest.mark.parametrize("n", [3, 5, 17, 63, 127, 128, 129, 255, 257, 383, 640])
def test_mixed_size_sweep(ora, dpt, n):
    """Tile edges and ragged tails of the 128 x 128 tiles and 64-wide K blocks."""
    cfg = inputs.full_unsymmetric(n=n)
    Ao, Eo, io = ora.solve_full(cfg["theta"], cfg["delta"], cfg["lam"], tol=1e-13)
    assert io["status"] == "OK"
    th, D = _dev(cfg)
    A, E, info = dpt.solve_full(th, D, cfg["lam"], prec="mixed")
    ee, ve = _parity(A, E, Ao, Eo)
    assert ee <= EIG_RTOL and ve <= VEC_TOL, (n, ee, ve, info)


def test_repeated_solves_identical(dpt):
    """The same problem twice through the pooled workspace gives identical bits
    (deterministic reductions, no state leaking between calls)."""
    cfg = inputs.full_unsymmetric(n=700)
    th, D = _dev(cfg)
    A1, E1, _ = dpt.solve_full(th, D, cfg["lam"])
    other = inputs.full_symmetric(n=333)
    dpt.solve_full(*_dev(other), other["lam"])
    A2, E2, _ = dpt.solve_full(th, D, cfg["lam"])
    assert torch.equal(A1, A2) and torch.equal(E1, E2)


def test_prepared_solve_replays_its_graph(dpt):
    """A prepared solve called again replays the iteration graph kept with its workspace
    (same buffers, form and parameters); another problem, another lambda or another
    chunk size in between capture a new one, and inputs changed in place are read
    afresh.  Each result equals that of a fresh call (new output buffers, so a new
    graph) bit for bit."""
    cfg = inputs.full_unsymmetric(n=300)
    th, D = _dev(cfg)
    fs = dpt.FullSolve(th, D, cfg["lam"], prec="mixed", tol=1e-12)

    def fresh(lam=cfg["lam"], **kw):
        return dpt.solve_full(th, D, lam, prec="mixed", tol=1e-12, **kw)

    fs.solve()
    A1 = fs.A.clone()
    fs.solve()                                        # replayed
    assert torch.equal(fs.A, A1)
    other = inputs.full_symmetric(n=333)
    dpt.solve_full(*_dev(other), other["lam"])        # another problem, same pool
    fs.solve()
    assert torch.equal(fs.A, A1)
    assert torch.equal(fresh()[0], A1)
    fs2 = dpt.FullSolve(th, D, 0.5 * cfg["lam"], prec="mixed", tol=1e-12, A_out=fs.A,
                        E_out=fs.E)                   # another lambda, same outputs
    fs2.solve()
    assert torch.equal(fs.A, fresh(0.5 * cfg["lam"])[0])
    fs3 = dpt.FullSolve(th, D, cfg["lam"], prec="mixed", tol=1e-12, graph_iters=2,
                        A_out=fs.A, E_out=fs.E)       # another chunk size
    fs3.solve()
    assert torch.equal(fs.A, A1)
    D.mul_(0.5)                                       # new values in the same buffer
    fs.solve()
    ref = fresh()[0]
    assert not torch.equal(ref, A1)
    assert torch.equal(fs.A, ref)


@pytest.mark.parametrize("graph_iters", [0, 1, 2, 3, 4, 5, 7])
def test_profiled_solves_any_chunk_size(dpt, graph_iters):
    """Per-launch profiling with every chunk size, including chunks that end exactly at
    convergence: the counted product launches equal the iterations."""
    cfg = inputs.full_unsymmetric(n=512, rep=21)
    th = torch.tensor(cfg["theta"], device="cuda")
    D = dpt.colmajor_tensor(cfg["delta"], "cuda")
    _, _, info = dpt.solve_full(th, D, cfg["lam"], profile=True, graph_iters=graph_iters)
    assert info["status"] == "OK"
    assert info["product_launches"] == info["iters"] - info["fp64_iters"]
    assert info["product_ms"] > 0


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_workspace_bytes_matches_pool_growth(dpt, prec):
    """dpt_workspace_bytes equals what a solve with device buffers takes from the
    pool: device memory drops by that figure (up to allocation granularity) when an
    empty pool serves one solve."""
    n = 2048
    cfg = inputs.full_unsymmetric(n=n)
    th, D = _dev(cfg)
    A = torch.empty((n, n), dtype=torch.float64, device="cuda").t()
    E = torch.empty(n, dtype=torch.float64, device="cuda")
    dpt.solve_full(th, D, cfg["lam"], prec=prec, A_out=A, E_out=E)   # modules loaded
    torch.cuda.synchronize()
    dpt.release_workspace()
    free0 = torch.cuda.mem_get_info()[0]
    dpt.solve_full(th, D, cfg["lam"], prec=prec, A_out=A, E_out=E)
    torch.cuda.synchronize()
    used = free0 - torch.cuda.mem_get_info()[0]
    ws = dpt.workspace_bytes(n, prec=prec)
    assert ws > 0 and abs(used - ws) <= 8 * 2**20, (used, ws)
    dpt.release_workspace()


def test_prepared_solve_matches_solve_full(dpt):
    """FullSolve (arguments marshalled once) is the same C-ABI call as solve_full: the
    same bits, call after call, into the caller's buffers."""
    cfg = inputs.full_unsymmetric(n=300)
    th, D = _dev(cfg)
    A0, E0, i0 = dpt.solve_full(th, D, cfg["lam"])
    A = torch.empty((300, 300), dtype=torch.float64, device="cuda").t()
    E = torch.empty(300, dtype=torch.float64, device="cuda")
    fs = dpt.FullSolve(th, D, cfg["lam"], A_out=A, E_out=E, profile=True)
    for _ in range(2):
        info = fs.solve()
        assert info["status"] == "OK" and info["iters"] == i0["iters"]
        assert info["product_ms"] > 0
        assert torch.equal(A, A0) and torch.equal(E, E0)
