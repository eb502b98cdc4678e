"""The CTA-pair forms of the product kernel (tcgen05 cta_group::2: 256-row tiles whose
operands are split over the two SMs of a pair; cta_pair = 2 stacks two pairs in a
cluster of four that share each increment tile through TMA multicast) against the
oracle and against the one-CTA form, through dpt_solve_full with the cta_pair
option."""
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


def _dev(cfg, dpt):
    return torch.tensor(cfg["theta"], device="cuda"), dpt.colmajor_tensor(cfg["delta"], "cuda")


@pytest.mark.parametrize("form", [1, 2])
@pytest.mark.parametrize("n", [1, 3, 64, 65, 200, 255, 256, 257, 300, 513, 1000])
def test_pair_parity(ora, dpt, n, form):
    """Ragged sizes: with form 2, n = 300 leaves the fourth CTA of the only row tile
    beyond the matrix, n = 513 a second row tile with one row, n = 1000 every
    cluster row tile partly filled."""
    cfg = inputs.full_unsymmetric(n=n, rep=11)
    th, D = _dev(cfg, dpt)
    A, E, info = dpt.solve_full(th, D, cfg["lam"], cta_pair=form)
    Ao, Eo, io = ora.solve_full(cfg["theta"], cfg["delta"], cfg["lam"], tol=1e-13)
    assert info["status"] == "OK" and io["status"] == "OK"
    assert info["cta_pair"] == form or info["iters"] == 0
    assert eig_err(to_np(E), Eo) <= EIG_RTOL, (n, info)
    assert vec_err(to_np(A), Ao) <= VEC_TOL, (n, info)


@pytest.mark.parametrize("form", [1, 2])
def test_pair_matches_single_cta_form(dpt, form):
    cfg = inputs.full_unsymmetric(n=777, rep=12)
    th, D = _dev(cfg, dpt)
    A1, E1, i1 = dpt.solve_full(th, D, cfg["lam"], cta_pair=0)
    A2, E2, i2 = dpt.solve_full(th, D, cfg["lam"], cta_pair=form)
    assert i1["cta_pair"] == 0 and i2["cta_pair"] == form
    assert i1["iters"] == i2["iters"]
    assert eig_err(to_np(E2), to_np(E1)) <= EIG_RTOL and vec_err(to_np(A2), to_np(A1)) <= VEC_TOL


@pytest.mark.parametrize("form", [1, 2])
def test_pair_bench_size_sampled(ora, dpt, form):
    """n = 4096 (the bench workload) with each pair form; sampled columns vs the oracle."""
    cfg = inputs.full_unsymmetric(n=4096)
    th, D = _dev(cfg, dpt)
    A, E, info = dpt.solve_full(th, D, cfg["lam"], cta_pair=form)
    assert info["status"] == "OK" and info["cta_pair"] == form
    cols = np.array([0, 1, 1000, 2047, 2048, 4094, 4095])
    Ao, Eo, io = ora.solve_full(cfg["theta"], cfg["delta"], cfg["lam"], tol=1e-13, cols=cols)
    A, E = to_np(A), to_np(E)
    assert eig_err(E[cols], Eo) <= EIG_RTOL and vec_err(A[:, cols], Ao) <= VEC_TOL


@pytest.mark.parametrize("n,rep", [(256, 1), (1000, 4)])
def test_two_slice_stages_keep_the_accuracy(ora, dpt, n, rep):
    """The pair form loads both slices per K-block after the first product (the
    increment tile fetched once); the first product, whose increment is the largest,
    keeps the per-slice accumulation order.  The eigenvector error against the FP64
    fixed point then stays that of the one-CTA form, which uses the per-slice order
    throughout (interleaving the slices in the first product too doubled it)."""
    cfg = inputs.full_unsymmetric(n=n, rep=rep)
    th, D = _dev(cfg, dpt)
    Ao, Eo, io = ora.solve_full(cfg["theta"], cfg["delta"], cfg["lam"], tol=1e-14, max_iter=60)
    assert io["status"] == "OK"
    errs = []
    for form in (1, 0):
        A, E, info = dpt.solve_full(th, D, cfg["lam"], cta_pair=form)
        assert info["status"] == "OK" and info["cta_pair"] == form
        errs.append(vec_err(to_np(A), Ao))
    assert errs[0] <= 1.25 * errs[1] + 1e-12, errs
    assert errs[0] <= VEC_TOL, errs


# Few clusters (pair_clusters): several tiles per cluster and, where they cut the
# padding, column tiles of two widths (bn, then bn - 32; the narrow ones load
# increment boxes of their own height).  In each case here the schedule has narrow
# tiles (14 wide and 5 narrow ones per row block at the bench's n = 4096); the last
# case of each form keeps one width.
@pytest.mark.parametrize("form,n,clusters", [(1, 390, 3), (1, 520, 2), (1, 1000, 5),
                                             (1, 1200, 3), (1, 777, 2), (2, 390, 1),
                                             (2, 700, 2), (2, 1000, 5), (2, 1500, 3),
                                             (2, 1000, 2)])
def test_few_clusters_two_tile_widths(ora, dpt, form, n, clusters):
    cfg = inputs.full_unsymmetric(n=n, rep=13)
    th, D = _dev(cfg, dpt)
    A, E, info = dpt.solve_full(th, D, cfg["lam"], cta_pair=form, pair_clusters=clusters)
    Ao, Eo, io = ora.solve_full(cfg["theta"], cfg["delta"], cfg["lam"], tol=1e-13)
    assert info["status"] == "OK" and io["status"] == "OK" and info["cta_pair"] == form
    assert eig_err(to_np(E), Eo) <= EIG_RTOL, (n, clusters, info)
    assert vec_err(to_np(A), Ao) <= VEC_TOL, (n, clusters, info)
    # against the schedule over every resident cluster: the tile widths differ, and
    # with them the K order of every accumulation (each tile takes its diagonal
    # K-blocks last), so the two differ by the rounding of two orders: at most twice
    # the accumulation error each keeps against the fixed point (VEC_TOL / 2 here)
    A2, E2, i2 = dpt.solve_full(th, D, cfg["lam"], cta_pair=form)
    E, E2 = to_np(E), to_np(E2)
    assert np.max(np.abs(E - E2) / np.maximum(1.0, np.abs(E2))) <= 1e-11
    assert vec_err(to_np(A), to_np(A2)) <= VEC_TOL / 2
