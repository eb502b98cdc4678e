"""Pins of the oracle's dominant-eigenvector form (single-vector map of
Eq. (single_line_dyn) for n* = argmax theta, Sec. II.H) against the full-spectrum
oracle and a library eigensolver on small sparse problems."""
import numpy as np
import pytest

from paper_2002_12872_gb300 import inputs


@pytest.mark.parametrize("n,k", [(50, 4), (300, 16)])
def test_dominant_matches_full_column_and_library(ora, n, k):
    cfg = inputs.dominant_csr(n=n, nnz_per_row=k)
    th, lam = cfg["theta"], cfg["lam"]
    z, E, info = ora.solve_dominant_csr(th, cfg["row_ptr"], cfg["col_idx"], cfg["vals"],
                                        lam, tol=1e-14)
    assert info["status"] == "OK"
    D = inputs.csr_to_dense(cfg["row_ptr"], cfg["col_idx"], cfg["vals"], n)
    A, Ef, infof = ora.solve_full(th, D, lam, tol=1e-14, cols=[0])
    assert abs(E - Ef[0]) < 1e-13 and np.abs(z - A[:, 0]).max() < 1e-13
    w = np.linalg.eigvals(np.diag(th) + lam * D)   # test-only library cross-check
    assert abs(E - w.real.max()) < 1e-12
    M = np.diag(th) + lam * D
    assert np.linalg.norm(M @ z - E * z) < 1e-12 * np.linalg.norm(z) * 3


def test_dominant_default_nstar_is_argmax(ora):
    cfg = inputs.dominant_csr(n=40, nnz_per_row=3)
    th = cfg["theta"].copy()
    th[0], th[7] = 0.5, 2.0
    z, E, info = ora.solve_dominant_csr(th, cfg["row_ptr"], cfg["col_idx"], cfg["vals"],
                                        0.01, tol=1e-14)
    assert info["status"] == "OK" and z[7] == 1.0


def test_dominant_rejects_bad_csr(ora):
    th = np.array([2.0, 1.0, 0.5])
    z, E, info = ora.solve_dominant_csr(th, [0, 1, 2, 3], [0, 5, 1], [1, 1, 1], 0.01)
    assert info["status"] == "ARG"
