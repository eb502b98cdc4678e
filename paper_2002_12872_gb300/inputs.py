"""Seeded synthetic inputs for the DPT workloads.

This module only draws random problems.  It holds none of the method's
arithmetic, so the oracle tests and the CUDA path can share it without sharing
any part of the computation.  Every generator uses NumPy's PCG64 with the seed
``2002_12872 + 1000 * config + rep``.

Shapes follow the problem statement of arXiv:2002.12872 (Sec. II.B):
M = diag(theta) + lam * Delta with simple unperturbed eigenvalues theta.  Dense
matrices are returned column-major (``order="F"``); CSR arrays are int32 / FP32.

Workloads (the paper has no public data set for this path; its random dense and
sparse perturbations, Sec. II.G-H, are synthetic, so these stand in for them):

  full_symmetric     theta_i = i, Delta symmetric with iid N(0, 1/n) entries
                     (upper triangle and diagonal drawn, then mirrored), lam 0.05
  full_unsymmetric   theta = sorted uniforms on [0, (n+1)/2] plus 0.5*i (values in
                     [0, n], every gap >= 0.5), Delta iid N(0, 1/n), lam 0.1
  dominant_csr       theta_m ~ U[0, 1] with theta_0 = 2, 16 distinct sorted column
                     indices per row drawn uniformly, values N(0, 1) in FP32,
                     lam 0.01
  dominant_dense     theta_m ~ U[0, 1] with theta_0 = 2, Delta iid N(0, 1/n)
                     dense FP64, lam 0.1 (the GEMV form; drawn on the device
                     by torch's seeded generator at sizes beyond a few thousand)
  batched_symmetric  n log-uniform in [32, 512], theta_i = i + U(-0.2, 0.2),
                     symmetric Delta as above, lam ~ U[0.01, 0.1]
  served_hermitian   Poisson arrivals, n log-uniform in [64, 4096], theta_i = i,
                     Hermitian Delta with E|x|^2 = 1/n (real N(0, 1/n) diagonal,
                     off-diagonal real and imaginary parts N(0, 1/(2n))),
                     lam ~ U[0.02, 0.08]
  near_degenerate    theta_i = base + i with one pair moved to a gap of ratio x its
                     coupling lambda |Delta|, Delta iid N(0, 1/n), lam 0.1 (the
                     edge case of the gaps in Eq. (dyn))
  delta_oscillator   the harmonic oscillator with a delta potential (Sec. II.F):
                     theta_n = 2n + 1/2, rank-one Delta from Hermite functions at 0
  served_pool /      the same requests drawn from a pool of distinct Hermitian
  served_stream      problems at stratified quantiles of the log-uniform size law
                     (each request its own lambda), so that long streams need not
                     hold one matrix per request
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 2002_12872


def seed_for(config: int, rep: int = 0) -> int:
    return SEED_BASE + 1000 * config + rep


def rng_for(config: int, rep: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed_for(config, rep)))


def symmetric_gaussian(n: int, var: float, rng: np.random.Generator) -> np.ndarray:
    """Symmetric n x n matrix: upper triangle (with diagonal) iid N(0, var), mirrored."""
    g = rng.standard_normal((n, n)) * np.sqrt(var)
    u = np.triu(g)
    return np.asfortranarray(u + np.triu(u, 1).T)


def hermitian_gaussian(n: int, var: float, rng: np.random.Generator) -> np.ndarray:
    """Hermitian n x n matrix with E|x_jk|^2 = var off the diagonal (real and
    imaginary parts N(0, var/2)) and a real N(0, var) diagonal."""
    re = rng.standard_normal((n, n)) * np.sqrt(var / 2.0)
    im = rng.standard_normal((n, n)) * np.sqrt(var / 2.0)
    dg = rng.standard_normal(n) * np.sqrt(var)
    up = np.triu(re + 1j * im, 1)
    h = up + up.conj().T
    h[np.arange(n), np.arange(n)] = dg
    return np.asfortranarray(h)


def full_symmetric(n: int = 256, rep: int = 0, lam: float = 0.05) -> dict:
    """Dense real symmetric workload (theta_i = i)."""
    rng = rng_for(1, rep)
    theta = np.arange(n, dtype=np.float64)
    delta = symmetric_gaussian(n, 1.0 / n, rng)
    return {"n": n, "theta": theta, "delta": delta, "lam": lam, "tol": 1e-12}


def spaced_uniform(n: int, min_gap: float, rng: np.random.Generator) -> np.ndarray:
    """n sorted values in [0, n] with every gap >= min_gap: sorted uniforms on
    [0, n - min_gap*(n-1)] shifted by min_gap * i (a uniform hard-core spacing)."""
    span = n - min_gap * (n - 1)
    u = np.sort(rng.uniform(0.0, span, size=n))
    return u + min_gap * np.arange(n)


def full_unsymmetric(n: int = 4096, rep: int = 0, lam: float = 0.1) -> dict:
    """Dense real unsymmetric workload (gaps >= 0.5, Delta iid N(0, 1/n))."""
    rng = rng_for(2, rep)
    theta = spaced_uniform(n, 0.5, rng)
    delta = np.asfortranarray(rng.standard_normal((n, n)) / np.sqrt(n))
    return {"n": n, "theta": theta, "delta": delta, "lam": lam, "tol": 1e-12}


def near_degenerate(n: int = 260, base: float = 0.0, ratio: float = 10.0, rep: int = 0,
                    lam: float = 0.1) -> dict:
    """A near-degenerate, strongly coupled pair in an otherwise regular spectrum (the
    edge the gaps theta_i - theta_j of Eq. (dyn) put at risk): theta_i = base + i,
    Delta iid N(0, 1/n) unsymmetric, and level i0 + 1 (i0 = n // 2) moved to
    theta_i0 + g with g = ratio * lam * max(|Delta_{i0,i0+1}|, |Delta_{i0+1,i0}|), so
    that the pair's coupling over its gap is 1 / ratio.  The map converges here for
    ratio >= 5 (at ratio 3 this draw's iteration diverges); base moves the spectrum to
    large |theta| without changing any gap.  Returns the pair's indices as "pair"."""
    rng = rng_for(6, rep)
    theta = base + np.arange(n, dtype=np.float64)
    delta = np.asfortranarray(rng.standard_normal((n, n)) / np.sqrt(n))
    i0 = n // 2
    g = ratio * lam * max(abs(delta[i0, i0 + 1]), abs(delta[i0 + 1, i0]))
    theta[i0 + 1] = theta[i0] + g
    return {"n": n, "theta": theta, "delta": delta, "lam": lam, "tol": 1e-15,
            "pair": (i0, i0 + 1), "gap": g}


def full_unsymmetric_device(n: int = 32768, rep: int = 0, lam: float = 0.1, device="cuda"):
    """full_unsymmetric's recipe at sizes whose host generation would dominate a run:
    theta from the same NumPy draw, Delta iid N(0, 1/n) drawn on the device with
    torch's seeded generator (column-major: the transpose view of a row-major
    tensor)."""
    import torch
    theta = spaced_uniform(n, 0.5, rng_for(2, rep))
    g = torch.Generator(device=device)
    g.manual_seed(seed_for(2, rep))
    rows = torch.randn(n, n, generator=g, device=device, dtype=torch.float64)
    rows.mul_(1.0 / np.sqrt(n))
    return {"n": n, "theta": theta, "delta": rows.t(), "lam": lam, "tol": 1e-12}


def dominant_csr(n: int = 2_000_000, nnz_per_row: int = 16, rep: int = 0,
                 lam: float = 0.01) -> dict:
    """Sparse unsymmetric CSR workload for the dominant-eigenvector form."""
    rng = rng_for(3, rep)
    theta = rng.uniform(0.0, 1.0, size=n)
    theta[0] = 2.0
    k = min(nnz_per_row, n)
    cols = rng.integers(0, n, size=(n, k), dtype=np.int64)
    cols.sort(axis=1)
    # redraw rows with a repeated index until every row has k distinct columns
    while True:
        dup = np.any(cols[:, 1:] == cols[:, :-1], axis=1) if k > 1 else np.zeros(n, bool)
        bad = np.nonzero(dup)[0]
        if bad.size == 0:
            break
        redraw = np.stack([np.sort(rng.choice(n, size=k, replace=False)) for _ in bad])
        cols[bad] = redraw
    col_idx = cols.reshape(-1).astype(np.int32)
    row_ptr = (np.arange(n + 1, dtype=np.int64) * k).astype(np.int32)
    vals = rng.standard_normal(n * k).astype(np.float32)
    return {"n": n, "theta": theta, "row_ptr": row_ptr, "col_idx": col_idx,
            "vals": vals, "lam": lam, "nstar": 0, "tol": 1e-12}


def dominant_dense(n: int = 32768, rep: int = 0, lam: float = 0.1) -> dict:
    """Dense unsymmetric workload for the dominant-eigenvector form (GEMV):
    theta_m ~ U[0, 1] with theta_0 = 2 set apart, Delta iid N(0, 1/n) (column-major
    FP64)."""
    rng = rng_for(6, rep)
    theta = rng.uniform(0.0, 1.0, size=n)
    theta[0] = 2.0
    delta = np.asfortranarray(rng.standard_normal((n, n)) / np.sqrt(n))
    return {"n": n, "theta": theta, "delta": delta, "lam": lam, "nstar": 0, "tol": 1e-12}


def dominant_dense_device(n: int = 32768, rep: int = 0, lam: float = 0.1, device="cuda"):
    """dominant_dense's recipe drawn on the device with torch's seeded generator
    (sizes whose host generation would dominate a run).  Returns theta (n) and the
    column-major Delta as the transpose view of a row-major tensor."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed_for(6, rep))
    theta = torch.rand(n, generator=g, device=device, dtype=torch.float64)
    theta[0] = 2.0
    rows = torch.randn(n, n, generator=g, device=device, dtype=torch.float64)
    rows.mul_(1.0 / np.sqrt(n))
    return {"n": n, "theta": theta, "delta": rows.t(), "lam": lam, "nstar": 0, "tol": 1e-12}


def delta_oscillator(N: int = 100) -> dict:
    """The harmonic oscillator with a delta potential at the origin (Sec. II.F), on
    the even Hermite functions: theta_n = 2n + 1/2 and the rank-one Delta_nm =
    phi_2n(0) phi_2m(0), with phi_k(x) = (2^k k! sqrt(pi))^(-1/2) H_k(x) exp(-x^2/2),
    so phi_0(0) = pi^(-1/4) and phi_2n(0) = -phi_2n-2(0) sqrt((2n-1)/(2n)) (from
    H_2n(0) = (-1)^n (2n)!/n!).  Deterministic: no random draw."""
    phi = np.zeros(N)
    phi[0] = np.pi ** -0.25
    for n in range(1, N):
        phi[n] = -phi[n - 1] * np.sqrt((2 * n - 1) / (2 * n))
    return {"n": N, "theta": 2 * np.arange(N) + 0.5, "delta": np.outer(phi, phi)}


def csr_to_dense(row_ptr, col_idx, vals, n) -> np.ndarray:
    """Dense column-major FP64 copy of a CSR matrix (values promoted exactly)."""
    d = np.zeros((n, n), order="F")
    for m in range(n):
        for q in range(row_ptr[m], row_ptr[m + 1]):
            d[m, col_idx[q]] += float(vals[q])
    return d


def batch_sizes(count: int, rep: int = 0, lo: int = 32, hi: int = 512) -> np.ndarray:
    rng = rng_for(4, rep)
    return np.rint(np.exp(rng.uniform(np.log(lo), np.log(hi), size=count))).astype(np.int64)


def batched_symmetric(count: int = 20_000, rep: int = 0, lo: int = 32,
                      hi: int = 512) -> list:
    """Independent dense symmetric problems of uneven size."""
    rng = rng_for(4, rep)
    sizes = np.rint(np.exp(rng.uniform(np.log(lo), np.log(hi), size=count))).astype(np.int64)
    lams = rng.uniform(0.01, 0.1, size=count)
    out = []
    for p in range(count):
        n = int(sizes[p])
        theta = np.arange(n, dtype=np.float64) + rng.uniform(-0.2, 0.2, size=n)
        delta = symmetric_gaussian(n, 1.0 / n, rng)
        out.append({"n": n, "theta": theta, "delta": delta, "lam": float(lams[p]),
                    "tol": 1e-12})
    return out


def served_hermitian(count: int, rate: float = 2000.0, rep: int = 0, lo: int = 64,
                     hi: int = 4096) -> list:
    """A Poisson request stream of dense complex Hermitian problems."""
    rng = rng_for(5, rep)
    gaps = rng.exponential(1.0 / rate, size=count)
    arrivals = np.cumsum(gaps)
    sizes = np.rint(np.exp(rng.uniform(np.log(lo), np.log(hi), size=count))).astype(np.int64)
    lams = rng.uniform(0.02, 0.08, size=count)
    out = []
    for p in range(count):
        n = int(sizes[p])
        out.append({"n": n, "arrival_s": float(arrivals[p]),
                    "theta": np.arange(n, dtype=np.float64),
                    "delta": hermitian_gaussian(n, 1.0 / n, rng),
                    "lam": float(lams[p]), "tol": 1e-12})
    return out


def served_pool(size: int = 48, rep: int = 0, lo: int = 64, hi: int = 4096) -> list:
    """Distinct served problems at the `size` stratified quantiles of the
    log-uniform size law on [lo, hi]: n_q = round(exp(ln lo + (q + 1/2) / size *
    ln(hi / lo))), theta_i = i, Hermitian Delta of variance 1/n."""
    rng = rng_for(5, 100 + rep)
    out = []
    for q in range(size):
        n = int(round(np.exp(np.log(lo) + (q + 0.5) / size * np.log(hi / lo))))
        out.append({"n": n, "theta": np.arange(n, dtype=np.float64),
                    "delta": hermitian_gaussian(n, 1.0 / n, rng)})
    return out


def served_stream(count: int, rate: float, pool_size: int, rep: int = 0) -> dict:
    """Poisson arrivals at `rate` per second (exponential gaps), the pool entry of
    each request (uniform over the pool) and its lambda ~ U[0.02, 0.08]."""
    rng = rng_for(5, 200 + rep)
    return {"arrival_s": np.cumsum(rng.exponential(1.0 / rate, size=count)),
            "pool": rng.integers(0, pool_size, size=count),
            "lam": rng.uniform(0.02, 0.08, size=count)}
