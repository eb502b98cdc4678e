"""Benchmark: full-spectrum DPT solves per second on one GB300 (and N GPUs, weak
scaling over independent problems).

Workload: the dense real unsymmetric problem of size n = 4096 (theta sorted
uniforms with every gap >= 0.5, Delta iid N(0, 1/n), lambda = 0.1), solved from
A_0 = I to a normalised residual <= 1e-12 (well below the 1e-10 the metric asks
for) with the mixed-precision path (tcgen05 products on FP16 operands with
power-of-two scales, FP32 accumulation, extended-precision state).  One step = one complete solve through the C ABI
with the inputs already resident in HBM; L2 is flushed between steps.

The JSON line also carries the plain-FP64 comparator (same problem, same
tolerance), the end-to-end number through the C ABI with pinned host buffers,
the roofline of the product kernel (timed per launch with CUDA events on the
stream it runs on), sampled SM clocks, and the CPU oracle timed on a bounded
sample of columns as a reported baseline.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N = 4096
WORKLOAD = "full-spectrum DPT, n=4096 dense real unsymmetric, lambda=0.1, tol=1e-12"
METRIC = "solves/s at residual<=1e-10 (mixed-precision DPT, n=4096)"
PROFILE = os.path.join(ROOT, "profiles", "k_gemm_epi_pair_n4096.md")
KERNEL_SRC = os.path.join(ROOT, "paper_2002_12872_gb300", "csrc", "dpt_full_mixed.cu")


STREAMS = 3   # default: independent solve streams per GPU in the timed throughput regions


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-check", action="store_true",
                    help="skip the oracle's error checks of the GPU results (never timed)")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the dominant (CSR and dense), batched and served workloads")
    ap.add_argument("--only", default="all",
                    choices=["all", "dominant", "dominant_dense", "homotopy", "rs",
                             "batched", "served", "served_pool", "full_variants"],
                    help="time one secondary workload alone and print its JSON object")
    ap.add_argument("--dense-n", type=int, default=32768,
                    help="dominant_dense: problem size")
    ap.add_argument("--streams", type=int, default=STREAMS,
                    help="independent solve streams (one host thread each) in the timed "
                         "throughput region of the headline solve")
    ap.add_argument("--pool-max-n", type=int, default=None,
                    help="served_pool: keep pool entries with n up to this size")
    return ap.parse_args()


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def kernel_hash():
    """Hash of the product kernels' section of their source file (from the section on
    the tensor-core iteration to the output section): the committed ncu summary names
    the hash it was taken with, so its traffic is only reported for that kernel code."""
    txt = open(KERNEL_SRC, "rb").read()
    a = txt.index(b"// The tensor-core iteration")
    b = txt.index(b"// Output: A (float-float -> FP64) and E of the returned iterate.")
    return hashlib.sha256(txt[a:b]).hexdigest()[:16]


def ncu_traffic():
    """DRAM bytes per launch of the product kernel from the committed ncu summary,
    or None if it is missing or was taken on a different version of the kernel."""
    if not os.path.exists(PROFILE):
        return None
    txt = open(PROFILE).read()
    m = re.search(r"dram_bytes_per_launch_full_size:\s*([0-9.eE+]+)", txt)
    h = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", txt)
    if not m or not h or h.group(1) != kernel_hash():
        return None
    return float(m.group(1))


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_init(args, backend=None):
    """Process group from the torchrun environment (RANK / LOCAL_RANK / WORLD_SIZE /
    MASTER_*): NCCL with one GPU per rank, or gloo where there is no GPU."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if backend is None:
            backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group("gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    """The largest of the ranks' values (the job's time is its slowest rank's)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, world, seconds_max):
    """Whole-job throughput of weak scaling: every rank processes units_per_rank
    independent units; the job takes the slowest rank's time."""
    return world * units_per_rank / seconds_max


# ---------------------------------------------------------------------------
# CPU oracle baseline (bounded sample of columns; each column is its own map)
# ---------------------------------------------------------------------------
def cpu_oracle(cfg, ncols, seed=0):
    import oracle
    oracle.build()
    rng = np.random.Generator(np.random.PCG64(seed))
    cols = np.sort(rng.choice(cfg["n"], size=ncols, replace=False))
    t0 = time.perf_counter()
    A, E, info = oracle.solve_full(cfg["theta"], cfg["delta"], cfg["lam"], tol=cfg["tol"],
                                   cols=cols)
    dt = time.perf_counter() - t0
    full = dt * cfg["n"] / ncols     # seconds for all n columns
    return 1.0 / full, dt, info


def run_reference(args, world, rank):
    """The oracle, as it stands, on this machine's host cores: each step solves a
    bounded sample of the same workload's columns (sized from a one-column
    calibration so the whole run stays within a few minutes); solves/s is scaled
    to the whole problem (all n columns)."""
    if rank != 0:
        return
    from paper_2002_12872_gb300 import inputs
    import oracle
    oracle.build()
    cores = oracle.set_threads(os.cpu_count() or 1)
    cfg = inputs.full_unsymmetric(n=N)
    _, t1, _ = cpu_oracle(cfg, 1, seed=12345)            # calibration, not timed
    budget = 150.0 / max(1, args.steps + args.warmup)   # seconds per step
    ncols = int(max(1, min(64, budget / max(t1, 1e-3))))
    walls = []
    for s in range(args.warmup + args.steps):
        v, dt, info = cpu_oracle(cfg, ncols, seed=s)
        if s >= args.warmup:
            walls.append(dt)
    wall = float(np.sum(walls))
    # a step solves ncols of the n columns (independent maps): ncols / n of a solve
    value = args.steps * (ncols / N) / wall
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * wall / args.steps,
            "ms_per_solve_equivalent": 1e3 / value, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": N, "lambda": cfg["lam"], "tol": 1e-12},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores,
                             "kind": "oracle",
                             "sample": f"{ncols} of {N} columns per step, scaled by n/{ncols}"},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline_sized(cfg, target_s=15.0, single_s=8.0):
    """The oracle on a column sample sized to about target_s seconds of work on all
    host threads, and on a smaller sample (about single_s seconds) on one thread."""
    import oracle
    oracle.build()
    cores = oracle.set_threads(os.cpu_count() or 1)
    _, t, _ = cpu_oracle(cfg, cores, seed=1)             # calibration
    ncols = int(min(cfg["n"], max(1, cores * max(1, round(target_s / max(t, 1e-3))))))
    v, dt, info = cpu_oracle(cfg, ncols, seed=2)
    oracle.set_threads(1)
    n1 = int(min(cfg["n"], max(1, round(single_s / max(t, 1e-3)))))
    v1, dt1, info1 = cpu_oracle(cfg, n1, seed=3)
    oracle.set_threads(cores)
    return {"value": v, "unit": "solves/s", "cores": cores, "kind": "oracle",
            "sample": f"{ncols} of {cfg['n']} columns ({dt:.1f} s on {cores} threads), "
                      f"scaled by n/{ncols}; status {info['status']}",
            "single_core": {"value": v1, "unit": "solves/s", "cores": 1,
                            "sample": f"{n1} of {cfg['n']} columns ({dt1:.1f} s on 1 thread), "
                                      f"scaled by n/{n1}; status {info1['status']}"}}


# ---------------------------------------------------------------------------
# The oracle as the checker: errors of GPU results against it (never timed)
# ---------------------------------------------------------------------------
def _unit(A):
    A = np.asarray(A)
    return A / np.linalg.norm(A, axis=0)


def checker_full(theta, delta, lam, A_cols, E_cols, cols, note):
    """Errors of GPU eigenpairs (columns `cols` of a full solve) against the oracle's
    map iterated to tol 1e-13 on the same columns (each column is its own map,
    Sec. II.B): |E - E_ora| / max(1, |E_ora|) and || a/|a| - a_ora/|a_ora| ||."""
    import oracle
    oracle.build()
    Ao, Eo, io = oracle.solve_full(theta, delta, lam, tol=1e-13, cols=np.asarray(cols))
    A_cols, E_cols = np.asarray(A_cols), np.asarray(E_cols)
    return {"max_eig_rel": float(np.max(np.abs(E_cols - Eo) / np.maximum(1.0, np.abs(Eo)))),
            "max_vec": float(np.max(np.linalg.norm(_unit(A_cols) - _unit(Ao), axis=0))),
            "columns": int(len(cols)), "sample": note, "oracle_status": io["status"]}


def tight_columns(theta, k=8):
    """The k columns whose nearest level is closest (the smallest gaps the map divides
    by)."""
    t = np.asarray(theta)
    if len(t) > 8192:
        o = np.argsort(t, kind="stable")
        d = np.diff(t[o])
        near = np.full(len(t), np.inf)
        near[o[:-1]] = np.minimum(near[o[:-1]], d)
        near[o[1:]] = np.minimum(near[o[1:]], d)
    else:
        g = np.abs(t[:, None] - t[None, :])
        np.fill_diagonal(g, np.inf)
        near = g.min(axis=0)
    return np.argsort(near, kind="stable")[:k]


# ---------------------------------------------------------------------------
# Secondary workloads (reported beside the headline)
# ---------------------------------------------------------------------------
DOM_BYTES_PER_ITER = None   # set from the workload: 8 B per nonzero + 36 B per row


def bench_dominant(dpt, inputs, dev, pk, steps=20, warmup=3, check=True):
    """Dominant eigenvector, n = 2e6 CSR with 16 nonzeros per row, lambda = 0.01.
    Algorithmic bytes per SpMV pass: FP32 value + int32 index per nonzero, and per
    row the row pointer (4 B), theta (8 B float-float), z read and written (8 + 8 B)
    and one gather of z (8 B)."""
    import torch
    cfg = inputs.dominant_csr()
    n = cfg["n"]
    t = lambda a: torch.tensor(np.ascontiguousarray(a), device=dev)
    th, rp, ci, va = t(cfg["theta"]), t(cfg["row_ptr"]), t(cfg["col_idx"]), t(cfg["vals"])
    z = torch.empty(n, dtype=torch.float64, device=dev)
    nnz = int(cfg["row_ptr"][-1])
    bytes_iter = 8.0 * nnz + 36.0 * n
    out = {"workload": "dominant eigenvector, CSR n=2e6, 16 nnz/row, lambda=0.01, tol=1e-12"}
    zo = Eo = None
    if check:
        import oracle
        oracle.build()
        zo, Eo, io = oracle.solve_dominant_csr(cfg["theta"], cfg["row_ptr"], cfg["col_idx"],
                                               cfg["vals"], cfg["lam"], tol=1e-13)
    for prec in ("mixed", "fp64"):
        for _ in range(warmup):
            dpt.solve_dominant(th, rp, ci, va, cfg["lam"], prec=prec, z_out=z, profile=True)
        torch.cuda.synchronize()
        stream = torch.cuda.current_stream(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        pm, pl, its = 0.0, 0, []
        e0.record(stream)
        for _ in range(steps):
            _, E, info = dpt.solve_dominant(th, rp, ci, va, cfg["lam"], prec=prec, z_out=z)
            its.append(info["iters"])
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        # per-pass SpMV durations: a separate pass with per-launch CUDA events
        for _ in range(3):
            _, E, info = dpt.solve_dominant(th, rp, ci, va, cfg["lam"], prec=prec, z_out=z,
                                            profile=True)
            pm += info["product_ms"]
            pl += info["product_launches"]
        per_pass = pm / max(1, pl)
        gbs = bytes_iter / (per_pass * 1e-3) / 1e9
        out[prec] = {"solves_per_s": 1e3 / ms, "ms_per_solve": ms, "iters": float(np.mean(its)),
                     "spmv_ms_per_pass": per_pass, "achieved_GBs": gbs,
                     "hbm_frac": gbs / pk["hbm_gbs"], "E": E}
        if zo is not None:
            zz = z.cpu().numpy()
            out[prec]["errors_vs_oracle"] = {
                "eig_rel": abs(E - Eo) / max(1.0, abs(Eo)),
                "vec": float(np.linalg.norm(zz / np.linalg.norm(zz) - zo / np.linalg.norm(zo))),
                "sample": "the whole eigenvector (oracle: single-vector map to tol 1e-13)"}
    out["roofline"] = {"bound": "hbm", "kernel": "k_dom_iter (+ y* pre-pass)",
                       "achieved": out["mixed"]["achieved_GBs"], "peak": pk["hbm_gbs"],
                       "unit": "GB/s", "frac": out["mixed"]["hbm_frac"],
                       "algorithmic_bytes_per_pass": bytes_iter}
    # the gather ceiling: the pass's index stream and random 8-byte gathers of the
    # (L2-resident, 16 MB) float-float iterate without its arithmetic or value loads
    zprobe = torch.ones((n, 2), dtype=torch.float32, device=dev)
    gms = dpt.probe_gather(rp, ci, zprobe, reps=20)
    out["gather_ceiling"] = {
        "ms_per_pass": gms,
        "gathers_per_s": nnz / (gms * 1e-3),
        "spmv_frac_of_ceiling": gms / out["mixed"]["spmv_ms_per_pass"],
        "probe": "dpt_probe_gather: same grid, row groups, index stream and 8-byte gathers "
                 f"({nnz / 1e6:.0f} M per pass into a {8 * n / 1e6:.0f} MB vector), no "
                 "arithmetic, no value loads"}
    # a solve against its passes: set-up, checks, host reads and the output outside them
    out["solve_over_passes"] = out["mixed"]["ms_per_solve"] / (
        (out["mixed"]["iters"] + 1) * out["mixed"]["spmv_ms_per_pass"])
    return out


def bench_dominant_dense(dpt, inputs, dev, pk, steps=10, warmup=3, n=32768):
    """Dominant eigenvector with a dense FP64 Delta (GEMV form), n = 32768, lambda =
    0.1.  Algorithmic bytes per GEMV pass: Delta once (8 n^2) and z (8 n).  Delta
    (8.6 GB) is far larger than L2, so no flush is needed between passes."""
    import torch
    cfg = inputs.dominant_dense_device(n=n, device=dev)
    th, D, lam = cfg["theta"], cfg["delta"], cfg["lam"]
    z = torch.empty(n, dtype=torch.float64, device=dev)
    bytes_pass = 8.0 * n * n + 8.0 * n
    out = {"workload": f"dominant eigenvector, dense FP64 n={n}, Delta iid N(0,1/n), "
                       f"theta U[0,1] with theta_0=2, lambda={lam}, tol=1e-12"}
    for prec in ("mixed", "fp64"):
        for _ in range(warmup):
            dpt.solve_dominant_dense(th, D, lam, prec=prec, z_out=z, profile=True)
        torch.cuda.synchronize()
        stream = torch.cuda.current_stream(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        pm, pl, its = 0.0, 0, []
        e0.record(stream)
        for _ in range(steps):
            _, E, info = dpt.solve_dominant_dense(th, D, lam, prec=prec, z_out=z)
            its.append(info["iters"])
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        # per-pass GEMV durations: a separate pass with per-launch CUDA events
        for _ in range(2):
            _, E, info = dpt.solve_dominant_dense(th, D, lam, prec=prec, z_out=z, profile=True)
            pm += info["product_ms"]
            pl += info["product_launches"]
        per_pass = pm / max(1, pl)
        gbs = bytes_pass / (per_pass * 1e-3) / 1e9
        out[prec] = {"solves_per_s": 1e3 / ms, "ms_per_solve": ms, "iters": float(np.mean(its)),
                     "gemv_ms_per_pass": per_pass, "achieved_GBs": gbs,
                     "hbm_frac": gbs / pk["hbm_gbs"], "E": E}
    # the non-autonomous iteration (lambda (1 - 0.5^k)) on the same problem: same fixed
    # point, more steps
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dpt.solve_dominant_dense(th, D, lam, z_out=z, ramp_alpha=0.5)
    torch.cuda.synchronize()
    e0.record(stream)
    _, Er, infor = dpt.solve_dominant_dense(th, D, lam, z_out=z, ramp_alpha=0.5)
    e1.record(stream)
    torch.cuda.synchronize()
    msr = e0.elapsed_time(e1)
    out["ramp_alpha_0.5"] = {"solves_per_s": 1e3 / msr, "ms_per_solve": msr,
                             "iters": infor["iters"], "status": infor["status"],
                             "E_minus_autonomous": Er - out["mixed"]["E"]}
    # polisher: start from the solution perturbed by 1e-4 (relative, seeded)
    g = torch.Generator(device=dev)
    g.manual_seed(77)
    zs = z.clone() * (1.0 + 1e-4 * torch.randn(n, generator=g, device=dev, dtype=torch.float64))
    dpt.solve_dominant_dense(th, D, lam, z_out=z, start=zs)
    torch.cuda.synchronize()
    e0.record(stream)
    _, Es, infos = dpt.solve_dominant_dense(th, D, lam, z_out=z, start=zs)
    e1.record(stream)
    torch.cuda.synchronize()
    mss = e0.elapsed_time(e1)
    out["start_1e-4"] = {"solves_per_s": 1e3 / mss, "ms_per_solve": mss,
                         "iters": infos["iters"], "status": infos["status"],
                         "E_minus_autonomous": Es - out["mixed"]["E"]}
    out["roofline"] = {"bound": "hbm", "kernel": "k_dd_gemv (float-float GEMV)",
                       "achieved": out["mixed"]["achieved_GBs"], "peak": pk["hbm_gbs"],
                       "unit": "GB/s", "frac": out["mixed"]["hbm_frac"],
                       "algorithmic_bytes_per_pass": bytes_pass}
    del D, cfg
    torch.cuda.empty_cache()
    return out


def bench_full_variants(dpt, inputs, dev, reps=5, check=True):
    """The mixed full solve of the headline workload (n = 4096) with the generalised
    start (the polisher of the closing remark of Sec. II.H: the first increment is the
    start's offset from I) and with the non-autonomous iteration (ramp alpha = 0.5):
    time per solve, map applications, FP64 steps, against the solve from I."""
    import torch
    cfg = inputs.full_unsymmetric(n=N)
    th = torch.tensor(cfg["theta"], device=dev)
    D = dpt.colmajor_tensor(cfg["delta"], dev)
    Aref, _, _ = dpt.solve_full(th, D, cfg["lam"])
    g = torch.Generator(device=dev)
    g.manual_seed(2024)
    pert = Aref * (1.0 + 1e-6 * torch.randn(Aref.shape, generator=g, device=dev,
                                            dtype=torch.float64))
    A = torch.empty((N, N), dtype=torch.float64, device=dev).t()
    E = torch.empty(N, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    out = {"workload": WORKLOAD}
    rng_c = np.random.Generator(np.random.PCG64(11))
    ccols = np.unique(np.concatenate([rng_c.choice(N, 16, replace=False),
                                      tight_columns(cfg["theta"], 8)]))
    cases = {"from_identity": {}, "start_solution_x_(1+1e-6_N(0,1))": {"start": pert},
             "start_solution": {"start": Aref}, "ramp_alpha_0.5": {"ramp_alpha": 0.5}}
    for name, kw in cases.items():
        dpt.solve_full(th, D, cfg["lam"], A_out=A, E_out=E, **kw)      # warm-up
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        r = 1 if "ramp" in name else reps
        e0.record(stream)
        for _ in range(r):
            _, _, info = dpt.solve_full(th, D, cfg["lam"], A_out=A, E_out=E, **kw)
        e1.record(stream)
        torch.cuda.synchronize()
        out[name] = {"ms_per_solve": e0.elapsed_time(e1) / r, "iters": info["iters"],
                     "fp64_iters": info["fp64_iters"], "refined_cols": info["refined_cols"],
                     "status": info["status"],
                     "max_abs_diff_to_solution": float((A - Aref).abs().max())}
        if check:
            ct = torch.tensor(ccols, device=dev)
            out[name]["errors_vs_oracle"] = checker_full(
                cfg["theta"], cfg["delta"], cfg["lam"], A[:, ct].cpu().numpy(),
                E[ct].cpu().numpy(), ccols, "16 seeded columns and the 8 with the smallest "
                "gaps; oracle (autonomous map) to tol 1e-13")
    return out


def bench_homotopy(dpt, dev, n=2048, lam=2.5, stages=3, steps=3):
    """Homotopy continuation (lambda in `stages` steps with a change of basis) on a
    seeded symmetric problem, theta_i = i, Delta = (S + S^T)/sqrt(2) with S iid
    N(0, 1/n), beside the direct solve of the same problem.  The basis changes are
    FP64 matrix products (2 n^3 flop each: six per stage, three in the last, plus
    the FP64 refinement steps of the last stage)."""
    import torch
    rng = np.random.Generator(np.random.PCG64(2002_12872 + 7000))
    th_h = np.arange(n, dtype=float)
    S = rng.standard_normal((n, n)) / np.sqrt(n)
    D_h = (S + S.T) / np.sqrt(2)
    th = torch.tensor(th_h, device=dev)
    D = dpt.colmajor_tensor(D_h, dev)
    stream = torch.cuda.current_stream(dev)
    out = {"workload": f"homotopy continuation, symmetric n={n}, theta_i=i, "
                       f"Delta GOE-like N(0,1/n), lambda={lam}, {stages} stages, tol=1e-12"}
    for name, fn in (("direct", lambda: dpt.solve_full(th, D, lam, max_iter=2000, check=False)),
                     ("homotopy", lambda: dpt.solve_homotopy(th, D, lam, stages, max_iter=2000,
                                                             check=False))):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            _, E, info = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        out[name] = {"ms_per_solve": ms, "solves_per_s": 1e3 / ms, "iters": info["iters"],
                     "status": info["status"]}
    gemms = 6 * stages - 3
    out["homotopy"]["fp64_basis_gemm_tflop"] = gemms * 2.0 * n**3 / 1e12
    del D
    torch.cuda.empty_cache()
    return out


def bench_rs_comparator(dpt, inputs, dev, N=100, big=2000):
    """The paper's D-PT vs RS comparison (Sec. II.F) on the GPU, delta-potential
    oscillator: for N = 100 the D-PT iterations (plain FP64 map) and the RS orders
    (dpt_rs_series, FP64) needed to reach 1e-12 of the converged eigenvectors at
    lambda = 1.5, and the RS error growth at lambda = 2.5; for N = `big` the time of a
    D-PT solve (mixed and FP64) and of 70 RS orders at lambda = 1.5."""
    import torch
    w = inputs.delta_oscillator(N)
    th = torch.tensor(w["theta"], device=dev)
    D = dpt.colmajor_tensor(w["delta"], dev)
    out = {"workload": f"delta-potential oscillator (Sec. II.F), N={N} and N={big}"}
    A, _, info = dpt.solve_full(th, D, 1.5, prec="fp64", tol=1e-14, max_iter=500)
    A = A.cpu().numpy()
    kd = next((k for k in range(1, 200)
               if np.linalg.norm(dpt.solve_full(th, D, 1.5, prec="fp64", tol=1e-300, max_iter=k,
                                                check=False)[0].cpu().numpy() - A) < 1e-12), None)
    kr = next((k for k in range(5, 201, 5)
               if np.linalg.norm(dpt.rs_series(th, D, 1.5, k)[0].cpu().numpy() - A) < 1e-12), None)
    A25, _, _ = dpt.solve_full(th, D, 2.5, prec="fp64", tol=1e-13, max_iter=3000)
    A25 = A25.cpu().numpy()
    errs = {k: float(np.linalg.norm(dpt.rs_series(th, D, 2.5, k)[0].cpu().numpy() - A25))
            for k in (20, 40, 60)}
    out["N100"] = {"lambda_1.5": {"dpt_iterations_to_1e-12": kd, "rs_orders_to_1e-12": kr},
                   "lambda_2.5": {"rs_error_by_order": errs, "dpt_status": "OK"}}
    w = inputs.delta_oscillator(big)
    th = torch.tensor(w["theta"], device=dev)
    D = dpt.colmajor_tensor(w["delta"], dev)
    stream = torch.cuda.current_stream(dev)
    timing = {}
    for name, fn in (("dpt_mixed", lambda: dpt.solve_full(th, D, 1.5, max_iter=500)),
                     ("dpt_fp64", lambda: dpt.solve_full(th, D, 1.5, prec="fp64", max_iter=500)),
                     ("rs_70_orders", lambda: dpt.rs_series(th, D, 1.5, 70))):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        timing[name] = {"ms": e0.elapsed_time(e1)}
        if name.startswith("dpt"):
            timing[name]["iters"] = r[2]["iters"]
            # the mixed solve of this strongly coupled problem ends with plain FP64
            # map steps (its float recursion cannot vouch for 1e-12 here)
            timing[name]["fp64_iters"] = r[2].get("fp64_iters", 0)
    out[f"N{big}"] = timing
    return out


def bench_batched(dpt, inputs, dev, pk, steps=3, warmup=2, check=True, fp64_tflops=None):
    """20,000 independent symmetric problems, n log-uniform in [32, 512], one
    grouped solve per step (inputs resident in HBM; the pointer arrays of the call
    are built once, outside the timed region).

    Roofline: at these sizes the grouped product is bound by its epilogue's memory
    traffic, so it is quoted against HBM with the algorithmic bytes of one map
    application per matrix element: read A (float-float, 8 B), the carried remainder
    (4 B), the previous increment (2 B) and the S BF16 slices of Delta (2 S B); write
    A (8 B), the remainder (4 B) and the new increment (2 B): 28 + 2 S bytes, summed
    over every problem's iterations (its slice count per product from dpt_info) and
    divided by the product kernels' summed device time (per-launch CUDA events, in a
    separate pass from the timed solves)."""
    import torch
    probs = inputs.batched_symmetric(count=20000)
    th = [torch.tensor(p["theta"], device=dev) for p in probs]
    D = [dpt.colmajor_tensor(p["delta"], dev) for p in probs]
    lams = [p["lam"] for p in probs]
    batch = dpt.Batch(th, D, lams)          # argument arrays built once, outside the timing
    # tile shape (grouped product form) chosen by the library's tuner on this group,
    # outside the timing; the timed solves use it
    try:
        form, tune_ms = batch.tune()
    except RuntimeError as e:               # the default form then
        form, tune_ms = None, {"error": str(e)}
    for _ in range(warmup):
        batch.solve()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        _, _, infos = batch.solve()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    # per-launch product times: a separate pass (events recorded inside the graphs)
    As, Es, pinfos = batch.solve(profile=True)
    prod_ms = pinfos[0]["product_ms"]
    its = [i["iters"] for i in infos]
    n3 = float(np.sum([2.0 * p["n"] ** 3 for p in probs]))
    nn = np.array([p["n"] for p in probs], dtype=float)
    bytes_alg = float(np.sum(nn ** 2 * (28.0 * np.array(its) +
                                        2.0 * np.array([i["slice_gemms"] for i in infos]))))
    gbs = bytes_alg / (prod_ms * 1e-3) / 1e9
    # the plain FP64 map cannot beat its FP64 pipe: sum over the problems of
    # 2 n^3 flop per iteration (the same iteration counts) at the measured FP64 rate
    f64 = fp64_tflops if fp64_tflops else 1.25
    flop64 = float(np.sum(2.0 * nn ** 3 * np.array(its)))
    ceiling64 = len(probs) / (flop64 / (f64 * 1e12))
    # plain FP64 map on a stratified sample (every 200th problem in size order), one
    # solve at a time: the comparator; the sample's mean time per problem estimates
    # the batch's
    order = np.argsort([p["n"] for p in probs])
    sample = [int(q) for q in order[::200]]
    for q in sample[:3]:
        dpt.solve_full(th[q], D[q], lams[q], prec="fp64")
    torch.cuda.synchronize()
    e0.record(stream)
    for q in sample:
        dpt.solve_full(th[q], D[q], lams[q], prec="fp64")
    e1.record(stream)
    torch.cuda.synchronize()
    ms64 = e0.elapsed_time(e1)
    fp64 = {"solves_per_s_estimated": len(sample) * 1e3 / ms64,
            "sample": f"{len(sample)} problems (every 200th by size), one solve at a time, "
                      f"{ms64:.0f} ms",
            "ceiling_solves_per_s": ceiling64,
            "ceiling": f"sum of 2 n^3 x iterations over the batch at {f64:.2f} TFLOP/s "
                       f"(the measured FP64 GEMM rate): no plain FP64 map can be faster"}
    errs = None
    if check:
        samp = [int(q) for q in order[::1667]]          # 12 problems across the sizes
        e = [checker_full(probs[q]["theta"], probs[q]["delta"], probs[q]["lam"],
                          As[q].cpu().numpy(), Es[q].cpu().numpy(), np.arange(probs[q]["n"]),
                          "") for q in samp]
        errs = {"max_eig_rel": max(x["max_eig_rel"] for x in e),
                "max_vec": max(x["max_vec"] for x in e),
                "sample": f"{len(samp)} problems (every 1667th by size), all columns, oracle "
                          f"to tol 1e-13",
                "n": [probs[q]["n"] for q in samp]}
    return {"workload": "20,000 dense symmetric problems, n log-uniform [32, 512], "
                        "lambda U[0.01, 0.1], tol=1e-12",
            "solves_per_s": 20000 * 1e3 / ms, "ms_per_batch": ms,
            "grouped_form": form,
            "tuner_product_ms_by_form": {str(f): v for f, v in tune_ms.items()},
            "fp64_comparator": fp64,
            "iters_mean": float(np.mean(its)), "iters_max": int(np.max(its)),
            "product_ms_per_batch": prod_ms,
            "product_ms_per_launch": prod_ms / max(1, pinfos[0]["product_launches"]),
            "algorithmic_tflop_per_iteration": n3 / 1e12,
            "roofline": {"bound": "hbm", "kernel": "k_g_gemm_epi (grouped product + update)",
                         "achieved": gbs, "peak": pk["hbm_gbs"], "unit": "GB/s",
                         "frac": gbs / pk["hbm_gbs"],
                         "algorithmic": "(28 + 2 S) bytes per element and iteration",
                         "algorithmic_bytes_per_batch": bytes_alg},
            "errors_vs_oracle": errs,
            "all_converged": all(i["status"] == "OK" for i in infos)}


def bench_served_pool(dpt, inputs, dev, pk, steps=3, warmup=2, max_n=None, check=True):
    """The served problem mix (the 48-entry pool of complex Hermitian problems,
    lambda = 0.05) as one grouped solve: the complex tcgen05 product's throughput
    without the request loop.  max_n keeps only pool entries up to that size."""
    import torch
    pool = [p for p in inputs.served_pool(48) if max_n is None or p["n"] <= max_n]
    th = [torch.tensor(p["theta"], device=dev) for p in pool]
    D = [dpt.colmajor_tensor(p["delta"], dev) for p in pool]
    lams = [0.05] * len(pool)
    batch = dpt.Batch(th, D, lams)
    for _ in range(warmup):
        batch.solve()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        _, _, infos = batch.solve()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    # per-launch product times: a separate pass (events recorded inside the graphs)
    As, Es, pinfos = batch.solve(profile=True)
    prod_ms = pinfos[0]["product_ms"]
    pl = pinfos[0]["product_launches"]
    ns = np.array([p["n"] for p in pool], dtype=float)
    it = np.array([i["iters"] for i in infos])
    sl = np.array([i["slice_gemms"] for i in infos])
    alg = float(np.sum(8 * ns**3 * it)) / (prod_ms * 1e-3) / 1e12
    errs = None
    if check:
        # three small entries in full, and eight columns of the largest one
        small = [q for q in np.argsort(ns, kind="stable")[:3]]
        big = int(np.argmax(ns))
        e = [checker_full(pool[q]["theta"], pool[q]["delta"], 0.05, As[q].cpu().numpy(),
                          Es[q].cpu().numpy(), np.arange(pool[q]["n"]), "") for q in small]
        nb = pool[big]["n"]
        cb = np.unique(np.concatenate([[0, nb - 1], np.linspace(1, nb - 2, 6).astype(int)]))
        e.append(checker_full(pool[big]["theta"], pool[big]["delta"], 0.05,
                              As[big][:, torch.tensor(cb, device=dev)].cpu().numpy(),
                              Es[big].cpu().numpy()[cb], cb, ""))
        errs = {"max_eig_rel": max(x["max_eig_rel"] for x in e),
                "max_vec": max(x["max_vec"] for x in e),
                "sample": f"the 3 smallest entries (all columns) and {len(cb)} columns of the "
                          f"largest (n = {nb}); oracle (complex128) to tol 1e-13"}
    return {"workload": f"{len(pool)} served complex Hermitian problems (pool entries"
                        f"{'' if max_n is None else f' with n <= {max_n}'}), lambda 0.05, one grouped solve",
            "solves_per_s": len(pool) * 1e3 / ms, "ms_per_batch": ms,
            "product_ms_per_batch": prod_ms, "product_launches": pl,
            "executed_tflops_in_product": float(np.sum(8 * ns**3 * sl)) / (prod_ms * 1e-3) / 1e12,
            "algorithmic_tflops_in_product": alg,
            "roofline": {"bound": "tensor", "kernel": "k_g_gemm_epi<complex> (real embedding)",
                         "achieved": alg, "peak": pk["bf16_tflops"], "unit": "TFLOP/s",
                         "frac": alg / pk["bf16_tflops"],
                         "algorithmic": "8 n^3 flop per problem and iteration",
                         "peak_source": "bf16_tflops (burst), measured"},
            "errors_vs_oracle": errs,
            "iters_max": int(it.max()), "all_converged": all(i["status"] == "OK" for i in infos)}


def _run_stream(srv, stream, th, D, outs, wait_all=True):
    """Open-loop submission at the scheduled arrival times; returns per-request
    (info, lateness) and the wall time from the first arrival to the last result."""
    arr, pool, lam = stream["arrival_s"], stream["pool"], stream["lam"]
    ids, late = [], []
    t0 = time.perf_counter()
    for k in range(len(arr)):
        while True:
            now = time.perf_counter() - t0
            if now >= arr[k]:
                break
            if arr[k] - now > 2e-3:
                time.sleep(0.5e-3)
        late.append(time.perf_counter() - t0 - arr[k])
        A, E = outs(k)
        ids.append(srv.submit(th[pool[k]], D[pool[k]], float(lam[k]), A_out=A, E_out=E))
    infos = [srv.wait(i)[2] for i in ids]
    wall = time.perf_counter() - t0
    return infos, np.array(late), wall


def bench_served(dpt, inputs, dev, rates=(250, 500, 1000, 2000), window_s=1.0, pool_size=48,
                 check=True):
    """Served complex Hermitian problems (n log-uniform in [64, 4096], theta_i = i,
    Delta of variance 1/n, lambda U[0.02, 0.08]) arriving as Poisson streams; the
    requests draw their matrices from a pool of 48 distinct problems at stratified
    size quantiles (inputs resident in HBM; each request its own lambda and its
    own outputs).  Per rate: goodput, p50/p99 submit-to-result latency, queue depth
    and memory use of the solve server."""
    import torch
    pool = inputs.served_pool(pool_size)
    th = [torch.tensor(p["theta"], device=dev) for p in pool]
    D = [dpt.colmajor_tensor(p["delta"], dev) for p in pool]
    ns = np.array([p["n"] for p in pool])
    out = {"workload": "served complex Hermitian, n log-uniform [64, 4096] (pool of 48 at "
                       "stratified quantiles), theta_i = i, Delta var 1/n, lambda U[0.02, 0.08], "
                       "tol=1e-12, Poisson arrivals",
           "budget_bytes": 96 << 30, "max_active": 256, "rates": {}}
    srv = dpt.Server(hbm_budget=96 << 30, max_active=256)
    try:
        # warm-up: every pool entry once
        warm = [srv.submit(th[q], D[q], 0.05) for q in range(pool_size)]
        for i in warm:
            srv.wait(i)
        for rate in rates:
            st = inputs.served_stream(int(rate * window_s), rate, pool_size, rep=int(rate))
            cnt = len(st["pool"])
            bufs = [(torch.empty((ns[q], ns[q]), dtype=torch.complex128, device=dev).t(),
                     torch.empty(ns[q], dtype=torch.complex128, device=dev)) for q in st["pool"]]
            torch.cuda.synchronize()
            s0 = srv.stats()
            infos, late, wall = _run_stream(srv, st, th, D, lambda k: bufs[k])
            s1 = srv.stats()
            lat = np.array([i["seconds"] for i in infos])
            ok = sum(i["status"] == "OK" for i in infos)
            flop = sum(8.0 * float(ns[q]) ** 3 * i["iters"] for q, i in zip(st["pool"], infos))
            out["rates"][str(rate)] = {
                "requests": cnt, "completed_ok": ok, "window_s": float(st["arrival_s"][-1]),
                "goodput_per_s": ok / wall, "wall_s": wall,
                "p50_ms": 1e3 * float(np.percentile(lat, 50)),
                "p99_ms": 1e3 * float(np.percentile(lat, 99)),
                "max_ms": 1e3 * float(lat.max()),
                "submit_lateness_max_ms": 1e3 * float(late.max()),
                "max_queued": s1["max_queued"], "hbm_peak_gb": s1["hbm_peak"] / 1e9,
                "steps": s1["steps"] - s0["steps"],
                "iters_mean": float(np.mean([i["iters"] for i in infos])),
                "algorithmic_tflops": flop / wall / 1e12}
            if rate == rates[-1]:
                # sampled requests equal their solo solves bit for bit
                rng = np.random.Generator(np.random.PCG64(5))
                same, errs, nsamp = [], [], []
                for k in rng.choice(cnt, size=4, replace=False):
                    q = st["pool"][k]
                    nsamp.append(int(ns[q]))
                    A1, E1, _ = dpt.solve_full(th[q], D[q], float(st["lam"][k]))
                    same.append(bool(torch.equal(A1, bufs[k][0]) and torch.equal(E1, bufs[k][1])))
                    if check:
                        # the request's own result against the oracle (all columns up to
                        # n = 256, else eight spread over the spectrum)
                        nq = int(ns[q])
                        cq = (np.arange(nq) if nq <= 256 else np.unique(
                            np.linspace(0, nq - 1, 8).astype(int)))
                        Aq = bufs[k][0][:, torch.tensor(cq, device=dev)].cpu().numpy()
                        errs.append(checker_full(pool[q]["theta"], pool[q]["delta"],
                                                 float(st["lam"][k]), Aq,
                                                 bufs[k][1].cpu().numpy()[cq], cq, ""))
                out["sampled_equal_to_solo"] = same
                if errs:
                    out["errors_vs_oracle"] = {
                        "max_eig_rel": max(x["max_eig_rel"] for x in errs),
                        "max_vec": max(x["max_vec"] for x in errs),
                        "sample": "4 requests of the 2,000 req/s window (their own outputs; "
                                  "all columns up to n = 256, else 8), oracle (complex128) to "
                                  "tol 1e-13",
                        "n": nsamp}
            del bufs
        # end to end at the highest rate: pinned host inputs and outputs (requests on
        # the same pool entry share their host output buffers)
        rate = rates[-1]
        th_h = [torch.tensor(p["theta"]).pin_memory() for p in pool]
        D_h = [dpt.colmajor_tensor(p["delta"], pin=True) for p in pool]
        ob = [(torch.empty((n, n), dtype=torch.complex128).pin_memory().t(),
               torch.empty(n, dtype=torch.complex128).pin_memory()) for n in ns]
        st = inputs.served_stream(int(rate * window_s / 2), rate, pool_size, rep=7)
        infos, late, wall = _run_stream(srv, st, th_h, D_h, lambda k: ob[st["pool"][k]])
        lat = np.array([i["seconds"] for i in infos])
        nb = sum(16.0 * float(ns[q]) ** 2 for q in st["pool"])
        out["e2e_host_buffers"] = {
            "rate": rate, "requests": len(infos),
            "goodput_per_s": sum(i["status"] == "OK" for i in infos) / wall,
            "p50_ms": 1e3 * float(np.percentile(lat, 50)),
            "p99_ms": 1e3 * float(np.percentile(lat, 99)),
            "h2d_bytes_per_request": nb / len(infos), "d2h_bytes_per_request": nb / len(infos)}
    finally:
        srv.close()
    # solo solves of a stratified sample of the pool: mixed vs plain FP64
    samp = list(range(3, pool_size, 8))
    t = {"mixed": [], "fp64": []}
    for prec in ("mixed", "fp64"):
        dpt.solve_full(th[samp[0]], D[samp[0]], 0.05, prec=prec)      # warm-up
        for q in samp:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, _, info = dpt.solve_full(th[q], D[q], 0.05, prec=prec)
            torch.cuda.synchronize()
            t[prec].append(time.perf_counter() - t0)
    out["solo_sample"] = {
        "n": [int(ns[q]) for q in samp],
        "mixed_s": t["mixed"], "fp64_s": t["fp64"],
        "mixed_solves_per_s_est": 1.0 / float(np.mean(t["mixed"])),
        "fp64_solves_per_s_est": 1.0 / float(np.mean(t["fp64"])),
        "note": "one solo solve per sampled pool entry (every 8th of 48, stratified); "
                "the mean over the sample estimates the mean over the size law"}
    return out


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------


def run_streams(calls, streams, nsolves):
    """nsolves calls spread over len(calls) streams, one host thread each (every call
    returns after its own solve, so one solve's host work and set-up kernels overlap
    another's products).  Device time from an event on the first stream, which every
    other stream waits for, to one after all of them; returns (seconds, infos)."""
    import torch
    ns = len(calls)
    per = [nsolves // ns + (1 if k < nsolves % ns else 0) for k in range(ns)]
    infos = [[] for _ in range(ns)]
    errors = []

    def worker(k):
        try:
            for _ in range(per[k]):
                infos[k].append(calls[k]())
        except Exception as e:   # re-raised on the calling thread
            errors.append(e)

    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(streams[0])
    for st in streams[1:]:
        st.wait_event(t0)
    if ns == 1:
        worker(0)   # one stream: on this thread
    else:
        threads = [threading.Thread(target=worker, args=(k,)) for k in range(ns)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
    if errors:
        raise errors[0]
    for st in streams[1:]:
        e = torch.cuda.Event()
        e.record(st)
        streams[0].wait_event(e)
    t1.record(streams[0])
    torch.cuda.synchronize()
    return t0.elapsed_time(t1) / 1e3, [i for lst in infos for i in lst]


def run_ours(args, world, rank, local):
    import torch

    from paper_2002_12872_gb300 import build, dpt, inputs

    build.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    cfg = inputs.full_unsymmetric(n=N, rep=rank)
    th = torch.tensor(cfg["theta"], device=dev)
    D = dpt.colmajor_tensor(cfg["delta"], dev)                      # column-major, no copy per call
    A = torch.empty((N, N), dtype=torch.float64, device=dev).t()
    E = torch.empty((N,), dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def solve(prof=False, prec="mixed"):
        return dpt.solve_full(th, D, cfg["lam"], prec=prec, tol=1e-12, A_out=A, E_out=E,
                              profile=prof)

    # the timed calls go through the C ABI with their arguments marshalled once, and
    # record no per-launch events (profile off)
    prepared = dpt.FullSolve(th, D, cfg["lam"], prec="mixed", tol=1e-12, A_out=A, E_out=E)
    for _ in range(max(3, args.warmup)):
        prepared.solve()
    torch.cuda.synchronize()

    # latency: back-to-back solves on one stream, L2 flushed before each (untimed flush)
    nlat = max(10, min(args.steps, 200))
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(nlat)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(nlat)]
    for k in range(nlat):
        flush.zero_()
        starts[k].record(stream)
        prepared.solve()
        ends[k].record(stream)
    torch.cuda.synchronize()
    step_ms = np.array([s.elapsed_time(e) for s, e in zip(starts, ends)])
    one_stream = {"value": job_throughput(nlat, 1, float(step_ms.sum()) / 1e3),
                  "unit": "solves/s", "solves": nlat,
                  "l2": "flushed before each solve (256 MB write, untimed)"}

    # throughput, the timed region: K solves over the independent solve streams (--streams);
    # a solve's working set (Delta 134 MB, about 0.5 GB of iterate state) exceeds L2,
    # so nothing is flushed between solves
    nstr = args.streams
    if nstr < 1:
        raise ValueError("--streams must be at least 1")
    sts = [stream] + [torch.cuda.Stream(dev) for _ in range(nstr - 1)]
    outs = [(A, E)] + [(torch.empty((N, N), dtype=torch.float64, device=dev).t(),
                        torch.empty((N,), dtype=torch.float64, device=dev))
                       for _ in range(nstr - 1)]
    # each stream its own copy of the inputs (no stream reads lines another just loaded)
    ins = [(th, D)] + [(th.clone(), dpt.colmajor_tensor(cfg["delta"], dev))
                       for _ in range(nstr - 1)]
    solvers = [prepared] + [dpt.FullSolve(ins[k][0], ins[k][1], cfg["lam"], prec="mixed",
                                          tol=1e-12, A_out=outs[k][0], E_out=outs[k][1],
                                          stream=sts[k].cuda_stream)
                            for k in range(1, nstr)]
    for f in solvers[1:]:
        for _ in range(max(3, args.warmup)):
            f.solve()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        barrier(world)
        torch.cuda.synchronize()
        wall0 = time.perf_counter()
        total_s, tinfos = run_streams([f.solve for f in solvers], sts, args.steps)
        wall = time.perf_counter() - wall0
        barrier(world)
    launches = sum(i["launches"] for i in tinfos)
    iters = [i["iters"] for i in tinfos]
    refined = max(i["refined_cols"] for i in tinfos)
    bad = [i for i in tinfos if i["status"] != "OK"]
    if bad:
        raise RuntimeError(f"solve failed: {bad[0]}")
    same = all(torch.equal(outs[0][0], o[0]) and torch.equal(outs[0][1], o[1]) for o in outs[1:])
    total_s = max_over_ranks(total_s, world)
    value = job_throughput(args.steps, world, total_s)

    # per-launch durations of the product kernel: a separate, untimed pass whose solves
    # record CUDA events around every product launch on the stream it runs on
    profiled = dpt.FullSolve(th, D, cfg["lam"], prec="mixed", tol=1e-12, A_out=A, E_out=E,
                             profile=True)
    prod_ms, prod_launches, slices, pair = 0.0, 0, [], 0
    for _ in range(max(10, min(args.steps, 50))):
        flush.zero_()
        info = profiled.solve()
        prod_ms += info["product_ms"]
        prod_launches += info["product_launches"]
        slices.append(info["slice_gemms"] / max(1, info["product_launches"]))
        pair = info["cta_pair"]
    torch.cuda.synchronize()

    # verification of the last solve: explicit FP64 residual of sampled columns
    rng = np.random.Generator(np.random.PCG64(7))
    cols = torch.tensor(np.sort(rng.choice(N, 16, replace=False)), device=dev)
    Ac = A[:, cols]
    M_A = th[:, None] * Ac + cfg["lam"] * (D @ Ac)
    R = M_A - Ac * E[cols][None, :]
    s = float(th.abs().max()) + cfg["lam"] * float(D.abs().sum(1).max())
    rho = float((R.norm(dim=0) / (s * Ac.norm(dim=0))).max())

    # roofline of the product kernel: algorithmic 2 n^3 flop per launch (one DPT
    # iteration's product) over its measured average launch duration
    pk, src = peaks()
    # the products take FP16 operands: FP16 and BF16 have the same nominal dense
    # tensor-core rate, so the measured BF16 peak times 1 is the FP16 peak; the kernel
    # runs in launches of about 0.2 ms inside a solve of about 1.2 ms, so the burst
    # figure (not the seconds-long sustained one) is its ceiling
    peak = pk["bf16_tflops"]
    per_launch_ms = prod_ms / max(1, prod_launches)
    achieved = 2.0 * N**3 / (per_launch_ms * 1e-3) / 1e12
    executed = 2.0 * N**3 * float(np.mean(slices)) / (per_launch_ms * 1e-3) / 1e12
    traffic = ncu_traffic() if pair else None   # the committed capture is of the pair form

    # the oracle as the checker (not timed): 16 seeded columns and the 8 columns with
    # the smallest gaps to another level
    errs = None
    if rank == 0 and not args.no_check:
        rng_c = np.random.Generator(np.random.PCG64(11))
        ccols = np.unique(np.concatenate([rng_c.choice(N, 16, replace=False),
                                          tight_columns(cfg["theta"], 8)]))
        ct = torch.tensor(ccols, device=dev)
        errs = checker_full(cfg["theta"], cfg["delta"], cfg["lam"], A[:, ct].cpu().numpy(),
                            E[ct].cpu().numpy(), ccols,
                            "16 seeded columns and the 8 with the smallest gaps; oracle to "
                            "tol 1e-13 on the same columns")

    # end to end through the C ABI with pinned host buffers (copies inside the call)
    th_h = torch.tensor(cfg["theta"]).pin_memory()
    D_h = dpt.colmajor_tensor(cfg["delta"], pin=True)   # column-major pinned buffer
    A_h = torch.empty((N, N), dtype=torch.float64).pin_memory().t()
    E_h = torch.empty((N,), dtype=torch.float64).pin_memory()
    # enough solves that the first input copy and the last output copy (about 1.3 ms,
    # which no other solve overlaps) are a small part of the timed region
    e2e_steps = max(4, min(args.steps, 60))
    outs_h = [(A_h, E_h)] + [(torch.empty((N, N), dtype=torch.float64).pin_memory().t(),
                              torch.empty((N,), dtype=torch.float64).pin_memory())
                             for _ in range(nstr - 1)]
    e2e_calls = [lambda k=k: dpt.solve_full(th_h, D_h, cfg["lam"], A_out=outs_h[k][0],
                                            E_out=outs_h[k][1], stream=sts[k].cuda_stream)
                 for k in range(nstr)]
    for c in e2e_calls:
        c()
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    run_streams(e2e_calls, sts, e2e_steps)
    e2e_s = max_over_ranks(time.perf_counter() - t0, world)
    e2e = {"value": job_throughput(e2e_steps, world, e2e_s), "unit": "solves/s",
           "h2d_bytes_per_step": 8 * N + 8 * N * N, "d2h_bytes_per_step": 8 * N * N + 8 * N,
           "streams": nstr}

    # plain FP64 comparator (same problem, same tolerance)
    fp64 = None
    if not args.no_fp64:
        solve(prec="fp64")
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, _, info64 = solve(prec="fp64", prof=True)
        e1.record(stream)
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1)
        fp64 = {"solves_per_s": 1e3 / ms64, "ms_per_solve": ms64, "iters": info64["iters"],
                "gemm_ms_per_launch": info64["product_ms"] / max(1, info64["product_launches"]),
                "gemm_fp64_tflops": 2.0 * N**3 / (info64["product_ms"] /
                                                  max(1, info64["product_launches"]) * 1e-3) / 1e12}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_sized(cfg)

    extra = {}
    if not args.no_extra:
        chk = not args.no_check
        f64 = fp64["gemm_fp64_tflops"] if fp64 else None
        extra["dominant_csr"] = bench_dominant(dpt, inputs, dev, pk, check=chk)
        extra["dominant_dense"] = bench_dominant_dense(dpt, inputs, dev, pk)
        extra["full_variants"] = bench_full_variants(dpt, inputs, dev, check=chk)
        extra["homotopy"] = bench_homotopy(dpt, dev)
        extra["rs_comparator"] = bench_rs_comparator(dpt, inputs, dev)
        extra["batched"] = bench_batched(dpt, inputs, dev, pk, check=chk, fp64_tflops=f64)
        extra["served"] = bench_served(dpt, inputs, dev, check=chk)
        extra["served_pool"] = bench_served_pool(dpt, inputs, dev, pk, check=chk)

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f16", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": N, "lambda": cfg["lam"], "tol": 1e-12,
                   "prec": "mixed (FP16 tensor-core slices and increments with power-of-two "
                           "scales, FP32 accumulate, float-float state)",
                   "l2": "inputs larger than L2: a solve's working set (Delta 134 MB, about "
                         "0.5 GB of iterate state) exceeds the 129 MB L2; no flush",
                   "parallelism": f"{nstr} independent solve stream(s) per GPU (one host "
                                  f"thread each), {world} GPU(s)"},
        "one_stream": one_stream,
        "streams_results_equal": bool(same),
        "latency_ms": {"p50": float(np.percentile(step_ms, 50)),
                       "p99": float(np.percentile(step_ms, 99)),
                       "mean": float(step_ms.mean())},
        "iters": {"mean": float(np.mean(iters)),
                  "slices_per_product_mean": float(np.mean(slices)),
                  "fp64_refined_columns_max": int(refined)},
        "verified_residual": rho,
        "verified": bool(rho <= 1e-10),
        "errors_vs_oracle": errs,
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak,
                     "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
                     "kernel": ("k_gemm_epi_pair (tcgen05 cta_group::2 product + fused update)"
                                if pair else "k_gemm_epi (tcgen05 product + fused update)"),
                     "peak_source": f"bf16_tflops (burst) x 1 (FP16 nominal rate = BF16), {src}",
                     "algorithmic": "2 n^3 flop per launch (one DPT iteration's product)",
                     "executed_tflops": executed,
                     "executed_frac": executed / peak,
                     "ms_per_launch": per_launch_ms,
                     "launch_timing": f"CUDA events around each product launch, "
                                      f"{prod_launches} launches in a separate untimed pass"},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "fp64_comparator": fp64,
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
        "wall_s": wall,
    }
    line.update(extra)
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    world, rank, local = dist_init(args)
    if args.only != "all":
        import torch
        from paper_2002_12872_gb300 import build, dpt, inputs
        build.build()
        dev = torch.device("cuda", local)
        pk, _ = peaks()
        if args.only == "dominant":
            out = bench_dominant(dpt, inputs, dev, pk, check=not args.no_check)
        elif args.only == "dominant_dense":
            out = bench_dominant_dense(dpt, inputs, dev, pk, steps=max(1, min(args.steps, 10)),
                                       warmup=max(1, min(args.warmup, 3)), n=args.dense_n)
        elif args.only == "homotopy":
            out = bench_homotopy(dpt, dev)
        elif args.only == "full_variants":
            out = bench_full_variants(dpt, inputs, dev, check=not args.no_check)
        elif args.only == "rs":
            out = bench_rs_comparator(dpt, inputs, dev)
        elif args.only == "batched":
            out = bench_batched(dpt, inputs, dev, pk, check=not args.no_check)
        elif args.only == "served_pool":
            out = bench_served_pool(dpt, inputs, dev, pk, steps=max(1, min(args.steps, 10)),
                                    warmup=max(1, min(args.warmup, 3)), max_n=args.pool_max_n,
                                    check=not args.no_check)
        else:
            out = bench_served(dpt, inputs, dev, check=not args.no_check)
        if rank == 0:
            print(json.dumps({args.only: out}), flush=True)
        return
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
