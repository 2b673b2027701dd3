#!/usr/bin/env python
"""Benchmark: filtered Newton-Schulz sign solves/s on one GB300.

Workload (one "step"): the batch of 512 independent symmetric banded matrices
(n log-uniform in [200, 8000], half-bandwidth uniform in {1..10}, seeded
synthetic inputs from workloads/), each solved to ||S^2 - I||_F/sqrt(n) <= 1e-8
with the EXACT filter: FP32 iterations until the residual is below 1e-4, then
FP64, all 512 in one sign_solve_batch call. Every step runs the whole path:
1-norm scale, the two sparse products per iteration, residuals, budgets,
thresholds, filtering and compaction, stage switches and stopping tests.

The serving leg (rank 0) streams Poisson arrivals at 50, 200 and 800 requests/s
through the continuous-batching server and reports p50/p99 latency and
throughput per rate.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun each rank solves its own batch of 512 (weak scaling, no
collective on the data path); the time is the maximum over ranks.

--impl reference times the CPU oracle (oracle/, plain C) on a bounded sample of
the same workload with the host's cores, as the reference arm.
"""
from __future__ import annotations

import argparse
import gc
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as w  # noqa: E402

METRIC = "filtered-NS sign solves/s at ||S^2-I||_F/sqrt(n)<=1e-8 (vs unfiltered FP64 NS on the same GPU)"
UNIT = "solves/s"
BATCH = 512
TOL = 1e-8
WORKLOAD = ("banded batch: 512 symmetric banded matrices, n log-uniform [200,8000], "
            "half-bandwidth U{1..10}, diag +-(1+U[0,1)), off-diag U[-1,1] scaled to row sum <= 0.8; "
            "EXACT filter, FP32 until resid<1e-4 then FP64, tol 1e-8")
# Unit-count peaks, for reference beside the measured ones (fma_peak_leg):
# FP64 152 SMs x 2 FMA/clk x 2 flop x 2.07 GHz; FP32 152 x 128 x 2 x 2.07 GHz
FP64_UNIT_GFLOPS = 152 * 2 * 2 * 2.07
FP32_UNIT_GFLOPS = 152 * 128 * 2 * 2.07
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per algorithmic
# byte of each product class, from ncu captures of the first 128 matrices of
# the batch: FP64 from profiles/k_num_group_f64_lanes_dram_banded128.md, FP32
# (row-wise kernels) from profiles/dram_traffic_products_banded128.md. A
# full-size launch is taken to move DRAM bytes in the same proportion to its
# algorithmic bytes. Valid for the product kernels as those captures built them.
DRAM_PER_ALG_BYTE = {"numeric_square_f64": 0.911, "numeric_update_f64": 0.563,
                     "numeric_square_f32": 0.851, "numeric_update_f32": 0.871}


def rank_seed0(rank: int, count: int = BATCH) -> int:
    """First seed of rank `rank`'s batch: the ranks' batches never share a seed."""
    return w.BASE_SEED + 3000 + rank * count


def batch_mats(rank: int, count: int = BATCH):
    return [w.banded(n, b, s) for n, b, s in w.banded_batch_shapes(count, rank_seed0(rank, count))]


def max_over_ranks(ms: float, dist=None, device=None) -> float:
    """The slowest rank's timed milliseconds (every rank gets the same value)."""
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(per_rank: int, world: int, steps: int, ms_max: float) -> float:
    """Whole-job solves/s: every rank's matrices over the slowest rank's time."""
    return per_rank * world * steps / (ms_max / 1000.0)


def step_hbm(prof: dict, steps: int, ms_per_step: float, hbm_gbs: float) -> dict:
    """The step's HBM roofline: the algorithmic bytes of the timed classes that
    count them (sparse products, filter, assembly: operands read once, outputs
    written once) per step, over the whole step's time."""
    per_step = sum(v["bytes"] for v in prof.values()) / max(steps, 1)
    gbs = per_step / (ms_per_step / 1e3) / 1e9 if ms_per_step > 0 else 0.0
    return {"algorithmic_bytes_per_step": per_step, "achieved_gbs": gbs, "peak_gbs": hbm_gbs,
            "frac": gbs / hbm_gbs if hbm_gbs else None,
            "covers": sorted(k for k, v in prof.items() if v["bytes"] > 0)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ---------------------------------------------------------------------- CPU oracle
def _oracle_one(args):
    idx, rank = args
    import oracle
    a = _mat_by_index(rank, idx)
    t = time.perf_counter()
    r = oracle.nsf(a, tol=TOL, filter="exact", mixed=True)
    return time.perf_counter() - t, r.status


def _mat_by_index(rank, idx):
    shapes = w.banded_batch_shapes(BATCH, w.BASE_SEED + 3000 + rank * BATCH)
    n, b, s = shapes[idx]
    return w.banded(n, b, s)


def oracle_sample(indices, rank=0, cores=None):
    """Times the oracle on the given batch members with a spawn pool."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    cores = cores or min(len(indices), os.cpu_count() or 1)
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(cores) as pool:
        res = pool.map(_oracle_one, [(i, rank) for i in indices])
    wall = time.perf_counter() - t0
    cpu = sum(r[0] for r in res)
    return wall, cpu, cores, [r[1] for r in res]


def cpu_baseline_leg(idx):
    """The oracle timed on the host's cores on a sample of the batch (the
    reported CPU baseline), and the same sample solved by the oracle in FP64
    throughout: the references of the per-result error of the mixed GPU
    results. Returns (cpu_baseline, {index: FP64 oracle result})."""
    import oracle
    wall, cpu_s, cores, st = oracle_sample(idx)
    cpu = {"value": len(idx) / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"{len(idx)} of the 512 matrices (every {BATCH // len(idx)}th), "
                     f"same solve settings; {cpu_s:.1f} s of CPU work in {wall:.1f} s wall"}
    refs = oracle.nsf_many([_mat_by_index(0, i) for i in idx], tol=TOL, filter="exact",
                           mixed=False)
    return cpu, {i: (r.rowptr, r.col, r.val) for i, r in zip(idx, refs)}


def result_errors(mats, results, ref64):
    """Per-result error of the GPU results (host CSR triples, one per matrix):
    ||S - S_ref64||_F / ||S_ref64||_F against the FP64 oracle on its sample, and
    for every result the commutator ||S A - A S||_F / ||A||_F (sign(A) commutes
    with A) and the involution residual ||S^2 - I||_F / sqrt(n)."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spl

    def m(n, rp, col, val):
        return sp.csr_matrix((val, col, rp), shape=(n, n))

    rel = {}
    for i, (rp, col, val) in (ref64 or {}).items():
        n = mats[i].n
        s_ref = m(n, rp, col, val)
        rel[i] = float(spl.norm(m(n, *results[i]) - s_ref) / spl.norm(s_ref))
    comm = []
    for a, (rp, col, val) in zip(mats, results):
        A, S = m(a.n, a.rowptr, a.col, a.val), m(a.n, rp, col, val)
        comm.append(float(spl.norm(S @ A - A @ S) / spl.norm(A)))
    out = {"commutator": {"definition": "||S A - A S||_F / ||A||_F, every result of the batch",
                          "max": max(comm), "median": statistics.median(comm),
                          "count": len(comm)}}
    if rel:
        v = list(rel.values())
        out.update({"definition": "||S_gpu - S_ref64||_F / ||S_ref64||_F, S_ref64 the FP64 "
                                  "oracle (FP64 throughout, EXACT, tol 1e-8)",
                    "sample": sorted(rel), "max": max(v), "median": statistics.median(v),
                    "per_result": [rel[i] for i in sorted(rel)],
                    "note": "the mixed result converges to the sign of the switched FP32 "
                            "iterate, not of A: its error is reported, not bounded by 1e-10"})
    return out


def sample_indices(k: int, offset: int = 0):
    step = BATCH // k
    return [(offset + i * step) % BATCH for i in range(k)]


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    k = args.ref_sample
    for s in range(args.warmup):
        oracle_sample(sample_indices(k, s))
    walls = []
    cores = 0
    for s in range(args.steps):
        wall, cpu, cores, st = oracle_sample(sample_indices(k, args.warmup + s))
        walls.append(wall)
    total = sum(walls)
    value = k * args.steps / total
    sample = f"{k} of the 512 matrices per step (every {BATCH // k}th, offset by step), mixed FP32->FP64, EXACT, tol 1e-8"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "fp32+fp64 (mixed)",
            "data": "synthetic", "config": {"workload": WORKLOAD, "global_batch": BATCH},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------- serving
SERVE_MIX = ("Poisson arrivals; each request drawn from the generators: 45% banded (n log-uniform "
             "[1000,8000], half-bandwidth U{1..10}), 35% tridiagonal (n log-uniform [1000,262144]), "
             "14% shifted 2-D Laplacian (m U{32..48}, n 1024-2304), 5% shifted 3-D Laplacian "
             "(m U{10..16}, n 1000-4096), 1% shifted 3-D Laplacian m=64 (n=262,144, refused by "
             "the footprint budget); mixed FP32->FP64, EXACT, tol 1e-8")


def serve_pool(seed: int = w.BASE_SEED + 4000, size: int = 160):
    """Distinct request matrices and their draw weights (host CSR)."""
    rng = np.random.default_rng(seed)
    pool, weights = [], []
    for i in range(size):
        u = rng.random()
        if u < 0.45:
            n = int(round(math.exp(rng.uniform(math.log(1000), math.log(8000)))))
            pool.append(w.banded(n, int(rng.integers(1, 11)), seed + i))
        elif u < 0.80:
            n = int(round(math.exp(rng.uniform(math.log(1000), math.log(262144)))))
            pool.append(w.tridiagonal(n, seed + i))
        elif u < 0.94:
            pool.append(w.laplacian(int(rng.integers(32, 49)), 2))
        else:
            pool.append(w.laplacian(int(rng.integers(10, 17)), 3))
        weights.append(1.0)
    pool.append(w.laplacian(64, 3))
    weights = np.array(weights + [len(weights) / 99.0])
    return pool, weights / weights.sum()


def serve_leg(sg, rates, seconds: float, seed: int = 7, max_wait_s: float = 0.0):
    """Open-loop Poisson stream per rate through a fresh server; latency is
    completion minus scheduled arrival (both CLOCK_MONOTONIC). max_wait_s > 0:
    the server refuses (SIGN_EAGAIN) submissions predicted to wait longer."""
    pool, p = serve_pool()
    rng = np.random.default_rng(seed)
    opts = sg.default_opts(tol=TOL, filter="exact", prec="mixed")
    with sg.Server(opts) as srv:  # warm-up: allocations, first launches
        ts = [srv.submit(pool[i]) for i in range(0, 40, 2)]
        for t in ts:
            srv.poll(t, wait_ms=120000)
    out = []
    for rate in rates:
        k = max(1, int(rng.poisson(rate * seconds)))
        arrivals = np.cumsum(rng.exponential(1.0 / rate, k))
        picks = rng.choice(len(pool), size=k, p=p)
        tickets, refused, late, t_arr = [], 0, 0, []
        with sg.Server(opts, max_wait_s=max_wait_s) as srv:
            t0 = time.monotonic() + 0.05
            for at, i in zip(arrivals, picks):
                wait = t0 + at - time.monotonic()
                if wait > 0:
                    time.sleep(wait)
                try:
                    tickets.append(srv.submit(pool[i]))
                    t_arr.append(t0 + at)
                except sg.SignError as e:
                    if e.status == sg.SIGN_EAGAIN:
                        late += 1
                    elif e.status != sg.SIGN_ENOMEM:
                        raise
                    refused += 1
            lat, done, lanes, bad = [], [], [], 0
            for t, ta in zip(tickets, t_arr):
                r = None
                while r is None:
                    r = srv.poll(t, wait_ms=10000)
                bad += r["status"] != sg.SIGN_OK
                lat.append(r["t_done"] - ta)
                done.append(r["t_done"])
                lanes.append(r["lane"])
            st = srv.stats()
        lat_ms, lanes = np.array(lat) * 1e3, np.array(lanes)
        span = (max(done) - t0) if done else float("nan")

        def pct(x):
            if not len(x):
                return None
            return {"count": int(len(x)), "p50_ms": float(np.percentile(x, 50)),
                    "p99_ms": float(np.percentile(x, 99)), "mean_ms": float(x.mean())}

        row = {"rate_req_per_s": rate, "requests": k, "refused": refused,
               "refused_for_wait": late,
               "completed": len(tickets), "not_converged": int(bad),
               "solves_per_s": len(tickets) / span if done else 0.0,
               "max_active_seen": st["max_active_seen"], "rounds": st["rounds"]}
        row.update(pct(lat_ms) or {})
        row["sparse_lane"] = pct(lat_ms[lanes == 0])
        row["fill_in_lane"] = pct(lat_ms[lanes == 1])
        out.append(row)
    return {"mix": SERVE_MIX, "seconds_per_rate": seconds, "mem_budget_bytes": 120e9,
            "lanes": "2: requests predicted to fill in (no Gershgorin gap) on a lane of their own",
            "latency": "completion minus scheduled arrival, both on CLOCK_MONOTONIC",
            "max_wait_s": max_wait_s, "rates": out}


# ---------------------------------------------------------------------- fill tracking
def fill_leg(sg, iters: int):
    """The 2-D shifted Laplacian at m = 256 (n = 65,536) for a bounded number
    of updates: nnz(X), nnz(T), residual and wall time per iteration, filtered
    (EXACT, FP64 and mixed) against unfiltered FP64."""
    import torch
    a = w.laplacian(256, 2)
    # unfiltered NS fills in fastest; its FP64 products are capped at 4 updates
    runs = {"filtered_fp64": (dict(filter="exact", prec="fp64"), iters),
            "filtered_mixed": (dict(filter="exact", prec="mixed"), iters),
            "unfiltered_fp64": (dict(filter="none", prec="fp64"), min(iters, 4))}
    out = {"workload": "laplacian2d m=256 (n=65,536), sigma mid-gap, tol 1e-8",
           "max_updates": iters}
    for name, (kw, k) in runs.items():
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = sg.solve(a, tol=TOL, max_iter=k, **kw)
        torch.cuda.synchronize()
        tr = r.trace
        out[name] = {"status": int(r.status), "updates": int(r.iters),
                     "seconds": time.perf_counter() - t0,
                     "nnz_x": [int(x) for x in tr["nnz_x"]], "nnz_t": [int(x) for x in tr["nnz_t"]],
                     "resid": [float(x) for x in tr["resid_k"]],
                     "prec": [int(x) for x in tr["prec_k"]]}
    return out


# ---------------------------------------------------------------------- 2-D Laplacian, solved
def laplacian2d_leg(sg, m: int = 256, rows: int = 100, per_row: int = 100):
    """The 2-D shifted Laplacian on m x m points (m = 256: n = 65,536) solved
    to ||X^2 - I||_F/sqrt(n) <= 1e-8, filtered (EXACT), mixed FP32 -> FP64;
    once its iterate holds a quarter of n^2 it runs on the dense tensor-core
    path. Reports the fill and residual per iteration, the time, the time of
    the dense products, and the error against the closed-form sign at
    rows x per_row seeded entries (half near the diagonal, half anywhere)."""
    import torch
    from workloads import closed_form
    a = w.laplacian(m, 2)
    n = a.n
    sg.trim_memory()
    sg.prof_reset()
    sg.prof_enable(True)
    import ctypes
    from paper_2210_03356_gb300 import _Info
    o = sg.default_opts(tol=TOL, filter="exact", prec="mixed", max_iter=200)
    info = _Info(256)
    with sg.Handle(a) as h:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = sg.load().sign_solve(h.h, ctypes.byref(o), ctypes.byref(info.s))
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
        sg.prof_enable(False)
        if st not in (sg.SIGN_OK, sg.SIGN_ENOTCONV, sg.SIGN_EDIVERGED):
            raise sg.SignError(st, "sign_solve")
        sg.trim_memory()  # the solve's cached memory back to the device before the copy
        rpd, cold, vald = h.result(device=True)
    prof = sg.prof_read()
    tr = info.trace()
    status, iters, resid = info.s.status, info.s.iters, info.s.resid
    rng = np.random.default_rng(m)
    p = np.sort(rng.choice(n, rows, replace=False))
    rp = rpd.cpu().numpy()
    got, pi, ppi = [], [], []
    for i in p:
        lo, hi = int(rp[i]), int(rp[i + 1])
        col = cold[lo:hi].cpu().numpy()
        val = vald[lo:hi].cpu().numpy()
        near = (i + rng.integers(-3 * m, 3 * m, per_row // 2)) % n
        far = rng.integers(0, n, per_row - per_row // 2)
        for j in np.r_[near, far]:
            k = np.searchsorted(col, j)
            got.append(val[k] if k < col.size and col[k] == j else 0.0)
            pi.append(i)
            ppi.append(j)
    got = np.array(got)
    ref = closed_form.laplacian_sign_entries(m, 2, np.array(pi), np.array(ppi))
    dense = {k: {"launches": v["launches"], "ms": v["ms"]} for k, v in prof.items()
             if k.startswith("dense") and v["launches"]}
    out = {"workload": f"laplacian2d m={m} (n={n}), sigma mid-gap, EXACT, mixed FP32->FP64, "
                       "tol 1e-8", "status": int(status), "updates": int(iters),
           "resid": float(resid), "seconds": secs, "nnz_final": int(rp[-1]),
           "density_final": float(rp[-1]) / n / n,
           "err_vs_closed_form": float(np.linalg.norm(got - ref) / np.linalg.norm(ref)),
           "max_abs_err": float(np.abs(got - ref).max()), "samples": int(got.size),
           "nnz_x": [int(x) for x in tr["nnz_x"]], "nnz_t": [int(x) for x in tr["nnz_t"]],
           "resid_k": [float(x) for x in tr["resid_k"]], "prec_k": [int(x) for x in tr["prec_k"]],
           "dense_classes": dense}
    del rpd, cold, vald
    torch.cuda.empty_cache()
    print(f"laplacian2d m={m}: {secs:.1f} s, {out['updates']} updates, error "
          f"{out['err_vs_closed_form']:.3g}", file=sys.stderr, flush=True)
    return out


# ---------------------------------------------------------------------- 3-D Laplacian (scaled)
def laplacian3d_leg(sg, m: int, samples: int = 4000):
    """The 3-D shifted Laplacian on m^3 points (scaled variants of the 64^3
    workload): mixed and FP64 solves with their fill per iteration, and the
    error of each against the closed-form sign at seeded sampled entries."""
    import torch
    from workloads import closed_form
    a = w.laplacian(m, 3)
    rng = np.random.default_rng(m)
    p = rng.integers(0, a.n, samples)
    pp = np.where(rng.random(samples) < 0.5, p + rng.integers(-3 * m * m, 3 * m * m, samples),
                  rng.integers(0, a.n, samples)) % a.n
    ref = closed_form.laplacian_sign_entries(m, 3, p, pp)
    out = {"workload": f"laplacian3d m={m} (n={a.n}), sigma = 6, EXACT, tol 1e-8",
           "samples": samples}
    # FP64 throughout only up to n = 16384: before the iterate reaches the dense
    # path's quarter, every FP64 iteration is a sparse product on filling rows
    modes = (("mixed", "mixed"), ("fp64", "fp64")) if a.n <= 16384 else (("mixed", "mixed"),)
    for name, prec in modes:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = sg.solve(a, tol=TOL, filter="exact", prec=prec, max_iter=200)
        torch.cuda.synchronize()
        got = closed_form.csr_entries(r.rowptr, r.col, r.val, p, pp)
        tr = r.trace
        out[name] = {"status": int(r.status), "updates": int(r.iters), "resid": float(r.resid),
                     "seconds": time.perf_counter() - t0,
                     "err_vs_closed_form": float(np.linalg.norm(got - ref) / np.linalg.norm(ref)),
                     "nnz_x": [int(x) for x in tr["nnz_x"]], "prec": [int(x) for x in tr["prec_k"]]}
        print(f"laplacian3d m={m} {name}: {out[name]['seconds']:.1f} s, "
              f"error {out[name]['err_vs_closed_form']:.3g}", file=sys.stderr, flush=True)
    return out


# Table 4.2.1's NSF times (MATLAB on the paper's CPU), tol 1e-12, for context
ODE_PAPER_NSF_SECONDS = {500: 0.0098, 1000: 0.011, 3000: 0.0268, 5000: 0.0481}


def ode_leg(sg, sizes, reps: int = 3):
    """Sec. 4.2's ODE block matrix A = [[0, B], [I, 0]], B = tridiag(1/16, 7/8,
    1/16), solved as in Table 4.2.1: FP64 NSF (EXACT) to tol 1e-12 from X0 = A
    (unscaled; A's eigenvalues are +-sqrt(eig B), within [0.87, 1] in modulus).
    The table's n is read both ways: as the order of B and as the order of A.
    Reports the device time per solve (one matrix per sign_solve_batch call,
    after a warm-up) and the error against the closed form (Eq. 1.26)."""
    import torch
    from workloads import closed_form
    out = []
    o = sg.default_opts(tol=1e-12, filter="exact", prec="fp64", scale_1norm=0)
    for n in sizes:
        for reading, nb in (("n = order of B", n), ("n = order of A", n // 2)):
            a = w.ode_block(nb)
            b = sg.Batch([a])
            try:
                b.solve(o)  # warm-up
                secs = []
                for _ in range(reps):
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    (st, iters, resid), = b.solve(o)
                    torch.cuda.synchronize()
                    secs.append(time.perf_counter() - t0)
                rp, col, val = b.handles[0].result()
            finally:
                b.close()
            D = np.zeros((a.n, a.n))
            D[np.repeat(np.arange(a.n), np.diff(rp)), col] = val
            S = closed_form.ode_block_sign(nb)
            out.append({"n": n, "reading": reading, "order_of_A": int(a.n), "status": int(st),
                        "iters": int(iters), "resid": float(resid),
                        "seconds_per_solve": statistics.median(secs),
                        "max_abs_err": float(np.abs(D - S).max()),
                        "rel_fro_err": float(np.linalg.norm(D - S) / np.linalg.norm(S)),
                        "paper_nsf_seconds": ODE_PAPER_NSF_SECONDS.get(n)})
            print(f"ode n={n} ({reading}): {out[-1]['seconds_per_solve'] * 1e3:.2f} ms, "
                  f"max abs err {out[-1]['max_abs_err']:.2e}", file=sys.stderr, flush=True)
    return out


def filter_error_leg(solve, sizes, seeds: int = 5, tol: float = 1e-12, make=None):
    """Sec. 4.1's second test (Fig. 4.1.2): random sparse SPD matrices of
    density 1% (the stand-in for sprandsym(n, 0.01, 1); workloads.spd_random),
    NS and NSF (EXACT) in FP64 to tol 1e-12 (make: another matrix family, as
    Sec. 4.1's first test with Newton's method). For every iteration k, the
    filtered and unfiltered iterates after k updates give
    dX_k = Xhat_k - X_k and dR_k = Rhat_k - R_k (R = I - X^2), in RMS-Frobenius
    norm; the paper shows both below tol. solve(a, filter, max_iter) returns
    (status, iters, rowptr, col, val) of a run stopped after max_iter updates."""
    out = []
    make = make or (lambda n, s: w.spd_random(n, 0.01, seed=w.BASE_SEED + 7000 + 10 * n + s))
    for n in sizes:
        for s in range(seeds):
            a = make(n, s)
            st, K, *_ = solve(a, "none", 100)
            dX, dR, r = [], [], []
            for k in range(1, K + 1):
                mats = []
                for filt in ("none", "exact"):
                    _, _, rp, col, val = solve(a, filt, k)
                    X = np.zeros((n, n))
                    X[np.repeat(np.arange(n), np.diff(rp)), col] = val
                    mats.append(X)
                X, Xh = mats
                R = np.eye(n) - X @ X
                Rh = np.eye(n) - Xh @ Xh
                rms = lambda M: float(np.linalg.norm(M) / np.sqrt(n))  # noqa: E731
                dX.append(rms(Xh - X))
                dR.append(rms(Rh - R))
                r.append(rms(R))
            out.append({"n": n, "seed": s, "ns_status": int(st), "iters": int(K), "dX": dX,
                        "dR": dR, "resid": r, "max_dX": max(dX), "max_dR": max(dR)})
            print(f"filter error n={n} seed {s}: {K} iterations, max dX {max(dX):.2e}, "
                  f"max dR {max(dR):.2e}", file=sys.stderr, flush=True)
    return out


# ---------------------------------------------------------------------- FMA peaks
def fma_peak_leg(sg, gpu_index: int, seconds: float = 1.0):
    """Measured FP64 and FP32 fused multiply-add peaks of this GPU: the
    library's probe (register-resident FMA chains on every SM) timed with CUDA
    events, the median of the launches, with the SM clock sampled while it
    runs. The sparse products' rooflines divide by these."""
    import ctypes
    import torch
    L = sg.load()
    stream = torch.cuda.current_stream()
    sp = ctypes.c_void_p(stream.cuda_stream)
    sms = torch.cuda.get_device_properties(gpu_index).multi_processor_count
    out = {}
    for name, fp64, iters in (("fp64", 1, 4096), ("fp32", 0, 65536)):
        fl = ctypes.c_double()

        def launch():
            st = L.sign_fma_probe(fp64, sms * 8, 256, iters, sp, ctypes.byref(fl))
            if st != sg.SIGN_OK:
                raise sg.SignError(st, "sign_fma_probe")

        for _ in range(3):
            launch()
        torch.cuda.synchronize()
        ck = Clocks(gpu_index)
        ck.start()
        times = []
        t_end = time.perf_counter() + seconds
        while time.perf_counter() < t_end or len(times) < 5:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            launch()
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        clk = ck.stop()
        ms = statistics.median(times)
        out[name] = {"gflops": fl.value / (ms / 1e3) / 1e9, "ms_per_launch": ms,
                     "launches": len(times), "clocks": clk,
                     "unit_count_gflops": FP64_UNIT_GFLOPS if fp64 else FP32_UNIT_GFLOPS}
    out["how"] = (f"sign_fma_probe: {sms * 8} CTAs x 256 threads, 8 independent FMA chains per "
                  "thread; median of the launches over ~1 s each, CUDA events")
    return out


# ---------------------------------------------------------------------- variants
VARIANTS = (("default", {}), ("filter_t", {"filter_t": 1}), ("budget_norm_2", {"budget_norm": 1}),
            ("both", {"filter_t": 1, "budget_norm": 1}))


def variants_leg(sg, mats, reps: int = 2):
    """The two variants of the readings against the default, on the banded
    batch: T filtered with the same budget (filter_t) and the 2-norm in Eq.
    (1.18) (budget_norm). Two workloads: the whole batch as benchmarked (mixed,
    tol 1e-8) and every 8th matrix in FP64 to tol 1e-12, where the adaptive
    budget of Eq. (1.18) is reached. Per variant: solves/s (CUDA events, after
    a warm-up), iterations, and the entries per iteration summed over the
    matrices (X, T and the T the update multiplies by)."""
    import torch
    out = []
    for label, sub, base in (("banded batch, mixed, EXACT, tol 1e-8", mats,
                              dict(tol=TOL, filter="exact", prec="mixed")),
                             ("every 8th matrix, FP64, EXACT, tol 1e-12", mats[::8],
                              dict(tol=1e-12, filter="exact", prec="fp64"))):
        b = sg.Batch(sub)
        try:
            rows = {}
            for name, kw in VARIANTS:
                o = sg.default_opts(**base, **kw)
                b.solve(o)
                ms = []
                for _ in range(reps):
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record()
                    b.solve(o)
                    e1.record()
                    e1.synchronize()
                    ms.append(e0.elapsed_time(e1))
                res = b.solve(o, trace_cap=64)
                tr = b.traces()
                depth = max(len(t["nnz_x"]) for t in tr)

                def per_iter(key):
                    return [int(sum(int(t[key][k]) for t in tr if k < len(t[key])))
                            for k in range(depth)]

                rows[name] = {"solves_per_s": len(sub) / (statistics.median(ms) / 1e3),
                              "ms_per_batch": statistics.median(ms),
                              "all_converged": all(s == sg.SIGN_OK for s, _, _ in res),
                              "mean_updates": float(np.mean([it for _, it, _ in res])),
                              "max_resid": float(max(r for _, _, r in res)),
                              "nnz_x_per_iter": per_iter("nnz_x"),
                              "nnz_t_per_iter": per_iter("nnz_t"),
                              "nnz_t_used_per_iter": per_iter("nnz_that")}
            out.append({"workload": label, "matrices": len(sub), "variants": rows})
        finally:
            b.close()
    return out


def tune_leg(sg, mats, reps: int = 3):
    """sign_tune_batch on two workloads: the banded batch as benchmarked and a
    Laplacian-heavy batch (shifted 2-D Laplacians, m = 24..46, and 3-D ones,
    m = 8..13). Per workload: the schedule the tuner chose, its own best times
    of a batch solve (base schedule and chosen one, host wall time), then the
    solves/s of the default and of the chosen schedule (CUDA events, median of
    reps after a warm-up). Every schedule gives the same results bit for bit."""
    import torch
    lap = [w.laplacian(m, 2) for m in range(24, 48, 2)] + [w.laplacian(m, 3) for m in range(8, 14)]
    out = []
    for label, sub in (("banded batch, mixed, EXACT, tol 1e-8", mats),
                       ("Laplacian-heavy batch: 12 shifted 2-D (m 24..46) + 6 shifted 3-D "
                        "(m 8..13) Laplacians, mixed, EXACT, tol 1e-8", lap)):
        b = sg.Batch(sub)
        try:
            base = sg.default_opts(tol=TOL, filter="exact", prec="mixed")
            best, rep = b.tune(base, reps=2, force=True)

            def median_ms(o):
                b.solve(o)
                ms = []
                for _ in range(reps):
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record()
                    b.solve(o)
                    e1.record()
                    e1.synchronize()
                    ms.append(e0.elapsed_time(e1))
                return statistics.median(ms)

            m0, m1 = median_ms(base), median_ms(best)
            out.append({"workload": label, "matrices": len(sub),
                        "chosen": {"band_min_eff": best.band_min_eff,
                                   "group_margin": best.group_margin,
                                   "pair_rows": best.pair_rows},
                        "default": {"band_min_eff": base.band_min_eff,
                                    "group_margin": base.group_margin,
                                    "pair_rows": base.pair_rows},
                        "tuner_solves_timed": rep["timed"],
                        "tuner_ms_base": rep["ms_base"], "tuner_ms_best": rep["ms_best"],
                        "solves_per_s_default": len(sub) / (m0 / 1e3),
                        "solves_per_s_tuned": len(sub) / (m1 / 1e3), "gain": m0 / m1})
        finally:
            b.close()
    return out


# ---------------------------------------------------------------------- clocks
class Clocks:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.rows = []
        self.proc = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu)], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        rows = [r for r in self.rows if len(r) >= 9]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# ---------------------------------------------------------------------- our arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--legs", default="all", choices=["all", "timed"],
                    help="timed: only the device-timed leg (for profiler runs)")
    ap.add_argument("--ref-sample", type=int, default=8)
    ap.add_argument("--cpu-sample", type=int, default=16)
    ap.add_argument("--unfiltered-sample", type=int, default=8)
    ap.add_argument("--batch", type=int, default=BATCH,
                    help="matrices per batch (smaller only for profiler captures)")
    ap.add_argument("--serve-seconds", type=float, default=5.0,
                    help="length of the Poisson stream at each serving rate (0: skip)")
    ap.add_argument("--serve-rates", default="50,200,800")
    ap.add_argument("--laplacian3d", default="",
                    help="comma-separated m: also solve the m^3 3-D Laplacian against its closed form")
    ap.add_argument("--fill-iters", type=int, default=0,
                    help="also track fill on the n=65,536 2-D Laplacian for this many updates")
    ap.add_argument("--laplacian2d", type=int, default=0,
                    help="m: also solve the m x m 2-D Laplacian (m = 256: n = 65,536) to tol")
    ap.add_argument("--ode", default="",
                    help="comma-separated n: also solve Sec. 4.2's ODE block matrix as in Table 4.2.1")
    ap.add_argument("--filter-error", default="",
                    help="comma-separated n: also run Sec. 4.1's NS vs NSF test (Fig. 4.1.2)")
    ap.add_argument("--filter-error-nm", default="",
                    help="comma-separated n: also run Sec. 4.1's NM vs NMF test (Fig. 4.1.1)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    # CPU baseline first: the spawn pool runs before this process touches CUDA
    cpu = ref64 = None
    if args.legs == "all" and rank == 0 and world == 1:
        idx = sample_indices(args.cpu_sample)
        cpu, ref64 = cpu_baseline_leg(idx)

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import __graft_entry__
    __graft_entry__.build()
    import paper_2210_03356_gb300 as sg
    L = sg.load()

    mats = batch_mats(rank)[:args.batch]
    opts = sg.default_opts(tol=TOL, filter="exact", prec="mixed")
    stream = torch.cuda.current_stream()
    batch = sg.Batch(mats, stream=None if stream.cuda_stream == 0 else
                     __import__("ctypes").c_void_p(stream.cuda_stream))

    def barrier():
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        out = batch.solve(opts)
    assert all(s == sg.SIGN_OK for s, _, _ in out), out[:4]
    # the inputs and handles made so far live until the end: keep them out of
    # the interpreter's full collections, which otherwise pause a step now and
    # then (about 30 ms scanning them; the usual setting of a long-lived service)
    gc.freeze()

    clocks = Clocks(local)
    clocks.start()
    barrier()
    sg.prof_reset()
    sg.prof_enable(True)
    l0 = sg.kernel_launches()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        out = batch.solve(opts)
    e1.record(stream)
    barrier()
    launches = sg.kernel_launches() - l0
    sg.prof_enable(False)
    prof_all = sg.prof_read()
    prof = {k: v for k, v in prof_all.items() if not k.startswith("host_")}
    host = {k: round(v["ms"] / args.steps, 3) for k, v in prof_all.items()
            if k.startswith("host_") and v["launches"]}
    ck = clocks.stop()
    ms = e0.elapsed_time(e1)
    assert all(s == sg.SIGN_OK and r <= TOL for s, _, r in out)
    ms_max = max_over_ranks(ms, dist, "cuda")
    value = job_throughput(len(mats), world, args.steps, ms_max)

    # roofline of the dominant kernel class; the FMA peaks are measured here
    peaks, peak_kind = measured_peaks()
    fma = fma_peak_leg(sg, local)
    FP64_PEAK_GFLOPS, FP32_PEAK_GFLOPS = fma["fp64"]["gflops"], fma["fp32"]["gflops"]
    top = max(prof.items(), key=lambda kv: kv[1]["ms"])
    name, p = top
    per_launch_ms = p["ms"] / max(p["launches"], 1)
    if "numeric" in name and name.endswith("f64"):
        bound, peak, unit = "alu", FP64_PEAK_GFLOPS, "GFLOP/s"
        achieved = p["flops"] / (p["ms"] / 1e3) / 1e9
        per_launch = p["flops"] / max(p["launches"], 1)
    elif "numeric" in name:
        fl = p["flops"] / (p["ms"] / 1e3) / 1e9
        by = p["bytes"] / (p["ms"] / 1e3) / 1e9
        if fl / FP32_PEAK_GFLOPS >= by / peaks["hbm_gbs"]:
            bound, peak, unit, achieved = "alu", FP32_PEAK_GFLOPS, "GFLOP/s", fl
            per_launch = p["flops"] / max(p["launches"], 1)
        else:
            bound, peak, unit, achieved = "hbm", peaks["hbm_gbs"], "GB/s", by
            per_launch = p["bytes"] / max(p["launches"], 1)
    else:
        bound, peak, unit = "hbm", peaks["hbm_gbs"], "GB/s"
        achieved = p["bytes"] / (p["ms"] / 1e3) / 1e9 if p["ms"] else 0.0
        per_launch = p["bytes"] / max(p["launches"], 1)
    total_ms = sum(v["ms"] for v in prof.values())
    alg_bytes = p["bytes"] / max(p["launches"], 1)
    traffic = DRAM_PER_ALG_BYTE[name] * alg_bytes if name in DRAM_PER_ALG_BYTE else None
    roofline = {"kernel": name, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
                "frac": achieved / peak, "traffic": traffic,
                "traffic_source": ("ncu DRAM bytes per algorithmic byte on the first 128 matrices, "
                                   "times this launch's algorithmic bytes" if traffic else None),
                "algorithmic_bytes_per_launch": alg_bytes,
                "peak_source": (f"{peak_kind} MEASURED_PEAKS.json hbm_gbs" if bound == "hbm"
                                else "measured in this run: FMA probe (fma_peaks), "
                                     f"{'FP64' if name.endswith('f64') else 'FP32'}"),
                "unit_count_peak": (None if bound == "hbm" else
                                    FP64_UNIT_GFLOPS if name.endswith("f64") else FP32_UNIT_GFLOPS),
                "per_launch_work": per_launch, "avg_launch_ms": per_launch_ms,
                "share_of_kernel_time": p["ms"] / total_ms if total_ms else None}
    by_kernel = {k: {"share": v["ms"] / total_ms if total_ms else 0.0, "launches": v["launches"],
                     "ms": round(v["ms"], 3),
                     "gflops": v["flops"] / (v["ms"] / 1e3) / 1e9 if v["ms"] else 0.0,
                     "gbs": v["bytes"] / (v["ms"] / 1e3) / 1e9 if v["ms"] else 0.0}
                 for k, v in prof.items() if v["launches"]}
    for k, v in by_kernel.items():  # the sparse products against their FMA pipe
        if k.startswith("numeric_"):
            v["frac_of_fma_peak"] = v["gflops"] / (FP64_PEAK_GFLOPS if k.endswith("f64")
                                                   else FP32_PEAK_GFLOPS)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "fp32+fp64 (mixed)", "data": "synthetic",
            "config": {"workload": WORKLOAD if len(mats) == BATCH else
                       f"first {len(mats)} matrices of: " + WORKLOAD, "global_batch": len(mats) * world,
                       "rows_per_batch": int(sum(a.n for a in mats)),
                       "parallelism": f"{world} independent batches (one per GPU)",
                       "l2": "working set of every step (iterates, products) is several GB, > 129 MB L2"},
            "gpu_launches": int(launches), "clocks": ck, "roofline": roofline,
            "hbm_roofline_step": step_hbm(prof, args.steps, ms_max / args.steps,
                                          peaks["hbm_gbs"]),
            "kernels": by_kernel, "host_ms_per_step": host, "fma_peaks": fma}

    if args.legs == "all":
        # end to end through the public API: pinned host inputs -> device -> host result
        pinned = []
        h2d = d2h = 0
        for a in mats:
            rp = torch.from_numpy(a.rowptr).pin_memory()
            col = torch.from_numpy(a.col).pin_memory()
            val = torch.from_numpy(a.val).pin_memory()
            pinned.append(type("P", (), {"n": a.n, "rowptr": rp.numpy(), "col": col.numpy(),
                                         "val": val.numpy(), "_keep": (rp, col, val)}))
            h2d += rp.numel() * 8 + col.numel() * 4 + val.numel() * 8
        # result buffers in pinned memory, sized by an untimed first pass and
        # reused by every step (a caller sizes them from result_nnz())
        outs = []

        last = []

        def e2e_step():
            b2 = sg.Batch(pinned)
            b2.solve(opts)
            for i, (hnd, nnz) in enumerate(zip(b2.handles, b2.result_nnz())):
                if i == len(outs) or outs[i][1].size < nnz:
                    buf = (torch.empty(hnd.n + 1, dtype=torch.int64, pin_memory=True),
                           torch.empty(max(nnz, 1), dtype=torch.int32, pin_memory=True),
                           torch.empty(max(nnz, 1), dtype=torch.float64, pin_memory=True))
                    views = tuple(t.numpy() for t in buf)
                    if i == len(outs):
                        outs.append(views)
                    else:
                        outs[i] = views
            res = b2.results(outs)  # every copy queued, one wait
            nbytes = sum(rp.nbytes + col.nbytes + val.nbytes for rp, col, val in res)
            b2.close()
            last[:] = res
            return nbytes

        for _ in range(args.warmup):  # untimed, as for the device-timed steps
            e2e_step()
        gc.freeze()  # the pinned inputs and result buffers, as above
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            d2h = e2e_step()
        barrier()
        e2e_s = time.perf_counter() - t0
        line["e2e"] = {"value": len(mats) * world * args.steps / e2e_s, "unit": UNIT,
                       "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                       "python_gc": "objects made before the timed steps frozen (gc.freeze)"}
        # the results of the last end-to-end step: identical to the timed steps'
        # (every solve is deterministic); their errors, outside any timed region
        if rank == 0:
            line["err_vs_fp64_oracle"] = result_errors(mats, last, ref64)

        # unfiltered FP64 Newton-Schulz on the same GPU: two disjoint samples of
        # the batch (every 64th matrix from 0 and from 32), each batch call
        # timed three times, filtered (the benchmarked options) and unfiltered
        o_f = sg.default_opts(tol=TOL, filter="exact", prec="mixed")
        o_u = sg.default_opts(tol=TOL, filter="none", prec="fp64")
        samples = []
        for off in (0, BATCH // (2 * args.unfiltered_sample)):
            idx = sample_indices(args.unfiltered_sample, off)
            sub = sg.Batch([mats[i] for i in idx])
            times = {}
            for name, o in (("filtered", o_f), ("unfiltered", o_u)):
                sub.solve(o)  # warm-up
                ts = []
                for _ in range(3):
                    barrier()
                    t0 = time.perf_counter()
                    r = sub.solve(o)
                    barrier()
                    ts.append(time.perf_counter() - t0)
                    assert all(st == sg.SIGN_OK for st, _, _ in r)
                times[name] = ts
            sub.close()
            tf, tu = statistics.median(times["filtered"]), statistics.median(times["unfiltered"])
            samples.append({"indices": idx, "filtered_mixed_solves_per_s": len(idx) / tf,
                            "unfiltered_fp64_solves_per_s": len(idx) / tu,
                            "speedup_median": tu / tf,
                            "speedup_range": [min(times["unfiltered"]) / max(times["filtered"]),
                                              max(times["unfiltered"]) / min(times["filtered"])]})
        tf_all = sum(len(x["indices"]) / x["filtered_mixed_solves_per_s"] for x in samples)
        tu_all = sum(len(x["indices"]) / x["unfiltered_fp64_solves_per_s"] for x in samples)
        n_all = sum(len(x["indices"]) for x in samples)
        line["vs_unfiltered_fp64"] = {
            "sample": f"2 x {args.unfiltered_sample} of the 512 matrices (every "
                      f"{BATCH // args.unfiltered_sample}th from 0 and from "
                      f"{BATCH // (2 * args.unfiltered_sample)}), one batch call per sample, "
                      "median of 3 timed calls after a warm-up",
            "filtered_mixed_solves_per_s": n_all / tf_all,
            "unfiltered_fp64_solves_per_s": n_all / tu_all, "speedup": tu_all / tf_all,
            "samples": samples}
        if cpu:
            line["cpu_baseline"] = cpu
    batch.close()
    if args.legs == "all" and rank == 0:
        line["variants"] = variants_leg(sg, mats)
        line["tuning"] = tune_leg(sg, mats)
    if args.legs == "all" and args.serve_seconds > 0 and rank == 0:
        rates = [float(x) for x in args.serve_rates.split(",") if x]
        line["serving"] = serve_leg(sg, rates, args.serve_seconds)
        # past capacity with a latency target: refusals instead of a growing queue
        line["serving_latency_target"] = serve_leg(sg, [rates[-1]], args.serve_seconds,
                                                   max_wait_s=0.25)
    if args.fill_iters > 0 and rank == 0:
        line["laplacian2d_fill"] = fill_leg(sg, args.fill_iters)
    if args.laplacian2d and rank == 0:
        line["laplacian2d_solve"] = laplacian2d_leg(sg, args.laplacian2d)
    if args.laplacian3d and rank == 0:
        line["laplacian3d"] = [laplacian3d_leg(sg, int(m)) for m in args.laplacian3d.split(",")]
    if args.ode and rank == 0:
        line["ode_table_4_2_1"] = ode_leg(sg, [int(n) for n in args.ode.split(",")])
    if args.filter_error and rank == 0:
        def gpu_solve(a, filt, max_iter):
            r = sg.solve(a, tol=1e-12, filter=filt, prec=0, max_iter=max_iter)
            return r.status, r.iters, r.rowptr, r.col, r.val
        line["filter_error_fig_4_1_2"] = filter_error_leg(
            gpu_solve, [int(n) for n in args.filter_error.split(",")])
    if args.filter_error_nm and rank == 0:
        def gpu_nmf(a, filt, max_iter):
            r = sg.solve(a, tol=1e-12, filter=filt, method="nmf", max_iter=max_iter)
            return r.status, r.iters, r.rowptr, r.col, r.val
        line["filter_error_fig_4_1_1"] = filter_error_leg(
            gpu_nmf, [int(n) for n in args.filter_error_nm.split(",")],
            make=lambda n, s: w.sprand_like(n, 0.01, seed=w.BASE_SEED + 8000 + 10 * n + s))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
