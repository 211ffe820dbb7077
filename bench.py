#!/usr/bin/env python
"""Ridge-path benchmark: IHS-BIN on GB300 through the C ABI.

Workload (default `c4`, the largest single-GPU configuration): dense BF16 A 262144 x 2048 with
power-law columns (1+j)^-1, B 262144 x 64 from a planted X* plus 1% noise, Gaussian sketch
m = 4096 with BF16 entries, T = 500 lambdas log-spaced in [1e-4, 1e-2] * ||A||_2^2, L = 9
intervals, per-interval (rho1, rho2, k) from tests/golden/c4_params.json.  `--config c2` (dense
FP32 65536 x 1024, SRHT) and the other workloads of synthetic/configs.py stay available.

One step = one whole path: sketch (a1), factor + inverse (a2), Gram + rhs
(a3), basis recursion (a4), evaluation of all T lambdas (a6), with A and B
resident in HBM.  `value` and the latencies come from K steps run without
per-kernel events; the per-kernel table and the roofline come from the same K
steps repeated with CUDA events around every launch.  `e2e` repeats the step through the same C ABI from pinned
host buffers (problem creation with its host->device copy, and the device->
host read of X, inside the timed region).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun (N > 1) every rank solves its own replica of the workload
(weak scaling, no collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ridge paths/sec at rel-err≤1e-6 vs FP64 oracle; p50/p99 latency; %HBM peak"
WORKLOADS = {
    "c2": "dense FP32 A 65536x1024, sigma_k=1/k with Haar factors, b=Ax*+1% noise, SRHT m=2048, "
          "T=200 lambdas log-spaced in [1e-6,1]*||A||_2^2, L=27",
    "c1": "dense FP64 A 2000x100, columns (1+j)^-0.8, Gaussian sketch m=200, T=50 lambdas in "
          "[1e-4,1e2]*||A||_2^2, L=27",
    "c3": "CSR A 1048576x4096, 40 distinct uniform columns/row, N(0,1) FP32 values, b=Ax*+0.1z, SJLT s=8 "
          "m=8192, T=1000 lambdas in [1e-4,1e-2]*||A||_2^2, L=9",
    "c3t": "under-determined CSR A 4096x1048576 (transpose of c3), through the dual, SJLT s=8 m=8192, "
           "T=1000 lambdas in [1e-4,1e-2]*||A||_2^2, L=9",
    "c4": "dense BF16 A 262144x2048, columns (1+j)^-1, B 262144x64 from a planted X* + 1% noise, Gaussian "
          "sketch m=4096 with BF16 entries, T=500 lambdas in [1e-4,1e-2]*||A||_2^2, L=9",
    "c5": "serving: Poisson arrivals 2000/s, n~U[4096,65536], d~U[64,1024], T~U[20,500], 50% dense FP32 "
          "(columns (1+j)^-0.8, SRHT) / 50% CSR 1% density (CountSketch s=1), m=2d, lambda in "
          "[1e-3,1e-1]*||A||_F^2/d, parameters from the sketch (Theorem 4, eps=1e-7), jmax=32",
}
L2_NOTE = {"c2": "inputs larger than L2 (A is 256 MiB)", "c4": "inputs larger than L2 (A is 1 GiB)",
           "c3": "inputs larger than L2 (CSR A is 344 MB)", "c3t": "inputs larger than L2 (CSR A is 344 MB)",
           "c1": "A is 1.5 MiB: L2-resident, latency-bound"}
# FP32 lanes per SM and SM count of GB300; max SM clock 2070 MHz
FP32_INSTR_PEAK = 152 * 128 * 2.07e9
FP64_FMA_PEAK = 152 * 2 * 2.07e9
# FP32 instructions per float-float multiply-add as implemented (common.cuh):
# two_prod 2, cross terms 2 (dd x dd) / 1 (float x dd), TwoSum 6, low-word add 2
INSTR_PER_MAC = {"gram": 10, "sketch_gram": None, "loop_gram_product": 12, "loop_precond_update": 12,
                 "inverse_syrk": 12, "factor_syrk": 12, "factor_trsm": 12, "rhs": 11, "dual_map": 11}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ihsbin", choices=["ihsbin", "reference"])
    ap.add_argument("--config", default="c4")
    ap.add_argument("--compute", default="f32x2", choices=["f32x2", "f64"])
    ap.add_argument("--jmax", type=int, default=16)
    ap.add_argument("--slice-weight", type=int, default=0,
                    help="slice pairs kept by the recursion's tensor-core products (0 = 6: float-float class)")
    ap.add_argument("--form", default="auto", choices=["auto", "residual", "increment"],
                    help="how the tensor-core recursion carries the basis (auto = residual where it runs)")
    ap.add_argument("--precond-weight", type=int, default=0,
                    help="residual form: slice pairs kept by P_l r (0 = from the conditioning bound)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-check", action="store_true")
    ap.add_argument("--auto", action="store_true",
                    help="parameters from the sketch (rho from d_e, k from Theorem 4 at --eps) on both sides")
    ap.add_argument("--eps", type=float, default=1e-7)
    ap.add_argument("--requests", type=int, default=4096, help="serving workload (c5): number of requests")
    ap.add_argument("--rows", type=int, default=0,
                    help="the workload's structure at this many rows (for profiling captures on a few GB; "
                         "0 = the workload's own size)")
    ap.add_argument("--slots", type=int, default=6, help="serving workload (c5): concurrent slots")
    ap.add_argument("--adaptive", type=int, default=0, metavar="M0",
                    help="a step starts with Algorithm 4 from sketch dimension M0 at lambda_min (the path then "
                         "runs on the m it settles on, parameters from the sketch as with --auto)")
    ap.add_argument("--losses", type=int, default=0, metavar="N_TEST",
                    help="validation workload: N_TEST held-out rows drawn with the training rows; a step "
                         "returns the training and test losses of every lambda (Section 6.1) instead of X")
    return ap.parse_args()


def load_params(config):
    with open(os.path.join(ROOT, "tests", "golden", f"{config}_params.json")) as f:
        return json.load(f)


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region (read-only query)."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9 and f[1].replace(".", "").isdigit():
                    rows.append(f)
        except OSError:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]), "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows if r[3] not in ("", "[N/A]"))}


# ------------------------------------------------------------------------ CPU oracle
def _timed(fn, *a):
    t = time.perf_counter()
    r = fn(*a)
    return r, time.perf_counter() - t


def oracle_sample(prob, par, jmax=0, target_s=1.5, A=None):
    """The FP64 oracle, as it stands, on a bounded sample of the path (about 5 s), extrapolated to
    one whole path:
      * the sketch: all of it, except for the Gaussian sketch, whose rows are drawn and applied in
        blocks (r rows of S timed, x m / r);
      * the Gram of A_hat: all of it up to 2^34 multiply-adds, else a block of rows (x N / rows);
      * the right-hand side A_hat^T B and one factor of G_S + lam0 I: whole (x L for the factor);
      * the basis of the median-k interval with the same truncation jmax as the GPU run, its first
        k_s terms (k_s doubled until a sample takes `target_s`), extrapolated by the product
        columns of the recursion, sum over steps i of min(i, J) K, to every interval, plus its
        evaluation.
    A: the oracle's matrix when the caller already holds it (data preparation, not timed)."""
    from oracle import ihsbin as ob
    from oracle import sketch as osk
    A = oracle_matrix(prob) if A is None else A
    if "tau" in par:   # the library's own plan (sketch-derived parameters)
        plan = ob.Plan(prob.lambda_min, prob.lambda_max, par["L"], np.array(par["edges"]), np.array(par["lam0"]),
                       np.array(par["tau"]), np.array(par["k"]))
    else:
        plan = ob.make_plan(prob.lambda_min, prob.lambda_max, par["rho1"], par["rho2"], par["k"], L=par["L"])
    (Ahat, c, _), t_rhs = _timed(ob.tall_form, A, prob.B)
    N, D = Ahat.shape
    bf16 = prob.storage == "bf16"
    if prob.sketch == "gaussian" and prob.m * N * D > (1 << 32):
        r = 8
        while True:
            S, t_s = _timed(lambda rr: osk._round_bf16(osk.gaussian_entries(prob.m, N, prob.sketch_seed,
                                                                                 rows=np.arange(rr)))
                            if bf16 else osk.gaussian_entries(prob.m, N, prob.sketch_seed, rows=np.arange(rr)), r)
            SAr, t_a = _timed(lambda: S @ Ahat)
            if t_s + t_a >= target_s or 2 * r > prob.m:
                break
            r *= 2
        t_sketch = (t_s + t_a) * prob.m / r
        SA = np.tile(SAr, (prob.m // r + 1, 1))[:prob.m]   # stand-in of the right shape for the timing below
        sk_note = f"Gaussian sketch: {r} of {prob.m} rows of S drawn and applied ({t_s + t_a:.2f}s, x m/{r})"
    else:
        SA, t_sketch = _timed(osk.apply, prob.sketch, Ahat, prob.m, prob.s, prob.sketch_seed, bf16)
        sk_note = f"sketch whole ({t_sketch:.2f}s)"
    GS, t_gs = _timed(lambda: SA.T @ SA)
    if hasattr(Ahat, "tocsr") or N * D * D <= (1 << 34):
        G, t_gram = _timed(lambda: Ahat.T @ Ahat)
        G = np.asarray(G.todense()) if hasattr(G, "todense") else G
        gr_note = f"Gram whole ({t_gram:.2f}s)"
    else:
        nb = max(1024, min(N, (1 << 34) // (D * D)))
        G, t_b = _timed(lambda: Ahat[:nb].T @ Ahat[:nb])
        t_gram = t_b * N / nb
        G = G * (N / nb)
        gr_note = f"Gram: {nb} of {N} rows ({t_b:.2f}s, x N/{nb})"
    t_fixed = t_sketch + t_gs + t_gram + t_rhs
    ks = np.array(plan.k)
    L = len(ks)
    K = c.shape[1] if c.ndim == 2 else 1
    l = int(np.argsort(ks)[L // 2])          # the median-k interval
    P, t_factor = _timed(ob.precond, GS, plan.lam0[l])
    J = lambda k: k if jmax <= 0 else min(k, jmax)
    cols = lambda k: sum(min(i, J(k)) for i in range(1, k)) + 1    # product columns (per rhs column) of a basis
    lams = prob.lambdas[(prob.lambdas >= plan.edges[l]) & (prob.lambdas <= plan.edges[l + 1])]
    k_s = min(4, int(ks[l]))
    while True:
        t1 = time.perf_counter()
        ut = ob.basis(lambda V: G @ V, P, c, plan.tau[l], k_s, jmax=jmax)
        for lam in lams:
            ob.evaluate(ut, plan.tau[l], plan.lam0[l], lam)
        t_cols = time.perf_counter() - t1
        if k_s >= int(ks[l]) or t_cols > target_s:
            break
        k_s = min(2 * k_s, int(ks[l]))
    per_path = t_fixed + L * t_factor + t_cols * sum(cols(int(k)) for k in ks) / cols(k_s)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return dict(value=1.0 / per_path, unit="paths/s", cores=cores, kind="oracle",
                sample=f"FP64 numpy oracle on the {prob.name} path: {sk_note}; {gr_note}; rhs ({t_rhs:.2f}s); "
                       f"the factor of interval {l} ({t_factor:.2f}s, x L={L}); its first {k_s} of k={int(ks[l])} "
                       f"basis terms (jmax={jmax if jmax > 0 else 'all'}, K={K}) with evaluation ({t_cols:.2f}s), "
                       f"extrapolated to all intervals by product columns; per-path time {per_path:.1f}s",
                t_fixed=t_fixed)


def oracle_matrix(prob):
    """A as the oracle consumes it: FP64 dense, or scipy CSR for sparse workloads (TF32 storage
    rounded by the oracle's TF32 rounding first)."""
    from oracle.precision import round_tf32
    tf32 = prob.storage == "tf32"
    if prob.layout == "csr":
        import scipy.sparse as sp
        val = round_tf32(prob.val) if tf32 else prob.val
        return sp.csr_matrix((val.astype(np.float64), prob.col_idx, prob.row_ptr), shape=(prob.n, prob.d))
    return round_tf32(prob.A).astype(np.float64) if tf32 else prob.dense_f64()


def config_for(args, prob, par, world=1):
    """The `config` object of both arms' JSON lines (identical keys and values)."""
    return {"workload": WORKLOADS.get(args.config, args.config) + (
                f"; plus {args.losses} held-out rows of the same model, a step returns the training "
                f"and test losses of every lambda (X not formed)" if args.losses else "") + (
                f"; the sketch dimension chosen by Algorithm 4 from m0={args.adaptive} at lambda_min "
                f"inside each step" if args.adaptive else ""),
            "jmax": args.jmax,
            "slice_weight": args.slice_weight or 6,
            "form": args.form, "precond_weight": args.precond_weight or "auto",
            "storage": prob.storage,
            "l2": L2_NOTE.get(args.config, "see workload"),
            "params": (f"tests/golden/{args.config[:-1] if args.config == 'c3t' else args.config}_params.json"
                       if par is not None and "tau" not in par else
                       "from the sketch (rho from d_e, k from Theorem 4 at eps)"),
            "parallelism": f"replicas x{world}", **({"rows": args.rows} if args.rows else {})}


def reference_arm(args, prob, par):
    """--impl reference: the FP64 oracle as it stands on the host cores (rank 0 only), each step a
    bounded sample of the same path (oracle_sample), with the GPU arm's truncation jmax."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    A = oracle_matrix(prob)            # data preparation, outside every sample
    for _ in range(args.warmup):
        oracle_sample(prob, par, jmax=args.jmax, A=A)
    times, vals = [], []
    info = None
    for _ in range(args.steps):
        t1 = time.perf_counter()
        info = oracle_sample(prob, par, jmax=args.jmax, A=A)
        times.append(time.perf_counter() - t1)
        vals.append(info["value"])
    value = statistics.median(vals)
    line = {"metric": METRIC, "value": value, "unit": "paths/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_for(args, prob, par, args.gpus),
            "impl": "reference",
            "cpu_baseline": {"value": value, "unit": "paths/s", "cores": info["cores"], "kind": "oracle",
                             "sample": info["sample"]},
            "e2e": {"value": value, "unit": "paths/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------ multi-rank
def max_over_ranks(value: float, dist=None, device="cpu") -> float:
    """The slowest rank's time (replicas: the job is done when the last rank is)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, units_per_rank: float, seconds: float) -> float:
    """Whole-job rate: units processed by all ranks / the max-over-ranks time."""
    return world * units_per_rank / seconds


# ---------------------------------------------------------------------------- GPU arm
def serving_arm(args):
    """Serving workload: the served float-float form (`--slots` concurrent requests) against the plain
    FP64 GPU method processing the same trace FIFO, one request at a time."""
    import torch
    from paper_2210_12212_gb300 import ihsbin as ihs
    from synthetic import serving_requests
    from synthetic.configs import _csr_uniform
    torch.cuda.set_device(0)
    trace = serving_requests(args.requests)
    rng = np.random.default_rng(12345)
    # one device buffer of FP32 data with (1+j)^-0.8 column scales; a dense request uses its
    # top-left n x d block in place (row stride 1024)
    big = (rng.standard_normal((65536, 1024), dtype=np.float32)
           * (1.0 + np.arange(1024, dtype=np.float32)) ** -0.8).astype(np.float32)
    big_dev = torch.from_numpy(big).cuda()
    colsq = np.cumsum(np.cumsum(big.astype(np.float64) ** 2, axis=0), axis=1)  # prefix sums for ||A||_F^2
    reqs = []
    for r in trace:
        n, d, T = r["n"], r["d"], r["T"]
        rr = np.random.default_rng(1000 + r["seed"])
        b = rr.standard_normal(n)
        if r["layout"] == "dense":
            fro2 = colsq[n - 1, d - 1]
            entry = dict(kind="dense", n=n, d=d, T=T, b=b, fro2=fro2)
        else:
            per = max(1, int(round(0.01 * d)))
            rp, cols, vals = _csr_uniform(rr, n, d, per)
            entry = dict(kind="csr", n=n, d=d, T=T, b=b, csr=(rp, cols, vals),
                         fro2=float(np.sum(vals.astype(np.float64) ** 2)))
        scale = entry["fro2"] / d
        entry["lambdas"] = np.geomspace(1e-3 * scale, 1e-1 * scale, T)
        entry["arrival"] = r["arrival_s"]
        reqs.append(entry)
    arrivals = np.array([e["arrival"] for e in reqs])

    def build(compute):
        built = []
        for e in reqs:
            kw = dict(m=2 * min(e["n"], e["d"]), seed=7, eps=1e-7, auto_rho=True, jmax=32, compute=compute)
            if e["kind"] == "dense":
                A = big_dev[:e["n"], :e["d"]]
                built.append(ihs.make_request(A, e["b"], e["lambdas"], dtype="f32", sketch="srht", **kw))
            else:
                built.append(ihs.make_request(B=e["b"], lambdas=e["lambdas"], dtype="f32", csr=e["csr"],
                                              shape=(e["n"], e["d"]), sketch="countsketch", s=1, **kw))
        return built

    ctx = ihs.Context(0)

    def run(compute, slots):
        built = build(compute)
        arr = (ihs.Request * len(built))(*[b[0] for b in built])
        res = np.zeros(len(built), dtype=np.int32)
        lat = np.zeros(len(built))
        cfg = ihs.ServeConfig(slots, 120 << 30)
        t0 = time.perf_counter()
        ihs._check(ihs._lib.ihsbin_serve(ctx.h, ihs.C.byref(cfg), ihs.C.cast(arr, ihs.C.c_void_p), len(built),
                                         ihs._ptr(arrivals), ihs._ptr(res), ihs._ptr(lat)))
        wall = time.perf_counter() - t0
        outs = [b[2] for b in built]
        return dict(wall=wall, lat=lat, res=res, outs=outs)

    served = run("f32x2", args.slots)
    note("served run done")
    fifo = run("f64", 1)
    note("FIFO run done")
    errs = [float(np.max(np.linalg.norm((a - b).reshape(len(a), -1), axis=1)
                         / np.maximum(np.linalg.norm(b.reshape(len(b), -1), axis=1), 1e-300)))
            for a, b in zip(served["outs"], fifo["outs"])]
    # a sample of served results against the FP64 oracle (its own sketch-derived plan, as the library's)
    oracle_check = serving_oracle_sample(reqs, served["outs"], big, n_each=3)
    note("oracle sample done")

    def summary(r):
        lat = np.sort(r["lat"])
        return {"paths_per_s": len(lat) / r["wall"], "p50_ms": 1e3 * float(np.percentile(lat, 50)),
                "p99_ms": 1e3 * float(np.percentile(lat, 99)), "wall_s": r["wall"],
                "failed": int(np.sum(r["res"] != 0))}
    line = {"metric": METRIC, "value": summary(served)["paths_per_s"], "unit": "paths/s", "n_gpus": 1,
            "steps": args.requests, "warmup": 0, "ms_per_step": 1e3 * served["wall"] / args.requests,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32x2",
            "data": "synthetic", "config": {"workload": WORKLOADS["c5"], "requests": args.requests,
                                            "slots": args.slots, "budget_gb": 120},
            "served_f32x2": summary(served), "fifo_f64": summary(fifo),
            "max_rel_err_served_vs_fp64": max(errs), "oracle_sample": oracle_check}
    print(json.dumps(line), flush=True)


def serving_oracle_sample(reqs, outs, big, n_each=3):
    """The n_each smallest dense and CSR requests of the trace through the FP64 oracle, with the plan
    the oracle derives from its own sketch (rho from d_e, k from Theorem 4 at eps = 1e-7): max
    relative error of the served x(lambda) over each request's lambdas."""
    import scipy.sparse as sp
    from oracle import ihsbin as ob
    from oracle import sketch as osk
    res = []
    for kind in ("dense", "csr"):
        idx = sorted((i for i, e in enumerate(reqs) if e["kind"] == kind), key=lambda i: reqs[i]["n"] * reqs[i]["d"])
        for i in idx[:n_each]:
            e = reqs[i]
            n, d = e["n"], e["d"]
            if kind == "dense":
                A = big[:n, :d].astype(np.float64)
                sk, s = "srht", 1
            else:
                rp, ci, va = e["csr"]
                A = sp.csr_matrix((va.astype(np.float64), ci, rp), shape=(n, d))
                sk, s = "countsketch", 1
            m = 2 * min(n, d)
            B = e["b"].reshape(-1, 1)
            Ahat, c, _ = ob.tall_form(A, B)
            SA = osk.apply(sk, Ahat, m, s, 7)
            GS = SA.T @ SA
            lam = e["lambdas"]
            plan = ob.auto_plan(GS, m, lam[0], lam[-1], eps=1e-7)
            X = ob.ihs_bin_path(A, B, sk, m, s, 7, plan, lam).X
            got = outs[i].reshape(X.shape)
            err = float(np.max(np.linalg.norm((got - X).reshape(len(X), -1), axis=1)
                               / np.linalg.norm(X.reshape(len(X), -1), axis=1)))
            res.append({"request": i, "kind": kind, "n": n, "d": d, "T": len(lam), "max_rel_err": err})
    return {"requests": res, "max_rel_err": max(r["max_rel_err"] for r in res), "pass": all(r["max_rel_err"] <= 1e-6
                                                                                            for r in res)}


_T0 = time.perf_counter()


def note(msg):
    """Progress of the run on stderr (the JSON result line alone goes to stdout)."""
    print(f"[bench {time.perf_counter() - _T0:8.1f}s] {msg}", file=sys.stderr, flush=True)


def main():
    args = parse()
    if args.impl == "reference" and int(os.environ.get("RANK", "0")) != 0:
        return  # the reference arm runs on rank 0 alone; the other ranks exit without work
    if args.config == "c5":
        serving_arm(args)
        return
    from synthetic import make_problem, make_split
    A_test = B_test = None
    if args.losses > 0:
        prob, A_test, B_test = make_split(args.config, args.losses, seed=0)
    else:
        prob = make_problem(args.config, seed=0, **({"n": args.rows} if args.rows else {}))
    note(f"workload {args.config} generated")
    if args.adaptive:
        args.auto = True
    par = None if args.auto else load_params(args.config[:-1] if args.config == "c3t" else args.config)
    if args.impl == "reference":
        reference_arm(args, prob, par)
        return

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2210_12212_gb300 import ihsbin as ihs

    ctx = ihs.Context(local)
    B_dev = torch.from_numpy(np.ascontiguousarray(prob.B)).cuda()
    B_pin = torch.from_numpy(np.ascontiguousarray(prob.B)).pin_memory()  # the end-to-end path's host inputs are pinned
    T = len(prob.lambdas)
    X_dev = torch.empty((T, prob.d, prob.K), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    if par is None:
        bkw = dict(k=None, k_default=0, eps=args.eps, auto_rho=True, jmax=args.jmax, compute=args.compute,
                   slice_weight=args.slice_weight)
    else:
        bkw = dict(L=par["L"], k=par["k"], rho1=par["rho1"], rho2=par["rho2"], jmax=args.jmax,
                   compute=args.compute, slice_weight=args.slice_weight)
    bkw.update(form=args.form, precond_weight=args.precond_weight)
    entries = "bf16" if prob.storage == "bf16" else "f64"
    if prob.layout == "csr":
        csr_dev = tuple(torch.from_numpy(np.ascontiguousarray(a)).cuda()
                        for a in (prob.row_ptr, prob.col_idx, prob.val))
        make_dev = lambda: ihs.Problem(ctx, B=B_dev, dtype=prob.storage, csr=csr_dev, shape=(prob.n, prob.d))
        csr_pin = tuple(torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
                        for a in (prob.row_ptr, prob.col_idx, prob.val))
        make_host = lambda: ihs.Problem(ctx, B=B_pin, dtype=prob.storage, csr=csr_pin, shape=(prob.n, prob.d))
        host_bytes = prob.row_ptr.nbytes + prob.col_idx.nbytes + prob.val.nbytes
    else:
        A_np = np.ascontiguousarray(prob.A)
        A_dev = torch.from_numpy(A_np.view(np.int16) if prob.storage == "bf16" else A_np).cuda()
        A_pin = torch.from_numpy(A_np.view(np.int16) if prob.storage == "bf16" else A_np).pin_memory()
        make_dev = lambda: ihs.Problem(ctx, A_dev, B_dev, dtype=prob.storage)
        make_host = lambda: ihs.Problem(ctx, A_pin, B_pin, dtype=prob.storage)
        host_bytes = A_pin.numel() * A_pin.element_size()
    p = make_dev()
    if A_test is not None:
        At_np = np.ascontiguousarray(A_test)
        At_dev = torch.from_numpy(At_np.view(np.int16) if prob.storage == "bf16" else At_np).cuda()
        Bt_dev = torch.from_numpy(np.ascontiguousarray(B_test)).cuda()
        At_pin = torch.from_numpy(At_np.view(np.int16) if prob.storage == "bf16" else At_np).pin_memory()
        Bt_pin = torch.from_numpy(np.ascontiguousarray(B_test)).pin_memory()
        host_bytes += At_pin.numel() * At_pin.element_size() + Bt_pin.numel() * 8

    adapt = {}

    def step(pp, out=None):
        if args.adaptive:
            adapt.update(pp.adaptive_sketch(prob.sketch, args.adaptive, prob.lambda_min, s=prob.s,
                                            seed=prob.sketch_seed, entries=entries, compute=args.compute,
                                            stream=stream))
        else:
            pp.sketch(prob.sketch, prob.m, prob.s, prob.sketch_seed, entries=entries, stream=stream)
        pp.build_basis(prob.lambda_min, prob.lambda_max, stream=stream, **bkw)
        if A_test is not None:  # losses of every lambda, X never formed
            dev = out is not None
            return pp.path_losses(prob.lambdas, At_dev if dev else At_pin, Bt_dev if dev else Bt_pin,
                                  test_dtype=prob.storage, stream=stream)
        return pp.eval_path(prob.lambdas, out=out, stream=stream)

    # untimed steps until the library's autotuner has settled every launch site the steps use (each
    # candidate geometry is timed on a few launches first: the table stops changing), then the W
    # warm-up steps
    prev = None
    for _ in range(32):
        step(p, X_dev)
        torch.cuda.synchronize()
        rep = ihs.tuning_report()
        if rep == prev:
            break
        prev = rep
    for _ in range(max(args.warmup, 0)):
        step(p, X_dev)
    torch.cuda.synchronize()
    note("warm-up done")
    recursion = None
    if args.warmup > 0 and not args.adaptive:
        f, w = p.recursion_form()
        recursion = {"form": f, "precond_weight": w}

    # ---- timed region: K steps as a user runs them (no per-kernel events)
    def timed_steps(instrumented):
        p.set_timing(instrumented)
        p.reset_stats()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        e_start = torch.cuda.Event(enable_timing=True)
        e_stop = torch.cuda.Event(enable_timing=True)
        e_start.record(stream)
        for s in range(args.steps):
            evs[s][0].record(stream)
            step(p, X_dev)
            evs[s][1].record(stream)
        e_stop.record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        out = (max_over_ranks(e_start.elapsed_time(e_stop), dist, "cuda"), sorted(a.elapsed_time(b) for a, b in evs),
               p.kernel_stats(), p.phase_times())
        p.set_timing(False)
        return out

    # clocks sampled every 50 ms through both timed regions
    with ClockSampler(local) as clk:
        elapsed_ms, lat, stats_clean, phases = timed_steps(False)
        # ---- the same K steps again with CUDA events around every launch, on the launching stream:
        # the per-kernel device times of the roofline and of the kernel table
        inst_ms, _, stats, _ = timed_steps(True)
        xstats = p.kernel_exec()

    # ---- end to end through the C ABI from pinned host buffers
    e2e = None
    if not args.no_e2e:
        ke = max(1, min(args.steps, 5))
        # X is read back every step into pinned host memory allocated once, like the pinned inputs
        X_pin = torch.empty(tuple(X_dev.shape), dtype=torch.float64).pin_memory() if A_test is None else None
        q = make_host()   # warm the host path once
        step(q, X_pin)
        q.close()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(ke):
            q = make_host()
            Xh = step(q, X_pin)
            q.close()
        torch.cuda.synchronize()
        te = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
        e2e = {"value": job_throughput(world, ke, te), "unit": "paths/s",
               "h2d_bytes_per_step": int(host_bytes + prob.B.nbytes + prob.lambdas.nbytes),
               "d2h_bytes_per_step": int(sum(a.nbytes for a in Xh if a is not None) if isinstance(Xh, tuple)
                                         else Xh.numel() * Xh.element_size())}

    # ---- parity of the timed result against the FP64 oracle (sampled lambdas, rank 0)
    check = None
    note("timed region done")
    if rank == 0 and not args.no_check:
        if A_test is not None:
            losses = step(p, X_dev)
            p.eval_path(prob.lambdas, out=X_dev, stream=stream)
            torch.cuda.synchronize()
        pprob = prob
        if args.adaptive:  # the path ran on the sketch Algorithm 4 left behind
            import dataclasses
            pprob = dataclasses.replace(prob, m=int(adapt["m"]), sketch_seed=prob.sketch_seed + int(adapt["doublings"]))
        check = parity_sample(pprob, par, X_dev.cpu().numpy(), tol=1e-9 if args.compute == "f64" else 1e-6,
                              eps=args.eps)
        if args.adaptive:
            check["adaptive"] = adaptive_check(prob, args.adaptive, adapt)
        if A_test is not None:
            check["losses"] = losses_check(prob, A_test, B_test, X_dev.cpu().numpy(), losses)

    # ---- roofline of the dominant kernel (largest device time in the timed region)
    dom = max(stats.items(), key=lambda kv: kv[1][1])
    name, (launches, ms, flops, byts) = dom
    bound, peak, peak_note = kernel_peak(name, args.compute)
    xf0, xb0 = xstats.get(name, (flops, byts))
    if (xf0, xb0) != (flops, byts) and ms > 0:
        # an exact-slice product: its bound is the resource its executed work uses most (the tensor pipe
        # for wide column panels, HBM for the slice images of thin ones)
        ft = xf0 / (ms * 1e-3) / 1e12 / measured_peak("bf16_tflops_sustained", 1700.0)[0]
        fh = xb0 / (ms * 1e-3) / 1e9 / measured_peak("hbm_gbs", 6800.0)[0]
        if ft >= fh:
            peak, how = measured_peak("bf16_tflops_sustained", 1700.0)
            bound, peak_note = "tensor", f"cuBLAS bf16 sustained (MEASURED_PEAKS.json), {how}"
        else:
            peak, how = measured_peak("hbm_gbs", 6800.0)
            bound, peak_note = "hbm", f"copy bandwidth (MEASURED_PEAKS.json hbm_gbs), {how}"
    if bound == "hbm":
        achieved, unit = (byts / (ms * 1e-3) / 1e9 if ms > 0 else 0.0), "GB/s"
    else:
        achieved, unit = (flops / (ms * 1e-3) / 1e12 if ms > 0 else 0.0), "TFLOP/s"
    traffic = read_traffic(name, launches / args.steps if args.steps else 0)
    roof = {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit, "frac": achieved / peak,
            "algorithmic_bytes_per_launch": byts / launches if launches else 0.0,
            "algorithmic_flops_per_launch": flops / launches if launches else 0.0,
            "traffic": traffic, "kernel": name, "launches_per_step": launches / args.steps,
            "avg_launch_ms": ms / launches, "peak_basis": peak_note}
    xf, xb = xstats.get(name, (flops, byts))
    if (xf, xb) != (flops, byts):
        # what the launches execute: the BF16 products of every kept slice pair and the slice images
        roof["executed"] = {"flops_per_launch": xf / launches, "bytes_per_launch": xb / launches,
                            "tflops": xf / (ms * 1e-3) / 1e12, "gbs": xb / (ms * 1e-3) / 1e9,
                            "frac_tensor": xf / (ms * 1e-3) / 1e12 / measured_peak("bf16_tflops_sustained", 1700.0)[0],
                            "frac_hbm": xb / (ms * 1e-3) / 1e9 / measured_peak("hbm_gbs", 6800.0)[0]}
    # the basis build as a phase (step a4): the method's bytes of every recursion launch per path
    # over the recursion's device time per path, against the copy bandwidth
    loop_cats = [k for k in stats if k.startswith("loop_")]
    bb = sum(stats[k][3] for k in loop_cats) / args.steps
    hbm_pk = measured_peak("hbm_gbs", 6800.0)[0]
    tb = phases["basis"]
    basis_roof = {"bound": "hbm", "bytes_per_path": bb, "ms_per_path": tb,
                  "achieved": bb / (tb * 1e-3) / 1e9 if tb > 0 else 0.0, "peak": hbm_pk,
                  "unit": "GB/s", "categories": loop_cats}
    basis_roof["frac"] = basis_roof["achieved"] / hbm_pk

    cpu = None
    note("parity done")
    if rank == 0 and not args.no_cpu and world == 1:
        info = oracle_sample(prob, par if par is not None else p.plan_dict_for_oracle(), jmax=args.jmax)
        cpu = {k: info[k] for k in ("value", "unit", "cores", "kind", "sample")}

    gpu_launches = int(sum(v[0] for v in stats_clean.values()))
    value = job_throughput(world, args.steps, elapsed_ms * 1e-3)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "paths/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": args.compute, "data": "synthetic",
            "config": config_for(args, prob, par, world),
            "latency_ms": {"p50": lat[len(lat) // 2], "p99": lat[min(len(lat) - 1, int(math.ceil(0.99 * len(lat))) - 1)]},
            "instrumented_ms_per_step": inst_ms / args.steps,
            "phase_ms": phases, "recursion": recursion,
            "tuning": [" ".join(x.split()[:1] + x.split()[2:3]) for x in ihs.tuning_report().splitlines()],
            "roofline": roof, "basis_roofline": basis_roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": gpu_launches,
            "clocks": clk.summary(), "parity": check,
            "kernels": {k: {"launches": v[0], "ms": v[1], "tflops": (v[2] / (v[1] * 1e-3) / 1e12 if v[1] else 0)}
                        for k, v in stats.items()},
        }
        print(json.dumps(line), flush=True)
    p.close()
    if dist:
        dist.destroy_process_group()


def parity_sample(prob, par, X, tol=1e-6, eps=1e-7):
    """Max relative error of the GPU path against the oracle's k_l-step IHS (Gram space) at 9 lambdas
    (the endpoints and 7 interior grid points), plus the distance of the oracle to x*(lambda).
    With par None the oracle derives its own plan from its sketch (oracle.ihsbin.auto_plan)."""
    from oracle import ihsbin as ob
    from oracle import sketch as osk
    A = oracle_matrix(prob)
    idx = np.unique(np.linspace(0, len(prob.lambdas) - 1, 9).round().astype(int))
    lams = prob.lambdas[idx]
    Ahat, c, dual = ob.tall_form(A, prob.B)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    SA = osk.apply(prob.sketch, Ahat, prob.m, prob.s, prob.sketch_seed, bf16_entries=prob.storage == "bf16",
                   workers=max(1, min(16, cores - 1)))
    GS = SA.T @ SA
    if par is None:
        plan = ob.auto_plan(GS, prob.m, prob.lambda_min, prob.lambda_max, eps=eps)
    else:
        plan = ob.make_plan(prob.lambda_min, prob.lambda_max, par["rho1"], par["rho2"], par["k"], L=par["L"])
    ref = ob.direct_path(A, prob.B, GS, plan, lams)
    err = [float(np.linalg.norm(X[i] - ref[t]) / np.linalg.norm(ref[t])) for t, i in enumerate(idx)]
    G = Ahat.T @ Ahat
    G = np.asarray(G.todense()) if hasattr(G, "todense") else G
    conv = []
    for t, lam in enumerate(lams):
        z = np.linalg.solve(G + lam * np.eye(G.shape[0]), c)
        xs = Ahat @ z if dual else z
        conv.append(float(np.linalg.norm(ref[t] - xs) / np.linalg.norm(ref[t])))
    return {"max_rel_err_vs_oracle": max(err), "lambdas_checked": len(idx), "pass": max(err) <= tol,
            "oracle_max_rel_dist_to_exact_ridge": max(conv)}


def adaptive_check(prob, m0, g):
    """Algorithm 4 on the device against the oracle's run: the m and step sequences (exact) and the
    decrements relative to the first."""
    from oracle import adaptive as oa
    o = oa.adaptive_for_problem(oracle_matrix(prob), prob.B, prob.sketch, m0, prob.s, prob.sketch_seed,
                                prob.lambda_min, bf16_entries=prob.storage == "bf16")
    n = min(len(o.delta), len(g["deltas"]))
    return {"m0": m0, "m": int(g["m"]), "iterations": int(g["iterations"]), "doublings": int(g["doublings"]),
            "m_sequence_equal": list(map(int, g["ms"])) == o.ms, "steps_equal": list(g["steps"]) == o.steps,
            "max_rel_err_delta": float(np.max(np.abs(np.asarray(g["deltas"][:n]) - np.asarray(o.delta[:n])))
                                       / o.delta[0])}


def losses_check(prob, A_test, B_test, X, losses):
    """The device losses against the oracle's losses of the same X at 9 lambdas (relative)."""
    from oracle import ihsbin as ob
    from synthetic.configs import bf16_bits_to_f32
    idx = np.unique(np.linspace(0, len(prob.lambdas) - 1, 9).round().astype(int))
    At = bf16_bits_to_f32(A_test).astype(np.float64) if prob.storage == "bf16" else A_test.astype(np.float64)
    tr, te = ob.path_losses(oracle_matrix(prob), prob.B, At, B_test, X[idx], prob.lambdas[idx])
    rel = lambda a, b: float(np.max(np.abs(a - b) / np.abs(b)))
    return {"max_rel_err_train": rel(losses[0][idx], tr), "max_rel_err_test": rel(losses[1][idx], te),
            "lambdas_checked": len(idx), "n_test": int(A_test.shape[0]),
            "test_loss_argmin_lambda": float(prob.lambdas[int(np.argmin(losses[1]))])}


def measured_peak(key, fallback):
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)[key]), "of measured"
    except (OSError, KeyError, ValueError):
        return fallback, "of fallback"


# Categories whose binding resource is HBM: every step of the recursion streams the live
# intervals' preconditioner slices (12 bytes per entry), which do not stay in L2; the
# elementwise steps of the recursion and the slicing / joining kernels move data only.
HBM_BOUND = ("loop_precond_tc", "loop_precond_update", "loop_slice", "factor_slice", "gram_slice", "gram_combine",
             "loss_slice", "loss_resid")


def kernel_peak(name, compute):
    """(bound, peak, how the peak was obtained) for a kernel category; TFLOP/s, or GB/s for hbm."""
    if name in HBM_BOUND:
        pk, how = measured_peak("hbm_gbs", 6800.0)
        return "hbm", pk, f"copy bandwidth (MEASURED_PEAKS.json hbm_gbs), {how}"
    if name in ("gram_tc_mma", "loop_gram_tc", "loss_image_tc", "sketch_tc", "sketch_gram", "rhs", "inverse_tc",
                "trtri_tc", "factor_syrk_tc"):  # tensor-core products, inside a long step
        pk, how = measured_peak("bf16_tflops_sustained", 1700.0)
        return "tensor", pk, f"cuBLAS bf16 sustained (MEASURED_PEAKS.json), {how}"
    if compute == "f64":
        return "alu", 2 * FP64_FMA_PEAK / 1e12, "FP64 FMA rate from unit counts (152 SMs x 2 DFMA/clk x 2070 MHz)"
    instr = INSTR_PER_MAC.get(name) or 12
    return "alu", 2 * FP32_INSTR_PEAK / instr / 1e12, (
        f"float-float multiply-add rate from unit counts: 152 SMs x 128 FP32 lanes x 2070 MHz "
        f"/ {instr} FP32 instructions per multiply-add")


def read_traffic(kernel, launches_per_step):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it matches the current
    kernel source (the summary records a hash of csrc/); otherwise null."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2210_12212_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        h.update(open(os.path.join(csrc, f), "rb").read())
    digest = h.hexdigest()[:16]
    for line in open(path):
        f = line.split()
        if len(f) >= 3 and f[0] == kernel and f[1] == digest:
            return float(f[2])
    return None


if __name__ == "__main__":
    main()
