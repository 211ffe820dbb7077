"""Per-interval iteration parameters for a workload, chosen by the FP64 oracle.

TEST INFRASTRUCTURE: this script calls only ``oracle/`` and ``synthetic`` and
writes ``tests/golden/<config>_params.json``, which tests and the benchmark
pass unchanged to both the CUDA path and the oracle.

Rule (a reading; the paper leaves rho1, rho2 and k to the user):
* rho_l = min(d_e(lam0_l) / m, 0.95) with the effective dimension of
  Section 4.2, d_e = ||D||_F^2 / ||D||_2^2, D = diag(sigma_i / sqrt(sigma_i^2 + lam0)),
  computed from the exact spectrum of A^T A; rho1/rho2 from the Gaussian-sketch
  theorem with ||D||_2 = 1 and eta -> 0: (1 +- sqrt(rho_l))^2.
* tau_l from Theorem 4 (proof form), see oracle.ihsbin.step_size.
* k_l = the smallest k for which k plain IHS steps (the quantity IHS-BIN
  reproduces exactly, Proposition 1) are within `eps` of x*(lam) in relative
  2-norm at every grid lambda of the interval and at its two edges.

Usage:  python -m oracle.tune c2 [--eps 1e-7] [--seed 0]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np
import scipy.linalg as sla

from . import ihsbin as ob
from . import sketch as sk

GOLDEN = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests", "golden")


def _tall(prob):
    import scipy.sparse as sp
    if prob.layout == "csr":
        A = sp.csr_matrix((prob.val.astype(np.float64), prob.col_idx, prob.row_ptr), shape=(prob.n, prob.d))
    else:
        A = prob.dense_f64()
    B = prob.B
    if prob.n >= prob.d:
        G = A.T @ A
        c = A.T @ B
        Ahat = A
    else:
        Ahat = A.T.tocsr() if hasattr(A, "tocsr") else A.T
        G = A @ A.T
        c = B.copy()
    G = np.asarray(G.todense()) if hasattr(G, "todense") else np.asarray(G)
    return Ahat, G, np.asarray(c)


def tune(prob, eps: float = 1e-7, kmax: int = 3000, rho_cap: float = 0.95, bf16_sketch: bool = False):
    t0 = time.time()
    Ahat, G, c = _tall(prob)
    D = G.shape[0]
    lmin, lmax = prob.lambda_min, prob.lambda_max
    L = ob.num_intervals(lmin, lmax)
    edges = ob.interval_edges(lmin, lmax, L)
    lam0 = np.sqrt(edges[:-1] * edges[1:])
    sig2 = np.clip(np.linalg.eigvalsh(G), 0.0, None)
    rho = np.empty(L)
    for l in range(L):
        Dd = sig2 / (sig2 + lam0[l])
        de = Dd.sum() / Dd.max()
        rho[l] = min(de / prob.m, rho_cap)
    r1 = (1 + np.sqrt(rho)) ** 2
    r2 = (1 - np.sqrt(rho)) ** 2
    SA = sk.apply(prob.sketch, Ahat, prob.m, prob.s, prob.sketch_seed, bf16_entries=bf16_sketch)
    GS = SA.T @ SA
    ks, conv = [], []
    for l in range(L):
        tau = ob.step_size(edges[l], edges[l + 1], r1[l], r2[l])
        lams = [edges[l], edges[l + 1]] + [x for x in prob.lambdas if edges[l] <= x <= edges[l + 1]]
        lams = np.array(sorted(set(lams)))
        P = ob.precond(GS, lam0[l])
        Xs = np.stack([sla.cho_solve(sla.cho_factor(G + lam * np.eye(D), lower=True), c) for lam in lams])
        K = c.shape[1]
        # all lambdas of the interval side by side: column block t holds x(lams[t]) (D x K)
        Xs_cat = np.concatenate(list(Xs), axis=1)
        C_cat = np.tile(c, (1, len(lams)))
        lam_cols = np.repeat(lams, K)[None, :]
        nrm = np.array([np.linalg.norm(Xs[t]) for t in range(len(lams))])
        X = np.zeros_like(Xs_cat)
        k_need = kmax
        err = np.inf
        for k in range(1, kmax + 1):
            X = X - tau * P.solve(G @ X - C_cat + lam_cols * X)      # one IHS step for every lambda
            diff = (X - Xs_cat).reshape(D, len(lams), K)
            err = float(np.max(np.linalg.norm(diff, axis=(0, 2)) / nrm))
            if err <= eps:
                k_need = k
                break
        ks.append(int(k_need))
        conv.append(float(err))
    return dict(L=int(L), rho=rho.tolist(), rho1=r1.tolist(), rho2=r2.tolist(), k=ks, eps=eps,
                conv_err=conv, lambda_min=lmin, lambda_max=lmax, seconds=time.time() - t0)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("config")
    ap.add_argument("--eps", type=float, default=1e-7)
    ap.add_argument("--seed", type=int, default=0)
    a = ap.parse_args()
    from synthetic import make_problem
    prob = make_problem(a.config, seed=a.seed)
    out = tune(prob, eps=a.eps, bf16_sketch=(prob.storage == "bf16"))
    out.update(config=a.config, seed=a.seed, generated_by="python -m oracle.tune " + a.config)
    os.makedirs(GOLDEN, exist_ok=True)
    path = os.path.join(GOLDEN, f"{a.config}_params.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(path, "L", out["L"], "k", out["k"], "sum k^2/2", sum(k * (k - 1) // 2 for k in out["k"]),
          f"{out['seconds']:.1f}s")


if __name__ == "__main__":
    main()
