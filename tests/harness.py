"""Shared test/bench plumbing: run a workload through the C ABI and through the oracle.

Only argument preparation lives here (no IHS-BIN arithmetic): the parameters
(rho per interval, k per interval) are passed identically to both sides.
"""
from __future__ import annotations

import numpy as np

from synthetic import make_problem


def rel_err_max(X, Xref):
    """max over lambda of ||X_t - Xref_t||_F / ||Xref_t||_F."""
    X = np.asarray(X, dtype=np.float64)
    Xref = np.asarray(Xref, dtype=np.float64)
    num = np.linalg.norm((X - Xref).reshape(X.shape[0], -1), axis=1)
    den = np.linalg.norm(Xref.reshape(X.shape[0], -1), axis=1)
    return float(np.max(num / np.maximum(den, 1e-300)))


def oracle_A(prob):
    """A as the oracle consumes it: FP64 dense array or scipy CSR (values widened exactly; TF32
    storage rounded by the oracle's own TF32 rounding first)."""
    from oracle.precision import round_tf32
    tf32 = prob.storage == "tf32"
    if prob.layout == "csr":
        import scipy.sparse as sp
        val = round_tf32(prob.val) if tf32 else prob.val
        return sp.csr_matrix((val.astype(np.float64), prob.col_idx, prob.row_ptr), shape=(prob.n, prob.d))
    return round_tf32(prob.A).astype(np.float64) if tf32 else prob.dense_f64()


def gpu_problem(ihs, ctx, prob, device_inputs=False):
    """Create the library problem for a synthetic workload (host copies unless device_inputs)."""
    if prob.layout == "csr":
        arrs = (prob.row_ptr, prob.col_idx, prob.val)
        if device_inputs:
            import torch
            arrs = tuple(torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs)
        return ihs.Problem(ctx, B=prob.B, dtype=prob.storage, csr=arrs, shape=(prob.n, prob.d))
    A = prob.A
    if device_inputs:
        import torch
        A = torch.from_numpy(np.ascontiguousarray(A).view(np.int16) if prob.storage == "bf16"
                             else np.ascontiguousarray(A)).cuda()
    return ihs.Problem(ctx, A, prob.B, dtype=prob.storage)


def default_params(prob, L, k, rho=None):
    """Per-interval (rho1, rho2, k) arrays: the Gaussian-sketch rule with a single rho."""
    D = min(prob.n, prob.d)
    if rho is None:
        rho = min(D / prob.m, 0.81)
    r1 = (1 + np.sqrt(rho)) ** 2
    r2 = (1 - np.sqrt(rho)) ** 2
    return np.full(L, r1), np.full(L, r2), np.full(L, k, dtype=np.int32)


def small(name, **kw):
    return make_problem(name, seed=kw.pop("seed", 0), **kw)
