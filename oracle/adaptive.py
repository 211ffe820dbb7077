"""Adaptive choice of the sketch dimension (Section 5.1, Algorithm 4), in plain FP64.

TEST INFRASTRUCTURE: the oracle of the repository's tests and benchmark
baseline; the CUDA library neither imports nor calls it.

The method runs preconditioned Newton-sketch (IHS) steps with an Armijo line
search on the ridge problem at lam = lambda_min and doubles m whenever one
step fails to shrink the decrement enough.  Readings of Algorithm 4 taken
here (the printed listing puts the doubling test after the loop):

* The problem is the tall form of Section 5.2 (A_hat = A for n >= d, the dual
  with A_hat = A^T for n < d): f(x) = 1/2 x^T (A_hat^T A_hat + lam I) x - c^T x
  with c = A_hat^T b (primal) or c = b (dual).  For n >= d this is the paper's
  1/2||Ax - b||^2 + lam/2||x||^2 less the constant 1/2||b||^2, which neither
  the Armijo test nor the decrement sees.  The gradient is
  A_hat^T A_hat x + lam x - c (the printed A^T(Ax - b + lam x) is read as in
  the IHS update).  With K right-hand sides f is the sum over the columns and
  one step size serves all of them.
* d_k = P_S grad f(x_k) with P_S = ((S A_hat)^T S A_hat + lam I)^-1, and the
  decrement delta_k = d_k^T grad f(x_k) (the printed delta and delta-tilde are
  the same quantity).
* Armijo: the smallest j >= 0 with
  f(x_k - g1^j d_k) <= f(x_k) - g2 g1^j d_k^T grad f(x_k); tau_k = g1^j.
* After x_{k+1} = x_k - tau_k d_k the new direction and decrement are formed;
  if delta_{k+1} >= g3 delta_k, m is doubled (while 2m <= m_max), a new sketch
  is drawn (seed + number of doublings so far) and d_{k+1}, delta_{k+1} are
  recomputed with it; the loop then continues from x_{k+1}.
* The loop stops when delta_k <= eps * delta_0 (the paper's absolute epsilon
  is taken relative to the first decrement, the problem's scale being
  arbitrary) or after max_iter steps.  The output is the final m.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, List

import numpy as np
import scipy.linalg as sla

from . import sketch as osk
from .ihsbin import tall_form


@dataclass
class AdaptiveResult:
    m: int                       # the final sketch dimension
    iterations: int              # line-search steps taken
    doublings: int
    x: np.ndarray                # final iterate (D x K; the dual variable for n < d)
    delta: List[float] = field(default_factory=list)   # delta_0, delta_1, ... (after any re-sketch)
    ms: List[int] = field(default_factory=list)        # m in force for each delta
    steps: List[float] = field(default_factory=list)   # tau_k
    curv: List[float] = field(default_factory=list)    # d_k^T H d_k (the quadratic's curvature along d_k)


def sketcher_for(kind: str, Ahat, s: int, seed: int, bf16_entries: bool = False) -> Callable[[int, int], np.ndarray]:
    """S A_hat for sketch dimension m and doubling count r (seed + r)."""
    return lambda m, r: osk.apply(kind, Ahat, m, s, seed + r, bf16_entries=bf16_entries)


def adaptive_sketch_dim(Ahat, c, lam: float, m0: int, sketcher: Callable[[int, int], np.ndarray],
                        eps: float = 1e-10, g1: float = 0.5, g2: float = 0.25, g3: float = 0.5,
                        max_iter: int = 100, m_max: int = 1 << 40, max_backtrack: int = 200) -> AdaptiveResult:
    """Algorithm 4 on f(x) = 1/2 x^T (A_hat^T A_hat + lam I) x - c^T x (see the module notes)."""
    c = c[:, None] if c.ndim == 1 else np.asarray(c, dtype=np.float64)
    G = Ahat.T @ Ahat
    G = np.asarray(G.todense()) if hasattr(G, "todense") else np.asarray(G, dtype=np.float64)
    D, K = c.shape
    H = G + lam * np.eye(D)

    def f(X):
        return 0.5 * float(np.sum(X * (H @ X))) - float(np.sum(c * X))

    def grad(X):
        return H @ X - c

    def factor(m, r):
        SA = sketcher(m, r)
        return sla.cho_factor(SA.T @ SA + lam * np.eye(D), lower=True)

    m, r = m0, 0
    P = factor(m, r)
    x = np.zeros((D, K))
    g = grad(x)
    d = sla.cho_solve(P, g)
    delta = float(np.sum(d * g))
    res = AdaptiveResult(m=m, iterations=0, doublings=0, x=x, delta=[delta], ms=[m])
    delta0 = delta
    k = 0
    while delta > eps * delta0 and k < max_iter:
        fx = f(x)
        j = 0
        while f(x - g1 ** j * d) > fx - g2 * g1 ** j * delta:
            j += 1
            if j > max_backtrack:
                raise RuntimeError("Armijo search found no step")
        t = g1 ** j
        res.steps.append(t)
        res.curv.append(float(np.sum(d * (H @ d))))
        x = x - t * d
        g = grad(x)
        d = sla.cho_solve(P, g)
        dnew = float(np.sum(d * g))
        if dnew >= g3 * delta and 2 * m <= m_max:
            m, r = 2 * m, r + 1
            P = factor(m, r)
            d = sla.cho_solve(P, g)
            dnew = float(np.sum(d * g))
        delta = dnew
        k += 1
        res.delta.append(delta)
        res.ms.append(m)
    res.m, res.iterations, res.doublings, res.x = m, k, r, x
    return res


def adaptive_for_problem(A, B, kind: str, m0: int, s: int, seed: int, lam: float, bf16_entries: bool = False,
                         **kw) -> AdaptiveResult:
    """Algorithm 4 on a data matrix A (n x d, dense FP64 or scipy CSR) and right-hand side(s) B."""
    B = B[:, None] if B.ndim == 1 else B
    Ahat, c, _ = tall_form(A, B)
    if hasattr(Ahat, "tocsr"):
        Ahat = Ahat.tocsr()
    return adaptive_sketch_dim(Ahat, c, lam, m0, sketcher_for(kind, Ahat, s, seed, bf16_entries), **kw)
