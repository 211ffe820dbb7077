"""IHS-BIN in plain FP64: interval plan, preconditioner, basis, path, and direct checks.

Notation follows the paper: A (n x d), b / B (n x K), ridge problem (eq. 1)
x*(lam) = (A^T A + lam I)^-1 A^T b (Section 2.1), sketch S, preconditioner
P_S = (A^T S^T S A + lam0 I)^-1 (Section 3, after eq. (equ:ihs)).

Readings of the paper taken here (each is listed with its reason in the
design notes of the repository):

* IHS update (eq. equ:ihs): the gradient is A^T(Ax - b) + lam x (the printed
  A^T(Ax - b + lam x) is dimensionally inconsistent; the second line of the
  same equation fixes M = I - tau P_S (A^T A + lam I)).
* Proposition 1's initial condition u_00 = +P_S A^T b; Algorithm 2 prints
  -P_S A^T b, which with Algorithm 3's composition returns -x.
* The basis is built once per lambda interval, not inside the lambda loop of
  Algorithm 3 / 6 (its cost statement O(Tdk) for evaluation needs that).
* Interval split (Section 4.2): L = floor(2 ln(lmax/lmin)) (natural log,
  at least 1), lambda^(l) = lmin beta^(l/L), lam0_l = sqrt(lambda^(l) lambda^(l+1));
  a lambda belongs to the half-open interval [lambda^(l), lambda^(l+1)), the
  last interval is closed.
* Step size (Theorem 4): the proof gives alpha / lam0 = 2 (lmin/rho1 + lmax/rho2)^-1,
  i.e. tau = 2 lam0 / (lo/rho1 + hi/rho2) on the interval [lo, hi]; the printed
  closed form 2 sqrt(1/(rho1 rho2)) / (sqrt(kt) + 1/sqrt(kt)) disagrees with it.
* Re-centred, re-scaled expansion.  Writing M(lam) = I - tau P (A^T A + lam I)
  = B0 - theta Q with B0 = I - tau P (A^T A + lam0 I), Q = lam0 P and
  theta = tau (lam - lam0) / lam0, Proposition 1's induction goes through
  unchanged with (B, P, tau lam) replaced by (B0, Q, theta):
      u_{i+1,0} = B0 u_{i,0},  u_{i+1,j} = B0 u_{i,j} - Q u_{i,j-1},
      u_{i+1,i+1} = -Q u_{i,i},  u_00 = P A^T b,
      x_k(lam) = tau sum_j theta^j utilde_j,  utilde_j = sum_{i>=j} u_{i,j}.
  It is the same polynomial in lam as the printed form (which expands in
  powers of tau lam around 0 and loses all accuracy in FP64 for large k), with
  every term O(1) because ||Q|| <= 1 and |theta| <= tau (sqrt(beta^(1/L)) - 1).
  ``basis_literal`` keeps the printed form for small-k cross-checks.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable, List, Optional, Sequence

import numpy as np
import scipy.linalg as sla


# --------------------------------------------------------------------------- plan
@dataclass
class Plan:
    lambda_min: float
    lambda_max: float
    L: int
    edges: np.ndarray      # L+1
    lam0: np.ndarray       # L
    tau: np.ndarray        # L
    k: np.ndarray          # L (int)


def num_intervals(lmin: float, lmax: float) -> int:
    """Section 6.1: L = floor(2 log(lmax/lmin)), natural log, at least one interval."""
    return max(1, int(math.floor(2.0 * math.log(lmax / lmin))))


def interval_edges(lmin: float, lmax: float, L: int) -> np.ndarray:
    """Section 4.2: lambda^(l) = lmin * beta^(l/L), l = 0..L (endpoints exact)."""
    beta = lmax / lmin
    e = np.array([lmin * beta ** (l / L) for l in range(L + 1)])
    e[0], e[-1] = lmin, lmax
    return e


def rho_gaussian(rho: float):
    """Theorem (Gaussian sketch, Section 3.1) with ||D||_2 = 1 and eta -> 0:
    rho1 = (1 + sqrt(rho))^2, rho2 = (1 - sqrt(rho))^2, rho = d_e / m."""
    r = math.sqrt(rho)
    return (1.0 + r) ** 2, (1.0 - r) ** 2


def center(lo: float, hi: float, sigma_d2: float = 0.0) -> float:
    """lam0 of the interval [lo, hi]: sqrt(lo hi) (Section 4.2); with a known sigma_d^2 (the smallest
    eigenvalue of A^T A; the remark after Theorem 4) sqrt((hi + s)(lo + s)) - s."""
    return math.sqrt((hi + sigma_d2) * (lo + sigma_d2)) - sigma_d2


def step_size(lo: float, hi: float, rho1: float, rho2: float, sigma_d2: float = 0.0) -> float:
    """Theorem 4 (proof): alpha = 2 lam0 / (lo/rho1 + hi/rho2) with lam0 = sqrt(lo hi); with sigma_d^2
    (the proof's equation for alpha / (lam0 + sigma_d^2)): 2 (lam0 + s) / ((lo + s)/rho1 + (hi + s)/rho2)."""
    lam0 = center(lo, hi, sigma_d2)
    return 2.0 * (lam0 + sigma_d2) / ((lo + sigma_d2) / rho1 + (hi + sigma_d2) / rho2)


def make_plan(lmin: float, lmax: float, rho1: Sequence[float], rho2: Sequence[float],
              k: Sequence[int], L: int = 0, sigma_d2: float = 0.0) -> Plan:
    if L <= 0:
        L = num_intervals(lmin, lmax)
    edges = interval_edges(lmin, lmax, L)
    lam0 = np.array([center(edges[l], edges[l + 1], sigma_d2) for l in range(L)])
    r1 = np.broadcast_to(np.asarray(rho1, dtype=float), (L,))
    r2 = np.broadcast_to(np.asarray(rho2, dtype=float), (L,))
    tau = np.array([step_size(edges[l], edges[l + 1], r1[l], r2[l], sigma_d2) for l in range(L)])
    kk = np.broadcast_to(np.asarray(k, dtype=np.int64), (L,)).copy()
    return Plan(lmin, lmax, L, edges, lam0, tau, kk)


def theorem4_k(rho1: float, rho2: float, lo: float, hi: float, eps: float, sigma_d2: float = 0.0) -> int:
    """Theorem 4: the error contracts by (kt-1)/(kt+1) per step, kt = rho1 hi / (rho2 lo) (with sigma_d^2:
    rho1 (hi + s) / (rho2 (lo + s))); the smallest k with ((kt-1)/(kt+1))^k <= eps (capped at 20000)."""
    kt = rho1 * (hi + sigma_d2) / (rho2 * (lo + sigma_d2))
    rate = (kt - 1.0) / (kt + 1.0)
    k = math.ceil(math.log(eps) / math.log(rate)) if rate > 0 else 1
    return int(min(max(k, 1), 20000))


def auto_plan(GS: np.ndarray, m: int, lmin: float, lmax: float, eps: float = 1e-7, L: int = 0,
              rho_cap: float = 0.95, sigma_d2: float = 0.0) -> Plan:
    """Parameters from the sketch alone: rho_l = min(d_e/m, rho_cap) with the effective dimension of
    Section 4.2 estimated from the sketched Hessian, d_e = tr(G_S (G_S + lam0 I)^-1)
    = D - lam0 tr((G_S + lam0 I)^-1) (||D||_2 taken as 1); rho1/rho2 by the Gaussian-sketch theorem;
    tau by Theorem 4 (proof form); k by Theorem 4's rate for relative error eps."""
    if L <= 0:
        L = num_intervals(lmin, lmax)
    edges = interval_edges(lmin, lmax, L)
    lam0 = np.array([center(edges[l], edges[l + 1], sigma_d2) for l in range(L)])
    D = GS.shape[0]
    r1, r2, ks = [], [], []
    for l in range(L):
        Pinv = np.linalg.inv(GS + lam0[l] * np.eye(D))
        de = max(1.0, D - lam0[l] * np.trace(Pinv))
        rho = min(de / m, rho_cap)
        a, b = rho_gaussian(rho)
        r1.append(a)
        r2.append(b)
        ks.append(theorem4_k(a, b, edges[l], edges[l + 1], eps, sigma_d2))
    return make_plan(lmin, lmax, r1, r2, ks, L=L, sigma_d2=sigma_d2)


def interval_of(lam: float, plan: Plan) -> int:
    """Half-open [lambda^(l), lambda^(l+1)), last interval closed."""
    l = int(np.searchsorted(plan.edges, lam, side="right")) - 1
    return min(max(l, 0), plan.L - 1)


# ------------------------------------------------------------------- operators
def gram_operator(Ahat) -> Callable[[np.ndarray], np.ndarray]:
    """v -> A^T A v with G = A^T A formed once (FP64)."""
    G = np.asarray((Ahat.T @ Ahat).todense()) if hasattr(Ahat, "todense") else Ahat.T @ Ahat
    return lambda V: G @ V


def path_losses(A, B, A_test, B_test, X, lambdas):
    """The training and test losses of Section 6.1 along a path X (T x d x K):
    L_train(lam) = 1/2 ||A x - B||_F^2 + lam/2 ||x||_F^2,  L_test(lam) = 1/2 ||A_test x - B_test||_F^2."""
    B = B[:, None] if B.ndim == 1 else B
    train, test = np.empty(len(lambdas)), np.empty(len(lambdas))
    for t, lam in enumerate(lambdas):
        x = X[t]
        r = A @ x - B
        train[t] = 0.5 * float(np.sum(r * r)) + 0.5 * lam * float(np.sum(x * x))
        if A_test is not None:
            rt = A_test @ x - B_test
            test[t] = 0.5 * float(np.sum(rt * rt))
    return train, test


def gram_extended(Ahat) -> np.ndarray:
    """G = A^T A (the Hessian of the least-squares term, Section 2) with every sum
    accumulated in numpy's extended precision (longdouble: a 64-bit significand on
    x86-64, 113 bits on AArch64) and rounded once to FP64.  For data stored in
    FP32/BF16 every product is exact there, so the result is the exact Gram up to
    the final rounding and the extended accumulation; it checks Gram kernels whose
    error is below that of an FP64 GEMM."""
    A = np.asarray(Ahat.todense() if hasattr(Ahat, "todense") else Ahat, dtype=np.longdouble)
    return (A.T @ A).astype(np.float64)


def gram_entries_extended(Ahat, rows, cols) -> np.ndarray:
    """Entries G[rows[q], cols[q]] of A^T A, accumulated as in gram_extended."""
    A = np.asarray(Ahat, dtype=np.longdouble)
    return (A[:, rows] * A[:, cols]).sum(axis=0).astype(np.float64)


def aspace_operator(Ahat) -> Callable[[np.ndarray], np.ndarray]:
    """v -> A^T (A v), the two products of Algorithm 2 line 'tau A^T A u_j'."""
    return lambda V: Ahat.T @ (Ahat @ V)


@dataclass
class Precond:
    """P = (G_S + lam0 I)^-1 through its Cholesky factor (textbook, FP64)."""
    chol: np.ndarray
    lam0: float

    def solve(self, V):
        return sla.cho_solve((self.chol, True), V)


def precond(GS: np.ndarray, lam0: float) -> Precond:
    D = GS.shape[0]
    return Precond(np.linalg.cholesky(GS + lam0 * np.eye(D)), lam0)


def precond_svd_apply(SA: np.ndarray, lam0: float, V: np.ndarray) -> np.ndarray:
    """P_S v from the SVD of SA (Section 3, equations after Proposition 1): both m<d and m>=d forms."""
    m, D = SA.shape
    _, sig, V1 = np.linalg.svd(SA, full_matrices=False)     # SA = U1 diag(sig) V1, rows of V1 orthonormal
    V = np.asarray(V, dtype=float)
    if m < D:
        return V / lam0 + V1.T @ (((1.0 / (sig ** 2 + lam0)) - 1.0 / lam0)[:, None] * (V1 @ V)) \
            if V.ndim == 2 else V / lam0 + V1.T @ ((1.0 / (sig ** 2 + lam0) - 1.0 / lam0) * (V1 @ V))
    w = 1.0 / (sig ** 2 + lam0)
    return V1.T @ (w[:, None] * (V1 @ V)) if V.ndim == 2 else V1.T @ (w * (V1 @ V))


# ----------------------------------------------------------------------- basis
def basis(AtA: Callable, P: Precond, c: np.ndarray, tau: float, k: int, jmax: int = 0) -> np.ndarray:
    """Algorithm 2 (matrix form: Algorithm 5) in the re-centred, re-scaled form.

    Returns utilde with shape (k, D, K) (jmax > 0: only the terms j < min(k, jmax), shape
    (min(k, jmax), D, K)).  The in-place descending-j order of Algorithm 2 is kept: u_i is
    formed from the old u_{i-1}, then u_j for j = i-1..1 from the old u_j and old u_{j-1},
    then u_0; the products A^T A u_j of one outer step all use the values from before that
    step.  u_j is updated from u_j and u_{j-1} only, so the terms j < jmax do not depend on
    the higher ones and truncating at jmax leaves them unchanged.
    """
    lam0 = P.lam0
    c = np.atleast_2d(c.T).T if c.ndim == 1 else c
    D, K = c.shape
    J = k if jmax <= 0 else min(k, jmax)
    u: List[Optional[np.ndarray]] = [None] * J
    ut = np.zeros((J, D, K))
    u[0] = P.solve(c)                                   # u_00 = P A^T b
    ut[0] += u[0]
    for i in range(1, k):
        n_old = min(i, J)
        Y = AtA(np.concatenate(u[:n_old], axis=1)).reshape(D, n_old, K)   # A^T A u_j, j < i (old values)
        if i < J:
            u[i] = -lam0 * P.solve(u[i - 1])            # u_{i,i} = -Q u_{i-1,i-1}
        for j in range(n_old - 1, 0, -1):
            u[j] = u[j] - P.solve(tau * (Y[:, j] + lam0 * u[j]) + lam0 * u[j - 1])
        u[0] = u[0] - P.solve(tau * (Y[:, 0] + lam0 * u[0]))
        for j in range(min(i + 1, J)):
            ut[j] += u[j]
    return ut


def basis_partial_sums(AtA: Callable, P: Precond, c: np.ndarray, tau: float, k: int, jmax: int = 0,
                       solve: Optional[Callable] = None) -> np.ndarray:
    """The recursion of `basis` carried as its partial sums v_{i,j} = sum_{i' <= i} u_{i',j}.

    Summing the re-centred recursion u_{i+1,j} = B0 u_{i,j} - Q u_{i,j-1} (B0 = I - tau P H0,
    H0 = A^T A + lam0 I, Q = lam0 P) over the steps 0..i gives, with u_00 = P c,
        v_{i+1,j} = v_{i,j} + P r_{i,j},
        r_{i,j} = [j = 0] c - tau H0 v_{i,j} - lam0 v_{i,j-1},
    i.e. the fixed-preconditioner IHS update (Section 3, eq. equ:ihs) x <- x + tau P (A^T b -
    (A^T A + lam I) x) taken coefficient by coefficient in theta.  v_{k-1,j} = utilde_j, so the
    result equals `basis` in exact arithmetic (same shape, same truncation at jmax: r_j reads
    v_j and v_{j-1} only).  `solve` replaces P.solve (tests apply a perturbed preconditioner).
    """
    lam0 = P.lam0
    solve = solve or P.solve
    c = np.atleast_2d(c.T).T if c.ndim == 1 else c
    D, K = c.shape
    J = k if jmax <= 0 else min(k, jmax)
    v = np.zeros((J, D, K))
    v[0] = solve(c)                                     # v_00 = u_00 = P A^T b
    for i in range(1, k):
        live = min(i, J)                                # v_j != 0 for j < i before the step
        Y = AtA(np.concatenate(list(v[:live]), axis=1)).reshape(D, live, K)
        new = v.copy()
        for j in range(min(i + 1, J)):
            r = -lam0 * v[j - 1] if j > 0 else c.astype(float).copy()
            if j < live:
                r = r - tau * (Y[:, j] + lam0 * v[j])
            new[j] = v[j] + solve(r)
        v = new
    return v


def evaluate(ut: np.ndarray, tau: float, lam0: float, lam: float) -> np.ndarray:
    """x_k(lam) = tau * sum_j theta^j utilde_j, theta = tau (lam - lam0) / lam0."""
    theta = tau * (lam - lam0) / lam0
    coef = tau
    x = np.zeros(ut.shape[1:])
    for j in range(ut.shape[0]):
        x += coef * ut[j]
        coef *= theta
    return x


def basis_literal(AtA: Callable, Psolve: Callable, c: np.ndarray, tau: float, k: int) -> np.ndarray:
    """Proposition 1 exactly as printed (powers of tau*lam around 0), for small k only.

    u_{i+1,0} = (I - tau P A^T A) u_{i,0}, u_{i+1,j} = (I - tau P A^T A) u_{i,j} - P u_{i,j-1},
    u_{i+1,i+1} = -P u_{i,i}, u_00 = P A^T b;  x_k = tau sum_j (tau lam)^j utilde_j.
    """
    c = c[:, None] if c.ndim == 1 else c
    D, K = c.shape
    rows = [[Psolve(c)]]
    for i in range(k - 1):
        prev = rows[-1]
        Y = [AtA(v) for v in prev]
        new = [prev[0] - tau * Psolve(Y[0])]
        for j in range(1, i + 1):
            new.append(prev[j] - tau * Psolve(Y[j]) - Psolve(prev[j - 1]))
        new.append(-Psolve(prev[i]))
        rows.append(new)
    ut = np.zeros((k, D, K))
    for i, row in enumerate(rows):
        for j, v in enumerate(row):
            ut[j] += v
    return ut


def evaluate_literal(ut: np.ndarray, tau: float, lam: float) -> np.ndarray:
    return tau * sum((tau * lam) ** j * ut[j] for j in range(ut.shape[0]))


# ------------------------------------------------------------------ direct checks
def direct_ihs(AtA: Callable, P: Precond, c: np.ndarray, tau: float, lam: float, k: int):
    """k steps of fixed-preconditioner IHS from x0 = 0 (eq. equ:ihs, gradient A^T(Ax-b) + lam x)."""
    x = np.zeros_like(c, dtype=float)
    for _ in range(k):
        x = x - tau * P.solve(AtA(x) - c + lam * x)
    return x


def exact_ridge(Ahat_dense: np.ndarray, B: np.ndarray, lam: float) -> np.ndarray:
    """x*(lam) = (A^T A + lam I)^-1 A^T B by a textbook Cholesky solve (Section 2.1)."""
    G = Ahat_dense.T @ Ahat_dense
    return sla.cho_solve(sla.cho_factor(G + lam * np.eye(G.shape[0]), lower=True),
                         Ahat_dense.T @ B)


def svd_path(A: np.ndarray, B: np.ndarray, lams: Sequence[float]) -> np.ndarray:
    """Section 2.1: x*(lam) = V (Sigma^2 + lam I)^-1 Sigma U^T b, for every lam."""
    U, sig, Vt = np.linalg.svd(A, full_matrices=False)
    UtB = U.T @ B
    return np.stack([Vt.T @ ((sig / (sig ** 2 + lam))[:, None] * UtB) for lam in lams])


# -------------------------------------------------------------------- pipeline
@dataclass
class PathResult:
    plan: Plan
    SA: np.ndarray
    GS: np.ndarray
    c: np.ndarray
    bases: List[np.ndarray] = field(default_factory=list)   # per interval (k_l, D, K)
    X: Optional[np.ndarray] = None                         # (T, d, K)
    Z: Optional[np.ndarray] = None                         # dual path (T, n, K) if under-determined
    dual: bool = False


def tall_form(A, B):
    """Section 5.2: for n < d the dual problem min_z 1/2||A^T z||^2 + lam/2 ||z||^2 - b^T z is solved,
    whose data matrix is A_hat = A^T (d x n) and whose right-hand side enters as c = b; x = A^T z."""
    n, d = A.shape
    if n >= d:
        c = A.T @ B
        return A, c, False
    return A.T, B.copy(), True


def ihs_bin_path(A, B: np.ndarray, sketch_kind: str, m: int, s: int, seed: int, plan: Plan,
                 lambdas: Sequence[float], product: str = "gram", bf16_sketch: bool = False,
                 keep_bases: bool = True) -> PathResult:
    """Algorithm 3 (Algorithm 6 for K > 1) with the readings above.

    A: dense (n x d) FP64 array or scipy CSR.  B: (n x K).
    product: "gram" forms A_hat^T A_hat once (FP64); "aspace" applies A_hat^T (A_hat v).
    """
    from . import sketch as sk
    B = B[:, None] if B.ndim == 1 else B
    Ahat, c, dual = tall_form(A, B)
    if hasattr(Ahat, "tocsr"):
        Ahat = Ahat.tocsr()
    SA = sk.apply(sketch_kind, Ahat, m, s, seed, bf16_entries=bf16_sketch)
    GS = SA.T @ SA
    AtA = gram_operator(Ahat) if product == "gram" else aspace_operator(Ahat)
    res = PathResult(plan, SA, GS, c, dual=dual)
    for l in range(plan.L):
        P = precond(GS, plan.lam0[l])
        res.bases.append(basis(AtA, P, c, plan.tau[l], int(plan.k[l])))
    T = len(lambdas)
    D = c.shape[0]
    Zt = np.zeros((T, D, c.shape[1]))
    for t, lam in enumerate(lambdas):
        l = interval_of(lam, plan)
        Zt[t] = evaluate(res.bases[l], plan.tau[l], plan.lam0[l], lam)
    if dual:
        res.Z = Zt
        res.X = np.stack([Ahat @ Zt[t] for t in range(T)])
    else:
        res.X = Zt
    if not keep_bases:
        res.bases = []
    return res


def direct_path(A, B: np.ndarray, GS: np.ndarray, plan: Plan, lambdas: Sequence[float]):
    """Ground truth for parity without the polynomial: per lambda, k_l steps of IHS in Gram space."""
    B = B[:, None] if B.ndim == 1 else B
    Ahat, c, dual = tall_form(A, B)
    AtA = gram_operator(Ahat)
    out = []
    cache = {}
    for lam in lambdas:
        l = interval_of(lam, plan)
        if l not in cache:
            cache[l] = precond(GS, plan.lam0[l])
        z = direct_ihs(AtA, cache[l], c, plan.tau[l], lam, int(plan.k[l]))
        out.append(Ahat @ z if dual else z)
    return np.stack(out)
