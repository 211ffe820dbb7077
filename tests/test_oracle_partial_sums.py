"""The partial-sums (residual) form of the basis recursion, on the CPU.

Summing Proposition 1's re-centred recursion over the steps gives the recursion of the partial
sums v_{i,j} = sum_{i' <= i} u_{i',j}: v_j <- v_j + P r_j with r_j = [j = 0] c - tau H0 v_j -
lam0 v_{j-1}, the IHS update of Section 3 (eq. equ:ihs) taken coefficient by coefficient.  Pins:

* in exact arithmetic it is Algorithm 2: `basis_partial_sums` equals `basis` to rounding, with
  and without the truncation at jmax, for one and several right-hand sides;
* the property the tensor-core recursion relies on: an error made in applying P is carried into
  the next residual and removed by the later steps.  With every application of P perturbed by
  relative noise eps, Algorithm 2's increments keep an error of order eps in x(lambda), while the
  partial sums end within a small multiple of eps times the convergence level of the plan.
"""
import numpy as np
import pytest

from oracle import ihsbin as ob


def _problem(K, seed=0, n=300, d=40, m=160):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, d)) * np.logspace(0, -1.5, d)
    b = rng.standard_normal((n, K))
    S = rng.standard_normal((m, n)) / np.sqrt(m)
    SA = S @ A
    rho = d / m
    r1, r2 = (1 + np.sqrt(rho)) ** 2, (1 - np.sqrt(rho)) ** 2
    return A.T @ A, A.T @ b, SA.T @ SA, r1, r2


@pytest.mark.parametrize("K,k,jmax", [(1, 25, 0), (3, 30, 8), (2, 12, 20)])
def test_partial_sums_equal_algorithm2(K, k, jmax):
    G, c, GS, r1, r2 = _problem(K)
    for lam0, tau in ((0.05, 0.6), (1.3, 0.9)):
        P = ob.precond(GS, lam0)
        u = ob.basis(lambda V: G @ V, P, c, tau, k, jmax=jmax)
        v = ob.basis_partial_sums(lambda V: G @ V, P, c, tau, k, jmax=jmax)
        assert u.shape == v.shape == (min(k, jmax) if jmax else k, G.shape[0], K)
        assert np.max(np.abs(u - v)) <= 1e-13 * np.max(np.abs(u))


class _NoisyP:
    """P applied with relative Gaussian noise eps on every entry of every product."""

    def __init__(self, P, eps, seed):
        self.P, self.lam0, self.eps = P, P.lam0, eps
        self.rng = np.random.default_rng(seed)

    def solve(self, V):
        X = self.P.solve(V)
        return X * (1.0 + self.eps * self.rng.standard_normal(X.shape))


@pytest.mark.parametrize("eps", [1e-6, 1e-4])
def test_partial_sums_correct_preconditioner_errors(eps):
    G, c, GS, r1, r2 = _problem(2)
    lmin, lmax = 0.02, 2.0
    L = ob.num_intervals(lmin, lmax)
    k = 60
    plan = ob.make_plan(lmin, lmax, np.full(L, r1), np.full(L, r2), np.full(L, k), L=L)
    for l in (0, L - 1):
        lam0, tau = plan.lam0[l], plan.tau[l]
        P = ob.precond(GS, lam0)
        lams = np.linspace(plan.edges[l], plan.edges[l + 1], 4)
        u = ob.basis(lambda V: G @ V, P, c, tau, k)
        xs = [ob.evaluate(u, tau, lam0, lm) for lm in lams]
        conv = max(np.linalg.norm(x - np.linalg.solve(G + lm * np.eye(G.shape[0]), c)) / np.linalg.norm(x)
                   for lm, x in zip(lams, xs))
        assert conv < 1e-4  # the plan converges (Theorem 4's rate at these rho)

        def err(ut):
            return max(np.linalg.norm(ob.evaluate(ut, tau, lam0, lm) - x) / np.linalg.norm(x) for lm, x in zip(lams, xs))

        e_inc = err(ob.basis(lambda V: G @ V, _NoisyP(P, eps, 1), c, tau, k))
        e_sum = err(ob.basis_partial_sums(lambda V: G @ V, P, c, tau, k, solve=_NoisyP(P, eps, 1).solve))
        assert e_inc >= 0.1 * eps          # the increments keep the preconditioner's error ...
        assert e_sum <= 10 * eps * conv    # ... the partial sums damp it to the convergence level
