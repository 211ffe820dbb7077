"""Pins of the oracle's adaptive sketch dimension (Section 5.1, Algorithm 4) against facts the
mathematics fixes: an exact sketch makes the direction the Newton step (one unit step solves the
quadratic), the line search's step is the closed form of the Armijo test on a quadratic, the
iterate converges to the ridge solution of the tall form (and, through the dual, to the primal
one), and the doubling rule's two limits (never / every step)."""
import numpy as np
import pytest

from oracle import adaptive as oa
from oracle.ihsbin import exact_ridge, tall_form


def _small_dense(n=400, d=30, K=1, seed=0):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, d)) * (1.0 + np.arange(d)) ** -1.0
    B = A @ rng.standard_normal((d, K)) + 0.05 * rng.standard_normal((n, K))
    return A, B


def test_exact_sketch_gives_one_newton_step():
    A, B = _small_dense()
    Ahat, c, _ = tall_form(A, B)
    res = oa.adaptive_sketch_dim(Ahat, c, 1e-2, 5, lambda m, r: Ahat, eps=1e-20, max_iter=5)
    # P = (A^T A + lam I)^-1 exactly: d_0 = -x*, f(x - t d) - f(x) = -(t - t^2/2) delta, t = 1 accepted
    assert res.steps[0] == 1.0
    assert res.doublings == 0
    assert res.delta[1] <= 1e-24 * res.delta[0]
    xs = exact_ridge(A, B, 1e-2)
    assert np.linalg.norm(res.x - xs) <= 1e-12 * np.linalg.norm(xs)


@pytest.mark.parametrize("kind,m0,s", [("gaussian", 4, 1), ("countsketch", 8, 2), ("srht", 4, 1)])
def test_armijo_step_is_the_quadratic_closed_form(kind, m0, s):
    """On a quadratic, f(x - t d) <= f(x) - g2 t delta  <=>  t q <= 2 (1 - g2) delta with
    q = d^T (A^T A + lam I) d, so the step is g1^j with j = max(0, ceil(log(2(1-g2) delta / q) / log g1))."""
    A, B = _small_dense(seed=1)
    g1, g2 = 0.5, 0.3
    res = oa.adaptive_for_problem(A, B, kind, m0, s, 7, 1e-3, g1=g1, g2=g2, eps=1e-12, max_iter=40)
    assert len(res.steps) == res.iterations >= 3
    for k, t in enumerate(res.steps):
        ratio = 2 * (1 - g2) * res.delta[k] / res.curv[k]
        j = max(0, int(np.ceil(np.log(ratio) / np.log(g1) - 1e-12)))
        assert t == g1 ** j


def test_converges_to_the_ridge_solution_and_decrement_shrinks():
    A, B = _small_dense(n=600, d=40, K=3, seed=2)
    lam = 1e-3
    res = oa.adaptive_for_problem(A, B, "gaussian", 2, 1, 11, lam, eps=1e-20, max_iter=200)
    xs = exact_ridge(A, B, lam)
    # delta = g^T P g >= lambda_min(P H) ||x - x*||_H^2: at delta <= 1e-20 delta_0 the iterate is within 1e-6
    assert np.linalg.norm(res.x - xs) <= 1e-6 * np.linalg.norm(xs)
    assert all(v >= 0 for v in res.delta)
    assert res.doublings >= 1 and res.m == 2 * 2 ** res.doublings
    assert res.ms == sorted(res.ms)


def test_dual_iterate_maps_to_the_primal_ridge_solution():
    rng = np.random.default_rng(4)
    A = rng.standard_normal((25, 300))
    B = rng.standard_normal((25, 1))
    lam = 0.5
    res = oa.adaptive_for_problem(A, B, "gaussian", 4, 1, 3, lam, eps=1e-22, max_iter=200)
    xs = exact_ridge(A, B, lam)              # primal (A^T A + lam I)^-1 A^T b
    assert np.linalg.norm(A.T @ res.x - xs) <= 1e-8 * np.linalg.norm(xs)


def test_doubling_limits():
    A, B = _small_dense(seed=5)
    never = oa.adaptive_for_problem(A, B, "gaussian", 4, 1, 1, 1e-2, g3=1e300, eps=1e-8, max_iter=30)
    assert never.doublings == 0 and set(never.ms) == {4}
    # g3 -> 0: every step doubles until 2m would pass m_max
    always = oa.adaptive_for_problem(A, B, "gaussian", 4, 1, 1, 1e-2, g3=1e-300, eps=1e-30, max_iter=8,
                                     m_max=64)
    assert always.ms[:5] == [4, 8, 16, 32, 64] and always.m == 64 and always.doublings == 4
