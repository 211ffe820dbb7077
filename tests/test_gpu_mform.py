"""The recursion's two-product form (GPU), part of the increment form (form="increment").

Once the basis is truncated to jmax columns (jmax K a multiple of 16) and at most six
intervals are still running, every step forms [M_q U, P_l U] with M_q = P_l (G + lam0_l I) in
one tensor-core launch and updates u_{i+1,j} = u_{i,j} - tau M_q u_{i,j} - lam0 P_l u_{i,j-1}:
the same polynomial as the four-launch step R = tau (G u_j + lam0 u_j) + lam0 u_{j-1},
u_j <- u_j - P_l R (Proposition 1, re-centred).  The per-interval k below leave a few long
intervals running after the truncation, so the form takes over part-way through the recursion.
Checked against the CUDA-core float-float recursion with the same truncation (which keeps the
four-launch form), against the oracle's full basis terms, and against the oracle's path.
"""
import numpy as np
import pytest

from oracle import ihsbin as ob
from tests.harness import default_params, gpu_problem, oracle_A, rel_err_max, small

pytestmark = pytest.mark.gpu

JMAX = 16


@pytest.fixture(scope="module")
def ctx(lib):
    from paper_2210_12212_gb300 import ihsbin as ihs
    return ihs.Context(0)


def _k_profile(L, long_k, short_k, n_long):
    """n_long intervals with long_k steps, the rest with short_k (so few remain after short_k)."""
    k = np.full(L, short_k, dtype=np.int32)
    k[:n_long] = long_k
    k[1] = long_k - 7  # unequal lengths: the running set shrinks inside the two-product steps
    return k


def _run(ctx, prob, loop, kk, r1, r2, L, basis=False):
    from paper_2210_12212_gb300 import ihsbin as ihs
    gp = gpu_problem(ihs, ctx, prob)
    gp.sketch(prob.sketch, prob.m, prob.s, prob.sketch_seed)
    gp.build_basis(prob.lambda_min, prob.lambda_max, L=L, k=kk, rho1=r1, rho2=r2, jmax=JMAX, compute="f32x2",
                   loop=loop, form="increment")
    X = gp.eval_path(prob.lambdas)
    terms = [gp.basis(l, min(prob.n, prob.d)) for l in range(L)] if basis else None
    gp.close()
    return X, terms


CASES = [
    ("c2_small", {}, 60, 25),
    ("c4_small", {}, 50, 20),        # K = 5 right-hand sides
    ("c3_small", {}, 45, 22),        # CSR
    ("ar1u_small", {}, 40, 20),      # under-determined: the dual, D = n = 400 (the last cluster CTA owns no rows)
    ("c1_small", dict(n=30, d=70, m=50), 40, 20),  # dual with D = 30: one k-block, a cluster of one CTA
]


@pytest.mark.parametrize("name,over,long_k,short_k", CASES, ids=[c[0] + ("_dual" if c[1] else "") for c in CASES])
def test_two_product_form_matches_four_launch_form_and_oracle(ctx, name, over, long_k, short_k):
    prob = small(name, **over)
    L = ob.num_intervals(prob.lambda_min, prob.lambda_max)
    r1, r2, _ = default_params(prob, L, 1)
    kk = _k_profile(L, long_k, short_k, min(5, L - 1))
    Xs, terms = _run(ctx, prob, "slices", kk, r1, r2, L, basis=True)
    Xf, terms_f = _run(ctx, prob, "fma", kk, r1, r2, L, basis=True)
    # same truncation, same polynomial: the tensor-core two-product form against CUDA-core products
    assert rel_err_max(Xs, Xf) <= 1e-10
    for Ug, Uf in zip(terms, terms_f):
        assert np.max(np.abs(Ug - Uf)) <= 1e-9 * np.max(np.abs(Uf))
    plan = ob.make_plan(prob.lambda_min, prob.lambda_max, r1, r2, kk, L=L)
    ref = ob.ihs_bin_path(oracle_A(prob), prob.B, prob.sketch, prob.m, prob.s, prob.sketch_seed, plan,
                          prob.lambdas)
    # the basis terms j < jmax do not depend on the truncated ones; float-float carries about 47 bits,
    # less what the conditioning of G_S + lam0 I takes (ar1u_small: AR(1) rows, m below D)
    for l, Ug in enumerate(terms):
        Uo = ref.bases[l][:Ug.shape[0]]
        assert Ug.shape == Uo.shape
        assert np.max(np.abs(Ug - Uo)) <= 1e-9 * np.max(np.abs(Uo))
    # the omitted terms weigh at most about 0.29^16 of the leading one
    assert rel_err_max(Xs, ref.X) <= 1e-7
