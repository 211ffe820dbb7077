"""GPU path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (max over lambda of the relative Frobenius error of x(lambda)):
FP64 compute 1e-9, float-float compute 1e-6; sketch indices and signs bit-exact.
"""
import math

import numpy as np
import pytest

from oracle import ihsbin as ob
from oracle import sketch as osk
from tests.harness import default_params, gpu_problem, oracle_A, rel_err_max, small

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-9, "f32x2": 1e-6}


@pytest.fixture(scope="module")
def ctx(lib):
    from paper_2210_12212_gb300 import ihsbin as ihs
    c = ihs.Context(0)
    yield c


def run_both(ctx, prob, compute, k=25, L=0, rho=None, jmax=0, product="auto", lambdas=None):
    from paper_2210_12212_gb300 import ihsbin as ihs
    lmin, lmax = prob.lambda_min, prob.lambda_max
    Lr = L if L > 0 else ob.num_intervals(lmin, lmax)
    r1, r2, kk = default_params(prob, Lr, k, rho)
    lams = prob.lambdas if lambdas is None else lambdas
    gp = gpu_problem(ihs, ctx, prob)
    gp.sketch(prob.sketch, prob.m, prob.s, prob.sketch_seed)
    gp.build_basis(lmin, lmax, L=Lr, k=kk, rho1=r1, rho2=r2, jmax=jmax, compute=compute, product=product)
    Xg = gp.eval_path(lams)
    plan = ob.make_plan(lmin, lmax, r1, r2, kk, L=Lr)
    res = ob.ihs_bin_path(oracle_A(prob), prob.B, prob.sketch, prob.m, prob.s, prob.sketch_seed, plan, lams)
    return gp, Xg, res, plan


@pytest.mark.parametrize("compute", ["f64", "f32x2"])
def test_c1_small_gaussian(ctx, compute):
    prob = small("c1_small")
    gp, Xg, res, plan = run_both(ctx, prob, compute, k=30)
    assert Xg.shape == res.X.shape
    assert rel_err_max(Xg, res.X) <= TOL[compute]
    gp.close()


@pytest.mark.parametrize("compute", ["f64", "f32x2"])
def test_c2_small_srht(ctx, compute):
    prob = small("c2_small")
    gp, Xg, res, plan = run_both(ctx, prob, compute, k=40)
    assert rel_err_max(Xg, res.X) <= TOL[compute]
    gp.close()


def test_plan_matches_oracle(ctx):
    prob = small("c2_small")
    gp, Xg, res, plan = run_both(ctx, prob, "f64", k=7)
    p = gp.plan()
    assert p["L"] == plan.L
    np.testing.assert_allclose(p["edges"], plan.edges, rtol=1e-15)
    np.testing.assert_allclose(p["lam0"], plan.lam0, rtol=1e-15)
    np.testing.assert_allclose(p["tau"], plan.tau, rtol=1e-14)
    gp.close()


def test_srht_draws_bit_exact(ctx):
    from paper_2210_12212_gb300 import ihsbin as ihs
    prob = small("c2_small")
    gp = gpu_problem(ihs, ctx, prob)
    gp.sketch("srht", prob.m, 1, 1234)
    Np = osk.next_pow2(prob.n)
    idx, sign, cnt = gp.sketch_export(Np)
    assert cnt == prob.m
    np.testing.assert_array_equal(idx[:cnt], osk.srht_rows(Np, prob.m, 1234))
    np.testing.assert_array_equal(sign[:Np].astype(float), osk.srht_signs(Np, 1234))
    SA, GS = gp.sketch_matrices(prob.m, prob.d)
    SAo = osk.apply_srht(oracle_A(prob), prob.m, 1234)
    np.testing.assert_allclose(SA, SAo, rtol=0, atol=1e-12 * np.abs(SAo).max())
    np.testing.assert_allclose(GS, SAo.T @ SAo, rtol=0, atol=1e-12 * np.abs(GS).max())
    gp.close()


def test_countsketch_draws_bit_exact(ctx):
    from paper_2210_12212_gb300 import ihsbin as ihs
    prob = small("c1_small")
    gp = gpu_problem(ihs, ctx, prob)
    gp.sketch("countsketch", 40, 4, 99)
    idx, sign, cnt = gp.sketch_export(prob.n * 4)
    rows, sg = osk.countsketch_map(prob.n, 40, 4, 99)
    assert cnt == prob.n * 4
    np.testing.assert_array_equal(idx[:cnt].reshape(prob.n, 4), rows)
    np.testing.assert_array_equal(sign[:cnt].reshape(prob.n, 4).astype(float), sg)
    SA, _ = gp.sketch_matrices(40, prob.d)
    SAo = osk.apply_countsketch(oracle_A(prob), 40, 4, 99)
    np.testing.assert_allclose(SA, SAo, rtol=0, atol=1e-12 * np.abs(SAo).max())
    gp.close()


def test_gaussian_sketch_values(ctx):
    from paper_2210_12212_gb300 import ihsbin as ihs
    prob = small("c1_small")
    gp = gpu_problem(ihs, ctx, prob)
    gp.sketch("gaussian", prob.m, 1, 5)
    SA, GS = gp.sketch_matrices(prob.m, prob.d)
    SAo = osk.apply_gaussian(oracle_A(prob), prob.m, 5)
    np.testing.assert_allclose(SA, SAo, rtol=0, atol=1e-12 * np.abs(SAo).max())
    gp.close()


@pytest.mark.parametrize("compute", ["f64", "f32x2"])
def test_basis_terms_match_oracle(ctx, compute):
    prob = small("c1_small")
    gp, Xg, res, plan = run_both(ctx, prob, compute, k=12, L=3)
    for l in range(plan.L):
        Ug = gp.basis(l, prob.d)
        Uo = res.bases[l]
        assert Ug.shape == Uo.shape
        scale = np.abs(Uo).max()
        np.testing.assert_allclose(Ug, Uo, rtol=0, atol=TOL[compute] * 10 * scale)
    gp.close()


@pytest.mark.parametrize("product", ["gram", "aspace"])
def test_product_modes_agree(ctx, product):
    prob = small("c1_small")
    gp, Xg, res, plan = run_both(ctx, prob, "f64", k=20, product=product)
    assert rel_err_max(Xg, res.X) <= 1e-9
    gp.close()


def test_underdetermined_dense_dual(ctx):
    prob = small("c1_small", n=30, d=70, m=50)
    gp, Xg, res, plan = run_both(ctx, prob, "f64", k=25)
    assert res.dual and Xg.shape == (len(prob.lambdas), 70, 1)
    assert rel_err_max(Xg, res.X) <= 1e-9
    gp.close()


@pytest.mark.parametrize("compute", ["f64", "f32x2"])
def test_matrix_valued_bf16(ctx, compute):
    prob = small("c4_small")
    gp, Xg, res, plan = run_both(ctx, prob, compute, k=18)
    assert Xg.shape == (len(prob.lambdas), prob.d, prob.K)
    assert rel_err_max(Xg, res.X) <= TOL[compute]
    gp.close()


def test_truncated_basis_matches_full(ctx):
    prob = small("c2_small")
    gp, Xg, res, plan = run_both(ctx, prob, "f64", k=60, jmax=30)
    assert rel_err_max(Xg, res.X) <= 1e-9
    gp.close()


def test_lambda_out_of_range_writes_nothing(ctx):
    from paper_2210_12212_gb300 import ihsbin as ihs
    prob = small("c1_small")
    gp = gpu_problem(ihs, ctx, prob)
    gp.sketch(prob.sketch, prob.m, 1, 0)
    gp.build_basis(prob.lambda_min, prob.lambda_max, k_default=3)
    out = np.full((2, prob.d, 1), 7.0)
    from paper_2210_12212_gb300.ihsbin import _check, _lib, _ptr, ERR_LAMBDA_RANGE
    lam = np.array([prob.lambda_min, prob.lambda_max * 1.5])
    st = _lib.ihsbin_eval_path(gp.h, _ptr(lam), 2, _ptr(out), 0, 0, None)
    assert st == ERR_LAMBDA_RANGE
    assert np.all(out == 7.0)
    gp.close()


def test_call_order_enforced(ctx):
    from paper_2210_12212_gb300 import ihsbin as ihs
    prob = small("c1_small")
    gp = gpu_problem(ihs, ctx, prob)
    with pytest.raises(ihs.IhsbinError) as ei:
        gp.build_basis(prob.lambda_min, prob.lambda_max, k_default=3)
    assert ei.value.status == ihs.ERR_STATE
    gp.close()


def csr_under(prob, seed=3):
    """Under-determined CSR variant: A_u = A^T of a CSR workload, fresh b_u."""
    t = prob.transpose()
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((t.n, 1))
    import dataclasses
    return dataclasses.replace(t, B=B, x_star=np.zeros((t.d, 1)))


@pytest.mark.parametrize("compute", ["f64", "f32x2"])
def test_c3_small_csr_sjlt(ctx, compute):
    prob = small("c3_small")
    gp, Xg, res, plan = run_both(ctx, prob, compute, k=30)
    assert rel_err_max(Xg, res.X) <= TOL[compute]
    gp.close()


@pytest.mark.parametrize("compute", ["f64", "f32x2"])
def test_c3_small_csr_underdetermined_dual(ctx, compute):
    prob = csr_under(small("c3_small"))
    assert prob.n < prob.d
    gp, Xg, res, plan = run_both(ctx, prob, compute, k=30)
    assert res.dual and Xg.shape == (len(prob.lambdas), prob.d, 1)
    assert rel_err_max(Xg, res.X) <= TOL[compute]
    gp.close()


def test_csr_countsketch_draws_bit_exact(ctx):
    from paper_2210_12212_gb300 import ihsbin as ihs
    prob = small("c3_small")
    gp = gpu_problem(ihs, ctx, prob)
    gp.sketch("countsketch", prob.m, prob.s, 77)
    idx, sign, cnt = gp.sketch_export(prob.n * prob.s)
    rows, sg = osk.countsketch_map(prob.n, prob.m, prob.s, 77)
    np.testing.assert_array_equal(idx[:cnt].reshape(prob.n, prob.s), rows)
    np.testing.assert_array_equal(sign[:cnt].reshape(prob.n, prob.s).astype(float), sg)
    SA, GS = gp.sketch_matrices(prob.m, prob.d)
    SAo = osk.apply_countsketch(oracle_A(prob), prob.m, prob.s, 77)
    np.testing.assert_allclose(SA, SAo, rtol=0, atol=1e-12 * np.abs(SAo).max())
    gp.close()


@pytest.mark.parametrize("compute", ["f64", "f32x2"])
def test_auto_parameters_match_oracle(ctx, compute):
    # rho from the sketch's effective dimension, k from Theorem 4: both sides derive them independently
    from paper_2210_12212_gb300 import ihsbin as ihs
    prob = small("c2_small")
    gp = gpu_problem(ihs, ctx, prob)
    gp.sketch(prob.sketch, prob.m, prob.s, prob.sketch_seed)
    gp.build_basis(prob.lambda_min, prob.lambda_max, k=None, k_default=0, eps=1e-6, auto_rho=True,
                   compute=compute, jmax=40)
    Xg = gp.eval_path(prob.lambdas)
    SA = osk.apply_srht(oracle_A(prob), prob.m, prob.sketch_seed)
    plan = ob.auto_plan(SA.T @ SA, prob.m, prob.lambda_min, prob.lambda_max, eps=1e-6)
    got = gp.plan()
    np.testing.assert_allclose(got["tau"], plan.tau, rtol=1e-9)
    assert np.abs(got["k"] - plan.k).max() <= 1
    res = ob.ihs_bin_path(oracle_A(prob), prob.B, prob.sketch, prob.m, prob.s, prob.sketch_seed, plan,
                          prob.lambdas)
    assert rel_err_max(Xg, res.X) <= TOL[compute]
    gp.close()


@pytest.mark.parametrize("compute", ["f64", "f32x2"])
def test_bf16_gaussian_sketch_entries(ctx, compute):
    # BF16 data with BF16 sketch entries on the CUDA cores: exact products, float-float accumulation of S A
    from paper_2210_12212_gb300 import ihsbin as ihs
    prob = small("c4_small")
    gp = gpu_problem(ihs, ctx, prob)
    gp.sketch("gaussian", prob.m, 1, 21, entries="bf16", apply="fma")
    SA, GS = gp.sketch_matrices(prob.m, prob.d)
    SAo = osk.apply_gaussian(oracle_A(prob), prob.m, 21, bf16_entries=True)
    np.testing.assert_allclose(SA, SAo, rtol=0, atol=1e-13 * np.abs(SAo).max())
    L = ob.num_intervals(prob.lambda_min, prob.lambda_max)
    r1, r2, kk = default_params(prob, L, 16)
    gp.build_basis(prob.lambda_min, prob.lambda_max, L=L, k=kk, rho1=r1, rho2=r2, compute=compute)
    Xg = gp.eval_path(prob.lambdas)
    plan = ob.make_plan(prob.lambda_min, prob.lambda_max, r1, r2, kk, L=L)
    res = ob.ihs_bin_path(oracle_A(prob), prob.B, "gaussian", prob.m, 1, 21, plan, prob.lambdas, bf16_sketch=True)
    assert rel_err_max(Xg, res.X) <= TOL[compute]
    gp.close()


@pytest.mark.parametrize("compute", ["f64", "f32x2"])
def test_known_sigma_d_rule(ctx, compute):
    """The remark after Theorem 4: interval centres and steps from a known smallest eigenvalue
    (A = U diag(1/k) V^T, so sigma_d^2 = 1/d^2), fixed and sketch-derived parameters."""
    from paper_2210_12212_gb300 import ihsbin as ihs
    prob = small("c2_small")
    s2 = 1.0 / prob.d ** 2
    L = ob.num_intervals(prob.lambda_min, prob.lambda_max)
    r1, r2, kk = default_params(prob, L, 40)
    gp = gpu_problem(ihs, ctx, prob)
    gp.sketch(prob.sketch, prob.m, prob.s, prob.sketch_seed)
    gp.build_basis(prob.lambda_min, prob.lambda_max, L=L, k=kk, rho1=r1, rho2=r2, compute=compute, sigma_d2=s2)
    Xg = gp.eval_path(prob.lambdas)
    got = gp.plan()
    plan = ob.make_plan(prob.lambda_min, prob.lambda_max, r1, r2, kk, L=L, sigma_d2=s2)
    np.testing.assert_allclose(got["lam0"], plan.lam0, rtol=1e-14)
    np.testing.assert_allclose(got["tau"], plan.tau, rtol=1e-14)
    # sqrt((hi+s)(lo+s)) - s lies between the geometric and arithmetic means of the edges (AM-GM)
    lo, hi = plan.edges[:-1], plan.edges[1:]
    assert np.all(got["lam0"] > np.sqrt(lo * hi)) and np.all(got["lam0"] < 0.5 * (lo + hi))
    res = ob.ihs_bin_path(oracle_A(prob), prob.B, prob.sketch, prob.m, prob.s, prob.sketch_seed, plan, prob.lambdas)
    assert rel_err_max(Xg, res.X) <= TOL[compute]
    # sketch-derived rho and Theorem 4's k with the refined rate
    gp.build_basis(prob.lambda_min, prob.lambda_max, k=None, k_default=0, eps=1e-6, auto_rho=True,
                   compute=compute, sigma_d2=s2)
    Xa = gp.eval_path(prob.lambdas)
    got = gp.plan()
    gp.close()
    SA = osk.apply_srht(oracle_A(prob), prob.m, prob.sketch_seed)
    ap = ob.auto_plan(SA.T @ SA, prob.m, prob.lambda_min, prob.lambda_max, eps=1e-6, sigma_d2=s2)
    np.testing.assert_allclose(got["tau"], ap.tau, rtol=1e-9)
    assert np.abs(got["k"] - ap.k).max() <= 1
    ap.k = np.asarray(got["k"])
    res = ob.ihs_bin_path(oracle_A(prob), prob.B, prob.sketch, prob.m, prob.s, prob.sketch_seed, ap, prob.lambdas)
    assert rel_err_max(Xa, res.X) <= TOL[compute]
