"""The basis recursion's products on the tensor cores (exact slices of G / P_l and of each
step's columns) against the oracle and against the CUDA-core float-float products: dense,
CSR, several right-hand sides (wider column tiles), the A-space product mode, the dual, the
basis terms themselves, and the refusal outside the float-float compute mode."""
import numpy as np
import pytest

from oracle import ihsbin as ob
from tests.harness import default_params, gpu_problem, oracle_A, rel_err_max, small

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(lib):
    from paper_2210_12212_gb300 import ihsbin as ihs
    return ihs.Context(0)


def _run(ctx, prob, loop, k=30, product="auto", basis=False):
    from paper_2210_12212_gb300 import ihsbin as ihs
    L = ob.num_intervals(prob.lambda_min, prob.lambda_max)
    r1, r2, kk = default_params(prob, L, k)
    gp = gpu_problem(ihs, ctx, prob)
    gp.sketch(prob.sketch, prob.m, prob.s, prob.sketch_seed)
    gp.build_basis(prob.lambda_min, prob.lambda_max, L=L, k=kk, rho1=r1, rho2=r2, compute="f32x2",
                   product=product, loop=loop)
    X = gp.eval_path(prob.lambdas)
    terms = [gp.basis(l, min(prob.n, prob.d)) for l in range(L)] if basis else None
    gp.close()
    plan = ob.make_plan(prob.lambda_min, prob.lambda_max, r1, r2, kk, L=L)
    return X, terms, plan


def _oracle(prob, plan):
    return ob.ihs_bin_path(oracle_A(prob), prob.B, prob.sketch, prob.m, prob.s, prob.sketch_seed, plan, prob.lambdas)


@pytest.mark.parametrize("name,k", [("c2_small", 40), ("c3_small", 30), ("c4_small", 30), ("c1_small", 30)])
def test_loop_slices_match_oracle_and_fma(ctx, name, k):
    prob = small(name)
    Xs, _, plan = _run(ctx, prob, "slices", k)
    Xf, _, _ = _run(ctx, prob, "fma", k)
    Xo = _oracle(prob, plan).X
    # both product kernels carry about 44-47 significant bits
    assert rel_err_max(Xs, Xo) <= 1e-10
    assert rel_err_max(Xs, Xf) <= 1e-10


def test_loop_slices_basis_terms(ctx):
    prob = small("c2_small")
    _, terms, plan = _run(ctx, prob, "slices", 25, basis=True)
    ref = _oracle(prob, plan)
    for l, Ug in enumerate(terms):
        Uo = ref.bases[l]
        assert Ug.shape == Uo.shape
        assert np.max(np.abs(Ug - Uo)) <= 1e-10 * np.max(np.abs(Uo))


def test_loop_slices_aspace_product(ctx):
    prob = small("c2_small")
    Xs, _, plan = _run(ctx, prob, "slices", 30, product="aspace")
    assert rel_err_max(Xs, _oracle(prob, plan).X) <= 1e-10


def test_loop_slices_dense_dual(ctx):
    import dataclasses
    base = small("c1_small")
    # an under-determined problem: the transpose of the over-determined data, its own right-hand side
    A = np.ascontiguousarray(base.A.T)
    rng = np.random.default_rng(3)
    B = rng.standard_normal((A.shape[0], 1))
    prob = dataclasses.replace(base, A=A, n=A.shape[0], d=A.shape[1], B=B, m=2 * A.shape[0])
    Xs, _, plan = _run(ctx, prob, "slices", 30)
    assert Xs.shape == (len(prob.lambdas), prob.d, 1)
    assert rel_err_max(Xs, _oracle(prob, plan).X) <= 1e-10


def test_loop_slices_refused_outside_f32x2(ctx):
    from paper_2210_12212_gb300 import ihsbin as ihs
    prob = small("c2_small")
    gp = gpu_problem(ihs, ctx, prob)
    gp.sketch(prob.sketch, prob.m, prob.s, prob.sketch_seed)
    with pytest.raises(ihs.IhsbinError) as e:
        gp.build_basis(prob.lambda_min, prob.lambda_max, L=1, k_default=2, compute="f64", loop="slices")
    assert e.value.status == ihs.ERR_UNSUPPORTED
    gp.close()


@pytest.mark.parametrize("name,k", [("c2_small", 40), ("c4_small", 30), ("c1_small", 30)])
def test_inverse_slices_match_fma(ctx, name, k):
    """P_l = W_l^T W_l on the tensor cores (triangular and symmetric blocks skipped) against the
    float-float CUDA-core product, through the whole path."""
    from paper_2210_12212_gb300 import ihsbin as ihs
    prob = small(name)
    L = ob.num_intervals(prob.lambda_min, prob.lambda_max)
    r1, r2, kk = default_params(prob, L, k)
    out = {}
    for factor in ("slices", "fma"):
        gp = gpu_problem(ihs, ctx, prob)
        gp.sketch(prob.sketch, prob.m, prob.s, prob.sketch_seed)
        gp.build_basis(prob.lambda_min, prob.lambda_max, L=L, k=kk, rho1=r1, rho2=r2, compute="f32x2", factor=factor)
        out[factor] = gp.eval_path(prob.lambdas)
        gp.close()
    plan = ob.make_plan(prob.lambda_min, prob.lambda_max, r1, r2, kk, L=L)
    assert rel_err_max(out["slices"], _oracle(prob, plan).X) <= 1e-10
    assert rel_err_max(out["slices"], out["fma"]) <= 1e-10


@pytest.mark.parametrize("name,k", [("c2_small", 40), ("c4_small", 30)])
@pytest.mark.parametrize("w", [4, 5])
def test_slice_weight_keeps_float32_class_accuracy(ctx, name, k, w):
    """Dropping the slice pairs with s + t > w (each weighs below 2^(-8(w+1)) of an entry's leading
    product) in the recursion and inverse products: the path stays within the FP32/TF32 tolerance."""
    from paper_2210_12212_gb300 import ihsbin as ihs
    prob = small(name)
    L = ob.num_intervals(prob.lambda_min, prob.lambda_max)
    r1, r2, kk = default_params(prob, L, k)
    gp = gpu_problem(ihs, ctx, prob)
    gp.sketch(prob.sketch, prob.m, prob.s, prob.sketch_seed)
    gp.build_basis(prob.lambda_min, prob.lambda_max, L=L, k=kk, rho1=r1, rho2=r2, compute="f32x2", slice_weight=w)
    Xw = gp.eval_path(prob.lambdas)
    gp.close()
    plan = ob.make_plan(prob.lambda_min, prob.lambda_max, r1, r2, kk, L=L)
    assert rel_err_max(Xw, _oracle(prob, plan).X) <= (1e-6 if w == 4 else 1e-8)
