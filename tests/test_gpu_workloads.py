"""The paper's own workload forms (Section 6.1) through the CUDA path against the oracle: AR(1)
correlated rows over- and under-determined with CountSketch (sketch dimension below D, as in the
paper's random experiments), and matrix-valued Gaussian-kernel ridge regression; the path and the
training / test losses, both compute modes, and the sketch-derived parameters."""
import numpy as np
import pytest

from oracle import ihsbin as ob
from oracle import sketch as osk
from synthetic import make_split
from tests.harness import default_params, gpu_problem, oracle_A, rel_err_max

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-9, "f32x2": 1e-6}


@pytest.fixture(scope="module")
def ctx(lib):
    from paper_2210_12212_gb300 import ihsbin as ihs
    return ihs.Context(0)


def _rel(a, b):
    return float(np.max(np.abs(a - b) / np.abs(b)))


@pytest.mark.parametrize("compute", ["f64", "f32x2"])
@pytest.mark.parametrize("name,n_test,k", [("ar1_small", 300, 30), ("ar1u_small", 0, 30), ("gkernel_small", 150, 25)])
def test_workload_path_and_losses(ctx, name, n_test, k, compute):
    from paper_2210_12212_gb300 import ihsbin as ihs
    if n_test:
        prob, A_test, B_test = make_split(name, n_test, seed=0)
    else:
        from synthetic import make_problem
        prob, A_test, B_test = make_problem(name), None, None
    assert prob.m < min(prob.n, prob.d) or name == "gkernel_small"
    L = ob.num_intervals(prob.lambda_min, prob.lambda_max)
    r1, r2, kk = default_params(prob, L, k)
    gp = gpu_problem(ihs, ctx, prob)
    gp.sketch(prob.sketch, prob.m, prob.s, prob.sketch_seed)
    gp.build_basis(prob.lambda_min, prob.lambda_max, L=L, k=kk, rho1=r1, rho2=r2, compute=compute)
    X = gp.eval_path(prob.lambdas)
    tr, te = gp.path_losses(prob.lambdas, A_test, B_test)
    gp.close()
    plan = ob.make_plan(prob.lambda_min, prob.lambda_max, r1, r2, kk, L=L)
    A = oracle_A(prob)
    ref = ob.ihs_bin_path(A, prob.B, prob.sketch, prob.m, prob.s, prob.sketch_seed, plan, prob.lambdas)
    assert X.shape == ref.X.shape
    assert rel_err_max(X, ref.X) <= TOL[compute]
    otr, ote = ob.path_losses(A, prob.B, None if A_test is None else A_test.astype(np.float64), B_test, X,
                              prob.lambdas)
    assert _rel(tr, otr) <= 1e-10
    if te is not None:
        assert _rel(te, ote) <= 1e-10


def test_ar1_sketch_derived_parameters(ctx):
    """rho from the sketch's effective dimension and k from Theorem 4 with m < D."""
    from paper_2210_12212_gb300 import ihsbin as ihs
    from synthetic import make_problem
    prob = make_problem("ar1_small")
    gp = gpu_problem(ihs, ctx, prob)
    gp.sketch(prob.sketch, prob.m, prob.s, prob.sketch_seed)
    gp.build_basis(prob.lambda_min, prob.lambda_max, k=None, k_default=0, eps=1e-6, auto_rho=True,
                   compute="f32x2")
    Xg = gp.eval_path(prob.lambdas)
    got = gp.plan()
    gp.close()
    A = oracle_A(prob)
    SA = osk.apply(prob.sketch, A, prob.m, prob.s, prob.sketch_seed)
    plan = ob.auto_plan(SA.T @ SA, prob.m, prob.lambda_min, prob.lambda_max, eps=1e-6)
    np.testing.assert_allclose(got["tau"], plan.tau, rtol=1e-9)
    assert np.abs(got["k"] - plan.k).max() <= 1
    plan.k = np.asarray(got["k"])
    res = ob.ihs_bin_path(A, prob.B, prob.sketch, prob.m, prob.s, prob.sketch_seed, plan, prob.lambdas)
    assert rel_err_max(Xg, res.X) <= TOL["f32x2"]
