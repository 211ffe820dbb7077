"""Error paths and explicit parameters through the C ABI (GPU).

* a non-finite entry of A comes back as IHSBIN_ERR_NAN from the factor it reaches (no trap);
* an allocation that fails (made to fail on the host by the context's test hook) comes back as
  IHSBIN_ERR_OUT_OF_MEMORY; the failed build leaves the problem sketched without a basis, with
  its sketch untouched, and a build after the hook is lifted gives the same result as before;
* an explicit per-interval tau (Theorem 4's step chosen by the caller) is used as given and
  matches the oracle run with the same plan.
"""
import numpy as np
import pytest

from oracle import ihsbin as ob
from tests.harness import default_params, gpu_problem, oracle_A, rel_err_max, small

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(lib):
    from paper_2210_12212_gb300 import ihsbin as ihs
    yield ihs.Context(0)


@pytest.mark.parametrize("bad", [np.nan, np.inf])
@pytest.mark.parametrize("name", ["c2_small", "c1_small"])
def test_nonfinite_data_reports_nan(ctx, name, bad):
    import dataclasses
    from paper_2210_12212_gb300 import ihsbin as ihs
    prob = small(name)
    A = np.array(prob.A, copy=True)
    A[7, 3] = bad
    prob = dataclasses.replace(prob, A=A)
    gp = gpu_problem(ihs, ctx, prob)
    gp.sketch(prob.sketch, prob.m, prob.s, prob.sketch_seed)
    L = ob.num_intervals(prob.lambda_min, prob.lambda_max)
    r1, r2, kk = default_params(prob, L, 8)
    with pytest.raises(ihs.IhsbinError) as e:
        gp.build_basis(prob.lambda_min, prob.lambda_max, L=L, k=kk, rho1=r1, rho2=r2, compute="f32x2")
    assert e.value.status == ihs.ERR_NAN
    with pytest.raises(ihs.IhsbinError) as e:
        gp.eval_path(prob.lambdas)
    assert e.value.status == ihs.ERR_STATE
    gp.close()


@pytest.mark.parametrize("after", [0, 3, 12])
def test_allocation_failure_leaves_problem_sketched(ctx, after):
    from paper_2210_12212_gb300 import ihsbin as ihs
    prob = small("c2_small")
    L = ob.num_intervals(prob.lambda_min, prob.lambda_max)
    r1, r2, kk = default_params(prob, L, 20)
    gp = gpu_problem(ihs, ctx, prob)
    gp.sketch(prob.sketch, prob.m, prob.s, prob.sketch_seed)
    SA0, GS0 = gp.sketch_matrices(prob.m, prob.d)
    gp.build_basis(prob.lambda_min, prob.lambda_max, L=L, k=kk, rho1=r1, rho2=r2, compute="f32x2")
    X0 = gp.eval_path(prob.lambdas)
    ctx.fail_allocations(after)
    try:
        with pytest.raises(ihs.IhsbinError) as e:
            gp.build_basis(prob.lambda_min, prob.lambda_max, L=L, k=kk, rho1=r1, rho2=r2, compute="f32x2")
        assert e.value.status == ihs.ERR_OUT_OF_MEMORY
    finally:
        ctx.fail_allocations(-1)
    with pytest.raises(ihs.IhsbinError) as e:
        gp.eval_path(prob.lambdas)                     # the basis was discarded ...
    assert e.value.status == ihs.ERR_STATE
    SA1, GS1 = gp.sketch_matrices(prob.m, prob.d)      # ... the sketch was not
    assert np.array_equal(SA0, SA1) and np.array_equal(GS0, GS1)
    gp.build_basis(prob.lambda_min, prob.lambda_max, L=L, k=kk, rho1=r1, rho2=r2, compute="f32x2")
    assert np.array_equal(gp.eval_path(prob.lambdas), X0)
    gp.close()


def test_allocation_failure_in_sketch(ctx):
    from paper_2210_12212_gb300 import ihsbin as ihs
    prob = small("c1_small")
    gp = gpu_problem(ihs, ctx, prob)
    ctx.fail_allocations(1)
    try:
        with pytest.raises(ihs.IhsbinError) as e:
            gp.sketch(prob.sketch, prob.m, prob.s, prob.sketch_seed)
        assert e.value.status == ihs.ERR_OUT_OF_MEMORY
    finally:
        ctx.fail_allocations(-1)
    with pytest.raises(ihs.IhsbinError) as e:          # a failed sketch leaves the problem unsketched
        gp.build_basis(prob.lambda_min, prob.lambda_max, L=2, k_default=5)
    assert e.value.status == ihs.ERR_STATE
    gp.sketch(prob.sketch, prob.m, prob.s, prob.sketch_seed)
    gp.close()


@pytest.mark.parametrize("compute", ["f64", "f32x2"])
def test_explicit_tau(ctx, compute):
    from paper_2210_12212_gb300 import ihsbin as ihs
    prob = small("c1_small")
    L = ob.num_intervals(prob.lambda_min, prob.lambda_max)
    r1, r2, kk = default_params(prob, L, 30)
    rule = ob.make_plan(prob.lambda_min, prob.lambda_max, r1, r2, kk, L=L)
    tau = rule.tau * np.linspace(0.8, 1.0, L)          # smaller steps than Theorem 4's, per interval
    gp = gpu_problem(ihs, ctx, prob)
    gp.sketch(prob.sketch, prob.m, prob.s, prob.sketch_seed)
    gp.build_basis(prob.lambda_min, prob.lambda_max, L=L, k=kk, rho1=r1, rho2=r2, tau=tau, compute=compute)
    got = gp.plan()
    np.testing.assert_array_equal(got["tau"], tau)
    Xg = gp.eval_path(prob.lambdas)
    plan = ob.Plan(prob.lambda_min, prob.lambda_max, L, rule.edges, rule.lam0, tau, rule.k)
    res = ob.ihs_bin_path(oracle_A(prob), prob.B, prob.sketch, prob.m, prob.s, prob.sketch_seed, plan, prob.lambdas)
    assert rel_err_max(Xg, res.X) <= (1e-9 if compute == "f64" else 1e-6)
    with pytest.raises(ihs.IhsbinError) as e:
        bad = tau.copy()
        bad[2] = -1.0
        gp.build_basis(prob.lambda_min, prob.lambda_max, L=L, k=kk, rho1=r1, rho2=r2, tau=bad, compute=compute)
    assert e.value.status == ihs.ERR_INVALID_ARG
    gp.close()


@pytest.mark.parametrize("fault", ["column_out_of_range", "column_not_increasing", "row_ptr_decreasing",
                                   "row_ptr_end"])
def test_invalid_csr_structure_is_rejected(ctx, fault):
    """CSR structure is checked on the device before any kernel indexes with it (every read of the
    check stays inside the arrays' stated sizes), so bad input is INVALID_ARG, not a fault."""
    import dataclasses
    from paper_2210_12212_gb300 import ihsbin as ihs
    prob = small("c3_small")
    rp, ci = prob.row_ptr.copy(), prob.col_idx.copy()
    if fault == "column_out_of_range":
        ci[rp[7]] = prob.d                      # one past the last column
    elif fault == "column_not_increasing":
        ci[rp[3] + 1] = ci[rp[3]]               # a duplicate within row 3
    elif fault == "row_ptr_decreasing":
        rp[5] = rp[4] - 1
    else:
        rp[-1] = rp[-1] - 1                     # does not end at nnz
    bad = dataclasses.replace(prob, row_ptr=rp, col_idx=ci)
    before = ctx.memory()
    with pytest.raises(ihs.IhsbinError) as e:
        gpu_problem(ihs, ctx, bad)
    assert e.value.status == ihs.ERR_INVALID_ARG
    assert ctx.memory() == before
    gp = gpu_problem(ihs, ctx, prob)           # the valid structure still goes through
    gp.close()
