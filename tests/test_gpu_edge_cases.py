"""Edge cases of the CUDA path against the oracle: empty CSR rows, one column, several
right-hand sides on CSR data, a single lambda, and a degenerate range lambda_min = lambda_max."""
import dataclasses

import numpy as np
import pytest

from oracle import ihsbin as ob
from tests.harness import default_params, gpu_problem, oracle_A, rel_err_max, small

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(lib):
    from paper_2210_12212_gb300 import ihsbin as ihs
    return ihs.Context(0)


def _both(ctx, prob, compute="f64", k=20, lambdas=None, L=0):
    from paper_2210_12212_gb300 import ihsbin as ihs
    lams = prob.lambdas if lambdas is None else lambdas
    Lr = L if L > 0 else ob.num_intervals(prob.lambda_min, prob.lambda_max)
    r1, r2, kk = default_params(prob, Lr, k)
    gp = gpu_problem(ihs, ctx, prob)
    gp.sketch(prob.sketch, prob.m, prob.s, prob.sketch_seed)
    gp.build_basis(prob.lambda_min, prob.lambda_max, L=Lr, k=kk, rho1=r1, rho2=r2, compute=compute)
    Xg = gp.eval_path(lams)
    gp.close()
    plan = ob.make_plan(prob.lambda_min, prob.lambda_max, r1, r2, kk, L=Lr)
    Xo = ob.ihs_bin_path(oracle_A(prob), prob.B, prob.sketch, prob.m, prob.s, prob.sketch_seed, plan, lams).X
    return Xg, Xo


def _with_empty_rows(prob, every=7):
    """Drop the nonzeros of every `every`-th row of a CSR workload."""
    counts = np.diff(prob.row_ptr)
    keep_row = np.arange(prob.n) % every != 0
    keep = np.repeat(keep_row, counts)
    counts = np.where(keep_row, counts, 0)
    rp = np.zeros(prob.n + 1, dtype=np.int64)
    np.cumsum(counts, out=rp[1:])
    return dataclasses.replace(prob, row_ptr=rp, col_idx=prob.col_idx[keep], val=prob.val[keep])


@pytest.mark.parametrize("compute", ["f64", "f32x2"])
def test_csr_with_empty_rows(ctx, compute):
    prob = _with_empty_rows(small("c3_small"))
    assert (np.diff(prob.row_ptr) == 0).sum() > 0
    Xg, Xo = _both(ctx, prob, compute)
    assert rel_err_max(Xg, Xo) <= (1e-9 if compute == "f64" else 1e-6)


def test_single_column(ctx):
    prob = small("c1_small", d=1, m=8)
    Xg, Xo = _both(ctx, prob, "f64", k=8)
    assert Xg.shape == (len(prob.lambdas), 1, 1)
    assert rel_err_max(Xg, Xo) <= 1e-9


def test_csr_several_right_hand_sides(ctx):
    prob = small("c3_small", K=3)
    assert prob.B.shape[1] == 3
    Xg, Xo = _both(ctx, prob, "f32x2")
    assert rel_err_max(Xg, Xo) <= 1e-6


def test_single_lambda(ctx):
    prob = small("c2_small")
    lam = np.array([np.sqrt(prob.lambda_min * prob.lambda_max)])
    Xg, Xo = _both(ctx, prob, "f64", lambdas=lam)
    assert Xg.shape[0] == 1 and rel_err_max(Xg, Xo) <= 1e-9


def test_degenerate_range(ctx):
    prob = small("c2_small")
    lam = prob.lambda_min * 3.0
    prob = dataclasses.replace(prob, lambda_min=lam, lambda_max=lam, lambdas=np.array([lam]))
    Xg, Xo = _both(ctx, prob, "f64", k=30)
    assert rel_err_max(Xg, Xo) <= 1e-9
