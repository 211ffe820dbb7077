"""The Gram of A and A^T b started by ihsbin_sketch in the background (GPU).

For dense FP32/BF16 data with at least 32 right-hand sides, the sketch call starts the Gram of A
and A^T b (which do not depend on the sketch) on the problem's side stream; a float-float build
with the sliced Gram takes them, any other build waits for them and forms its own.  Per-launch
timing turns the background launch off, so a problem with timing on computes the same path with
the Gram inside the build: the two must agree bit for bit (the Gram's tiles are combined in a
fixed order whatever its launch geometry).  Also: a build in another mode after the sketch, two
sketches in a row, a sketch without a build before the problem is destroyed, and the oracle.
"""
import numpy as np
import pytest

from oracle import ihsbin as ob
from synthetic import make_problem
from tests.harness import default_params, gpu_problem, oracle_A, rel_err_max

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(lib):
    from paper_2210_12212_gb300 import ihsbin as ihs
    return ihs.Context(0)


def _prob():
    # BF16 data with 40 right-hand sides: the configuration the background Gram serves
    return make_problem("c4_small", seed=5, n=6000, d=200, m=400, K=40)


def _path(ctx, prob, timing, compute="f32x2", sketch_twice=False):
    from paper_2210_12212_gb300 import ihsbin as ihs
    L = ob.num_intervals(prob.lambda_min, prob.lambda_max)
    r1, r2, kk = default_params(prob, L, 25)
    gp = gpu_problem(ihs, ctx, prob)
    gp.set_timing(timing)
    gp.sketch(prob.sketch, prob.m, prob.s, prob.sketch_seed, entries="bf16")
    if sketch_twice:
        gp.sketch(prob.sketch, prob.m, prob.s, prob.sketch_seed, entries="bf16")
    gp.build_basis(prob.lambda_min, prob.lambda_max, L=L, k=kk, rho1=r1, rho2=r2, compute=compute)
    X = gp.eval_path(prob.lambdas)
    G = gp.gram()
    gp.close()
    return X, G, ob.make_plan(prob.lambda_min, prob.lambda_max, r1, r2, kk, L=L)


def test_background_gram_matches_build_gram_bit_for_bit(ctx):
    prob = _prob()
    Xb, Gb, plan = _path(ctx, prob, timing=False)
    Xt, Gt, _ = _path(ctx, prob, timing=True)
    assert np.array_equal(Gb, Gt)
    assert np.array_equal(Xb, Xt)
    ref = ob.ihs_bin_path(oracle_A(prob), prob.B, prob.sketch, prob.m, prob.s, prob.sketch_seed, plan,
                          prob.lambdas, bf16_sketch=True)
    assert rel_err_max(Xb, ref.X) <= 1e-5


def test_other_mode_and_repeated_sketch(ctx):
    prob = _prob()
    Xb, _, plan = _path(ctx, prob, timing=False)
    X2, _, _ = _path(ctx, prob, timing=False, sketch_twice=True)
    assert np.array_equal(Xb, X2)
    X64, _, _ = _path(ctx, prob, timing=False, compute="f64")   # the background Gram is not taken
    assert rel_err_max(X64, Xb) <= 1e-5


def test_sketch_without_build(ctx):
    from paper_2210_12212_gb300 import ihsbin as ihs
    prob = _prob()
    before = ctx.memory()
    gp = gpu_problem(ihs, ctx, prob)
    gp.sketch(prob.sketch, prob.m, prob.s, prob.sketch_seed, entries="bf16")
    gp.close()   # waits for the background Gram and frees it
    assert ctx.memory() == before


def test_many_right_hand_sides_fp32(ctx):
    """FP32 data with 40 right-hand sides (the background Gram, the fused right-hand side and the
    tiled path evaluation for K >= 16) against the oracle at the float-float tolerance."""
    from paper_2210_12212_gb300 import ihsbin as ihs
    prob = make_problem("c2_small", seed=2, K=40)
    L = ob.num_intervals(prob.lambda_min, prob.lambda_max)
    r1, r2, kk = default_params(prob, L, 30)
    gp = gpu_problem(ihs, ctx, prob)
    gp.sketch(prob.sketch, prob.m, prob.s, prob.sketch_seed)
    gp.build_basis(prob.lambda_min, prob.lambda_max, L=L, k=kk, rho1=r1, rho2=r2, compute="f32x2")
    X = gp.eval_path(prob.lambdas)
    gp.close()
    plan = ob.make_plan(prob.lambda_min, prob.lambda_max, r1, r2, kk, L=L)
    ref = ob.ihs_bin_path(oracle_A(prob), prob.B, prob.sketch, prob.m, prob.s, prob.sketch_seed, plan, prob.lambdas)
    assert X.shape == ref.X.shape
    assert rel_err_max(X, ref.X) <= 1e-9
