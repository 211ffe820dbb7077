"""TF32 data (FP32 storage, values rounded to TF32 to nearest with ties away from zero) through
the C ABI against the oracle, which rounds the same FP32 values by its own definition.

The Gram of the rounded data is compared entry by entry (a single value rounded differently
would move its entries far above the tolerance), and x(lambda) at the tolerance of the FP32/TF32
precision form (1e-6; 1e-9 in FP64 compute): dense with the SRHT, dense with the Gaussian sketch
(BF16 entries: exact BF16 x TF32 products), CSR with CountSketch, and the dense dual.
"""
import dataclasses

import numpy as np
import pytest

from oracle import ihsbin as ob
from tests.harness import default_params, gpu_problem, oracle_A, rel_err_max, small

pytestmark = pytest.mark.gpu
TOL = {"f64": 1e-9, "f32x2": 1e-6}


@pytest.fixture(scope="module")
def ctx(lib):
    from paper_2210_12212_gb300 import ihsbin as ihs
    yield ihs.Context(0)


def _tf32(name, **kw):
    return small(name, storage="tf32", **kw)


@pytest.mark.parametrize("compute", ["f64", "f32x2"])
@pytest.mark.parametrize("name,device", [("c2_small", False), ("c2_small", True), ("c3_small", False),
                                         ("c3_small", True)])
def test_tf32_path_matches_oracle(ctx, name, device, compute):
    from paper_2210_12212_gb300 import ihsbin as ihs
    prob = _tf32(name)
    L = ob.num_intervals(prob.lambda_min, prob.lambda_max)
    r1, r2, kk = default_params(prob, L, 30)
    gp = gpu_problem(ihs, ctx, prob, device_inputs=device)
    gp.sketch(prob.sketch, prob.m, prob.s, prob.sketch_seed)
    gp.build_basis(prob.lambda_min, prob.lambda_max, L=L, k=kk, rho1=r1, rho2=r2, compute=compute)
    Xg = gp.eval_path(prob.lambdas)
    A = oracle_A(prob)
    G = gp.gram()
    Ah = A if prob.n >= prob.d else A.T
    Go = np.asarray((Ah.T @ Ah).todense()) if hasattr(Ah, "todense") else Ah.T @ Ah
    np.testing.assert_allclose(G, Go, rtol=0, atol=1e-11 * np.abs(Go).max())
    plan = ob.make_plan(prob.lambda_min, prob.lambda_max, r1, r2, kk, L=L)
    res = ob.ihs_bin_path(A, prob.B, prob.sketch, prob.m, prob.s, prob.sketch_seed, plan, prob.lambdas)
    assert rel_err_max(Xg, res.X) <= TOL[compute]
    gp.close()


def test_tf32_gaussian_bf16_entries(ctx):
    from paper_2210_12212_gb300 import ihsbin as ihs
    from oracle import sketch as osk
    prob = _tf32("c2_small")
    gp = gpu_problem(ihs, ctx, prob)
    gp.sketch("gaussian", prob.m, 1, 3, entries="bf16")
    SA, _ = gp.sketch_matrices(prob.m, prob.d)
    SAo = osk.apply_gaussian(oracle_A(prob), prob.m, 3, bf16_entries=True)
    np.testing.assert_allclose(SA, SAo, rtol=0, atol=1e-12 * np.abs(SAo).max())
    gp.close()


def test_tf32_dense_dual(ctx):
    from paper_2210_12212_gb300 import ihsbin as ihs
    base = _tf32("c2_small")
    A = np.ascontiguousarray(base.A[:80].T)          # 96 x 80: under-determined
    rng = np.random.default_rng(3)
    prob = dataclasses.replace(base, n=A.shape[0], d=A.shape[1], A=A, B=rng.standard_normal((A.shape[0], 1)))
    L = ob.num_intervals(prob.lambda_min, prob.lambda_max)
    r1, r2, kk = default_params(prob, L, 30)
    gp = gpu_problem(ihs, ctx, prob)
    gp.sketch("srht", 64, 1, 5)
    gp.build_basis(prob.lambda_min, prob.lambda_max, L=L, k=kk, rho1=r1, rho2=r2, compute="f32x2")
    Xg = gp.eval_path(prob.lambdas)
    plan = ob.make_plan(prob.lambda_min, prob.lambda_max, r1, r2, kk, L=L)
    res = ob.ihs_bin_path(oracle_A(prob), prob.B, "srht", 64, 1, 5, plan, prob.lambdas)
    assert rel_err_max(Xg, res.X) <= 1e-6
    gp.close()
