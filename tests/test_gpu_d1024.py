"""Parity at the dimension of the dense FP32 benchmark workload (D = 1024), through the C ABI.

The small workloads stop at D <= 600; this one has the structure of the 65536 x 1024 SRHT
workload (Haar factors, singular values 1/k) at n = 8192, so that the float-float recursion on
the tensor cores runs with several 128-row tiles, items split over the contraction, per-column
kernels on full 8-CTA clusters (and the smaller clusters the autotuner tries), and the
two-product steps once at most six intervals are left (term counts falling from 45 to 14,
jmax = 16).  x(lambda) and every kept basis term are compared with the oracle element by
element; the oracle keeps the same terms (the truncation does not change them), and its full
expansion differs from the truncated one by at most 0.29^16 relative.
"""
import numpy as np
import pytest

from oracle import ihsbin as ob
from synthetic import make_problem
from tests.harness import gpu_problem, oracle_A, rel_err_max

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(lib):
    from paper_2210_12212_gb300 import ihsbin as ihs
    yield ihs.Context(0)


@pytest.mark.parametrize("K", [1, 3])
def test_d1024_recursion_matches_oracle(ctx, K):
    from paper_2210_12212_gb300 import ihsbin as ihs
    prob = make_problem("c2_small", n=8192, d=1024, m=2048, T=40, K=K)
    L = ob.num_intervals(prob.lambda_min, prob.lambda_max)
    rho = 1024 / 2048
    r1 = np.full(L, (1 + np.sqrt(rho)) ** 2)
    r2 = np.full(L, (1 - np.sqrt(rho)) ** 2)
    kk = np.linspace(45, 14, L).round().astype(np.int32)
    jmax = 16
    gp = gpu_problem(ihs, ctx, prob)
    gp.sketch(prob.sketch, prob.m, prob.s, prob.sketch_seed)
    for rep in range(2):  # the second build runs on the geometry the autotuner settled on
        gp.build_basis(prob.lambda_min, prob.lambda_max, L=L, k=kk, rho1=r1, rho2=r2, jmax=jmax, compute="f32x2")
        Xg = gp.eval_path(prob.lambdas)
        terms = [gp.basis(l, prob.d) for l in range(L)]
        plan = ob.make_plan(prob.lambda_min, prob.lambda_max, r1, r2, kk, L=L)
        if rep == 0:
            ref = ob.ihs_bin_path(oracle_A(prob), prob.B, prob.sketch, prob.m, prob.s, prob.sketch_seed, plan,
                                  prob.lambdas)
            Ahat, c, _ = ob.tall_form(oracle_A(prob), prob.B)
            G = Ahat.T @ Ahat
            cut = [ob.basis(lambda V: G @ V, ob.precond(ref.GS, plan.lam0[l]), c, plan.tau[l], int(kk[l]), jmax=jmax)
                   for l in range(L)]
        assert rel_err_max(Xg, ref.X) <= 1e-6
        for l in range(L):
            Ug, Uo = terms[l], cut[l]  # both (j, D, K)
            assert Ug.shape == Uo.shape and Ug.shape[0] == min(int(kk[l]), jmax)
            assert np.max(np.abs(Ug - Uo)) <= 1e-8 * np.max(np.abs(Uo)), l
    gp.close()
