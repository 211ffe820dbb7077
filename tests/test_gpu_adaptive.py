"""Algorithm 4 (adaptive sketch dimension) on the device against the oracle: the sequence of sketch
dimensions and line-search steps bit for bit, the decrements and the final iterate to the compute
mode's accuracy, for every sketch family, dense and CSR data, K > 1, the dual, both compute modes;
then the path built on the sketch the procedure leaves behind."""
import numpy as np
import pytest

from oracle import adaptive as oa
from oracle import ihsbin as ob
from synthetic.configs import make_transposed
from tests.harness import default_params, gpu_problem, oracle_A, rel_err_max, small

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(lib):
    from paper_2210_12212_gb300 import ihsbin as ihs
    return ihs.Context(0)


def _oracle(prob, m0, lam, **kw):
    return oa.adaptive_for_problem(oracle_A(prob), prob.B, prob.sketch, m0, prob.s, prob.sketch_seed, lam,
                                   bf16_entries=prob.storage == "bf16", **kw)


def _compare(g, o, tol):
    assert list(g["ms"]) == o.ms, (list(g["ms"]), o.ms)
    assert list(g["steps"]) == o.steps
    assert g["m"] == o.m and g["iterations"] == o.iterations and g["doublings"] == o.doublings
    d_g, d_o = np.asarray(g["deltas"]), np.asarray(o.delta)
    # decrements: relative to the first one (they fall by many orders of magnitude)
    assert np.max(np.abs(d_g - d_o)) <= tol * d_o[0]
    assert np.linalg.norm(g["x"] - o.x) <= tol * np.linalg.norm(o.x)


CASES = [("c1_small", 8, "f32x2"), ("c1_small", 8, "f64"), ("c2_small", 16, "f32x2"), ("c3_small", 32, "f32x2"),
         ("c4_small", 16, "f32x2")]


@pytest.mark.parametrize("name,m0,compute", CASES)
def test_adaptive_matches_oracle(ctx, name, m0, compute):
    from paper_2210_12212_gb300 import ihsbin as ihs
    prob = small(name)
    lam = prob.lambda_min
    o = _oracle(prob, m0, lam, eps=1e-10)
    assert o.doublings >= 1
    gp = gpu_problem(ihs, ctx, prob)
    g = gp.adaptive_sketch(prob.sketch, m0, lam, s=prob.s, seed=prob.sketch_seed,
                           entries="bf16" if prob.storage == "bf16" else "f64", eps=1e-10, compute=compute,
                           want_x=True, apply="fma")  # the float-float sketch: decrements compared at 1e-9
    gp.close()
    _compare(g, o, 1e-9)


def test_adaptive_dual_csr(ctx):
    from paper_2210_12212_gb300 import ihsbin as ihs
    prob = make_transposed("c3_small")
    lam = prob.lambda_min
    o = _oracle(prob, 16, lam, eps=1e-10)
    gp = gpu_problem(ihs, ctx, prob)
    g = gp.adaptive_sketch(prob.sketch, 16, lam, s=prob.s, seed=prob.sketch_seed, eps=1e-10, want_x=True)
    gp.close()
    _compare(g, o, 1e-9)


def test_adaptive_parameters_and_limits(ctx):
    """Custom gammas, the m cap, the iteration cap."""
    from paper_2210_12212_gb300 import ihsbin as ihs
    prob = small("c2_small")
    lam = prob.lambda_min
    kw = dict(g1=0.3, g2=0.1, g3=0.8, eps=1e-12, max_iter=12, m_max=64)
    o = _oracle(prob, 8, lam, **kw)
    gp = gpu_problem(ihs, ctx, prob)
    g = gp.adaptive_sketch(prob.sketch, 8, lam, s=prob.s, seed=prob.sketch_seed, gamma1=0.3, gamma2=0.1,
                           gamma3=0.8, eps=1e-12, max_iter=12, m_max=64, want_x=True)
    gp.close()
    assert g["m"] <= 64 and g["iterations"] <= 12
    _compare(g, o, 1e-9)


def test_path_on_the_adapted_sketch(ctx):
    """build_basis after Algorithm 4 uses the sketch it left: the oracle path with m_final and the
    seed advanced by the number of doublings."""
    from paper_2210_12212_gb300 import ihsbin as ihs
    prob = small("c2_small")
    gp = gpu_problem(ihs, ctx, prob)
    g = gp.adaptive_sketch(prob.sketch, 16, prob.lambda_min, s=prob.s, seed=prob.sketch_seed, eps=1e-10)
    L = ob.num_intervals(prob.lambda_min, prob.lambda_max)
    pr = __import__("dataclasses").replace(prob, m=int(g["m"]), sketch_seed=prob.sketch_seed + g["doublings"])
    r1, r2, kk = default_params(pr, L, 40)
    gp.build_basis(prob.lambda_min, prob.lambda_max, L=L, k=kk, rho1=r1, rho2=r2, compute="f32x2")
    X = gp.eval_path(prob.lambdas)
    gp.close()
    plan = ob.make_plan(prob.lambda_min, prob.lambda_max, r1, r2, kk, L=L)
    Xo = ob.ihs_bin_path(oracle_A(pr), pr.B, pr.sketch, pr.m, pr.s, pr.sketch_seed, plan, prob.lambdas).X
    assert rel_err_max(X, Xo) <= 1e-10


def test_adaptive_argument_checks(ctx):
    from paper_2210_12212_gb300 import ihsbin as ihs
    prob = small("c2_small")
    gp = gpu_problem(ihs, ctx, prob)
    for kw in (dict(lam=0.0), dict(lam=-1.0), dict(gamma1=1.5), dict(gamma2=1.0)):
        lam = kw.pop("lam", prob.lambda_min)
        with pytest.raises(ihs.IhsbinError) as e:
            gp.adaptive_sketch(prob.sketch, 16, lam, **kw)
        assert e.value.status == ihs.ERR_INVALID_ARG
    gp.close()
