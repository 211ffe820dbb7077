"""The residual form of the tensor-core recursion (GPU).

The fused tensor-core recursion can carry the basis as the partial sums v_{i,j} of Proposition 1's
terms and apply P_l to the residual r_j = [j = 0] c - tau (G + lam0 I) v_j - lam0 v_{j-1};
G v keeps the float-float class (26 slice pairs), P_l r only the pairs s + t <= precond_weight:
an error in applying P_l is removed by the later steps (pinned on the CPU by
tests/test_oracle_partial_sums.py), down to about k eps_w kappa times the plan's convergence
level.  The cases therefore run converged plans (rho from the sketch, k_l from Theorem 4 at eps = 1e-9,
the basis truncated at 16 terms).  Checked:
x(lambda) and the basis terms against the oracle (Algorithm 2 in FP64) and against the increment
form of the same library, for every precond_weight down to one (three pairs); the form and
weight the build reports; AUTO's choice (the residual form only when its weight rule drops
pairs; unconverged plans keep the increment form); the argument checks.
"""
import numpy as np
import pytest

from oracle import ihsbin as ob
from tests.harness import default_params, gpu_problem, oracle_A, rel_err_max, small

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(lib):
    from paper_2210_12212_gb300 import ihsbin as ihs
    return ihs.Context(0)


JMAX = 16


def _run(ctx, prob, form, pw=0, basis=False, k=None):
    """k None: a converged plan (rho from the sketch, k_l from Theorem 4 at eps = 1e-9); else k
    steps everywhere with the default rho.  The basis is truncated at JMAX terms."""
    from paper_2210_12212_gb300 import ihsbin as ihs
    L = ob.num_intervals(prob.lambda_min, prob.lambda_max)
    gp = gpu_problem(ihs, ctx, prob)
    gp.sketch(prob.sketch, prob.m, prob.s, prob.sketch_seed)
    if k is None:
        kw = dict(k=None, k_default=0, eps=1e-9, auto_rho=True)
    else:
        r1, r2, kk = default_params(prob, L, k)
        kw = dict(k=kk, rho1=r1, rho2=r2)
    gp.build_basis(prob.lambda_min, prob.lambda_max, L=L, jmax=JMAX, compute="f32x2", loop="slices", form=form,
                   precond_weight=pw, **kw)
    X = gp.eval_path(prob.lambdas)
    ran = gp.recursion_form()
    got = gp.plan()
    terms = [gp.basis(l, min(prob.n, prob.d)) for l in range(L)] if basis else None
    gp.close()
    plan = ob.Plan(prob.lambda_min, prob.lambda_max, L, got["edges"], got["lam0"], got["tau"], got["k"])
    return X, ran, terms, plan


def _oracle(prob, plan):
    """x(lambda) and the terms of Algorithm 2 in FP64 with the same plan and truncation."""
    from oracle import sketch as osk
    Ahat, c, dual = ob.tall_form(oracle_A(prob), prob.B)
    SA = osk.apply(prob.sketch, Ahat, prob.m, prob.s, prob.sketch_seed)
    GS = SA.T @ SA
    AtA = ob.gram_operator(Ahat)
    bases = [ob.basis(AtA, ob.precond(GS, plan.lam0[l]), c, plan.tau[l], int(plan.k[l]), jmax=JMAX)
             for l in range(plan.L)]
    Z = []
    for lam in prob.lambdas:
        l = ob.interval_of(lam, plan)
        Z.append(ob.evaluate(bases[l], plan.tau[l], plan.lam0[l], lam))
    Z = np.stack(Z)
    X = np.stack([Ahat @ z for z in Z]) if dual else Z
    return X, bases


_REF = {}
CASES = [("c2_small", {}), ("c4_small", {}), ("c3_small", {}), ("c1_small", {}), ("ar1u_small", {}),
         ("c1_small", dict(n=30, d=70, m=50))]


@pytest.mark.parametrize("name,over", CASES, ids=[c[0] + ("_dual" if c[1] else "") for c in CASES])
@pytest.mark.parametrize("pw", [1, 2, 3, 0])
def test_residual_form_matches_oracle_and_increment_form(ctx, name, over, pw):
    prob = small(name, **over)
    Xr, ran, _, plan = _run(ctx, prob, "residual", pw)
    assert ran[0] == "residual"
    assert ran[1] == pw if pw else 2 <= ran[1] <= 6
    key = (name, tuple(sorted(over.items())))
    if key not in _REF:  # the increment form and the oracle, once per case (the plan is the same)
        Xi, ran_i, _, plan_i = _run(ctx, prob, "increment")
        assert ran_i == ("increment", 6)
        assert np.array_equal(plan_i.k, plan.k)
        _REF[key] = (Xi, _oracle(prob, plan)[0])
    Xi, Xo = _REF[key]
    assert rel_err_max(Xi, Xo) <= 1e-10
    # one pair weight (three pairs, eps_w = 2^-16) stays inside the BF16 tolerance; from two on,
    # the partial sums end in the float-float class of the increment form
    tol = 1e-5 if pw == 1 else 1e-9
    assert rel_err_max(Xr, Xo) <= tol
    assert rel_err_max(Xr, Xi) <= tol


@pytest.mark.parametrize("pw,tol", [(2, 1e-8), (3, 1e-9)])
def test_residual_form_basis_terms(ctx, pw, tol):
    """The terms themselves (the highest, least converged ones carry the largest error): within
    about k eps_w kappa of the plan's convergence level, 1e-8 of the largest term with two pair
    weights and 1e-9 with three."""
    prob = small("c4_small")
    _, _, terms, plan = _run(ctx, prob, "residual", pw, basis=True)
    _, bases = _oracle(prob, plan)
    for l, (Ug, Uo) in enumerate(zip(terms, bases)):
        assert Ug.shape == Uo.shape
        assert np.max(np.abs(Ug - Uo)) <= tol * np.max(np.abs(Uo)), l


def test_auto_form_choice(ctx):
    prob = small("c2_small")
    # a converged plan: AUTO's rule drops pairs, so the residual form runs
    _, ran, _, _ = _run(ctx, prob, "auto")
    assert ran[0] == "residual" and 2 <= ran[1] <= 5
    # the same data with 12 steps everywhere (Theorem 4's bound leaves k rate^(k-1) near 11):
    # the rule keeps more pairs
    _, ran12, _, _ = _run(ctx, prob, "auto", k=12)
    assert ran12[1] >= ran[1]
    # kappa near 1e6 and the same unconverged plan: no weight below 6 passes, the increment form runs
    _, ran, _, _ = _run(ctx, small("c3_small"), "auto", k=12)
    assert ran == ("increment", 6)


def test_form_default_and_fma_loop(ctx):
    from paper_2210_12212_gb300 import ihsbin as ihs
    prob = small("c2_small")
    gp = gpu_problem(ihs, ctx, prob)
    gp.sketch(prob.sketch, prob.m, prob.s, prob.sketch_seed)
    with pytest.raises(ihs.IhsbinError) as e:
        gp.recursion_form()                       # no basis yet
    assert e.value.status == ihs.ERR_STATE
    gp.build_basis(prob.lambda_min, prob.lambda_max, L=2, k_default=10, compute="f32x2", form="increment")
    assert gp.recursion_form() == ("increment", 6)
    gp.build_basis(prob.lambda_min, prob.lambda_max, L=2, k_default=10, compute="f32x2", form="residual")
    assert gp.recursion_form()[0] == "residual"
    gp.build_basis(prob.lambda_min, prob.lambda_max, L=2, k_default=10, compute="f32x2", loop="fma")
    assert gp.recursion_form() == ("increment", 6)
    gp.build_basis(prob.lambda_min, prob.lambda_max, L=2, k_default=10, compute="f64", form="residual")
    assert gp.recursion_form() == ("increment", 6)  # CUDA-core products: Algorithm 2's increments
    for bad in (-1, 7):
        with pytest.raises(ihs.IhsbinError) as e:
            gp.build_basis(prob.lambda_min, prob.lambda_max, L=2, k_default=10, compute="f32x2", precond_weight=bad)
        assert e.value.status == ihs.ERR_INVALID_ARG
    gp.close()
