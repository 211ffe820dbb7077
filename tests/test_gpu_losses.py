"""Section 6.1's training and test losses along the path, formed on the device from the
basis's images (A utilde_j, A_test utilde_j) without X: against the oracle's losses of the
same X (the loss arithmetic alone) and of the oracle's own path (the whole method), for
dense FP64 / FP32 / BF16 data, CSR data, several right-hand sides, both duals, the F64
compute mode, and the argument checks."""
import dataclasses

import numpy as np
import pytest

from oracle import ihsbin as ob
from synthetic import make_split
from synthetic.configs import bf16_bits_to_f32, make_transposed
from tests.harness import default_params, gpu_problem, oracle_A

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(lib):
    from paper_2210_12212_gb300 import ihsbin as ihs
    return ihs.Context(0)


def _dense_f64(A, storage):
    return bf16_bits_to_f32(A).astype(np.float64) if storage == "bf16" else np.asarray(A, dtype=np.float64)


def _rel(a, b):
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300)))


def _run(ctx, prob, A_test, B_test, lambdas, k=30, compute="f32x2", train=True, loop="auto"):
    from paper_2210_12212_gb300 import ihsbin as ihs
    L = ob.num_intervals(prob.lambda_min, prob.lambda_max)
    r1, r2, kk = default_params(prob, L, k)
    gp = gpu_problem(ihs, ctx, prob)
    gp.sketch(prob.sketch, prob.m, prob.s, prob.sketch_seed)
    gp.build_basis(prob.lambda_min, prob.lambda_max, L=L, k=kk, rho1=r1, rho2=r2, compute=compute, loop=loop)
    X = gp.eval_path(lambdas)
    tr, te = gp.path_losses(lambdas, A_test, B_test, test_dtype=prob.storage if A_test is not None else None,
                            train=train)
    gp.close()
    plan = ob.make_plan(prob.lambda_min, prob.lambda_max, r1, r2, kk, L=L)
    return X, tr, te, plan


def _check(prob, A_test, B_test, lambdas, X, tr, te, plan, tol_same=1e-10, tol_path=1e-8):
    A = oracle_A(prob)
    At = _dense_f64(A_test, prob.storage)
    # the same X through the oracle: checks the loss arithmetic itself
    otr, ote = ob.path_losses(A, prob.B, At, B_test, X, lambdas)
    assert _rel(tr, otr) <= tol_same
    assert _rel(te, ote) <= tol_same
    # the oracle's own path: the losses of the method end to end
    Xo = ob.ihs_bin_path(A, prob.B, prob.sketch, prob.m, prob.s, prob.sketch_seed, plan, lambdas).X
    ptr, pte = ob.path_losses(A, prob.B, At, B_test, Xo, lambdas)
    assert _rel(tr, ptr) <= tol_path
    assert _rel(te, pte) <= tol_path


@pytest.mark.parametrize("name,n_test,k", [("c2_small", 700, 40), ("c3_small", 900, 30), ("c4_small", 500, 30),
                                           ("c1_small", 77, 30)])
def test_losses_match_oracle(ctx, name, n_test, k):
    prob, A_test, B_test = make_split(name, n_test, seed=0)
    lam = prob.lambdas
    X, tr, te, plan = _run(ctx, prob, A_test, B_test, lam, k)
    assert tr.shape == te.shape == (len(lam),)
    _check(prob, A_test, B_test, lam, X, tr, te, plan)


def test_losses_tensor_core_images_match_cuda_core_images(ctx):
    """The exact-slice images (tensor cores) against the float-float GEMM of the CUDA cores."""
    prob, A_test, B_test = make_split("c2_small", 700, seed=0)
    lam = prob.lambdas
    _, tr_s, te_s, _ = _run(ctx, prob, A_test, B_test, lam, 40, loop="slices")
    _, tr_f, te_f, _ = _run(ctx, prob, A_test, B_test, lam, 40, loop="fma")
    assert _rel(tr_s, tr_f) <= 1e-10
    assert _rel(te_s, te_f) <= 1e-10


def test_losses_many_row_blocks(ctx):
    """More training and test rows than one block of the image (32768 rows): ragged last blocks, K=2."""
    prob, A_test, B_test = make_split("c4_small", 33001, seed=3, n=70001, d=40, K=2, storage="f32")
    lam = prob.lambdas
    X, tr, te, plan = _run(ctx, prob, A_test, B_test, lam, 30)
    _check(prob, A_test, B_test, lam, X, tr, te, plan)


def test_losses_f64_compute(ctx):
    prob, A_test, B_test = make_split("c1_small", 50, seed=1)
    lam = prob.lambdas
    X, tr, te, plan = _run(ctx, prob, A_test, B_test, lam, 30, compute="f64")
    _check(prob, A_test, B_test, lam, X, tr, te, plan)


def test_losses_unsorted_lambdas_with_edges_and_repeats(ctx):
    """lambdas in any order, both ends of the range, repeats, more than one chunk per interval."""
    prob, A_test, B_test = make_split("c2_small", 300, seed=2)
    rng = np.random.default_rng(5)
    lam = np.concatenate([[prob.lambda_min, prob.lambda_max], prob.lambdas, prob.lambdas[:7],
                          np.exp(rng.uniform(np.log(prob.lambda_min), np.log(prob.lambda_max), 45))])
    rng.shuffle(lam)
    X, tr, te, plan = _run(ctx, prob, A_test, B_test, lam, 40)
    _check(prob, A_test, B_test, lam, X, tr, te, plan)
    # the same lambda gives the same loss, bit for bit
    for t in range(len(lam)):
        same = np.nonzero(lam == lam[t])[0]
        assert np.all(tr[same] == tr[t]) and np.all(te[same] == te[t])


def test_losses_dense_dual(ctx):
    base = make_split("c1_small", 10, seed=0)[0]
    A = np.ascontiguousarray(base.A.T)  # 37 x 300: under-determined
    rng = np.random.default_rng(3)
    B = rng.standard_normal((A.shape[0], 1))
    prob = dataclasses.replace(base, A=A, n=A.shape[0], d=A.shape[1], B=B, m=2 * A.shape[0])
    A_test = rng.standard_normal((29, A.shape[1]))
    B_test = rng.standard_normal((29, 1))
    X, tr, te, plan = _run(ctx, prob, A_test, B_test, prob.lambdas, 30)
    _check(prob, A_test, B_test, prob.lambdas, X, tr, te, plan)


def test_losses_csr_dual(ctx):
    prob = make_transposed("c3_small")
    rng = np.random.default_rng(4)
    A_test = rng.standard_normal((64, prob.d)).astype(np.float32)
    B_test = rng.standard_normal((64, prob.K))
    X, tr, te, plan = _run(ctx, prob, A_test, B_test, prob.lambdas, 30)
    _check(prob, A_test, B_test, prob.lambdas, X, tr, te, plan)


def test_losses_train_only_and_test_only(ctx):
    prob, A_test, B_test = make_split("c4_small", 200, seed=0)
    lam = prob.lambdas
    X, tr, te, plan = _run(ctx, prob, None, None, lam, 30)
    assert te is None
    otr, _ = ob.path_losses(oracle_A(prob), prob.B, None, None, X, lam)
    assert _rel(tr, otr) <= 1e-10
    X2, tr2, te2, _ = _run(ctx, prob, A_test, B_test, lam, 30, train=False)
    assert tr2 is None
    _, ote = ob.path_losses(oracle_A(prob), prob.B, _dense_f64(A_test, prob.storage), B_test, X2, lam)
    assert _rel(te2, ote) <= 1e-10


def test_losses_argument_checks(ctx):
    from paper_2210_12212_gb300 import ihsbin as ihs
    prob, A_test, B_test = make_split("c2_small", 100, seed=0)
    gp = gpu_problem(ihs, ctx, prob)
    with pytest.raises(ihs.IhsbinError) as e:  # before build_basis
        gp.path_losses(prob.lambdas)
    assert e.value.status == ihs.ERR_STATE
    gp.sketch(prob.sketch, prob.m, prob.s, prob.sketch_seed)
    gp.build_basis(prob.lambda_min, prob.lambda_max, k_default=10, compute="f32x2")
    with pytest.raises(ihs.IhsbinError) as e:
        gp.path_losses([prob.lambda_max * 1.5])
    assert e.value.status == ihs.ERR_LAMBDA_RANGE
    with pytest.raises(ihs.IhsbinError) as e:  # A_test with the wrong column count
        gp.path_losses(prob.lambdas, np.ascontiguousarray(A_test[:, :-1]), B_test)
    assert e.value.status == ihs.ERR_INVALID_ARG
    gp.close()
