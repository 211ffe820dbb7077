"""The Gaussian sketch with BF16 entries of BF16 data on the tensor cores, against the oracle.

* Entries (Section 3, Gaussian sketch; BF16 rounding FP64 -> FP32 -> BF16, ties to even): the
  device draws in FP32 and redraws in FP64 only the entries whose FP32 value lies near a BF16
  rounding midpoint, so every BF16 entry must equal the oracle's bit for bit.
* S A_hat: every product of two BF16 numbers is exact; the tensor cores accumulate in FP32 over
  one k-split (at most N products per entry here) and the splits are added in FP64.  With one
  rounding of at most 2^-23 of the running |sum| per MMA of K = 16 products, the error of an
  entry is at most (N / 16 + 2) 2^-23 sum_k |S_ik A_kj|; the test asserts that bound and a
  typical (median) error far below it.
* x(lambda) through the whole path: the BF16 precision form's tolerance, 1e-5, against the oracle
  that uses the exact S A_hat (the sketch only sets the preconditioner).
"""
import numpy as np
import pytest

from oracle import ihsbin as ob
from oracle import sketch as osk
from synthetic import make_problem
from synthetic.configs import bf16_bits_to_f32
from tests.harness import default_params, gpu_problem, oracle_A, rel_err_max

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(lib):
    from paper_2210_12212_gb300 import ihsbin as ihs
    yield ihs.Context(0)


def _bf16_bits(x):
    return (osk._round_bf16(x).astype(np.float32).view(np.uint32) >> 16).astype(np.uint16)


def _problem(n, d, m, seed=0):
    # BF16 data with power-law columns and ragged sizes against the 128 x 256 x 64 tiles
    return make_problem("c4_small", seed=seed, n=n, d=d, m=m, K=2)


@pytest.mark.parametrize("window", [(0, 64, 0, 131072), (37, 5, 100001, 3000)])
def test_entries_bit_exact(ctx, window):
    from paper_2210_12212_gb300 import ihsbin as ihs
    prob = _problem(131072 + 77, 8, 300)
    gp = gpu_problem(ihs, ctx, prob)
    gp.sketch("gaussian", prob.m, 1, 5, entries="bf16", apply="tensor")
    r0, nr, c0, nc = window
    got = gp.sketch_entries(r0, nr, c0, nc)
    Sref = osk.gaussian_entries(prob.m, prob.n, 5, rows=np.arange(r0, r0 + nr))[:, c0:c0 + nc]
    want = _bf16_bits(Sref)
    bad = int(np.count_nonzero(got != want))
    assert bad == 0, f"{bad} of {got.size} BF16 entries differ from the oracle's rounding"
    gp.close()


@pytest.mark.parametrize("shape", [(5000, 300, 300), (70000, 520, 136), (256, 256, 128)])
def test_sketch_matches_oracle(ctx, shape):
    from paper_2210_12212_gb300 import ihsbin as ihs
    n, d, m = shape
    prob = _problem(n, d, m, seed=3)
    gp = gpu_problem(ihs, ctx, prob)
    gp.sketch("gaussian", m, 1, 11, entries="bf16", apply="tensor")
    SA, GS = gp.sketch_matrices(m, d)
    A = oracle_A(prob)
    S = osk._round_bf16(osk.gaussian_entries(m, n, 11))
    SAo = S @ A
    absum = np.abs(S) @ np.abs(A)
    err = np.abs(SA - SAo)
    bound = (n / 16 + 2) * 2.0 ** -23 * absum
    assert np.all(err <= bound), float(np.max(err / bound))
    # typical accuracy: FP32 accumulation with cancellation, far inside the worst case
    assert float(np.median(err / absum)) <= 1e-6
    # the sketched Gram is the FP64-class Gram of the device's S A_hat
    np.testing.assert_allclose(GS, SA.T @ SA, rtol=0, atol=1e-12 * np.abs(GS).max())
    gp.close()


def test_tensor_and_fma_paths_agree(ctx):
    from paper_2210_12212_gb300 import ihsbin as ihs
    prob = _problem(9000, 260, 200, seed=4)
    out = {}
    for apply in ("tensor", "fma"):
        gp = gpu_problem(ihs, ctx, prob)
        gp.sketch("gaussian", prob.m, 1, 2, entries="bf16", apply=apply)
        out[apply] = gp.sketch_matrices(prob.m, prob.d)[0]
        gp.close()
    A = oracle_A(prob)
    S = osk._round_bf16(osk.gaussian_entries(prob.m, prob.n, 2))
    absum = np.abs(S) @ np.abs(A)
    assert np.all(np.abs(out["tensor"] - out["fma"]) <= (prob.n / 16 + 3) * 2.0 ** -23 * absum)


def test_tensor_needs_bf16_data_and_entries(ctx):
    from paper_2210_12212_gb300 import ihsbin as ihs
    prob = make_problem("c1_small")  # FP64 data
    gp = gpu_problem(ihs, ctx, prob)
    with pytest.raises(ihs.IhsbinError) as e:
        gp.sketch("gaussian", prob.m, 1, 0, entries="bf16", apply="tensor")
    assert e.value.status == 9  # IHSBIN_ERR_UNSUPPORTED
    gp.close()


@pytest.mark.parametrize("compute", ["f64", "f32x2"])
def test_path_with_tensor_sketch(ctx, compute):
    from paper_2210_12212_gb300 import ihsbin as ihs
    prob = make_problem("c4_small")
    gp = gpu_problem(ihs, ctx, prob)
    gp.sketch("gaussian", prob.m, 1, 21, entries="bf16", apply="tensor")
    L = ob.num_intervals(prob.lambda_min, prob.lambda_max)
    r1, r2, kk = default_params(prob, L, 16)
    gp.build_basis(prob.lambda_min, prob.lambda_max, L=L, k=kk, rho1=r1, rho2=r2, compute=compute)
    Xg = gp.eval_path(prob.lambdas)
    plan = ob.make_plan(prob.lambda_min, prob.lambda_max, r1, r2, kk, L=L)
    res = ob.ihs_bin_path(oracle_A(prob), prob.B, "gaussian", prob.m, 1, 21, plan, prob.lambdas, bf16_sketch=True)
    assert rel_err_max(Xg, res.X) <= 1e-5
    gp.close()
