"""The tensor-core Gram (dense FP32/BF16 data cut into exact integer BF16 slices, tcgen05
products, FP64 combination) against the oracle's extended-precision Gram: several 128-wide
tiles with ragged edges, several row splits, the dual, zero columns, entries spread over a
wide exponent range, and the path it feeds."""
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


def _gram(ctx, prob, compute="f64", gram="slices"):
    from paper_2210_12212_gb300 import ihsbin as ihs
    gp = gpu_problem(ihs, ctx, prob)
    gp.sketch(prob.sketch, prob.m, prob.s, prob.sketch_seed)
    gp.build_basis(prob.lambda_min, prob.lambda_max, L=1, k_default=2, compute=compute, gram=gram)
    G = gp.gram()
    gp.close()
    return G


def _scaled_err(G, Gref):
    d = np.sqrt(np.abs(np.diag(Gref)))
    den = np.maximum(np.outer(d, d), 1e-300)
    return float(np.max(np.abs(G - Gref) / den))


def _ahat(prob):
    A = oracle_A(prob)
    return A if prob.n >= prob.d else A.T


def _with_dense(prob, A32):
    """The workload with its dense FP32 matrix replaced (B kept; only the Gram is compared)."""
    return dataclasses.replace(prob, A=np.ascontiguousarray(A32, dtype=np.float32))


# Error bound of the sliced Gram for FP32 data, relative to sqrt(G_ii G_jj):
#  * six slices hold every entry to |delta_kj| <= 2^-48 2^e_j <= 2^-47 max_k |a_kj| <= 2^-47 sqrt(G_jj),
#    so by Cauchy-Schwarz the representation error is <= 2 sqrt(N) 2^-47;
#  * the dropped pairs (s + t >= 7) weigh <= 2^-52 max|a_ki| max|a_kj| per row, <= N 2^-52 in all;
#  * plus the final FP64 rounding.
def _slice_bound(N):
    return np.sqrt(N) * 2.0 ** -46 + N * 2.0 ** -52 + 4e-16


@pytest.mark.parametrize("name", ["c2_small", "c4_small"])
@pytest.mark.parametrize("compute", ["f64", "f32x2"])
def test_slices_gram_matches_extended(ctx, name, compute):
    prob = small(name)
    G = _gram(ctx, prob, compute)
    Gref = ob.gram_extended(_ahat(prob))
    # F64 compute keeps G in FP64; float-float keeps about 48 significant bits
    assert _scaled_err(G, Gref) <= (1e-15 if compute == "f64" else 1e-14)
    assert np.array_equal(G, G.T)


def test_fma_gram_still_matches(ctx):
    prob = small("c2_small")
    G = _gram(ctx, prob, "f64", gram="fma")
    assert _scaled_err(G, ob.gram_extended(_ahat(prob))) <= prob.n * 2.0 ** -52


@pytest.mark.parametrize("n,d", [(65, 1), (129, 128), (700, 130), (100, 260)])
def test_ragged_and_wide_exponent_range(ctx, n, d):
    # the generator makes over-determined matrices; the dual case (n < d) takes its shape's transpose
    base = small("c2_small", n=max(n, d), d=min(n, d), m=max(8, 2 * min(n, d)))
    rng = np.random.default_rng(n * 1000 + d)
    col_scale = np.exp2(rng.integers(-40, 41, size=d).astype(np.float64))
    entry_scale = np.exp2(rng.integers(-12, 1, size=(n, d)).astype(np.float64))
    A32 = (rng.standard_normal((n, d)) * col_scale * entry_scale).astype(np.float32)
    prob = dataclasses.replace(_with_dense(base, A32), n=n, d=d, B=np.ascontiguousarray(base.B[:n]))
    # lambda relative to the largest diagonal entry keeps the preconditioner's factor well posed
    gmax = float(np.max(np.sum(A32.astype(np.float64) ** 2, axis=0 if n >= d else 1)))
    prob = dataclasses.replace(prob, lambda_min=1e-3 * gmax, lambda_max=1e-2 * gmax)
    G = _gram(ctx, prob, "f64")
    Gref = ob.gram_extended(_ahat(prob))
    assert _scaled_err(G, Gref) <= _slice_bound(max(n, d))


def test_zero_columns(ctx):
    prob = small("c2_small")
    A = prob.A.astype(np.float32).copy()
    A[:, 5] = 0.0
    A[:, 90] = 0.0
    G = _gram(ctx, _with_dense(prob, A), "f64")
    for j in (5, 90):
        assert np.all(G[j, :] == 0.0) and np.all(G[:, j] == 0.0)
    Gref = ob.gram_extended(A)
    keep = np.setdiff1d(np.arange(prob.d), [5, 90])
    assert _scaled_err(G[np.ix_(keep, keep)], Gref[np.ix_(keep, keep)]) <= 1e-15


def test_several_row_splits_sampled(ctx):
    # 20000 rows -> 313 row blocks of 64; with 3 x 3 tiles the rows are split across work items
    prob = small("c2_small", n=20000, d=300, m=600)
    G = _gram(ctx, prob, "f64")
    A = _ahat(prob)
    rng = np.random.default_rng(5)
    rows = np.concatenate([np.arange(300), rng.integers(0, 300, 1500)])
    cols = np.concatenate([np.arange(300), rng.integers(0, 300, 1500)])
    ref = ob.gram_entries_extended(A, rows, cols)
    dg = np.sqrt(ref[:300])
    err = np.abs(G[rows, cols] - ref) / (dg[rows] * dg[cols])
    assert float(err.max()) <= 1e-15


@pytest.mark.parametrize("compute", ["f64", "f32x2"])
def test_path_parity_both_gram_kernels(ctx, compute):
    """x(lambda) through the sliced Gram and through the CUDA-core Gram agree with the oracle."""
    from paper_2210_12212_gb300 import ihsbin as ihs
    prob = small("c2_small")
    L = ob.num_intervals(prob.lambda_min, prob.lambda_max)
    r1, r2, kk = default_params(prob, L, 20)
    plan = ob.make_plan(prob.lambda_min, prob.lambda_max, r1, r2, kk, L=L)
    Xo = ob.ihs_bin_path(oracle_A(prob), prob.B, prob.sketch, prob.m, prob.s, prob.sketch_seed, plan,
                         prob.lambdas).X
    out = {}
    for gram in ("slices", "fma"):
        gp = gpu_problem(ihs, ctx, prob)
        gp.sketch(prob.sketch, prob.m, prob.s, prob.sketch_seed)
        gp.build_basis(prob.lambda_min, prob.lambda_max, L=L, k=kk, rho1=r1, rho2=r2, compute=compute, gram=gram)
        out[gram] = gp.eval_path(prob.lambdas)
        gp.close()
        assert rel_err_max(out[gram], Xo) <= (1e-10 if compute == "f64" else 1e-8)
    assert rel_err_max(out["slices"], out["fma"]) <= (1e-10 if compute == "f64" else 1e-8)


def test_slices_refused_for_f64_data(ctx):
    from paper_2210_12212_gb300 import ihsbin as ihs
    prob = small("c1_small")
    gp = gpu_problem(ihs, ctx, prob)
    gp.sketch(prob.sketch, prob.m, prob.s, prob.sketch_seed)
    with pytest.raises(ihs.IhsbinError) as e:
        gp.build_basis(prob.lambda_min, prob.lambda_max, L=1, k_default=2, gram="slices")
    assert e.value.status == ihs.ERR_UNSUPPORTED
    gp.close()
