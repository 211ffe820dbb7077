"""Pins of the FP64 oracle to things other than itself (CPU only).

Each test checks the oracle against a closed form, a textbook or library
routine on tiny inputs, brute force, an invariant the paper states, or a
published known-answer vector, chosen so that a dropped term, a wrong sign or
index, or a transposed operand fails at least one of them.
"""
import math

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import ihsbin as ob
from oracle import philox
from oracle import sketch as sk


def rand_problem(n, d, K=1, seed=0, decay=0.5):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, d)) * (1.0 + np.arange(d)) ** (-decay)
    B = rng.standard_normal((n, K))
    return A, B


# ------------------------------------------------------------------ generator
def test_philox_known_answers():
    # Known-answer vectors published with the Philox4x32-10 reference implementation.
    cases = [
        ((0, 0, 0, 0, 0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
        ((0xFFFFFFFF,) * 6, (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
        ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344, 0xA4093822, 0x299F31D0),
         (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
    ]
    for args, want in cases:
        got = tuple(int(x) for x in philox.philox4x32_10(*args))
        assert got == want


def test_philox_stream_layout():
    w = philox.draw(0x0123456789ABCDEF, 5, np.array([0, 1, (1 << 40) + 3], dtype=np.uint64))
    # counter = (idx lo, idx hi, stream, 0), key = (seed lo, seed hi)
    ref = philox.philox4x32_10(3, 256, 5, 0, 0x89ABCDEF, 0x01234567)
    assert all(int(w[q][2]) == int(ref[q]) for q in range(4))


def test_uniform_open_interval():
    u = philox.uniform_open(np.array([0, 0xFFFFFFFF], dtype=np.uint32))
    assert 0.0 < u[0] < 1e-9 and 1 - 1e-9 < u[1] < 1.0


# -------------------------------------------------------------------- sketches
@pytest.mark.parametrize("n", [1, 2, 8, 64, 256])
def test_fwht_equals_sylvester_hadamard(n):
    X = np.random.default_rng(n).standard_normal((n, 3))
    assert np.allclose(sk.fwht_rows(X), sla.hadamard(n) @ X, atol=1e-12)


def test_fwht_involution():
    X = np.random.default_rng(1).standard_normal((128, 2))
    assert np.allclose(sk.fwht_rows(sk.fwht_rows(X)), 128 * X)


def test_srht_rows_brute_force():
    N_pad, m, seed = 512, 37, 11
    rows = sk.srht_rows(N_pad, m, seed)
    keys = []
    for r in range(N_pad):
        w0, w1, _, _ = philox.philox4x32_10(r, 0, 7, 0, seed, 0)
        keys.append(((int(w1) << 32) | int(w0), r))
    want = sorted(r for _, r in sorted(keys)[:m])
    assert list(rows) == want
    assert len(set(rows)) == m and np.all(np.diff(rows) > 0)


def test_srht_expectation_identity():
    # E[S^T S] = I for S = (1/sqrt m) R H D with m of N_pad rows sampled without replacement.
    N, m = 16, 4
    acc = np.zeros((N, N))
    reps = 3000
    for seed in range(reps):
        acc += (lambda S: S.T @ S)(sk.apply_srht(np.eye(N), m, seed))
    acc /= reps
    assert np.allclose(np.diag(acc), 1.0, atol=1e-12)          # diagonal is exactly 1 each draw
    assert np.abs(acc - np.eye(N)).max() < 0.08


def test_countsketch_structure_and_diag():
    N, m, s, seed = 300, 24, 4, 5
    S = sk.apply_countsketch(np.eye(N), m, s, seed)            # = S itself (m x N)
    nz = S != 0
    assert np.all(nz.sum(axis=0) == s)
    for t in range(s):
        assert np.all(nz[t * (m // s):(t + 1) * (m // s)].sum(axis=0) == 1)
    assert np.allclose(np.abs(S[nz]), 1 / math.sqrt(s))
    assert np.allclose(np.diag(S.T @ S), 1.0)                  # exact: s entries of 1/s each


def test_countsketch_bucket_bruteforce():
    rows, sign = sk.countsketch_map(5, 12, 3, 99)
    for i in range(5):
        for t in range(3):
            w0, w1, _, _ = philox.philox4x32_10(i * 3 + t, 0, 3, 0, 99, 0)
            assert rows[i, t] == t * 4 + ((int(w0) * 4) >> 32)
            assert sign[i, t] == (-1.0 if int(w1) & 1 else 1.0)


def test_countsketch_csr_equals_dense():
    import scipy.sparse as sp
    rng = np.random.default_rng(3)
    A = rng.standard_normal((80, 9)) * (rng.random((80, 9)) < 0.3)
    d1 = sk.apply_countsketch(A, 16, 2, 4)
    d2 = sk.apply_countsketch(sp.csr_matrix(A), 16, 2, 4)
    assert np.allclose(d1, d2)


def test_gaussian_moments_and_scale():
    m, N = 64, 2000
    S = sk.gaussian_entries(m, N, 123)
    z = S.ravel() * math.sqrt(m)
    assert abs(z.mean()) < 0.02 and abs(z.var() - 1) < 0.02
    assert abs(np.mean(z ** 4) - 3) < 0.1
    # Box-Muller brute force for one entry
    w0, w1, _, _ = philox.philox4x32_10(5 * N + 7, 0, 5, 0, 123, 0)
    u0, u1 = (int(w0) + 0.5) / 2 ** 32, (int(w1) + 0.5) / 2 ** 32
    assert math.isclose(S[5, 7] * math.sqrt(m),
                        math.sqrt(-2 * math.log(u0)) * math.cos(2 * math.pi * u1), rel_tol=1e-14)


# ----------------------------------------------------------------------- plan
def test_interval_count_rule():
    assert ob.num_intervals(1.0, 1e6) == 27
    assert ob.num_intervals(1.0, 100.0) == 9
    assert ob.num_intervals(1.0, 1.2) == 1


def test_interval_assignment_half_open():
    p = ob.make_plan(1.0, 100.0, 2.0, 0.5, 5, L=4)
    assert ob.interval_of(1.0, p) == 0
    assert ob.interval_of(p.edges[1], p) == 1
    assert ob.interval_of(np.nextafter(p.edges[1], 0), p) == 0
    assert ob.interval_of(100.0, p) == 3


def test_step_size_matches_proof_and_not_printed_form():
    lo, hi, r1, r2 = 2.0, 9.0, 1.7, 0.4
    tau = ob.step_size(lo, hi, r1, r2)
    kt = r1 * hi / (r2 * lo)
    assert math.isclose(tau, 2 * math.sqrt(r1 * r2) / (math.sqrt(kt) + 1 / math.sqrt(kt)))
    printed = 2 * math.sqrt(1 / (r1 * r2)) / (math.sqrt(kt) + 1 / math.sqrt(kt))
    assert not math.isclose(tau, printed, rel_tol=1e-3)


# ---------------------------------------------------------------- exact paths
@pytest.mark.parametrize("n,d", [(40, 7), (6, 11)])
def test_exact_ridge_equals_svd_path(n, d):
    A, B = rand_problem(n, d, K=2, seed=n)
    lams = [1e-3, 0.1, 3.0]
    want = ob.svd_path(A, B, lams)
    for t, lam in enumerate(lams):
        assert np.allclose(ob.exact_ridge(A, B, lam), want[t], rtol=1e-10, atol=1e-12)


def test_ridge_norm_strictly_decreasing():
    A, B = rand_problem(50, 8, seed=2)
    lams = np.geomspace(1e-4, 1e3, 40)
    norms = [np.linalg.norm(x) for x in ob.svd_path(A, B, lams)]
    assert np.all(np.diff(norms) < 0)


def test_precond_cholesky_equals_svd_formula():
    rng = np.random.default_rng(4)
    for m, d in [(5, 9), (14, 9)]:           # m < d and m >= d forms
        SA = rng.standard_normal((m, d))
        V = rng.standard_normal((d, 3))
        P = ob.precond(SA.T @ SA, 0.37)
        assert np.allclose(P.solve(V), ob.precond_svd_apply(SA, 0.37, V), rtol=1e-10)


# ------------------------------------------------------------ basis identities
def test_identity_sketch_one_step_is_exact_ridge():
    # S = I, lam = lam0, tau = 1, k = 1: x = P A^T b = x*(lam0).
    A, B = rand_problem(30, 6, seed=5)
    lam0 = 0.25
    P = ob.precond(A.T @ A, lam0)
    ut = ob.basis(ob.aspace_operator(A), P, A.T @ B, 1.0, 1)
    assert np.allclose(ob.evaluate(ut, 1.0, lam0, lam0), ob.exact_ridge(A, B, lam0), rtol=1e-12)


@pytest.mark.parametrize("k", [1, 2, 5, 17])
def test_identity_sketch_closed_form(k):
    # S = I: in the right singular basis x_k = sum_i [1 - (1 - tau (s_i^2+lam)/(s_i^2+lam0))^k] x*_i(lam).
    A, B = rand_problem(25, 5, seed=k)
    lo, hi = 0.05, 0.4
    lam0 = math.sqrt(lo * hi)
    tau = 0.8
    P = ob.precond(A.T @ A, lam0)
    ut = ob.basis(ob.aspace_operator(A), P, A.T @ B, tau, k)
    U, s, Vt = np.linalg.svd(A, full_matrices=False)
    for lam in [lo, lam0, 0.21, hi]:
        xs = Vt.T @ ((s / (s ** 2 + lam))[:, None] * (U.T @ B))
        factor = 1.0 - (1.0 - tau * (s ** 2 + lam) / (s ** 2 + lam0)) ** k
        want = Vt.T @ (factor[:, None] * (Vt @ xs))
        assert np.allclose(ob.evaluate(ut, tau, lam0, lam), want, rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("m", [6, 30])
def test_bin_equals_k_ihs_steps(m):
    # Proposition 1: the basis composition equals k plain IHS steps, for every lambda.
    A, B = rand_problem(60, 12, K=2, seed=m)
    SA = sk.apply_gaussian(A, m, 77)
    lo, hi = 0.02, 0.06
    lam0 = math.sqrt(lo * hi)
    tau = ob.step_size(lo, hi, 1.8, 0.3)
    P = ob.precond(SA.T @ SA, lam0)
    c = A.T @ B
    k = 25
    ut = ob.basis(ob.aspace_operator(A), P, c, tau, k)
    for lam in np.linspace(lo, hi, 5):
        want = ob.direct_ihs(ob.aspace_operator(A), P, c, tau, lam, k)
        assert np.allclose(ob.evaluate(ut, tau, lam0, lam), want, rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("jmax", [1, 4, 9])
def test_truncated_basis_keeps_its_terms(jmax):
    # u_j is updated from u_j and u_{j-1} only, so the terms j < jmax are the full basis's terms,
    # and the truncated expansion differs from k IHS steps only by the omitted terms.
    A, B = rand_problem(60, 12, K=2, seed=jmax)
    SA = sk.apply_gaussian(A, 30, 5)
    lo, hi = 0.02, 0.06
    lam0 = math.sqrt(lo * hi)
    tau = ob.step_size(lo, hi, 1.8, 0.3)
    P = ob.precond(SA.T @ SA, lam0)
    c = A.T @ B
    full = ob.basis(ob.aspace_operator(A), P, c, tau, 14)
    cut = ob.basis(ob.aspace_operator(A), P, c, tau, 14, jmax=jmax)
    assert cut.shape[0] == jmax
    np.testing.assert_allclose(cut, full[:jmax], rtol=1e-13, atol=1e-15 * np.abs(full).max())


def test_recentred_equals_printed_form_small_k():
    A, B = rand_problem(40, 6, seed=9)
    SA = sk.apply_srht(A, 16, 3)
    lam0, tau, k = 0.3, 0.7, 6
    P = ob.precond(SA.T @ SA, lam0)
    c = A.T @ B
    ut = ob.basis(ob.aspace_operator(A), P, c, tau, k)
    ul = ob.basis_literal(ob.aspace_operator(A), P.solve, c, tau, k)
    for lam in [0.2, 0.3, 0.45]:
        assert np.allclose(ob.evaluate(ut, tau, lam0, lam), ob.evaluate_literal(ul, tau, lam),
                           rtol=1e-9)


def test_gd_bin_closed_form_with_identity_preconditioner():
    # With P := I the printed recursion is gradient descent; eq. before Algorithm 1:
    # x_k = tau sum_j (-tau lam)^j u_j,  u_j = sum_{i=0}^{k-1-j} C(i+j, j) (I - tau A^T A)^i A^T b.
    A, B = rand_problem(20, 4, seed=3)
    A = A / np.linalg.norm(A, 2)
    tau, k = 0.9, 7
    c = A.T @ B
    ul = ob.basis_literal(ob.aspace_operator(A), lambda v: v, c, tau, k)
    M = np.eye(4) - tau * A.T @ A
    for j in range(k):
        uj = sum(math.comb(i + j, j) * np.linalg.matrix_power(M, i) @ c for i in range(k - j))
        assert np.allclose(ul[j], (-1) ** j * uj, rtol=1e-10, atol=1e-12)
    lam = 0.13
    x_gd = tau * sum((-tau * lam) ** j * (-1) ** j * ul[j] for j in range(k))
    assert np.allclose(ob.evaluate_literal(ul, tau, lam), x_gd)


def test_matrix_valued_equals_column_solves():
    A, B = rand_problem(50, 7, K=3, seed=12)
    plan = ob.make_plan(0.01, 1.0, 2.0, 0.3, 12, L=3)
    lams = np.geomspace(0.01, 1.0, 7)
    full = ob.ihs_bin_path(A, B, "gaussian", 20, 1, 8, plan, lams).X
    for r in range(3):
        col = ob.ihs_bin_path(A, B[:, r], "gaussian", 20, 1, 8, plan, lams).X
        assert np.allclose(full[:, :, r], col[:, :, 0], rtol=1e-12, atol=1e-14)


def test_gram_and_aspace_products_agree():
    A, B = rand_problem(45, 6, seed=1)
    plan = ob.make_plan(0.01, 1.0, 2.0, 0.3, 9, L=2)
    lams = np.geomspace(0.01, 1.0, 5)
    x1 = ob.ihs_bin_path(A, B, "srht", 16, 1, 2, plan, lams, product="gram").X
    x2 = ob.ihs_bin_path(A, B, "srht", 16, 1, 2, plan, lams, product="aspace").X
    assert np.allclose(x1, x2, rtol=1e-11)


def test_dual_converges_to_primal_ridge():
    # Section 5.2: under-determined A (n < d) through the dual; x = A^T z.
    A, B = rand_problem(12, 40, K=2, seed=6, decay=0.0)
    lams = np.geomspace(0.5, 5.0, 6)
    plan = ob.make_plan(0.5, 5.0, 1.5, 0.4, 200, L=2)
    res = ob.ihs_bin_path(A, B, "gaussian", 36, 1, 1, plan, lams)
    assert res.dual and res.X.shape == (6, 40, 2)
    want = ob.svd_path(A, B, lams)
    assert np.allclose(res.X, want, rtol=1e-10, atol=1e-12)
    # the dual solution itself: z = (A A^T + lam I)^-1 b
    z0 = np.linalg.solve(A @ A.T + lams[0] * np.eye(12), B)
    assert np.allclose(res.Z[0], z0, rtol=1e-10)


def test_direct_path_equals_bin_path():
    A, B = rand_problem(70, 9, seed=8)
    plan = ob.make_plan(1e-3, 1.0, 2.2, 0.2, 30, L=0)
    lams = np.geomspace(1e-3, 1.0, 11)
    res = ob.ihs_bin_path(A, B, "countsketch", 24, 2, 5, plan, lams)
    assert np.allclose(res.X, ob.direct_path(A, B, res.GS, plan, lams), rtol=1e-9, atol=1e-12)


def test_theorem4_contraction_bound_holds_with_exact_rhos():
    # Theorem 4 with rho1/rho2 = extreme eigenvalues of C_S (generalised eigenvalues of
    # (G_S + lam0 I, G + lam0 I)): delta_{k+1}/delta_k <= ((kt-1)/(kt+1))^2 on [lmin, lmax]
    # with the step size of the proof; the printed closed form of alpha breaks the bound.
    A, B = rand_problem(200, 10, seed=21)
    b = B[:, 0]
    G = A.T @ A
    c = A.T @ b
    lmin, lmax = 0.5, 2.0
    lam0 = math.sqrt(lmin * lmax)

    def worst_ratio(GS, tau):
        P = ob.precond(GS, lam0)
        worst = 0.0
        for lam in np.linspace(lmin, lmax, 9):
            H = G + lam * np.eye(10)
            xs = np.linalg.solve(H, c)
            x = np.zeros(10)
            prev = 0.5 * (x - xs) @ H @ (x - xs)
            for _ in range(12):
                x = x - tau * P.solve(G @ x - c + lam * x)
                cur = 0.5 * (x - xs) @ H @ (x - xs)
                worst = max(worst, cur / prev)
                prev = cur
        return worst

    for m in (14, 20, 40):
        SA = sk.apply_gaussian(A, m, 31)
        GS = SA.T @ SA
        gam = sla.eigh(GS + lam0 * np.eye(10), G + lam0 * np.eye(10), eigvals_only=True)
        r1, r2 = gam.max() * (1 + 1e-9), gam.min() / (1 + 1e-9)
        kt = r1 * lmax / (r2 * lmin)
        bound = ((kt - 1) / (kt + 1)) ** 2
        assert worst_ratio(GS, ob.step_size(lmin, lmax, r1, r2)) <= bound
        if m == 14:
            tau_printed = 2 * math.sqrt(1 / (r1 * r2)) / (math.sqrt(kt) + 1 / math.sqrt(kt))
            assert worst_ratio(GS, tau_printed) > 1.0 > bound


def test_known_sigma_d_rule_bound_holds_and_tightens():
    # Remark after Theorem 4: with sigma_d^2 = the smallest eigenvalue of A^T A, lam0 =
    # sqrt((lmax + s)(lmin + s)) - s and alpha = 2 (lam0 + s) / ((lmin + s)/rho1 + (lmax + s)/rho2),
    # the energy error contracts per step by at most ((kh-1)/(kh+1))^2, kh = rho1 (lmax + s) / (rho2 (lmin + s)),
    # with rho1/rho2 the extreme generalised eigenvalues of (G_S + lam0 I, G + lam0 I)
    rng = np.random.default_rng(21)
    A = rng.standard_normal((200, 10)) * (1 + np.arange(10)) ** -0.5
    b = A @ rng.standard_normal(10) + 0.1 * rng.standard_normal(200)
    G, c = A.T @ A, A.T @ b
    s2 = np.linalg.eigvalsh(G).min()
    lmin, lmax = 0.5, 2.0
    for sig in (s2, 0.5 * s2):
        lam0 = ob.center(lmin, lmax, sig)
        assert abs((lam0 + sig) ** 2 - (lmin + sig) * (lmax + sig)) <= 1e-12 * (lmax + sig) ** 2
        for m in (14, 20, 40):
            SA = sk.apply_gaussian(A, m, 31)
            GS = SA.T @ SA
            gam = sla.eigh(GS + lam0 * np.eye(10), G + lam0 * np.eye(10), eigvals_only=True)
            r1, r2 = gam.max() * (1 + 1e-9), gam.min() / (1 + 1e-9)
            tau = ob.step_size(lmin, lmax, r1, r2, sig)
            P = ob.precond(GS, lam0)
            worst = 0.0
            for lam in np.linspace(lmin, lmax, 9):
                H = G + lam * np.eye(10)
                xs = np.linalg.solve(H, c)
                x = np.zeros(10)
                prev = 0.5 * (x - xs) @ H @ (x - xs)
                for _ in range(12):
                    x = x - tau * P.solve(G @ x - c + lam * x)
                    cur = 0.5 * (x - xs) @ H @ (x - xs)
                    worst = max(worst, cur / prev)
                    prev = cur
            kh = r1 * (lmax + sig) / (r2 * (lmin + sig))
            kt = r1 * lmax / (r2 * lmin)
            assert worst <= ((kh - 1) / (kh + 1)) ** 2 < ((kt - 1) / (kt + 1)) ** 2
    # sigma_d^2 = 0 is the default rule
    assert ob.center(lmin, lmax, 0.0) == math.sqrt(lmin * lmax)
    assert ob.step_size(lmin, lmax, 2.0, 0.5, 0.0) == 2 * math.sqrt(lmin * lmax) / (lmin / 2.0 + lmax / 0.5)


def test_theorem4_k_meets_its_rate():
    # the chosen k is the first with rate^k <= eps
    lo, hi, r1, r2, eps = 1.0, 1.6, 2.0, 0.3, 1e-7
    k = ob.theorem4_k(r1, r2, lo, hi, eps)
    kt = r1 * hi / (r2 * lo)
    rate = (kt - 1) / (kt + 1)
    assert rate ** k <= eps < rate ** (k - 1)


def test_auto_plan_effective_dimension_limits():
    # d_e from the sketch tends to rank(G_S) as lam0 -> 0 and to 0 as lam0 -> inf
    rng = np.random.default_rng(2)
    SA = rng.standard_normal((6, 9))
    GS = SA.T @ SA
    p_small = ob.auto_plan(GS, 100, 1e-9, 2e-9, L=1)
    p_large = ob.auto_plan(GS, 100, 1e9, 2e9, L=1)
    de_small = 9 - p_small.lam0[0] * np.trace(np.linalg.inv(GS + p_small.lam0[0] * np.eye(9)))
    de_large = 9 - p_large.lam0[0] * np.trace(np.linalg.inv(GS + p_large.lam0[0] * np.eye(9)))
    assert abs(de_small - 6) < 1e-6 and de_large < 1e-6
    assert p_small.k[0] > p_large.k[0] >= 1


# ---- extended-precision Gram (checks the tensor-core Gram below FP64 GEMM rounding)
def test_gram_extended_exact_on_integers():
    rng = np.random.default_rng(11)
    A = rng.integers(-1000, 1001, size=(50, 7))
    exact = [[sum(int(A[k, i]) * int(A[k, j]) for k in range(50)) for j in range(7)] for i in range(7)]
    assert np.array_equal(ob.gram_extended(A.astype(np.float64)), np.array(exact, dtype=np.float64))


def test_gram_extended_rational_reference():
    from fractions import Fraction
    rng = np.random.default_rng(12)
    A = (rng.standard_normal((20, 4)) * np.exp2(rng.integers(-20, 20, size=(20, 4)))).astype(np.float32)
    G = ob.gram_extended(A)
    for i in range(4):
        for j in range(4):
            ref = float(sum(Fraction(float(A[k, i])) * Fraction(float(A[k, j])) for k in range(20)))
            assert abs(G[i, j] - ref) <= np.spacing(abs(ref))


def test_gram_entries_extended_match_full():
    rng = np.random.default_rng(13)
    A = rng.standard_normal((300, 9)).astype(np.float32)
    rows, cols = rng.integers(0, 9, 40), rng.integers(0, 9, 40)
    assert np.array_equal(ob.gram_entries_extended(A, rows, cols), ob.gram_extended(A)[rows, cols])


# ---- losses along the path (Section 6.1)
def test_train_loss_closed_form_at_ridge_solution():
    # at x*(lam) the normal equations give ||A x - b||^2 + lam ||x||^2 = ||b||^2 - b^T A x*
    rng = np.random.default_rng(21)
    A = rng.standard_normal((60, 9))
    b = rng.standard_normal((60, 2))
    lams = np.array([0.01, 0.5, 7.0])
    X = np.stack([ob.exact_ridge(A, b, lam) for lam in lams])
    train, _ = ob.path_losses(A, b, None, None, X, lams)
    closed = [0.5 * (np.sum(b * b) - np.sum(b * (A @ X[t]))) for t in range(3)]
    np.testing.assert_allclose(train, closed, rtol=1e-12)


def test_test_loss_on_training_data_drops_the_ridge_term():
    rng = np.random.default_rng(22)
    A = rng.standard_normal((40, 6))
    b = rng.standard_normal((40, 1))
    lams = np.array([0.1, 1.0])
    X = rng.standard_normal((2, 6, 1))
    train, test = ob.path_losses(A, b, A, b, X, lams)
    np.testing.assert_allclose(test, train - 0.5 * lams * np.sum(X * X, axis=(1, 2)), rtol=1e-13)


def test_split_keeps_the_model():
    from synthetic import make_problem, make_split
    full = make_problem("c2_small", seed=0, n=3400)
    train, At, Bt = make_split("c2_small", 400, seed=0)
    assert train.n == 3000 and At.shape == (400, train.d) and Bt.shape == (400, 1)
    assert np.array_equal(train.A, full.A[:3000]) and np.array_equal(At, full.A[3000:])
    tr, A2, B2 = make_split("c3_small", 50, seed=0)
    assert tr.row_ptr.shape == (tr.n + 1,) and A2.shape == (50, tr.d)


def test_tf32_rounding_known_values():
    # TF32 keeps 10 fraction bits: 1 + k 2^-10 are representable; halfway points go away from zero
    from oracle.precision import round_tf32
    u = 2.0 ** -10
    x = np.array([1.0, 1.0 + u, 1.0 + u / 2, 1.0 + u / 2 - 2.0 ** -23, 1.0 + 3 * u / 2, -(1.0 + u / 2),
                  2.0 ** -126, 3.0e38, 0.0, -0.0, np.inf], dtype=np.float32)
    want = np.array([1.0, 1.0 + u, 1.0 + u, 1.0, 1.0 + 2 * u, -(1.0 + u), 2.0 ** -126, np.float32(3.0e38),
                     0.0, -0.0, np.inf], dtype=np.float32)
    got = round_tf32(x)
    # 3e38 = 0x7F61B1E6: its 13 low bits 0x11E6 >= 0x1000 round the magnitude up
    want[7] = np.uint32(0x7F61C000).view(np.float32)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))
    assert np.isnan(round_tf32(np.array([np.nan], dtype=np.float32)))[0]


def test_tf32_rounding_is_nearest():
    # against the definition on a grid: the result is one of the two neighbours at 2^-10 relative
    # spacing, the nearer one, and the error is at most half the spacing
    from oracle.precision import round_tf32
    rng = np.random.default_rng(4)
    x = (rng.standard_normal(100000) * 10.0 ** rng.integers(-8, 8, 100000)).astype(np.float32)
    r = round_tf32(x).astype(np.float64)
    e = np.floor(np.log2(np.abs(x.astype(np.float64))))
    ulp = 2.0 ** (e - 10)
    assert np.all(np.abs(r - x) <= ulp / 2 * (1 + 1e-12))
    assert np.all(np.abs(r / ulp - np.round(r / ulp)) == 0)   # on the TF32 grid of x's binade (or the next)
