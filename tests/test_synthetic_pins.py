"""The workload generators of Section 6.1 against their definitions: the AR(1) rows equal
(n d)^(-1/4) Sigma z with the explicit Toeplitz Sigma_ij = alpha^|i-j| (the generator runs two
recursive filters instead), their covariance is Sigma^2 / sqrt(n d), and the Gaussian kernel
matrix is symmetric, positive semidefinite, one on the diagonal, and its test rows are the
kernel between the held-out and the training points."""
import numpy as np
import scipy.linalg as sla

from synthetic import configs as sc
from synthetic import make_problem, make_split


def test_ar1_filters_equal_the_toeplitz_product():
    n, d, alpha, seed = 37, 29, 0.9, 5
    A = sc._ar1_rows(np.random.default_rng(seed), n, d, alpha)
    Z = np.random.default_rng(seed).standard_normal((d, n))       # the generator's draw for one block
    Sigma = sla.toeplitz(alpha ** np.arange(d))
    ref = ((n * d) ** -0.25 * (Sigma @ Z)).T
    np.testing.assert_allclose(A, ref.astype(np.float32), rtol=2e-6, atol=2e-6 * np.abs(ref).max())


def test_ar1_row_covariance():
    n, d, alpha = 40000, 12, 0.99
    A = sc._ar1_rows(np.random.default_rng(1), n, d, alpha).astype(np.float64)
    Sigma = sla.toeplitz(alpha ** np.arange(d))
    expect = Sigma @ Sigma / np.sqrt(n * d)
    emp = A.T @ A / n
    assert np.max(np.abs(emp - expect)) <= 0.05 * np.max(np.abs(expect))


def test_ar1_workload_model():
    prob = make_problem("ar1_small")
    assert prob.A.shape == (2000, 400) and prob.sketch == "countsketch" and prob.s == 1 and prob.m == 160
    assert (prob.lambda_min, prob.lambda_max) == (1.0, 100.0)
    # b = A v* + noise with sigma = 0.02
    r = prob.B - prob.A.astype(np.float64) @ prob.x_star
    assert abs(np.std(r) - 0.02) <= 0.003
    assert abs(np.mean(prob.x_star ** 2) * prob.d - 1.0) <= 0.2      # v* ~ N(0, I/d)


def test_kernel_matrix_properties():
    prob, A_test, B_test = make_split("gkernel_small", 50, seed=2)
    A = prob.A.astype(np.float64)
    assert prob.n == prob.d == 600 and prob.K == 10
    np.testing.assert_allclose(A, A.T, rtol=0, atol=1e-7)
    np.testing.assert_allclose(np.diag(A), 1.0, rtol=0, atol=1e-7)
    assert A.min() > 0 and A.max() <= 1.0
    assert np.linalg.eigvalsh(A).min() >= -1e-4
    assert np.all(prob.B.sum(axis=1) == 1) and np.all(B_test.sum(axis=1) == 1)
    # the test rows are the kernel of new points against the same training points: a training point
    # placed among the test points reproduces its row of A
    rng = np.random.default_rng(2)
    f, _ = sc._kernel_features(rng, 650, 3072, 10)
    K_all = sc._gauss_kernel(f, f[:600], 1000.0)
    np.testing.assert_allclose(K_all[:600], prob.A, rtol=0, atol=1e-6)
    np.testing.assert_allclose(K_all[600:], A_test, rtol=0, atol=1e-6)
