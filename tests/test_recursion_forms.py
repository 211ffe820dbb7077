"""Two restatements the CUDA path relies on, checked on the CPU against the oracle.

* The two-product step of the basis recursion.  Proposition 1's recursion, re-centred at lam0,
  forms R = tau (G u_j + lam0 u_j) + lam0 u_{j-1} and then u_j <- u_j - P R.  With
  M = P (G + lam0 I) the same step is u_{i+1,j} = u_{i,j} - tau M u_{i,j} - lam0 P u_{i,j-1}: both
  products then act on the old columns.  The basis terms it accumulates must be the oracle's.
* The Hadamard transform of the SRHT in int64 fixed point.  Each column is scaled by 2^k_c,
  k_c = 61 - log2(N_pad) - e_c (the column maximum below 2^e_c), and rounded once.  The butterflies
  are then exact integer additions that cannot leave int64.  The result differs from the exact
  transform by at most N_pad / 2 units of 2^-k_c.
"""
import math

import numpy as np

from oracle import ihsbin as ob
from oracle import sketch as osk


def _two_product_basis(G, GS, c, lam0, tau, k):
    D = G.shape[0]
    P = np.linalg.inv(GS + lam0 * np.eye(D))
    M = P @ (G + lam0 * np.eye(D))
    u = [P @ c]
    ut = [u[0].copy()]
    for i in range(1, k):
        new = [u[0] - tau * (M @ u[0])]
        new += [u[j] - tau * (M @ u[j]) - lam0 * (P @ u[j - 1]) for j in range(1, i)]
        new.append(-lam0 * (P @ u[i - 1]))
        u = new
        ut[:] = [ut[j] + u[j] for j in range(i)] + [u[i].copy()]
    return np.stack(ut)


def test_two_product_step_gives_the_oracle_basis():
    rng = np.random.default_rng(3)
    n, d, m, K, k = 80, 14, 40, 2, 11
    A = rng.standard_normal((n, d)) / (1.0 + np.arange(d)) ** 0.8
    B = rng.standard_normal((n, K))
    S = rng.standard_normal((m, n)) / math.sqrt(m)
    SA = S @ A
    GS, G, c = SA.T @ SA, A.T @ A, A.T @ B
    for lam0, tau in [(0.05, 0.7), (0.6, 1.1)]:
        ref = ob.basis(lambda V: G @ V, ob.precond(GS, lam0), c, tau, k)
        got = _two_product_basis(G, GS, c, lam0, tau, k)
        assert got.shape == ref.shape
        assert np.max(np.abs(got - ref)) <= 1e-11 * np.max(np.abs(ref))


def _fixed_point_transform(X):
    """H X with X scaled per column to integers, exact integer butterflies, scaled back."""
    N, D = X.shape
    pbits = int(round(math.log2(N)))
    out = np.empty((N, D))
    for col in range(D):
        cmax = float(np.max(np.abs(X[:, col])))
        e = math.frexp(cmax)[1] if cmax > 0 else 0           # cmax < 2^e
        kc = 61 - pbits - e
        v = [int(math.copysign(math.floor(abs(x) * 2.0 ** kc + 0.5), x)) for x in X[:, col]]
        h = 1
        while h < N:
            for s in range(0, N, 2 * h):
                for t in range(s, s + h):
                    a, b = v[t], v[t + h]
                    v[t], v[t + h] = a + b, a - b
            h *= 2
        assert max(abs(x) for x in v) < 2 ** 63                 # no int64 overflow
        out[:, col] = [math.ldexp(x, -kc) for x in v]
    return out


def test_fixed_point_hadamard_transform_within_its_bound():
    rng = np.random.default_rng(7)
    N, D = 512, 6
    X = rng.standard_normal((N, D)).astype(np.float32).astype(np.float64)
    X[:, 1] *= 1e-30                                           # tiny column: its own scale
    X[:, 2] = 0.0                                              # zero column
    X[:, 3] = np.abs(X[:, 3]) * 1e20                           # one sign, large values: the largest growth
    X[::7, 4] *= 1e-12                                         # wide exponent range inside one column
    ref = osk.fwht_rows(X)
    got = _fixed_point_transform(X)
    pbits = int(math.log2(N))
    for col in range(D):
        cmax = float(np.max(np.abs(X[:, col])))
        if cmax == 0:
            assert np.all(got[:, col] == 0)
            continue
        e = math.frexp(cmax)[1]
        unit = 2.0 ** -(61 - pbits - e)                         # 2^-k_c
        # N roundings of at most half a unit each, plus the FP64 reference's own rounding
        bound = N * unit / 2 + 4 * pbits * np.finfo(float).eps * N * cmax
        assert np.max(np.abs(got[:, col] - ref[:, col])) <= bound
        # relative to the column maximum, the rounding is at 2^-(62 - pbits) per entry
        assert unit / 2 <= 2.0 ** -(62 - pbits) * 2.0 ** e
