"""Seeded problem generators (data only; no IHS-BIN arithmetic).

Every generator is deterministic in its seed and uses numpy's PCG64 stream.
The sketch's own random draws are NOT generated here: each side (oracle and
CUDA path) derives them from a counter-based generator it implements itself.

Workloads (sizes are the full ones; ``*_small`` variants keep the structure
at sizes the FP64 oracle finishes in seconds):

* ``c1``  dense over-determined 2000x100 FP64, columns scaled (1+j)^-0.8,
          b = A x* + 0.1 z, Gaussian sketch m=200, T=50 lambdas log-spaced in
          [1e-4, 1e2] * ||A||_2^2.
* ``c2``  dense FP32 65536x1024, A = U diag(1/k) V^T with Haar U, V,
          b = A x* + e with ||e|| = 0.01 ||A x*||, SRHT m=2048, T=200 lambdas
          in [1e-6, 1] * ||A||_2^2 (||A||_2 = 1 by construction).
* ``c3``  CSR 1,048,576x4096, 40 distinct uniform columns per row, N(0,1)
          FP32 values, b = A x* + 0.1 z, SJLT s=8 m=8192, T=1000 lambdas in
          [1e-4, 1e-2] * ||A||_2^2.  ``c3t`` is the under-determined
          transpose 4096x1,048,576.
* ``c4``  dense BF16 262144x2048, columns scaled (1+j)^-1, B = A X* + E with
          K=64 and ||E||_F = 0.01 ||A X*||_F, Gaussian sketch m=4096 in BF16,
          T=500 lambdas in [1e-4, 1e-2] * ||A||_2^2.
* ``c5``  serving mix: request shapes drawn per request seed.
* ``ar1`` / ``ar1u``  the paper's random data (Section 6.1): rows of A drawn
          from N(0, Sigma^2 / sqrt(n d)) with the AR(1) correlation
          Sigma_ij = 0.99^|i-j|, v* ~ N(0, I/d), b = A v* + N(0, 0.02^2), CountSketch
          (s = 1), lambdas in [1, 100]; over-determined 20000 x 4000 with m = 1600
          and under-determined 4000 x 20000 with m = 2400 (the shapes of the
          paper's random over- and under-determined experiments), FP32 storage.
* ``gkernel``  matrix-valued kernel ridge regression (Section 6.1, the CIFAR-10
          experiment's form): A_ij = exp(-||f_i - f_j||^2 / (2h)), h = 1000, on
          synthetic class-structured features in [0,1]^3072, B = one-hot labels of 10
          classes, n = d = 8192, Gaussian sketch m = 4096, lambdas in [0.1, 10].
"""
from __future__ import annotations

import dataclasses
import os
from typing import Optional

import numpy as np

__all__ = ["Problem", "CONFIGS", "make_problem", "make_split", "spectral_norm_sq", "lambda_grid",
           "to_bf16_bits", "bf16_bits_to_f32", "serving_requests"]


@dataclasses.dataclass
class Problem:
    name: str
    n: int
    d: int
    K: int
    layout: str                 # "dense" | "csr"
    storage: str                # "f64" | "f32" | "tf32" | "bf16"  (element type of A as stored; "tf32"
                                #  data is held as FP32 and the library rounds it, as the oracle does)
    A: Optional[np.ndarray]     # dense n x d (float64/float32, or uint16 bf16 bit patterns)
    row_ptr: Optional[np.ndarray]  # CSR int64 (n+1)
    col_idx: Optional[np.ndarray]  # CSR int32 (nnz), sorted within a row, no duplicates
    val: Optional[np.ndarray]      # CSR float32/float64 (nnz)
    B: np.ndarray               # n x K float64
    x_star: np.ndarray          # d x K planted solution
    sketch: str                 # "gaussian" | "srht" | "countsketch"
    m: int
    s: int                      # SJLT sparsity (countsketch only)
    sketch_seed: int
    lambda_min: float
    lambda_max: float
    lambdas: np.ndarray         # T float64, ascending
    norm2_sq: float             # ||A||_2^2 used to scale the lambda range

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1]) if self.layout == "csr" else self.n * self.d

    def dense_f64(self) -> np.ndarray:
        """A widened exactly to float64 (dense n x d)."""
        if self.layout == "csr":
            out = np.zeros((self.n, self.d))
            rows = np.repeat(np.arange(self.n), np.diff(self.row_ptr))
            out[rows, self.col_idx] = self.val
            return out
        if self.storage == "bf16":
            return bf16_bits_to_f32(self.A).astype(np.float64)
        return self.A.astype(np.float64)

    def transpose(self) -> "Problem":
        """Under-determined variant: A_u = A^T (CSR of the transpose)."""
        assert self.layout == "csr"
        n, d = self.n, self.d
        rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(self.row_ptr))
        order = np.lexsort((rows, self.col_idx))
        t_cols = rows[order].astype(np.int32)
        t_vals = self.val[order]
        counts = np.bincount(self.col_idx, minlength=d)
        t_ptr = np.zeros(d + 1, dtype=np.int64)
        np.cumsum(counts, out=t_ptr[1:])
        return dataclasses.replace(self, name=self.name + "t", n=d, d=n, row_ptr=t_ptr,
                                   col_idx=t_cols, val=t_vals)


def to_bf16_bits(x: np.ndarray) -> np.ndarray:
    """Round float32 to bfloat16 (round to nearest, ties to even); returns uint16 bits."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32)
    r = (b + np.uint32(0x7FFF) + ((b >> np.uint32(16)) & np.uint32(1))) >> np.uint32(16)
    return r.astype(np.uint16)


def bf16_bits_to_f32(bits: np.ndarray) -> np.ndarray:
    return (bits.astype(np.uint32) << np.uint32(16)).view(np.float32)


def spectral_norm_sq(matvec, rmatvec, d: int, iters: int, seed: int) -> float:
    """||A||_2^2 by power iteration on A^T A from a seeded start (input scaling only)."""
    rng = np.random.default_rng(seed + 7919)
    v = rng.standard_normal(d)
    v /= np.linalg.norm(v)
    est = 0.0
    for _ in range(iters):
        w = rmatvec(matvec(v))
        est = float(np.linalg.norm(w))
        v = w / est
    return est


def lambda_grid(lmin: float, lmax: float, T: int) -> np.ndarray:
    """T values log-spaced in [lmin, lmax] (endpoints included exactly)."""
    if T == 1:
        return np.array([lmin])
    g = lmin * (lmax / lmin) ** (np.arange(T) / (T - 1))
    g[0], g[-1] = lmin, lmax
    return g


def _cache_path(key: str) -> Optional[str]:
    root = os.environ.get("IHSBIN_DATA_CACHE")
    if not root:
        return None
    os.makedirs(root, exist_ok=True)
    return os.path.join(root, key + ".npz")


def _power_law_dense(rng, n, d, expo, dtype):
    scale = (1.0 + np.arange(d)) ** (-expo)
    A = rng.standard_normal((n, d)) * scale
    return A.astype(dtype)


def _haar_lowrank(rng, n, d):
    """A = U diag(1/k) V^T with Haar-distributed orthonormal U (n x d) and V (d x d)."""
    G1 = rng.standard_normal((n, d))
    U, R = np.linalg.qr(G1)
    U *= np.sign(np.diag(R))
    del G1
    G2 = rng.standard_normal((d, d))
    V, R2 = np.linalg.qr(G2)
    V *= np.sign(np.diag(R2))
    sig = 1.0 / np.arange(1, d + 1)
    return (U * sig) @ V.T


def _csr_uniform(rng, n, d, per_row, chunk=1 << 17):
    """Each row: `per_row` distinct uniform columns (draw, reject duplicates, sort), N(0,1) values."""
    cand_w = per_row + 16
    cols_out = np.empty(n * per_row, dtype=np.int32)
    for r0 in range(0, n, chunk):
        r1 = min(n, r0 + chunk)
        rows = r1 - r0
        while True:
            cand = rng.integers(0, d, size=(rows, cand_w), dtype=np.int32)
            order = np.argsort(cand, axis=1, kind="stable")
            srt = np.take_along_axis(cand, order, axis=1)
            dup_sorted = np.zeros_like(srt, dtype=bool)
            dup_sorted[:, 1:] = srt[:, 1:] == srt[:, :-1]
            dup = np.empty_like(dup_sorted)
            np.put_along_axis(dup, order, dup_sorted, axis=1)
            keep = ~dup
            rank = np.cumsum(keep, axis=1)
            sel = keep & (rank <= per_row)
            if np.all(sel.sum(axis=1) == per_row):
                break
        picked = cand[sel].reshape(rows, per_row)
        picked.sort(axis=1)
        cols_out[r0 * per_row:r1 * per_row] = picked.ravel()
    vals = rng.standard_normal(n * per_row, dtype=np.float32)
    row_ptr = np.arange(0, n * per_row + 1, per_row, dtype=np.int64)
    return row_ptr, cols_out, vals


def _ar1_rows(rng, n, d, alpha, chunk=1 << 12):
    """n rows a_i = (n d)^(-1/4) Sigma z_i with Sigma_ij = alpha^|i-j| (so Cov(a_i) = Sigma^2 / sqrt(n d)):
    Sigma z = F + G - z with the forward and backward AR(1) filters F_j = alpha F_{j-1} + z_j,
    G_j = alpha G_{j+1} + z_j (O(n d) instead of the d x d product)."""
    A = np.empty((n, d), dtype=np.float32)
    scale = (float(n) * d) ** -0.25
    for r0 in range(0, n, chunk):
        r1 = min(n, r0 + chunk)
        Zt = rng.standard_normal((d, r1 - r0))  # column j of the rows' block is row j here
        F = np.empty_like(Zt)
        Gb = np.empty_like(Zt)
        F[0] = Zt[0]
        for j in range(1, d):
            F[j] = alpha * F[j - 1] + Zt[j]
        Gb[d - 1] = Zt[d - 1]
        for j in range(d - 2, -1, -1):
            Gb[j] = alpha * Gb[j + 1] + Zt[j]
        A[r0:r1] = (scale * (F + Gb - Zt)).T
    return A


def _kernel_features(rng, n, p, classes):
    """Class-structured features in [0, 1]^p: f_i = clip(mu_{y_i} + 0.15 z_i), class means mu_c ~ U[0,1]^p."""
    mu = rng.uniform(0.0, 1.0, size=(classes, p))
    y = rng.integers(0, classes, size=n)
    f = np.clip(mu[y] + 0.15 * rng.standard_normal((n, p)), 0.0, 1.0)
    return f, y


def _gauss_kernel(F1, F2, h, chunk=2048):
    """exp(-||f_i - g_j||^2 / (2h)) in FP64 (the constant (2 pi h)^(-p/2) of Section 6.1 is dropped), FP32 out."""
    out = np.empty((F1.shape[0], F2.shape[0]), dtype=np.float32)
    n2 = np.sum(F2 * F2, axis=1)
    for r0 in range(0, F1.shape[0], chunk):
        X = F1[r0:r0 + chunk]
        d2 = np.sum(X * X, axis=1)[:, None] + n2[None, :] - 2.0 * (X @ F2.T)
        out[r0:r0 + chunk] = np.exp(-np.maximum(d2, 0.0) / (2.0 * h))
    return out


def _csr_matvec(row_ptr, col, val, n, d):
    rows = np.repeat(np.arange(n), np.diff(row_ptr))
    v64 = val.astype(np.float64)

    def mv(x):
        return np.bincount(rows, weights=v64 * x[col], minlength=n)

    def rmv(y):
        return np.bincount(col, weights=v64 * y[rows], minlength=d)
    return mv, rmv


# name -> parameters.  `small` variants keep the structure at oracle-friendly sizes.
CONFIGS = {
    "c1": dict(kind="powerlaw", n=2000, d=100, K=1, expo=0.8, storage="f64", sketch="gaussian",
               m=200, s=1, T=50, lrange=(1e-4, 1e2), noise=0.1),
    "c2": dict(kind="haar", n=65536, d=1024, K=1, storage="f32", sketch="srht", m=2048, s=1,
               T=200, lrange=(1e-6, 1.0), noise_rel=0.01),
    "c3": dict(kind="csr", n=1 << 20, d=4096, K=1, per_row=40, storage="f32", sketch="countsketch",
               m=8192, s=8, T=1000, lrange=(1e-4, 1e-2), noise=0.1),
    "c4": dict(kind="powerlaw", n=262144, d=2048, K=64, expo=1.0, storage="bf16",
               sketch="gaussian", m=4096, s=1, T=500, lrange=(1e-4, 1e-2), noise_rel=0.01),
    # Section 6.1's random data and the kernel form of its CIFAR-10 experiment
    "ar1": dict(kind="ar1", n=20000, d=4000, K=1, alpha=0.99, sigma=0.02, storage="f32", sketch="countsketch",
                m=1600, s=1, T=100, lrange_abs=(1.0, 100.0)),
    "ar1u": dict(kind="ar1", n=4000, d=20000, K=1, alpha=0.99, sigma=0.02, storage="f32", sketch="countsketch",
                 m=2400, s=1, T=100, lrange_abs=(1.0, 100.0)),
    "gkernel": dict(kind="gkernel", n=8192, d=8192, K=10, p=3072, h=1000.0, storage="f32", sketch="gaussian",
                    m=4096, s=1, T=100, lrange_abs=(0.1, 10.0)),
    # structure-preserving small variants (ragged against 64-wide tiles)
    "c1_small": dict(kind="powerlaw", n=300, d=37, K=1, expo=0.8, storage="f64", sketch="gaussian",
                     m=80, s=1, T=23, lrange=(1e-3, 1e1), noise=0.1),
    "c2_small": dict(kind="haar", n=3000, d=96, K=1, storage="f32", sketch="srht", m=192, s=1,
                     T=40, lrange=(1e-3, 1.0), noise_rel=0.01),
    "c3_small": dict(kind="csr", n=5000, d=200, K=1, per_row=12, storage="f32",
                     sketch="countsketch", m=400, s=4, T=60, lrange=(1e-4, 1e-2), noise=0.1),
    "c4_small": dict(kind="powerlaw", n=2048, d=72, K=5, expo=1.0, storage="bf16",
                     sketch="gaussian", m=160, s=1, T=30, lrange=(1e-4, 1e-2), noise_rel=0.01),
    "ar1_small": dict(kind="ar1", n=2000, d=400, K=1, alpha=0.99, sigma=0.02, storage="f32", sketch="countsketch",
                      m=160, s=1, T=30, lrange_abs=(1.0, 100.0)),
    "ar1u_small": dict(kind="ar1", n=400, d=2000, K=1, alpha=0.99, sigma=0.02, storage="f32", sketch="countsketch",
                       m=240, s=1, T=30, lrange_abs=(1.0, 100.0)),
    "gkernel_small": dict(kind="gkernel", n=600, d=600, K=10, p=3072, h=1000.0, storage="f32", sketch="gaussian",
                          m=300, s=1, T=30, lrange_abs=(0.1, 10.0)),
}


def make_transposed(name: str, seed: int = 0, **overrides) -> Problem:
    """Under-determined variant of a CSR workload: A_u = A^T (d x n), with its own planted x*_u and
    b_u = A_u x*_u + 0.1 z; the lambda range keeps the base workload's fractions of ||A||_2^2."""
    base = make_problem(name, seed=seed, **overrides)
    t = base.transpose()
    rng = np.random.default_rng(seed + 31337)
    x_u = rng.standard_normal((t.d, base.K))
    mv, _ = _csr_matvec(t.row_ptr, t.col_idx, t.val, t.n, t.d)
    B = np.stack([mv(x_u[:, r]) for r in range(base.K)], axis=1) + 0.1 * rng.standard_normal((t.n, base.K))
    return dataclasses.replace(t, name=name + "t", B=B, x_star=x_u)


def make_problem(name: str, seed: int = 0, **overrides) -> Problem:
    """Build the named workload deterministically from `seed`.

    `overrides` may replace any entry of the config table (n, d, m, T, lrange, ...).
    Set IHSBIN_DATA_CACHE to a directory to cache large generated inputs.
    """
    if name.endswith("t") and name[:-1] in CONFIGS and CONFIGS[name[:-1]]["kind"] == "csr":
        return make_transposed(name[:-1], seed=seed, **overrides)
    cfg = dict(CONFIGS[name])
    cfg.update(overrides)
    key = f"{name}_s{seed}_" + "_".join(f"{k}{cfg[k]}" for k in sorted(cfg))
    key = "".join(ch if ch.isalnum() or ch in "_.-" else "_" for ch in key)[:180]
    cpath = _cache_path(key)
    if cpath and os.path.exists(cpath):
        z = np.load(cpath, allow_pickle=False)
        return _from_cached(name, cfg, {f: z[f] for f in z.files})

    rng = np.random.default_rng(seed)
    n, d, K = cfg["n"], cfg["d"], cfg["K"]
    A = row_ptr = col = val = None
    layout = "dense"
    if cfg["kind"] == "powerlaw":
        if cfg["storage"] == "bf16":
            scale = (1.0 + np.arange(d)) ** (-cfg["expo"])
            A = np.empty((n, d), dtype=np.uint16)
            step = max(1, (1 << 24) // d)
            for r0 in range(0, n, step):
                r1 = min(n, r0 + step)
                z = rng.standard_normal((r1 - r0, d), dtype=np.float32)
                A[r0:r1] = to_bf16_bits((z * scale).astype(np.float32))
            Af = None
        else:
            A = _power_law_dense(rng, n, d, cfg["expo"], np.float64 if cfg["storage"] == "f64"
                                 else np.float32)
            Af = A
    elif cfg["kind"] == "haar":
        A = _haar_lowrank(rng, n, d).astype(np.float32 if cfg["storage"] in ("f32", "tf32") else np.float64)
        Af = A
    elif cfg["kind"] == "csr":
        layout = "csr"
        row_ptr, col, val = _csr_uniform(rng, n, d, cfg["per_row"])
    elif cfg["kind"] == "ar1":
        A = _ar1_rows(rng, n, d, cfg["alpha"])
        Af = A
    elif cfg["kind"] == "gkernel":
        return _kernel_problem(name, cfg, seed, n_test=0)[0]
    else:
        raise ValueError(cfg["kind"])

    # planted solution and right-hand side (float64 on the host); Section 6.1 draws v* ~ N(0, I/d)
    x_star = rng.standard_normal((d, K))
    if cfg["kind"] == "ar1":
        x_star /= np.sqrt(d)
    if layout == "csr":
        mv, rmv = _csr_matvec(row_ptr, col, val, n, d)
        Ax = np.stack([mv(x_star[:, r]) for r in range(K)], axis=1)
    elif cfg["storage"] == "bf16":
        Ax = np.empty((n, K))
        step = max(1, (1 << 24) // d)
        for r0 in range(0, n, step):
            r1 = min(n, r0 + step)
            Ax[r0:r1] = bf16_bits_to_f32(A[r0:r1]).astype(np.float64) @ x_star
    else:
        Ax = Af.astype(np.float64) @ x_star
    if "sigma" in cfg:
        B = Ax + cfg["sigma"] * rng.standard_normal((n, K))
    elif "noise" in cfg:
        B = Ax + cfg["noise"] * rng.standard_normal((n, K))
    else:
        E = rng.standard_normal((n, K))
        E *= cfg["noise_rel"] * np.linalg.norm(Ax) / np.linalg.norm(E)
        B = Ax + E

    # lambda range scale ||A||_2^2
    if cfg["kind"] == "haar":
        norm2_sq = 1.0                                   # sigma_1 = 1 by construction
    elif layout == "csr":
        mv, rmv = _csr_matvec(row_ptr, col, val, n, d)
        norm2_sq = spectral_norm_sq(mv, rmv, d, 60, seed)
    elif cfg["storage"] == "bf16":
        A32 = bf16_bits_to_f32(A)
        norm2_sq = spectral_norm_sq(lambda v: A32 @ v.astype(np.float32),
                                    lambda w: A32.T @ w.astype(np.float32), d, 30, seed)
        del A32
    else:
        A64 = A.astype(np.float64)
        norm2_sq = spectral_norm_sq(lambda v: A64 @ v, lambda w: A64.T @ w, d,
                                    200 if n * d <= (1 << 24) else 40, seed)
    if "lrange_abs" in cfg:  # the paper's absolute lambda range
        lmin, lmax = cfg["lrange_abs"]
    else:
        lmin, lmax = cfg["lrange"][0] * norm2_sq, cfg["lrange"][1] * norm2_sq
    lambdas = lambda_grid(lmin, lmax, cfg["T"])
    p = Problem(name=name, n=n, d=d, K=K, layout=layout, storage=cfg["storage"], A=A,
                row_ptr=row_ptr, col_idx=col, val=val, B=B, x_star=x_star, sketch=cfg["sketch"],
                m=cfg["m"], s=cfg["s"], sketch_seed=seed, lambda_min=lmin, lambda_max=lmax,
                lambdas=lambdas, norm2_sq=norm2_sq)
    if cpath:
        np.savez(cpath, **{f.name: getattr(p, f.name) for f in dataclasses.fields(p)
                           if f.name not in ("name", "layout", "storage", "sketch")
                           and getattr(p, f.name) is not None})
    return p


def _kernel_problem(name, cfg, seed, n_test):
    """Kernel ridge regression data: n training and n_test test feature vectors with labels;
    A = k(train, train) (n x n), A_test = k(test, train), B / B_test one-hot (K classes)."""
    rng = np.random.default_rng(seed)
    n, K = cfg["n"], cfg["K"]
    f, y = _kernel_features(rng, n + n_test, cfg["p"], K)
    A = _gauss_kernel(f[:n], f[:n], cfg["h"])
    onehot = np.eye(K)[y]
    A64 = A.astype(np.float64)
    norm2_sq = spectral_norm_sq(lambda v: A64 @ v, lambda w: A64.T @ w, n, 40, seed)
    lmin, lmax = cfg["lrange_abs"]
    p = Problem(name=name, n=n, d=n, K=K, layout="dense", storage=cfg["storage"], A=A, row_ptr=None,
                col_idx=None, val=None, B=np.ascontiguousarray(onehot[:n]), x_star=np.zeros((n, K)),
                sketch=cfg["sketch"], m=cfg["m"], s=cfg["s"], sketch_seed=seed, lambda_min=lmin,
                lambda_max=lmax, lambdas=lambda_grid(lmin, lmax, cfg["T"]), norm2_sq=norm2_sq)
    if n_test == 0:
        return p, None, None
    return p, _gauss_kernel(f[n:], f[:n], cfg["h"]), np.ascontiguousarray(onehot[n:])


def make_split(name: str, n_test: int, seed: int = 0, **overrides):
    """A held-out split as in Section 6 (part of the data kept as the test set): the workload is drawn
    with n + n_test rows from one model and split by rows.  Returns (train Problem, A_test, B_test):
    A_test dense (n_test x d, the training problem's storage type; CSR test rows are densified),
    B_test (n_test x K) float64."""
    if CONFIGS[name]["kind"] == "gkernel":  # test rows: the kernel between new points and the training points
        cfg = dict(CONFIGS[name])
        cfg.update(overrides)
        cfg["d"] = cfg["n"]
        return _kernel_problem(name, cfg, seed, n_test)
    n = overrides.pop("n", CONFIGS[name]["n"])
    full = make_problem(name, seed=seed, n=n + n_test, **overrides)
    B_test = np.ascontiguousarray(full.B[n:])
    if full.layout == "csr":
        e0, e1 = int(full.row_ptr[n]), int(full.row_ptr[-1])
        A_test = np.zeros((n_test, full.d), dtype=full.val.dtype)
        rows = np.repeat(np.arange(n_test), np.diff(full.row_ptr[n:]))
        A_test[rows, full.col_idx[e0:e1]] = full.val[e0:e1]
        train = dataclasses.replace(full, n=n, row_ptr=np.ascontiguousarray(full.row_ptr[:n + 1]),
                                    col_idx=np.ascontiguousarray(full.col_idx[:e0]),
                                    val=np.ascontiguousarray(full.val[:e0]), B=np.ascontiguousarray(full.B[:n]))
    else:
        A_test = np.ascontiguousarray(full.A[n:])
        train = dataclasses.replace(full, n=n, A=np.ascontiguousarray(full.A[:n]), B=np.ascontiguousarray(full.B[:n]))
    return train, A_test, B_test


def _from_cached(name, cfg, z) -> Problem:
    layout = "csr" if cfg["kind"] == "csr" else "dense"

    def g(f):
        return z.get(f)
    return Problem(name=name, n=int(z["n"]), d=int(z["d"]), K=int(z["K"]), layout=layout,
                   storage=cfg["storage"], A=g("A"), row_ptr=g("row_ptr"), col_idx=g("col_idx"),
                   val=g("val"), B=z["B"], x_star=z["x_star"], sketch=cfg["sketch"],
                   m=int(z["m"]), s=int(z["s"]), sketch_seed=int(z["sketch_seed"]),
                   lambda_min=float(z["lambda_min"]), lambda_max=float(z["lambda_max"]),
                   lambdas=z["lambdas"], norm2_sq=float(z["norm2_sq"]))


def serving_requests(count: int = 4096, rate_per_s: float = 2000.0, seed: int = 0,
                     n_range=(4096, 65536), d_range=(64, 1024), T_range=(20, 500)):
    """Request shapes and Poisson arrival times for the serving workload.

    Returns a list of dicts: arrival_s, n, d, T, layout ("dense"|"csr"), seed (= request index).
    """
    rng = np.random.default_rng(seed + 104729)
    gaps = rng.exponential(1.0 / rate_per_s, size=count)
    t = np.cumsum(gaps) - gaps[0]
    out = []
    for r in range(count):
        out.append(dict(arrival_s=float(t[r]),
                        n=int(rng.integers(n_range[0], n_range[1] + 1)),
                        d=int(rng.integers(d_range[0], d_range[1] + 1)),
                        T=int(rng.integers(T_range[0], T_range[1] + 1)),
                        layout="dense" if rng.random() < 0.5 else "csr",
                        seed=r))
    return out
