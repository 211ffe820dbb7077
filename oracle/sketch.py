"""Sketching matrices S (m x N) applied to the tall data matrix A_hat (N x D), in FP64.

Section 3 lists the sketch families; the entries are drawn from the Philox
stream layout documented in ``oracle/philox.py``.

* Gaussian (Section 3, first item): S_ij ~ N(0, 1/m).  z_ij by Box-Muller on
  the two uniforms (w0, w1) of counter index i*N + j on stream 5:
  z = sqrt(-2 ln u0) * cos(2 pi u1).
* CountSketch / SJLT (Section 3, items 2-3): s stacked CountSketches of m/s
  rows each.  Column i of S has, in block t, the value +-1/sqrt(s) at row
  t*(m/s) + h_t(i), with (w0, w1) = draw(index i*s + t, stream 3),
  h_t(i) = (w0 * (m/s)) >> 32 and sign -1 iff w1 is odd.  (The paper writes
  h(i) in {1..n}; the bucket range is the block height, and the 1/sqrt(s)
  scale makes E[S^T S] = I.)
* SRHT (Section 3, item 4, left undefined in the paper): S = (1/sqrt(m)) R H D
  on A_hat zero-padded to N_pad = 2^ceil(log2 N) rows; D_ii = -1 iff word w0
  of draw(i, stream 6) is odd; H is the unnormalised Sylvester-Hadamard
  matrix H_{r,i} = (-1)^popcount(r & i); R keeps the m rows r with the
  smallest 64-bit keys (w1 << 32 | w0) of draw(r, stream 7), ties to the lower
  index, listed in ascending r.  E[S^T S] = I.
"""
import math

import numpy as np

from . import philox


def gaussian_entries(m: int, N: int, seed: int, rows=None) -> np.ndarray:
    """Explicit Gaussian sketch rows (FP64), S[i, j] = z_ij / sqrt(m)."""
    rows = np.arange(m) if rows is None else np.asarray(rows)
    idx = (rows[:, None].astype(np.uint64) * np.uint64(N) + np.arange(N, dtype=np.uint64)[None, :])
    w0, w1, _, _ = philox.draw(seed, philox.STREAM_GAUSSIAN, idx)
    u0 = philox.uniform_open(w0)
    u1 = philox.uniform_open(w1)
    z = np.sqrt(-2.0 * np.log(u0)) * np.cos(2.0 * np.pi * u1)
    return z / math.sqrt(m)


def countsketch_map(N: int, m: int, s: int, seed: int):
    """(row index in S, sign) for every (input row i, block t): arrays of shape (N, s)."""
    if m % s:
        raise ValueError("m must be a multiple of s")
    mb = m // s
    idx = np.arange(N, dtype=np.uint64)[:, None] * np.uint64(s) + np.arange(s, dtype=np.uint64)
    w0, w1, _, _ = philox.draw(seed, philox.STREAM_COUNTSKETCH, idx)
    bucket = ((w0.astype(np.uint64) * np.uint64(mb)) >> np.uint64(32)).astype(np.int64)
    rows = bucket + (np.arange(s, dtype=np.int64) * mb)[None, :]
    sign = np.where((w1 & np.uint32(1)) == 1, -1.0, 1.0)
    return rows, sign


def srht_signs(N_pad: int, seed: int) -> np.ndarray:
    w0, _, _, _ = philox.draw(seed, philox.STREAM_SRHT_SIGN, np.arange(N_pad, dtype=np.uint64))
    return np.where((w0 & np.uint32(1)) == 1, -1.0, 1.0)


def srht_rows(N_pad: int, m: int, seed: int) -> np.ndarray:
    """Indices of the m rows of H kept by R: smallest keys, ties to the lower index, ascending."""
    w0, w1, _, _ = philox.draw(seed, philox.STREAM_SRHT_KEY, np.arange(N_pad, dtype=np.uint64))
    key = (w1.astype(np.uint64) << np.uint64(32)) | w0.astype(np.uint64)
    order = np.lexsort((np.arange(N_pad), key))        # by key, then by index
    return np.sort(order[:m])


def next_pow2(N: int) -> int:
    return 1 << max(0, (N - 1).bit_length())


def fwht_rows(X: np.ndarray) -> np.ndarray:
    """Unnormalised Walsh-Hadamard transform along axis 0 (length a power of two): returns H X."""
    X = np.array(X, dtype=np.float64, copy=True)
    N = X.shape[0]
    h = 1
    while h < N:
        Y = X.reshape(N // (2 * h), 2, h, -1)
        a = Y[:, 0].copy()
        b = Y[:, 1].copy()
        Y[:, 0] = a + b
        Y[:, 1] = a - b
        X = Y.reshape(X.shape)
        h *= 2
    return X


def _gaussian_rows(args):
    """Rows [r0, r1) of S (BF16-rounded when asked), for a worker process."""
    m, N, seed, r0, r1, bf16_entries = args
    S = gaussian_entries(m, N, seed, rows=np.arange(r0, r1))
    return _round_bf16(S).astype(np.float32) if bf16_entries else S


def apply_gaussian(Ahat: np.ndarray, m: int, seed: int, bf16_entries: bool = False,
                   block: int = 512, workers: int = 0) -> np.ndarray:
    """SA for the Gaussian sketch; S is generated in row blocks (never all at once).

    workers > 1 draws the row blocks in that many spawned processes (BF16 entries travel as
    float32, which holds them exactly); each block's product is the same as in the serial loop."""
    N, D = Ahat.shape
    out = np.empty((m, D))
    jobs = [(m, N, seed, r0, min(m, r0 + block), bf16_entries) for r0 in range(0, m, block)]
    if workers > 1:
        import concurrent.futures as cf
        import multiprocessing as mp
        with cf.ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
            for job, S in zip(jobs, ex.map(_gaussian_rows, jobs)):
                out[job[3]:job[4]] = S.astype(np.float64) @ Ahat
        return out
    for job in jobs:
        out[job[3]:job[4]] = _gaussian_rows(job).astype(np.float64) @ Ahat
    return out


def apply_countsketch(Ahat, m: int, s: int, seed: int) -> np.ndarray:
    """SA for CountSketch (s = 1) / SJLT (s > 1).  Ahat: dense (N x D) array or scipy CSR."""
    N, D = Ahat.shape
    rows, sign = countsketch_map(N, m, s, seed)
    out = np.zeros((m, D))
    scale = 1.0 / math.sqrt(s)
    if hasattr(Ahat, "tocsr"):
        import scipy.sparse as sp
        S = sp.csr_matrix((np.repeat(sign.ravel() * scale, 1), (rows.ravel(),
                           np.repeat(np.arange(N), s))), shape=(m, N))
        return np.asarray((S @ Ahat).todense())
    for t in range(s):
        np.add.at(out, rows[:, t], (sign[:, t] * scale)[:, None] * Ahat)
    return out


def apply_srht(Ahat: np.ndarray, m: int, seed: int) -> np.ndarray:
    N, D = Ahat.shape
    N_pad = next_pow2(N)
    X = np.zeros((N_pad, D))
    X[:N] = Ahat
    X *= srht_signs(N_pad, seed)[:, None]
    HX = fwht_rows(X)
    return HX[srht_rows(N_pad, m, seed)] / math.sqrt(m)


def _round_bf16(x: np.ndarray) -> np.ndarray:
    f = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32)
    r = ((f + np.uint32(0x7FFF) + ((f >> np.uint32(16)) & np.uint32(1))) >> np.uint32(16))
    return (r.astype(np.uint32) << np.uint32(16)).view(np.float32).astype(np.float64)


def apply(kind: str, Ahat, m: int, s: int, seed: int, bf16_entries: bool = False, workers: int = 0) -> np.ndarray:
    if kind == "gaussian":
        dense = Ahat.toarray() if hasattr(Ahat, "toarray") else Ahat
        return apply_gaussian(dense, m, seed, bf16_entries, block=128 if workers > 1 else 512, workers=workers)
    if kind == "countsketch":
        return apply_countsketch(Ahat, m, s, seed)
    if kind == "srht":
        dense = Ahat.toarray() if hasattr(Ahat, "toarray") else Ahat
        return apply_srht(dense, m, seed)
    raise ValueError(kind)
