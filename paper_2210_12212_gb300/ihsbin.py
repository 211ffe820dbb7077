"""ctypes binding of libihsbin (include/ihsbin.h): argument marshalling only.

Every computation happens in the CUDA library; this module converts Python
arguments (numpy arrays, torch tensors, integers) into the C ABI's plain
pointers and sizes and turns non-zero statuses into exceptions.  Loading
fails loudly when the in-tree library has not been built: there is no other
code path.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libihsbin.so")

# ---- enums (mirror include/ihsbin.h)
OK, ERR_INVALID_ARG, ERR_OUT_OF_MEMORY, ERR_CUDA, ERR_NOT_SPD, ERR_LAMBDA_RANGE, ERR_STATE, \
    ERR_TIMEOUT, ERR_ADMISSION, ERR_UNSUPPORTED = range(10)
ERR_NAN = 11
F64, F32, BF16, TF32 = 0, 1, 2, 3
COMPUTE_F64, COMPUTE_F32X2 = 0, 1
DENSE, CSR = 0, 1
SK_GAUSSIAN, SK_SRHT, SK_COUNTSKETCH = 0, 1, 2
PRODUCT_AUTO, PRODUCT_GRAM, PRODUCT_ASPACE = 0, 1, 2

SKETCH_KIND = {"gaussian": SK_GAUSSIAN, "srht": SK_SRHT, "countsketch": SK_COUNTSKETCH}
DTYPE = {"f64": F64, "f32": F32, "bf16": BF16, "tf32": TF32}
SKETCH_APPLY = {"auto": 0, "tensor": 1, "fma": 2}
COMPUTE = {"f64": COMPUTE_F64, "f32x2": COMPUTE_F32X2}
PRODUCT = {"auto": PRODUCT_AUTO, "gram": PRODUCT_GRAM, "aspace": PRODUCT_ASPACE}
GRAM_AUTO, GRAM_SLICES, GRAM_FMA = 0, 1, 2
GRAM = {"auto": GRAM_AUTO, "slices": GRAM_SLICES, "fma": GRAM_FMA}
LOOP = {"auto": 0, "slices": 1, "fma": 2}
FACTOR = {"auto": 0, "slices": 1, "fma": 2}
FORM = {"auto": 0, "residual": 1, "increment": 2}


class IhsbinError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"ihsbin status {status}: {msg}")
        self.status = status


class Matrix(C.Structure):
    _fields_ = [("n", C.c_int64), ("d", C.c_int64), ("layout", C.c_int), ("dtype", C.c_int),
                ("values", C.c_void_p), ("ld", C.c_int64), ("row_ptr", C.c_void_p),
                ("col_idx", C.c_void_p), ("nnz", C.c_int64), ("on_device", C.c_int)]


class SketchDesc(C.Structure):
    _fields_ = [("kind", C.c_int), ("m", C.c_int64), ("s", C.c_int32), ("seed", C.c_uint64), ("entries", C.c_int),
                ("apply", C.c_int)]


class PathDesc(C.Structure):
    _fields_ = [("lambda_min", C.c_double), ("lambda_max", C.c_double), ("L", C.c_int32),
                ("k", C.c_void_p), ("k_default", C.c_int32), ("rho1", C.c_void_p),
                ("rho2", C.c_void_p), ("rho", C.c_double), ("jmax", C.c_int32),
                ("compute", C.c_int), ("product", C.c_int), ("eps", C.c_double), ("auto_rho", C.c_int32),
                ("gram", C.c_int), ("loop", C.c_int), ("factor", C.c_int), ("sigma_d2", C.c_double),
                ("tau", C.c_void_p), ("slice_weight", C.c_int32), ("form", C.c_int32),
                ("precond_weight", C.c_int32)]


class AdaptiveDesc(C.Structure):
    _fields_ = [("sketch", SketchDesc), ("lam", C.c_double), ("eps", C.c_double), ("gamma1", C.c_double),
                ("gamma2", C.c_double), ("gamma3", C.c_double), ("max_iter", C.c_int32), ("m_max", C.c_int64),
                ("compute", C.c_int)]


class AdaptiveResult(C.Structure):
    _fields_ = [("m", C.c_int64), ("iterations", C.c_int32), ("doublings", C.c_int32), ("delta0", C.c_double),
                ("delta", C.c_double)]


class Request(C.Structure):
    _fields_ = [("A", Matrix), ("B", C.c_void_p), ("K", C.c_int64), ("ldb", C.c_int64), ("b_dtype", C.c_int),
                ("b_on_device", C.c_int), ("sketch", SketchDesc), ("path", PathDesc), ("lambdas", C.c_void_p),
                ("T", C.c_int64), ("X", C.c_void_p), ("x_dtype", C.c_int), ("x_on_device", C.c_int)]


class ServeConfig(C.Structure):
    _fields_ = [("slots", C.c_int32), ("hbm_budget_bytes", C.c_uint64)]


_lib = None

EXPORTED = [
    "ihsbin_ctx_create", "ihsbin_ctx_destroy", "ihsbin_ctx_memory", "ihsbin_last_error",
    "ihsbin_problem_create", "ihsbin_problem_destroy", "ihsbin_sketch", "ihsbin_sketch_export",
    "ihsbin_sketch_matrix_export", "ihsbin_build_basis", "ihsbin_plan_export", "ihsbin_basis_export",
    "ihsbin_eval_path", "ihsbin_phase_times", "ihsbin_set_timing", "ihsbin_reset_stats",
    "ihsbin_kernel_stats", "ihsbin_sketch_gram_noalloc", "ihsbin_request_footprint", "ihsbin_serve_create",
    "ihsbin_serve_submit", "ihsbin_serve_wait", "ihsbin_serve_destroy", "ihsbin_serve", "ihsbin_gram_export",
    "ihsbin_path_losses", "ihsbin_adaptive_sketch", "ihsbin_sketch_entries_export", "ihsbin_kernel_exec",
    "ihsbin_ctx_fail_allocations", "ihsbin_tuning_report", "ihsbin_tuning_reset", "ihsbin_recursion_form",
]
KCAT_COUNT = 40


def load(path: Optional[str] = None):
    """Load the in-tree library (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"libihsbin not built ({path} missing): run "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(path)
    vp, i64, i32, dbl = C.c_void_p, C.c_int64, C.c_int32, C.c_double
    sig = {
        "ihsbin_ctx_create": [C.c_int, C.c_uint64, C.POINTER(vp)],
        "ihsbin_ctx_destroy": [vp],
        "ihsbin_ctx_memory": [vp, C.POINTER(C.c_uint64)],
        "ihsbin_problem_create": [vp, C.POINTER(Matrix), vp, i64, i64, C.c_int, C.c_int, C.POINTER(vp)],
        "ihsbin_problem_destroy": [vp],
        "ihsbin_sketch": [vp, C.POINTER(SketchDesc), vp],
        "ihsbin_sketch_export": [vp, vp, vp, i64, C.POINTER(i64)],
        "ihsbin_sketch_matrix_export": [vp, vp, vp],
        "ihsbin_sketch_entries_export": [vp, i64, i64, i64, i64, vp],
        "ihsbin_build_basis": [vp, C.POINTER(PathDesc), vp],
        "ihsbin_plan_export": [vp, vp, vp, vp, vp, vp, i32, C.POINTER(i32)],
        "ihsbin_basis_export": [vp, i32, vp, i64, C.POINTER(i64)],
        "ihsbin_eval_path": [vp, vp, i64, vp, C.c_int, C.c_int, vp],
        "ihsbin_phase_times": [vp, vp],
        "ihsbin_set_timing": [vp, C.c_int],
        "ihsbin_reset_stats": [vp],
        "ihsbin_kernel_stats": [vp, i32, vp, vp, vp, vp, vp],
        "ihsbin_kernel_exec": [vp, i32, vp, vp],
        "ihsbin_ctx_fail_allocations": [vp, i64],
        "ihsbin_tuning_report": [vp, i64, C.POINTER(i64)],
        "ihsbin_tuning_reset": [],
        "ihsbin_recursion_form": [vp, C.POINTER(i32), C.POINTER(i32)],
        "ihsbin_sketch_gram_noalloc": [vp, i64, i64, vp, vp],
        "ihsbin_request_footprint": [C.POINTER(Request), C.POINTER(C.c_uint64)],
        "ihsbin_serve_create": [vp, C.POINTER(ServeConfig), C.POINTER(vp)],
        "ihsbin_serve_submit": [vp, C.POINTER(Request), C.POINTER(C.c_uint64)],
        "ihsbin_serve_wait": [vp, C.c_uint64, i64, C.POINTER(C.c_int), vp],
        "ihsbin_serve_destroy": [vp],
        "ihsbin_serve": [vp, C.POINTER(ServeConfig), vp, i64, vp, vp, vp],
        "ihsbin_gram_export": [vp, vp],
        "ihsbin_path_losses": [vp, vp, i64, C.POINTER(Matrix), vp, i64, C.c_int, C.c_int, vp, vp, vp],
        "ihsbin_adaptive_sketch": [vp, C.POINTER(AdaptiveDesc), C.POINTER(AdaptiveResult), vp, vp, vp, i32, vp, vp],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = C.c_int
    lib.ihsbin_last_error.argtypes = []
    lib.ihsbin_last_error.restype = C.c_char_p
    _lib = lib
    return lib


def _check(status: int):
    if status != OK:
        raise IhsbinError(status, _lib.ihsbin_last_error().decode())


def _ptr(a) -> int:
    """Address of a numpy array or torch tensor (0 for None)."""
    if a is None:
        return 0
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def _on_device(a) -> int:
    return int(bool(getattr(a, "is_cuda", False)))


def _stream(stream) -> int:
    if stream is None:
        return 0
    return int(getattr(stream, "cuda_stream", stream))


class Context:
    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        load()
        h = C.c_void_p()
        _check(_lib.ihsbin_ctx_create(device, hbm_budget_bytes, C.byref(h)))
        self.h = h

    def memory(self) -> int:
        v = C.c_uint64()
        _check(_lib.ihsbin_ctx_memory(self.h, C.byref(v)))
        return v.value

    def fail_allocations(self, after: int):
        """Test hook: after `after` more successful device allocations every one fails (< 0: off)."""
        _check(_lib.ihsbin_ctx_fail_allocations(self.h, after))

    def close(self):
        if self.h:
            _check(_lib.ihsbin_ctx_destroy(self.h))
            self.h = None


class Problem:
    """A problem handle: ihsbin_problem_create / _sketch / _build_basis / _eval_path."""

    def __init__(self, ctx: Context, A=None, B=None, *, dtype: str = "f64", csr=None, shape=None):
        """A: dense (n x d) numpy array or CUDA tensor, or csr=(row_ptr, col_idx, values) with shape=(n, d).
        B: (n,) or (n x K) numpy array (float64/float32) or CUDA tensor."""
        self.ctx = ctx
        m = Matrix()
        self._keep = []
        if csr is not None:
            rp, ci, val = csr
            n, d = shape
            m.n, m.d, m.layout, m.dtype = n, d, CSR, DTYPE[dtype]
            m.values, m.row_ptr, m.col_idx, m.nnz = _ptr(val), _ptr(rp), _ptr(ci), int(len(ci))
            m.ld = 0
            m.on_device = _on_device(val)
            self._keep += [rp, ci, val]
        else:
            n, d = A.shape
            m.n, m.d, m.layout, m.dtype = n, d, DENSE, DTYPE[dtype]
            m.values = _ptr(A)
            m.ld = A.stride(0) if hasattr(A, "stride") and callable(A.stride) else A.strides[0] // A.itemsize
            m.on_device = _on_device(A)
            self._keep.append(A)
        if B.ndim == 1:
            B = B.reshape(-1, 1)
        K = B.shape[1]
        if hasattr(B, "is_cuda"):
            bdt = F64 if str(B.dtype) == "torch.float64" else F32
            ldb = B.stride(0)
        else:
            B = np.ascontiguousarray(B)
            bdt = F64 if B.dtype == np.float64 else F32
            ldb = B.shape[1]
        self._keep.append(B)
        h = C.c_void_p()
        _check(_lib.ihsbin_problem_create(ctx.h, C.byref(m), _ptr(B), K, ldb, bdt, _on_device(B),
                                          C.byref(h)))
        self.h = h
        self.n, self.d, self.K = n, d, K

    # -- hot path -------------------------------------------------------------------------
    def sketch(self, kind: str, m: int, s: int = 1, seed: int = 0, entries: str = "f64", apply: str = "auto",
               stream=None):
        sd = SketchDesc(SKETCH_KIND[kind], m, s, seed, DTYPE[entries], SKETCH_APPLY[apply])
        _check(_lib.ihsbin_sketch(self.h, C.byref(sd), _stream(stream)))

    def build_basis(self, lambda_min: float, lambda_max: float, *, L: int = 0,
                    k: Optional[Sequence[int]] = None, k_default: int = 20,
                    rho1: Optional[Sequence[float]] = None, rho2: Optional[Sequence[float]] = None,
                    rho: float = 0.0, jmax: int = 0, compute: str = "f64", product: str = "auto",
                    eps: float = 0.0, auto_rho: bool = False, gram: str = "auto", loop: str = "auto",
                    factor: str = "auto", sigma_d2: float = 0.0, tau: Optional[Sequence[float]] = None,
                    slice_weight: int = 0, form: str = "auto", precond_weight: int = 0, stream=None):
        """k=None with k_default <= 0 selects Theorem 4's k for `eps`; auto_rho takes rho from the sketch;
        gram / loop / factor select the Gram kernel, the recursion's product kernel and the inverse's
        product kernel ("auto", "slices" = tensor-core exact slices, "fma" = CUDA cores); form selects
        how the tensor-core recursion carries the basis ("auto", "residual", "increment") and
        precond_weight the slice pairs of the residual form's P_l r (0 = from the conditioning bound)."""
        pd = PathDesc()
        pd.lambda_min, pd.lambda_max, pd.L = lambda_min, lambda_max, L
        ka = np.ascontiguousarray(k, dtype=np.int32) if k is not None else None
        r1 = np.ascontiguousarray(rho1, dtype=np.float64) if rho1 is not None else None
        r2 = np.ascontiguousarray(rho2, dtype=np.float64) if rho2 is not None else None
        pd.k = _ptr(ka)
        pd.k_default = k_default
        pd.rho1, pd.rho2 = _ptr(r1), _ptr(r2)
        pd.rho, pd.jmax = rho, jmax
        pd.compute, pd.product = COMPUTE[compute], PRODUCT[product]
        pd.eps, pd.auto_rho = eps, int(auto_rho)
        pd.gram = GRAM[gram]
        pd.loop = LOOP[loop]
        pd.factor = FACTOR[factor]
        pd.sigma_d2 = sigma_d2
        ta = np.ascontiguousarray(tau, dtype=np.float64) if tau is not None else None
        pd.tau = _ptr(ta)
        pd.slice_weight = slice_weight
        pd.form = FORM[form]
        pd.precond_weight = precond_weight
        _check(_lib.ihsbin_build_basis(self.h, C.byref(pd), _stream(stream)))

    def recursion_form(self):
        """(form, precond_weight) the last build ran with: form "residual" or "increment"."""
        f, w = C.c_int32(), C.c_int32()
        _check(_lib.ihsbin_recursion_form(self.h, C.byref(f), C.byref(w)))
        return {v: k for k, v in FORM.items() if k != "auto"}[f.value], w.value

    def adaptive_sketch(self, kind: str, m0: int, lam: float, *, s: int = 1, seed: int = 0, entries: str = "f64",
                        eps: float = 0.0, gamma1: float = 0.0, gamma2: float = 0.0, gamma3: float = 0.0,
                        max_iter: int = 0, m_max: int = 0, compute: str = "f32x2", trace_cap: int = 256,
                        want_x: bool = False, apply: str = "auto", stream=None):
        """Algorithm 4: returns dict(m, iterations, doublings, delta0, delta, deltas, ms, steps[, x]);
        the problem is left sketched with the final m."""
        sd = SketchDesc(SKETCH_KIND[kind], m0, s, seed, DTYPE[entries], SKETCH_APPLY[apply])
        ad = AdaptiveDesc(sd, lam, eps, gamma1, gamma2, gamma3, max_iter, m_max, COMPUTE[compute])
        res = AdaptiveResult()
        dl = np.zeros(trace_cap)
        ms = np.zeros(trace_cap, dtype=np.int64)
        st = np.zeros(trace_cap)
        D = min(self.n, self.d)
        x = np.empty((D, self.K)) if want_x else None
        _check(_lib.ihsbin_adaptive_sketch(self.h, C.byref(ad), C.byref(res), _ptr(dl), _ptr(ms), _ptr(st),
                                           trace_cap, _ptr(x), _stream(stream)))
        it = res.iterations
        out = dict(m=res.m, iterations=it, doublings=res.doublings, delta0=res.delta0, delta=res.delta,
                   deltas=dl[:min(it + 1, trace_cap)].copy(), ms=ms[:min(it + 1, trace_cap)].copy(),
                   steps=st[:min(it, trace_cap)].copy())
        if want_x:
            out["x"] = x
        return out

    def eval_path(self, lambdas, out=None, x_dtype: str = "f64", stream=None):
        """Returns X (T x d x K) as a numpy array, or fills `out` (a CUDA tensor) in place."""
        lam = np.ascontiguousarray(lambdas, dtype=np.float64)
        T = lam.shape[0]
        if out is None:
            out = np.empty((T, self.d, self.K), dtype=np.float64 if x_dtype == "f64" else np.float32)
            on_dev = 0
        else:
            on_dev = _on_device(out)
        _check(_lib.ihsbin_eval_path(self.h, _ptr(lam), T, _ptr(out), DTYPE[x_dtype], on_dev,
                                     _stream(stream)))
        return out

    def path_losses(self, lambdas, A_test=None, B_test=None, *, test_dtype: Optional[str] = None,
                    train: bool = True, stream=None):
        """Section 6.1's losses without forming X: (train, test) arrays of T doubles (either None
        when not asked for).  A_test: dense n_test x d numpy array or CUDA tensor (element type
        `test_dtype`, default the array's own); B_test: (n_test,) or (n_test x K)."""
        lam = np.ascontiguousarray(lambdas, dtype=np.float64)
        T = lam.shape[0]
        tr = np.empty(T) if train else None
        te = None
        keep = []
        mref, bptr, ldb, bdt, bdev = None, None, 0, F64, 0
        if A_test is not None:
            if test_dtype is None:
                test_dtype = {"float64": "f64", "float32": "f32", "torch.float64": "f64",
                              "torch.float32": "f32", "torch.bfloat16": "bf16"}[str(A_test.dtype)]
            m = _matrix(A_test, dtype=test_dtype, keep=keep)
            mref = C.byref(m)
            if B_test.ndim == 1:
                B_test = B_test.reshape(-1, 1)
            if hasattr(B_test, "is_cuda"):
                bdt = F64 if str(B_test.dtype) == "torch.float64" else F32
                ldb = B_test.stride(0)
            else:
                B_test = np.ascontiguousarray(B_test)
                bdt = F64 if B_test.dtype == np.float64 else F32
                ldb = B_test.shape[1]
            keep.append(B_test)
            bptr, bdev = _ptr(B_test), _on_device(B_test)
            te = np.empty(T)
        _check(_lib.ihsbin_path_losses(self.h, _ptr(lam), T, mref, bptr, ldb, bdt, bdev, _ptr(tr), _ptr(te),
                                       _stream(stream)))
        return tr, te

    # -- exports ---------------------------------------------------------------------------
    def sketch_export(self, cap: int):
        idx = np.empty(cap, dtype=np.int64)
        sign = np.empty(cap, dtype=np.int8)
        cnt = C.c_int64()
        _check(_lib.ihsbin_sketch_export(self.h, _ptr(idx), _ptr(sign), cap, C.byref(cnt)))
        return idx, sign, cnt.value

    def sketch_entries(self, row0: int, nrows: int, col0: int, ncols: int):
        """BF16 bits (uint16, nrows x ncols) of a window of the Gaussian sketch with BF16 entries."""
        out = np.empty((nrows, ncols), dtype=np.uint16)
        _check(_lib.ihsbin_sketch_entries_export(self.h, row0, nrows, col0, ncols, _ptr(out)))
        return out

    def sketch_matrices(self, m: int, D: int):
        SA = np.empty((m, D))
        GS = np.empty((D, D))
        _check(_lib.ihsbin_sketch_matrix_export(self.h, _ptr(SA), _ptr(GS)))
        return SA, GS

    def gram(self):
        """G = A_hat^T A_hat (D x D, FP64) as built by the last build_basis (Gram product mode)."""
        D = min(self.n, self.d)
        G = np.empty((D, D))
        _check(_lib.ihsbin_gram_export(self.h, _ptr(G)))
        return G

    def plan(self):
        Lv = C.c_int32()
        _check(_lib.ihsbin_plan_export(self.h, None, None, None, None, None, 0, C.byref(Lv)))
        L = Lv.value
        edges = np.empty(L + 1)
        lam0, tau = np.empty(L), np.empty(L)
        k, jc = np.empty(L, np.int32), np.empty(L, np.int32)
        _check(_lib.ihsbin_plan_export(self.h, _ptr(edges), _ptr(lam0), _ptr(tau), _ptr(k), _ptr(jc),
                                       L + 1, C.byref(Lv)))
        return dict(L=L, edges=edges, lam0=lam0, tau=tau, k=k, jcount=jc)

    def plan_dict_for_oracle(self):
        """The library's plan as (L, rho1, rho2, k) arrays, for timing the oracle on the same plan."""
        p = self.plan()
        # tau = 2 lam0 / (lo/rho1 + hi/rho2): report rho via the oracle-compatible fields the library used
        return dict(L=p["L"], k=p["k"].tolist(), tau=p["tau"].tolist(), lam0=p["lam0"].tolist(),
                    edges=p["edges"].tolist())

    def basis(self, l: int, D: int):
        need = C.c_int64()
        _check(_lib.ihsbin_basis_export(self.h, l, None, 0, C.byref(need)))
        buf = np.empty(need.value)
        _check(_lib.ihsbin_basis_export(self.h, l, _ptr(buf), need.value, C.byref(need)))
        return buf.reshape(-1, self.K, D).transpose(0, 2, 1)   # (j, D, K)

    def phase_times(self):
        out = np.zeros(5, dtype=np.float32)
        _check(_lib.ihsbin_phase_times(self.h, _ptr(out)))
        return dict(zip(["sketch", "factor", "gram_rhs", "basis", "eval"], out.tolist()))

    def set_timing(self, enable: bool = True):
        _check(_lib.ihsbin_set_timing(self.h, int(enable)))

    def reset_stats(self):
        _check(_lib.ihsbin_reset_stats(self.h))

    def kernel_stats(self):
        """{category: (launches, ms, flops, bytes)} for every category with launches."""
        out = {}
        for cat in range(KCAT_COUNT):
            n, ms, fl, by = C.c_int64(), C.c_double(), C.c_double(), C.c_double()
            name = C.c_char_p()
            _check(_lib.ihsbin_kernel_stats(self.h, cat, C.byref(n), C.byref(ms), C.byref(fl), C.byref(by),
                                            C.byref(name)))
            if n.value:
                out[name.value.decode()] = (n.value, ms.value, fl.value, by.value)
        return out

    def kernel_exec(self):
        """{category: (executed flops, executed bytes)} for every category with launches."""
        out = {}
        for cat in range(KCAT_COUNT):
            n, xf, xb = C.c_int64(), C.c_double(), C.c_double()
            name = C.c_char_p()
            _check(_lib.ihsbin_kernel_stats(self.h, cat, C.byref(n), None, None, None, C.byref(name)))
            if n.value:
                _check(_lib.ihsbin_kernel_exec(self.h, cat, C.byref(xf), C.byref(xb)))
                out[name.value.decode()] = (xf.value, xb.value)
        return out

    def close(self):
        if getattr(self, "h", None):
            _check(_lib.ihsbin_problem_destroy(self.h))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --------------------------------------------------------------------------- serving
def tuning_report() -> str:
    """The autotuner's table: one line per tuned launch site and shape class."""
    need = C.c_int64()
    _check(_lib.ihsbin_tuning_report(None, 0, C.byref(need)))
    buf = C.create_string_buffer(max(1, need.value))
    _check(_lib.ihsbin_tuning_report(buf, need.value, C.byref(need)))
    return buf.value.decode()


def tuning_reset():
    _check(_lib.ihsbin_tuning_reset())


def _matrix(A=None, *, dtype="f32", csr=None, shape=None, keep=None):
    m = Matrix()
    if csr is not None:
        rp, ci, val = csr
        n, d = shape
        m.n, m.d, m.layout, m.dtype = n, d, CSR, DTYPE[dtype]
        m.values, m.row_ptr, m.col_idx, m.nnz = _ptr(val), _ptr(rp), _ptr(ci), int(len(ci))
        m.on_device = _on_device(val)
        keep += [rp, ci, val]
    else:
        n, d = A.shape
        m.n, m.d, m.layout, m.dtype = n, d, DENSE, DTYPE[dtype]
        m.values = _ptr(A)
        m.ld = A.stride(0) if hasattr(A, "stride") and callable(A.stride) else A.strides[0] // A.itemsize
        m.on_device = _on_device(A)
        keep.append(A)
    return m


def make_request(A=None, B=None, lambdas=None, *, dtype="f32", csr=None, shape=None, sketch="srht", m=None,
                 s=1, seed=0, lambda_min=None, lambda_max=None, L=0, k=None, k_default=0, eps=1e-7,
                 auto_rho=True, jmax=32, compute="f32x2", out=None, x_dtype="f64"):
    """Build an ihsbin_request (returns (request, keep-alive list, output array))."""
    keep = []
    req = Request()
    req.A = _matrix(A, dtype=dtype, csr=csr, shape=shape, keep=keep)
    n, d = req.A.n, req.A.d
    if B.ndim == 1:
        B = B.reshape(-1, 1)
    B = np.ascontiguousarray(B, dtype=np.float64)
    keep.append(B)
    req.B, req.K, req.ldb, req.b_dtype, req.b_on_device = _ptr(B), B.shape[1], B.shape[1], F64, 0
    req.sketch = SketchDesc(SKETCH_KIND[sketch], m if m else 2 * min(n, d), s, seed, F64)
    lam = np.ascontiguousarray(lambdas, dtype=np.float64)
    keep.append(lam)
    pd = PathDesc()
    pd.lambda_min = lambda_min if lambda_min is not None else float(lam.min())
    pd.lambda_max = lambda_max if lambda_max is not None else float(lam.max())
    pd.L = L
    ka = np.ascontiguousarray(k, dtype=np.int32) if k is not None else None
    keep.append(ka)
    pd.k, pd.k_default = _ptr(ka), k_default
    pd.jmax, pd.compute, pd.product, pd.eps, pd.auto_rho = jmax, COMPUTE[compute], PRODUCT_AUTO, eps, int(auto_rho)
    req.path = pd
    req.lambdas, req.T = _ptr(lam), lam.shape[0]
    if out is None:
        out = np.zeros((lam.shape[0], d, B.shape[1]), dtype=np.float64 if x_dtype == "f64" else np.float32)
    keep.append(out)
    req.X, req.x_dtype, req.x_on_device = _ptr(out), DTYPE[x_dtype], _on_device(out)
    return req, keep, out


def request_footprint(req) -> int:
    v = C.c_uint64()
    _check(_lib.ihsbin_request_footprint(C.byref(req), C.byref(v)))
    return v.value


class Server:
    """ihsbin_serve_create / _submit / _wait / _destroy."""

    def __init__(self, ctx: Context, slots: int = 4, hbm_budget_bytes: int = 0):
        load()
        cfg = ServeConfig(slots, hbm_budget_bytes)
        h = C.c_void_p()
        _check(_lib.ihsbin_serve_create(ctx.h, C.byref(cfg), C.byref(h)))
        self.h = h
        self._keep = {}

    def submit(self, req, keep) -> int:
        t = C.c_uint64()
        _check(_lib.ihsbin_serve_submit(self.h, C.byref(req), C.byref(t)))
        self._keep[t.value] = (req, keep)
        return t.value

    def wait(self, ticket: int, timeout_us: int = 60_000_000):
        """(request status, [queue_s, service_s, total_s, device_s]); raises IhsbinError(ERR_TIMEOUT)."""
        res = C.c_int()
        t4 = np.zeros(4)
        _check(_lib.ihsbin_serve_wait(self.h, ticket, timeout_us, C.byref(res), _ptr(t4)))
        self._keep.pop(ticket, None)
        return res.value, t4

    def close(self):
        if getattr(self, "h", None):
            _check(_lib.ihsbin_serve_destroy(self.h))
            self.h = None
