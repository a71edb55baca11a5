"""Python binding of the C ABI in include/tucker_gb300.h (ctypes).

Argument marshalling only: every step of the computation runs in the CUDA
library libtucker_gb300.so.  Device memory and streams come from PyTorch;
tensors are passed as raw device pointers.  If the library has not been
built, every call raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtucker_gb300.so")
MAX_MODES = 8

STATUS = {0: "OK", 1: "INVALID", 2: "OOM", 3: "NONFINITE", 4: "EIG_NOCONV", 5: "CUDA",
          6: "UNSUPPORTED"}
F32, F64 = 0, 1
PREC = {"fp64": 0, "fp32": 1, "mixed": 2, "tensor": 3}
OPT_TIMING, OPT_MAX_SWEEPS, OPT_JACOBI_TOL, OPT_EIG_SOLVER = 1, 2, 3, 4
OPT_BARRIER_POLLS, OPT_MEM_LIMIT, OPT_GRAM_DIGITS, OPT_AUTOTUNE = 5, 6, 7, 8
OPT_HOST_CHUNK = 9
EIG_SOLVER = {"auto": 0, "jacobi": 1, "tridiag": 2}

EXPORTS = ["tucker_create", "tucker_destroy", "tucker_last_error", "tucker_set_option",
           "tucker_sthosvd", "tucker_sthosvd_batched", "tucker_result_destroy",
           "tucker_reconstruct",
           "tucker_multi_ttm", "tucker_ttm_order", "tucker_norm_sq", "tucker_gram",
           "tucker_eig", "tucker_eig_trunc", "tucker_rank_cut", "tucker_ttm",
           "tucker_kernel_launches", "tucker_gram_noalloc", "tucker_hosvd",
           "tucker_sthosvd_order", "tucker_slice_stats", "tucker_slice_transform",
           "tucker_preprocess", "tucker_selftest_rcp64", "tucker_autotune_entries",
           "tucker_sthosvd_host"]
STATS = ("mean", "std", "max", "min", "norm1", "norm2")
PRE_METHOD = {"standardize": 0, "max": 1}


class TuckerError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status
        self.name = STATUS.get(status, str(status))


class CResult(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int),
        ("core_dtype", ctypes.c_int),
        ("dims", ctypes.c_int64 * MAX_MODES),
        ("ranks", ctypes.c_int64 * MAX_MODES),
        ("mode_order", ctypes.c_int * MAX_MODES),
        ("core", ctypes.c_void_p),
        ("factors", ctypes.c_void_p * MAX_MODES),
        ("eigvals", ctypes.c_void_p * MAX_MODES),
        ("norm_x_sq", ctypes.c_double),
        ("threshold", ctypes.c_double),
        ("discarded_sq", ctypes.c_double * MAX_MODES),
        ("jacobi_sweeps", ctypes.c_int * MAX_MODES),
        ("gram_kernel", ctypes.c_int * MAX_MODES),
        ("ttm_kernel", ctypes.c_int * MAX_MODES),
        ("eig_kernel", ctypes.c_int * MAX_MODES),
        ("ms_norm", ctypes.c_float),
        ("ms_gram", ctypes.c_float * MAX_MODES),
        ("ms_eig", ctypes.c_float * MAX_MODES),
        ("ms_ttm", ctypes.c_float * MAX_MODES),
        ("ms_total", ctypes.c_float),
    ]


_lib = None


def lib():
    """The loaded CUDA library (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library missing: {LIB_PATH} (run __graft_entry__.build())")
        L = ctypes.CDLL(LIB_PATH)
        vp, i64p, c_int = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.c_int
        L.tucker_create.argtypes = [ctypes.POINTER(vp), vp]
        L.tucker_destroy.argtypes = [vp]
        L.tucker_last_error.argtypes = [vp]
        L.tucker_last_error.restype = ctypes.c_char_p
        L.tucker_set_option.argtypes = [vp, c_int, ctypes.c_double]
        L.tucker_sthosvd.argtypes = [vp, vp, c_int, c_int, i64p, ctypes.c_double, i64p,
                                     ctypes.POINTER(c_int), c_int, ctypes.POINTER(ctypes.POINTER(CResult))]
        L.tucker_sthosvd_batched.argtypes = [vp, c_int, ctypes.POINTER(vp), c_int,
                                             ctypes.POINTER(c_int), ctypes.POINTER(i64p),
                                             ctypes.c_double, c_int,
                                             ctypes.POINTER(ctypes.POINTER(CResult))]
        L.tucker_result_destroy.argtypes = [ctypes.POINTER(CResult)]
        L.tucker_reconstruct.argtypes = [vp, ctypes.POINTER(CResult), i64p, i64p,
                                         ctypes.POINTER(c_int), c_int, vp, c_int]
        L.tucker_multi_ttm.argtypes = [vp, vp, c_int, c_int, i64p, ctypes.POINTER(vp), i64p, i64p,
                                       ctypes.POINTER(c_int), c_int, vp, c_int]
        L.tucker_ttm_order.argtypes = [c_int, i64p, i64p, c_int, ctypes.POINTER(c_int)]
        L.tucker_norm_sq.argtypes = [vp, vp, c_int, ctypes.c_int64, ctypes.POINTER(ctypes.c_double)]
        L.tucker_gram.argtypes = [vp, vp, c_int, c_int, i64p, c_int, c_int, vp]
        L.tucker_eig.argtypes = [vp, vp, ctypes.c_int64, vp, vp, ctypes.POINTER(c_int)]
        L.tucker_eig_trunc.argtypes = [vp, vp, ctypes.c_int64, ctypes.c_double, ctypes.c_int64,
                                       vp, vp, i64p, ctypes.POINTER(ctypes.c_double)]
        L.tucker_rank_cut.argtypes = [vp, vp, ctypes.c_int64, ctypes.c_double, i64p,
                                      ctypes.POINTER(ctypes.c_double)]
        L.tucker_ttm.argtypes = [vp, vp, c_int, c_int, i64p, c_int, vp, ctypes.c_int64,
                                 ctypes.c_int64, c_int, c_int, vp, c_int]
        for name in EXPORTS:
            if name not in ("tucker_last_error", "tucker_kernel_launches",
                            "tucker_autotune_entries"):
                getattr(L, name).restype = c_int
        L.tucker_kernel_launches.argtypes = []
        L.tucker_kernel_launches.restype = ctypes.c_uint64
        L.tucker_autotune_entries.argtypes = []
        L.tucker_autotune_entries.restype = ctypes.c_int64
        L.tucker_gram_noalloc.argtypes = [vp, c_int, c_int, i64p, c_int, c_int, vp, vp]
        L.tucker_hosvd.argtypes = [vp, vp, c_int, c_int, i64p, ctypes.c_double, i64p, c_int,
                                   ctypes.POINTER(ctypes.POINTER(CResult))]
        L.tucker_sthosvd_host.argtypes = L.tucker_sthosvd.argtypes
        L.tucker_sthosvd_order.argtypes = [c_int, i64p, i64p, ctypes.POINTER(c_int)]
        L.tucker_selftest_rcp64.argtypes = [vp, vp, ctypes.c_int64, vp]
        L.tucker_slice_stats.argtypes = [vp, vp, c_int, c_int, i64p, c_int, vp]
        L.tucker_slice_transform.argtypes = [vp, vp, c_int, c_int, i64p, c_int, vp, vp, c_int, vp]
        L.tucker_preprocess.argtypes = [vp, vp, c_int, c_int, i64p, c_int, c_int, vp, vp, vp]
        _lib = L
    return _lib


def _i64(vals):
    return (ctypes.c_int64 * MAX_MODES)(*[int(v) for v in vals])


def _ints(vals):
    return (ctypes.c_int * MAX_MODES)(*[int(v) for v in vals])


def _dtype_code(t):
    import torch
    if t.dtype == torch.float32:
        return F32
    if t.dtype == torch.float64:
        return F64
    raise TypeError(f"unsupported dtype {t.dtype}")


def _torch_dtype(code):
    import torch
    return torch.float64 if code == F64 else torch.float32


class _CAI:
    """Minimal __cuda_array_interface__ carrier for a library-owned pointer."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3,
                                         "strides": None}


def _view(ptr, shape, code):
    import torch
    return torch.as_tensor(_CAI(ptr, shape, "<f8" if code == F64 else "<f4"), device="cuda")


def _check_dev(t, name):
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA tensor")


def _host_buffer(x):
    """(address, dtype code, element count) of a contiguous host array: a CPU
    torch tensor or a numpy array of float32 / float64."""
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("x must be a contiguous host array")
        if x.dtype == np.float32:
            code = F32
        elif x.dtype == np.float64:
            code = F64
        else:
            raise TypeError(f"unsupported dtype {x.dtype}")
        return x.ctypes.data, code, x.size
    if getattr(x, "is_cuda", True) or not x.is_contiguous():
        raise ValueError("x must be a contiguous host (CPU) tensor or numpy array")
    return x.data_ptr(), _dtype_code(x), x.numel()


class Result:
    """ST-HOSVD result.  Scalars are read at once; the device arrays (core,
    factors, eigenvalues) are copied into torch tensors on first access."""

    def __init__(self, ctx, ptr):
        self._ctx, self._p = ctx, ptr
        r = ptr.contents
        N = r.ndim
        self.ndim = N
        self.dims = tuple(r.dims[k] for k in range(N))
        self.ranks = tuple(r.ranks[k] for k in range(N))
        self.mode_order = tuple(r.mode_order[k] for k in range(N))
        self.norm_sq = r.norm_x_sq
        self.threshold = r.threshold
        self.discarded = [r.discarded_sq[k] for k in range(N)]
        self.sweeps = [r.jacobi_sweeps[k] for k in range(N)]
        names = {0: "simt-fp64", 1: "simt-fp32", 2: "tcgen05", 3: "small-fp64", 4: "simt-fp32c",
                 5: "tcgen05-x3", 6: "tcgen05-x2"}
        self.gram_kernel = [names.get(r.gram_kernel[k], "?") for k in range(N)]
        self.ttm_kernel = [names.get(r.ttm_kernel[k], "?") for k in range(N)]
        self.eig_kernel = [{0: "jacobi", 1: "tridiag"}.get(r.eig_kernel[k], "?") for k in range(N)]
        self.core_dtype = r.core_dtype
        self.ms = {"norm": r.ms_norm, "total": r.ms_total,
                   "gram": [r.ms_gram[k] for k in range(N)],
                   "eig": [r.ms_eig[k] for k in range(N)],
                   "ttm": [r.ms_ttm[k] for k in range(N)]}
        self._core = self._factors = self._eigvals = None

    def _r(self):
        if self._p is None:
            raise RuntimeError("result was closed")
        return self._p.contents

    @property
    def core(self):
        if self._core is None:
            self._core = _view(self._r().core, (int(np.prod(self.ranks)),), self.core_dtype).clone()
        return self._core

    @property
    def factors(self):
        # U_n is I_n x R_n column-major == (R_n, I_n) row-major
        if self._factors is None:
            r = self._r()
            self._factors = [_view(r.factors[k], (self.ranks[k], self.dims[k]), F64).clone().t()
                             for k in range(self.ndim)]
        return self._factors

    @property
    def eigvals(self):
        if self._eigvals is None:
            r = self._r()
            self._eigvals = [_view(r.eigvals[k], (self.dims[k],), F64).clone()
                             for k in range(self.ndim)]
        return self._eigvals

    def to_host(self):
        """Device -> host copy of core and factors (numpy), straight from
        the library-owned buffers."""
        import torch
        r = self._r()
        core = _view(r.core, (int(np.prod(self.ranks)),), self.core_dtype).cpu().numpy()
        fac = [_view(r.factors[k], (self.ranks[k], self.dims[k]), F64).cpu().numpy().T
               for k in range(self.ndim)]
        return core, fac

    def reconstruct(self, begin=None, end=None, mode_order=None, prec="fp64", out_dtype=None):
        return self._ctx.reconstruct(self, begin, end, mode_order, prec, out_dtype)

    def close(self):
        if self._p is not None:
            lib().tucker_result_destroy(self._p)
            self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Context:
    """Owns a tucker_ctx bound to a CUDA stream (default: torch's current)."""

    def __init__(self, stream=None, timing=False):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self._c = ctypes.c_void_p()
        self._check(lib().tucker_create(ctypes.byref(self._c), ctypes.c_void_p(stream)))
        if timing:
            self.set_option(OPT_TIMING, 1)

    def _check(self, st):
        if st != 0:
            msg = lib().tucker_last_error(self._c).decode() if self._c else ""
            raise TuckerError(st, msg)

    def set_option(self, key, value):
        self._check(lib().tucker_set_option(self._c, int(key), float(value)))

    def close(self):
        if self._c:
            lib().tucker_destroy(self._c)
            self._c = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- whole path
    def sthosvd(self, x, dims, eps=None, ranks=None, mode_order=None, prec="fp64"):
        _check_dev(x, "x")
        N = len(dims)
        out = ctypes.POINTER(CResult)()
        st = lib().tucker_sthosvd(
            self._c, ctypes.c_void_p(x.data_ptr()), _dtype_code(x), N, _i64(dims),
            float(eps) if eps is not None else 0.0,
            _i64(ranks) if ranks is not None else None,
            _ints(mode_order) if mode_order is not None else None,
            PREC[prec], ctypes.byref(out))
        if st != 0 and out:
            lib().tucker_result_destroy(out)   # EIG_NOCONV still returns a result
        self._check(st)
        return Result(self, out)

    def sthosvd_host(self, x, dims, eps=None, ranks=None, mode_order=None, prec="fp64"):
        """ST-HOSVD of a tensor in host memory (tucker_sthosvd_host): x is a
        contiguous CPU torch tensor (page-locked for an overlapped copy) or
        numpy array of float32/float64 with prod(dims) elements."""
        ptr, code, n = _host_buffer(x)
        if n != int(np.prod([int(d) for d in dims])):
            raise ValueError(f"x has {n} elements, dims {tuple(dims)} need {int(np.prod(dims))}")
        out = ctypes.POINTER(CResult)()
        st = lib().tucker_sthosvd_host(
            self._c, ctypes.c_void_p(ptr), code, len(dims), _i64(dims),
            float(eps) if eps is not None else 0.0,
            _i64(ranks) if ranks is not None else None,
            _ints(mode_order) if mode_order is not None else None,
            PREC[prec], ctypes.byref(out))
        if st != 0 and out:
            lib().tucker_result_destroy(out)
        self._check(st)
        return Result(self, out)

    def hosvd(self, x, dims, eps=None, ranks=None, prec="fp64"):
        """HOSVD (tucker_hosvd): every factor from the Gram of x itself."""
        _check_dev(x, "x")
        out = ctypes.POINTER(CResult)()
        st = lib().tucker_hosvd(
            self._c, ctypes.c_void_p(x.data_ptr()), _dtype_code(x), len(dims), _i64(dims),
            float(eps) if eps is not None else 0.0,
            _i64(ranks) if ranks is not None else None, PREC[prec], ctypes.byref(out))
        if st != 0 and out:
            lib().tucker_result_destroy(out)
        self._check(st)
        return Result(self, out)

    def slice_stats(self, x, dims, mode):
        """(I_n, 6) FP64 device tensor of hyperslice statistics (STATS order)."""
        import torch
        _check_dev(x, "x")
        I = int(dims[mode])
        st = torch.empty((I, 6), dtype=torch.float64, device=x.device)
        self._check(lib().tucker_slice_stats(self._c, ctypes.c_void_p(x.data_ptr()),
                                             _dtype_code(x), len(dims), _i64(dims), int(mode),
                                             ctypes.c_void_p(st.data_ptr())))
        return st

    def slice_transform(self, x, dims, mode, shift, scale, inverse=False, out=None):
        """y = (x - shift_i) * scale_i per mode-`mode` hyperslice (inverse:
        x / scale_i + shift_i); out may be x (in place)."""
        import torch
        _check_dev(x, "x")
        I = int(dims[mode])
        for t, nm in ((shift, "shift"), (scale, "scale")):
            _check_dev(t, nm)
            if t.dtype != torch.float64 or t.numel() < I:
                raise ValueError(f"{nm} must hold {I} float64 values")
        y = torch.empty_like(x) if out is None else out
        _check_dev(y, "out")
        if y.dtype != x.dtype or y.numel() != x.numel():
            raise ValueError("out must match x in dtype and size")
        self._check(lib().tucker_slice_transform(
            self._c, ctypes.c_void_p(x.data_ptr()), _dtype_code(x), len(dims), _i64(dims),
            int(mode), ctypes.c_void_p(shift.data_ptr()), ctypes.c_void_p(scale.data_ptr()),
            1 if inverse else 0, ctypes.c_void_p(y.data_ptr())))
        return y

    def preprocess(self, x, dims, mode, method="standardize", out=None):
        """Section 3.5 pre-processing; returns (y, shift, scale)."""
        import torch
        _check_dev(x, "x")
        I = int(dims[mode])
        shift = torch.empty(I, dtype=torch.float64, device=x.device)
        scale = torch.empty(I, dtype=torch.float64, device=x.device)
        y = torch.empty_like(x) if out is None else out
        _check_dev(y, "out")
        if y.dtype != x.dtype or y.numel() != x.numel():
            raise ValueError("out must match x in dtype and size")
        self._check(lib().tucker_preprocess(
            self._c, ctypes.c_void_p(x.data_ptr()), _dtype_code(x), len(dims), _i64(dims),
            int(mode), PRE_METHOD[method], ctypes.c_void_p(shift.data_ptr()),
            ctypes.c_void_p(scale.data_ptr()), ctypes.c_void_p(y.data_ptr())))
        return y, shift, scale

    def sthosvd_batched(self, xs, dims_list, eps, prec="fp64"):
        """ST-HOSVD of several tensors at once (tucker_sthosvd_batched);
        xs: contiguous CUDA tensors of one dtype, dims_list: their dims."""
        n = len(xs)
        if n != len(dims_list) or n < 1:
            raise ValueError("xs and dims_list must have the same, nonzero length")
        for t in xs:
            _check_dev(t, "x")
        codes = {_dtype_code(t) for t in xs}
        if len(codes) != 1:
            raise TypeError("all tensors of a batch must have one dtype")
        ptrs = (ctypes.c_void_p * n)(*[t.data_ptr() for t in xs])
        nd = (ctypes.c_int * n)(*[len(d) for d in dims_list])
        dim_arrs = [(ctypes.c_int64 * len(d))(*[int(v) for v in d]) for d in dims_list]
        dptrs = (ctypes.POINTER(ctypes.c_int64) * n)(
            *[ctypes.cast(a, ctypes.POINTER(ctypes.c_int64)) for a in dim_arrs])
        outs = (ctypes.POINTER(CResult) * n)()
        self._check(lib().tucker_sthosvd_batched(self._c, n, ptrs, codes.pop(), nd, dptrs,
                                                 float(eps), PREC[prec], outs))
        return [Result(self, outs[i]) for i in range(n)]

    def reconstruct(self, res, begin=None, end=None, mode_order=None, prec="fp64", out_dtype=None):
        import torch
        N = res.ndim
        b = list(begin) if begin is not None else [0] * N
        e = list(end) if end is not None else list(res.dims)
        shape = int(np.prod([e[k] - b[k] for k in range(N)]))
        odt = res.core_dtype if out_dtype is None else out_dtype
        out = torch.empty(shape, dtype=_torch_dtype(odt), device="cuda")
        st = lib().tucker_reconstruct(self._c, res._p, _i64(b), _i64(e),
                                      _ints(mode_order) if mode_order is not None else None,
                                      PREC[prec], ctypes.c_void_p(out.data_ptr()), odt)
        self._check(st)
        return out

    def multi_ttm(self, core, core_dims, mats, out_dims, mode_order=None, prec="fp64",
                  out_dtype=None):
        """mats[n]: torch FP64 tensor (K_n, R_n) on the device (any strides
        with unit row stride are passed as column-major with lda)."""
        import torch
        _check_dev(core, "core")
        N = len(core_dims)
        ptrs, lda, keep = (ctypes.c_void_p * MAX_MODES)(), [], []
        for n, A in enumerate(mats):
            At = A.t().contiguous().t() if A.stride(0) != 1 else A   # column-major
            keep.append(At)
            ptrs[n] = At.data_ptr()
            lda.append(At.stride(1) if At.shape[1] > 1 else At.shape[0])
        odt = _dtype_code(core) if out_dtype is None else out_dtype
        out = torch.empty(int(np.prod(out_dims)), dtype=_torch_dtype(odt), device="cuda")
        st = lib().tucker_multi_ttm(self._c, ctypes.c_void_p(core.data_ptr()), _dtype_code(core), N,
                                    _i64(core_dims), ptrs, _i64(lda), _i64(out_dims),
                                    _ints(mode_order) if mode_order is not None else None,
                                    PREC[prec], ctypes.c_void_p(out.data_ptr()), odt)
        self._check(st)
        return out

    # ---- single steps
    def norm_sq(self, y):
        _check_dev(y, "y")
        v = ctypes.c_double()
        self._check(lib().tucker_norm_sq(self._c, ctypes.c_void_p(y.data_ptr()), _dtype_code(y),
                                         y.numel(), ctypes.byref(v)))
        return v.value

    def gram(self, y, dims, mode, prec="fp64"):
        import torch
        _check_dev(y, "y")
        I = int(dims[mode])
        S = torch.empty((I, I), dtype=torch.float64, device="cuda")
        self._check(lib().tucker_gram(self._c, ctypes.c_void_p(y.data_ptr()), _dtype_code(y),
                                      len(dims), _i64(dims), int(mode), PREC[prec],
                                      ctypes.c_void_p(S.data_ptr())))
        return S

    def eig(self, S):
        """Descending eigenvalues and column eigenvectors (torch (I, I))."""
        import torch
        _check_dev(S, "S")
        I = S.shape[0]
        w = torch.empty(I, dtype=torch.float64, device="cuda")
        Vt = torch.empty((I, I), dtype=torch.float64, device="cuda")   # column-major V
        sw = ctypes.c_int()
        self._check(lib().tucker_eig(self._c, ctypes.c_void_p(S.data_ptr()), I,
                                     ctypes.c_void_p(w.data_ptr()), ctypes.c_void_p(Vt.data_ptr()),
                                     ctypes.byref(sw)))
        return w, Vt.t(), sw.value

    def eig_trunc(self, S, thr=0.0, R=0):
        """All eigenvalues (descending) and the leading R eigenvectors (torch
        (I, R)) of S; R from the cut at thr, or given.  Returns (w, U, R,
        discarded)."""
        import torch
        _check_dev(S, "S")
        I = S.shape[0]
        w = torch.empty(I, dtype=torch.float64, device="cuda")
        Ut = torch.empty((I, I), dtype=torch.float64, device="cuda")
        Rv, d = ctypes.c_int64(), ctypes.c_double()
        self._check(lib().tucker_eig_trunc(self._c, ctypes.c_void_p(S.data_ptr()), I, float(thr),
                                           int(R), ctypes.c_void_p(w.data_ptr()),
                                           ctypes.c_void_p(Ut.data_ptr()), ctypes.byref(Rv),
                                           ctypes.byref(d)))
        k = Rv.value
        U = Ut.view(-1)[:I * k].view(k, I).t()
        return w, U, k, d.value

    def rank_cut(self, w, thr):
        R, d = ctypes.c_int64(), ctypes.c_double()
        self._check(lib().tucker_rank_cut(self._c, ctypes.c_void_p(w.data_ptr()), w.numel(),
                                          float(thr), ctypes.byref(R), ctypes.byref(d)))
        return R.value, d.value

    def ttm(self, y, dims, mode, A, prec="fp64", out_dtype=None):
        """Z = Y x_mode A with A a (K, J_mode) FP64 device tensor."""
        import torch
        _check_dev(y, "y")
        K = A.shape[0]
        if A.stride(1) == 1:
            arow, lda = 1, A.stride(0) if K > 1 else A.shape[1]
        elif A.stride(0) == 1:
            arow, lda = 0, A.stride(1) if A.shape[1] > 1 else K
        else:
            A = A.contiguous()
            arow, lda = 1, A.shape[1]
        zd = list(dims)
        zd[mode] = K
        odt = _dtype_code(y) if out_dtype is None else out_dtype
        z = torch.empty(int(np.prod(zd)), dtype=_torch_dtype(odt), device="cuda")
        self._check(lib().tucker_ttm(self._c, ctypes.c_void_p(y.data_ptr()), _dtype_code(y),
                                     len(dims), _i64(dims), int(mode),
                                     ctypes.c_void_p(A.data_ptr()), K, lda, arow, PREC[prec],
                                     ctypes.c_void_p(z.data_ptr()), odt))
        return z


def ttm_order(core_dims, out_dims, objective="flops"):
    """Mode order of a multi-TTM chain (host-only C call)."""
    N = len(core_dims)
    out = (ctypes.c_int * MAX_MODES)()
    st = lib().tucker_ttm_order(N, _i64(core_dims), _i64(out_dims),
                                0 if objective == "flops" else 1, out)
    if st != 0:
        raise TuckerError(st, "tucker_ttm_order")
    return tuple(out[k] for k in range(N))


def sthosvd_order(dims, ranks):
    """Flop-minimal ST-HOSVD mode order for given ranks (host-only C call)."""
    N = len(dims)
    out = (ctypes.c_int * MAX_MODES)()
    st = lib().tucker_sthosvd_order(N, _i64(dims), _i64(ranks), out)
    if st != 0:
        raise TuckerError(st, "tucker_sthosvd_order")
    return tuple(out[k] for k in range(N))


def selftest_rcp64(x):
    """The tridiagonal eigensolver's FP64 reciprocal of every entry of the
    FP64 device tensor x (diagnostics)."""
    import torch
    _check_dev(x, "x")
    if x.dtype != torch.float64:
        raise ValueError("x must be float64")
    y = torch.empty_like(x)
    st = lib().tucker_selftest_rcp64(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                     x.numel(), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    if st != 0:
        raise TuckerError(st, "tucker_selftest_rcp64")
    return y


def autotune_entries():
    """(kernel, shape) entries the split-K autotuner has cached so far."""
    return int(lib().tucker_autotune_entries())


def kernel_launches():
    """Kernels launched by the library in this process so far."""
    return int(lib().tucker_kernel_launches())


def _check_gram_out(y, dims, mode, S):
    """Shape, dtype and device checks of a Gram call whose output S the
    caller supplies: the kernels write I_n x I_n FP64 values through S's
    pointer and read prod(dims) elements of y, so a mismatch would reach
    memory outside both tensors.  Raises ValueError before anything runs."""
    import torch
    if not 0 <= int(mode) < len(dims):
        raise ValueError(f"mode {mode} out of range for {len(dims)} modes")
    if y.numel() != int(np.prod([int(d) for d in dims])):
        raise ValueError(f"y holds {y.numel()} elements, dims {tuple(dims)} need "
                         f"{int(np.prod([int(d) for d in dims]))}")
    I = int(dims[mode])
    if S.dtype != torch.float64:
        raise ValueError(f"S must be float64, got {S.dtype}")
    if tuple(S.shape) != (I, I):
        raise ValueError(f"S must have shape ({I}, {I}), got {tuple(S.shape)}")
    if S.device != y.device:
        raise ValueError(f"S is on {S.device}, y on {y.device}")


def gram_noalloc(y, dims, mode, S, prec="fp64", stream=None):
    """tucker_gram_noalloc: the Gram of one mode into the caller's FP64
    (I, I) device tensor S, with the library's fixed device scratch instead
    of any allocation.  Asynchronous on `stream` (default: torch's current).
    For callers that cannot allocate device memory; calls that overlap on
    the GPU share the scratch and race."""
    import torch
    _check_gram_out(y, dims, mode, S)
    _check_dev(y, "y")
    _check_dev(S, "S")
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    st = lib().tucker_gram_noalloc(ctypes.c_void_p(y.data_ptr()), _dtype_code(y), len(dims),
                                   _i64(dims), int(mode), PREC[prec],
                                   ctypes.c_void_p(S.data_ptr()), ctypes.c_void_p(stream))
    if st != 0:
        raise TuckerError(st, "tucker_gram_noalloc")
    return S


# MIXED precision (exact-digit tensor-core Grams, tensor-core TTMs) is built.
MIXED_AVAILABLE = True
