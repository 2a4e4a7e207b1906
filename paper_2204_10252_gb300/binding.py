"""Thin ctypes binding of libpp (include/pp.h): argument marshalling only.

Every function below has the name and argument order of the C entry point
it wraps.  Device arrays are torch complex64 CUDA tensors (PyTorch provides
memory and streams; all arithmetic runs in libpp's kernels).  A call that
returns a status other than PP_OK raises PPError with pp_last_error().
There is no fallback: when libpp.so is missing or cannot be loaded, the
first call raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libpp.so")

PP_OK, PP_ERR_INVALID_ARG, PP_ERR_UNSUPPORTED, PP_ERR_OOM, PP_ERR_CUDA, PP_ERR_NONFINITE, \
    PP_ERR_TIMEOUT = range(7)
PP_CARTESIAN, PP_NONCARTESIAN, PP_NONCARTESIAN_TOEPLITZ = 0, 1, 2
STATUS_NAMES = {0: "PP_OK", 1: "PP_ERR_INVALID_ARG", 2: "PP_ERR_UNSUPPORTED", 3: "PP_ERR_OOM",
                4: "PP_ERR_CUDA", 5: "PP_ERR_NONFINITE", 6: "PP_ERR_TIMEOUT"}


class PPError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__("%s: %s (%s)" % (where, message, STATUS_NAMES.get(status, status)))
        self.status = status


class pp_dims(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("n", ctypes.c_int * 3)]


class pp_sampling(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("mask", ctypes.c_void_p), ("traj", ctypes.c_void_p),
                ("K", ctypes.c_int64), ("kb_width", ctypes.c_int), ("oversamp", ctypes.c_float)]


class pp_solve_info(ctypes.Structure):
    _fields_ = [("rescale", ctypes.c_int), ("levels", ctypes.c_int), ("no_momentum", ctypes.c_int),
                ("history", ctypes.c_void_p), ("ref", ctypes.c_void_p),
                ("bnorm", ctypes.c_double), ("L", ctypes.c_double), ("launches", ctypes.c_int64),
                ("wavelet", ctypes.c_int), ("safe_scale", ctypes.c_int)]


_lib = None

_SIGS = {
    "pp_plan_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), pp_dims, ctypes.c_int,
                                      ctypes.c_void_p, ctypes.POINTER(pp_sampling), ctypes.c_uint64,
                                      ctypes.c_int, ctypes.c_void_p]),
    "pp_plan_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "pp_plan_scale": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    "pp_plan_set_scale": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double]),
    "pp_plan_mu": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64,
                                  ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]),
    "pp_plan_tuning": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "pp_plan_set_tuning": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "pp_plan_sizes": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64),
                                     ctypes.POINTER(ctypes.c_int64)]),
    "pp_forward_apply": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "pp_adjoint_apply": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "pp_adjoint_apply_static": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "pp_normal_apply": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "pp_poly_coeffs_l2": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "pp_poly_coeffs_cheb": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]),
    "pp_poly_coeffs_wl2": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_double)]),
    "pp_poly_max_zp": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                                      ctypes.POINTER(ctypes.c_double)]),
    "pp_poly_apply": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "pp_prox_l1_haar": (ctypes.c_int, [pp_dims, ctypes.c_int, ctypes.c_float, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p]),
    "pp_prox_l1_db4": (ctypes.c_int, [pp_dims, ctypes.c_int, ctypes.c_float, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_void_p]),
    "pp_fista_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_float, ctypes.c_int,
                                      ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_void_p,
                                      ctypes.POINTER(pp_solve_info), ctypes.c_void_p]),
    "pp_fista_solve_prox": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                                           ctypes.c_float, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                           ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(pp_solve_info),
                                           ctypes.c_void_p]),
    "pp_profile_normal": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                         ctypes.c_int, ctypes.c_char_p, ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_int), ctypes.c_void_p]),
    "pp_batch_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64,
                                       ctypes.c_int, ctypes.c_void_p]),
    "pp_batch_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "pp_batch_offsets": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "pp_batch_scales": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "pp_batch_set_scales": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "pp_batch_tile": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "pp_batch_set_tile": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "pp_batch_forward_apply": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "pp_batch_adjoint_apply": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "pp_batch_normal_apply": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "pp_batch_fista_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_float, ctypes.c_int,
                                            ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_void_p,
                                            ctypes.POINTER(pp_solve_info), ctypes.c_void_p]),
    "pp_batch_unrolled_forward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_float, ctypes.c_int,
                                                 ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_int,
                                                 ctypes.c_void_p, ctypes.c_void_p]),
    "pp_batch_unrolled_backward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_float, ctypes.c_int,
                                                  ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_int,
                                                  ctypes.c_void_p, ctypes.c_void_p,
                                                  ctypes.POINTER(ctypes.c_double),
                                                  ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]),
    "pp_selftest_wait": (ctypes.c_int, [ctypes.c_int64, ctypes.c_void_p]),
    "pp_prox_llr": (ctypes.c_int, [pp_dims, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_float,
                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "pp_last_error": (ctypes.c_char_p, []),
}


def lib(path: Optional[str] = None):
    """Load libpp.so (once).  Raises when it is missing: there is no fallback."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError("libpp.so not found at %s: build it with "
                           "paper_2204_10252_gb300.build.build_library()" % p)
    L = ctypes.CDLL(p)
    for name, (res, args) in _SIGS.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(status: int, where: str):
    if status != PP_OK:
        msg = lib().pp_last_error()
        raise PPError(status, where, msg.decode() if msg else "")


def _dims(shape: Sequence[int]) -> pp_dims:
    """Image shape in C order ([ny, nx] or [nz, ny, nx]) -> pp_dims."""
    shape = tuple(int(s) for s in shape)
    d = pp_dims()
    d.ndim = len(shape)
    rev = list(reversed(shape)) + [1] * (3 - len(shape))
    for i in range(3):
        d.n[i] = rev[i]
    return d


def _dev_ptr(t, what: str) -> int:
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError("%s must be a torch tensor" % what)
    if not t.is_cuda or t.dtype != torch.complex64 or not t.is_contiguous():
        raise ValueError("%s must be a contiguous complex64 CUDA tensor" % what)
    return t.data_ptr()


def _numel(t, n: int, what: str):
    """Raise before any device work when a tensor's size does not match what
    the plan will read or write (the C ABI cannot see buffer sizes)."""
    size = int(t.numel()) if hasattr(t, "numel") else int(np.size(t))
    if size != n:
        raise ValueError("%s has %d elements; the plan expects %d" % (what, size, n))


def _img(plan, t, what):
    _numel(t, int(np.prod(plan.shape)), what)
    return _dev_ptr(t, what)


def _ksp(plan, t, what):
    _numel(t, int(np.prod(plan.kspace_shape)), what)
    return _dev_ptr(t, what)


def _stream(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Plan:
    """Handle of a pp_plan.  Keeps the borrowed sensitivity tensor alive."""

    def __init__(self, handle: int, shape, coils: int, sens, kspace_shape):
        self.handle = ctypes.c_void_p(handle)
        self.shape = tuple(shape)
        self.coils = coils
        self.kspace_shape = tuple(kspace_shape)
        self._sens = sens

    def destroy(self):
        if self.handle:
            _check(lib().pp_plan_destroy(self.handle), "pp_plan_destroy")
            self.handle = ctypes.c_void_p(0)
            self._sens = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.destroy()

    def __del__(self):
        try:
            if self.handle:
                lib().pp_plan_destroy(self.handle)
        except Exception:
            pass


def pp_plan_create(shape, coils: int, sens, mask=None, traj=None, kb_width: int = 4,
                   oversamp: float = 1.25, seed: int = 0, power_iters: int = 50,
                   stream=None, toeplitz: bool = False) -> Plan:
    """shape: image shape [ny, nx] or [nz, ny, nx]; sens: CUDA complex64
    [C, *shape]; mask: uint8 array of the image shape (Cartesian) or
    traj: float32 [K, 2] (non-Cartesian; toeplitz=True evaluates the normal
    operator as the exact F^H F through its Toeplitz embedding)."""
    s = pp_sampling()
    keep = []
    if mask is not None:
        m = np.ascontiguousarray(mask, dtype=np.uint8)
        keep.append(m)
        s.kind = PP_CARTESIAN
        s.mask = m.ctypes.data
        s.traj = None
        s.K = 0
        kshape = (coils,) + tuple(shape)
    elif traj is not None:
        t = np.ascontiguousarray(traj, dtype=np.float32)
        keep.append(t)
        s.kind = PP_NONCARTESIAN_TOEPLITZ if toeplitz else PP_NONCARTESIAN
        s.mask = None
        s.traj = t.ctypes.data
        s.K = int(t.shape[0])
        kshape = (coils, int(t.shape[0]))
    else:
        raise ValueError("need a mask or a trajectory")
    s.kb_width = int(kb_width)
    s.oversamp = float(oversamp)
    out = ctypes.c_void_p(0)
    _numel(sens, int(coils) * int(np.prod(shape)), "sens")
    if mask is not None:
        _numel(m, int(np.prod(shape)), "mask")
    _check(lib().pp_plan_create(ctypes.byref(out), _dims(shape), int(coils), _dev_ptr(sens, "sens"),
                                ctypes.byref(s), ctypes.c_uint64(seed), int(power_iters),
                                _stream(stream)), "pp_plan_create")
    return Plan(out.value, shape, coils, sens, kshape)


def pp_plan_destroy(plan: Plan):
    plan.destroy()


def pp_plan_scale(plan: Plan) -> float:
    L = ctypes.c_double(0.0)
    _check(lib().pp_plan_scale(plan.handle, ctypes.byref(L)), "pp_plan_scale")
    return L.value


def pp_plan_set_scale(plan: Plan, L: float):
    _check(lib().pp_plan_set_scale(plan.handle, float(L)), "pp_plan_set_scale")


def pp_plan_mu(plan: Plan, iters: int = 50, seed: int = 0, stream=None) -> float:
    """mu = smallest eigenvalue of N_hat by power iteration on I - N_hat."""
    mu = ctypes.c_double(0.0)
    _check(lib().pp_plan_mu(plan.handle, int(iters), ctypes.c_uint64(seed), ctypes.byref(mu),
                            _stream(stream)), "pp_plan_mu")
    return mu.value


def pp_plan_tuning(plan: Plan):
    """(row_ifft_variant, stencil_kind, stencil_coils) chosen at plan creation."""
    a, b, c = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
    _check(lib().pp_plan_tuning(plan.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
           "pp_plan_tuning")
    return a.value, b.value, c.value


def pp_plan_set_tuning(plan: Plan, row_ifft_variant: int, stencil_kind: int, stencil_coils: int = 8):
    _check(lib().pp_plan_set_tuning(plan.handle, int(row_ifft_variant), int(stencil_kind),
                                    int(stencil_coils)), "pp_plan_set_tuning")


def pp_plan_sizes(plan: Plan):
    a, b = ctypes.c_int64(0), ctypes.c_int64(0)
    _check(lib().pp_plan_sizes(plan.handle, ctypes.byref(a), ctypes.byref(b)), "pp_plan_sizes")
    return a.value, b.value


def pp_forward_apply(plan: Plan, x, y, stream=None):
    _check(lib().pp_forward_apply(plan.handle, _img(plan, x, "x"), _ksp(plan, y, "y"), _stream(stream)),
           "pp_forward_apply")


def pp_adjoint_apply(plan: Plan, y, x, stream=None):
    _check(lib().pp_adjoint_apply(plan.handle, _ksp(plan, y, "y"), _img(plan, x, "x"), _stream(stream)),
           "pp_adjoint_apply")


def pp_adjoint_apply_static(plan: Plan, y, x, stream=None):
    """A^H y without allocating device memory: for callers that cannot
    allocate at call time; intermediates live in a fixed 16 MiB library
    array (see include/pp.h)."""
    _check(lib().pp_adjoint_apply_static(plan.handle, _ksp(plan, y, "y"), _img(plan, x, "x"),
                                         _stream(stream)), "pp_adjoint_apply_static")


def pp_normal_apply(plan: Plan, x, y, stream=None):
    _check(lib().pp_normal_apply(plan.handle, _img(plan, x, "x"), _img(plan, y, "y"), _stream(stream)),
           "pp_normal_apply")


def pp_poly_coeffs_l2(d: int) -> np.ndarray:
    c = (ctypes.c_double * (d + 1))() if d >= 0 else (ctypes.c_double * 1)()
    _check(lib().pp_poly_coeffs_l2(int(d), c), "pp_poly_coeffs_l2")
    return np.array(list(c), dtype=np.float64)


def pp_poly_coeffs_cheb(d: int, mu: float) -> np.ndarray:
    c = (ctypes.c_double * (max(d, 0) + 1))()
    _check(lib().pp_poly_coeffs_cheb(int(d), float(mu), c), "pp_poly_coeffs_cheb")
    return np.array(list(c), dtype=np.float64)


def pp_poly_coeffs_wl2(d: int, moments) -> np.ndarray:
    """Eq. "wl2cost" design; moments[k] = int_0^1 w(z) z^k dz, k = 0..2d+2."""
    m = np.ascontiguousarray(moments, dtype=np.float64)
    if m.ndim != 1 or m.size < 2 * max(d, 0) + 3:
        raise ValueError("need the moments m_0 .. m_{2d+2}")
    c = (ctypes.c_double * (max(d, 0) + 1))()
    mv = (ctypes.c_double * m.size)(*m.tolist())
    _check(lib().pp_poly_coeffs_wl2(int(d), mv, c), "pp_poly_coeffs_wl2")
    return np.array(list(c), dtype=np.float64)


def pp_poly_max_zp(c, d: int) -> float:
    """max over z in [0, 1] of z p(z) (the preconditioned step's Lipschitz constant)."""
    m = ctypes.c_double(0.0)
    cc = np.ascontiguousarray(c, dtype=np.float64)
    cv = (ctypes.c_double * len(cc))(*cc.tolist())
    _check(lib().pp_poly_max_zp(cv, int(d), ctypes.byref(m)), "pp_poly_max_zp")
    return m.value


def _cvec(c):
    c = np.ascontiguousarray(c, dtype=np.float64)
    return (ctypes.c_double * len(c))(*c.tolist())


def pp_poly_apply(plan: Plan, c, d: int, v, out, stream=None):
    _check(lib().pp_poly_apply(plan.handle, _cvec(c), int(d), _img(plan, v, "v"), _img(plan, out, "out"),
                               _stream(stream)), "pp_poly_apply")


def pp_prox_l1_haar(shape, levels: int, lam: float, x_in, x_out, stream=None):
    _numel(x_in, int(np.prod(shape)), "in")
    _numel(x_out, int(np.prod(shape)), "out")
    _check(lib().pp_prox_l1_haar(_dims(shape), int(levels), float(lam), _dev_ptr(x_in, "in"),
                                 _dev_ptr(x_out, "out"), _stream(stream)), "pp_prox_l1_haar")


def pp_prox_l1_db4(shape, levels: int, lam: float, x_in, x_out, stream=None):
    _numel(x_in, int(np.prod(shape)), "in")
    _numel(x_out, int(np.prod(shape)), "out")
    _check(lib().pp_prox_l1_db4(_dims(shape), int(levels), float(lam), _dev_ptr(x_in, "in"),
                                _dev_ptr(x_out, "out"), _stream(stream)), "pp_prox_l1_db4")


def pp_prox_llr(shape, T: int, block: int, lam: float, x_in, x_out, shift=None, stream=None):
    """Locally-low-rank prox of T coefficient images of `shape` ([ny, nx] or
    [nz, ny, nx]); x_in/x_out are complex64 CUDA tensors of T * prod(shape)
    elements; shift (x, y, z) moves the block grid circularly."""
    n = int(T) * int(np.prod(shape))
    _numel(x_in, n, "in")
    _numel(x_out, n, "out")
    sh = None
    if shift is not None:
        sv = [int(v) for v in shift] + [0] * (3 - len(shift))
        sh = (ctypes.c_int * 3)(*sv[:3])
    _check(lib().pp_prox_llr(_dims(shape), int(T), int(block), sh, float(lam), _dev_ptr(x_in, "in"),
                             _dev_ptr(x_out, "out"), _stream(stream)), "pp_prox_llr")


WAVELETS = {"haar": 0, "db4": 1}


class SolveResult:
    """What pp_fista_solve reports besides x_out."""

    def __init__(self, history, bnorm, L, launches):
        self.history = history      # [iters, 3] or None
        self.bnorm = bnorm
        self.L = L
        self.launches = launches


def pp_fista_solve(plan: Plan, b, lam: float, iters: int, c, d: int, x_out, stream=None,
                   history: bool = False, rescale: bool = False, levels: int = 2,
                   ref=None, momentum: bool = True, wavelet: str = "haar",
                   safe_scale: bool = False) -> SolveResult:
    """c None with d = 0: plain FISTA.  history: per-iteration FP64
    ||y_{k+1}-y_k||^2, ||y_{k+1}||^2, ||y_{k+1}-ref||^2 (ref optional).
    wavelet: "haar" or "db4" (Daubechies-4, 2-D) for the prox's W.
    safe_scale: divide c by max over [0, 1] of z p(z) (FISTA's step rule)."""
    info = pp_solve_info()
    info.wavelet = WAVELETS[wavelet]
    info.safe_scale = 1 if safe_scale else 0
    info.rescale = 1 if rescale else 0
    info.levels = int(levels)
    info.no_momentum = 0 if momentum else 1
    hist = None
    if history:
        hist = np.zeros((max(iters, 1), 3), dtype=np.float64)
        info.history = hist.ctypes.data
    else:
        info.history = None
    info.ref = _img(plan, ref, "ref") if ref is not None else None
    cptr = _cvec(c) if c is not None else None
    _check(lib().pp_fista_solve(plan.handle, _ksp(plan, b, "b"), float(lam), int(iters), cptr, int(d),
                                _img(plan, x_out, "x_out"), ctypes.byref(info), _stream(stream)),
           "pp_fista_solve")
    return SolveResult(hist[:iters] if hist is not None else None, info.bnorm, info.L,
                       int(info.launches))


def pp_fista_solve_prox(plan: Plan, b, v, sigma: float, lam: float, iters: int, c, d: int, x_out,
                        stream=None, history: bool = False, levels: int = 2, ref=None,
                        momentum: bool = True, wavelet: str = "haar") -> SolveResult:
    """argmin_x 1/2||A x - b||^2 + sigma/2 ||x - v||^2 + lam ||W x||_1 (the
    consensus-ADMM subproblem, rho = 1/sigma); b or v may be None."""
    info = pp_solve_info()
    info.wavelet = WAVELETS[wavelet]
    info.levels = int(levels)
    info.no_momentum = 0 if momentum else 1
    hist = None
    if history:
        hist = np.zeros((max(iters, 1), 3), dtype=np.float64)
        info.history = hist.ctypes.data
    else:
        info.history = None
    info.ref = _img(plan, ref, "ref") if ref is not None else None
    cptr = _cvec(c) if c is not None else None
    _check(lib().pp_fista_solve_prox(plan.handle, _ksp(plan, b, "b") if b is not None else None,
                                     _img(plan, v, "v") if v is not None else None, float(sigma),
                                     float(lam), int(iters), cptr, int(d), _img(plan, x_out, "x_out"),
                                     ctypes.byref(info), _stream(stream)), "pp_fista_solve_prox")
    return SolveResult(hist[:iters] if hist is not None else None, info.bnorm, info.L,
                       int(info.launches))


def pp_profile_normal(plan: Plan, x, y, reps: int = 20, stream=None, max_stages: int = 32):
    """Average milliseconds per normal apply for each kernel (CUDA events)."""
    names = ctypes.create_string_buffer(48 * max_stages)
    ms = (ctypes.c_double * max_stages)()
    n = ctypes.c_int(0)
    _check(lib().pp_profile_normal(plan.handle, _img(plan, x, "x"), _img(plan, y, "y"), int(reps),
                                   int(max_stages), names, ms, ctypes.byref(n), _stream(stream)),
           "pp_profile_normal")
    raw = names.raw
    return {raw[48 * i:48 * i + 48].split(b"\0", 1)[0].decode(): ms[i] for i in range(n.value)}


class Batch:
    """Handle of a pp_batch.  Keeps the borrowed sensitivity tensors alive."""

    def __init__(self, handle, shapes, coils, sens, image_off, kspace_off):
        self.handle = ctypes.c_void_p(handle)
        self.shapes = [tuple(s) for s in shapes]
        self.coils = list(coils)
        self.image_off = image_off
        self.kspace_off = kspace_off
        self._sens = list(sens)

    @property
    def n(self):
        return len(self.shapes)

    def destroy(self):
        if self.handle:
            _check(lib().pp_batch_destroy(self.handle), "pp_batch_destroy")
            self.handle = ctypes.c_void_p(0)
            self._sens = []

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.destroy()

    def __del__(self):
        try:
            if self.handle:
                lib().pp_batch_destroy(self.handle)
        except Exception:
            pass


def pp_batch_create(shapes, coils, sens, masks, seed: int = 0, power_iters: int = 50,
                    stream=None) -> Batch:
    """shapes: list of (ny, nx); coils: list of C_s; sens: list of CUDA
    complex64 [C_s, ny, nx]; masks: list of uint8 [ny, nx] (constant along x)."""
    n = len(shapes)
    dims = (pp_dims * n)(*[_dims(s) for s in shapes])
    cs = (ctypes.c_int * n)(*[int(c) for c in coils])
    for i, (t, shp, c) in enumerate(zip(sens, shapes, coils)):
        _numel(t, int(c) * int(np.prod(shp)), "sens[%d]" % i)
    sp = (ctypes.c_void_p * n)(*[_dev_ptr(t, "sens[%d]" % i) for i, t in enumerate(sens)])
    ms = [np.ascontiguousarray(m, dtype=np.uint8) for m in masks]
    for i, (m, shp) in enumerate(zip(ms, shapes)):
        if m.size != int(np.prod(shp)):
            raise ValueError("masks[%d] has %d elements; expected %d" % (i, m.size, int(np.prod(shp))))
    mp = (ctypes.c_void_p * n)(*[m.ctypes.data for m in ms])
    out = ctypes.c_void_p(0)
    _check(lib().pp_batch_create(ctypes.byref(out), n, dims, cs, sp, mp, ctypes.c_uint64(seed),
                                 int(power_iters), _stream(stream)), "pp_batch_create")
    io = np.zeros(n + 1, dtype=np.int64)
    ko = np.zeros(n + 1, dtype=np.int64)
    _check(lib().pp_batch_offsets(out, io.ctypes.data, ko.ctypes.data), "pp_batch_offsets")
    return Batch(out.value, shapes, coils, sens, io, ko)


def pp_batch_destroy(batch: Batch):
    batch.destroy()


def pp_batch_offsets(batch: Batch):
    return batch.image_off.copy(), batch.kspace_off.copy()


def pp_batch_scales(batch: Batch) -> np.ndarray:
    L = np.zeros(batch.n, dtype=np.float64)
    _check(lib().pp_batch_scales(batch.handle, L.ctypes.data), "pp_batch_scales")
    return L


def pp_batch_set_scales(batch: Batch, L):
    L = np.ascontiguousarray(L, dtype=np.float64)
    _check(lib().pp_batch_set_scales(batch.handle, L.ctypes.data), "pp_batch_set_scales")


def pp_batch_tile(batch: Batch):
    a, b = ctypes.c_int(0), ctypes.c_int(0)
    _check(lib().pp_batch_tile(batch.handle, ctypes.byref(a), ctypes.byref(b)), "pp_batch_tile")
    return a.value, b.value


def _bimg(batch, t, what):
    _numel(t, int(batch.image_off[-1]), what)
    return _dev_ptr(t, what)


def _bksp(batch, t, what):
    _numel(t, int(batch.kspace_off[-1]), what)
    return _dev_ptr(t, what)


def pp_batch_set_tile(batch: Batch, cols_per_cta: int):
    _check(lib().pp_batch_set_tile(batch.handle, int(cols_per_cta)), "pp_batch_set_tile")


def pp_batch_forward_apply(batch: Batch, x, y, stream=None):
    _check(lib().pp_batch_forward_apply(batch.handle, _bimg(batch, x, "x"), _bksp(batch, y, "y"),
                                        _stream(stream)), "pp_batch_forward_apply")


def pp_batch_adjoint_apply(batch: Batch, y, x, stream=None):
    _check(lib().pp_batch_adjoint_apply(batch.handle, _bksp(batch, y, "y"), _bimg(batch, x, "x"),
                                        _stream(stream)), "pp_batch_adjoint_apply")


def pp_batch_normal_apply(batch: Batch, x, y, stream=None):
    _check(lib().pp_batch_normal_apply(batch.handle, _bimg(batch, x, "x"), _bimg(batch, y, "y"),
                                       _stream(stream)), "pp_batch_normal_apply")


def pp_batch_fista_solve(batch: Batch, b, lam: float, iters: int, c, d: int, x_out, stream=None,
                         history: bool = False, rescale: bool = False, ref=None,
                         momentum: bool = True, safe_scale: bool = False) -> SolveResult:
    info = pp_solve_info()
    info.rescale = 1 if rescale else 0
    info.safe_scale = 1 if safe_scale else 0
    info.levels = 2
    info.no_momentum = 0 if momentum else 1
    hist = None
    if history:
        hist = np.zeros((max(iters, 1), 3), dtype=np.float64)
        info.history = hist.ctypes.data
    else:
        info.history = None
    info.ref = _bimg(batch, ref, "ref") if ref is not None else None
    cptr = _cvec(c) if c is not None else None
    _check(lib().pp_batch_fista_solve(batch.handle, _bksp(batch, b, "b"), float(lam), int(iters), cptr,
                                      int(d), _bimg(batch, x_out, "x_out"), ctypes.byref(info),
                                      _stream(stream)), "pp_batch_fista_solve")
    return SolveResult(hist[:iters] if hist is not None else None, info.bnorm, info.L,
                       int(info.launches))


def pp_batch_unrolled_forward(batch: Batch, b, lam: float, iters: int, c, d: int,
                              checkpoint_every: int, x_out, stream=None):
    _check(lib().pp_batch_unrolled_forward(batch.handle, _bksp(batch, b, "b"), float(lam), int(iters),
                                           _cvec(c), int(d), int(checkpoint_every),
                                           _bimg(batch, x_out, "x_out"), _stream(stream)),
           "pp_batch_unrolled_forward")


def pp_batch_unrolled_backward(batch: Batch, b, lam: float, iters: int, c, d: int,
                               checkpoint_every: int, grad_out, grad_b, stream=None):
    """Returns (grad_lambda, grad_c ndarray [d+1]); grad_b is written in place."""
    gl = ctypes.c_double(0.0)
    gc = (ctypes.c_double * (d + 1))()
    _check(lib().pp_batch_unrolled_backward(batch.handle, _bksp(batch, b, "b"), float(lam), int(iters),
                                            _cvec(c), int(d), int(checkpoint_every),
                                            _bimg(batch, grad_out, "grad_out"), _bksp(batch, grad_b, "grad_b"),
                                            ctypes.byref(gl), gc, _stream(stream)),
           "pp_batch_unrolled_backward")
    return gl.value, np.array(list(gc), dtype=np.float64)


def pp_selftest_wait(limit_ns: int, stream=None):
    """One block waits on a counter nothing increments; raises PPError with
    PP_ERR_TIMEOUT when the bounded wait gives up (the expected outcome)."""
    _check(lib().pp_selftest_wait(int(limit_ns), _stream(stream)), "pp_selftest_wait")


def pp_last_error() -> str:
    m = lib().pp_last_error()
    return m.decode() if m else ""
