"""Python binding of the sk C ABI (include/sk.h): the same entry points, same
names, argument marshalling only.  Every step of the computation runs in the
CUDA library; if the library has not been built this module refuses to import.

Arrays may be torch tensors (CUDA or CPU) or numpy arrays; they must be
float64 and contiguous.  Streams are torch.cuda.Stream objects, raw
cudaStream_t integers, or None for the current torch stream.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_LIB_PATH = _build.LIB
if not os.path.exists(_LIB_PATH):
    raise ImportError("the sk CUDA library is not built (%s); run __graft_entry__.build() first" % _LIB_PATH)
_lib = ctypes.CDLL(_LIB_PATH)

# status codes / enums (include/sk.h)
SK_OK, SK_ERR_ARG, SK_ERR_DOMAIN, SK_ERR_WEIGHTS, SK_ERR_NOMEM = 0, 1, 2, 3, 4
SK_ERR_UNDERFLOW, SK_ERR_NOT_CONVERGED, SK_ERR_TIMEOUT, SK_ERR_CUDA, SK_ERR_UNSUPPORTED = 5, 6, 7, 8, 9
SK_ERR_TOO_LARGE = 10
SK_FP32, SK_FP64 = 0, 1
SK_METHOD_NFFT, SK_METHOD_DIRECT = 0, 1
SK_DOMAIN_SCALING, SK_DOMAIN_LOG = 0, 1
SK_KERNELS_SIMT, SK_KERNELS_TENSOR = 0, 1
SK_FFT_PASSES, SK_FFT_PLANES = 0, 1
SK_FAULT_NONE, SK_FAULT_TC_WAIT = 0, 1
SK_SET_X, SK_SET_Y = 0, 1
SK_STAGE_SPREAD, SK_STAGE_FFT, SK_STAGE_INTERP, SK_STAGE_OTHER, SK_STAGE_DIRECT, SK_STAGE_NEAR = 0, 1, 2, 3, 4, 5
SK_NSTAGES = 6
STAGE_NAMES = ("spread", "fft", "interp", "other", "direct", "near")


class sk_nfft_params(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("sigma", ctypes.c_double), ("m_w", ctypes.c_int), ("p", ctypes.c_int),
                ("eps_B", ctypes.c_double), ("eps_I", ctypes.c_double), ("precision", ctypes.c_int),
                ("user_geometry", ctypes.c_int), ("center", ctypes.c_double * 3), ("scale", ctypes.c_double)]


class sk_result(ctypes.Structure):
    _fields_ = [("s", ctypes.c_double), ("s_upper", ctypes.c_double), ("err_row", ctypes.c_double),
                ("err_col", ctypes.c_double), ("marg_err", ctypes.c_double), ("iters", ctypes.c_int),
                ("total_iters", ctypes.c_int)]


class sk_info(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("n", ctypes.c_int64), ("m", ctypes.c_int64), ("N", ctypes.c_int),
                ("n_os", ctypes.c_int), ("m_w", ctypes.c_int), ("p", ctypes.c_int), ("precision", ctypes.c_int),
                ("nearfield", ctypes.c_int), ("eps", ctypes.c_double), ("r", ctypes.c_double),
                ("eps_scaled", ctypes.c_double), ("center", ctypes.c_double * 3), ("scale", ctypes.c_double),
                ("eps_B", ctypes.c_double), ("eps_I", ctypes.c_double), ("n_subproblems_x", ctypes.c_int),
                ("n_subproblems_y", ctypes.c_int), ("device_bytes", ctypes.c_int64), ("tensor_cores", ctypes.c_int),
                ("fft_planes", ctypes.c_int)]


_P = ctypes.c_void_p
_D = ctypes.c_void_p          # double* (host or device)
_S = ctypes.c_void_p          # cudaStream_t
_SIGS = {
    "sk_error_string": (ctypes.c_char_p, [ctypes.c_int]),
    "sk_last_error": (ctypes.c_char_p, []),
    "sk_default_params": (ctypes.c_int, [ctypes.POINTER(sk_nfft_params)]),
    "sk_init": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.c_int64, _D, _D, ctypes.c_int64, _D, _D,
                               ctypes.c_double, ctypes.c_double, ctypes.POINTER(sk_nfft_params), _S]),
    "sk_destroy": (None, [_P]),
    "sk_set_method": (ctypes.c_int, [_P, ctypes.c_int]),
    "sk_set_domain": (ctypes.c_int, [_P, ctypes.c_int]),
    "sk_set_kernels": (ctypes.c_int, [_P, ctypes.c_int]),
    "sk_set_fft": (ctypes.c_int, [_P, ctypes.c_int]),
    "sk_inject_fault": (ctypes.c_int, [_P, ctypes.c_int]),
    "sk_autotune": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), _S]),
    "sk_kernel_apply": (ctypes.c_int, [_P, ctypes.c_int, _D, _D, _S]),
    "sk_solve": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_double, ctypes.c_int, _D, _D,
                                ctypes.POINTER(sk_result), _S]),
    "sk_grad": (ctypes.c_int, [_P, _D, _D, _D, _D, _S]),
    "sk_solve_batch": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.c_int, ctypes.POINTER(sk_result), _S]),
    "sk_divergence": (ctypes.c_int, [ctypes.c_int, ctypes.c_int64, _D, _D, ctypes.c_int64, _D, _D, ctypes.c_double,
                                     ctypes.c_double, ctypes.POINTER(sk_nfft_params), ctypes.c_int, ctypes.c_double,
                                     _D, _D, _D, _D, _D, _S]),
    "sk_get_state": (ctypes.c_int, [_P, _D, _D, ctypes.POINTER(ctypes.c_int)]),
    "sk_set_state": (ctypes.c_int, [_P, _D, _D, ctypes.c_int]),
    "sk_plan_info": (ctypes.c_int, [_P, ctypes.POINTER(sk_info)]),
    "sk_fourier_coefficients": (ctypes.c_int, [_P, _D, _S]),
    "sk_adjoint_nfft": (ctypes.c_int, [_P, ctypes.c_int, _D, _D, _S]),
    "sk_nfft": (ctypes.c_int, [_P, ctypes.c_int, _D, _D, _S]),
    "sk_spectrum": (ctypes.c_int, [_P, ctypes.c_int, _D, _D, _S]),
    "sk_apply_spectrum": (ctypes.c_int, [_P, ctypes.c_int, _D, _D, _S]),
    "sk_stage_times": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_int64)]),
    "sk_launch_count": (ctypes.c_int64, [_P]),
    "sk_fp32_peak": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(ctypes.c_int), _S]),
    "sk_direct_residual_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int64, _D, _D, _D, ctypes.c_int64, _D, _D,
                                                  ctypes.c_double, ctypes.c_double, _D, _D, _S]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


class SkError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        detail = _lib.sk_last_error().decode() if status in (SK_ERR_CUDA, SK_ERR_NOMEM) else ""
        super().__init__("%s: %s (status %d)%s" % (where, _lib.sk_error_string(status).decode(), status,
                                                    " [" + detail + "]" if detail else ""))


def _check(status, where):
    if status != SK_OK:
        raise SkError(status, where)
    return status


def _ptr(arr, n=None, name="array"):
    """Raw pointer of a float64 contiguous tensor / ndarray (None -> NULL)."""
    if arr is None:
        return None
    if hasattr(arr, "data_ptr"):
        import torch
        if arr.dtype != torch.float64 or not arr.is_contiguous():
            raise TypeError("%s must be a contiguous float64 tensor" % name)
        if n is not None and arr.numel() != n:
            raise ValueError("%s must have %d elements, has %d" % (name, n, arr.numel()))
        return arr.data_ptr()
    if not isinstance(arr, np.ndarray) or arr.dtype != np.float64 or not arr.flags["C_CONTIGUOUS"]:
        raise TypeError("%s must be a C-contiguous float64 ndarray" % name)
    if n is not None and arr.size != n:
        raise ValueError("%s must have %d elements, has %d" % (name, n, arr.size))
    return arr.ctypes.data


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def sk_error_string(status):
    return _lib.sk_error_string(status).decode()


def sk_last_error():
    return _lib.sk_last_error().decode()


def sk_default_params(**overrides):
    p = sk_nfft_params()
    _check(_lib.sk_default_params(ctypes.byref(p)), "sk_default_params")
    for k, v in overrides.items():
        if k == "center":
            for t, c in enumerate(v):
                p.center[t] = c
        else:
            setattr(p, k, v)
    return p


class Plan:
    """Owning handle of an sk_plan*; sk_destroy runs on close() or garbage collection."""

    def __init__(self, handle, d, n, m):
        self.handle = handle
        self.d, self.n, self.m = d, n, m

    def close(self):
        if self.handle:
            _lib.sk_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def sk_init(x, a, y, b, eps, r, params=None, stream=None):
    n, d = x.shape
    m = y.shape[0]
    h = _P()
    prm = ctypes.byref(params) if params is not None else None
    st = _lib.sk_init(ctypes.byref(h), int(d), int(n), _ptr(x, n * d, "x"), _ptr(a, n, "a"), int(m),
                      _ptr(y, m * d, "y"), _ptr(b, m, "b"), float(eps), float(r), prm, _stream(stream))
    _check(st, "sk_init")
    return Plan(h, int(d), int(n), int(m))


def sk_destroy(plan):
    plan.close()


def sk_set_method(plan, method):
    _check(_lib.sk_set_method(plan.handle, int(method)), "sk_set_method")


def sk_set_domain(plan, domain):
    _check(_lib.sk_set_domain(plan.handle, int(domain)), "sk_set_domain")


def sk_set_kernels(plan, kernels):
    _check(_lib.sk_set_kernels(plan.handle, int(kernels)), "sk_set_kernels")


def sk_set_fft(plan, form):
    _check(_lib.sk_set_fft(plan.handle, int(form)), "sk_set_fft")


def sk_autotune(plan, stream=None):
    """Keeps the faster interpolation kernel kind for the plan; returns it."""
    chosen = ctypes.c_int(0)
    _check(_lib.sk_autotune(plan.handle, ctypes.byref(chosen), _stream(stream)), "sk_autotune")
    return chosen.value


def sk_inject_fault(plan, kind):
    _check(_lib.sk_inject_fault(plan.handle, int(kind)), "sk_inject_fault")


def sk_kernel_apply(plan, transpose, vin, out, stream=None):
    nin, nout = (plan.n, plan.m) if transpose else (plan.m, plan.n)
    _check(_lib.sk_kernel_apply(plan.handle, int(transpose), _ptr(vin, nin, "in"), _ptr(out, nout, "out"),
                                _stream(stream)), "sk_kernel_apply")
    return out


def sk_solve(plan, max_iter, tol=0.0, check_every=10, u_out=None, v_out=None, result=True, stream=None,
             raise_on_error=True):
    """Returns (status, result dict or None)."""
    res = sk_result() if result else None
    st = _lib.sk_solve(plan.handle, int(max_iter), float(tol), int(check_every), _ptr(u_out, plan.n, "u_out"),
                       _ptr(v_out, plan.m, "v_out"), ctypes.byref(res) if res is not None else None,
                       _stream(stream))
    if raise_on_error and st not in (SK_OK, SK_ERR_NOT_CONVERGED):
        raise SkError(st, "sk_solve")
    out = None
    if res is not None:
        out = {f: getattr(res, f) for f, _ in sk_result._fields_}
    return st, out


def sk_solve_batch(plans, max_iter, result=True, stream=None, raise_on_error=True):
    """Returns (status, list of result dicts or None); see include/sk.h."""
    arr = (_P * len(plans))(*[p.handle for p in plans])
    res = (sk_result * len(plans))() if result else None
    st = _lib.sk_solve_batch(arr, len(plans), int(max_iter), res, _stream(stream))
    if raise_on_error and st != SK_OK:
        raise SkError(st, "sk_solve_batch")
    out = None
    if result:
        out = [{f: getattr(r, f) for f, _ in sk_result._fields_} for r in res]
    return st, out


def sk_grad(plan, grad_a=None, grad_b=None, grad_x=None, grad_y=None, stream=None):
    """Gradient of the value at the plan's current state (see include/sk.h);
    grad_x / grad_y are n x d / m x d row-major."""
    _check(_lib.sk_grad(plan.handle, _ptr(grad_a, plan.n, "grad_a"), _ptr(grad_b, plan.m, "grad_b"),
                        _ptr(grad_x, plan.n * plan.d, "grad_x"), _ptr(grad_y, plan.m * plan.d, "grad_y"),
                        _stream(stream)), "sk_grad")


def sk_divergence(x, a, y, b, eps, r, max_iter, tol=0.0, params=None, grad_a=None, grad_b=None, grad_x=None,
                  grad_y=None, stream=None):
    """Returns (sd, s_xy, s_xx, s_yy) and fills the optional gradients; see include/sk.h."""
    n, d = x.shape
    m = y.shape[0]
    out = np.zeros(4)
    prm = ctypes.byref(params) if params is not None else None
    st = _lib.sk_divergence(int(d), int(n), _ptr(x, n * d, "x"), _ptr(a, n, "a"), int(m), _ptr(y, m * d, "y"),
                            _ptr(b, m, "b"), float(eps), float(r), prm, int(max_iter), float(tol), out.ctypes.data,
                            _ptr(grad_a, n, "grad_a"), _ptr(grad_b, m, "grad_b"), _ptr(grad_x, n * d, "grad_x"),
                            _ptr(grad_y, m * d, "grad_y"), _stream(stream))
    if st not in (SK_OK, SK_ERR_NOT_CONVERGED):
        _check(st, "sk_divergence")
    return tuple(float(v) for v in out)


def sk_get_state(plan, u=None, v=None):
    it = ctypes.c_int(0)
    _check(_lib.sk_get_state(plan.handle, _ptr(u, plan.n, "u"), _ptr(v, plan.m, "v"), ctypes.byref(it)),
           "sk_get_state")
    return it.value


def sk_set_state(plan, u=None, v=None, iters=0):
    _check(_lib.sk_set_state(plan.handle, _ptr(u, plan.n, "u"), _ptr(v, plan.m, "v"), int(iters)), "sk_set_state")


def sk_plan_info(plan):
    info = sk_info()
    _check(_lib.sk_plan_info(plan.handle, ctypes.byref(info)), "sk_plan_info")
    out = {}
    for f, _ in sk_info._fields_:
        v = getattr(info, f)
        out[f] = list(v) if f == "center" else v
    return out


def sk_fourier_coefficients(plan, out, stream=None):
    _check(_lib.sk_fourier_coefficients(plan.handle, _ptr(out, name="out"), _stream(stream)),
           "sk_fourier_coefficients")
    return out


def sk_adjoint_nfft(plan, which, w, fhat, stream=None):
    n = plan.n if which == SK_SET_X else plan.m
    _check(_lib.sk_adjoint_nfft(plan.handle, int(which), _ptr(w, n, "w"), _ptr(fhat, name="fhat"),
                                _stream(stream)), "sk_adjoint_nfft")
    return fhat


def sk_nfft(plan, which, fhat, f, stream=None):
    n = plan.n if which == SK_SET_X else plan.m
    _check(_lib.sk_nfft(plan.handle, int(which), _ptr(fhat, name="fhat"), _ptr(f, n, "f"), _stream(stream)),
           "sk_nfft")
    return f


def spectrum_size(plan):
    """Number of complex values of a spectrum of this plan, (N+1)^d."""
    info = sk_plan_info(plan)
    return (info["N"] + 1) ** info["d"]


def sk_spectrum(plan, which, w, spec, stream=None):
    """Adjoint NFFT of w on cloud `which` into spec ((N+1)^d interleaved complex); see include/sk.h."""
    n = plan.n if which == SK_SET_X else plan.m
    _check(_lib.sk_spectrum(plan.handle, int(which), _ptr(w, n, "w"), _ptr(spec, 2 * spectrum_size(plan), "spec"),
                            _stream(stream)), "sk_spectrum")
    return spec


def sk_apply_spectrum(plan, which, spec, out, stream=None):
    """Outer sum of Eq. (fastsum) with the plan's b_k, from a (summed) spectrum, at cloud `which`."""
    n = plan.n if which == SK_SET_X else plan.m
    _check(_lib.sk_apply_spectrum(plan.handle, int(which), _ptr(spec, 2 * spectrum_size(plan), "spec"),
                                  _ptr(out, n, "out"), _stream(stream)), "sk_apply_spectrum")
    return out


def sk_stage_times(plan, enable):
    ms = (ctypes.c_double * SK_NSTAGES)()
    cnt = (ctypes.c_int64 * SK_NSTAGES)()
    _check(_lib.sk_stage_times(plan.handle, int(enable), ms, cnt), "sk_stage_times")
    return {STAGE_NAMES[s]: (ms[s], cnt[s]) for s in range(SK_NSTAGES)}


def sk_launch_count(plan):
    return int(_lib.sk_launch_count(plan.handle))


def sk_fp32_peak(packed=False, iters=20000, stream=None):
    """Measured FP32 FMA rate of the current device: (TFLOP/s, SM count)."""
    tf = ctypes.c_double(0.0)
    sms = ctypes.c_int(0)
    _check(_lib.sk_fp32_peak(int(bool(packed)), int(iters), ctypes.byref(tf), ctypes.byref(sms), _stream(stream)),
           "sk_fp32_peak")
    return tf.value, sms.value


def sk_direct_residual_noalloc(x, u, a, y, v, eps, r, t_out, stats_out, stream=None):
    """Direct-sum t = K v plus (sum (u t - a)^2, sum u t) into caller-owned device
    buffers, with no device allocation (see include/sk.h)."""
    n, d = x.shape
    m = y.shape[0]
    _check(_lib.sk_direct_residual_noalloc(int(d), int(n), _ptr(x, n * d, "x"), _ptr(u, n, "u"), _ptr(a, n, "a"),
                                           int(m), _ptr(y, m * d, "y"), _ptr(v, m, "v"), float(eps), float(r),
                                           _ptr(t_out, n, "t_out"), _ptr(stats_out, 2, "stats_out"),
                                           _stream(stream)), "sk_direct_residual_noalloc")
    return t_out, stats_out


def _divergence_function():
    """torch.autograd.Function over sk_divergence (built on first use, so that
    importing this module does not require torch)."""
    import torch

    class SinkhornDivergence(torch.autograd.Function):
        """Sinkhorn divergence S = s(x, y) - s(x, x)/2 - s(y, y)/2 as a function
        of the positions and weights (CUDA float64 tensors).  The forward pass
        solves the three problems through sk_divergence, which also returns the
        gradients (the dual variables and the position gradients at the final
        iterates, see sk_grad); the backward pass scales those by the incoming
        gradient.  No iterate is stored."""

        @staticmethod
        def forward(ctx, x, a, y, b, eps, r, max_iter, tol, params):
            x, a, y, b = (t.detach().contiguous() for t in (x, a, y, b))
            ga, gb = torch.zeros_like(a), torch.zeros_like(b)
            gx, gy = torch.zeros_like(x), torch.zeros_like(y)
            sd, _, _, _ = sk_divergence(x, a, y, b, eps, r, max_iter, tol, params, grad_a=ga, grad_b=gb,
                                        grad_x=gx, grad_y=gy)
            ctx.save_for_backward(gx, ga, gy, gb)
            return torch.tensor(sd, dtype=torch.float64, device=x.device)

        @staticmethod
        def backward(ctx, g):
            gx, ga, gy, gb = ctx.saved_tensors
            return g * gx, g * ga, g * gy, g * gb, None, None, None, None, None

    return SinkhornDivergence


_SinkhornDivergence = None


def sinkhorn_divergence(x, a, y, b, eps, r=2.0, max_iter=200, tol=0.0, params=None):
    """Differentiable Sinkhorn divergence of (x, a) and (y, b): x is n x d, y is
    m x d, a and b the weights, all CUDA float64 tensors.  Returns a 0-d tensor;
    torch.autograd gives its gradient with respect to all four."""
    global _SinkhornDivergence
    if _SinkhornDivergence is None:
        _SinkhornDivergence = _divergence_function()
    return _SinkhornDivergence.apply(x, a, y, b, eps, r, max_iter, tol, params)
