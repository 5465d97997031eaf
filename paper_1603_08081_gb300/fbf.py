"""Thin ctypes binding over ``libfbf.so`` (the C ABI declared in ``include/fbf.h``).

Argument marshalling only: every step of the filter runs in the library's CUDA
kernels or its host FP64 fit.  PyTorch supplies device memory and the current
stream.  Importing this module loads the library and raises if it has not been
built; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import math
import os

from . import build as _build

KMAX = 256
WMAX = 48

FBF_OK, FBF_ERR_INVALID_ARGUMENT, FBF_ERR_NOT_CONVERGED, FBF_ERR_RANGE = 0, 1, 2, 3
FBF_ERR_UNSUPPORTED, FBF_ERR_CUDA, FBF_ERR_TIMEOUT = 4, 5, 6
FBF_RANGE_GAUSSIAN, FBF_RANGE_EXPONENTIAL = 0, 1
FBF_SPATIAL_GAUSSIAN, FBF_SPATIAL_BOX, FBF_SPATIAL_GAUSSIAN_RECURSIVE = 0, 1, 2
FBF_BORDER_REFLECT, FBF_BORDER_TRUNCATE = 0, 1
FBF_U8, FBF_F32 = 0, 1
FBF_FORM_AUTO, FBF_FORM_FP32, FBF_FORM_TC_FP16, FBF_FORM_TC_BF16, FBF_FORM_TC_FP16_SINGLE = 0, 1, 2, 3, 4
FBF_FORM_TC_BF16_SINGLE = 5

SCHEDULES = ["persistent", "persistent_wide", "per_image_fp32", "per_image_form", "per_image_fp32_streams",
             "per_image_form_streams", "persistent_tc"]

_NAMES = {"gaussian": 0, "exponential": 1, "box": 1, "gaussian_recursive": 2, "reflect": 0, "truncate": 1,
          "auto": 0, "fp32": 1, "tc_fp16": 2, "tc_bf16": 3, "tc_fp16_single": 4, "tc_bf16_single": 5}


class fbf_coeffs(C.Structure):
    _fields_ = [("K", C.c_int), ("levels", C.c_int), ("T", C.c_double), ("omega", C.c_double),
                ("resid_l2", C.c_double), ("resid_linf", C.c_double), ("d", C.c_double * KMAX)]

    @property
    def coefficients(self):
        return [self.d[k] for k in range(self.K)]

    def __repr__(self):
        return "fbf_coeffs(K=%d, T=%g, resid_l2=%.3g, resid_linf=%.3g)" % (
            self.K, self.T, self.resid_l2, self.resid_linf)


class fbf_params(C.Structure):
    _fields_ = [("spatial", C.c_int), ("sigma_s", C.c_double), ("W", C.c_int), ("border", C.c_int),
                ("form", C.c_int), ("coeffs", C.POINTER(fbf_coeffs))]


class fbf_image_desc(C.Structure):
    _fields_ = [("d_in", C.c_void_p), ("d_out", C.c_void_p), ("H", C.c_int), ("Wd", C.c_int),
                ("in_pitch", C.c_size_t), ("out_pitch", C.c_size_t), ("spatial", C.c_int),
                ("sigma_s", C.c_double), ("W", C.c_int), ("range", C.c_int), ("sigma_r", C.c_double),
                ("T", C.c_double), ("eps", C.c_double), ("K_fixed", C.c_int), ("levels", C.c_int)]


class FbfError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__("%s%s" % (what + ": " if what else "", fbf_status_string(status)))


def _load():
    path = _build.lib_path()
    if not os.path.exists(path):
        raise ImportError("libfbf.so is not built (%s); run `python -m paper_1603_08081_gb300.build`"
                          " or __graft_entry__.build()" % path)
    lib = C.CDLL(path)
    i, d, p, sz = C.c_int, C.c_double, C.c_void_p, C.c_size_t
    lib.fbf_fit_coeffs.argtypes = [i, d, d, d, i, i, C.POINTER(fbf_coeffs)]
    lib.fbf_fit_coeffs.restype = i
    lib.fbf_fit_coeffs_samples.argtypes = [C.POINTER(C.c_double), i, d, d, i, C.POINTER(fbf_coeffs)]
    lib.fbf_fit_coeffs_samples.restype = i
    lib.fbf_filter.argtypes = [C.POINTER(fbf_params), p, i, i, i, sz, p, sz, p]
    lib.fbf_filter.restype = i
    lib.fbf_filter_backward.argtypes = [C.POINTER(fbf_params), p, p, p, p, i, i, sz, p]
    lib.fbf_filter_backward.restype = i
    lib.fbf_filter_backward_noalloc.argtypes = [C.POINTER(fbf_params), p, p, p, p, i, i, sz, p]
    lib.fbf_filter_backward_noalloc.restype = i
    lib.fbf_filter_stack.argtypes = [C.POINTER(fbf_params), p, i, i, i, i, sz, sz, p, sz, sz, p]
    lib.fbf_filter_stack.restype = i
    lib.fbf_filter_backward_stack.argtypes = [C.POINTER(fbf_params), p, p, p, i, i, i, sz, sz, p]
    lib.fbf_filter_backward_stack.restype = i
    lib.fbf_plan_create.argtypes = [C.POINTER(fbf_image_desc), i, i, i, C.POINTER(p)]
    lib.fbf_plan_create.restype = i
    lib.fbf_plan_create_schedule.argtypes = [C.POINTER(fbf_image_desc), i, i, i, i, C.POINTER(p)]
    lib.fbf_plan_create_schedule.restype = i
    lib.fbf_filter_batched.argtypes = [p, p]
    lib.fbf_filter_batched.restype = i
    lib.fbf_plan_destroy.argtypes = [p]
    lib.fbf_plan_destroy.restype = i
    lib.fbf_plan_size.argtypes = [p, C.POINTER(i), C.POINTER(i)]
    lib.fbf_plan_size.restype = i
    lib.fbf_plan_schedule.argtypes = [p, C.POINTER(i), C.POINTER(d)]
    lib.fbf_plan_schedule.restype = i
    lib.fbf_local_range.argtypes = [p, i, i, i, sz, i, p, p]
    lib.fbf_local_range.restype = i
    lib.fbf_resolve_window.argtypes = [C.POINTER(fbf_params)]
    lib.fbf_resolve_window.restype = i
    lib.fbf_set_wait_limit.argtypes = [C.c_longlong]
    lib.fbf_set_wait_limit.restype = i
    lib.fbf_device_error.argtypes = [C.POINTER(C.c_uint)]
    lib.fbf_device_error.restype = i
    lib.fbf_measure_fp32_peak.argtypes = [i, i, C.POINTER(C.c_double)]
    lib.fbf_measure_fp32_peak.restype = i
    lib.fbf_status_string.argtypes = [i]
    lib.fbf_status_string.restype = C.c_char_p
    lib.fbf_version.argtypes = []
    lib.fbf_version.restype = i
    return lib


lib = _load()


def _enum(v) -> int:
    return _NAMES[v.lower()] if isinstance(v, str) else int(v)


def fbf_status_string(status: int) -> str:
    return lib.fbf_status_string(int(status)).decode()


def fbf_version() -> int:
    return int(lib.fbf_version())


def fbf_fit_coeffs(kernel="gaussian", sigma_r: float = 30.0, T: float = 255.0, eps: float = 1e-3,
                   K_fixed: int = 0, levels: int = 0, allow_not_converged: bool = False) -> fbf_coeffs:
    """Algorithm 2 on the host in FP64 (see fbf.h)."""
    out = fbf_coeffs()
    st = lib.fbf_fit_coeffs(_enum(kernel), float(sigma_r), float(T), float(eps), int(K_fixed),
                            int(levels), C.byref(out))
    if st != FBF_OK and not (st == FBF_ERR_NOT_CONVERGED and allow_not_converged):
        raise FbfError(st, "fbf_fit_coeffs")
    return out


def fbf_fit_coeffs_samples(phi, T: float, eps: float = 1e-3, K_fixed: int = 0,
                           allow_not_converged: bool = False) -> fbf_coeffs:
    """Algorithm 2 for a range kernel given by samples phi(t_l), t_l = l T / (L - 1)
    (see fbf.h)."""
    vals = [float(v) for v in phi]
    arr = (C.c_double * max(len(vals), 1))(*vals)
    out = fbf_coeffs()
    st = lib.fbf_fit_coeffs_samples(arr, len(vals), float(T), float(eps), int(K_fixed), C.byref(out))
    if st != FBF_OK and not (st == FBF_ERR_NOT_CONVERGED and allow_not_converged):
        raise FbfError(st, "fbf_fit_coeffs_samples")
    return out


def make_params(coeffs: fbf_coeffs, sigma_s: float = 3.0, W: int = 0, spatial="gaussian",
                border="reflect", form="fp32") -> fbf_params:
    p = fbf_params()
    p.spatial = _enum(spatial)
    p.sigma_s = float(sigma_s)
    p.W = int(W)
    p.border = _enum(border)
    p.form = _enum(form)
    p.coeffs = C.pointer(coeffs)
    p._keep = coeffs  # keep the struct alive with the params
    return p


def fbf_resolve_window(params: fbf_params) -> int:
    return int(lib.fbf_resolve_window(C.byref(params)))


def _stream_handle(stream):
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(int(stream.cuda_stream))


def fbf_filter(params: fbf_params, x, out=None, stream=None):
    """Filter a 2-D CUDA tensor (uint8 or float32), or a 3-D stack (N, H, W) of
    images under the same parameters (fbf_filter_stack).  Returns the float32
    output of the same shape.

    Rows may be padded (any row stride); columns must be contiguous.
    """
    import torch

    if x.dim() == 3 and x.is_cuda:
        return _filter_stack(params, x, out, stream)
    if x.dim() != 2 or not x.is_cuda:
        raise ValueError("fbf_filter expects a 2-D (or 3-D stacked) CUDA tensor")
    if x.dtype == torch.uint8:
        dt, esz = FBF_U8, 1
    elif x.dtype == torch.float32:
        dt, esz = FBF_F32, 4
    else:
        raise TypeError("fbf_filter: dtype must be uint8 or float32")
    if x.stride(1) != 1:
        x = x.contiguous()
    H, Wd = x.shape
    if out is None:
        out = torch.empty((H, Wd), dtype=torch.float32, device=x.device)
    if out.dtype != torch.float32 or out.dim() != 2 or out.shape != x.shape or out.stride(1) != 1:
        raise ValueError("fbf_filter: out must be float32 (H, W) with contiguous rows")
    st = lib.fbf_filter(C.byref(params), C.c_void_p(x.data_ptr()), dt, H, Wd,
                        x.stride(0) * esz, C.c_void_p(out.data_ptr()), out.stride(0) * 4,
                        _stream_handle(stream))
    if st != FBF_OK:
        raise FbfError(st, "fbf_filter")
    return out


def fbf_local_range(x, W: int, out=None, stream=None) -> int:
    """Dynamic range T of a uint8 CUDA image over the window [-W, W]^2 (see
    include/fbf.h).  Writes it to `out` (a 1-element int32 CUDA tensor, allocated
    when None) and returns it as an int (synchronises the stream)."""
    import torch

    if x.dim() != 2 or not x.is_cuda or x.dtype != torch.uint8:
        raise TypeError("fbf_local_range expects a 2-D uint8 CUDA tensor")
    if x.stride(1) != 1:
        x = x.contiguous()
    if out is None:
        out = torch.empty(1, dtype=torch.int32, device=x.device)
    H, Wd = x.shape
    sh = _stream_handle(stream)
    st = lib.fbf_local_range(C.c_void_p(x.data_ptr()), FBF_U8, H, Wd, x.stride(0), int(W),
                             C.c_void_p(out.data_ptr()), sh)
    if st != FBF_OK:
        raise FbfError(st, "fbf_local_range")
    (stream or torch.cuda.current_stream()).synchronize()
    return int(out.item())


def _filter_stack(params, x, out, stream):
    import torch

    if x.dtype == torch.uint8:
        dt, esz = FBF_U8, 1
    elif x.dtype == torch.float32:
        dt, esz = FBF_F32, 4
    else:
        raise TypeError("fbf_filter: dtype must be uint8 or float32")
    x = x.contiguous()
    N, H, Wd = x.shape
    if out is None:
        out = torch.empty((N, H, Wd), dtype=torch.float32, device=x.device)
    if out.dtype != torch.float32 or out.shape != x.shape or not out.is_contiguous():
        raise ValueError("fbf_filter: out must be a contiguous float32 (N, H, W) tensor")
    st = lib.fbf_filter_stack(C.byref(params), C.c_void_p(x.data_ptr()), dt, N, H, Wd, Wd * esz, H * Wd * esz,
                              C.c_void_p(out.data_ptr()), Wd * 4, H * Wd * 4, _stream_handle(stream))
    if st != FBF_OK:
        raise FbfError(st, "fbf_filter_stack")
    return out


def fbf_filter_backward(params: fbf_params, x, g, grad=None, stream=None):
    """dL/dx for L = sum(g * fbf_filter(params, x)); x and g float32 CUDA, one
    image (H, W) or a stack (N, H, W) (fbf_filter_backward_stack)."""
    import torch

    if x.dtype != torch.float32 or g.dtype != torch.float32 or not (x.is_cuda and g.is_cuda):
        raise TypeError("fbf_filter_backward: x and g must be float32 CUDA tensors")
    x = x.contiguous()
    g = g.contiguous()
    if g.shape != x.shape or x.dim() not in (2, 3):
        raise ValueError("fbf_filter_backward: x and g must have the same 2-D or 3-D shape")
    if grad is None:
        grad = torch.empty_like(x)
    elif (grad.dtype != torch.float32 or grad.shape != x.shape or grad.device != x.device
          or not grad.is_contiguous()):
        # the library writes grad with x's (contiguous) layout
        raise ValueError("fbf_filter_backward: grad must be a contiguous float32 tensor of x's shape and device")
    if x.dim() == 3:
        N, H, Wd = x.shape
        st = lib.fbf_filter_backward_stack(C.byref(params), C.c_void_p(x.data_ptr()), C.c_void_p(g.data_ptr()),
                                           C.c_void_p(grad.data_ptr()), N, H, Wd, Wd * 4, H * Wd * 4,
                                           _stream_handle(stream))
        if st != FBF_OK:
            raise FbfError(st, "fbf_filter_backward_stack")
        return grad
    H, Wd = x.shape
    st = lib.fbf_filter_backward(C.byref(params), C.c_void_p(x.data_ptr()), C.c_void_p(g.data_ptr()), None,
                                 C.c_void_p(grad.data_ptr()), H, Wd, x.stride(0) * 4, _stream_handle(stream))
    if st != FBF_OK:
        raise FbfError(st, "fbf_filter_backward")
    return grad


def _autograd_function():
    import torch

    class FBFFunction(torch.autograd.Function):
        """Differentiable shiftable bilateral filter (in x only): forward is
        fbf_filter (FP32 form, float input), backward the hand-written adjoint;
        x is one image (H, W) or a stack (N, H, W) under the same parameters."""

        @staticmethod
        def forward(ctx, x, params):
            ctx.params = params
            ctx.save_for_backward(x)
            return fbf_filter(params, x.contiguous())

        @staticmethod
        def backward(ctx, g):
            (x,) = ctx.saved_tensors
            return fbf_filter_backward(ctx.params, x, g.contiguous().float()), None

    return FBFFunction


def __getattr__(name):
    if name == "FBFFunction":
        fn = _autograd_function()
        globals()["FBFFunction"] = fn
        return fn
    raise AttributeError(name)


class Plan:
    """A batched-filter plan (fbf_plan_create); keeps its images alive."""

    def __init__(self, handle, keep):
        self.handle = handle
        self._keep = keep

    def size(self):
        ni, nt = C.c_int(0), C.c_int(0)
        st = lib.fbf_plan_size(self.handle, C.byref(ni), C.byref(nt))
        if st != FBF_OK:
            raise FbfError(st, "fbf_plan_size")
        return ni.value, nt.value

    def schedule(self):
        """(name of the replayed schedule, ms measured by autotuning)."""
        k, ms = C.c_int(0), C.c_double(0.0)
        st = lib.fbf_plan_schedule(self.handle, C.byref(k), C.byref(ms))
        if st != FBF_OK:
            raise FbfError(st, "fbf_plan_schedule")
        return SCHEDULES[k.value], ms.value

    def destroy(self):
        if self.handle:
            lib.fbf_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def fbf_plan_create(images, outs, specs, form="fp32", border="reflect", schedule=None, tune_cache=None):
    """images / outs: lists of uint8 / float32 CUDA tensors; specs: list of dicts
    with sigma_s, sigma_r and optionally W, spatial, range, T, eps, K_fixed, levels.
    schedule: None autotunes (fbf_plan_create); a name of SCHEDULES captures
    that schedule only (fbf_plan_create_schedule).
    tune_cache: path of a JSON autotuning cache (tune_cache.py), or None for
    the FBF_TUNE_CACHE environment variable (unset: no cache).  With a cache
    and schedule None, a request seen before on this GPU model captures the
    recorded schedule without autotuning; otherwise the autotuned choice is
    recorded."""
    if schedule is None:
        cache = tune_cache if tune_cache is not None else os.environ.get("FBF_TUNE_CACHE") or None
        if cache:
            return _plan_create_cached(images, outs, specs, form, border, cache)
    n = len(images)
    arr = (fbf_image_desc * max(n, 1))()
    for k, (x, y, sp) in enumerate(zip(images, outs, specs)):
        d = arr[k]
        d.d_in, d.d_out = x.data_ptr(), y.data_ptr()
        d.H, d.Wd = x.shape
        d.in_pitch, d.out_pitch = x.stride(0), y.stride(0) * 4
        d.spatial = _enum(sp.get("spatial", "gaussian"))
        d.sigma_s = float(sp.get("sigma_s", 3.0))
        d.W = int(sp.get("W", 0))
        d.range = _enum(sp.get("range", "gaussian"))
        d.sigma_r = float(sp["sigma_r"])
        d.T = float(sp.get("T", 255.0))
        d.eps = float(sp.get("eps", 1e-3))
        d.K_fixed = int(sp.get("K_fixed", 0))
        d.levels = int(sp.get("levels", 0))
    h = C.c_void_p()
    if schedule is None:
        st = lib.fbf_plan_create(arr, n, _enum(form), _enum(border), C.byref(h))
    else:
        st = lib.fbf_plan_create_schedule(arr, n, _enum(form), _enum(border), SCHEDULES.index(schedule), C.byref(h))
    if st != FBF_OK:
        raise FbfError(st, "fbf_plan_create")
    return Plan(h, (list(images), list(outs)))


def _plan_create_cached(images, outs, specs, form, border, cache):
    import torch

    from . import tune_cache as TC

    dev = images[0].device if images else torch.device("cuda", torch.cuda.current_device())
    gpu = torch.cuda.get_device_name(dev)
    tma_ok = [x.data_ptr() % 16 == 0 and x.stride(0) % 16 == 0 for x in images]
    sig = TC.signature(form, border, [tuple(x.shape) for x in images], tma_ok, specs)
    hit = TC.lookup(cache, gpu, sig)
    if hit is not None and hit["schedule"] in SCHEDULES:
        try:
            return fbf_plan_create(images, outs, specs, form, border, schedule=hit["schedule"])
        except FbfError as e:  # no longer a candidate of the form: autotune again
            if e.status != FBF_ERR_INVALID_ARGUMENT:
                raise
    plan = fbf_plan_create(images, outs, specs, form, border, tune_cache="")
    kind, ms = plan.schedule()
    TC.record(cache, gpu, sig, {"schedule": kind, "ms": round(ms, 4), "form": form, "n_images": len(images)})
    return plan


def fbf_filter_batched(plan: Plan, stream=None):
    st = lib.fbf_filter_batched(plan.handle, _stream_handle(stream))
    if st != FBF_OK:
        raise FbfError(st, "fbf_filter_batched")


def fbf_plan_destroy(plan: Plan):
    plan.destroy()


def fbf_device_error() -> int:
    """Read and clear the device error word (synchronises the device); non-zero
    when a bounded wait inside a kernel gave up (fbf_device_error returns
    FBF_ERR_TIMEOUT then)."""
    v = C.c_uint(0)
    st = lib.fbf_device_error(C.byref(v))
    if st not in (FBF_OK, FBF_ERR_TIMEOUT):
        raise FbfError(st, "fbf_device_error")
    return int(v.value)


def fbf_set_wait_limit(polls: int):
    """Poll limit of the tensor-core kernels' bounded waits (< 0: the default)."""
    st = lib.fbf_set_wait_limit(int(polls))
    if st != FBF_OK:
        raise FbfError(st, "fbf_set_wait_limit")


def fbf_measure_fp32_peak(device: int = 0, packed=None) -> float:
    """Measured FP32 FMA throughput in TFLOP/s (max of scalar and packed when
    packed is None)."""
    vals = []
    for pk in ((0, 1) if packed is None else (int(bool(packed)),)):
        v = C.c_double(0.0)
        st = lib.fbf_measure_fp32_peak(int(device), pk, C.byref(v))
        if st != FBF_OK:
            raise FbfError(st, "fbf_measure_fp32_peak")
        vals.append(v.value)
    return max(vals)


def bilateral_filter(x, sigma_s: float = 3.0, sigma_r: float = 30.0, eps: float = 1e-3,
                     T: float | None = None, kernel="gaussian", K: int = 0, W: int = 0,
                     spatial="gaussian", border="reflect", form="fp32", levels: int = 0):
    """Convenience: fit the coefficients (host) and filter ``x``.

    ``x`` may be a CUDA tensor, or a CPU tensor (pinned for speed), in which case
    it is copied to the current device and the result is copied back.
    """
    import torch

    if T is None:
        T = 255.0 if x.dtype == torch.uint8 else 1.0
    if levels == 0 and T != math.floor(T):
        levels = 256
    c = fbf_fit_coeffs(kernel, sigma_r, T, eps, K, levels)
    p = make_params(c, sigma_s, W, spatial, border, form)
    if x.is_cuda:
        return fbf_filter(p, x)
    xd = x.to("cuda", non_blocking=True)
    y = fbf_filter(p, xd)
    host = torch.empty(y.shape, dtype=y.dtype, pin_memory=True)
    host.copy_(y, non_blocking=True)
    torch.cuda.current_stream().synchronize()
    return host
