"""ctypes wrapper over the FP64 CPU oracle (``oracle/fbf_oracle.c``).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package.  The product library in
``paper_1603_08081_gb300`` never imports it, and this package imports nothing
from there.

The C source is compiled on first use with the system ``gcc`` (plain C99 +
OpenMP, no architecture flags, so the same source builds on x86-64 and aarch64).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fbf_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")

RANGE_GAUSSIAN, RANGE_EXPONENTIAL = 0, 1
SPATIAL_GAUSSIAN, SPATIAL_BOX = 0, 1
BORDER_REFLECT, BORDER_TRUNCATE = 0, 1
KMAX = 256

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library in-tree; returns its path."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c99", "-fopenmp", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            d, i, p, dp, ip, lp = C.c_double, C.c_int, C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int), C.c_long
            lib.orc_num_threads.restype = i
            lib.orc_phi.argtypes = [i, d, d]
            lib.orc_phi.restype = d
            lib.orc_phi_n.argtypes = [dp, i, d, d]
            lib.orc_phi_n.restype = d
            lib.orc_fit_samples.argtypes = [dp, dp, i, d, d, i, i, dp, ip, dp, dp]
            lib.orc_fit_samples.restype = i
            lib.orc_fit.argtypes = [i, d, d, d, i, i, i, dp, ip, dp, dp]
            lib.orc_fit.restype = i
            lib.orc_weights_1d.argtypes = [i, d, i, dp]
            lib.orc_weights_1d.restype = i
            lib.orc_direct.argtypes = [dp, i, i, dp, i, i, i, i, d, dp, i, d, ip, ip, lp, dp, dp, dp]
            lib.orc_direct.restype = None
            lib.orc_alg1.argtypes = [dp, i, i, dp, i, i, dp, i, d, i, i, dp, dp, dp, dp, dp]
            lib.orc_alg1.restype = i
            lib.orc_grad_direct.argtypes = [dp, dp, i, i, dp, i, i, dp, i, d, dp]
            lib.orc_grad_direct.restype = None
            lib.orc_grad_at.argtypes = [dp, dp, i, i, dp, i, i, dp, i, d, ip, ip, lp, dp]
            lib.orc_grad_at.restype = i
            lib.orc_set_threads.argtypes = [i]
            lib.orc_set_threads.restype = None
            lib.orc_local_range.argtypes = [dp, i, i, i, i]
            lib.orc_local_range.restype = d
            lib.orc_rec_kernel.argtypes = [d, C.c_long]
            lib.orc_rec_kernel.restype = d
            lib.orc_rec_coeffs.argtypes = [d, dp, dp, dp]
            lib.orc_rec_coeffs.restype = None
            lib.orc_rec_filter_line.argtypes = [dp, C.c_long, d, dp]
            lib.orc_rec_filter_line.restype = None
            lib.orc_alg1_rec.argtypes = [dp, i, i, d, i, dp, i, d, dp, dp, dp]
            lib.orc_alg1_rec.restype = i
            _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double)) if a is not None else None


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int)) if a is not None else None


def num_threads() -> int:
    return int(_load().orc_num_threads())


def set_threads(n: int) -> None:
    """Threads of the oracle's parallel loops from now on (for timing)."""
    _load().orc_set_threads(int(n))


def phi(kernel: int, sigma_r: float, t: float) -> float:
    return float(_load().orc_phi(int(kernel), float(sigma_r), float(t)))


def phi_n(d, T: float, t: float) -> float:
    d = np.ascontiguousarray(d, np.float64)
    return float(_load().orc_phi_n(_dp(d), len(d), float(T), float(t)))


class Fit:
    __slots__ = ("d", "K", "E", "linf", "status", "T")

    def __init__(self, d, K, E, linf, status, T):
        self.d, self.K, self.E, self.linf, self.status, self.T = d, K, E, linf, status, T

    @property
    def converged(self) -> bool:
        return self.status == 0

    def __repr__(self):
        return "Fit(K=%d, E=%.3g, linf=%.3g, status=%d)" % (self.K, self.E, self.linf, self.status)


def fit(kernel: int, sigma_r: float, T: float, eps: float = 0.0, K: int = 0,
        levels: int = 0, Kmax: int = KMAX) -> Fit:
    """Least-squares cosine fit (eqs. (6)-(8)); see ``orc_fit`` in the C source."""
    d = np.zeros(KMAX, np.float64)
    Ko, E, li = C.c_int(0), C.c_double(0), C.c_double(0)
    st = _load().orc_fit(int(kernel), float(sigma_r), float(T), float(eps), int(K), int(levels),
                         int(Kmax), _dp(d), C.byref(Ko), C.byref(E), C.byref(li))
    if st < 0:
        raise ValueError("oracle fit: bad arguments")
    return Fit(d[: Ko.value].copy(), Ko.value, E.value, li.value, st, float(T))


def fit_samples(t, b, T: float, eps: float = 0.0, K: int = 0, Kmax: int = KMAX) -> Fit:
    t = np.ascontiguousarray(t, np.float64)
    b = np.ascontiguousarray(b, np.float64)
    d = np.zeros(max(KMAX, len(t)), np.float64)
    Ko, E, li = C.c_int(0), C.c_double(0), C.c_double(0)
    st = _load().orc_fit_samples(_dp(t), _dp(b), len(t), float(T), float(eps), int(K),
                                 int(min(Kmax, len(t))), _dp(d), C.byref(Ko), C.byref(E),
                                 C.byref(li))
    if st < 0:
        raise ValueError("oracle fit_samples: bad arguments")
    return Fit(d[: Ko.value].copy(), Ko.value, E.value, li.value, st, float(T))


def default_W(sigma_s: float) -> int:
    """W = ceil(3 sigma_s) (Sec. I gives W = 3 sigma_s)."""
    return int(np.ceil(3.0 * sigma_s - 1e-12))


def weights_1d(spatial: int, sigma_s: float, W: int) -> np.ndarray:
    w = np.zeros(2 * W + 1, np.float64)
    if _load().orc_weights_1d(int(spatial), float(sigma_s), int(W), _dp(w)) < 0:
        raise ValueError("bad window")
    return w


def _img(f):
    f = np.ascontiguousarray(np.asarray(f, dtype=np.float64))
    assert f.ndim == 2
    return f


def _points(points):
    if points is None:
        return None, None, 0
    ys = np.ascontiguousarray(np.asarray(points[0]), np.int32)
    xs = np.ascontiguousarray(np.asarray(points[1]), np.int32)
    return ys, xs, len(ys)


def direct_bf(f, w1, border: int, kernel: int, sigma_r: float, points=None):
    """Eq. (1) with the exact range kernel.  Returns (out, P, Q)."""
    f = _img(f)
    H, Wd = f.shape
    w1 = np.ascontiguousarray(w1, np.float64)
    W = (len(w1) - 1) // 2
    ys, xs, n = _points(points)
    m = n if ys is not None else H * Wd
    out, P, Q = (np.empty(m, np.float64) for _ in range(3))
    _load().orc_direct(_dp(f), H, Wd, _dp(w1), W, int(border), 0, int(kernel), float(sigma_r),
                       None, 0, 1.0, _ip(ys), _ip(xs), n, _dp(out), _dp(P), _dp(Q))
    if ys is None:
        return out.reshape(H, Wd), P.reshape(H, Wd), Q.reshape(H, Wd)
    return out, P, Q


def direct_sbf(f, w1, border: int, d, T: float, points=None):
    """Eq. (9): eq. (1) with phi_N in place of phi, summed directly.  (out, P, Q)."""
    f = _img(f)
    H, Wd = f.shape
    w1 = np.ascontiguousarray(w1, np.float64)
    W = (len(w1) - 1) // 2
    d = np.ascontiguousarray(d, np.float64)
    ys, xs, n = _points(points)
    m = n if ys is not None else H * Wd
    out, P, Q = (np.empty(m, np.float64) for _ in range(3))
    _load().orc_direct(_dp(f), H, Wd, _dp(w1), W, int(border), 1, 0, 1.0, _dp(d), len(d),
                       float(T), _ip(ys), _ip(xs), n, _dp(out), _dp(P), _dp(Q))
    if ys is None:
        return out.reshape(H, Wd), P.reshape(H, Wd), Q.reshape(H, Wd)
    return out, P, Q


def alg1(f, w1, border: int, d, T: float, rows=None):
    """Algorithm 1 (complex form) on output rows [r0, r1).  Returns
    (out, P, Q, Pim, Qim), each (r1-r0, W)."""
    f = _img(f)
    H, Wd = f.shape
    r0, r1 = (0, H) if rows is None else (int(rows[0]), int(rows[1]))
    w1 = np.ascontiguousarray(w1, np.float64)
    W = (len(w1) - 1) // 2
    d = np.ascontiguousarray(d, np.float64)
    shp = (r1 - r0, Wd)
    out, P, Q, Pi, Qi = (np.empty(shp, np.float64) for _ in range(5))
    st = _load().orc_alg1(_dp(f), H, Wd, _dp(w1), W, int(border), _dp(d), len(d), float(T),
                          r0, r1, _dp(out), _dp(P), _dp(Q), _dp(Pi), _dp(Qi))
    if st != 0:
        raise ValueError("oracle alg1: bad arguments")
    return out, P, Q, Pi, Qi


def grad_direct(f, g, w1, border: int, d, T: float):
    """d/df of sum(g * fhat), fhat from eq. (9); FP64, direct window sums."""
    f = _img(f)
    g = _img(g)
    H, Wd = f.shape
    w1 = np.ascontiguousarray(w1, np.float64)
    W = (len(w1) - 1) // 2
    d = np.ascontiguousarray(d, np.float64)
    out = np.empty((H, Wd), np.float64)
    _load().orc_grad_direct(_dp(f), _dp(g), H, Wd, _dp(w1), W, int(border), _dp(d), len(d),
                            float(T), _dp(out))
    return out


def grad_at(f, g, w1, border: int, d, T: float, points):
    """The gradient of grad_direct evaluated at the given pixels only."""
    f = _img(f)
    g = _img(g)
    H, Wd = f.shape
    w1 = np.ascontiguousarray(w1, np.float64)
    W = (len(w1) - 1) // 2
    d = np.ascontiguousarray(d, np.float64)
    ys, xs, n = _points(points)
    out = np.empty(n, np.float64)
    st = _load().orc_grad_at(_dp(f), _dp(g), H, Wd, _dp(w1), W, int(border), _dp(d), len(d), float(T),
                             _ip(ys), _ip(xs), n, _dp(out))
    if st != 0:
        raise MemoryError("orc_grad_at: could not allocate its preimage lists")
    return out


def local_range(f, W: int, border: int = 0) -> float:
    """Dynamic range T of f over the window [-W, W]^2 (the definition opening
    Sec. III); see ``orc_local_range`` in the C source."""
    f = _img(f)
    H, Wd = f.shape
    return float(_load().orc_local_range(_dp(f), H, Wd, int(W), int(border)))


def bound12(T: float, eps: float, w0: float) -> float:
    """Right-hand side of the accuracy bound, eq. (12): 2 T eps / (w(0) - eps)."""
    return 2.0 * T * eps / (w0 - eps)


def rec_kernel(sigma_s: float, k: int) -> float:
    """Deriche's approximation g(k) of exp(-k^2 / (2 sigma_s^2)), unscaled (the
    recursive Gaussian that Sec. II cites; see the C source)."""
    return float(_load().orc_rec_kernel(float(sigma_s), int(k)))


def rec_coeffs(sigma_s: float):
    """(causal numerator n[0..3], denominator d[0..4] with d[0] = 1, anticausal
    numerator m[0..4] with m[0] = 0) of the recursive Gaussian, unit gain."""
    nc, dd, na = np.zeros(4), np.zeros(5), np.zeros(5)
    _load().orc_rec_coeffs(float(sigma_s), _dp(nc), _dp(dd), _dp(na))
    return nc, dd, na


def rec_filter_line(x, sigma_s: float) -> np.ndarray:
    """One line through the causal + anticausal recursions (zero outside)."""
    x = np.ascontiguousarray(x, np.float64)
    y = np.empty_like(x)
    _load().orc_rec_filter_line(_dp(x), len(x), float(sigma_s), _dp(y))
    return y


def alg1_rec(f, sigma_s: float, border: int, d, T: float):
    """Algorithm 1 with the recursive Gaussian as the convolution (whole image).
    Returns (out, P, Q)."""
    f = _img(f)
    H, Wd = f.shape
    d = np.ascontiguousarray(d, np.float64)
    out, P, Q = (np.empty((H, Wd), np.float64) for _ in range(3))
    st = _load().orc_alg1_rec(_dp(f), H, Wd, float(sigma_s), int(border), _dp(d), len(d), float(T),
                              _dp(out), _dp(P), _dp(Q))
    if st != 0:
        raise ValueError("oracle alg1_rec: bad arguments")
    return out, P, Q
