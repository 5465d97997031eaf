"""Host-side checks of the C ABI: the library loads, exports what include/fbf.h
declares, the host FP64 fit (Algorithm 2) reaches the oracle's least-squares
solution, and argument validation returns the documented status codes before
any device work."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fbf():
    from paper_1603_08081_gb300 import build

    build.build()
    from paper_1603_08081_gb300 import fbf as mod

    return mod


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(fbf_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_library_exports_every_declared_symbol(fbf):
    names = _declared_functions()
    assert "fbf_filter" in names and "fbf_fit_coeffs" in names
    for n in names:
        assert hasattr(fbf.lib, n), n  # ctypes resolves the exported symbol
        assert C.cast(getattr(fbf.lib, n), C.c_void_p).value


@pytest.mark.parametrize("kernel,sigma_r,T,eps,K,levels", [
    ("gaussian", 30.0, 217.0, 1e-8, 0, 0),
    ("gaussian", 30.0, 217.0, 1e-3, 0, 0),
    ("gaussian", 30.0, 255.0, 1e-2, 0, 0),
    ("gaussian", 20.0, 255.0, 1e-3, 0, 0),
    ("gaussian", 40.0, 255.0, 1e-3, 0, 0),
    ("gaussian", 10.0, 255.0, 1e-3, 0, 0),
    ("exponential", 20.0, 255.0, 0.0, 40, 0),
    ("exponential", 20.0, 255.0, 1e-3, 0, 0),
    ("gaussian", 0.1, 1.0, 1e-3, 0, 256),
])
def test_host_fit_matches_oracle(fbf, kernel, sigma_r, T, eps, K, levels):
    c = fbf.fbf_fit_coeffs(kernel, sigma_r, T, eps, K, levels)
    o = O.fit(0 if kernel == "gaussian" else 1, sigma_r, T, eps, K, levels)
    assert c.K == o.K
    assert np.max(np.abs(np.array(c.coefficients) - o.d)) <= 1e-10
    assert c.resid_l2 == pytest.approx(o.E, rel=1e-8, abs=1e-13)
    assert c.resid_linf == pytest.approx(o.linf, rel=1e-8, abs=1e-13)
    assert c.omega == pytest.approx(np.pi / T)


def _tukey(t, c=60.0):
    # Tukey's biweight: (1 - (t/c)^2)^2 inside |t| <= c, 0 outside (continuous, C^1)
    u = np.clip(np.abs(t) / c, 0.0, 1.0)
    return (1.0 - u * u) ** 2


def _huber(t, k=25.0):
    # Huber-type weight: 1 inside |t| <= k, k/|t| outside (continuous, one kink)
    a = np.abs(t)
    return np.where(a <= k, 1.0, k / np.maximum(a, 1e-300))


@pytest.mark.parametrize("name,phi,T,L,eps,K", [
    ("tukey", _tukey, 255.0, 256, 1e-3, 0),
    ("huber", _huber, 255.0, 256, 1e-3, 0),
    ("lorentz", lambda t: 1.0 / (1.0 + (t / 30.0) ** 2), 255.0, 256, 1e-3, 0),
    ("tukey_fixed", _tukey, 255.0, 256, 0.0, 40),
    ("tukey_unit", lambda t: _tukey(t, 60.0 / 255.0), 1.0, 256, 1e-3, 0),
    ("huber_coarse", _huber, 255.0, 64, 1e-2, 0),
])
def test_fit_from_samples_matches_oracle(fbf, name, phi, T, L, eps, K):
    """Algorithm 2 on user samples of a kernel (Sec. III: any kernel whose Fourier
    series converges pointwise) reaches the oracle's least-squares solution
    (Householder QR of the same samples): same order, d within 1e-10."""
    t = np.arange(L) * T / (L - 1)
    b = phi(t)
    c = fbf.fbf_fit_coeffs_samples(b, T, eps, K)
    o = O.fit_samples(t, b, T, eps, K)
    assert c.K == o.K and c.levels == L
    assert np.max(np.abs(np.array(c.coefficients) - o.d)) <= 1e-10
    assert c.resid_l2 == pytest.approx(o.E, rel=1e-8, abs=1e-13)
    assert c.resid_linf == pytest.approx(o.linf, rel=1e-8, abs=1e-13)
    if K == 0:
        assert c.resid_l2 <= eps and c.resid_linf <= c.resid_l2 * (1 + 1e-12)


def test_fit_from_samples_equals_enum_fit_on_the_same_grid(fbf):
    """Samples of the Gaussian on {0..T} are what fbf_fit_coeffs fits."""
    t = np.arange(256.0)
    for sr, eps in ((20.0, 1e-3), (30.0, 1e-2)):
        a = fbf.fbf_fit_coeffs("gaussian", sr, 255.0, eps)
        b = fbf.fbf_fit_coeffs_samples(np.exp(-t * t / (2 * sr * sr)), 255.0, eps)
        assert a.K == b.K  # (numpy's exp and the library's may differ in the last bit)
        assert np.max(np.abs(np.array(a.coefficients) - np.array(b.coefficients))) <= 1e-13


def test_fit_from_samples_errors(fbf):
    L = fbf.lib
    out = fbf.fbf_coeffs()
    arr = (C.c_double * 4)(1.0, 0.5, 0.2, 0.1)
    assert L.fbf_fit_coeffs_samples(None, 4, 3.0, 1e-3, 0, C.byref(out)) == fbf.FBF_ERR_INVALID_ARGUMENT
    assert L.fbf_fit_coeffs_samples(arr, 1, 3.0, 1e-3, 0, C.byref(out)) == fbf.FBF_ERR_INVALID_ARGUMENT
    assert L.fbf_fit_coeffs_samples(arr, 4, 0.0, 1e-3, 0, C.byref(out)) == fbf.FBF_ERR_INVALID_ARGUMENT
    assert L.fbf_fit_coeffs_samples(arr, 4, 3.0, 0.0, 0, C.byref(out)) == fbf.FBF_ERR_INVALID_ARGUMENT
    assert L.fbf_fit_coeffs_samples(arr, 4, 3.0, 1e-3, 5, C.byref(out)) == fbf.FBF_ERR_RANGE
    assert L.fbf_fit_coeffs_samples(arr, 4, 3.0, 1e-3, 0, None) == fbf.FBF_ERR_INVALID_ARGUMENT
    nan = (C.c_double * 4)(1.0, float("nan"), 0.2, 0.1)
    assert L.fbf_fit_coeffs_samples(nan, 4, 3.0, 1e-3, 0, C.byref(out)) == fbf.FBF_ERR_INVALID_ARGUMENT
    # 4 samples are fitted exactly by 4 columns
    assert L.fbf_fit_coeffs_samples(arr, 4, 3.0, 1e-14, 0, C.byref(out)) in (fbf.FBF_OK, fbf.FBF_ERR_NOT_CONVERGED)
    assert out.K == 4 and out.resid_l2 < 1e-12


def test_host_fit_tables_3_and_4(fbf):
    for eps, N in ((1e-8, 15), (1e-5, 12), (1e-4, 11), (1e-3, 10), (1e-2, 8), (1e-1, 7)):
        assert fbf.fbf_fit_coeffs("gaussian", 30.0, 217.0, eps).K == N


def test_host_fit_errors(fbf):
    out = fbf.fbf_coeffs()
    L = fbf.lib
    assert L.fbf_fit_coeffs(0, 30.0, 255.0, 1e-3, 0, 0, None) == fbf.FBF_ERR_INVALID_ARGUMENT
    assert L.fbf_fit_coeffs(0, -1.0, 255.0, 1e-3, 0, 0, C.byref(out)) == fbf.FBF_ERR_INVALID_ARGUMENT
    assert L.fbf_fit_coeffs(0, 30.0, 0.0, 1e-3, 0, 0, C.byref(out)) == fbf.FBF_ERR_INVALID_ARGUMENT
    assert L.fbf_fit_coeffs(0, 30.0, 2.5, 1e-3, 0, 0, C.byref(out)) == fbf.FBF_ERR_INVALID_ARGUMENT
    assert L.fbf_fit_coeffs(0, 30.0, 255.0, 0.0, 0, 0, C.byref(out)) == fbf.FBF_ERR_INVALID_ARGUMENT
    assert L.fbf_fit_coeffs(7, 30.0, 255.0, 1e-3, 0, 0, C.byref(out)) == fbf.FBF_ERR_INVALID_ARGUMENT
    assert L.fbf_fit_coeffs(0, 30.0, 255.0, 1e-3, 0, 1, C.byref(out)) == fbf.FBF_ERR_INVALID_ARGUMENT
    assert L.fbf_fit_coeffs(0, 30.0, 255.0, 0.0, 300, 0, C.byref(out)) == fbf.FBF_ERR_RANGE
    # eps below what 256 columns reach: filled in, flagged.
    st = L.fbf_fit_coeffs(1, 1.0, 1000.0, 1e-12, 0, 0, C.byref(out))
    assert st == fbf.FBF_ERR_NOT_CONVERGED and out.K == fbf.KMAX


def test_fixed_order_and_full_grid(fbf):
    c = fbf.fbf_fit_coeffs("gaussian", 15.0, 63.0, 0.0, 64)
    assert c.K == 64 and c.resid_l2 < 1e-12
    c = fbf.fbf_fit_coeffs("gaussian", 1e12, 255.0, 1e-6)
    assert c.K == 1 and abs(c.d[0] - 1.0) < 1e-12


def test_filter_validation_without_device_work(fbf):
    """Invalid requests are rejected before any CUDA call (runs without a GPU)."""
    L = fbf.lib
    c = fbf.fbf_fit_coeffs("gaussian", 30.0, 255.0, 1e-2)
    p = fbf.make_params(c, 3.0)
    dummy = C.c_void_p(16)
    nul = C.c_void_p(0)
    st = L.fbf_filter(None, dummy, 0, 4, 4, 4, dummy, 16, nul)
    assert st == fbf.FBF_ERR_INVALID_ARGUMENT
    assert L.fbf_filter(C.byref(p), nul, 0, 4, 4, 4, dummy, 16, nul) == fbf.FBF_ERR_INVALID_ARGUMENT
    assert L.fbf_filter(C.byref(p), dummy, 0, 4, 4, 3, dummy, 16, nul) == fbf.FBF_ERR_INVALID_ARGUMENT
    assert L.fbf_filter(C.byref(p), dummy, 0, 4, 4, 4, dummy, 12, nul) == fbf.FBF_ERR_INVALID_ARGUMENT
    assert L.fbf_filter(C.byref(p), dummy, 0, -1, 4, 4, dummy, 16, nul) == fbf.FBF_ERR_INVALID_ARGUMENT
    assert L.fbf_filter(C.byref(p), dummy, 5, 4, 4, 4, dummy, 16, nul) == fbf.FBF_ERR_INVALID_ARGUMENT
    # empty image: a no-op, no launch
    assert L.fbf_filter(C.byref(p), nul, 0, 0, 4, 4, nul, 16, nul) == fbf.FBF_OK
    assert L.fbf_filter(C.byref(p), nul, 0, 4, 0, 4, nul, 16, nul) == fbf.FBF_OK
    big = fbf.make_params(c, 16.2)  # W = 49 > FBF_WMAX = 48
    assert fbf.fbf_resolve_window(big) == 49
    assert L.fbf_filter(C.byref(big), dummy, 0, 4, 4, 4, dummy, 16, nul) == fbf.FBF_ERR_RANGE
    neg = fbf.make_params(c, -1.0)
    assert L.fbf_filter(C.byref(neg), dummy, 0, 4, 4, 4, dummy, 16, nul) == fbf.FBF_ERR_INVALID_ARGUMENT
    box0 = fbf.make_params(c, 3.0, W=0, spatial="box")
    assert L.fbf_filter(C.byref(box0), dummy, 0, 4, 4, 4, dummy, 16, nul) == fbf.FBF_ERR_INVALID_ARGUMENT
    cf = fbf.fbf_fit_coeffs("gaussian", 0.1, 1.0, 1e-3, levels=256)
    pf = fbf.make_params(cf, 3.0)  # T = 1 is fine for f32 but the u8 path needs integer T >= 1
    assert fbf.fbf_resolve_window(pf) == 9
    bad = fbf.fbf_coeffs()
    bad.K, bad.T = 10, 2.5
    pb = fbf.make_params(bad, 3.0)
    assert L.fbf_filter(C.byref(pb), dummy, 0, 4, 4, 4, dummy, 16, nul) == fbf.FBF_ERR_UNSUPPORTED
    bad.K = 0
    assert L.fbf_filter(C.byref(pb), dummy, 0, 4, 4, 4, dummy, 16, nul) == fbf.FBF_ERR_INVALID_ARGUMENT
    bad.K, bad.T = 300, 255.0
    assert L.fbf_filter(C.byref(pb), dummy, 0, 4, 4, 4, dummy, 16, nul) == fbf.FBF_ERR_RANGE


def test_stack_and_alignment_validation_without_device_work(fbf):
    """Float images must stay 4-byte aligned: a misaligned base pointer or an
    image stride that is not a multiple of 4 is refused before any launch."""
    L = fbf.lib
    c = fbf.fbf_fit_coeffs("gaussian", 30.0, 255.0, 1e-2)
    p = fbf.make_params(c, 3.0)
    nul = C.c_void_p(0)
    a, odd = C.c_void_p(4096), C.c_void_p(4098)
    # fbf_filter: FP32 output (and FP32 input) base pointers
    assert L.fbf_filter(C.byref(p), a, 0, 4, 4, 4, odd, 16, nul) == fbf.FBF_ERR_INVALID_ARGUMENT
    assert L.fbf_filter(C.byref(p), odd, 1, 4, 4, 16, a, 16, nul) == fbf.FBF_ERR_INVALID_ARGUMENT
    # stacks: strides of float images
    assert L.fbf_filter_stack(C.byref(p), a, 0, 2, 4, 4, 4, 16, a, 16, 66, nul) == fbf.FBF_ERR_INVALID_ARGUMENT
    assert L.fbf_filter_stack(C.byref(p), a, 1, 2, 4, 4, 16, 66, a, 16, 64, nul) == fbf.FBF_ERR_INVALID_ARGUMENT
    assert L.fbf_filter_backward_stack(C.byref(p), a, a, a, 2, 4, 4, 16, 66, nul) == fbf.FBF_ERR_INVALID_ARGUMENT
    assert L.fbf_filter_backward_stack(C.byref(p), a, odd, a, 2, 4, 4, 16, 64, nul) == fbf.FBF_ERR_INVALID_ARGUMENT
    assert L.fbf_filter_backward_noalloc(C.byref(p), a, odd, None, a, 4, 4, 16, nul) == fbf.FBF_ERR_INVALID_ARGUMENT


def test_status_strings(fbf):
    for s in range(7):
        assert fbf.fbf_status_string(s).startswith("FBF_")
    assert fbf.fbf_version() >= 100
