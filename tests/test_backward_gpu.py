"""GPU parity of the float-input forward and of the hand-written adjoint
(fbf_filter_backward through the C ABI) against the FP64 oracle.

Tolerances.  Forward: 0.5 gray contract scaled to the image range (T = 1 here:
0.5 / 255), and the FP32 regression bound 1e-4 * T.  Gradient: FP32 sums of
eight channels per harmonic with weights n*omega up to ~40; relative rounding
~1e-6 per term, so 1e-3 of the largest gradient entry leaves a wide margin.
"""
import numpy as np
import pytest

import oracle as O
from paper_1603_08081_gb300.synth import make_grad, make_image_f32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fbf():
    import torch  # noqa: F401

    from paper_1603_08081_gb300 import build

    build.build()
    from paper_1603_08081_gb300 import fbf as mod

    return mod


def _fit(fbf, sigma_r=0.1, T=1.0, eps=1e-3, levels=256):
    return fbf.fbf_fit_coeffs("gaussian", sigma_r, T, eps, 0, levels)


def _w1(sigma_s, W):
    return O.weights_1d(O.SPATIAL_GAUSSIAN, sigma_s, W)


def _bd(border):
    return O.BORDER_REFLECT if border == "reflect" else O.BORDER_TRUNCATE


def _cuda(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


@pytest.mark.parametrize("border", ["reflect", "truncate"])
@pytest.mark.parametrize("shape,sigma_s", [((64, 64), 4.0), ((37, 53), 2.0), ((5, 7), 3.0), ((100, 33), 5.0),
                                           ((1, 40), 1.0), ((70, 90), 7.0), ((45, 61), 10.6), ((9, 6), 6.0)])
def test_float_forward_matches_oracle(fbf, border, shape, sigma_s):
    import torch

    img = make_image_f32(*shape, seed=1400)
    c = _fit(fbf)
    W = int(np.ceil(3 * sigma_s))
    p = fbf.make_params(c, sigma_s, 0, "gaussian", border, "fp32")
    y = fbf.fbf_filter(p, _cuda(img))
    torch.cuda.synchronize()
    ref = O.alg1(img.astype(np.float64), _w1(sigma_s, W), _bd(border), np.array(c.coefficients), 1.0)[0]
    err = np.abs(y.cpu().numpy() - ref).max()
    assert err <= 0.5 / 255 and err <= 1e-4, err


def test_float_forward_arbitrary_T(fbf):
    import torch

    img = make_image_f32(48, 50, seed=3) * np.float32(2.5)
    c = fbf.fbf_fit_coeffs("gaussian", 0.3, 2.5, 1e-4, 0, 300)
    p = fbf.make_params(c, 2.0)
    y = fbf.fbf_filter(p, _cuda(img))
    torch.cuda.synchronize()
    ref = O.alg1(img.astype(np.float64), _w1(2.0, 6), O.BORDER_REFLECT, np.array(c.coefficients), 2.5)[0]
    assert np.abs(y.cpu().numpy() - ref).max() <= 2.5e-4


@pytest.mark.parametrize("border", ["reflect", "truncate"])
@pytest.mark.parametrize("shape,sigma_s,W", [((24, 30), 1.0, 3), ((17, 13), 2.0, 6), ((40, 36), 4.0, 12),
                                             ((6, 9), 2.0, 6), ((9, 4), 1.0, 16), ((30, 41), 6.7, 20),
                                             ((36, 44), 10.0, 32), ((7, 5), 3.0, 20), ((50, 3), 8.0, 24)])
def test_backward_matches_oracle_gradient(fbf, border, shape, sigma_s, W):
    """Full FP64 gradient of sum(g * fhat), eq. (9), incl. windows wider than the
    image, for both kernel tile sets (W <= 16 and 17 <= W <= 32)."""
    import torch

    img = make_image_f32(*shape, seed=1401)
    g = make_grad(*shape, seed=1499)
    c = _fit(fbf)
    p = fbf.make_params(c, sigma_s, W, "gaussian", border, "fp32")
    gr = fbf.fbf_filter_backward(p, _cuda(img), _cuda(g))
    torch.cuda.synchronize()
    ref = O.grad_direct(img.astype(np.float64), g.astype(np.float64), _w1(sigma_s, W), _bd(border),
                        np.array(c.coefficients), 1.0)
    got = gr.cpu().numpy()
    assert np.all(np.isfinite(got))
    assert np.abs(got - ref).max() <= 1e-3 * np.abs(ref).max(), (np.abs(got - ref).max(), np.abs(ref).max())


def test_backward_512_sampled(fbf):
    """One 512x512 image of the differentiation workload (sigma_s = 4, W = 12,
    sigma_r = 0.1, T = 1, 256 levels, eps = 1e-3 -> K = 13): sampled pixels
    (random, corners, edges) against the FP64 gradient at those pixels."""
    import torch

    img = make_image_f32(512, 512, seed=1400)
    g = make_grad(512, 512, seed=1499)
    c = _fit(fbf)
    assert c.K == 13
    p = fbf.make_params(c, 4.0)
    gr = fbf.fbf_filter_backward(p, _cuda(img), _cuda(g))
    torch.cuda.synchronize()
    rng = np.random.default_rng(7)
    ys = np.concatenate([rng.integers(0, 512, 24), [0, 0, 511, 511, 5, 256, 500]])
    xs = np.concatenate([rng.integers(0, 512, 24), [0, 511, 0, 511, 256, 3, 256]])
    ref = O.grad_at(img.astype(np.float64), g.astype(np.float64), _w1(4.0, 12), O.BORDER_REFLECT,
                    np.array(c.coefficients), 1.0, (ys, xs))
    got = gr.cpu().numpy()[ys, xs]
    scale = np.abs(gr.cpu().numpy()).max()
    assert np.abs(got - ref).max() <= 1e-3 * scale


def test_autograd_function_and_finite_differences(fbf):
    """FBFFunction backward equals fbf_filter_backward, and agrees with central
    differences of the GPU forward (FP32, h = 1e-3) at a few pixels."""
    import torch

    img = make_image_f32(32, 40, seed=1402).astype(np.float64)
    g = make_grad(32, 40, seed=1499)
    c = _fit(fbf)
    p = fbf.make_params(c, 2.0)
    x = _cuda(img).requires_grad_(True)
    y = fbf.FBFFunction.apply(x, p)
    (y * _cuda(g)).sum().backward()
    direct = fbf.fbf_filter_backward(p, _cuda(img), _cuda(g))
    torch.cuda.synchronize()
    assert torch.allclose(x.grad, direct, rtol=0, atol=1e-6)
    h = 1e-3
    for (i, j) in ((0, 0), (5, 7), (16, 20), (31, 39), (10, 0)):
        vals = []
        for s in (h, -h):
            im = img.copy()
            im[i, j] += s
            out = fbf.fbf_filter(p, _cuda(im))
            torch.cuda.synchronize()
            vals.append(float((out.double().cpu().numpy() * g).sum()))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - float(direct[i, j])) <= 2e-2 * max(1.0, abs(fd)), (i, j, fd, float(direct[i, j]))


def test_backward_rejects_tensor_core_forms_and_big_windows(fbf):
    import ctypes as C

    c = _fit(fbf)
    x = _cuda(np.zeros((8, 8)))
    p = fbf.make_params(c, 2.0, 0, "gaussian", "reflect", "tc_fp16")
    st = fbf.lib.fbf_filter_backward(C.byref(p), C.c_void_p(x.data_ptr()), C.c_void_p(x.data_ptr()), None,
                                     C.c_void_p(x.data_ptr()), 8, 8, 32, None)
    assert st == fbf.FBF_ERR_UNSUPPORTED
    p = fbf.make_params(c, 11.0)  # W = 33 > 32, the adjoint's window limit
    st = fbf.lib.fbf_filter_backward(C.byref(p), C.c_void_p(x.data_ptr()), C.c_void_p(x.data_ptr()), None,
                                     C.c_void_p(x.data_ptr()), 8, 8, 32, None)
    assert st == fbf.FBF_ERR_RANGE


@pytest.mark.parametrize("form", ["fp32", "tc_fp16", "tc_fp16_single"])
def test_stack_forward_equals_each_image(fbf, form):
    """fbf_filter_stack (3-D input) gives every image exactly what fbf_filter
    gives it alone, for uint8 stacks in every form and float stacks (FP32)."""
    import torch

    from paper_1603_08081_gb300.synth import make_image

    c = fbf.fbf_fit_coeffs("gaussian", 25.0, 255.0, 1e-3)
    p = fbf.make_params(c, 3.0, 0, "gaussian", "reflect", form)
    x = torch.stack([torch.from_numpy(make_image(70, 90, seed=900 + k)) for k in range(5)]).cuda()
    y = fbf.fbf_filter(p, x)
    torch.cuda.synchronize()
    for k in range(5):
        assert torch.equal(y[k], fbf.fbf_filter(p, x[k]))
    if form == "fp32":
        cf = _fit(fbf)
        pf = fbf.make_params(cf, 2.0)
        xf = torch.stack([torch.from_numpy(make_image_f32(40, 75, 950 + k)) for k in range(4)]).cuda()
        yf = fbf.fbf_filter(pf, xf)
        torch.cuda.synchronize()
        for k in range(4):
            assert torch.equal(yf[k], fbf.fbf_filter(pf, xf[k]))


@pytest.mark.parametrize("border", ["reflect", "truncate"])
def test_stack_backward_and_autograd_equal_each_image(fbf, border):
    """fbf_filter_backward_stack and the autograd Function on a (N, H, W) stack
    give every image the gradient of the single-image adjoint, bit for bit."""
    import torch

    c = _fit(fbf)
    p = fbf.make_params(c, 3.0, 0, "gaussian", border)
    x = torch.stack([torch.from_numpy(make_image_f32(48, 66, 960 + k)) for k in range(4)]).cuda()
    g = torch.stack([torch.from_numpy(make_grad(48, 66, 970 + k)) for k in range(4)]).cuda()
    gin = fbf.fbf_filter_backward(p, x, g)
    xr = x.detach().requires_grad_(True)
    (fbf.FBFFunction.apply(xr, p) * g).sum().backward()
    torch.cuda.synchronize()
    for k in range(4):
        single = fbf.fbf_filter_backward(p, x[k], g[k])
        torch.cuda.synchronize()
        assert torch.equal(gin[k], single)
        assert torch.equal(xr.grad[k], single)


def test_stack_arguments(fbf):
    import ctypes as C

    import torch

    c = _fit(fbf)
    p = fbf.make_params(c, 2.0)
    x = torch.zeros((3, 8, 8), dtype=torch.float32, device="cuda")
    px, po = C.c_void_p(x.data_ptr()), C.c_void_p(x.data_ptr())
    lib = fbf.lib
    assert lib.fbf_filter_stack(C.byref(p), px, fbf.FBF_F32, -1, 8, 8, 32, 256, po, 32, 256, None) == \
        fbf.FBF_ERR_INVALID_ARGUMENT
    assert lib.fbf_filter_stack(C.byref(p), px, fbf.FBF_F32, 2, 8, 8, 32, 255, po, 32, 256, None) == \
        fbf.FBF_ERR_INVALID_ARGUMENT
    assert lib.fbf_filter_stack(C.byref(p), px, fbf.FBF_F32, 0, 8, 8, 32, 0, po, 32, 0, None) == fbf.FBF_OK
    assert lib.fbf_filter_backward_stack(C.byref(p), px, px, po, 2, 8, 8, 32, 128, None) == \
        fbf.FBF_ERR_INVALID_ARGUMENT
    assert lib.fbf_filter_backward_stack(C.byref(p), px, None, po, 2, 8, 8, 32, 256, None) == \
        fbf.FBF_ERR_INVALID_ARGUMENT
    pt = fbf.make_params(c, 2.0, 0, "gaussian", "reflect", "tc_fp16")
    assert lib.fbf_filter_backward_stack(C.byref(pt), px, px, po, 2, 8, 8, 32, 256, None) == \
        fbf.FBF_ERR_UNSUPPORTED
    # image strides that would misalign the float images after the first one
    assert lib.fbf_filter_stack(C.byref(p), px, fbf.FBF_F32, 2, 8, 8, 32, 258, po, 32, 256, None) == \
        fbf.FBF_ERR_INVALID_ARGUMENT
    assert lib.fbf_filter_stack(C.byref(p), px, fbf.FBF_F32, 2, 8, 8, 32, 256, po, 32, 258, None) == \
        fbf.FBF_ERR_INVALID_ARGUMENT
    assert lib.fbf_filter_backward_stack(C.byref(p), px, px, po, 2, 8, 8, 32, 258, None) == \
        fbf.FBF_ERR_INVALID_ARGUMENT
    # misaligned float base pointers (input, output, upstream gradient)
    odd = C.c_void_p(x.data_ptr() + 2)
    assert lib.fbf_filter_stack(C.byref(p), odd, fbf.FBF_F32, 1, 8, 8, 32, 256, po, 32, 256, None) == \
        fbf.FBF_ERR_INVALID_ARGUMENT
    assert lib.fbf_filter_stack(C.byref(p), px, fbf.FBF_F32, 1, 8, 8, 32, 256, odd, 32, 256, None) == \
        fbf.FBF_ERR_INVALID_ARGUMENT
    assert lib.fbf_filter_backward_stack(C.byref(p), px, odd, po, 2, 8, 8, 32, 256, None) == \
        fbf.FBF_ERR_INVALID_ARGUMENT
    assert lib.fbf_filter_backward(C.byref(p), px, odd, None, po, 8, 8, 32, None) == fbf.FBF_ERR_INVALID_ARGUMENT
    # a caller-supplied grad of the wrong shape, dtype or layout is refused before the call
    x2, g2 = x[0].clone(), torch.ones((8, 8), dtype=torch.float32, device="cuda")
    for bad in (torch.empty((4, 8), dtype=torch.float32, device="cuda"),
                torch.empty((8, 8), dtype=torch.float64, device="cuda"),
                torch.empty((8, 16), dtype=torch.float32, device="cuda")[:, ::2]):
        with pytest.raises(ValueError):
            fbf.fbf_filter_backward(p, x2, g2, grad=bad)
    torch.cuda.synchronize()
