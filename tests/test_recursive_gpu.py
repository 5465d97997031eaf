"""GPU parity of the recursive-Gaussian spatial kernel (the constant-time
Gaussian filtering that Sec. II cites: Deriche's recursive approximation),
FP32 form, against the oracle's FP64 recursive mode of Algorithm 1 with the
same coefficients and border, element by element.

Tolerance.  The library runs the filter as two second-order sections per
direction in FP32 (the oracle: one fourth-order recursion in FP64); the FP32
recursions accumulate rounding over a line like the FIR's window sums do, so
the FP32 form's regression bound of 0.05 gray level applies, inside the 0.5
contract.
"""
import numpy as np
import pytest

import oracle as O
from paper_1603_08081_gb300.synth import make_image

pytestmark = pytest.mark.gpu

TOL = 0.05


@pytest.fixture(scope="module")
def fbf():
    import torch  # noqa: F401

    from paper_1603_08081_gb300 import build

    build.build()
    from paper_1603_08081_gb300 import fbf as mod

    return mod


def _gpu(fbf, img, c, sigma_s, border="reflect", form="fp32", pad=0):
    import torch

    H, Wd = img.shape
    if pad:
        buf = torch.zeros((H, Wd + pad), dtype=torch.uint8, device="cuda")
        buf[:, :Wd] = torch.from_numpy(img).cuda()
        x = buf[:, :Wd]
    else:
        x = torch.from_numpy(np.ascontiguousarray(img)).cuda()
    p = fbf.make_params(c, sigma_s, 0, "gaussian_recursive", border, form)
    y = fbf.fbf_filter(p, x)
    torch.cuda.synchronize()
    return y.cpu().numpy().astype(np.float64)


def _oracle(img, c, sigma_s, border):
    bd = O.BORDER_REFLECT if border == "reflect" else O.BORDER_TRUNCATE
    return O.alg1_rec(img.astype(np.float64), sigma_s, bd, np.array(c.coefficients), c.T)[0]


@pytest.mark.parametrize("border", ["reflect", "truncate"])
@pytest.mark.parametrize("shape", [(1, 1), (1, 70), (70, 1), (5, 7), (33, 200), (130, 97), (256, 256)])
def test_ragged_images(fbf, shape, border):
    img = make_image(*shape, seed=shape[0] + 3 * shape[1])
    c = fbf.fbf_fit_coeffs("gaussian", 30.0, 255.0, 1e-2)
    got = _gpu(fbf, img, c, 3.0, border)
    assert np.all(np.isfinite(got))
    assert np.abs(got - _oracle(img, c, 3.0, border)).max() <= TOL


@pytest.mark.parametrize("border", ["reflect", "truncate"])
@pytest.mark.parametrize("sigma_s", [0.5, 1.0, 4.0, 12.0, 30.0])
def test_scales(fbf, sigma_s, border):
    """From half a pixel to windows far wider than any FIR instantiation."""
    img = make_image(150, 130, seed=int(sigma_s * 10))
    c = fbf.fbf_fit_coeffs("gaussian", 25.0, 255.0, 1e-3)
    got = _gpu(fbf, img, c, sigma_s, border)
    assert np.abs(got - _oracle(img, c, sigma_s, border)).max() <= TOL


@pytest.mark.parametrize("K_fixed", [1, 40])
def test_orders(fbf, K_fixed):
    """K = 1 (sigma_r -> infinity: plain Gaussian smoothing) and K = 40."""
    img = make_image(100, 90, seed=K_fixed)
    c = fbf.fbf_fit_coeffs("exponential", 20.0, 255.0, 0.0, K_fixed)
    got = _gpu(fbf, img, c, 5.0, "reflect")
    assert np.abs(got - _oracle(img, c, 5.0, "reflect")).max() <= TOL


def test_padded_pitch_and_chunked_harmonics_match(fbf):
    """A padded row pitch; and the time does not depend on sigma_s (the point of
    the recursive form): under TRUNCATE (no line extension) sigma_s = 2 and 40
    run within 50% of each other (the work is the same)."""
    import time

    import torch

    img = make_image(300, 260, seed=9)
    c = fbf.fbf_fit_coeffs("gaussian", 20.0, 255.0, 1e-3)
    got = _gpu(fbf, img, c, 6.0, "reflect", pad=13)
    assert np.abs(got - _oracle(img, c, 6.0, "reflect")).max() <= TOL
    big = torch.from_numpy(make_image(1024, 1024, seed=10)).cuda()
    ts = {}
    for s in (2.0, 40.0):
        p = fbf.make_params(c, s, 0, "gaussian_recursive", "truncate", "fp32")
        fbf.fbf_filter(p, big)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(3):
            fbf.fbf_filter(p, big)
        torch.cuda.synchronize()
        ts[s] = time.perf_counter() - t0
    assert ts[40.0] <= 1.5 * ts[2.0] and ts[2.0] <= 1.5 * ts[40.0]


def test_full_size_2048_rows(fbf):
    """The benchmark image (a 1024 x 512 crop) at sigma_s = 10, sigma_r = 20 (K = 17)."""
    img = make_image(2048, 2048, 1100)[:1024, :512].copy()
    c = fbf.fbf_fit_coeffs("gaussian", 20.0, 255.0, 1e-3)
    got = _gpu(fbf, img, c, 10.0, "reflect")
    ref = _oracle(img, c, 10.0, "reflect")
    assert np.abs(got - ref).max() <= TOL


def test_rejected_where_the_kernel_does_not_apply(fbf):
    import torch

    c = fbf.fbf_fit_coeffs("gaussian", 30.0, 255.0, 1e-2)
    x = torch.zeros((40, 40), dtype=torch.uint8, device="cuda")
    for form in ("tc_fp16", "tc_fp16_single"):
        with pytest.raises(fbf.FbfError) as e:
            fbf.fbf_filter(fbf.make_params(c, 3.0, 0, "gaussian_recursive", "reflect", form), x)
        assert e.value.status == fbf.FBF_ERR_UNSUPPORTED
    for s, code in ((0.3, fbf.FBF_ERR_RANGE), (300.0, fbf.FBF_ERR_RANGE), (float("nan"), fbf.FBF_ERR_INVALID_ARGUMENT)):
        with pytest.raises(fbf.FbfError) as e:
            fbf.fbf_filter(fbf.make_params(c, s, 0, "gaussian_recursive", "reflect", "fp32"), x)
        assert e.value.status == code
    cf = fbf.fbf_fit_coeffs("gaussian", 0.1, 1.0, 1e-3, levels=256)
    xf = torch.rand((40, 40), device="cuda")
    pf = fbf.make_params(cf, 3.0, 0, "gaussian_recursive", "reflect", "fp32")
    with pytest.raises(fbf.FbfError) as e:
        fbf.fbf_filter(pf, xf)
    assert e.value.status == fbf.FBF_ERR_UNSUPPORTED
    with pytest.raises(fbf.FbfError) as e:
        fbf.fbf_filter_backward(pf, xf, torch.ones_like(xf))
    assert e.value.status == fbf.FBF_ERR_UNSUPPORTED
