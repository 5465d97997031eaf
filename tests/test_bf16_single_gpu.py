"""GPU parity of the single BF16 tensor-core form (TC_BF16_SINGLE: data, with
the intensity centred f - T/2, and weights rounded to BF16 once, FP32
accumulation) against the FP64 oracle, element by element, inside the form's
stated domain: REFLECT border, sigma_r >= 15, sigma_s >= 1 (W >= 3).  Under
TRUNCATE the window near a corner keeps a quarter of its weight, Q is about
four times smaller there and so is the margin (0.48 gray measured at W = 16):
those cases are checked on the pixels at least W from every border.

Tolerance.  BF16 keeps 8 significand bits (relative rounding 2^-9 per
operand).  An FP64 emulation of the form's rounding steps (channels rounded
once, row results rounded once, FP32 sums) gives 0.08-0.31 gray level on
Gaussian windows W = 9..48 and box windows W = 3..30 at sigma_r = 15..60, both
borders, crops of the benchmark image and small synthetic images (0.11-0.20 on
the benchmark's six settings); 0.4 keeps a margin above that and stays inside
the 0.5 contract.  At sigma_r = 10 the emulation reaches 0.46-0.54, and a
window with one dominant tap (sigma_s = 1/3, W = 1: 0.45 measured) leaves the
rounding of a single channel value unaveraged: outside the domain, not tested.
"""
import numpy as np
import pytest

import oracle as O
from paper_1603_08081_gb300.synth import make_image

pytestmark = pytest.mark.gpu

TOL_BF16_SINGLE = 0.4
FORM = "tc_bf16_single"


@pytest.fixture(scope="module")
def fbf():
    import torch  # noqa: F401

    from paper_1603_08081_gb300 import build

    build.build()
    from paper_1603_08081_gb300 import fbf as mod

    return mod


def _gpu(fbf, img, c, sigma_s, W=0, spatial="gaussian", border="reflect", form=FORM):
    import torch

    x = torch.from_numpy(np.ascontiguousarray(img)).cuda()
    y = fbf.fbf_filter(fbf.make_params(c, sigma_s, W, spatial, border, form), x)
    torch.cuda.synchronize()
    return y.cpu().numpy().astype(np.float64)


def _oracle(img, c, sigma_s, W, spatial, border):
    w1 = O.weights_1d(O.SPATIAL_BOX if spatial == "box" else O.SPATIAL_GAUSSIAN, sigma_s, W)
    bd = O.BORDER_TRUNCATE if border == "truncate" else O.BORDER_REFLECT
    return O.alg1(img, w1, bd, np.array(c.coefficients), c.T)[0]


def _check(got, ref, tol=TOL_BF16_SINGLE, border="reflect", W=0):
    assert np.all(np.isfinite(got))
    if border == "truncate" and W > 0:  # interior: the full window inside the image
        got, ref = got[W:-W, W:-W], ref[W:-W, W:-W]
        if got.size == 0:  # no pixel with the full window inside the image
            return 0.0
    err = np.abs(got - ref).max()
    assert err <= tol, err
    return err


@pytest.mark.parametrize("border", ["reflect", "truncate"])
@pytest.mark.parametrize("shape", [(1, 1), (7, 5), (33, 200), (130, 197), (256, 256)])
def test_ragged_images(fbf, shape, border):
    img = make_image(*shape, seed=31 + shape[0])
    c = fbf.fbf_fit_coeffs("gaussian", 30.0, 255.0, 1e-2)
    _check(_gpu(fbf, img, c, 3.0, border=border), _oracle(img, c, 3.0, 9, "gaussian", border), border=border, W=9)


@pytest.mark.parametrize("border", ["reflect", "truncate"])
@pytest.mark.parametrize("W", [3, 9, 16, 17, 30, 32, 33, 48])
def test_every_instantiation_band(fbf, W, border):
    """Windows across the three instantiations (row chunks 4, 6, 8), Gaussian."""
    img = make_image(300, 260, seed=W + 50)
    c = fbf.fbf_fit_coeffs("gaussian", 25.0, 255.0, 1e-3)
    ss = max(W, 1) / 3.0
    _check(_gpu(fbf, img, c, ss, W=W, border=border), _oracle(img, c, ss, W, "gaussian", border), border=border, W=W)


@pytest.mark.parametrize("W", [3, 8, 30])
def test_box_windows(fbf, W):
    img = make_image(200, 170, seed=W + 70)
    c = fbf.fbf_fit_coeffs("gaussian", 20.0, 255.0, 1e-3)
    for border in ("reflect", "truncate"):
        _check(_gpu(fbf, img, c, 1.0, W=W, spatial="box", border=border), _oracle(img, c, 1.0, W, "box", border),
               border=border, W=W)


@pytest.mark.parametrize("W", [9, 30, 48])
def test_tile_row_edges(fbf, W):
    """Heights one below, at and one above the tile height 128 - 2W."""
    c = fbf.fbf_fit_coeffs("gaussian", 20.0, 255.0, 1e-3)
    rows = 128 - 2 * W
    for H in (rows - 1, rows, rows + 1, 2 * rows + 1):
        img = make_image(H, 75, seed=H + W)
        _check(_gpu(fbf, img, c, W / 3.0, W=W), _oracle(img, c, W / 3.0, W, "gaussian", "reflect"))


@pytest.mark.parametrize("sigma_s", [3.0, 5.0, 10.0])
@pytest.mark.parametrize("sigma_r", [20.0, 40.0])
def test_full_size_2048_sampled(fbf, sigma_s, sigma_r):
    """The benchmark's launches: sampled pixels against eq. (9) summed directly."""
    img = make_image(2048, 2048, 1100)
    c = fbf.fbf_fit_coeffs("gaussian", sigma_r, 255.0, 1e-3)
    got = _gpu(fbf, img, c, sigma_s)
    W = int(np.ceil(3 * sigma_s))
    rng = np.random.default_rng(int(sigma_s * 10 + sigma_r) + 7)
    ys = np.concatenate([rng.integers(0, 2048, 400), [0, 0, 2047, 2047]])
    xs = np.concatenate([rng.integers(0, 2048, 400), [0, 2047, 0, 2047]])
    w1 = O.weights_1d(O.SPATIAL_GAUSSIAN, sigma_s, W)
    ref = O.direct_sbf(img, w1, O.BORDER_REFLECT, np.array(c.coefficients), 255.0, points=(ys, xs))[0]
    _check(got[ys, xs], ref)


def test_bf16_operands_are_used(fbf):
    """The form runs BF16 operands, not FP16: its output differs from the single
    FP16 form's and is less accurate on the same launch, both within bounds."""
    img = make_image(160, 192, seed=3)
    c = fbf.fbf_fit_coeffs("gaussian", 20.0, 255.0, 1e-3)
    ref = _oracle(img, c, 3.0, 9, "gaussian", "reflect")
    e_bf = _check(_gpu(fbf, img, c, 3.0), ref)
    e_fp = _check(_gpu(fbf, img, c, 3.0, form="tc_fp16_single"), ref, 0.15)
    assert e_bf > 2 * e_fp


def test_batched_plan_equals_single_image_filter(fbf):
    """The persistent tensor-core batch in this form: bit-identical to fbf_filter."""
    import torch

    shapes = [(300, 260), (70, 90), (33, 200), (129, 97)]
    specs = [dict(sigma_s=3.0, sigma_r=30.0), dict(sigma_s=10.0, sigma_r=20.0), dict(sigma_s=1.5, sigma_r=40.0),
             dict(sigma_s=6.0, sigma_r=15.0)]
    imgs = [make_image(h, w, seed=900 + k) for k, (h, w) in enumerate(shapes)]
    xs = [torch.from_numpy(im).cuda() for im in imgs]
    ys = [torch.full(im.shape, float("nan"), dtype=torch.float32, device="cuda") for im in imgs]
    plan = fbf.fbf_plan_create(xs, ys, specs, FORM, "reflect", schedule="persistent_tc")
    fbf.fbf_filter_batched(plan)
    torch.cuda.synchronize()
    for im, x, y, sp in zip(imgs, xs, ys, specs):
        c = fbf.fbf_fit_coeffs("gaussian", sp["sigma_r"], 255.0, 1e-3)
        single = fbf.fbf_filter(fbf.make_params(c, sp["sigma_s"], 0, "gaussian", "reflect", FORM), x)
        torch.cuda.synchronize()
        assert torch.equal(single, y)
        W = int(np.ceil(3 * sp["sigma_s"] - 1e-12))
        _check(y.cpu().numpy().astype(np.float64), _oracle(im, c, sp["sigma_s"], W, "gaussian", "reflect"))
    plan.destroy()


def test_rejected_where_the_form_does_not_apply(fbf):
    """Float input and the adjoint take the FP32 form only."""
    import torch

    c = fbf.fbf_fit_coeffs("gaussian", 0.1, 1.0, 1e-3, levels=256)
    x = torch.rand((40, 40), device="cuda")
    p = fbf.make_params(c, 2.0, 0, "gaussian", "reflect", FORM)
    with pytest.raises(fbf.FbfError) as e:
        fbf.fbf_filter(p, x)
    assert e.value.status == fbf.FBF_ERR_UNSUPPORTED
    with pytest.raises(fbf.FbfError) as e:
        fbf.fbf_filter_backward(p, x, torch.ones_like(x))
    assert e.value.status == fbf.FBF_ERR_UNSUPPORTED
