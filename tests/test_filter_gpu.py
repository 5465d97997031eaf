"""GPU parity of the device filter forms (fbf_filter through the C ABI: FP32,
tensor-core FP16, tensor-core BF16, tensor-core single FP16) against the FP64
oracle, element by element.

Tolerance.  The contract is max-abs <= 0.5 gray level against the FP64 oracle
with the same coefficients and border.  The FP32 form is held to a tighter
regression bound, TOL_FP32 = 0.05 gray: its only error sources are FP32
rounding of the taps, coefficients, table entries (|rel| <= 2^-24 each) and of
the window sums, i.e. |dP|, |dQ| ~ 1e-5 * 255 relative to P, Q; divided by
Q >= w(0) - eps (>= ~5e-3 here) that stays below ~1e-2 gray.
"""
import numpy as np
import pytest

import oracle as O
from paper_1603_08081_gb300.synth import make_image

pytestmark = pytest.mark.gpu

TOL_CONTRACT = 0.5
TOL_FP32 = 0.05
# Tensor-core forms: data split into hi + lo 16-bit parts (and the weights too
# for BF16); an FP64 emulation of this arithmetic on the 2048x2048 image stays
# below 1e-3 gray, so 0.02 leaves a 20x margin while catching layout errors.
TOL_TC = 0.02
# Single FP16 form: data (with the intensity centred, f - T/2) and weights
# rounded to FP16 once, relative error 2^-11 per operand.  An emulation of its
# arithmetic gives 0.02-0.05 gray on these settings (sigma_r >= 20, binary
# 0/255 images included), so 0.15 keeps a 3x margin below the 0.5 contract.
TOL_TC1 = 0.15
FORMS = ["fp32", "tc_fp16", "tc_bf16", "tc_fp16_single"]
TOL = {"fp32": TOL_FP32, "tc_fp16": TOL_TC, "tc_bf16": TOL_TC, "tc_fp16_single": TOL_TC1}


@pytest.fixture(scope="module")
def fbf():
    import torch  # noqa: F401

    from paper_1603_08081_gb300 import build

    build.build()
    from paper_1603_08081_gb300 import fbf as mod

    return mod


def _gpu(fbf, img, coeffs, sigma_s, W=0, spatial="gaussian", border="reflect", stream=None,
         pad=0, offset=0, form="fp32"):
    import torch

    H, Wd = img.shape
    if pad or offset:
        buf = torch.zeros((H, Wd + pad + offset), dtype=torch.uint8, device="cuda")
        buf[:, offset:offset + Wd] = torch.from_numpy(img).cuda()
        x = buf[:, offset:offset + Wd]
    else:
        x = torch.from_numpy(np.ascontiguousarray(img)).cuda()
    p = fbf.make_params(coeffs, sigma_s, W, spatial, border, form)
    y = fbf.fbf_filter(p, x, stream=stream)
    torch.cuda.synchronize()
    return y.cpu().numpy().astype(np.float64)


def _oracle_full(img, coeffs, sigma_s, W, spatial, border):
    sp = O.SPATIAL_BOX if spatial == "box" else O.SPATIAL_GAUSSIAN
    w1 = O.weights_1d(sp, sigma_s, W)
    bd = O.BORDER_TRUNCATE if border == "truncate" else O.BORDER_REFLECT
    return O.alg1(img, w1, bd, np.array(coeffs.coefficients), coeffs.T)[0]


def _check(got, ref, tol=TOL_FP32):
    err = np.abs(got - ref)
    assert np.all(np.isfinite(got))
    assert err.max() <= TOL_CONTRACT
    assert err.max() <= tol, (err.max(), np.unravel_index(err.argmax(), err.shape))
    return err.max()


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("border", ["reflect", "truncate"])
def test_small_plain_config_256(fbf, border, form):
    """256x256, Gaussian sigma_s = 3 (W = 9), sigma_r = 30, eps = 1e-2 (K = 10)."""
    img = make_image(256, 256, 1000)
    c = fbf.fbf_fit_coeffs("gaussian", 30.0, 255.0, 1e-2)
    assert c.K == 10
    got = _gpu(fbf, img, c, 3.0, border=border, form=form)
    _check(got, _oracle_full(img, c, 3.0, 9, "gaussian", border), TOL[form])


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("shape", [(1, 1), (1, 300), (300, 1), (7, 5), (65, 64), (130, 197),
                                   (64, 64), (129, 33)])
@pytest.mark.parametrize("border", ["reflect", "truncate"])
def test_ragged_and_tiny_images(fbf, shape, border, form):
    """Sizes off the tile grid, single rows/columns, windows wider than the image."""
    img = make_image(*shape, seed=17)
    c = fbf.fbf_fit_coeffs("gaussian", 20.0, 255.0, 1e-3)
    for sigma_s in (3.0, 7.0):  # W = 9 and W = 21: the small- and wide-window tiles of each form
        W = int(np.ceil(3 * sigma_s))
        got = _gpu(fbf, img, c, sigma_s, border=border, form=form)
        _check(got, _oracle_full(img, c, sigma_s, W, "gaussian", border), TOL[form])


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("W", [0, 1, 2, 5, 8, 15, 16, 17, 23, 30, 31, 32, 33, 36, 40, 45, 48])
def test_every_window_tail(fbf, W, form):
    """All tap-count residues mod 8 and both tile configurations (box and Gaussian)."""
    img = make_image(96, 150, seed=W)
    c = fbf.fbf_fit_coeffs("gaussian", 30.0, 255.0, 1e-3)
    for spatial, ss in (("box", 1.0), ("gaussian", max(W, 1) / 3.0)):
        if spatial == "box" and W == 0:
            continue
        got = _gpu(fbf, img, c, ss, W=W if W > 0 else 1, spatial=spatial, form=form)
        _check(got, _oracle_full(img, c, ss, W if W > 0 else 1, spatial, "reflect"), TOL[form])


def _tc_tile_rows(form, W):
    """Output rows of one tensor-core tile: 128 - 2W in the second layout (the
    single form at every W, the split forms beyond W = 32); in the first layout
    min(BY, 128 - 2W) with BY = 112 computed rows for W <= 16, 96 for W <= 26
    and 64 above."""
    if form == "tc_fp16_single" or W > 32:
        return 128 - 2 * W
    return min(112, 128 - 2 * W) if W <= 16 else (128 - 2 * W if W <= 26 else 64)


@pytest.mark.parametrize("form", ["tc_fp16", "tc_bf16", "tc_fp16_single"])
@pytest.mark.parametrize("W", [1, 8, 9, 12, 15, 16, 17, 20, 24, 25, 26, 27, 30, 32, 33, 45, 48])
def test_tensor_core_tile_row_edges(fbf, W, form):
    """Heights at and across the tensor-core tiles' row count (both layouts),
    under both borders.  The single FP16 form is held to 0.25 gray here: on
    these small images under the box kernel with W >= 27 some pixels have a
    small Q, and an FP64 emulation of the form's roundings (data and row sums
    to FP16 once, FP32 accumulation) gives 0.17 gray (W = 27, 74 x 70,
    TRUNCATE) and 0.20 (W = 30, 69 x 70, TRUNCATE) -- the GPU matches the
    emulation to 1e-4 gray."""
    rows = _tc_tile_rows(form, W)
    tol = 0.25 if form == "tc_fp16_single" else TOL[form]
    c = fbf.fbf_fit_coeffs("gaussian", 30.0, 255.0, 1e-3)
    for H in (rows, rows + 1, 2 * rows - 1, 2 * rows + 3):
        img = make_image(H, 70, seed=H + W)
        for border in ("reflect", "truncate"):
            got = _gpu(fbf, img, c, W / 3.0, W=W, spatial="box", border=border, form=form)
            _check(got, _oracle_full(img, c, W / 3.0, W, "box", border), tol)


@pytest.mark.parametrize("form", FORMS)
def test_orders_from_one_to_255(fbf, form):
    img = make_image(80, 90, seed=3)
    for c in (fbf.fbf_fit_coeffs("gaussian", 1e12, 255.0, 1e-6),        # K = 1: spatial FIR
              fbf.fbf_fit_coeffs("exponential", 20.0, 255.0, 0.0, 40),   # fixed K = 40
              fbf.fbf_fit_coeffs("exponential", 20.0, 255.0, 1e-3)):     # K = 255
        got = _gpu(fbf, img, c, 2.0, form=form)
        _check(got, _oracle_full(img, c, 2.0, 6, "gaussian", "reflect"), TOL[form])


@pytest.mark.parametrize("form", FORMS)
def test_constant_and_extreme_images(fbf, form):
    c = fbf.fbf_fit_coeffs("gaussian", 30.0, 255.0, 1e-3)
    for v in (0, 1, 128, 255):
        img = np.full((70, 90), v, np.uint8)
        got = _gpu(fbf, img, c, 3.0, form=form)
        assert np.max(np.abs(got - v)) <= (TOL[form] if form == "tc_fp16_single" else 1e-3 * max(1, v))
    rng = np.random.default_rng(5)
    img = rng.choice(np.array([0, 255], np.uint8), size=(64, 80))  # every difference is +-T
    got = _gpu(fbf, img, c, 2.0, form=form)
    _check(got, _oracle_full(img, c, 2.0, 6, "gaussian", "reflect"), TOL[form])
    img = (np.arange(256, dtype=np.uint8)[None, :].repeat(40, 0))  # all 256 levels
    got = _gpu(fbf, img, c, 3.0, border="truncate", form=form)
    _check(got, _oracle_full(img, c, 3.0, 9, "gaussian", "truncate"), TOL[form])


@pytest.mark.parametrize("form", FORMS)
def test_pitch_offset_and_stream(fbf, form):
    import torch

    img = make_image(100, 123, seed=8)
    c = fbf.fbf_fit_coeffs("gaussian", 40.0, 255.0, 1e-3)
    ref = _oracle_full(img, c, 5.0, 15, "gaussian", "reflect")
    s = torch.cuda.Stream()
    _check(_gpu(fbf, img, c, 5.0, pad=37, offset=3, stream=s, form=form), ref, TOL[form])
    _check(_gpu(fbf, img, c, 5.0, pad=5, offset=0, form=form), ref, TOL[form])


@pytest.mark.parametrize("form", FORMS)
def test_subpixel_bound_against_direct_filter(fbf, form):
    """eps = 1e-5 gives K = 14 and bound (12) = 0.288 < 0.5 at sigma_s = 3: the GPU
    output is provably within a sub-pixel of the exact bilateral filter, eq. (1)."""
    img = make_image(256, 256, 1000)
    c = fbf.fbf_fit_coeffs("gaussian", 30.0, 255.0, 1e-5)
    assert c.K == 14
    got = _gpu(fbf, img, c, 3.0, form=form)
    w1 = O.weights_1d(O.SPATIAL_GAUSSIAN, 3.0, 9)
    bound = O.bound12(255.0, 1e-5, w1[9] ** 2)
    assert bound < 0.5
    ys, xs = np.mgrid[0:256:3, 0:256:3]
    ref = O.direct_bf(img, w1, O.BORDER_REFLECT, O.RANGE_GAUSSIAN, 30.0,
                      points=(ys.ravel(), xs.ravel()))[0]
    assert np.max(np.abs(got[ys, xs].ravel() - ref)) <= bound


def _sample_points(H, W, n, seed):
    rng = np.random.default_rng(seed)
    ys = list(rng.integers(0, H, n)) + [0, 0, H - 1, H - 1, H // 2, 0, H - 1, H // 2]
    xs = list(rng.integers(0, W, n)) + [0, W - 1, 0, W - 1, 0, W // 2, W // 2, W - 1]
    return np.array(ys), np.array(xs)


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("sigma_s", [3.0, 5.0, 10.0, 12.0])
@pytest.mark.parametrize("sigma_r", [20.0, 40.0])
def test_full_size_2048_sampled(fbf, sigma_s, sigma_r, form):
    """2048x2048, eps = 1e-3, the benchmark's launch configuration: sampled pixels
    (random + corners + edges) against eq. (9) summed directly in FP64."""
    img = make_image(2048, 2048, 1100)
    c = fbf.fbf_fit_coeffs("gaussian", sigma_r, 255.0, 1e-3)
    got = _gpu(fbf, img, c, sigma_s, form=form)
    W = int(np.ceil(3 * sigma_s))
    ys, xs = _sample_points(2048, 2048, 600, seed=int(sigma_s * 10 + sigma_r))
    w1 = O.weights_1d(O.SPATIAL_GAUSSIAN, sigma_s, W)
    ref = O.direct_sbf(img, w1, O.BORDER_REFLECT, np.array(c.coefficients), 255.0,
                       points=(ys, xs))[0]
    _check(got[ys, xs], ref, TOL[form])
    assert np.all(np.isfinite(got))
    assert got.min() >= -1.0 and got.max() <= 256.0


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("W", [33, 36, 45])
def test_windows_beyond_32(fbf, W, form):
    """Windows wider than 32 (sigma_s = 11 .. 15; Table 1 of Sec. V runs sigma_s up
    to 12): every form against Algorithm 1 in FP64, both borders, Gaussian and
    box kernels."""
    img = make_image(300, 260, seed=W + 5)
    c = fbf.fbf_fit_coeffs("gaussian", 25.0, 255.0, 1e-3)
    for border in ("reflect", "truncate"):
        got = _gpu(fbf, img, c, W / 3.0, W=W, border=border, form=form)
        _check(got, _oracle_full(img, c, W / 3.0, W, "gaussian", border), TOL[form])
    got = _gpu(fbf, img, c, 1.0, W=W, spatial="box", form=form)
    _check(got, _oracle_full(img, c, 1.0, W, "box", "reflect"), 0.25 if form == "tc_fp16_single" else TOL[form])


@pytest.mark.parametrize("sigma_r", [5.0, 10.0])
def test_single_form_small_range_scale(fbf, sigma_r):
    """The single FP16 form's error grows as sigma_r shrinks (K = 60 at sigma_r = 5):
    it stays within 0.2 gray there (emulation: 0.09), the split FP16 form within TOL_TC."""
    img = make_image(200, 160, seed=4)
    c = fbf.fbf_fit_coeffs("gaussian", sigma_r, 255.0, 1e-3)
    ref = _oracle_full(img, c, 3.0, 9, "gaussian", "reflect")
    _check(_gpu(fbf, img, c, 3.0, form="tc_fp16_single"), ref, 0.2)
    _check(_gpu(fbf, img, c, 3.0, form="tc_fp16"), ref, TOL_TC)


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("kernel", ["tukey", "huber"])
def test_user_sampled_range_kernel(fbf, kernel, form):
    """A range kernel given only by samples (Sec. III: any kernel with a pointwise-
    convergent Fourier series), fitted by fbf_fit_coeffs_samples: Tukey's biweight
    (1 - (t/60)^2)^2 on |t| <= 60, or the Huber-type weight min(1, 25/|t|).  Every
    form against Algorithm 1 in FP64 with the same coefficients, both borders."""
    t = np.arange(256.0)
    if kernel == "tukey":
        phi = (1.0 - np.clip(t / 60.0, 0.0, 1.0) ** 2) ** 2
    else:
        phi = np.minimum(1.0, 25.0 / np.maximum(t, 1e-300))
    c = fbf.fbf_fit_coeffs_samples(phi, 255.0, 1e-3)
    assert c.K > 5
    img = make_image(150, 130, seed=21)
    for border, ss in (("reflect", 3.0), ("truncate", 5.0)):
        got = _gpu(fbf, img, c, ss, border=border, form=form)
        _check(got, _oracle_full(img, c, ss, int(np.ceil(3 * ss)), "gaussian", border), TOL[form])


@pytest.mark.parametrize("border", ["reflect", "truncate"])
def test_box_4096_exponential_sampled(fbf, border):
    """The 4096x4096 exponential-kernel workload with the box kernel W = 8 (the
    FP32 form runs it as running window sums), K = 40 fixed: sampled pixels
    against eq. (9) summed directly, every form."""
    img = make_image(4096, 4096, 1200)
    c = fbf.fbf_fit_coeffs("exponential", 20.0, 255.0, 0.0, 40)
    ys, xs = _sample_points(4096, 4096, 400, seed=88)
    w1 = O.weights_1d(O.SPATIAL_BOX, 1.0, 8)
    bd = O.BORDER_REFLECT if border == "reflect" else O.BORDER_TRUNCATE
    ref = O.direct_sbf(img, w1, bd, np.array(c.coefficients), 255.0, points=(ys, xs))[0]
    for form in FORMS:
        got = _gpu(fbf, img, c, 1.0, W=8, spatial="box", border=border, form=form)
        _check(got[ys, xs], ref, TOL[form])


@pytest.mark.parametrize("spatial,W,expect", [("gaussian", 3, "fp32"), ("gaussian", 4, "tc_fp16"),
                                              ("gaussian", 6, "tc_fp16"), ("gaussian", 30, "tc_fp16"),
                                              ("box", 3, "fp32"), ("box", 4, "tc_fp16"),
                                              ("box", 10, "tc_fp16"), ("box", 17, "tc_fp16"),
                                              ("box", 26, "tc_fp16"), ("box", 30, "tc_fp16")])
def test_auto_form_picks_the_documented_kernel(fbf, spatial, W, expect):
    """AUTO runs exactly the kernel of the form its rule names (bit-identical output)."""
    img = make_image(150, 170, seed=W)
    c = fbf.fbf_fit_coeffs("gaussian", 25.0, 255.0, 1e-3)
    auto = _gpu(fbf, img, c, max(W, 1) / 3.0, W=W, spatial=spatial, form="auto")
    want = _gpu(fbf, img, c, max(W, 1) / 3.0, W=W, spatial=spatial, form=expect)
    assert np.array_equal(auto, want)
    _check(auto, _oracle_full(img, c, max(W, 1) / 3.0, W, spatial, "reflect"), TOL[expect])


@pytest.mark.parametrize("form,W", [("tc_fp16_single", 9), ("tc_fp16_single", 36), ("tc_fp16", 36),
                                    ("tc_bf16", 36)])
@pytest.mark.parametrize("pad", [0, 3])
def test_bounded_wait_gives_up_then_the_next_call_is_correct(fbf, form, W, pad):
    """With the poll limit set to 0 every bounded wait of the second tensor-core
    layout gives up at once (the TMA box wait when the image is TMA-aligned,
    pad = 0; the first MMA wait when rows are loaded directly, pad = 3): the
    kernel drains its copies and MMAs in flight, sets the device error word and
    returns; the context stays usable and the next call, at the default limit,
    is exact.  (The split forms run the second layout beyond W = 32.)"""
    import ctypes as C

    img = make_image(150, 144, seed=31)  # 144-byte rows: TMA-aligned unless padded
    c = fbf.fbf_fit_coeffs("gaussian", 30.0, 255.0, 1e-3)
    ref = _oracle_full(img, c, W / 3.0, W, "gaussian", "reflect")
    try:
        assert fbf.fbf_device_error() == 0
        fbf.fbf_set_wait_limit(0)
        _gpu(fbf, img, c, W / 3.0, W=W, pad=pad, form=form)
        v = C.c_uint(0)
        assert fbf.lib.fbf_device_error(C.byref(v)) == fbf.FBF_ERR_TIMEOUT
        assert v.value != 0
        assert fbf.fbf_device_error() == 0  # read and cleared
    finally:
        fbf.fbf_set_wait_limit(-1)
    _check(_gpu(fbf, img, c, W / 3.0, W=W, pad=pad, form=form), ref, TOL[form])
    assert fbf.fbf_device_error() == 0
