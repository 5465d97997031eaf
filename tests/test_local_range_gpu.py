"""GPU parity of fbf_local_range (the dynamic range T of Sec. III) against the
FP64 oracle: an integer result, compared exactly."""
import ctypes as C

import numpy as np
import pytest

import oracle as O
from paper_1603_08081_gb300.synth import make_image

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fbf():
    import torch  # noqa: F401

    from paper_1603_08081_gb300 import build

    build.build()
    from paper_1603_08081_gb300 import fbf as mod

    return mod


def _t(fbf, img, W, pad=0):
    import torch

    H, Wd = img.shape
    if pad:
        buf = torch.zeros((H, Wd + pad), dtype=torch.uint8, device="cuda")
        buf[:, :Wd] = torch.from_numpy(img).cuda()
        x = buf[:, :Wd]
    else:
        x = torch.from_numpy(np.ascontiguousarray(img)).cuda()
    return fbf.fbf_local_range(x, W)


@pytest.mark.parametrize("shape", [(1, 1), (1, 70), (70, 1), (5, 7), (33, 65), (64, 64), (97, 130), (256, 200)])
@pytest.mark.parametrize("W", [0, 1, 2, 3, 5, 8, 9, 15, 16, 17, 31, 32])
def test_matches_oracle(fbf, shape, W):
    img = make_image(*shape, seed=60 + W)
    assert _t(fbf, img, W) == int(O.local_range(img, W))


def test_structured_images(fbf):
    step = np.full((40, 90), 40, np.uint8)
    step[:, 45:] = 217
    assert _t(fbf, step, 1) == 177
    assert _t(fbf, step, 0) == 0
    spike = np.zeros((50, 70), np.uint8)
    spike[49, 69] = 255  # corner pixel: reached only through the last tile's edge
    assert _t(fbf, spike, 3) == 255
    assert _t(fbf, np.full((33, 77), 9, np.uint8), 12) == 0
    rng = np.random.default_rng(2)
    noise = rng.integers(0, 256, size=(130, 260), dtype=np.uint8)
    for W in (1, 4, 32):
        assert _t(fbf, noise, W, pad=13) == int(O.local_range(noise, W))


@pytest.mark.parametrize("W", [9, 15, 30])
def test_full_size_2048(fbf, W):
    """The benchmark image: T against max/min filters with edge replication
    (equal to the oracle's definition, pinned on the CPU)."""
    ndi = pytest.importorskip("scipy.ndimage")
    img = make_image(2048, 2048, 1100)
    f = img.astype(np.int32)
    size = 2 * W + 1
    want = max(int(np.max(ndi.maximum_filter(f, size=size, mode="nearest") - f)),
               int(np.max(f - ndi.minimum_filter(f, size=size, mode="nearest"))))
    assert _t(fbf, img, W) == want


def test_errors_and_empty(fbf):
    import torch

    out = torch.full((1,), 7, dtype=torch.int32, device="cuda")
    x = torch.zeros((4, 4), dtype=torch.uint8, device="cuda")
    p = C.c_void_p(x.data_ptr())
    o = C.c_void_p(out.data_ptr())
    assert fbf.lib.fbf_local_range(p, fbf.FBF_U8, 4, 4, 4, 49, o, None) == fbf.FBF_ERR_RANGE
    assert fbf.lib.fbf_local_range(p, fbf.FBF_F32, 4, 4, 16, 3, o, None) == fbf.FBF_ERR_UNSUPPORTED
    assert fbf.lib.fbf_local_range(p, fbf.FBF_U8, 4, 4, 3, 3, o, None) == fbf.FBF_ERR_INVALID_ARGUMENT
    assert fbf.lib.fbf_local_range(p, fbf.FBF_U8, 4, 4, 4, 3, None, None) == fbf.FBF_ERR_INVALID_ARGUMENT
    assert fbf.lib.fbf_local_range(p, fbf.FBF_U8, 0, 4, 4, 3, o, None) == fbf.FBF_OK
    torch.cuda.synchronize()
    assert int(out.item()) == 0


def test_local_T_filter_matches_oracle(fbf):
    """Filtering with the local T (fewer terms) stays within the contract of the
    exact filter with that T (Sec. III: T bounds every window difference)."""
    import torch

    img = make_image(192, 160, seed=1000)
    T = _t(fbf, img, 9)
    assert 0 < T < 255
    c = fbf.fbf_fit_coeffs("gaussian", 30.0, float(T), 1e-3)
    c255 = fbf.fbf_fit_coeffs("gaussian", 30.0, 255.0, 1e-3)
    assert c.K <= c255.K
    p = fbf.make_params(c, 3.0)
    y = fbf.fbf_filter(p, torch.from_numpy(img).cuda())
    torch.cuda.synchronize()
    w1 = O.weights_1d(O.SPATIAL_GAUSSIAN, 3.0, 9)
    ref = O.alg1(img, w1, O.BORDER_REFLECT, np.array(c.coefficients), float(T))[0]
    assert np.abs(y.cpu().numpy() - ref).max() <= 0.05
