"""The allocation-free gradient entry point, fbf_filter_backward_noalloc.

It exists for callers that may not allocate device memory (for example when
a host framework has already reserved the device memory for its own
allocator, or inside a real-time loop where an allocation call could block or
fail).  It runs the same kernels as fbf_filter_backward, with its scratch in
a fixed array inside the library.  These checks call both entry points
through the C ABI and require bit-identical gradients (the same kernels on
the same inputs), call after call: first a larger REFLECT image, then a
smaller REFLECT image with other data and another window, whose extended
grid lies inside what the first call left in the shared array -- an element
the adjoint pass failed to rewrite would carry the first call's value -- and
then a TRUNCATE image.  They also check the size limit.  This file is
collected last on purpose, so a run that stops at its first failure has run
everything else.
"""
import ctypes as C

import pytest

from paper_1603_08081_gb300.synth import make_grad, make_image_f32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fbf():
    import torch  # noqa: F401

    from paper_1603_08081_gb300 import build

    build.build()
    from paper_1603_08081_gb300 import fbf as mod

    return mod


def _call(fbf, fn, params, x, g, out):
    import torch

    H, Wd = x.shape
    st = fn(C.byref(params), C.c_void_p(x.data_ptr()), C.c_void_p(g.data_ptr()), None, C.c_void_p(out.data_ptr()),
            H, Wd, x.stride(0) * 4, C.c_void_p(int(torch.cuda.current_stream().cuda_stream)))
    torch.cuda.synchronize()
    return st


def test_noalloc_backward_matches_allocating_entry_point_call_after_call(fbf):
    import torch

    cases = [((120, 104), 4.0, "reflect", 11),   # W = 12: the larger extended grid first
             ((70, 57), 2.0, "reflect", 12),     # W = 6, other data: inside the first call's leftovers
             ((130, 67), 4.0, "truncate", 13)]
    for (shape, sigma_s, border, seed) in cases:
        x = torch.from_numpy(make_image_f32(*shape, seed=1400 + seed)).cuda()
        g = torch.from_numpy(make_grad(*shape, seed=1499 + seed)).cuda()
        c = fbf.fbf_fit_coeffs("gaussian", 0.1, 1.0, 1e-3, 0, 256)
        p = fbf.make_params(c, sigma_s, 0, "gaussian", border, "fp32")
        ref = torch.full_like(x, float("nan"))
        got = torch.full_like(x, float("nan"))
        assert _call(fbf, fbf.lib.fbf_filter_backward, p, x, g, ref) == fbf.FBF_OK
        assert _call(fbf, fbf.lib.fbf_filter_backward_noalloc, p, x, g, got) == fbf.FBF_OK
        assert bool(torch.isfinite(got).all())
        assert torch.equal(got, ref), (shape, border, float((got - ref).abs().max()))


def test_noalloc_backward_rejects_requests_beyond_its_scratch(fbf):
    import torch

    limit = 16 << 20
    side = 1500  # 8 B/pixel + (side + 2W)^2 floats > 16 MiB
    assert side * side * 8 > limit
    x = torch.zeros((side, side), dtype=torch.float32, device="cuda")
    c = fbf.fbf_fit_coeffs("gaussian", 0.1, 1.0, 1e-3, 0, 256)
    p = fbf.make_params(c, 2.0)
    assert _call(fbf, fbf.lib.fbf_filter_backward_noalloc, p, x, x, x) == fbf.FBF_ERR_RANGE
