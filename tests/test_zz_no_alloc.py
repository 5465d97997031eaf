"""The allocation-free gradient entry point, fbf_filter_backward_noalloc.

It exists for callers that may not allocate device memory (for example when
a host framework has already reserved the device memory for its own
allocator, or inside a real-time loop where an allocation call could block or
fail).  It runs the same kernels as fbf_filter_backward, with its scratch in
a fixed array inside the library.  These checks call both entry points
through the C ABI and compare them, twice in a row with different inputs so
that anything left in the shared array by the first call would show up in the
second; and they check the size limit.  This file is collected last on
purpose, so a run that stops at its first failure has run everything else.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1603_08081_gb300.synth import make_grad, make_image_f32

pytestmark = pytest.mark.gpu

# Same bound as the other gradient tests: 1e-3 of the largest entry.
REL_TOL = 1e-3


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


def test_noalloc_backward_matches_allocating_entry_point_twice(fbf):
    import torch

    cases = [((96, 80), 2.0, "reflect", 11), ((130, 67), 4.0, "truncate", 12)]
    for (shape, sigma_s, border, seed) in cases:
        x = torch.from_numpy(make_image_f32(*shape, seed=1400 + seed)).cuda()
        g = torch.from_numpy(make_grad(*shape, seed=1499 + seed)).cuda()
        c = fbf.fbf_fit_coeffs("gaussian", 0.1, 1.0, 1e-3, 0, 256)
        p = fbf.make_params(c, sigma_s, 0, "gaussian", border, "fp32")
        ref = torch.full_like(x, float("nan"))
        got = torch.full_like(x, float("nan"))
        assert _call(fbf, fbf.lib.fbf_filter_backward, p, x, g, ref) == fbf.FBF_OK
        assert _call(fbf, fbf.lib.fbf_filter_backward_noalloc, p, x, g, got) == fbf.FBF_OK
        r, o = ref.cpu().numpy(), got.cpu().numpy()
        assert np.all(np.isfinite(o))
        assert np.abs(o - r).max() <= REL_TOL * np.abs(r).max()


def test_noalloc_backward_rejects_requests_beyond_its_scratch(fbf):
    import torch

    limit = 16 << 20
    side = 1500  # 8 B/pixel + (side + 2W)^2 floats > 16 MiB
    assert side * side * 8 > limit
    x = torch.zeros((side, side), dtype=torch.float32, device="cuda")
    c = fbf.fbf_fit_coeffs("gaussian", 0.1, 1.0, 1e-3, 0, 256)
    p = fbf.make_params(c, 2.0)
    assert _call(fbf, fbf.lib.fbf_filter_backward_noalloc, p, x, x, x) == fbf.FBF_ERR_RANGE
