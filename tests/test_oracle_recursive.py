"""Pins of the oracle's recursive-Gaussian mode (the constant-time Gaussian
filtering that Sec. II cites: Deriche's recursive approximation) against what
the mathematics fixes, independently of the oracle's own recursion:

* Deriche's two damped sinusoids approximate the Gaussian closely (a wrong
  published constant breaks this);
* the causal + anticausal recursions reproduce, sample by sample, the kernel
  written as its closed form (a wrong z-transform coefficient breaks this);
* Algorithm 1 with the recursive filter equals eq. (9) summed directly with
  that closed-form kernel (TRUNCATE: over the whole image; REFLECT: within the
  tail bound of the line extension);
* a constant image maps to itself; sigma_r -> infinity reduces to Gaussian
  smoothing (scipy) within the approximation's own error.
"""
import numpy as np
import pytest

import oracle as O
from paper_1603_08081_gb300.synth import make_image


def _kernel(s, kmax):
    k = np.arange(-kmax, kmax + 1)
    return k, np.array([O.rec_kernel(s, int(v)) for v in k])


def _total(s):  # sum of g(k) over all k (the tail beyond 60 s is below 1e-40)
    return float(_kernel(s, int(np.ceil(60 * s)))[1].sum())


@pytest.mark.parametrize("s", [1.0, 2.0, 5.0, 10.0, 20.0])
def test_deriche_kernel_approximates_the_gaussian(s):
    k, g = _kernel(s, int(10 * s))
    ga = np.exp(-k * k / (2 * s * s))
    assert abs(O.rec_kernel(s, 0) - 1.0) < 1e-3  # g(0) = a1 + a2
    g, ga = g / g.sum(), ga / ga.sum()
    assert np.abs(g - ga).max() <= 1e-3 * ga.max()  # 3.2e-4 .. 4.7e-4 measured


@pytest.mark.parametrize("s", [0.7, 3.0, 12.0])
def test_recursions_reproduce_the_closed_form_kernel(s):
    n = int(np.ceil(40 * s))
    x = np.zeros(2 * n + 1)
    x[n] = 1.0
    y = O.rec_filter_line(x, s)
    k, g = _kernel(s, n)
    assert np.abs(y - g / _total(s)).max() <= 1e-12
    # the anticausal recursion mirrors the causal one: symmetric impulse response
    assert np.abs(y - y[::-1]).max() <= 1e-13


def _w1(s, W):
    return _kernel(s, W)[1] / _total(s)


@pytest.mark.parametrize("shape", [(9, 11), (13, 6), (1, 7)])
@pytest.mark.parametrize("s,K", [(1.5, 1), (1.5, 7), (4.0, 12)])
def test_truncate_equals_direct_eq9_with_the_kernel(shape, s, K):
    """TRUNCATE: the infinite-support kernel restricted to the image, i.e. eq. (9)
    with w = g(j_y) g(j_x) over a window covering the whole image."""
    img = make_image(*shape, seed=shape[0] * 7 + K).astype(np.float64)
    c = O.fit(O.RANGE_GAUSSIAN, 30.0, 255.0, K=K)
    W = max(shape)
    ref = O.direct_sbf(img, _w1(s, W), O.BORDER_TRUNCATE, c.d, 255.0)[0]
    got = O.alg1_rec(img, s, O.BORDER_TRUNCATE, c.d, 255.0)[0]
    assert np.abs(got - ref).max() <= 1e-9


@pytest.mark.parametrize("s", [0.8, 2.5])
def test_reflect_equals_direct_eq9_within_the_extension_tail(s):
    """REFLECT: lines extended by E = ceil(8 s) mirrored samples; eq. (9) with the
    kernel on [-E, E] and the mirrored border differs only by the kernel's weight
    beyond E."""
    img = make_image(12, 10, seed=5).astype(np.float64)
    c = O.fit(O.RANGE_GAUSSIAN, 25.0, 255.0, K=9)
    E = int(np.ceil(8 * s))
    ref = O.direct_sbf(img, _w1(s, E), O.BORDER_REFLECT, c.d, 255.0)[0]
    got = O.alg1_rec(img, s, O.BORDER_REFLECT, c.d, 255.0)[0]
    k, g = _kernel(s, int(np.ceil(60 * s)))
    tail = np.abs(g[np.abs(k) > E]).sum() / _total(s)
    # P and Q both move by at most 2 * tail of their totals; the ratio by ~4 * tail * 255
    assert np.abs(got - ref).max() <= max(4 * tail * 255.0, 1e-9)


@pytest.mark.parametrize("border", [O.BORDER_REFLECT, O.BORDER_TRUNCATE])
def test_constant_image_maps_to_itself(border):
    img = np.full((17, 23), 137.0)
    c = O.fit(O.RANGE_GAUSSIAN, 20.0, 255.0, 1e-3)
    out = O.alg1_rec(img, 3.0, border, c.d, 255.0)[0]
    assert np.abs(out - 137.0).max() <= 1e-9


@pytest.mark.parametrize("s", [1.0, 3.0, 6.0])
def test_flat_range_kernel_is_gaussian_smoothing(s):
    """sigma_r -> infinity (phi = 1, K = 1): the separable recursive Gaussian of the
    image, which is scipy's Gaussian filter up to the approximation's L1 error."""
    scipy_ndimage = pytest.importorskip("scipy.ndimage")
    img = make_image(40, 37, seed=11).astype(np.float64)
    got = O.alg1_rec(img, s, O.BORDER_REFLECT, [1.0], 255.0)[0]
    ref = scipy_ndimage.gaussian_filter(img, s, mode="reflect", truncate=8.0)
    k, g = _kernel(s, int(8 * s))
    ga = np.exp(-k * k / (2 * s * s))
    l1 = np.abs(g / g.sum() - ga / ga.sum()).sum()
    assert np.abs(got - ref).max() <= 2 * l1 * 255.0
    assert np.abs(got - ref).max() <= 0.5
