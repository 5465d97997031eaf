"""Pins for the FP64 oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself by retyping its formulas: each
check is a value the paper prints, a closed form, a library routine on a
special case, an invariant of the filter, or a bound the paper proves.
"""
import os

import numpy as np
import pytest

import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    out = []
    with open(os.path.join(GOLD, name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                out.append(line.split())
    return out


def _img(H, W, seed, lo=0, hi=255):
    from paper_1603_08081_gb300.synth import make_image

    a = make_image(H, W, seed).astype(np.float64)
    return np.clip(a, lo, hi)


# ---------------------------------------------------------------- the fit ---

def test_fit_order_matches_tables_3_and_4():
    """Table 3 / Table 4: order N versus eps at T = 217, sigma_r = 30."""
    for eps, N in _rows("table3_table4_order.txt"):
        f = O.fit(O.RANGE_GAUSSIAN, 30.0, 217.0, float(eps))
        assert f.converged
        assert f.K == int(N), (eps, f.K, N)


def test_predicted_bound_row_of_table_4():
    """Table 4 "Predicted": eq. (12) with the normalised sigma_s = 3, W = 9 weights."""
    w1 = O.weights_1d(O.SPATIAL_GAUSSIAN, 3.0, 9)
    w0 = w1[9] ** 2
    for eps, printed, sig in _rows("table4_predicted_bound.txt"):
        b = O.bound12(217.0, float(eps), w0)
        rounded = float("%.*g" % (int(sig), b))
        assert rounded == pytest.approx(float(printed), rel=1e-12), (eps, b, printed)
    # The misprinted 1e-3 entry: the same formula gives 25.9, not 29.5.
    assert round(O.bound12(217.0, 1e-3, w0), 1) == 25.9


@pytest.mark.parametrize("kernel,sigma_r,T,K,levels", [
    (O.RANGE_GAUSSIAN, 30.0, 217.0, 10, 0),
    (O.RANGE_GAUSSIAN, 20.0, 255.0, 17, 0),
    (O.RANGE_EXPONENTIAL, 20.0, 255.0, 40, 0),
    (O.RANGE_GAUSSIAN, 0.1, 1.0, 13, 256),
])
def test_fit_is_the_least_squares_solution(kernel, sigma_r, T, K, levels):
    """d agrees with LAPACK least squares, and b - A d is orthogonal to range(A)."""
    f = O.fit(kernel, sigma_r, T, K=K, levels=levels)
    L = int(T) + 1 if levels == 0 else levels
    t = np.arange(L, dtype=np.float64) if levels == 0 else np.arange(L) * T / (levels - 1)
    b = np.array([O.phi(kernel, sigma_r, x) for x in t])
    A = np.cos(np.outer(t, np.arange(K)) * np.pi / T)
    d_ref = np.linalg.lstsq(A, b, rcond=None)[0]
    assert f.K == K
    assert np.max(np.abs(f.d - d_ref)) <= 1e-10
    r = b - A @ f.d
    assert np.linalg.norm(A.T @ r) <= 1e-10 * np.linalg.norm(A) * np.linalg.norm(b)
    assert f.E == pytest.approx(np.linalg.norm(r), rel=1e-9, abs=1e-14)
    assert f.linf == pytest.approx(np.max(np.abs(r)), rel=1e-9, abs=1e-14)
    # The range kernels in closed form, eq. (3) and the exponential.
    if kernel == O.RANGE_GAUSSIAN:
        assert np.allclose(b, np.exp(-t ** 2 / (2 * sigma_r ** 2)), rtol=0, atol=1e-15)
    else:
        assert np.allclose(b, np.exp(-np.abs(t) / sigma_r), rtol=0, atol=1e-15)


@pytest.mark.parametrize("eps", [1e-1, 1e-2, 1e-3, 1e-5, 1e-8])
def test_kernel_error_guarantee_eq_10(eps):
    """|phi - phi_N| <= ||.||_2 = E <= eps on the grid (eq. (10))."""
    for sr in (10.0, 30.0, 60.0):
        f = O.fit(O.RANGE_GAUSSIAN, sr, 255.0, eps)
        assert f.converged and f.linf <= f.E <= eps
        t = np.arange(256.0)
        err = [abs(O.phi(0, sr, x) - O.phi_n(f.d, 255.0, x)) for x in t]
        assert max(err) <= eps


def test_decay_of_error_is_monotone():
    """Proposition (Decay of Error): E_K non-increasing in K, -> 0 at K = |Lambda_T|."""
    E = [O.fit(O.RANGE_GAUSSIAN, 15.0, 63.0, K=k).E for k in range(1, 65)]
    assert all(E[i + 1] <= E[i] * (1 + 1e-12) + 1e-15 for i in range(len(E) - 1))
    assert E[-1] < 1e-12  # square system (64 points, 64 columns) is solved exactly
    assert E[0] > 0.1


def test_flat_kernel_needs_one_term():
    """sigma_r -> infinity: phi == 1 on [0, T] is the constant column, K = 1, d_0 = 1."""
    f = O.fit(O.RANGE_GAUSSIAN, 1e12, 255.0, 1e-6)
    assert f.K == 1 and abs(f.d[0] - 1.0) < 1e-12


def test_exact_cosine_polynomial_is_recovered():
    """Samples of 0.3 + 0.5 cos(wt) + 0.2 cos(3wt): the fit must stop at K = 4 with
    exactly these coefficients (catches a wrong omega or column index)."""
    T = 40.0
    t = np.arange(41.0)
    w = np.pi / T
    b = 0.3 + 0.5 * np.cos(w * t) + 0.2 * np.cos(3 * w * t)
    f = O.fit_samples(t, b, T, eps=1e-10)
    assert f.K == 4
    assert np.allclose(f.d, [0.3, 0.5, 0.0, 0.2], atol=1e-12)
    assert O.fit_samples(t, b, T, K=3).E > 0.1


def test_fit_is_scale_equivariant():
    """(sigma_r, T) -> (sigma_r/255, T/255) on the 256-level grid is the same problem."""
    a = O.fit(O.RANGE_GAUSSIAN, 25.5, 255.0, 1e-3)
    b = O.fit(O.RANGE_GAUSSIAN, 0.1, 1.0, 1e-3, levels=256)
    assert a.K == b.K == 13
    assert np.max(np.abs(a.d - b.d)) < 1e-11


# -------------------------------------------------------------- the filter ---

def _setup(sigma_s=2.0, W=None, spatial=O.SPATIAL_GAUSSIAN, sigma_r=30.0, eps=1e-2, T=255.0,
           kernel=O.RANGE_GAUSSIAN):
    W = O.default_W(sigma_s) if W is None else W
    w1 = O.weights_1d(spatial, sigma_s, W)
    fit = O.fit(kernel, sigma_r, T, eps)
    return w1, fit


@pytest.mark.parametrize("shape", [(1, 1), (1, 7), (7, 1), (5, 3), (17, 23), (12, 12)])
@pytest.mark.parametrize("border", [O.BORDER_REFLECT, O.BORDER_TRUNCATE])
@pytest.mark.parametrize("W,spatial", [(0, O.SPATIAL_GAUSSIAN), (2, O.SPATIAL_BOX),
                                       (4, O.SPATIAL_GAUSSIAN), (9, O.SPATIAL_GAUSSIAN)])
def test_algorithm_1_equals_direct_eq_9(shape, border, W, spatial):
    """Algorithm 1 (modulate, convolve, demodulate) computes eq. (9) exactly:
    brute force over the window on tiny images, windows larger than the image."""
    f = _img(*shape, seed=7 + W)
    w1 = O.weights_1d(spatial, 3.0, W)
    fit = O.fit(O.RANGE_GAUSSIAN, 30.0, 255.0, 1e-3)
    a, Pa, Qa, Pi, Qi = O.alg1(f, w1, border, fit.d, 255.0)
    b, Pb, Qb = O.direct_sbf(f, w1, border, fit.d, 255.0)
    assert np.max(np.abs(a - b)) <= 1e-9
    assert np.max(np.abs(Pa - Pb)) <= 1e-9 and np.max(np.abs(Qa - Qb)) <= 1e-11
    assert np.max(np.abs(Pi)) <= 1e-9 and np.max(np.abs(Qi)) <= 1e-11


@pytest.mark.parametrize("border", [O.BORDER_REFLECT, O.BORDER_TRUNCATE])
def test_constant_image_is_fixed(border):
    """P = c Q for a constant image, so fhat = c (any phi_N with Q != 0)."""
    w1, fit = _setup()
    for c in (0.0, 17.0, 255.0):
        f = np.full((9, 13), c)
        assert np.max(np.abs(O.alg1(f, w1, border, fit.d, 255.0)[0] - c)) < 1e-10
        assert np.max(np.abs(O.direct_sbf(f, w1, border, fit.d, 255.0)[0] - c)) < 1e-10
        assert np.max(np.abs(O.direct_bf(f, w1, border, O.RANGE_GAUSSIAN, 30.0)[0] - c)) < 1e-10


@pytest.mark.parametrize("shape,sigma_s", [((20, 31), 2.0), ((40, 16), 3.0), ((5, 6), 2.0)])
def test_flat_range_kernel_reduces_to_spatial_filter(shape, sigma_s):
    """sigma_r -> infinity: the filter is the normalised spatial FIR, compared with
    scipy.ndimage.correlate ('reflect' = half-sample symmetric; 'constant' with the
    mask renormalised for the truncated border)."""
    nd = pytest.importorskip("scipy.ndimage")
    f = _img(*shape, seed=3)
    W = O.default_W(sigma_s)
    w1 = O.weights_1d(O.SPATIAL_GAUSSIAN, sigma_s, W)
    w2 = np.outer(w1, w1)
    fit = O.fit(O.RANGE_GAUSSIAN, 1e12, 255.0, 1e-6)
    ref = nd.correlate(f, w2, mode="reflect")
    if min(shape) > W:  # scipy's reflect extends once; deeper mirroring only tested above
        assert np.max(np.abs(O.alg1(f, w1, O.BORDER_REFLECT, fit.d, 255.0)[0] - ref)) < 1e-9
        assert np.max(np.abs(O.direct_bf(f, w1, O.BORDER_REFLECT, 0, 1e12)[0] - ref)) < 1e-9
    num = nd.correlate(f, w2, mode="constant", cval=0.0)
    den = nd.correlate(np.ones_like(f), w2, mode="constant", cval=0.0)
    assert np.max(np.abs(O.alg1(f, w1, O.BORDER_TRUNCATE, fit.d, 255.0)[0] - num / den)) < 1e-9
    assert np.max(np.abs(O.direct_bf(f, w1, O.BORDER_TRUNCATE, 0, 1e12)[0] - num / den)) < 1e-9


def test_direct_bf_against_padded_window_sum():
    """Eq. (1) evaluated with numpy's own symmetric padding and window views."""
    f = _img(14, 11, seed=5)
    W, sr = 3, 20.0
    w1 = O.weights_1d(O.SPATIAL_GAUSSIAN, 1.0, W)
    w2 = np.outer(w1, w1)
    pad = np.pad(f, W, mode="symmetric")
    win = np.lib.stride_tricks.sliding_window_view(pad, (2 * W + 1, 2 * W + 1))
    # window index (a, b) is neighbour offset (a - W, b - W); w is symmetric.
    ph = np.exp(-((win - f[:, :, None, None]) ** 2) / (2 * sr * sr))
    ref = (w2 * ph * win).sum((2, 3)) / (w2 * ph).sum((2, 3))
    out = O.direct_bf(f, w1, O.BORDER_REFLECT, O.RANGE_GAUSSIAN, sr)[0]
    assert np.max(np.abs(out - ref)) < 1e-10


@pytest.mark.parametrize("border", [O.BORDER_REFLECT, O.BORDER_TRUNCATE])
def test_shift_equivariance(border):
    """Only differences f(i-j) - f(i) enter phi: (f + c) -> fhat + c."""
    w1, fit = _setup(eps=1e-3)
    f = _img(16, 19, seed=11, lo=0, hi=200)
    a = O.direct_sbf(f, w1, border, fit.d, 255.0)[0]
    b = O.direct_sbf(f + 40.0, w1, border, fit.d, 255.0)[0]
    assert np.max(np.abs(b - (a + 40.0))) < 1e-9
    a = O.direct_bf(f, w1, border, O.RANGE_GAUSSIAN, 30.0)[0]
    b = O.direct_bf(f + 40.0, w1, border, O.RANGE_GAUSSIAN, 30.0)[0]
    assert np.max(np.abs(b - (a + 40.0))) < 1e-9


def test_flip_and_transpose_equivariance_reflect():
    w1, fit = _setup(eps=1e-3)
    f = _img(13, 18, seed=2)
    a = O.alg1(f, w1, O.BORDER_REFLECT, fit.d, 255.0)[0]
    assert np.max(np.abs(O.alg1(f.T, w1, O.BORDER_REFLECT, fit.d, 255.0)[0] - a.T)) < 1e-9
    assert np.max(np.abs(O.alg1(f[::-1], w1, O.BORDER_REFLECT, fit.d, 255.0)[0] - a[::-1])) < 1e-9
    assert np.max(np.abs(O.alg1(f[:, ::-1], w1, O.BORDER_REFLECT, fit.d, 255.0)[0] - a[:, ::-1])) < 1e-9


def test_scale_equivariance_filter():
    """(alpha f, alpha sigma_r, alpha T) -> alpha fhat: the [0, 1] / T = 1 workload
    is the uint8 problem scaled by 1/255."""
    f = _img(12, 15, seed=4)
    w1 = O.weights_1d(O.SPATIAL_GAUSSIAN, 2.0, 6)
    a = O.fit(O.RANGE_GAUSSIAN, 25.5, 255.0, 1e-3)
    b = O.fit(O.RANGE_GAUSSIAN, 0.1, 1.0, 1e-3, levels=256)
    oa = O.alg1(f, w1, O.BORDER_REFLECT, a.d, 255.0)[0]
    ob = O.alg1(f / 255.0, w1, O.BORDER_REFLECT, b.d, 1.0)[0]
    assert np.max(np.abs(ob * 255.0 - oa)) < 1e-8


@pytest.mark.parametrize("eps", [1e-5, 1e-3, 1e-2])
def test_accuracy_bound_eq_12_and_appendix(eps):
    """||f_BF - fhat_BF||_inf <= 2 T eps / (w(0) - eps), eq. (12); per pixel the
    Appendix's Q_1 >= w(0), |Q_1 - Q_2| <= eps, |P_1 - P_2| <= T eps."""
    T = 255.0
    f = _img(40, 36, seed=9)
    w1 = O.weights_1d(O.SPATIAL_GAUSSIAN, 3.0, 9)
    w0 = w1[9] ** 2
    fit = O.fit(O.RANGE_GAUSSIAN, 30.0, T, eps)
    o1, P1, Q1 = O.direct_bf(f, w1, O.BORDER_REFLECT, O.RANGE_GAUSSIAN, 30.0)
    o2, P2, Q2 = O.direct_sbf(f, w1, O.BORDER_REFLECT, fit.d, T)
    bound = O.bound12(T, eps, w0)
    assert np.max(np.abs(o1 - o2)) <= bound
    assert np.all(Q1 >= w0 * (1 - 1e-12))
    assert np.max(np.abs(Q1 - Q2)) <= eps
    assert np.max(np.abs(P1 - P2)) <= T * eps
    if eps == 1e-5:
        assert fit.K == 14 and bound < 0.5  # provably sub-pixel


def test_points_and_row_slabs_match_full_evaluation():
    w1, fit = _setup(sigma_s=3.0, eps=1e-3)
    f = _img(37, 29, seed=8)
    for border in (O.BORDER_REFLECT, O.BORDER_TRUNCATE):
        full = O.direct_sbf(f, w1, border, fit.d, 255.0)[0]
        ys = np.array([0, 36, 5, 20, 36, 0])
        xs = np.array([0, 28, 7, 14, 0, 28])
        pts = O.direct_sbf(f, w1, border, fit.d, 255.0, points=(ys, xs))[0]
        assert np.array_equal(pts, full[ys, xs])
        a = O.alg1(f, w1, border, fit.d, 255.0)[0]
        for r0, r1 in ((0, 4), (10, 21), (30, 37)):
            s = O.alg1(f, w1, border, fit.d, 255.0, rows=(r0, r1))[0]
            assert np.max(np.abs(s - a[r0:r1])) < 1e-10


@pytest.mark.parametrize("border", [O.BORDER_REFLECT, O.BORDER_TRUNCATE])
def test_gradient_against_central_differences(border):
    """d/df sum(g * fhat) of eq. (9): closed form vs central differences (FP64)."""
    rng = np.random.default_rng(0)
    f = rng.uniform(0.2, 0.8, size=(7, 9))
    g = rng.normal(size=(7, 9))
    W = 3
    w1 = O.weights_1d(O.SPATIAL_GAUSSIAN, 1.3, W)
    fit = O.fit(O.RANGE_GAUSSIAN, 0.1, 1.0, 1e-3, levels=256)
    gr = O.grad_direct(f, g, w1, border, fit.d, 1.0)
    h = 1e-5
    num = np.zeros_like(f)
    for i in range(f.shape[0]):
        for j in range(f.shape[1]):
            fp = f.copy()
            fp[i, j] += h
            fm = f.copy()
            fm[i, j] -= h
            num[i, j] = (np.sum(g * O.direct_sbf(fp, w1, border, fit.d, 1.0)[0])
                         - np.sum(g * O.direct_sbf(fm, w1, border, fit.d, 1.0)[0])) / (2 * h)
    assert np.max(np.abs(gr - num)) <= 1e-6 * max(1.0, np.max(np.abs(num)))


@pytest.mark.parametrize("border", [O.BORDER_REFLECT, O.BORDER_TRUNCATE])
@pytest.mark.parametrize("shape,W", [((9, 11), 2), ((6, 5), 4), ((12, 10), 3), ((1, 3), 32), ((2, 1), 33)])
def test_gradient_at_points_equals_full_gradient(border, shape, W):
    """The sampled-pixel gradient enumerates the same pairs as the full one
    (including windows wider than the image, where pixels reflect repeatedly:
    a one-row image under W = 32 has 65 row preimages per pixel)."""
    rng = np.random.default_rng(1)
    f = rng.uniform(0.1, 0.9, size=shape)
    g = rng.normal(size=shape)
    w1 = O.weights_1d(O.SPATIAL_GAUSSIAN, 1.5, W)
    fit = O.fit(O.RANGE_GAUSSIAN, 0.1, 1.0, 1e-3, levels=256)
    full = O.grad_direct(f, g, w1, border, fit.d, 1.0)
    ys, xs = np.mgrid[0:shape[0], 0:shape[1]]
    pts = O.grad_at(f, g, w1, border, fit.d, 1.0, (ys.ravel(), xs.ravel()))
    assert np.max(np.abs(pts - full.ravel())) <= 1e-11 * max(1.0, np.max(np.abs(full)))


# ---- local dynamic range T (the definition opening Sec. III) ----------------

@pytest.mark.parametrize("W", [0, 1, 2, 5, 9])
@pytest.mark.parametrize("shape", [(1, 1), (1, 17), (13, 1), (20, 31), (7, 40)])
def test_local_range_equals_max_min_filters(shape, W):
    """Max/min filters with edge replication (scipy) see the same values as the
    clipped window (a replicated pixel lies inside it), so
    T = max(maxfilt(f) - f, f - minfilt(f)) must hold for both borders."""
    ndi = pytest.importorskip("scipy.ndimage")
    from paper_1603_08081_gb300.synth import make_image

    f = make_image(*shape, seed=50 + W).astype(np.float64)
    size = 2 * W + 1
    want = max(np.max(ndi.maximum_filter(f, size=size, mode="nearest") - f),
               np.max(f - ndi.minimum_filter(f, size=size, mode="nearest")))
    for border in (O.BORDER_REFLECT, O.BORDER_TRUNCATE):
        assert O.local_range(f, W, border) == want


def test_local_range_closed_forms():
    rng = np.random.default_rng(3)
    f = rng.integers(0, 256, size=(12, 15)).astype(np.float64)
    # W = 0: every window is the pixel itself
    assert O.local_range(f, 0) == 0.0
    # a window covering the whole image: the full dynamic range
    assert O.local_range(f, 20) == f.max() - f.min()
    # constant image
    assert O.local_range(np.full((9, 9), 77.0), 4) == 0.0
    # a vertical step a | b: any window crossing it sees |a - b|, none sees more
    step = np.full((10, 12), 40.0)
    step[:, 6:] = 217.0
    for W in (1, 3, 11):
        assert O.local_range(step, W) == 177.0
    # an isolated spike of height s on a flat background is seen at distance <= W
    spike = np.zeros((15, 15))
    spike[7, 7] = 90.0
    assert O.local_range(spike, 2) == 90.0
    # monotone in W
    g = rng.integers(0, 256, size=(30, 30)).astype(np.float64)
    vals = [O.local_range(g, W) for W in range(0, 8)]
    assert all(a <= b for a, b in zip(vals, vals[1:]))


def test_local_range_gives_fewer_terms():
    """Sec. III: a smaller T needs fewer terms for the same sigma_r and eps (here
    K = 10 at T = 217 against K = 11 at T = 255 for sigma_r = 30, eps = 1e-3)."""
    assert O.fit(O.RANGE_GAUSSIAN, 30.0, 217.0, 1e-3).K == 10
    assert O.fit(O.RANGE_GAUSSIAN, 30.0, 255.0, 1e-3).K == 11
