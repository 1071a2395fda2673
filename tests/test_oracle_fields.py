"""Pins of the oracle's lattice fields (Sec. 3.1, Sec. 5, Sec. 1 (ii)) against things other than itself.

* two independent implementations (direct windowed sum vs separable passes);
* a library routine (``scipy.signal.correlate2d`` with the truncated kernel);
* closed forms (single pixel, all-ones interior, linearity, translation, transpose);
* the untruncated Parzen sum by brute force over all points, and the truncation bound.
"""
import numpy as np
import pytest
from scipy.signal import correlate2d

import oracle


def _g(d, s):
    return np.exp(-np.asarray(d, float) ** 2 / (2 * s * s))


def _rand_img(rng, H, W, p=0.3, weighted=False):
    on = rng.random((H, W)) < p
    if weighted:
        return on * rng.random((H, W))
    return on.astype(np.float64)


@pytest.mark.parametrize("sig", [(2.0, 2.0), (1.5, 2.5), (3.0, 1.0)])
@pytest.mark.parametrize("absolute", [False, True])
@pytest.mark.parametrize("weighted", [False, True])
def test_direct_equals_separable(sig, absolute, weighted):
    rng = np.random.default_rng(7)
    h = _rand_img(rng, 23, 31, 0.3, weighted)
    d = oracle.fields2d(h, sig, absolute=absolute, method="direct")
    s = oracle.fields2d(h, sig, absolute=absolute, method="separable")
    scale = np.abs(d[0]).max() * (40 if absolute else 10)
    for a, b in zip(d, s):
        np.testing.assert_allclose(a, b, rtol=1e-13, atol=1e-13 * scale)


@pytest.mark.parametrize("sigma", [1.0, 2.0, 3.0])
def test_fields_match_library_correlation(sigma):
    """A, F_u, F_v, B_u, B_v equal scipy's zero-padded 2-D correlation with the truncated mask."""
    rng = np.random.default_rng(11)
    h = _rand_img(rng, 40, 33, 0.25, weighted=True)
    R = oracle.radius(sigma)
    d = np.arange(-R, R + 1)
    K = np.outer(_g(d, sigma), _g(d, sigma))
    Ku = K * d[:, None]
    Kv = K * d[None, :]
    corr = lambda img, k: correlate2d(img, k, mode="same", boundary="fill", fillvalue=0.0)
    A, Fu, Fv = oracle.fields2d(h, sigma)
    np.testing.assert_allclose(A, corr(h, K), rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(Fu, corr(h, Ku), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(Fv, corr(h, Kv), rtol=1e-12, atol=1e-12)
    uu, vv = np.meshgrid(np.arange(40), np.arange(33), indexing="ij")
    _, Bu, Bv = oracle.fields2d(h, sigma, absolute=True)
    np.testing.assert_allclose(Bu, corr(uu * h, K), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(Bv, corr(vv * h, K), rtol=1e-12, atol=1e-12)


def test_single_pixel_is_the_kernel():
    H, W, s = 31, 29, 2.0
    h = np.zeros((H, W))
    h[14, 9] = 1.0
    A, Fu, Fv = oracle.fields2d(h, s)
    R = oracle.radius(s)
    uu, vv = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    inside = (np.abs(uu - 14) <= R) & (np.abs(vv - 9) <= R)
    ref = np.where(inside, _g(uu - 14, s) * _g(vv - 9, s), 0.0)
    np.testing.assert_allclose(A, ref, rtol=1e-14, atol=0)
    np.testing.assert_allclose(Fu, ref * (14 - uu), rtol=1e-14, atol=1e-300)
    np.testing.assert_allclose(Fv, ref * (9 - vv), rtol=1e-14, atol=1e-300)
    assert np.all(A[~inside] == 0) and np.all(Fu[~inside] == 0)


def test_all_ones_interior_closed_form():
    s = 2.5
    R = oracle.radius(s)
    h = np.ones((40, 40))
    A, Fu, Fv = oracle.fields2d(h, s)
    s1 = _g(np.arange(-R, R + 1), s).sum()
    interior = (slice(R, 40 - R), slice(R, 40 - R))
    np.testing.assert_allclose(A[interior], s1 * s1, rtol=1e-14)
    assert np.abs(Fu[interior]).max() < 1e-12 and np.abs(Fv[interior]).max() < 1e-12
    # at the top-left corner only the quadrant d >= 0 is inside the lattice
    q = _g(np.arange(0, R + 1), s).sum()
    np.testing.assert_allclose(A[0, 0], q * q, rtol=1e-14)


def test_linearity_translation_transpose():
    rng = np.random.default_rng(3)
    h1, h2 = _rand_img(rng, 20, 24, 0.3, True), _rand_img(rng, 20, 24, 0.3, True)
    f1, f2 = oracle.fields2d(h1, 1.7), oracle.fields2d(h2, 1.7)
    f12 = oracle.fields2d(2.0 * h1 - 0.5 * h2, 1.7)
    for a, b, c in zip(f1, f2, f12):
        np.testing.assert_allclose(c, 2.0 * a - 0.5 * b, rtol=1e-12, atol=1e-12)
    # translation: the same image placed at two offsets inside zero canvases; the centred fields
    # move with it
    fp = oracle.fields2d(np.pad(h1, ((15, 25), (20, 20))), 1.7)
    shifted = oracle.fields2d(np.pad(h1, ((17, 23), (25, 15))), 1.7)
    for a, b in zip(fp, shifted):
        np.testing.assert_allclose(a[15:35, 20:44], b[17:37, 25:49], rtol=1e-14, atol=1e-14)
    # transpose swaps the roles of u and v
    A, Fu, Fv = oracle.fields2d(h1, (1.2, 2.2))
    At, Fut, Fvt = oracle.fields2d(h1.T, (2.2, 1.2))
    np.testing.assert_allclose(At, A.T, rtol=1e-14)
    np.testing.assert_allclose(Fut, Fv.T, rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(Fvt, Fu.T, rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("sigma", [1.5, 2.0])
def test_untruncated_parzen_sum_and_truncation_bound(sigma):
    """With a wide mask the field is the Parzen sum over all points (Sec. 3.1 convolution identity);
    with the 3-sigma mask it is below it by at most the kernel mass outside the box."""
    rng = np.random.default_rng(5)
    h = _rand_img(rng, 30, 30, 0.2)
    X, w = oracle.image_points(h)
    uu, vv = np.meshgrid(np.arange(30), np.arange(30), indexing="ij")
    Y = np.stack([uu.ravel(), vv.ravel()], 1).astype(float)
    d2 = ((Y[:, None, :] - X[None, :, :]) ** 2).sum(-1)
    full = (np.exp(-d2 / (2 * sigma * sigma)) * w[None, :]).sum(1).reshape(30, 30)
    Awide = oracle.fields2d(h, sigma, trunc=12.0)[0]
    np.testing.assert_allclose(Awide, full, rtol=1e-12)
    A3 = oracle.fields2d(h, sigma, trunc=3.0)[0]
    R = oracle.radius(sigma)
    s_in = _g(np.arange(-R, R + 1), sigma).sum()
    s_all = _g(np.arange(-200, 201), sigma).sum()
    assert np.all(A3 <= full + 1e-12)
    assert np.all(full - A3 <= s_all ** 2 - s_in ** 2 + 1e-12)
    # for the 3-sigma mask the 2-D mass outside the box is below 0.6 % of the total
    assert (s_all ** 2 - s_in ** 2) / s_all ** 2 < 6e-3


def test_sites_equal_dense():
    rng = np.random.default_rng(9)
    h = _rand_img(rng, 25, 19, 0.3, True)
    dense = oracle.fields2d(h, 2.0, method="direct")
    sites = np.stack([rng.integers(0, 25, 40), rng.integers(0, 19, 40)], 1)
    sp = oracle.fields2d_sites(h, 2.0, sites)
    for a, b in zip(dense, sp):
        np.testing.assert_array_equal(a[sites[:, 0], sites[:, 1]], b)


# ----------------------------------------------------------------------------------- 3-D lattice
def _gray(rng, H, W, G):
    return rng.integers(0, G, (H, W))


@pytest.mark.parametrize("absolute", [False, True])
def test_3d_direct_equals_separable(absolute):
    rng = np.random.default_rng(21)
    gray = _gray(rng, 12, 13, 20)
    hw = rng.random((12, 13))
    sig = (1.5, 1.0, 2.0)
    d = oracle.fields3d(gray, 20, sig, hw=hw, absolute=absolute, method="direct")
    s = oracle.fields3d(gray, 20, sig, hw=hw, absolute=absolute, method="separable")
    scale = np.abs(d[0]).max() * 30
    for a, b in zip(d, s):
        np.testing.assert_allclose(a, b, rtol=1e-13, atol=1e-13 * scale)


def test_3d_reduces_to_2d_on_a_constant_gray_image():
    """A constant gray level c puts every pixel on slice c: slice g of the volume is the 2-D field
    scaled by the g-axis kernel at g - c, with F_g = (c - g) A."""
    rng = np.random.default_rng(4)
    hw = _rand_img(rng, 14, 16, 0.4, True)
    gray = np.full((14, 16), 5)
    sig = (1.5, 2.0, 1.7)
    A3, Fu3, Fv3, Fg3 = oracle.fields3d(gray, 12, sig, hw=hw)
    A2, Fu2, Fv2 = oracle.fields2d(hw, sig[:2])
    Rg = oracle.radius(sig[2])
    for g in range(12):
        k = _g(g - 5, sig[2]) if abs(g - 5) <= Rg else 0.0
        np.testing.assert_allclose(A3[g], k * A2, rtol=1e-13, atol=1e-300)
        np.testing.assert_allclose(Fu3[g], k * Fu2, rtol=1e-13, atol=1e-14)
        np.testing.assert_allclose(Fv3[g], k * Fv2, rtol=1e-13, atol=1e-14)
        np.testing.assert_allclose(Fg3[g], (5 - g) * k * A2, rtol=1e-13, atol=1e-14)


def test_3d_untruncated_brute_force():
    rng = np.random.default_rng(8)
    gray = _gray(rng, 9, 10, 15)
    sig = (1.2, 1.4, 2.0)
    A = oracle.fields3d(gray, 15, sig, trunc=12.0)[0]
    X, w = oracle.gray_points(gray)
    gg, uu, vv = np.meshgrid(np.arange(15), np.arange(9), np.arange(10), indexing="ij")
    Y = np.stack([uu.ravel(), vv.ravel(), gg.ravel()], 1).astype(float)
    s2 = np.array(sig) ** 2
    d2 = (((Y[:, None, :] - X[None, :, :]) ** 2) / (2 * s2)).sum(-1)
    full = np.exp(-d2).sum(1).reshape(15, 9, 10)
    np.testing.assert_allclose(A, full, rtol=1e-12)


def test_3d_sites_equal_dense():
    rng = np.random.default_rng(10)
    gray = _gray(rng, 11, 12, 16)
    dense = oracle.fields3d(gray, 16, (1.0, 1.5, 2.0), method="direct")
    sites = np.stack([rng.integers(0, 11, 30), rng.integers(0, 12, 30), rng.integers(0, 16, 30)], 1)
    sp = oracle.fields3d_sites(gray, sites, 16, (1.0, 1.5, 2.0))
    for a, b in zip(dense, sp):
        np.testing.assert_array_equal(a[sites[:, 2], sites[:, 0], sites[:, 1]], b)
