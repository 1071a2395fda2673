"""Pins of the oracle's recursive Gaussian fields (Sec. 3.1: recursive filters for large widths;
Deriche's damped-sinusoid fit computed by first-order complex recursions).

* the recursions equal the direct convolution with the fitted kernel, value and first moment,
  to rounding, for several widths (so the recursion adds nothing to the fit);
* the fit itself is within 6e-4 of exp(-x^2/2) everywhere (pins the published constants);
* 2-D recursive fields differ from the exact, untruncated Gaussian fields by no more than the
  fit error summed over the kernel (a rigorous bound computed in the test), for A and both
  centred moments;
* closed forms: a single pixel gives A = k(|du|/s) k(|dv|/s) and F_i = (x_i - y_i) A exactly;
  absolute moments are centred moments plus y_i A.
"""
import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("sigma", [1.5, 4.0, 15.0, 40.0])
def test_recursion_equals_direct_sum_of_the_fit(sigma):
    rng = np.random.default_rng(int(sigma * 10))
    x = rng.random(131) * (rng.random(131) < 0.5)
    y, yd = oracle.deriche_filter(x, sigma)
    n = np.arange(131)
    D = n[None, :] - n[:, None]
    K = oracle.deriche_kernel(np.abs(D).ravel() / sigma).reshape(D.shape)
    scale = np.abs(x).sum()
    assert np.abs(y - (K * x[None, :]).sum(1)).max() <= 1e-13 * scale
    assert np.abs(yd - (K * D * x[None, :]).sum(1)).max() <= 1e-13 * scale * 131


def test_fit_is_close_to_the_gaussian():
    t = np.linspace(0.0, 12.0, 4001)
    assert np.abs(oracle.deriche_kernel(t) - np.exp(-t * t / 2)).max() <= 6e-4


def _fit_bound(sigma, R, w=0):
    """sum over offsets of |k_u k_v |d_i|^w - g_u g_v |d_i|^w|: the largest change of a field per
    unit of h."""
    d = np.arange(-R, R + 1, dtype=float)
    k = oracle.deriche_kernel(np.abs(d) / sigma)
    g = np.exp(-d * d / (2 * sigma * sigma))
    m = np.abs(d) ** w
    return np.abs(np.outer(k * m, k) - np.outer(g * m, g)).sum()


@pytest.mark.parametrize("sigma", [3.0, 6.0])
def test_fields_within_the_fit_error_of_the_exact_gaussian(sigma):
    rng = np.random.default_rng(7)
    h = (rng.random((70, 90)) < 0.3) * rng.random((70, 90))
    A, Fu, Fv = oracle.fields2d_recursive(h, sigma)
    R = int(np.ceil(12 * sigma))
    Ae, Fue, Fve = oracle.fields2d(h, sigma, R=(R, R))     # untruncated in practice (12 sigma)
    hm = h.max()
    assert np.abs(A - Ae).max() <= hm * _fit_bound(sigma, R)
    assert np.abs(Fu - Fue).max() <= hm * _fit_bound(sigma, R, 1)
    assert np.abs(Fv - Fve).max() <= hm * _fit_bound(sigma, R, 1)
    # and the bound is tight enough to matter: under 1 % of the field's range
    assert hm * _fit_bound(sigma, R) <= 0.01 * A.max()


def test_single_pixel_closed_forms():
    h = np.zeros((40, 50))
    h[17, 23] = 2.0
    s = 5.0
    A, Fu, Fv = oracle.fields2d_recursive(h, s)
    u, v = np.meshgrid(np.arange(40), np.arange(50), indexing="ij")
    ku = oracle.deriche_kernel(np.abs(u - 17).ravel() / s).reshape(u.shape)
    kv = oracle.deriche_kernel(np.abs(v - 23).ravel() / s).reshape(v.shape)
    assert np.allclose(A, 2.0 * ku * kv, rtol=0, atol=1e-13)
    assert np.allclose(Fu, (17 - u) * A, rtol=0, atol=1e-12)
    assert np.allclose(Fv, (23 - v) * A, rtol=0, atol=1e-12)
    Aa, Fua, Fva = oracle.fields2d_recursive(h, s, absolute=True)
    assert np.allclose(Fua, Fu + u * A, atol=1e-11) and np.allclose(Fva, Fv + v * A, atol=1e-11)
