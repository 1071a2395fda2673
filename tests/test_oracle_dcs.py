"""Pins of the oracle's Cauchy-Schwarz divergence (Eq. (1)) and its gradient.

* Eq. (1) from normalised Parzen densities (Eq. (dens1)/(dens2), xi = omega = sigma/sqrt(2)) with
  every overlap integral done by dense numerical quadrature equals the oracle's unnormalised
  log S_WW + log S_XX - 2 log S_XW (this pins the reading of sigma and the cancelled constants);
* hand-derived closed forms (``tests/golden/two_pixels.json``);
* D_cs = 0 when the data are the codebook, D_cs >= 0 (Cauchy-Schwarz), invariance under h -> a h,
  <dD/dh, h> = 0 (degree-0 homogeneity);
* the analytic gradient against FP64 central differences, and the point-list gradient against
  the dense-image gradient;
* the step <-> gradient identity w' - w = -(sigma^2 S_XW / (2 a_k)) dD/dw_k.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_1310_7114_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _all_sites(h):
    H, W = h.shape
    u, v = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    return np.stack([u.ravel(), v.ravel()], 1).astype(float), h.ravel().astype(float)


def test_dcs_equals_quadrature_of_normalised_parzen_densities():
    sigma = 1.4
    xi = om = sigma / math.sqrt(2.0)
    pts = np.array([[2.0, 2.0], [3.0, 5.0], [6.0, 3.0], [5.0, 6.0]])
    hx = np.array([1.0, 0.6, 0.8, 0.3])
    W = np.array([[3.0, 3.0], [5.0, 5.0], [2.0, 6.0]])
    t = np.arange(-10.0, 18.0, 0.025)
    U, V = np.meshgrid(t, t, indexing="ij")

    def G(c, s):
        return np.exp(-((U - c[0]) ** 2 + (V - c[1]) ** 2) / (2 * s * s)) / (2 * np.pi * s * s)

    p = sum(w * G(x, xi) for x, w in zip(pts, hx)) / hx.sum()
    q = sum(G(w, om) for w in W) / len(W)
    V_xw, V_w, V_x = (p * q).sum(), (q * q).sum(), (p * p).sum()
    d_quad = -2 * math.log(V_xw) + math.log(V_w) + math.log(V_x)
    d_orc = oracle.dcs((9, 9), pts, hx, sigma, W, trunc=12.0)
    assert abs(d_quad - d_orc) < 1e-9, (d_quad, d_orc)


def test_golden_two_pixels():
    g = json.load(open(os.path.join(GOLDEN, "two_pixels.json")))
    ns = {"log": math.log, "exp": math.exp}
    h = np.zeros(g["lattice"])
    for u, v in g["pixels"]:
        h[u, v] = 1.0
    X, hx = oracle.image_points(h)
    A, Fu, Fv = oracle.fields2d(h, g["sigma"], trunc=g["trunc"])
    for case in g["cases"]:
        W = np.array(case["W"], float)
        d = oracle.dcs(h.shape, X, hx, g["sigma"], W, trunc=g["trunc"])
        assert abs(d - eval(case["dcs"], ns)) < 1e-14
        _, Wraw, _ = oracle.lattice_step(A, [Fu, Fv], g["sigma"], W, snap=False)
        np.testing.assert_allclose(Wraw[0], [eval(e, ns) for e in case["step"]], atol=1e-14)
        gW, _ = oracle.dcs_grad(h.shape, X, hx, g["sigma"], W, trunc=g["trunc"])
        np.testing.assert_allclose(gW[0], [eval(e, ns) for e in case["grad"]], atol=1e-14)


def test_dcs_zero_when_data_are_the_codebook_and_nonnegative():
    W = np.array([[2.0, 3.0], [7.0, 4.0], [5.0, 9.0]])
    assert abs(oracle.dcs((12, 12), W, np.ones(3), 1.5, W, trunc=12.0)) < 1e-13
    rng = np.random.default_rng(0)
    for _ in range(20):
        X = rng.integers(0, 16, (12, 2)).astype(float)
        hx = rng.random(12)
        Wr = rng.integers(0, 16, (4, 2)).astype(float)
        assert oracle.dcs((16, 16), X, hx, 2.0, Wr, trunc=12.0) >= -1e-12


def test_scale_invariance_and_homogeneity():
    rng = np.random.default_rng(1)
    h = (rng.random((18, 20)) < 0.4) * rng.random((18, 20))
    X, hx = _all_sites(h)
    W = np.array([[4.0, 5.0], [10.0, 12.0], [14.0, 3.0]])
    d1 = oracle.dcs(h.shape, X, hx, 2.0, W)
    d2 = oracle.dcs(h.shape, X, 3.7 * hx, 2.0, W)
    assert abs(d1 - d2) < 1e-13
    _, gh = oracle.dcs_grad(h.shape, X, hx, 2.0, W)
    assert abs(np.dot(gh, hx)) < 1e-12 * np.abs(gh).sum()


@pytest.mark.parametrize("sigma", [1.5, (2.0, 1.2)])
def test_gradient_matches_central_differences(sigma):
    rng = np.random.default_rng(2)
    h = (rng.random((16, 18)) < 0.5) * rng.random((16, 18))
    X, hx = _all_sites(h)
    W = np.array([[4.0, 5.0], [9.0, 12.0], [12.0, 3.0], [6.0, 9.0]])
    gW, gh = oracle.dcs_grad(h.shape, X, hx, sigma, W)
    eps = 1e-4
    fd_w = np.zeros_like(W)
    for k in range(W.shape[0]):
        for i in range(2):
            Wp, Wm = W.copy(), W.copy()
            Wp[k, i] += eps
            Wm[k, i] -= eps
            fd_w[k, i] = (oracle.dcs(h.shape, X, hx, sigma, Wp) - oracle.dcs(h.shape, X, hx, sigma, Wm)) / (2 * eps)
    np.testing.assert_allclose(gW, fd_w, rtol=1e-6, atol=1e-9)
    idx = rng.choice(hx.size, 24, replace=False)
    fd_h = []
    for p in idx:
        hp, hm = hx.copy(), hx.copy()
        hp[p] += eps
        hm[p] -= eps
        fd_h.append((oracle.dcs(h.shape, X, hp, sigma, W) - oracle.dcs(h.shape, X, hm, sigma, W)) / (2 * eps))
    np.testing.assert_allclose(gh[idx], fd_h, rtol=1e-6, atol=1e-9)


def test_dense_gradient_equals_point_list_gradient():
    rng = np.random.default_rng(3)
    h = (rng.random((21, 17)) < 0.5) * rng.random((21, 17))
    X, hx = _all_sites(h)
    W = np.array([[4.0, 5.0], [9.0, 12.0], [18.0, 3.0]])
    gW, gh = oracle.dcs_grad(h.shape, X, hx, 2.0, W)
    gW2, gh2, sums = oracle.dcs_grad2d_dense(h, 2.0, W)
    np.testing.assert_allclose(gW2, gW, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(gh2.ravel(), gh, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(sums, oracle.dcs_sums(h.shape, X, hx, 2.0, W), rtol=1e-13)


def test_step_gradient_identity():
    """w' - w = -(sigma^2 S_XW / (2 a_k)) dD/dw_k: the update is a preconditioned gradient step."""
    img = synth.c1_image(1)
    A, Fu, Fv = oracle.fields2d(img, 2.0)
    W = synth.init_codebook(synth.rng_for(1, 1), img.astype(np.float32), 8).astype(float)
    _, Wraw, st = oracle.lattice_step(A, [Fu, Fv], 2.0, W, snap=False)
    X, hx = oracle.image_points(img)
    gW, _ = oracle.dcs_grad(img.shape, X, hx, 2.0, W, with_h=False)
    a = A[W[:, 0].astype(int), W[:, 1].astype(int)]
    pred = W - (4.0 * st["sxw"] / (2 * a))[:, None] * gW
    np.testing.assert_allclose(Wraw, pred, rtol=0, atol=1e-10)


def test_3d_gradient_matches_central_differences():
    rng = np.random.default_rng(5)
    gray = rng.integers(0, 12, (8, 9))
    hw = rng.random((8, 9))
    X, hx = oracle.gray_points(gray, hw)
    sig = (1.3, 1.6, 2.0)
    W = np.array([[3.0, 4.0, 5.0], [6.0, 2.0, 8.0], [2.0, 7.0, 3.0]])
    shape = (8, 9, 12)
    gW, gh = oracle.dcs_grad(shape, X, hx, sig, W)
    eps = 1e-4
    for k in range(3):
        for i in range(3):
            Wp, Wm = W.copy(), W.copy()
            Wp[k, i] += eps
            Wm[k, i] -= eps
            fd = (oracle.dcs(shape, X, hx, sig, Wp) - oracle.dcs(shape, X, hx, sig, Wm)) / (2 * eps)
            assert abs(fd - gW[k, i]) < 1e-6 * max(1.0, abs(fd))
    for p in rng.choice(hx.size, 10, replace=False):
        hp, hm = hx.copy(), hx.copy()
        hp[p] += eps
        hm[p] -= eps
        fd = (oracle.dcs(shape, X, hp, sig, W) - oracle.dcs(shape, X, hm, sig, W)) / (2 * eps)
        assert abs(fd - gh[p]) < 1e-6 * max(1.0, abs(fd))


def test_planted_sign_error_in_the_update_is_caught():
    """A copy of the update with the repulsion term's sign flipped (a plausible transcription
    slip in Eq. (origupdate)) breaks the step <-> gradient identity the oracle satisfies."""
    img = synth.c1_image(2)
    A, Fu, Fv = oracle.fields2d(img, 2.0)
    W = synth.init_codebook(synth.rng_for(1, 2), img.astype(np.float32), 8).astype(float)
    _, Wraw, st = oracle.lattice_step(A, [Fu, Fv], 2.0, W, snap=False)
    X, hx = oracle.image_points(img)
    gW, _ = oracle.dcs_grad(img.shape, X, hx, 2.0, W, with_h=False)
    a = A[W[:, 0].astype(int), W[:, 1].astype(int)]
    # the correct update's repulsion part is Wraw - (W + D/a); flipping it moves the result by
    # twice that amount
    Dk = np.stack([Fu[W[:, 0].astype(int), W[:, 1].astype(int)], Fv[W[:, 0].astype(int), W[:, 1].astype(int)]], 1)
    mutated = 2 * (W + Dk / a[:, None]) - Wraw
    pred = W - (4.0 * st["sxw"] / (2 * a))[:, None] * gW
    assert np.abs(mutated - pred).max() > 1e-3
    assert np.abs(Wraw - pred).max() < 1e-10


def test_dense_dcs_equals_point_list_definition():
    rng = np.random.default_rng(7)
    h = (rng.random((20, 22)) < 0.4) * rng.random((20, 22))
    X, hx = _all_sites(h)
    for W in (np.array([[4.0, 5.0], [10.0, 12.0]]), np.array([[4.3, 5.8], [0.2, 21.0], [19.6, 3.1]])):
        assert abs(oracle.dcs2d_dense(h, 2.0, W) - oracle.dcs(h.shape, X, hx, 2.0, W)) < 1e-12
