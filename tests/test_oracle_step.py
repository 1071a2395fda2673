"""Pins of the oracle's fixed-point update (Sec. 2.1 Eq. (origupdate), Sec. 3.1 Eq. (accupdate),
Algorithm 1) against things other than itself.

* M = 1 removes the repulsion term: the update is one Gaussian mean-shift step (Sec. 2.2), i.e. the
  kernel-weighted average of the data in the window, computed here with ``numpy.average``;
* with a wide mask and integral W, the lattice step (centred-moment form) equals the three-term
  Eq. (origupdate) evaluated over the point list;
* Eq. (accupdate) with its integrals evaluated by dense numerical quadrature of the normalised
  Parzen densities equals the oracle step with step_scale 1/2 (the reading of the two update rules);
* mirror symmetry, merged codebooks, the fixed-point invariant, empty support.
"""
import numpy as np
import pytest

import oracle
from paper_1310_7114_gb300 import synth


def _g(d, s):
    return np.exp(-np.asarray(d, float) ** 2 / (2 * s * s))


def _fields(h, sigma, trunc=3.0):
    A, Fu, Fv = oracle.fields2d(h, sigma, trunc=trunc)
    return A, [Fu, Fv]


@pytest.mark.parametrize("sigma", [1.5, 2.0, 3.0])
def test_single_codebook_is_a_mean_shift_step(sigma):
    rng = np.random.default_rng(1)
    h = (rng.random((40, 40)) < 0.3) * rng.random((40, 40))
    A, F = _fields(h, sigma)
    R = oracle.radius(sigma)
    for w in [(20, 20), (3, 37), (0, 0), (39, 12)]:
        Wn, Wraw, st = oracle.lattice_step(A, F, sigma, np.array([w], float), snap=False)
        u0, u1 = max(0, w[0] - R), min(40, w[0] + R + 1)
        v0, v1 = max(0, w[1] - R), min(40, w[1] + R + 1)
        uu, vv = np.meshgrid(np.arange(u0, u1), np.arange(v0, v1), indexing="ij")
        wt = h[u0:u1, v0:v1] * _g(uu - w[0], sigma) * _g(vv - w[1], sigma)
        ref = [np.average(uu, weights=wt), np.average(vv, weights=wt)]
        np.testing.assert_allclose(Wraw[0], ref, rtol=0, atol=1e-12)
        snapped, _, _ = oracle.lattice_step(A, F, sigma, np.array([w], float), snap=True)
        np.testing.assert_array_equal(snapped[0], np.clip(np.floor(np.array(ref) + 0.5), 0, 39))


def test_single_pixel_in_window_attracts_exactly():
    h = np.zeros((30, 30))
    h[12, 17] = 1.0
    A, F = _fields(h, 2.0)
    Wn, Wraw, _ = oracle.lattice_step(A, F, 2.0, np.array([[15.0, 13.0]]), snap=False)
    np.testing.assert_allclose(Wraw[0], [12.0, 17.0], atol=1e-12)


def test_original_itc_single_codebook_is_untruncated_mean_shift():
    rng = np.random.default_rng(2)
    X = rng.uniform(0, 20, (50, 2))
    w = np.array([[8.0, 11.0]])
    out = oracle.original_step(X, 2.5, w)
    wt = np.exp(-((X - w) ** 2).sum(1) / (2 * 2.5 ** 2))
    np.testing.assert_allclose(out[0], np.average(X, axis=0, weights=wt), rtol=1e-13)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_lattice_step_equals_original_update_without_truncation(seed):
    """At integral W and with a mask wide enough that truncation is below FP64 resolution, the
    centred lattice form w + (D - cE)/a and the three terms of Eq. (origupdate) agree."""
    img = synth.c1_image(seed)
    rng = synth.rng_for(1, seed)
    W0 = synth.init_codebook(rng, img.astype(np.float32), 8).astype(float)
    for sigma in (2.0, (1.5, 2.5)):
        sig = (sigma, sigma) if np.isscalar(sigma) else sigma
        A, F = _fields(img, sig, trunc=10.0)
        _, Wraw, st = oracle.lattice_step(A, F, sig, W0, snap=False)
        X, hx = oracle.image_points(img)
        ref = oracle.original_step(X, sig, W0, hx)
        inside = np.all((ref >= 0) & (ref <= 63), axis=1)
        np.testing.assert_allclose(Wraw[inside], ref[inside], rtol=0, atol=1e-9)


def test_accupdate_by_quadrature_is_the_half_step():
    """Eq. (accupdate) with p, q the normalised Parzen densities of Eq. (dens1)/(dens2),
    xi = omega = sigma/sqrt(2), and every integral done by dense quadrature, equals the oracle
    step with step_scale 1/2 (wide mask, integral W, continuous state)."""
    sigma = 1.3
    xi = om = sigma / np.sqrt(2.0)
    h = np.zeros((8, 9))
    pts = [(2, 2, 1.0), (3, 5, 0.7), (5, 3, 0.4), (6, 7, 1.0), (4, 4, 0.9)]
    for u, v, w in pts:
        h[u, v] = w
    W = np.array([[3.0, 3.0], [5.0, 6.0]])
    t = np.arange(-9.0, 18.0, 0.02)
    U, V = np.meshgrid(t, t, indexing="ij")

    def G(cu, cv, s):
        return np.exp(-((U - cu) ** 2 + (V - cv) ** 2) / (2 * s * s)) / (2 * np.pi * s * s)

    N = sum(p[2] for p in pts)
    p = sum(w * G(u, v, xi) for u, v, w in pts) / N
    q = sum(G(a, b, om) for a, b in W) / len(W)
    c = (p * q).sum() / (q * q).sum()
    ref = []
    for a, b in W:
        Gk = G(a, b, om)
        den = (p * Gk).sum()
        num = np.array([(p * Gk * U).sum(), (p * Gk * V).sum()])
        qx = np.array([(q * Gk * U).sum(), (q * Gk * V).sum()])
        qd = (q * Gk).sum()
        ref.append((num - c * qx + c * qd * np.array([a, b])) / den)
    A, F = _fields(h, sigma, trunc=10.0)
    _, Wraw, _ = oracle.lattice_step(A, F, sigma, W, step_scale=0.5, snap=False)
    np.testing.assert_allclose(Wraw, np.array(ref), rtol=0, atol=1e-8)


def test_mirror_symmetry():
    rng = np.random.default_rng(4)
    half = (rng.random((32, 16)) < 0.3).astype(float)
    h = np.concatenate([half, half[:, ::-1]], axis=1)  # symmetric under v -> 31 - v
    A, F = _fields(h, 2.0)
    Wl = np.array([[5.0, 3.0], [20.0, 10.0], [28.0, 14.0]])
    W = np.concatenate([Wl, np.stack([Wl[:, 0], 31 - Wl[:, 1]], 1)])
    _, Wraw, _ = oracle.lattice_step(A, F, 2.0, W, snap=False)
    np.testing.assert_allclose(Wraw[3:, 0], Wraw[:3, 0], atol=1e-12)
    np.testing.assert_allclose(Wraw[3:, 1], 31 - Wraw[:3, 1], atol=1e-12)


def test_merged_codebooks_stay_merged():
    img = synth.c1_image(0)
    A, F = _fields(img, 2.0)
    W = synth.init_codebook(synth.rng_for(1, 0), img.astype(np.float32), 6).astype(float)
    W[3] = W[1]
    for _ in range(10):
        W, _, _ = oracle.lattice_step(A, F, 2.0, W)
        np.testing.assert_array_equal(W[3], W[1])


def test_fixed_point_invariant():
    img = synth.c1_image(0)
    A, F = _fields(img, 2.0)
    W0 = synth.init_codebook(synth.rng_for(1, 0), img.astype(np.float32), 8)
    Ws, dcs, tie, t = oracle.lattice_run(A, F, oracle.sxx(img, A), 2.0, W0, 200, stop_on_fixed=True)
    assert t < 200, "did not reach a lattice fixed point"
    W2, _, st = oracle.lattice_step(A, F, 2.0, Ws)
    assert st["moved"] == 0
    np.testing.assert_array_equal(W2, Ws)


def test_empty_support_keeps_codebook():
    h = np.zeros((40, 40))
    h[5:9, 5:9] = 1.0
    A, F = _fields(h, 2.0)
    W = np.array([[6.0, 6.0], [35.0, 35.0]])
    Wn, _, st = oracle.lattice_step(A, F, 2.0, W)
    assert st["empty"] == 1
    np.testing.assert_array_equal(Wn[1], W[1])


def test_stepped_codebooks_lie_on_the_shape():
    """ITC centres end on the shape (Sec. 4, Fig. 2 caption): after 50 iterations on C1 every
    codebook vector sits on or next to a foreground pixel."""
    img = synth.c1_image(0)
    A, F = _fields(img, 2.0)
    W0 = synth.init_codebook(synth.rng_for(1, 0), img.astype(np.float32), 8)
    Ws, dcs, tie, t = oracle.lattice_run(A, F, oracle.sxx(img, A), 2.0, W0, 50)
    u, v = np.nonzero(img)
    for w in Ws:
        assert np.min(np.abs(u - w[0]) + np.abs(v - w[1])) <= 2


def test_run_divergence_equals_direct_definition_and_both_iterations_descend():
    """The D_cs that the lattice run reports from its fields equals Eq. (1) evaluated directly
    from the point list at the same W; original (Eq. (origupdate)) and lattice iterations both
    lower D_cs from the initial codebook.  How close their final codebooks are is not pinned
    (Sec. 4 says only "almost identical"; at sigma = 2 the snapped iteration stops at a lattice
    fixed point once every update is below half a pixel)."""
    for seed in range(3):
        img = synth.c1_image(seed)
        A, F = _fields(img, 2.0)
        W0 = synth.init_codebook(synth.rng_for(1, seed), img.astype(np.float32), 8).astype(float)
        X, hx = oracle.image_points(img)
        Wl, dcs_run, _, t = oracle.lattice_run(A, F, oracle.sxx(img, A), 2.0, W0, 50)
        d0 = oracle.dcs(img.shape, X, hx, 2.0, W0)
        dl = oracle.dcs(img.shape, X, hx, 2.0, Wl)
        np.testing.assert_allclose(dcs_run[0], d0, rtol=1e-12)
        np.testing.assert_allclose(dcs_run[-1], dl, rtol=1e-12)
        Wo = oracle.original_run(X, 2.0, W0, 50, hx)
        assert dl < d0 and oracle.dcs(img.shape, X, hx, 2.0, Wo) < d0


def test_3d_step_mean_shift_and_original():
    rng = np.random.default_rng(6)
    gray = rng.integers(0, 24, (14, 15))
    sig = (1.5, 1.5, 3.0)
    A, Fu, Fv, Fg = oracle.fields3d(gray, 24, sig, trunc=10.0)
    W = np.array([[7.0, 7.0, 12.0], [3.0, 10.0, 5.0], [11.0, 2.0, 20.0]])
    _, Wraw, _ = oracle.lattice_step(A, [Fu, Fv, Fg], sig, W, snap=False)
    X, hx = oracle.gray_points(gray)
    ref = oracle.original_step(X, sig, W, hx)
    np.testing.assert_allclose(Wraw, ref, rtol=0, atol=1e-9)
    # M = 1: kernel-weighted mean of the voxels
    _, W1, _ = oracle.lattice_step(A, [Fu, Fv, Fg], sig, W[:1], snap=False)
    wt = np.exp(-(((X - W[0]) ** 2) / (2 * np.array(sig) ** 2)).sum(1))
    np.testing.assert_allclose(W1[0], np.average(X, axis=0, weights=wt), atol=1e-9)
