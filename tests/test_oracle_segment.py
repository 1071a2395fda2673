"""Pins of the oracle's segmentation (the reading of Figs. 3 and 6: each data pixel goes to the
codebook vector of largest kernel value at it, i.e. smallest sum_i d_i^2 / tau_i^2 to its lattice
site, evaluated in single precision, lowest index on ties).

* Voronoi property in exact arithmetic: a pixel's codebook is at most a few single-precision
  roundings farther (relative) than the nearest one, for isotropic and per-axis widths, 2-D and
  3-D;
* closed forms: one codebook labels every data pixel; a pixel at a codebook's own site (no other
  codebook there) takes that codebook; separated blobs each seeded by one codebook; pixels
  without data get -1; the lowest index wins among coincident codebooks.
"""
import numpy as np
import pytest

import oracle
from paper_1310_7114_gb300 import synth

U = 2.0 ** -24


def _exact_metric(X, R, tau):
    """Exact (float64 of exact integers / tau^2) metric of every point to every site: N x M."""
    t2 = np.asarray(np.broadcast_to(np.asarray(tau, np.float32), (X.shape[1],)), np.float64) ** 2
    d = X[:, None, :].astype(np.int64) - R[None, :, :].astype(np.int64)
    return ((d * d) / t2).sum(-1)


def _sites(W, shape):
    return np.clip(np.floor(np.asarray(W, np.float64) + 0.5), 0, np.asarray(shape) - 1).astype(np.int64)


def _check_voronoi(X, lab, R, tau):
    D = _exact_metric(X, R, tau)
    best = D.min(1)
    got = D[np.arange(len(X)), lab]
    assert np.all(got <= best * (1 + 8 * U)), np.max(got / np.maximum(best, 1e-300))
    # where the nearest site is unique by more than the rounding, the label is that site
    srt = np.sort(D, 1)
    clear = srt[:, 1] > srt[:, 0] * (1 + 8 * U) if D.shape[1] > 1 else np.ones(len(X), bool)
    assert np.all(lab[clear] == D.argmin(1)[clear])


@pytest.mark.parametrize("tau", [2.0, 3.0, (1.5, 2.5)])
@pytest.mark.parametrize("seed", range(3))
def test_voronoi_property_2d(seed, tau):
    img = synth.c1_image(seed)
    M = 12
    W = synth.init_codebook(synth.rng_for(1, 50 + seed), img.astype(np.float32), M).astype(np.float64)
    W += np.random.default_rng(seed).uniform(-0.45, 0.45, W.shape)   # real W: sites by rounding
    lab = oracle.segment2d(img, tau, W)
    u, v = np.nonzero(img)
    assert np.all(lab[img == 0] == -1)
    _check_voronoi(np.stack([u, v], 1), lab[u, v], _sites(W, img.shape), tau)


def test_voronoi_property_3d():
    gray = synth.c5_gray(1, size=40)
    hw = (np.random.default_rng(3).random(gray.shape) < 0.8).astype(np.float64)
    W = np.stack([np.random.default_rng(4).integers(0, 40, 9), np.random.default_rng(5).integers(0, 40, 9),
                  np.random.default_rng(6).integers(0, 256, 9)], 1).astype(np.float64)
    tau = (2.0, 2.0, 6.0)
    lab = oracle.segment3d(gray, tau, W, 256, hw)
    u, v = np.nonzero(hw)
    assert np.all(lab[hw == 0] == -1)
    _check_voronoi(np.stack([u, v, gray[u, v]], 1), lab[u, v], _sites(W, (40, 40, 256)), tau)


def test_closed_forms():
    img = np.zeros((40, 50), np.uint8)
    img[5:12, 4:15] = 1       # blob A
    img[25:35, 30:45] = 1     # blob B
    img[30, 5] = 1            # a lone pixel, nearest to A's codebook
    W = np.array([[8.0, 9.0], [30.0, 37.0]])
    lab = oracle.segment2d(img, 2.0, W)
    assert np.all(lab[5:12, 4:15] == 0) and np.all(lab[25:35, 30:45] == 1) and lab[30, 5] == 0
    assert np.all(lab[img == 0] == -1)
    # one codebook: every data pixel
    assert np.all(oracle.segment2d(img, 2.0, W[:1])[img != 0] == 0)
    # a pixel at a codebook's own site takes it; coincident codebooks: the lowest index
    W3 = np.array([[30.0, 37.0], [8.0, 9.0], [8.0, 9.0]])
    lab3 = oracle.segment2d(img, 3.0, W3)
    assert lab3[30, 37] == 0 and lab3[8, 9] == 1 and not np.any(lab3 == 2)
