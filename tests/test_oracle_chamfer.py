"""Pins of the oracle's chamfer transform (Sec. 5 weighting; Borgefors' 3-4 chamfer distance to
the nearest background pixel, the outside of the image counted as background), computed by
two raster passes:

* the definition written out by brute force -- the minimum over background pixels and the
  one-pixel frame around the image of the 3-4 chamfer path length 3 max(|du|,|dv|) +
  min(|du|,|dv|) -- on random images of several sizes and densities;
* closed forms: an all-foreground image is 3 times the distance to the nearest edge row or
  column plus one; background pixels are 0; a lone background pixel in a large foreground
  block is at the centre of the chamfer disc 3 max + min.
"""
import numpy as np
import pytest

import oracle


def brute(X):
    H, W = X.shape
    bu, bv = np.nonzero(X == 0)
    fu = np.concatenate([bu, np.full(W + 2, -1), np.full(W + 2, H), np.arange(-1, H + 1), np.arange(-1, H + 1)])
    fv = np.concatenate([bv, np.arange(-1, W + 1), np.arange(-1, W + 1), np.full(H + 2, -1), np.full(H + 2, W)])
    U, V = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    du = np.abs(U[..., None] - fu)
    dv = np.abs(V[..., None] - fv)
    d = 3 * np.maximum(du, dv) + np.minimum(du, dv)
    return np.where(X != 0, d.min(-1), 0)


@pytest.mark.parametrize("shape,p", [((9, 13), 0.7), ((31, 24), 0.9), ((40, 40), 0.5), ((1, 17), 0.8), ((23, 1), 1.0)])
@pytest.mark.parametrize("seed", range(3))
def test_two_pass_equals_definition(shape, p, seed):
    X = (np.random.default_rng(seed).random(shape) < p).astype(np.uint8)
    assert np.array_equal(oracle.chamfer34(X), brute(X))


def test_closed_forms():
    H, W = 11, 16
    T = oracle.chamfer34(np.ones((H, W)))
    U, V = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    assert np.array_equal(T, 3 * np.minimum.reduce([U + 1, H - U, V + 1, W - V]))
    X = np.ones((61, 61), np.uint8)
    X[30, 30] = 0
    T = oracle.chamfer34(X)
    du, dv = np.abs(U := np.arange(61)[:, None] - 30), np.abs(np.arange(61)[None, :] - 30)
    disc = 3 * np.maximum(du, dv) + np.minimum(du, dv)
    inner = slice(20, 41)
    assert np.array_equal(T[inner, inner], disc[inner, inner])
    assert np.array_equal(oracle.chamfer34(np.zeros((5, 6))), np.zeros((5, 6)))
