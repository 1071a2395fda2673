"""GPU parity of itc_segment (segments of Figs. 3 and 6, nearest codebook site by the
single-precision kernel metric, lowest index on ties) vs the oracle: bit-exact labels on C1
images after a run, a ragged C3-style batch, weighted images, per-axis widths, a gray image's
3-D lattice, the build's largest codebook and one codebook.  Every case is also checked against
the nearest site in exact arithmetic (up to ties within the single-precision rounding), which
does not rest on the oracle's own single-precision evaluation."""
import numpy as np
import pytest

import oracle
from gpuhelp import assert_nearest_sites, to_dev
from paper_1310_7114_gb300 import build, itc, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    itc.lib()


def _labels(images, Ms, W0s, params, iters=True, **kw):
    import torch
    plan = itc.Plan([to_dev(im) for im in images], Ms, params, **kw)
    W = plan.pack_W(W0s)
    if iters:
        itc.run(plan, W, itc.new_stats(len(images), W.device))
    lab = itc.segment(plan, W)
    torch.cuda.synchronize()
    return plan.unpack_W(W), [x.astype(np.int32) for x in plan.unpack_pixels(lab)]


def _exact(h, lab, W, tau):
    """Data pixels against the exact nearest site; pixels without data carry -1."""
    assert np.all(lab[h == 0] == -1)
    u, v = np.nonzero(h)
    assert_nearest_sites(np.stack([u, v], 1), lab[u, v], W, h.shape, tau)


def test_c1_after_a_run():
    imgs = [synth.c1_image(s) for s in range(4)]
    W0s = [synth.init_codebook(synth.rng_for(1, 300 + s), im.astype(np.float32), 8) for s, im in enumerate(imgs)]
    Ws, labs = _labels(imgs, [8] * 4, W0s, itc.make_params(2.0, 3.0, 20))
    for im, W, lab in zip(imgs, Ws, labs):
        assert np.array_equal(lab, oracle.segment2d(im, 2.0, W))
        _exact(im, lab, W, 2.0)


def test_ragged_batch_mixed_sigma():
    images, Ms, sig = synth.c3_batch(24, start=100)
    W0s = [synth.init_codebook(synth.rng_for(3, 20_000 + i), im.astype(np.float32), int(m))
           for i, (im, m) in enumerate(zip(images, Ms))]
    params = [itc.make_params(float(s), 3.0, 10) for s in sig]
    Ws, labs = _labels(images, Ms, W0s, params)
    for b in range(len(images)):
        assert np.array_equal(labs[b], oracle.segment2d(images[b], float(sig[b]), Ws[b])), b
        _exact(images[b], labs[b], Ws[b], float(sig[b]))


def test_weighted_and_anisotropic():
    h = synth.c4_weights(7)[:150, :170].copy()
    h[h < 0.3] = 0.0
    W0 = synth.init_codebook(synth.rng_for(4, 77), h, 20, 0.5)
    for sigma in (3.0, (2.0, 3.5)):
        Ws, labs = _labels([h], [20], [W0], itc.make_params(sigma, 3.0, 5))
        assert np.array_equal(labs[0], oracle.segment2d(h, sigma, Ws[0])), sigma
        _exact(h, labs[0], Ws[0], sigma)


def test_gray_lattice():
    gray = (synth.c5_gray(2, size=48).astype(np.int64) * 60 // 256).astype(np.uint8)
    W0 = synth.init_codebook_gray(synth.rng_for(5, 9), gray, 10)
    Ws, labs = _labels([gray], [10], [W0], itc.make_params((2.0, 2.0, 3.0), 3.0, 5), ndims=[3], Gs=[60])
    assert np.array_equal(labs[0], oracle.segment3d(gray, (2.0, 2.0, 3.0), Ws[0], 60))
    u, v = np.nonzero(np.ones_like(gray))
    assert_nearest_sites(np.stack([u, v, gray[u, v]], 1), labs[0][u, v], Ws[0], (*gray.shape, 60), (2.0, 2.0, 3.0),
                         "3-D")


@pytest.mark.parametrize("M", [1, 2048])
def test_codebook_extremes(M):
    rng = np.random.default_rng(M)
    img = (rng.random((160, 150)) < 0.35).astype(np.uint8)
    W0 = synth.init_codebook(synth.rng_for(9, M), img.astype(np.float32), M)
    Ws, labs = _labels([img], [M], [W0], itc.make_params(2.0, 3.0, 0), iters=False)
    ref = oracle.segment2d(img, 2.0, Ws[0])
    assert np.array_equal(labs[0], ref)
    assert np.all(labs[0][img == 0] == -1)
    _exact(img, labs[0], Ws[0], 2.0)
