"""GPU parity of itc_chamfer (the 3-4 chamfer distance transform that weights binary shapes in
Sec. 5, outside of the image = background) vs the oracle's two raster passes: bit-exact on
random images of every register-segment width (1 to 1024 columns), on a ragged C3-style batch,
and the chamfer-weighted clustering P = T(X) * G of Sec. 5 run through a weighted plan against
the oracle run on the same weights."""
import numpy as np
import pytest

import oracle
from gpuhelp import DCS_ATOL, assert_lattice_equal_except_ties, to_dev
from paper_1310_7114_gb300 import build, itc, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    itc.lib()


def _gpu_chamfer(images, align=16):
    import torch
    buf, views = itc.pack_images(images, "cuda", align=align)
    plan = itc.Plan(views, [1] * len(images), itc.make_params(2.0))
    _, T = itc.chamfer(plan)
    torch.cuda.synchronize()
    return [t.cpu().numpy() for t in T]


@pytest.mark.parametrize("shape", [(1, 1), (1, 40), (37, 1), (29, 31), (64, 64), (70, 129), (33, 257), (41, 513),
                                   (17, 1024), (200, 300), (7, 70), (3, 200), (2, 400), (1, 900), (5, 260)])
def test_random_images(shape):
    rng = np.random.default_rng(shape[0] * 7919 + shape[1])
    imgs = [(rng.random(shape) < p).astype(np.uint8) for p in (0.5, 0.9, 1.0)]
    for im, T in zip(imgs, _gpu_chamfer(imgs)):
        assert np.array_equal(T, oracle.chamfer34(im).astype(np.float32)), shape


@pytest.mark.parametrize("shape", [(29, 31), (41, 513), (12, 130)])
def test_rows_without_4_byte_alignment(shape):
    """Byte rows packed back to back (pitch = W): the input comes byte by byte instead of in
    32-bit words; the result is the same."""
    rng = np.random.default_rng(shape[0] * 31 + shape[1])
    imgs = [(rng.random(shape) < p).astype(np.uint8) for p in (0.6, 0.95)]
    for im, T in zip(imgs, _gpu_chamfer(imgs, align=1)):
        assert np.array_equal(T, oracle.chamfer34(im).astype(np.float32)), shape


def test_ragged_batch():
    images, _, _ = synth.c3_batch(24, start=200)
    for b, T in enumerate(_gpu_chamfer(images)):
        assert np.array_equal(T, oracle.chamfer34(images[b]).astype(np.float32)), b


def test_chamfer_weighted_clustering():
    """Sec. 5: the weights T(X) feed the weighted path; the run matches the oracle's weighted
    run on the oracle's T(X) (ties aside, lockstep otherwise)."""
    import torch
    img = synth.c1_image(6)
    buf, views = itc.pack_images([img], "cuda")
    bplan = itc.Plan(views, [8], itc.make_params(2.0))
    out, (Tv,) = itc.chamfer(bplan)
    T_ref = oracle.chamfer34(img).astype(np.float64)
    W0 = synth.init_codebook(synth.rng_for(1, 66), img.astype(np.float32), 8)
    wplan = itc.Plan([Tv], [8], itc.make_params(2.0, 3.0, 30))
    assert wplan.classes()[0]["staging"] == "tma"    # padded rows take the tensor tiles
    W = wplan.pack_W([W0])
    st = itc.new_stats(1, W.device)
    itc.run(wplan, W, st)
    torch.cuda.synchronize()
    Wg = wplan.unpack_W(W)[0]
    A, Fu, Fv = oracle.fields2d(T_ref, 2.0)
    Wo, dcs, tie, t = oracle.lattice_run(A, [Fu, Fv], oracle.sxx(T_ref, A), 2.0, W0, 30)
    if tie.min() > 1e-4:
        assert np.array_equal(Wg, Wo)
        assert abs(itc.stats_to_numpy(st)[0]["dcs"] - dcs[-1]) <= DCS_ATOL
    else:
        Wc = np.asarray(W0, np.float64)
        Fg, sg = itc.fields(Tv, 2.0)
        for _ in range(30):
            Wn, raw, _ = oracle.lattice_step(A, [Fu, Fv], 2.0, Wc)
            Wq, _, _ = itc.step(Tv, Fg, sg, to_dev(Wc.astype(np.float32)), 2.0)
            torch.cuda.synchronize()
            assert_lattice_equal_except_ties(Wq.cpu().numpy(), Wn, raw, what="chamfer lockstep")
            Wc = Wn
