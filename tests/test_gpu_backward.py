"""GPU parity of the hand-written adjoint of Eq. (1): itc_backward's dD/dW and dD/dh (weighted
ITC, Sec. 5) vs the oracle's analytic gradient, and vs FP64 central differences (h = 1e-4) on 64
random entries of W and of h of a full-size 512x512 weight image.  Bars: normwise relative error
<= 1e-4 (FP32 sums of ~1e-6 relative error, with the cancellation between the two terms of
dD/dh bounded by their magnitudes), and for dD/dh also element-wise, every pixel within 3e-5 of
the magnitudes of its two terms (gpuhelp.assert_grad_h_close)."""
import numpy as np
import pytest

import oracle
from gpuhelp import assert_grad_h_close, to_dev
from paper_1310_7114_gb300 import build, itc, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    itc.lib()


def gpu_forward_backward(images, Ms, W0s, sigma, grad_dcs=None):
    import torch
    ts = [to_dev(im) for im in images]
    plan = itc.Plan(ts, Ms, itc.make_params(sigma, 3.0, 0))
    W = plan.pack_W(W0s)
    st = itc.new_stats(len(images), W.device)
    itc.run(plan, W, st)   # forward: fields, S_XX and D_cs at W (no iterations)
    gW = torch.empty_like(W)
    gh = torch.empty(plan.pixels, dtype=torch.float32, device=W.device)
    gd = None if grad_dcs is None else torch.tensor(grad_dcs, dtype=torch.float32, device=W.device)
    st2 = itc.new_stats(len(images), W.device)
    itc.backward(plan, W, grad_dcs=gd, grad_W=gW, grad_h=gh, stats=st2)
    torch.cuda.synchronize()
    return plan, plan.unpack_W(gW), plan.unpack_pixels(gh), itc.stats_to_numpy(st), itc.stats_to_numpy(st2)


def _nrel(a, b):
    return np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300)


def test_backward_matches_oracle_gradient_weighted_and_binary():
    images = [synth.c4_weights(i)[:128, :160] for i in range(3)] + [synth.c1_image(0).astype(np.float32)]
    Ms = [32, 32, 16, 8]
    W0s = [synth.init_codebook(synth.rng_for(4, 100 + i), im, m, 0.5 if i < 3 else 0.0)
           for i, (im, m) in enumerate(zip(images, Ms))]
    plan, gW, gh, st, st2 = gpu_forward_backward(images, Ms, W0s, 3.0, grad_dcs=[1.0, 2.5, -0.5, 1.0])
    for b, (im, W0) in enumerate(zip(images, W0s)):
        gref, ghref, sums = oracle.dcs_grad2d_dense(im.astype(np.float64), 3.0, W0.astype(np.float64))
        scale = [1.0, 2.5, -0.5, 1.0][b]
        assert _nrel(gW[b], scale * gref) <= 1e-4, (b, _nrel(gW[b], scale * gref))
        assert _nrel(gh[b], scale * ghref) <= 1e-4, (b, _nrel(gh[b], scale * ghref))
        A = oracle.fields2d(im.astype(np.float64), 3.0)[0]
        assert_grad_h_close(gh[b], im, A, sums, scale * ghref, gD=scale, what=f"image {b}")
        d_ref = np.log(sums[1]) + np.log(sums[2]) - 2 * np.log(sums[0])
        assert abs(st[b]["dcs"] - d_ref) <= 4e-5 and abs(st2[b]["dcs"] - d_ref) <= 4e-5


def test_backward_uint8_binary_image():
    img = synth.c1_image(2)
    W0 = synth.init_codebook(synth.rng_for(1, 2), img.astype(np.float32), 8)
    _, gW, gh, _, _ = gpu_forward_backward([img], [8], [W0], 2.0)
    gref, ghref, sums = oracle.dcs_grad2d_dense(img.astype(np.float64), 2.0, W0.astype(np.float64))
    assert _nrel(gW[0], gref) <= 1e-4 and _nrel(gh[0], ghref) <= 1e-4
    assert_grad_h_close(gh[0], img, oracle.fields2d(img.astype(np.float64), 2.0)[0], sums, ghref, what="binary")


def test_backward_at_real_valued_codebook():
    """The window is tied to round(w_k) and the kernel is evaluated at the real w_k."""
    img = synth.c4_weights(1)[:100, :100]
    rng = np.random.default_rng(9)
    W0 = (synth.init_codebook(synth.rng_for(4, 7), img, 12, 0.5) + rng.uniform(-0.45, 0.45, (12, 2))).astype(np.float32)
    _, gW, gh, _, _ = gpu_forward_backward([img], [12], [W0], 3.0)
    gref, ghref, sums = oracle.dcs_grad2d_dense(img.astype(np.float64), 3.0, W0.astype(np.float64))
    assert _nrel(gW[0], gref) <= 1e-4 and _nrel(gh[0], ghref) <= 1e-4
    assert_grad_h_close(gh[0], img, oracle.fields2d(img.astype(np.float64), 3.0)[0], sums, ghref, what="real W")


def test_backward_full_size_c4_against_central_differences():
    """C4 at full size: 512x512 weights, M = 32, sigma = 3; FP64 central differences (step 1e-4)
    of the oracle's Eq. (1) on 64 random entries of W and 64 of h."""
    h = synth.c4_weights(0).astype(np.float64)
    W0 = synth.init_codebook(synth.rng_for(4, 0), h.astype(np.float32), 32, 0.5).astype(np.float64)
    _, gW, gh, _, _ = gpu_forward_backward([h.astype(np.float32)], [32], [W0.astype(np.float32)], 3.0)
    rng = np.random.default_rng(11)
    eps = 1e-4
    A = oracle.fields2d(h, 3.0)[0]
    # every pixel of the full image against the oracle's analytic gradient, element-wise
    _, ghref, sums = oracle.dcs_grad2d_dense(h, 3.0, W0, A=A)
    assert_grad_h_close(gh[0], h, A, sums, ghref, what="C4 full size")
    kw = rng.choice(64, 64, replace=True)
    fd_w, an_w = [], []
    for q in kw:
        k, i = divmod(int(q), 2)
        Wp, Wm = W0.copy(), W0.copy()
        Wp[k, i] += eps
        Wm[k, i] -= eps
        fd_w.append((oracle.dcs2d_dense(h, 3.0, Wp, A=A) - oracle.dcs2d_dense(h, 3.0, Wm, A=A)) / (2 * eps))
        an_w.append(gW[0][k, i])
    assert _nrel(an_w, np.array(fd_w)) <= 1e-4
    pix = rng.choice(h.size, 64, replace=False)
    fd_h, an_h = [], []
    for p in pix:
        hp, hm = h.copy(), h.copy()
        hp.flat[p] += eps
        hm.flat[p] -= eps
        fd_h.append((oracle.dcs2d_dense(hp, 3.0, W0) - oracle.dcs2d_dense(hm, 3.0, W0)) / (2 * eps))
        an_h.append(gh[0].flat[p])
    assert _nrel(an_h, np.array(fd_h)) <= 1e-4


def test_autograd_function_matches_direct_calls():
    import torch
    from paper_1310_7114_gb300.autograd import ITCDivergence
    images = [synth.c4_weights(i)[:96, :96] for i in range(2)]
    W0s = [synth.init_codebook(synth.rng_for(4, 50 + i), im, 10, 0.5) for i, im in enumerate(images)]
    hs = [to_dev(im).requires_grad_(True) for im in images]
    Wt = [to_dev(w).requires_grad_(True) for w in W0s]
    d = ITCDivergence.apply(3.0, 3.0, *hs, *Wt)
    (d * torch.tensor([1.0, -2.0], device=d.device)).sum().backward()
    for b in range(2):
        gref, ghref, sums = oracle.dcs_grad2d_dense(images[b].astype(np.float64), 3.0, W0s[b].astype(np.float64))
        s = [1.0, -2.0][b]
        assert _nrel(Wt[b].grad.cpu().numpy(), s * gref) <= 1e-4
        assert _nrel(hs[b].grad.cpu().numpy(), s * ghref) <= 1e-4
        assert abs(d[b].item() - (np.log(sums[1]) + np.log(sums[2]) - 2 * np.log(sums[0]))) <= 4e-5


def test_backward_rows_not_16_byte_aligned():
    """dD/dh rows that do not start on 16-byte boundaries (widths and per-image offsets that are
    not multiples of 4 floats) go out through the shared-memory transpose; rows that do go out as
    16-byte pieces.  Both against the oracle, in one plan (the 64 x 64 image comes after an offset
    of 101*97 + 63*61 + 70*131 pixels, not a multiple of 4, so it takes the transpose too)."""
    images = [synth.c4_weights(5)[:101, :97], synth.c1_image(3).astype(np.float32)[:63, :61],
              synth.c4_weights(6)[:70, :131], synth.c1_image(4).astype(np.float32),
              synth.c4_weights(7)[:64, :128]]
    Ms = [16, 8, 20, 8, 12]
    assert (101 * 97 + 63 * 61 + 70 * 131) % 4 != 0
    W0s = [synth.init_codebook(synth.rng_for(4, 70 + i), im, m, 0.5) for i, (im, m) in enumerate(zip(images, Ms))]
    plan, gW, gh, _, _ = gpu_forward_backward(images, Ms, W0s, 3.0)
    for b in range(len(images)):
        gref, ghref, sums = oracle.dcs_grad2d_dense(images[b].astype(np.float64), 3.0, W0s[b].astype(np.float64))
        assert _nrel(gW[b], gref) <= 1e-4, (b, _nrel(gW[b], gref))
        assert _nrel(gh[b], ghref) <= 1e-4, (b, _nrel(gh[b], ghref))
        assert_grad_h_close(gh[b], images[b], oracle.fields2d(images[b].astype(np.float64), 3.0)[0], sums, ghref,
                            what=f"image {b}")
