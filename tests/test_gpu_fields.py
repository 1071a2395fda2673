"""GPU parity of the lattice fields (Sec. 3.1, Sec. 5): itc_fields vs the FP64 oracle,
element by element, over tile-spanning sizes with ragged tails, every compiled radius and the
runtime-radius path, binary and weighted inputs, centred and absolute moments, and the edge
cases (1x1, single rows/columns, images smaller than the mask, empty and full images)."""
import numpy as np
import pytest

import oracle
from gpuhelp import assert_fields_close, radii, to_dev
from paper_1310_7114_gb300 import build, itc, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    itc.lib()


def gpu_fields(h, sigma, trunc=3.0, absolute=False, pad=0):
    import torch
    if pad:
        buf, views = itc.pack_images([h], "cuda", align=pad)
        t = views[0]
    else:
        t = to_dev(h)
    F, sxx = itc.fields(t, sigma, trunc, absolute)
    torch.cuda.synchronize()
    W = h.shape[1]
    return [F[i, 0, :, :W].cpu().numpy().astype(np.float64) for i in range(3)], float(sxx.item())


def check(h, sigma, trunc=3.0, absolute=False, pad=0, what=""):
    g, sxx = gpu_fields(h, sigma, trunc, absolute, pad)
    ref = oracle.fields2d(h.astype(np.float64), sigma, trunc, absolute)
    assert_fields_close(g, ref, radii(sigma, trunc), absolute, what)
    ref_sxx = oracle.sxx(h.astype(np.float64), ref[0]) if not absolute else None
    if ref_sxx is not None:
        assert abs(sxx - ref_sxx) <= 1e-5 * ref_sxx + 1e-30, (sxx, ref_sxx)
    return g, ref


def _binary(rng, H, W, p):
    return (rng.random((H, W)) < p).astype(np.uint8)


CASES = {
    "c1_sigma2": lambda: (synth.c1_image(0), 2.0),
    "binary_150x97_sigma3": lambda: (_binary(np.random.default_rng(1), 150, 97, 0.2), 3.0),
    "binary_130x300_sigma4": lambda: (_binary(np.random.default_rng(2), 130, 300, 0.15), 4.0),
    "weights_96x200_sigma3": lambda: (synth.c4_weights(0)[:96, :200], 3.0),
    "anisotropic_runtime_radius": lambda: (_binary(np.random.default_rng(3), 80, 90, 0.3), (1.5, 2.5)),
    "sigma1_runtime_radius": lambda: (_binary(np.random.default_rng(4), 70, 140, 0.3), 1.0),
    "sigma_10_wide_runtime": lambda: (_binary(np.random.default_rng(5), 90, 100, 0.05), 10.0),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_fields_centred(name):
    h, s = CASES[name]()
    check(h, s, what=name)


@pytest.mark.parametrize("name", ["c1_sigma2", "weights_96x200_sigma3", "binary_130x300_sigma4", "anisotropic_runtime_radius"])
def test_fields_absolute(name):
    h, s = CASES[name]()
    check(h, s, absolute=True, what=name)


def test_fields_with_row_pitch():
    h = _binary(np.random.default_rng(6), 70, 77, 0.25)
    check(h, 2.0, pad=32, what="pitched rows")


@pytest.mark.parametrize("shape", [(1, 1), (1, 70), (70, 1), (5, 5), (13, 200), (200, 13), (65, 65), (64, 128)])
def test_edge_shapes(shape):
    rng = np.random.default_rng(sum(shape))
    h = _binary(rng, *shape, 0.4)
    h.flat[0] = 1
    check(h, 3.0, what=str(shape))


def test_empty_image_is_exactly_zero():
    h = np.zeros((100, 130), np.uint8)
    g, sxx = gpu_fields(h, 3.0)
    assert all(np.all(x == 0) for x in g) and sxx == 0.0


def test_full_image():
    check(np.ones((77, 66), np.uint8), 4.0, what="all ones")


def test_c2_full_size_sampled_sites():
    """C2 at full size (1024^2, sigma 4): 4000 random sites plus two whole 64x64 windows."""
    img = synth.c2_image(0)
    g, sxx = gpu_fields(img, 4.0)
    rng = np.random.default_rng(0)
    sites = np.stack([rng.integers(0, 1024, 4000), rng.integers(0, 1024, 4000)], 1)
    win = np.stack(np.meshgrid(np.arange(500, 564), np.arange(960, 1024), indexing="ij"), -1).reshape(-1, 2)
    win2 = np.stack(np.meshgrid(np.arange(0, 64), np.arange(0, 64), indexing="ij"), -1).reshape(-1, 2)
    sites = np.concatenate([sites, win, win2])
    ref = oracle.fields2d_sites(img.astype(np.float64), 4.0, sites)
    gs = [x[sites[:, 0], sites[:, 1]] for x in g]
    assert_fields_close(gs, ref, [12, 12], False, "C2 sites")
    A_ref = oracle.fields2d(img.astype(np.float64), 4.0)[0]
    ref_sxx = oracle.sxx(img.astype(np.float64), A_ref)
    assert abs(sxx - ref_sxx) <= 1e-5 * ref_sxx


def test_fields_are_deterministic():
    h = synth.c2_image(0, size=512)
    a, s1 = gpu_fields(h, 3.0)
    b, s2 = gpu_fields(h, 3.0)
    assert s1 == s2 and all(np.array_equal(x, y) for x, y in zip(a, b))


@pytest.mark.parametrize("sigma", [2.0, 3.0, 4.0])
@pytest.mark.parametrize("dtype", ["u8", "f32"])
@pytest.mark.parametrize("absolute", [False, True])
@pytest.mark.parametrize("pattern", ["sparse", "solid", "levels"])
def test_tma_tiles_equal_plain_tiles_bit_for_bit(sigma, dtype, absolute, pattern):
    """Rows on 16-byte boundaries take the TMA-staged tiles; an odd row pitch takes the plain
    staging.  Both accumulate the same products in the same order, so they agree exactly.
    "solid" adds a disc and a band of ones touching the border: long runs of all-ones windows,
    tiles with no zero row, and ones against the image edges; its row windows are mostly single
    runs of 0/1 inputs, which the TMA tiles take from their run table at R >= 9 (entries made by
    the same FMA chains).  "levels" puts inputs 2 and 255 into runs of the solid shapes: windows
    that are runs of nonzero inputs but not of ones, which must take the FMAs."""
    import torch
    rng = np.random.default_rng(int(sigma * 10) + (dtype == "f32"))
    h = (rng.random((197, 203)) < 0.2)
    if dtype == "f32":
        h = (h * rng.random((197, 203))).astype(np.float32)
    if pattern == "solid":
        uu, vv = np.mgrid[0:197, 0:203]
        one = ((uu - 90) ** 2 + (vv - 110) ** 2 < 70 ** 2) | (vv >= 180) | (uu < 20)
        h = np.where(one, 1, h)
    if pattern == "levels":
        uu, vv = np.mgrid[0:197, 0:203]
        one = ((uu - 90) ** 2 + (vv - 110) ** 2 < 70 ** 2) | (vv >= 180)
        h = np.where(one, 1, h).astype(np.float32)
        h[100:104, 60:150] = 2          # a band of 2 inside the disc
        h[30:150:7, 185:200] = 255      # rows of 255 inside the right band
    h = h.astype(np.uint8) if dtype == "u8" else h.astype(np.float32)
    buf_a, (ta,) = itc.pack_images([h], "cuda", align=16)      # pitch multiple of 16 elements
    buf_b, (tb,) = itc.pack_images([h], "cuda", align=1)       # pitch 203: no tensor map
    Fa, sa = itc.fields(ta, sigma, 3.0, absolute)
    Fb, sb = itc.fields(tb, sigma, 3.0, absolute)
    torch.cuda.synchronize()
    assert torch.equal(Fa[..., :203], Fb[..., :203])
    assert sa.item() == sb.item()
    ref = oracle.fields2d(h.astype(np.float64), sigma, 3.0, absolute)
    assert_fields_close([Fa[i, 0, :, :203].cpu().numpy().astype(np.float64) for i in range(3)], ref,
                        radii(sigma), absolute, "tma")


def test_bounded_tile_wait_reports_instead_of_hanging():
    """The TMA tile wait is bounded: with the test hook one CTA waits for a copy phase that never
    completes and gives up after about a second.  The call reports ITC_ERR_TIMEOUT in the status
    word at the start of its workspace, with sxx given (S_XX = NaN) and with sxx NULL; a call
    without the hook reports ITC_OK there; the GPU context stays usable and the next call is
    correct."""
    import ctypes
    import torch
    h = (np.random.default_rng(0).random((256, 256)) < 0.3).astype(np.uint8)
    buf, (t,) = itc.pack_images([h], "cuda", align=16)   # aligned rows: the TMA path
    img = itc.make_image(t)
    out = torch.empty(itc.lib().itc_fields_bytes(ctypes.byref(img)) // 4, device="cuda")
    ws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    assert itc.lib().itc_fields_workspace_bytes(ctypes.byref(img)) <= ws.numel()
    stream = torch.cuda.current_stream().cuda_stream
    for with_sxx in (True, False):
        ws.fill_(0x5A)
        sxx = torch.zeros(1, dtype=torch.float64, device="cuda")
        p = itc.make_params(2.0, 3.0, flags=itc.ITC_TEST_STALL_WAIT)
        rc = itc.itc_fields(img, p, out.data_ptr(), sxx.data_ptr() if with_sxx else None, ws.data_ptr(),
                            ws.numel(), stream)
        assert rc == itc.ITC_OK
        torch.cuda.synchronize()
        assert int(ws[:4].view(torch.int32).item()) == itc.ITC_ERR_TIMEOUT, with_sxx
        if with_sxx:
            assert np.isnan(sxx.item())
        else:
            assert sxx.item() == 0.0   # untouched
        rc = itc.itc_fields(img, itc.make_params(2.0), out.data_ptr(), None, ws.data_ptr(), ws.numel(), stream)
        assert rc == itc.ITC_OK
        torch.cuda.synchronize()
        assert int(ws[:4].view(torch.int32).item()) == itc.ITC_OK
    check(h, 2.0, what="after a stalled call")


def test_bounded_tile_wait_in_a_plan_sets_the_image_status():
    """The same hook in a batch plan: the images whose tiles the stalled CTA owned report
    ITC_ERR_TIMEOUT in itc_stats (from itc_run and from itc_backward), every other image of the
    plan runs as in a plan without the hook, and the next run of the same plan is clean."""
    import torch
    images, Ms, sig = synth.c3_batch(12, start=300)
    W0s = [synth.init_codebook(synth.rng_for(3, 90_000 + i), im.astype(np.float32), int(m))
           for i, (im, m) in enumerate(zip(images, Ms))]
    buf, views = itc.pack_images(images, "cuda")
    outs = []
    for stall in (True, False):
        params = [itc.make_params(float(s), 3.0, 5, flags=itc.ITC_TEST_STALL_WAIT if stall else 0) for s in sig]
        plan = itc.Plan(views, [int(m) for m in Ms], params)
        assert any(c["staging"] == "tma" for c in plan.classes())
        W = plan.pack_W(W0s)
        st = itc.new_stats(len(images), W.device)
        itc.run(plan, W, st)
        gW = torch.empty_like(W)
        st2 = itc.new_stats(len(images), W.device)
        itc.backward(plan, W, grad_W=gW, stats=st2)
        torch.cuda.synchronize()
        outs.append((plan.unpack_W(W), itc.stats_to_numpy(st), itc.stats_to_numpy(st2)))
    (Ws, s1, b1), (Wc, s0, b0) = outs
    timed_out = [b for b in range(len(images)) if s1[b]["status"] == itc.ITC_ERR_TIMEOUT]
    assert timed_out, "no image reported the timeout"
    assert len(timed_out) < len(images)
    for b in range(len(images)):
        if b in timed_out:
            assert np.isnan(s1[b]["sxx"]) and b1[b]["status"] == itc.ITC_ERR_TIMEOUT
        else:
            assert s1[b]["status"] == s0[b]["status"] != itc.ITC_ERR_TIMEOUT
            assert np.array_equal(Ws[b], Wc[b]) and s1[b]["dcs"] == s0[b]["dcs"]
            assert b1[b]["status"] != itc.ITC_ERR_TIMEOUT
    assert all(s0[b]["status"] != itc.ITC_ERR_TIMEOUT for b in range(len(images)))
    check(synth.c1_image(5), 2.0, what="after a stalled plan")
