"""GPU parity of the fixed-point iteration (Algorithm 1 with Eq. (origupdate)): itc_step and the
batched itc_run vs the FP64 oracle.

Bar: one step from identical W gives identical lattice positions except coordinates whose
oracle value lies within 1e-4 of a half-integer; final codebooks are identical when the
oracle's trajectory has no such tie, otherwise every iteration is checked in lockstep (the GPU
step from the oracle's W).  D_cs and the sums agree to the derived FP32 bound."""
import numpy as np
import pytest

import oracle
import gpuhelp
from gpuhelp import DCS_ATOL, assert_lattice_equal_except_ties, to_dev
from paper_1310_7114_gb300 import build, itc, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    itc.lib()


def _oracle_fields(h, sigma):
    A, Fu, Fv = oracle.fields2d(h.astype(np.float64), sigma)
    return A, [Fu, Fv], oracle.sxx(h.astype(np.float64), A)


def gpu_step(h, sigma, W, step_scale=1.0, flags=0, F=None):
    import torch
    t = to_dev(h)
    if F is None:
        F = itc.fields(t, sigma)
    Wo, Wl, st = itc.step(t, F[0], F[1], to_dev(np.asarray(W, np.float32)), sigma, 3.0, step_scale, flags)
    torch.cuda.synchronize()
    return Wo.cpu().numpy(), Wl.cpu().numpy(), itc.stats_to_numpy(st)[0], F


def run_plan(images, Ms, W0s, params, ndims=None, Gs=None, weights=None):
    import torch
    ts = [to_dev(im) for im in images]
    plan = itc.Plan(ts, Ms, params, ndims=ndims, Gs=Gs, weights=weights)
    W = plan.pack_W(W0s)
    st = itc.new_stats(len(images), W.device)
    itc.run(plan, W, st)
    torch.cuda.synchronize()
    return plan, plan.unpack_W(W), itc.stats_to_numpy(st)


@pytest.mark.parametrize("seed", range(4))
def test_single_step_c1(seed):
    img = synth.c1_image(seed)
    W0 = synth.init_codebook(synth.rng_for(1, seed), img.astype(np.float32), 8)
    A, F, sxx = _oracle_fields(img, 2.0)
    Wn, raw, st = oracle.lattice_step(A, F, 2.0, W0)
    Wg, Wl, s, _ = gpu_step(img, 2.0, W0)
    assert_lattice_equal_except_ties(Wg, Wn, raw, what=f"seed {seed}")
    assert np.array_equal(Wl, Wg.astype(np.int32))
    assert abs(s["sxw"] - st["sxw"]) <= 1e-5 * st["sxw"]
    assert abs(s["sww"] - st["sww"]) <= 1e-5 * st["sww"]
    d_ref = np.log(st["sww"]) + np.log(sxx) - 2 * np.log(st["sxw"])
    assert abs(s["dcs"] - d_ref) <= DCS_ATOL
    assert s["moved"] == st["moved"]


def test_single_step_continuous_and_half_step():
    img = synth.c1_image(1)
    rng = synth.rng_for(1, 1)
    W0 = synth.init_codebook(rng, img.astype(np.float32), 8) + rng.uniform(-0.4, 0.4, (8, 2)).astype(np.float32)
    W0 = W0.astype(np.float32)
    A, F, _ = _oracle_fields(img, 2.0)
    for scale in (1.0, 0.5):
        _, raw, _ = oracle.lattice_step(A, F, 2.0, W0.astype(np.float64), step_scale=scale, snap=False)
        Wg, _, _, _ = gpu_step(img, 2.0, W0, step_scale=scale, flags=itc.ITC_CONTINUOUS)
        ref = np.clip(raw, 0, 63)
        # FP32 fields and sums: a step of (D - cE)/a carries ~1e-5 relative error of the moment
        # window (|D| <= R a), so positions agree to 1e-5 R = 6e-5 px; stored as float32.
        np.testing.assert_allclose(Wg, ref, rtol=0, atol=1e-4)


def test_step_with_absolute_fields_matches():
    import torch
    img = synth.c1_image(2)
    W0 = synth.init_codebook(synth.rng_for(1, 2), img.astype(np.float32), 8)
    A, F, _ = _oracle_fields(img, 2.0)
    Wn, raw, _ = oracle.lattice_step(A, F, 2.0, W0)
    t = to_dev(img)
    Fa = itc.fields(t, 2.0, absolute=True)
    Wo, _, _ = itc.step(t, Fa[0], Fa[1], to_dev(W0), 2.0, flags=itc.ITC_FIELDS_ABSOLUTE)
    torch.cuda.synchronize()
    assert_lattice_equal_except_ties(Wo.cpu().numpy(), Wn, raw, what="absolute")


def plan_lockstep(images, Ms, sigmas, W0s, iters, what="plan lockstep"):
    """The batched plan in lockstep with the oracle (see gpuhelp.plan_lockstep)."""
    ref = [_oracle_fields(im, float(s)) for im, s in zip(images, sigmas)]

    def ostep(b, W):
        Wn, raw, _ = oracle.lattice_step(ref[b][0], ref[b][1], float(sigmas[b]), W)
        return Wn, raw

    return gpuhelp.plan_lockstep(images, Ms, [itc.make_params(float(s), 3.0, 1) for s in sigmas], W0s, iters,
                                 ostep, what=what)


def _check_run(img, sigma, M, iters, W0, plan_W, stats, what, batch=None):
    """Final codebooks equal the oracle's when its trajectory has no rounding tie; otherwise the
    batched plan is run in lockstep with the oracle (``batch`` = (images, Ms, sigmas, W0s) of the
    plan that produced ``plan_W``; the image alone when None)."""
    A, F, sxx = _oracle_fields(img, sigma)
    Wo, dcs, tie, t = oracle.lattice_run(A, F, sxx, sigma, W0, iters)
    if tie.min() > 1e-4:
        assert np.array_equal(plan_W, Wo), f"{what}: final codebooks differ"
        assert abs(stats["dcs"] - dcs[-1]) <= DCS_ATOL, (what, stats["dcs"], dcs[-1])
    else:
        imgs, ms, sg, ws = batch if batch is not None else ([img], [M], [sigma], [W0])
        plan_lockstep(imgs, ms, sg, ws, iters, what=what)
    assert stats["iters_done"] == iters


@pytest.mark.parametrize("seed", range(3))
def test_run_c1_fifty_iterations(seed):
    img = synth.c1_image(seed)
    W0 = synth.init_codebook(synth.rng_for(1, seed), img.astype(np.float32), 8)
    _, Ws, st = run_plan([img], [8], [W0], itc.make_params(2.0, 3.0, 50))
    _check_run(img, 2.0, 8, 50, W0, Ws[0], st[0], f"C1 seed {seed}")


def test_run_c2_full_size():
    img = synth.c2_image(0)
    W0 = synth.init_codebook(synth.rng_for(2, 0), img.astype(np.float32), 64)
    _, Ws, st = run_plan([img], [64], [W0], itc.make_params(4.0, 3.0, 100))
    _check_run(img, 4.0, 64, 100, W0, Ws[0], st[0], "C2")


def test_batched_run_matches_oracle_per_image_and_single_fields():
    """A ragged C3-like batch in one plan: every image's result equals its own oracle run, and the
    batched fields equal the single-image itc_fields bit for bit."""
    import torch
    images, Ms, sig = synth.c3_batch(24)
    W0s = [synth.init_codebook(synth.rng_for(3, 10_000 + i), im.astype(np.float32), int(m))
           for i, (im, m) in enumerate(zip(images, Ms))]
    params = [itc.make_params(float(s), 3.0, 20) for s in sig]
    plan, Ws, st = run_plan(images, Ms, W0s, params)
    tied = []
    for b in range(len(images)):
        A, F, sxx = _oracle_fields(images[b], float(sig[b]))
        Wo, dcs, tie, t = oracle.lattice_run(A, F, sxx, float(sig[b]), W0s[b], 20)
        assert st[b]["iters_done"] == 20
        if tie.min() > 1e-4:
            assert np.array_equal(Ws[b], Wo), f"image {b}: final codebooks differ"
            assert abs(st[b]["dcs"] - dcs[-1]) <= DCS_ATOL
        else:
            tied.append(b)
    if tied:   # the whole batch, through the batched plan, in lockstep with the oracle
        plan_lockstep(images, Ms, sig, W0s, 20)
    for b in (0, 5, 11):
        H, W = images[b].shape
        single, _ = itc.fields(to_dev(images[b]), float(sig[b]))
        torch.cuda.synchronize()
        batched = plan.fields_of(b)
        assert torch.equal(single[..., :W], batched[..., :W])


def test_stop_on_fixed_point():
    img = synth.c1_image(0)
    W0 = synth.init_codebook(synth.rng_for(1, 0), img.astype(np.float32), 8)
    _, Ws, st = run_plan([img], [8], [W0], itc.make_params(2.0, 3.0, 200, flags=itc.ITC_STOP_ON_FIXED))
    A, F, sxx = _oracle_fields(img, 2.0)
    Wo, dcs, tie, t = oracle.lattice_run(A, F, sxx, 2.0, W0, 200, stop_on_fixed=True)
    assert st[0]["iters_done"] == t < 200 and st[0]["moved"] == 0
    assert np.array_equal(Ws[0], Wo)


def test_empty_support_warning_keeps_codebook():
    img = np.zeros((64, 64), np.uint8)
    img[5:12, 5:12] = 1
    W0 = np.array([[8, 8], [60, 60]], np.float32)
    _, Ws, st = run_plan([img], [2], [W0], itc.make_params(2.0, 3.0, 3))
    assert st[0]["status"] == itc.ITC_WARN_EMPTY_SUPPORT and st[0]["empty"] == 1
    assert np.array_equal(Ws[0][1], W0[1])


def test_all_codebooks_without_data_is_nonfinite():
    img = np.zeros((64, 64), np.uint8)
    img[0, 0] = 1
    W0 = np.array([[40, 40], [60, 20]], np.float32)
    _, Ws, st = run_plan([img], [2], [W0], itc.make_params(2.0, 3.0, 2))
    assert st[0]["status"] == itc.ITC_ERR_NONFINITE and np.isinf(st[0]["dcs"])
    assert np.array_equal(Ws[0], W0)


def test_single_codebook_is_mean_shift_on_gpu():
    """M = 1 (no repulsion, Sec. 2.2): the GPU step is a Gaussian mean-shift step."""
    rng = np.random.default_rng(3)
    img = (rng.random((50, 60)) < 0.3).astype(np.uint8)
    w = np.array([[25.0, 30.0]], np.float32)
    Wg, _, _, _ = gpu_step(img, 2.0, w, flags=itc.ITC_CONTINUOUS)
    uu, vv = np.meshgrid(np.arange(19, 32), np.arange(24, 37), indexing="ij")
    wt = img[19:32, 24:37] * np.exp(-((uu - 25.0) ** 2 + (vv - 30.0) ** 2) / 8.0)
    np.testing.assert_allclose(Wg[0], [np.average(uu, weights=wt), np.average(vv, weights=wt)], atol=1e-4)


def test_run_is_deterministic():
    images, Ms, sig = synth.c3_batch(6)
    W0s = [synth.init_codebook(synth.rng_for(3, 20_000 + i), im.astype(np.float32), int(m))
           for i, (im, m) in enumerate(zip(images, Ms))]
    params = [itc.make_params(float(s), 3.0, 10) for s in sig]
    _, W1, s1 = run_plan(images, Ms, W0s, params)
    _, W2, s2 = run_plan(images, Ms, W0s, params)
    assert all(np.array_equal(a, b) for a, b in zip(W1, W2))
    assert s1.tobytes() == s2.tobytes()


def test_pipelined_and_range_runs_equal_plain_run():
    """itc_run_pipelined (fields of chunk k+1 overlapping iterations of chunk k on a second
    stream) and explicit range calls give the same codebooks and stats as itc_run."""
    import ctypes
    import torch
    images, Ms, sig = synth.c3_batch(40)
    W0s = [synth.init_codebook(synth.rng_for(3, 30_000 + i), im.astype(np.float32), int(m))
           for i, (im, m) in enumerate(zip(images, Ms))]
    params = [itc.make_params(float(s), 3.0, 15) for s in sig]
    ts = [to_dev(im) for im in images]
    plan = itc.Plan(ts, Ms, params)
    outs = []
    for mode in ("plain", "pipelined", "ranges"):
        W = plan.pack_W(W0s)
        st = itc.new_stats(len(images), W.device)
        if mode == "plain":
            itc.run(plan, W, st)
        elif mode == "pipelined":
            itc.run_pipelined(plan, W, st, chunks=5)
        else:
            L = itc.lib()
            s = torch.cuda.current_stream().cuda_stream
            for b0, b1 in ((0, 7), (7, 7), (7, 31), (31, 40)):
                assert L.itc_run_fields_range(plan.host_ptr, plan.dev.data_ptr(), b0, b1, plan.ws.data_ptr(),
                                              plan.ws.numel(), s) == 0
                assert L.itc_run_iterate_range(plan.host_ptr, plan.dev.data_ptr(), b0, b1, W.data_ptr(),
                                               st.data_ptr(), plan.ws.data_ptr(), plan.ws.numel(), s) == 0
            assert L.itc_run_fields_range(plan.host_ptr, plan.dev.data_ptr(), 5, 41, plan.ws.data_ptr(),
                                          plan.ws.numel(), s) == itc.ITC_ERR_INVALID_ARG
        torch.cuda.synchronize()
        outs.append((W.cpu().numpy().copy(), st.cpu().numpy().tobytes()))
    for W, st in outs[1:]:
        assert np.array_equal(W, outs[0][0]) and st == outs[0][1]


def test_staged_run_from_host_equals_plain_run():
    """itc_run_staged (image bytes copied range by range on a second stream while earlier ranges
    compute) gives the codebooks and stats of itc_run on device-resident images."""
    import torch
    images, Ms, sig = synth.c3_batch(40, start=700)
    W0s = [synth.init_codebook(synth.rng_for(3, 60_000 + i), im.astype(np.float32), int(m))
           for i, (im, m) in enumerate(zip(images, Ms))]
    params = [itc.make_params(float(s), 3.0, 12) for s in sig]
    buf, views = itc.pack_images(images, "cuda")
    host = buf.cpu().pin_memory()
    plan = itc.Plan(views, Ms, params)
    W = plan.pack_W(W0s)
    st = itc.new_stats(len(images), W.device)
    itc.run(plan, W, st)
    torch.cuda.synchronize()
    ref = (W.cpu().numpy().copy(), st.cpu().numpy().tobytes())
    side = torch.cuda.Stream()
    for chunks in (1, 3, 8):
        buf.zero_()
        W2 = plan.pack_W(W0s)
        st2 = itc.new_stats(len(images), W.device)
        itc.run_staged(plan, host, buf, W2, st2, chunks=chunks, copy_stream=side)
        torch.cuda.synchronize()
        assert np.array_equal(W2.cpu().numpy(), ref[0]) and st2.cpu().numpy().tobytes() == ref[1], chunks


def _fields_and_run(plan, W0s, iters_plan):
    import torch
    itc.run_fields(plan)
    torch.cuda.synchronize()
    F = [plan.fields_of(b).cpu().numpy().copy() for b in range(plan.B)]
    W = plan.pack_W(W0s)
    st = itc.new_stats(plan.B, W.device)
    itc.run(plan, W, st)
    torch.cuda.synchronize()
    return F, W.cpu().numpy().copy(), itc.stats_to_numpy(st)


def _c3_plan(n, iters):
    images, Ms, sig = synth.c3_batch(n)
    W0s = [synth.init_codebook(synth.rng_for(3, 40_000 + i), im.astype(np.float32), int(m))
           for i, (im, m) in enumerate(zip(images, Ms))]
    params = [itc.make_params(float(s), 3.0, iters) for s in sig]
    buf, views = itc.pack_images(images, "cuda")   # rows padded to 16 bytes: tensor tiles possible
    plan = itc.Plan(views, Ms, params)
    plan._keep_buf = buf
    return plan, W0s


def test_every_fields_configuration_gives_the_same_result():
    """Tile height, persistent grid and staging change only the schedule: the fields are
    bit-for-bit identical, so are the codebooks after a run.  S_XX is a sum of per-tile
    partials, each built from FP32 per-thread sums of at most 16 non-negative products h*A, so a
    different tiling moves it by at most 16 FP32 roundings, relative (< 1e-6); D_cs moves by the
    same amount through log S_XX."""
    plan, W0s = _c3_plan(48, 12)
    base = _fields_and_run(plan, W0s, 12)
    configs = [(64, 0, "plain"), (64, 1, "tma"), (32, 0, "tma"), (32, 1, "tma"), (32, 2, "tma"), (128, 0, "tma"),
               (128, 1, "tma"), (64, 0, "tma")]
    classes = plan.classes()
    assert sum(info["staging"] == "tma" for info in classes) >= 2
    for c, info in enumerate(classes):
        if info["staging"] != "tma":
            continue
        for th, g, stg in configs:
            plan.configure(c, th, g, stg)
            got = plan.classes()[c]
            assert (got["tile_h"], got["ctas_per_sm"], got["staging"]) == (th, g, stg)
            F, W, st = _fields_and_run(plan, W0s, 12)
            assert all(np.array_equal(a, b) for a, b in zip(F, base[0])), (c, th, g, stg)
            assert np.array_equal(W, base[1]), (c, th, g, stg)
            assert np.allclose(st["sxx"], base[2]["sxx"], rtol=1e-6, atol=0)
            assert np.allclose(st["dcs"], base[2]["dcs"], rtol=0, atol=1e-6)


def test_autotuned_plan_keeps_results():
    plan, W0s = _c3_plan(64, 10)
    base = _fields_and_run(plan, W0s, 10)
    info = plan.autotune(reps=2)
    assert len(info) >= 2
    for c in info:
        assert c["tuned_ms"] > 0 and c["tile_h"] in (32, 64, 128) and c["staging"] in ("tma", "plain")
    F, W, st = _fields_and_run(plan, W0s, 10)
    assert all(np.array_equal(a, b) for a, b in zip(F, base[0]))
    assert np.array_equal(W, base[1])
    assert np.allclose(st["dcs"], base[2]["dcs"], rtol=0, atol=1e-6)


@pytest.mark.parametrize("M", [700, 2048])
def test_large_codebooks_against_oracle(M):
    """Many codebook vectors per image (up to the build's limit of 2048): each thread owns
    several codebooks; a few iterations must match the oracle (ties aside)."""
    rng = np.random.default_rng(M)
    img = (rng.random((160, 150)) < 0.35).astype(np.uint8)
    W0 = synth.init_codebook(synth.rng_for(9, M), img.astype(np.float32), M)
    _, Ws, st = run_plan([img], [M], [W0], itc.make_params(2.0, 3.0, 3))
    _check_run(img, 2.0, M, 3, W0, Ws[0], st[0], f"M={M}")


def test_mixed_2d_and_3d_plan():
    """One plan holding binary, weighted and gray-lattice images: every image's result equals
    its own single-image plan."""
    gray = (synth.c5_gray(3, size=48).astype(np.int64) * 40 // 256).astype(np.uint8)
    imgs = [synth.c1_image(4), gray, synth.c4_weights(5)[:70, :90]]
    W0s = [synth.init_codebook(synth.rng_for(1, 4), imgs[0].astype(np.float32), 8),
           synth.init_codebook_gray(synth.rng_for(5, 3), gray, 10),
           synth.init_codebook(synth.rng_for(4, 5), imgs[2], 12, 0.5)]
    params = [itc.make_params(2.0, 3.0, 10), itc.make_params((2.0, 2.0, 3.0), 3.0, 10), itc.make_params(3.0, 3.0, 10)]
    plan, Ws, st = run_plan(imgs, [8, 10, 12], W0s, params, ndims=[2, 3, 2], Gs=[1, 40, 1])
    for b in range(3):
        _, Wb, sb = run_plan([imgs[b]], [len(W0s[b])], [W0s[b]], params[b], ndims=[[2, 3, 2][b]], Gs=[[1, 40, 1][b]])
        assert np.array_equal(Ws[b], Wb[0]), b
        assert st[b]["dcs"] == sb[0]["dcs"], b


def test_grouped_images_stop_on_their_own():
    """Images that share an iteration CTA (up to 8 with M <= 16, 4 with M <= 32, 2 with M <= 64)
    run in lockstep, but each stops on its own test: mixed iteration counts, Algorithm 1's
    fixed-point stop on some images, odd M.  Every image must come out exactly as when it runs
    alone (range launches take one image per CTA), codebooks and stats alike."""
    import torch
    Ms = [3, 5, 8, 16, 17, 24, 31, 32, 33, 40, 64, 7, 12, 15, 2, 1]
    images, W0s, params = [], [], []
    for i, m in enumerate(Ms):
        img = synth.c1_image(100 + i)
        images.append(img)
        W0s.append(synth.init_codebook(synth.rng_for(1, 500 + i), img.astype(np.float32), m))
        iters = (1, 7, 20, 60)[i % 4]
        flags = itc.ITC_STOP_ON_FIXED if i % 3 == 0 else 0
        params.append(itc.make_params(2.0 + 0.5 * (i % 3), 3.0, iters, flags=flags))
    ts = [to_dev(im) for im in images]
    plan = itc.Plan(ts, Ms, params)
    W = plan.pack_W(W0s)
    st = itc.new_stats(len(images), W.device)
    itc.run(plan, W, st)
    Wr = plan.pack_W(W0s)
    sr = itc.new_stats(len(images), W.device)
    L = itc.lib()
    s = torch.cuda.current_stream().cuda_stream
    for b in range(len(images)):
        assert L.itc_run_fields_range(plan.host_ptr, plan.dev.data_ptr(), b, b + 1, plan.ws.data_ptr(),
                                      plan.ws.numel(), s) == 0
        assert L.itc_run_iterate_range(plan.host_ptr, plan.dev.data_ptr(), b, b + 1, Wr.data_ptr(),
                                       sr.data_ptr(), plan.ws.data_ptr(), plan.ws.numel(), s) == 0
    torch.cuda.synchronize()
    assert np.array_equal(W.cpu().numpy(), Wr.cpu().numpy())
    assert st.cpu().numpy().tobytes() == sr.cpu().numpy().tobytes()
    stats = itc.stats_to_numpy(st)
    done = [int(stats[b]["iters_done"]) for b in range(len(images))]
    # the iteration limits hold, and the stopping images stop early where the oracle does
    for b, p in enumerate(params):
        assert done[b] <= p.iters
    for b in (0, 3, 6):
        A, F, sxx = _oracle_fields(images[b], float(params[b].sigma[0]))
        Wo, dcs, tie, t = oracle.lattice_run(A, F, sxx, float(params[b].sigma[0]), W0s[b], params[b].iters,
                                             stop_on_fixed=True)
        if tie.min() > 1e-4:
            assert done[b] == t
            assert np.array_equal(plan.unpack_W(W)[b], Wo)


def _real_valued(W0, rng, nd=2):
    """Lattice sites moved by up to 0.45 px per axis: real-valued initial codebooks (as left by a
    continuous run, or by gradient steps on W)."""
    return (np.asarray(W0, np.float64) + rng.uniform(-0.45, 0.45, np.shape(W0))).astype(np.float32)


@pytest.mark.parametrize("seed", range(4))
def test_single_step_real_valued_codebook_snaps_to_lattice(seed):
    """Default (snap) mode from a real-valued W: one step rounds w_k + delta_k onto the lattice
    (Sec. 3.2; rounding floor(x + 0.5)), exactly as the oracle does, ties aside."""
    img = synth.c1_image(10 + seed)
    rng = np.random.default_rng(100 + seed)
    W0 = _real_valued(synth.init_codebook(synth.rng_for(1, 10 + seed), img.astype(np.float32), 8), rng)
    assert np.any(W0 != np.round(W0))
    A, F, _ = _oracle_fields(img, 2.0)
    Wn, raw, st = oracle.lattice_step(A, F, 2.0, W0.astype(np.float64))
    Wg, Wl, s, _ = gpu_step(img, 2.0, W0)
    assert_lattice_equal_except_ties(Wg, Wn, raw, what=f"seed {seed}")
    assert np.all(Wg == np.round(Wg)), "snap mode left the lattice"
    assert np.array_equal(Wl, Wg.astype(np.int32))
    assert s["moved"] == st["moved"]


def test_batched_run_real_valued_codebooks_grouped_ctas():
    """A batch whose images share iteration CTAs (M <= 16, 32, 64: 8, 4, 2 per CTA) and larger
    ones, every W_0 real-valued, default snap mode: each image's run equals the oracle's (or the
    batched plan passes the lockstep when the oracle trajectory has a tie)."""
    Ms = [5, 12, 16, 9, 20, 32, 27, 31, 40, 64, 50, 100, 128, 16, 3, 64]
    images, W0s, sig = [], [], []
    rng = np.random.default_rng(2024)
    for i, m in enumerate(Ms):
        img = synth.c3_batch(1, start=900 + i)[0][0][:160, :200].copy()
        if img.sum() < 2 * m:
            img = synth.c1_image(200 + i)
        images.append(img)
        W0s.append(_real_valued(synth.init_codebook(synth.rng_for(3, 80_000 + i), img.astype(np.float32), m), rng))
        sig.append((2.0, 3.0, 4.0)[i % 3])
    params = [itc.make_params(s, 3.0, 12) for s in sig]
    plan, Ws, st = run_plan(images, Ms, W0s, params)
    tied = 0
    for b in range(len(images)):
        assert np.all(Ws[b] == np.round(Ws[b])), f"image {b} left the lattice"
        A, F, sxx = _oracle_fields(images[b], sig[b])
        Wo, dcs, tie, t = oracle.lattice_run(A, F, sxx, sig[b], W0s[b], 12)
        if tie.min() > 1e-4:
            assert np.array_equal(Ws[b], Wo), f"image {b}: final codebooks differ"
            assert abs(st[b]["dcs"] - dcs[-1]) <= DCS_ATOL
        else:
            tied += 1
    if tied:
        plan_lockstep(images, Ms, sig, W0s, 12, what="real-valued W0")
