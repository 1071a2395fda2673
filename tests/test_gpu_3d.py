"""GPU parity on the gray-value lattice [u, v, g] (Sec. 1 (ii); the "memory overhead" of
Sec. 6 is exactly these four 3-D fields): itc_fields (ndim 3), the batched run and the backward
vs the FP64 oracle, including the full-size 256x256x256 workload (sampled sites, and the final
codebook after 100 iterations)."""
import numpy as np
import pytest

import oracle
from gpuhelp import DCS_ATOL, assert_fields_close, plan_lockstep, radii, to_dev
from paper_1310_7114_gb300 import build, itc, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    itc.lib()


def gpu_fields3d(gray, G, sigma, hw=None, absolute=False):
    import torch
    t = to_dev(gray)
    w = to_dev(hw.astype(np.float32)) if hw is not None else None
    F, sxx = itc.fields(t, sigma, 3.0, absolute, ndim=3, G=G, weight=w)
    torch.cuda.synchronize()
    W = gray.shape[1]
    return F[..., :W].cpu().numpy().astype(np.float64), float(sxx.item())


def _smooth_gray(seed, H, W, G):
    g = synth.c5_gray(seed, size=max(H, W))[:H, :W].astype(np.int64)
    return (g * G // 256).astype(np.uint8)


@pytest.mark.parametrize("sigma,G,weighted,absolute", [
    ((3.0, 3.0, 8.0), 64, False, False),
    ((3.0, 3.0, 8.0), 64, True, False),
    ((3.0, 3.0, 8.0), 50, True, True),
    ((2.0, 2.5, 4.0), 37, False, False),   # runtime-radius path, G not a multiple of the slice batch
])
def test_fields3d_full_volume(sigma, G, weighted, absolute):
    gray = _smooth_gray(1, 40, 36, G)
    hw = np.random.default_rng(2).random((40, 36)) if weighted else None
    g, sxx = gpu_fields3d(gray, G, sigma, hw, absolute)
    ref = oracle.fields3d(gray, G, sigma, hw=hw, absolute=absolute)
    assert_fields_close(list(g), ref, radii(sigma, 3.0, 3), absolute, f"3-D {sigma} G={G}")
    if not absolute:
        occ = np.zeros((G, 40, 36))
        uu, vv = np.meshgrid(np.arange(40), np.arange(36), indexing="ij")
        occ[gray, uu, vv] = 1.0 if hw is None else hw
        ref_sxx = float((occ * ref[0]).sum())
        assert abs(sxx - ref_sxx) <= 1e-5 * ref_sxx


def test_fields3d_c5_full_size_sampled():
    gray = synth.c5_gray(0)
    g, sxx = gpu_fields3d(gray, 256, (3.0, 3.0, 8.0))
    rng = np.random.default_rng(3)
    n = 3000
    sites = np.stack([rng.integers(0, 256, n), rng.integers(0, 256, n), rng.integers(0, 256, n)], 1)
    # half the sites on occupied voxels, where the fields are largest
    sites[: n // 2, 2] = gray[sites[: n // 2, 0], sites[: n // 2, 1]]
    ref = oracle.fields3d_sites(gray, sites, 256, (3.0, 3.0, 8.0))
    gs = [g[f][sites[:, 2], sites[:, 0], sites[:, 1]] for f in range(4)]
    assert_fields_close(gs, ref, [9, 9, 24], False, "C5 sites")


def _run3d(gray, G, sigma, M, iters, W0, hw=None):
    import torch
    t = to_dev(gray)
    w = to_dev(hw.astype(np.float32)) if hw is not None else None
    plan = itc.Plan([t], [M], itc.make_params(sigma, 3.0, iters), ndims=[3], Gs=[G], weights=[w])
    W = plan.pack_W([W0])
    st = itc.new_stats(1, W.device)
    itc.run(plan, W, st)
    torch.cuda.synchronize()
    return plan, W, plan.unpack_W(W)[0], itc.stats_to_numpy(st)[0]


def _check_run3d(gray, G, sigma, M, iters, W0, Wg, st, hw=None):
    A, Fu, Fv, Fg = oracle.fields3d(gray, G, sigma, hw=hw)
    occ = np.zeros((G,) + gray.shape)
    uu, vv = np.meshgrid(np.arange(gray.shape[0]), np.arange(gray.shape[1]), indexing="ij")
    occ[gray, uu, vv] = 1.0 if hw is None else hw
    sxx = float((occ * A).sum())
    Wo, dcs, tie, _ = oracle.lattice_run(A, [Fu, Fv, Fg], sxx, sigma, W0, iters)
    if tie.min() > 1e-4:
        assert np.array_equal(Wg, Wo)
        assert abs(st["dcs"] - dcs[-1]) <= DCS_ATOL
    else:
        # the plan in lockstep with the oracle's steps
        def ostep(b, W):
            Wn, raw, _ = oracle.lattice_step(A, [Fu, Fv, Fg], sigma, W)
            return Wn, raw

        plan_lockstep([gray], [M], itc.make_params(sigma, 3.0, 1), [W0], iters, ostep, ndims=[3], Gs=[G],
                      weights=[hw] if hw is not None else None, what="3-D lockstep")


def test_run3d_small():
    gray = _smooth_gray(4, 48, 40, 64)
    W0 = synth.init_codebook_gray(synth.rng_for(5, 7), gray, 12)
    _, _, Wg, st = _run3d(gray, 64, (3.0, 3.0, 8.0), 12, 30, W0)
    _check_run3d(gray, 64, (3.0, 3.0, 8.0), 12, 30, W0, Wg, st)


def test_run3d_c5_full_size():
    gray = synth.c5_gray(0)
    W0 = synth.init_codebook_gray(synth.rng_for(5, 0), gray, 64)
    _, _, Wg, st = _run3d(gray, 256, (3.0, 3.0, 8.0), 64, 100, W0)
    _check_run3d(gray, 256, (3.0, 3.0, 8.0), 64, 100, W0, Wg, st)


def test_backward3d_matches_oracle():
    import torch
    gray = _smooth_gray(6, 20, 18, 32)
    hw = np.random.default_rng(8).random((20, 18))
    W0 = synth.init_codebook_gray(synth.rng_for(5, 9), gray, 6)
    plan, W, _, _ = _run3d(gray, 32, (1.5, 1.5, 3.0), 6, 0, W0, hw)
    gW = torch.empty_like(W)
    gh = torch.empty(plan.pixels, dtype=torch.float32, device=W.device)
    itc.backward(plan, W, grad_W=gW, grad_h=gh)
    torch.cuda.synchronize()
    X, hx = oracle.gray_points(gray, None)
    gref, ghref = oracle.dcs_grad((20, 18, 32), X, hw.ravel(), (1.5, 1.5, 3.0), W0.astype(np.float64))
    g1 = gW.cpu().numpy().reshape(-1, 3)
    assert np.linalg.norm(g1 - gref) <= 1e-4 * np.linalg.norm(gref)
    g2 = gh.cpu().numpy()
    assert np.linalg.norm(g2 - ghref) <= 1e-4 * np.linalg.norm(ghref)


def test_fields3d_plan_of_several_images():
    """The fields launch of a 3-D plan gives each persistent CTA a run of slice tiles that crosses
    image boundaries (and windows, which it stages anew).  Every image's fields equal its own
    single-image call bit for bit (the same products in the same order) and match the oracle;
    its S_XX (one partial per slice tile) matches the oracle's."""
    import torch
    specs = [(37, 70, 48, False), (64, 33, 20, True), (20, 100, 64, False), (45, 45, 31, True), (9, 7, 5, False)]
    sigma = (3.0, 3.0, 8.0)
    grays, hws = [], []
    for i, (H, W, G, weighted) in enumerate(specs):
        grays.append(_smooth_gray(20 + i, H, W, G))
        hws.append(np.random.default_rng(30 + i).random((H, W)) if weighted else None)
    bufs, views = itc.pack_images(grays, "cuda")   # rows on 16-byte boundaries
    wts = []
    for v, h in zip(views, hws):   # weights share the image's row pitch
        if h is None:
            wts.append(None)
            continue
        wp = torch.zeros((v.shape[0], v.stride(0)), dtype=torch.float32, device="cuda")
        wp[:, :v.shape[1]] = torch.from_numpy(h.astype(np.float32)).cuda()
        wts.append(wp[:, :v.shape[1]])
    plan = itc.Plan(views, [4] * len(specs), itc.make_params(sigma, 3.0, 0), ndims=[3] * len(specs),
                    Gs=[s[2] for s in specs], weights=wts)
    W0 = [synth.init_codebook_gray(synth.rng_for(5, 40 + i), g, 4) for i, g in enumerate(grays)]
    W = plan.pack_W(W0)
    st = itc.new_stats(len(specs), "cuda")
    itc.run(plan, W, st)
    torch.cuda.synchronize()
    stats = itc.stats_to_numpy(st)
    for b, (H, W_, G, _) in enumerate(specs):
        mine = plan.fields_of(b)[..., :W_].cpu().numpy()
        single, _ = itc.fields(views[b], sigma, 3.0, ndim=3, G=G, weight=wts[b])
        torch.cuda.synchronize()
        assert np.array_equal(mine, single[..., :W_].cpu().numpy()), f"image {b}: plan vs single call"
        ref = oracle.fields3d(grays[b], G, sigma, hw=hws[b])
        assert_fields_close(list(mine.astype(np.float64)), ref, radii(sigma, 3.0, 3), False, f"plan image {b}")
        occ = np.zeros((G, H, W_))
        uu, vv = np.meshgrid(np.arange(H), np.arange(W_), indexing="ij")
        occ[grays[b], uu, vv] = 1.0 if hws[b] is None else hws[b]
        ref_sxx = float((occ * ref[0]).sum())
        assert abs(stats["sxx"][b] - ref_sxx) <= 1e-5 * ref_sxx, f"image {b}: S_XX"
