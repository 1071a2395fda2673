"""GPU parity with separate kernel widths (Sec. 2.1): fields at tau, codebook pair sums at rho,
V(X) at s, the pair factor tau^2/rho^2 of the update and the normalising constant of Eq. (1),
against the FP64 oracle; also the paper's width schedule of Sec. 4 (omega = sqrt(N/M)/2,
xi = omega/2) through itc_params_parzen.  Bars as for the single-width path: S_XX within 1e-5
relative, lattice positions identical except oracle values within 1e-4 of a half-integer
(lockstep otherwise), D_cs within the FP32 bound, gradients normwise within 1e-4."""
import numpy as np
import pytest

import oracle
from gpuhelp import DCS_ATOL, plan_lockstep, to_dev
from paper_1310_7114_gb300 import build, itc, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    itc.lib()


def _widths(p, ndim=2):
    tau = np.array(list(p.sigma)[:ndim], float)
    rho = np.array([x if x > 0 else t for x, t in zip(list(p.sigma_pair)[:ndim], tau)])
    s = np.array([x if x > 0 else t for x, t in zip(list(p.sigma_self)[:ndim], tau)])
    return tau, rho, s


def _oracle_run(img, p, W0, iters):
    tau, rho, s = _widths(p)
    h = img.astype(np.float64)
    A, Fu, Fv = oracle.fields2d(h, tau, p.trunc)
    sxx = oracle.sxx(h, oracle.fields2d(h, s, p.trunc)[0])
    K = oracle.dcs_const(tau, rho, s)
    return (A, [Fu, Fv], sxx, K), oracle.lattice_run(A, [Fu, Fv], sxx, tau, W0, iters, step_scale=p.step_scale,
                                                     rho=rho, dcs_const=K)


def _lockstep(img, p, W0, iters, ref):
    """The plan (one image, its widths) in lockstep with the oracle's steps."""
    A, F, sxx, K = ref
    tau, rho, s = _widths(p)

    def ostep(b, W):
        Wn, raw, _ = oracle.lattice_step(A, F, tau, W, step_scale=p.step_scale, rho=rho)
        return Wn, raw

    plan_lockstep([img], [len(W0)], p, [W0], iters, ostep, what="widths lockstep")


def _run(images, Ms, W0s, params):
    import torch
    plan = itc.Plan([to_dev(im) for im in images], Ms, params)
    W = plan.pack_W(W0s)
    st = itc.new_stats(len(images), W.device)
    itc.run(plan, W, st)
    torch.cuda.synchronize()
    return plan, plan.unpack_W(W), itc.stats_to_numpy(st)


def _check(img, p, W0, Wg, st, what):
    ref, (Wo, dcs, tie, t) = _oracle_run(img, p, W0, p.iters)
    assert abs(st["sxx"] - ref[2]) <= 1e-5 * ref[2], what
    if tie.min() > 1e-4:
        assert np.array_equal(Wg, Wo), f"{what}: final codebooks differ"
        assert abs(st["dcs"] - dcs[-1]) <= DCS_ATOL, (what, st["dcs"], dcs[-1])
    else:
        _lockstep(img, p, W0, p.iters, ref)


@pytest.mark.parametrize("xi,om", [(1.0, 1.5), (1.4, 0.8)])
def test_fields_sxx_at_the_self_width(xi, om):
    p = itc.params_parzen(2, xi=xi, omega=om)
    tau, rho, s = _widths(p)
    img = synth.c1_image(3)
    F, sxx = itc.fields(to_dev(img), tuple(tau), 3.0, sigma_self=tuple(s))
    h = img.astype(np.float64)
    want = oracle.sxx(h, oracle.fields2d(h, s)[0])
    assert abs(sxx.item() - want) <= 1e-5 * want
    A = oracle.fields2d(h, tau)[0]
    assert np.abs(F[0, 0, :, :64].cpu().numpy() - A).max() <= 1e-5 * A.max()


@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("seed", range(2))
def test_run_with_parzen_widths(seed, form):
    img = synth.c1_image(10 + seed)
    W0 = synth.init_codebook(synth.rng_for(1, 100 + seed), img.astype(np.float32), 8)
    p = itc.params_parzen(2, xi=1.0, omega=1.6, iters=30, form=form)
    _, Ws, st = _run([img], [8], [W0], p)
    _check(img, p, W0, Ws[0], st[0], f"seed {seed} form {form}")


def test_run_with_the_width_schedule():
    """omega = sqrt(N/M)/2, xi = omega/2 from the foreground count (Sec. 4), in a batch mixing
    schedule images and single-width images (self-overlap passes beside plain classes)."""
    imgs = [synth.c1_image(20 + i) for i in range(4)]
    Ms = [16, 12, 8, 16]
    W0s = [synth.init_codebook(synth.rng_for(1, 200 + i), im.astype(np.float32), m) for i, (im, m) in enumerate(zip(imgs, Ms))]
    params = [itc.params_parzen(2, mass=float(im.sum()), M=m, iters=20) for im, m in zip(imgs[:3], Ms[:3])]
    params.append(itc.make_params(2.0, 3.0, 20))
    plan, Ws, st = _run(imgs, Ms, W0s, params)
    assert any(c["staging"] == "self" for c in plan.classes())
    for b in range(4):
        _check(imgs[b], params[b], W0s[b], Ws[b], st[b], f"image {b}")


def test_backward_with_three_widths():
    import torch
    h = synth.c4_weights(3)[:96, :120].copy()
    W0 = synth.init_codebook(synth.rng_for(4, 33), h, 12, 0.5)
    p = itc.params_parzen(2, xi=1.2, omega=1.7)
    tau, rho, s = _widths(p)
    plan = itc.Plan([to_dev(h)], [12], p)
    W = plan.pack_W([W0])
    st = itc.new_stats(1, W.device)
    itc.run(plan, W, st)
    gW = torch.empty_like(W)
    gh = torch.empty(plan.pixels, dtype=torch.float32, device=W.device)
    st2 = itc.new_stats(1, W.device)
    itc.backward(plan, W, grad_W=gW, grad_h=gh, stats=st2)
    torch.cuda.synchronize()
    gW_ref, gh_ref, sums = oracle.dcs_grad2d_dense(h.astype(np.float64), tau, W0.astype(np.float64), rho=rho, s=s)
    d_ref = float(np.log(sums[1]) + np.log(sums[2]) - 2 * np.log(sums[0]) + oracle.dcs_const(tau, rho, s))
    gWg, ghg = plan.unpack_W(gW)[0], plan.unpack_pixels(gh)[0]

    def nrel(a, b):
        return np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b)

    assert nrel(gWg, gW_ref) <= 1e-4
    assert nrel(ghg, gh_ref) <= 1e-4
    assert abs(itc.stats_to_numpy(st2)[0]["dcs"] - d_ref) <= DCS_ATOL
    assert abs(itc.stats_to_numpy(st)[0]["dcs"] - d_ref) <= DCS_ATOL
