"""GPU parity of the recursive (large-width) fields, Sec. 3.1, against the oracle's recursion
(Deriche's fit by complex first-order recursions, FP64): field planes of a plan, S_XX, and
Algorithm 1 runs with the width schedule of Sec. 4 (large tau, separate V(X) width), in plans
that also hold mask classes.  Bars: fields within 2e-5 of the field's range (FP32 recursions of
~sigma effective length) and element-wise within the rounding envelope of the recursions
(`rounding_envelope`), S_XX within 1e-5 relative, lattice positions as for the mask fields
(ties aside, lockstep otherwise)."""
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


# Deriche's published fit of exp(-x^2/2) by two damped sinusoids: weight magnitudes |alpha_t - i beta_t|
# and decay rates b_t (alpha = 1.680, -0.6803; beta = 3.735, -0.2598; b = 1.783, 1.723).
DERICHE_WEIGHT = (float(np.hypot(1.680, 3.735)), float(np.hypot(0.6803, 0.2598)))
DERICHE_DECAY = (1.783, 1.723)
U32 = 2.0 ** -24


def _axis_envelope(n, sigma, power):
    """sum_t |c_t| (1 + |d|)^power rho_t^|d|, d = -(n-1) .. n-1, rho_t = exp(-b_t / sigma)."""
    d = np.abs(np.arange(-(n - 1), n, dtype=np.float64))
    return sum(w * (1.0 + d) ** power * np.exp(-b * d / sigma) for w, b in zip(DERICHE_WEIGHT, DERICHE_DECAY))


def _conv(x, k, axis):
    from scipy.ndimage import convolve1d
    return convolve1d(x, k, axis=axis, mode="constant", cval=0.0)


def rounding_envelope(h, sigma):
    """Element-wise bounds (A, F_u, F_v) on the FP32 error of the recursive fields.

    One complex first-order step s[n] = x[n] + z s[n-1] in FP32 commits at most about 4u
    (u = 2^-24) of |x[n]| + |z s[n-1]|; that error then decays by |z| = rho per step, so the
    accumulated error of a value recursion is at most 4u sum_m (1 + m) rho^m |x[n - m]|, and of a
    moment recursion (whose state sums the value state) 4u sum_m (1 + m)^2 rho^m |x[n - m]|; the
    poles and weights rounded once to FP32 stay inside the same (1 + m) factor.  Along one axis
    the field thus errs by at most 4u (e_p * |x|) with e_p(d) = sum_t |c_t| (1 + |d|)^p rho_t^|d|
    (p = 1 for values, 2 for moments), and since the fitted kernel and its moment are below e_1
    and e_2, the two passes give |dA| <= 8u e_1,u * e_1,v * |h|, |dF_u| <= 8u e_2,u * e_1,v * |h|,
    |dF_v| <= 8u e_1,u * e_2,v * |h|.  The bound used is twice that (16u), for the final
    combinations Re(c s) and the sums of the two terms."""
    su, sv = (float(sigma), float(sigma)) if np.isscalar(sigma) else map(float, sigma)
    H, W = h.shape
    a = np.abs(np.asarray(h, np.float64))
    rows1 = _conv(a, _axis_envelope(W, sv, 1), 1)
    rows2 = _conv(a, _axis_envelope(W, sv, 2), 1)
    c = 16.0 * U32
    return (c * _conv(rows1, _axis_envelope(H, su, 1), 0), c * _conv(rows1, _axis_envelope(H, su, 2), 0),
            c * _conv(rows2, _axis_envelope(H, su, 1), 0))


def _plan(images, Ms, params):
    import torch
    plan = itc.Plan([to_dev(im) for im in images], Ms, params)
    return plan


@pytest.mark.parametrize("sigma", [6.0, 12.5, 30.0, (8.0, 20.0)])
def test_recursive_fields_and_sxx(sigma):
    import torch
    rng = np.random.default_rng(int(np.sum(sigma) * 10))
    imgs = [(rng.random((97, 131)) < 0.3).astype(np.uint8), (rng.random((150, 70)) * (rng.random((150, 70)) < 0.5)).astype(np.float32)]
    params = [itc.make_params(sigma, 3.0, 0, flags=itc.ITC_RECURSIVE)] * 2
    plan = _plan(imgs, [4, 4], params)
    assert all(c["staging"] == "recursive" for c in plan.classes())
    W = plan.pack_W([synth.init_codebook(synth.rng_for(7, b), im.astype(np.float32), 4) for b, im in enumerate(imgs)])
    st = itc.new_stats(2, W.device)
    itc.run(plan, W, st)
    torch.cuda.synchronize()
    s = itc.stats_to_numpy(st)
    for b, im in enumerate(imgs):
        h = im.astype(np.float64)
        A, Fu, Fv = oracle.fields2d_recursive(h, sigma)
        F = plan.fields_of(b)[:, 0, :, :im.shape[1]].cpu().numpy().astype(np.float64)
        scale = A.max()
        sm = float(np.max(sigma))
        assert np.abs(F[0] - A).max() <= 2e-5 * scale, b
        assert np.abs(F[1] - Fu).max() <= 2e-5 * sm * scale, b
        assert np.abs(F[2] - Fv).max() <= 2e-5 * sm * scale, b
        # element-wise, also in the tails where the fields are small
        for i, (ref, env) in enumerate(zip((A, Fu, Fv), rounding_envelope(h, sigma))):
            err = np.abs(F[i] - ref)
            worst = float(np.max(err / np.maximum(env, 1e-300)))
            assert worst <= 1.0, (b, i, worst)
        sxx = oracle.sxx(h, A)
        assert abs(s[b]["sxx"] - sxx) <= 1e-5 * sxx


def _check_run(plan, b, img, p, W0, Wg, st):
    tau = np.array(list(p.sigma)[:2], float)
    rho = np.array([x if x > 0 else t for x, t in zip(list(p.sigma_pair)[:2], tau)])
    sw = np.array([x if x > 0 else t for x, t in zip(list(p.sigma_self)[:2], tau)])
    h = img.astype(np.float64)
    A, Fu, Fv = oracle.fields2d_recursive(h, tau)
    sxx = oracle.sxx(h, oracle.fields2d_recursive(h, sw)[0])
    K = oracle.dcs_const(tau, rho, sw)
    assert abs(st["sxx"] - sxx) <= 1e-5 * sxx
    Wo, dcs, tie, t = oracle.lattice_run(A, [Fu, Fv], sxx, tau, W0, p.iters, step_scale=p.step_scale, rho=rho,
                                         dcs_const=K)
    if tie.min() > 1e-4:
        assert np.array_equal(Wg, Wo)
        assert abs(st["dcs"] - dcs[-1]) <= DCS_ATOL
        return
    # lockstep: a one-iteration plan over this image (recursive fields, its widths) from the
    # oracle's W every iteration
    def ostep(_, W):
        Wn, raw, _ = oracle.lattice_step(A, [Fu, Fv], tau, W, step_scale=p.step_scale, rho=rho)
        return Wn, raw

    plan_lockstep([img], [len(W0)], p, [W0], p.iters, ostep, what="recursive lockstep")


def test_schedule_run_with_recursive_fields():
    """omega = sqrt(N/M)/2 and xi = omega/2 on whole images give widths far beyond the masks'
    reach; with ITC_RECURSIVE the plan runs them beside mask classes."""
    import torch
    imgs = [synth.c2_image(3)[:300, :260].copy(), synth.c1_image(31), synth.c1_image(32)]
    Ms = [6, 4, 8]
    W0s = [synth.init_codebook(synth.rng_for(2, 400 + i), im.astype(np.float32), m) for i, (im, m) in enumerate(zip(imgs, Ms))]
    params = [itc.params_parzen(2, mass=float(im.sum()), M=m, iters=15, flags=itc.ITC_RECURSIVE)
              for im, m in zip(imgs[:2], Ms[:2])]
    params.append(itc.make_params(2.0, 3.0, 15))
    assert params[0].sigma[0] > 10.0
    plan = _plan(imgs, Ms, params)
    kinds = sorted(c["staging"] for c in plan.classes())
    assert "recursive" in kinds and ("tma" in kinds or "plain" in kinds)
    W = plan.pack_W(W0s)
    st = itc.new_stats(3, W.device)
    itc.run(plan, W, st)
    torch.cuda.synchronize()
    Ws, s = plan.unpack_W(W), itc.stats_to_numpy(st)
    for b in range(2):
        _check_run(plan, b, imgs[b], params[b], W0s[b], Ws[b], s[b])
    # the mask-field image in the same plan is unchanged by its neighbours
    A, Fu, Fv = oracle.fields2d(imgs[2].astype(np.float64), 2.0)
    Wo, dcs, tie, t = oracle.lattice_run(A, [Fu, Fv], oracle.sxx(imgs[2].astype(np.float64), A), 2.0, W0s[2], 15)
    if tie.min() > 1e-4:
        assert np.array_equal(Ws[2], Wo)
