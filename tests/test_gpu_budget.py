"""Fields recomputed under a memory budget (the forward and the adjoint of Eq. (1) for weighted
ITC, Sec. 5, with the fields of Sec. 3.1 not kept for the whole batch): itc_run_budget and
itc_backward_budget against itc_run and itc_backward on the same plan.  Bar: bit for bit equal
codebooks, stats, dD/dW and dD/dh (the same kernels, tile configuration and summation order run
range by range), for budgets that cut the batch into many ranges down to one image each; the
stored path is itself held to the oracle by the other GPU tests, and one image here is checked
against the oracle gradient directly."""
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


def _batch():
    """Weighted images of ragged sizes, binary ones, and images with a separate V(X) width (their
    own A_s plane): a plan with several classes."""
    imgs, Ms, params = [], [], []
    for i in range(14):
        h = synth.c4_weights(20 + i, size=256)[: 96 + 11 * i, : 250 - 9 * i].copy()
        imgs.append(h)
        Ms.append((8, 16, 32, 12)[i % 4])
        params.append(itc.make_params((2.0, 3.0)[i % 2], 3.0, 6))
    for i in range(6):
        b = synth.c3_batch(1, start=1200 + i)[0][0].astype(np.float32)
        imgs.append(b)
        Ms.append(16)
        params.append(itc.params_parzen(2, xi=1.1, omega=1.7, iters=6) if i % 2 else itc.make_params(4.0, 3.0, 6))
    W0s = [synth.init_codebook(synth.rng_for(4, 7000 + i), im, m, 0.5 if i < 14 else 0.0)
           for i, (im, m) in enumerate(zip(imgs, Ms))]
    return imgs, Ms, params, W0s


def _stored(plan, W0s):
    import torch
    W = plan.pack_W(W0s)
    st = itc.new_stats(plan.B, W.device)
    itc.run(plan, W, st)
    gW = torch.empty_like(W)
    gh = torch.empty(plan.pixels, dtype=torch.float32, device=W.device)
    st2 = itc.new_stats(plan.B, W.device)
    gd = torch.linspace(-1.0, 2.0, plan.B, device=W.device)
    itc.backward(plan, W, grad_dcs=gd, grad_W=gW, grad_h=gh, stats=st2)
    torch.cuda.synchronize()
    return [x.cpu().numpy().copy() for x in (W, st, gW, gh, st2)]


def _budgeted(plan, W0s, ws):
    import torch
    W = plan.pack_W(W0s)
    st = itc.new_stats(plan.B, W.device)
    itc.run_budget(plan, W, ws, st)
    gW = torch.empty_like(W)
    gh = torch.empty(plan.pixels, dtype=torch.float32, device=W.device)
    st2 = itc.new_stats(plan.B, W.device)
    gd = torch.linspace(-1.0, 2.0, plan.B, device=W.device)
    itc.backward_budget(plan, W, ws, grad_dcs=gd, grad_W=gW, grad_h=gh, stats=st2)
    torch.cuda.synchronize()
    return [x.cpu().numpy().copy() for x in (W, st, gW, gh, st2)]


def test_budgeted_calls_equal_stored_fields_bit_for_bit():
    imgs, Ms, params, W0s = _batch()
    plan = itc.Plan([to_dev(im) for im in imgs], Ms, params)
    assert any(c["staging"] == "self" for c in plan.classes())
    ref = _stored(plan, W0s)
    fields = plan.ws_bytes
    for budget in (fields // 3, fields // 8, 0):
        ws = itc.budget_workspace(plan, budget)
        assert ws.numel() < fields
        ws.fill_(0xFF)   # NaN everywhere: nothing may be read that the call did not write
        got = _budgeted(plan, W0s, ws)
        for name, a, b in zip(("W", "stats", "grad_W", "grad_h", "backward stats"), got, ref):
            assert a.tobytes() == b.tobytes(), (budget, name)


def test_budgeted_gradient_against_the_oracle():
    """One weighted image in a budgeted plan whose window holds it alone, against the oracle's
    analytic gradient (normwise 1e-4, dD/dh element-wise)."""
    import torch
    imgs = [synth.c4_weights(40 + i)[:200, :230].copy() for i in range(3)]
    W0s = [synth.init_codebook(synth.rng_for(4, 7100 + i), im, 24, 0.5) for i, im in enumerate(imgs)]
    plan = itc.Plan([to_dev(im) for im in imgs], [24] * 3, itc.make_params(3.0, 3.0, 0), allocate_ws=False)
    ws = itc.budget_workspace(plan, 0)
    W = plan.pack_W(W0s)
    gW = torch.empty_like(W)
    gh = torch.empty(plan.pixels, dtype=torch.float32, device=W.device)
    itc.backward_budget(plan, W, ws, grad_W=gW, grad_h=gh)
    torch.cuda.synchronize()
    for b in range(3):
        h = imgs[b].astype(np.float64)
        A = oracle.fields2d(h, 3.0)[0]
        gref, ghref, sums = oracle.dcs_grad2d_dense(h, 3.0, W0s[b].astype(np.float64), A=A)
        g1, g2 = plan.unpack_W(gW)[b], plan.unpack_pixels(gh)[b]
        assert np.linalg.norm(g1 - gref) <= 1e-4 * np.linalg.norm(gref)
        assert np.linalg.norm(g2 - ghref) <= 1e-4 * np.linalg.norm(ghref)
        assert_grad_h_close(g2, h, A, sums, ghref, what=f"budgeted image {b}")


def test_budgeted_gray_lattice_and_mixed_plan():
    """A gray image as a 3-D lattice beside binary images, under the smallest budget."""
    gray = (synth.c5_gray(2, size=64).astype(np.int64) * 48 // 256).astype(np.uint8)
    imgs = [synth.c1_image(7), gray, synth.c1_image(8)]
    W0s = [synth.init_codebook(synth.rng_for(1, 77), imgs[0].astype(np.float32), 8),
           synth.init_codebook_gray(synth.rng_for(5, 77), gray, 10),
           synth.init_codebook(synth.rng_for(1, 78), imgs[2].astype(np.float32), 8)]
    params = [itc.make_params(2.0, 3.0, 8), itc.make_params((2.0, 2.0, 3.0), 3.0, 8), itc.make_params(2.0, 3.0, 8)]
    plan = itc.Plan([to_dev(im) for im in imgs], [8, 10, 8], params, ndims=[2, 3, 2], Gs=[1, 48, 1])
    ref = _stored(plan, W0s)
    got = _budgeted(plan, W0s, itc.budget_workspace(plan, 0))
    for a, b in zip(got, ref):
        assert a.tobytes() == b.tobytes()


def test_autograd_with_a_fields_budget_equals_stored_fields():
    import torch
    from paper_1310_7114_gb300.autograd import ITCDivergence, itc_divergence
    images = [synth.c4_weights(60 + i)[:120 + 10 * i, :140].copy() for i in range(5)]
    W0s = [synth.init_codebook(synth.rng_for(4, 7200 + i), im, 10, 0.5) for i, im in enumerate(images)]
    out = []
    for budget in (None, 1):
        hs = [to_dev(im).requires_grad_(True) for im in images]
        Wt = [to_dev(w).requires_grad_(True) for w in W0s]
        d = ITCDivergence.apply(3.0, 3.0, *hs, *Wt) if budget is None else itc_divergence(hs, Wt, 3.0, 3.0, budget)
        (d * torch.arange(1.0, 6.0, device=d.device)).sum().backward()
        out.append((d.detach().cpu().numpy(), [h.grad.cpu().numpy() for h in hs], [w.grad.cpu().numpy() for w in Wt]))
    (d0, gh0, gw0), (d1, gh1, gw1) = out
    assert d0.tobytes() == d1.tobytes()
    assert all(a.tobytes() == b.tobytes() for a, b in zip(gh0, gh1))
    assert all(a.tobytes() == b.tobytes() for a, b in zip(gw0, gw1))
