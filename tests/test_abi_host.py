"""Host-side checks of the C ABI (no GPU needed): the library loads, exports every function
include/itc.h declares, and rejects invalid arguments before touching the device; batch plans
(host-only) lay out offsets as documented."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1310_7114_gb300 import build as itc_build
from paper_1310_7114_gb300 import itc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    itc_build.build()
    return itc.lib()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "itc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(itc_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(L, n), n
    assert sorted(itc.EXPORTS) == names


def test_struct_sizes_match_the_header():
    assert ctypes.sizeof(itc.ItcImage) == 40
    assert ctypes.sizeof(itc.ItcParams) == 52
    assert ctypes.sizeof(itc.ItcStats) == 56


def test_queries(L):
    assert L.itc_field_pitch(1) == 4 and L.itc_field_pitch(64) == 64 and L.itc_field_pitch(65) == 68
    img = itc.ItcImage(2, 100, 70, 1, 80, itc.ITC_U8, 0x1000, None)
    assert L.itc_fields_bytes(ctypes.byref(img)) == 3 * 100 * 72 * 4
    img3 = itc.ItcImage(3, 10, 12, 256, 12, itc.ITC_U8, 0x1000, None)
    assert L.itc_fields_bytes(ctypes.byref(img3)) == 4 * 256 * 10 * 12 * 4
    bad = itc.ItcImage(2, 100, 70, 1, 60, itc.ITC_U8, 0x1000, None)  # pitch < W
    assert L.itc_fields_bytes(ctypes.byref(bad)) == 0
    for c in (0, 1, -1, -2, -3, -4, -5, -6, 99):
        assert isinstance(L.itc_status_string(c), bytes)


def _p(sigma=2.0, trunc=3.0, iters=0, step=1.0, flags=0):
    return itc.make_params(sigma, trunc, iters, step, flags)


@pytest.mark.parametrize("mutate,code", [
    (lambda i, p: setattr(i, "data", None), itc.ITC_ERR_INVALID_ARG),
    (lambda i, p: setattr(i, "ndim", 4), itc.ITC_ERR_INVALID_ARG),
    (lambda i, p: setattr(i, "H", 0), itc.ITC_ERR_INVALID_ARG),
    (lambda i, p: setattr(i, "dtype", 7), itc.ITC_ERR_INVALID_ARG),
    (lambda i, p: setattr(p, "trunc", 0.0), itc.ITC_ERR_INVALID_ARG),
    (lambda i, p: setattr(p, "trunc", float("nan")), itc.ITC_ERR_INVALID_ARG),
    (lambda i, p: p.sigma.__setitem__(0, -1.0), itc.ITC_ERR_INVALID_ARG),
    (lambda i, p: setattr(p, "flags", 64), itc.ITC_ERR_INVALID_ARG),
    (lambda i, p: p.sigma.__setitem__(1, 40.0), itc.ITC_ERR_UNSUPPORTED),
])
def test_fields_rejects_invalid_arguments_without_launching(L, mutate, code):
    img = itc.ItcImage(2, 64, 64, 1, 64, itc.ITC_U8, 0x1000, None)
    p = _p()
    mutate(img, p)
    rc = L.itc_fields(ctypes.byref(img), ctypes.byref(p), 0x2000, None, 0x3000, 1 << 20, None)
    assert rc == code


def test_fields_workspace_checks(L):
    img = itc.ItcImage(2, 64, 64, 1, 64, itc.ITC_U8, 0x1000, None)
    p = _p()
    need = L.itc_fields_workspace_bytes(ctypes.byref(img))
    assert need > 0
    assert L.itc_fields(ctypes.byref(img), ctypes.byref(p), 0x2000, None, None, need, None) == itc.ITC_ERR_WORKSPACE
    assert L.itc_fields(ctypes.byref(img), ctypes.byref(p), 0x2000, None, 0x3000, need - 8, None) == itc.ITC_ERR_WORKSPACE
    assert L.itc_fields(ctypes.byref(img), ctypes.byref(p), 0x2004, None, 0x3000, need, None) == itc.ITC_ERR_INVALID_ARG


def test_step_rejects_bad_codebook_sizes(L):
    img = itc.ItcImage(2, 64, 64, 1, 64, itc.ITC_U8, 0x1000, None)
    p = _p(iters=1)
    for M in (0, -3, 5000):
        assert L.itc_step(ctypes.byref(img), ctypes.byref(p), 0x2000, 0x3000, M, 0x4000, 0x5000, None, None,
                          None) == itc.ITC_ERR_INVALID_ARG
    assert L.itc_step(ctypes.byref(img), ctypes.byref(p), 0x2000, None, 8, 0x4000, 0x5000, None, None,
                      None) == itc.ITC_ERR_INVALID_ARG


def _plan(L, shapes, Ms, params, ndims=None):
    B = len(shapes)
    ndims = ndims or [2] * B
    imgs = (itc.ItcImage * B)(*[itc.ItcImage(d, h, w, 256 if d == 3 else 1, w + 3, itc.ITC_U8, 0x10000 * (b + 1), None)
                                for b, ((h, w), d) in enumerate(zip(shapes, ndims))])
    M = (ctypes.c_int * B)(*Ms)
    if isinstance(params, list):
        ps, stride = (itc.ItcParams * B)(*params), 1
    else:
        ps, stride = (itc.ItcParams * 1)(params), 0
    nb = L.itc_plan_bytes(B)
    buf = ctypes.create_string_buffer(nb)
    ws = ctypes.c_size_t(0)
    rc = L.itc_plan(B, imgs, M, ps, stride, ctypes.cast(buf, ctypes.c_void_p), nb, ctypes.byref(ws))
    return rc, buf, ws.value


def test_plan_layout(L):
    shapes = [(64, 64), (100, 70), (300, 513), (17, 9)]
    Ms = [8, 16, 128, 3]
    rc, buf, ws = _plan(L, shapes, Ms, [_p(2.0), _p(3.0), _p(2.0), _p(4.0)])
    assert rc == 0
    assert L.itc_plan_pixels(ctypes.cast(buf, ctypes.c_void_p)) == sum(h * w for h, w in shapes)
    # workspace holds at least the fields of every image (3 planes, rows padded to 4 floats)
    assert ws >= sum(3 * h * ((w + 3) // 4 * 4) * 4 for h, w in shapes)
    assert ws % 256 == 0


def test_plan_rejects_invalid_batches(L):
    assert _plan(L, [(64, 64)], [0], _p())[0] == itc.ITC_ERR_INVALID_ARG
    assert _plan(L, [(64, 64)], [4096], _p())[0] == itc.ITC_ERR_INVALID_ARG
    assert _plan(L, [(64, 64), (32, 32)], [8, 8], [_p(), _p(trunc=-1.0)])[0] == itc.ITC_ERR_INVALID_ARG
    # more parameter classes than a plan holds
    shapes = [(32, 32)] * 20
    rc = _plan(L, shapes, [4] * 20, [_p(1.0 + 0.1 * i) for i in range(20)])[0]
    assert rc == itc.ITC_ERR_UNSUPPORTED
    nb = L.itc_plan_bytes(1)
    assert nb > 0 and L.itc_plan_bytes(0) == 0


def test_run_rejects_bad_plan_and_workspace(L):
    rc, buf, ws = _plan(L, [(64, 64)], [8], _p(iters=5))
    assert rc == 0
    bogus = ctypes.create_string_buffer(len(buf.raw))
    assert L.itc_run(ctypes.cast(bogus, ctypes.c_void_p), 0x1000, 0x2000, None, 0x4000, ws, None) == itc.ITC_ERR_INVALID_ARG
    assert L.itc_run(ctypes.cast(buf, ctypes.c_void_p), 0x1000, 0x2000, None, 0x4000, ws - 1, None) == itc.ITC_ERR_WORKSPACE
    assert L.itc_run(ctypes.cast(buf, ctypes.c_void_p), 0x1000, 0x2000, None, 0x4010, ws, None) == itc.ITC_ERR_WORKSPACE
    assert L.itc_backward(ctypes.cast(buf, ctypes.c_void_p), 0x1000, 0x2000, None, None, None, None, None, ws,
                          None) == itc.ITC_ERR_WORKSPACE


def test_product_path_has_no_cpu_fallback():
    """The package never imports the oracle, and the binding fails loudly without the library."""
    pkg = os.path.join(ROOT, "paper_1310_7114_gb300")
    for f in os.listdir(pkg):
        if f.endswith(".py"):
            src = open(os.path.join(pkg, f)).read()
            assert "import oracle" not in src and "from oracle" not in src, f


def test_plan_class_queries_and_configuration_checks(L):
    """Class queries are host-only; configuration and tuning reject bad arguments before any
    device work.  Rows of 3 bytes past a multiple of 16 cannot use tensor tiles."""
    rc, buf, ws = _plan(L, [(64, 64), (100, 70), (300, 513), (17, 9)], [8, 16, 128, 3],
                        [_p(2.0), _p(3.0), _p(2.0), _p(4.0)])
    assert rc == 0
    hp = ctypes.cast(buf, ctypes.c_void_p)
    assert L.itc_plan_classes(hp) == 3
    assert L.itc_plan_classes(None) == itc.ITC_ERR_INVALID_ARG
    seen = []
    for c in range(3):
        nd, th, gp, st, ni = (ctypes.c_int(-9) for _ in range(5))
        sig, ms = (ctypes.c_float * 3)(), ctypes.c_float(-1.0)
        assert L.itc_plan_class(hp, c, ctypes.byref(nd), sig, ctypes.byref(th), ctypes.byref(gp), ctypes.byref(st),
                                ctypes.byref(ni), ctypes.byref(ms)) == 0
        assert nd.value == 2 and th.value == 64 and gp.value == 0 and st.value == 0 and ms.value == 0.0
        seen.append((sig[0], ni.value))
    assert sorted(seen) == [(2.0, 2), (3.0, 1), (4.0, 1)]
    assert L.itc_plan_class(hp, 3, None, None, None, None, None, None, None) == itc.ITC_ERR_INVALID_ARG
    assert L.itc_plan_class(hp, 0, None, None, None, None, None, None, None) == 0
    dev = 0x100000
    assert L.itc_plan_configure(hp, dev, 0, 64, 0, 1, None) == itc.ITC_ERR_UNSUPPORTED
    assert L.itc_plan_configure(hp, dev, 0, 32, 0, 0, None) == itc.ITC_ERR_INVALID_ARG
    assert L.itc_plan_configure(hp, dev, 5, 64, 0, 0, None) == itc.ITC_ERR_INVALID_ARG
    assert L.itc_plan_configure(hp, dev, 0, 64, -1, 0, None) == itc.ITC_ERR_INVALID_ARG
    assert L.itc_plan_configure(hp, dev, 0, 64, 0, 2, None) == itc.ITC_ERR_INVALID_ARG
    assert L.itc_autotune(hp, dev, 0x4000, ws, 0, None) == itc.ITC_ERR_INVALID_ARG
    assert L.itc_autotune(hp, dev, 0x4000, ws - 1, 3, None) == itc.ITC_ERR_WORKSPACE


def test_params_from_parzen_widths(L):
    """itc_params_parzen: tau = sqrt(xi^2 + omega^2), rho = sqrt(2) omega, s = sqrt(2) xi, the
    accupdate step omega^2/tau^2, and the schedule omega = sqrt(N/M)/2, xi = omega/2."""
    p = itc.params_parzen(2, xi=1.0, omega=2.0, iters=7)
    assert np.allclose(list(p.sigma)[:2], [5 ** 0.5] * 2) and np.allclose(list(p.sigma_pair)[:2], [8 ** 0.5] * 2)
    assert np.allclose(list(p.sigma_self)[:2], [2 ** 0.5] * 2) and p.step_scale == 1.0 and p.iters == 7
    p = itc.params_parzen(3, xi=(1.0, 1.0, 2.0), omega=(2.0, 2.0, 4.0), form=1)
    assert abs(p.step_scale - 0.8) < 1e-7
    p = itc.params_parzen(2, mass=400.0, M=4)
    assert np.allclose(list(p.sigma_pair)[:2], [2 ** 0.5 * 5.0] * 2) and np.allclose(list(p.sigma_self)[:2], [2 ** 0.5 * 2.5] * 2)
    out = itc.ItcParams()
    xi = (ctypes.c_float * 3)(1.0, 1.0, 0.0)
    om = (ctypes.c_float * 3)(2.0, 1.0, 0.0)
    assert L.itc_params_parzen(2, xi, om, 0.0, 0, 3.0, 0, 1, 0, ctypes.byref(out)) == itc.ITC_ERR_INVALID_ARG
    neg = (ctypes.c_float * 3)(-1.0, 1.0, 0.0)
    assert L.itc_params_parzen(2, neg, om, 0.0, 0, 3.0, 0, 0, 0, ctypes.byref(out)) == itc.ITC_ERR_INVALID_ARG
    assert L.itc_params_parzen(4, xi, om, 0.0, 0, 3.0, 0, 0, 0, ctypes.byref(out)) == itc.ITC_ERR_INVALID_ARG


def test_width_parameters_are_checked_and_classed(L):
    img = itc.ItcImage(2, 64, 64, 1, 64, itc.ITC_U8, 0x1000, None)
    fields = ctypes.c_void_p(0x2000)
    for kw, code in ((dict(sigma_pair=-1.0), itc.ITC_ERR_INVALID_ARG), (dict(sigma_self=float("nan")), itc.ITC_ERR_INVALID_ARG),
                     (dict(sigma_self=11.0), itc.ITC_ERR_UNSUPPORTED)):
        p = itc.make_params(2.0, 3.0, **kw)
        assert L.itc_fields(ctypes.byref(img), ctypes.byref(p), fields, None, 0x4000, 1 << 20, None) == code, kw
    # images whose V(X) width differs join a self-overlap class (staging 2); the workspace grows
    # by one A plane per such image
    ps = [itc.make_params(2.0), itc.make_params(2.0, sigma_self=1.5), itc.make_params(2.0, sigma_pair=3.0)]
    rc, buf, ws = _plan(L, [(64, 64), (64, 64), (64, 64)], [4, 4, 4], ps)
    assert rc == 0
    hp = ctypes.cast(buf, ctypes.c_void_p)
    assert L.itc_plan_classes(hp) == 2
    st = ctypes.c_int()
    sig = (ctypes.c_float * 3)()
    n = ctypes.c_int()
    assert L.itc_plan_class(hp, 1, None, sig, None, None, ctypes.byref(st), ctypes.byref(n), None) == 0
    assert st.value == 2 and n.value == 1 and abs(sig[0] - 1.5) < 1e-7
    rc2, _, ws2 = _plan(L, [(64, 64)] * 3, [4, 4, 4], [itc.make_params(2.0)] * 3)
    assert ws - ws2 >= 64 * 64 * 4
    assert L.itc_plan_configure(hp, 0x100000, 1, 64, 0, 0, None) == itc.ITC_ERR_UNSUPPORTED


def test_segment_rejects_invalid_arguments(L):
    rc, buf, ws = _plan(L, [(64, 64)], [8], _p())
    hp = ctypes.cast(buf, ctypes.c_void_p)
    assert L.itc_segment(hp, None, 0x1000, 0x2000, None) == itc.ITC_ERR_INVALID_ARG
    assert L.itc_segment(hp, 0x100000, None, 0x2000, None) == itc.ITC_ERR_INVALID_ARG
    assert L.itc_segment(hp, 0x100000, 0x1000, 0x2001, None) == itc.ITC_ERR_INVALID_ARG
    bogus = ctypes.create_string_buffer(len(buf.raw))
    assert L.itc_segment(ctypes.cast(bogus, ctypes.c_void_p), 0x100000, 0x1000, 0x2000, None) == itc.ITC_ERR_INVALID_ARG


def test_chamfer_checks_and_padded_layout(L):
    rc, buf, ws = _plan(L, [(10, 20), (7, 5)], [2, 2], _p())
    hp = ctypes.cast(buf, ctypes.c_void_p)
    assert L.itc_plan_padded_offset(hp, 0) == 0
    assert L.itc_plan_padded_offset(hp, 1) == 10 * 20
    assert L.itc_plan_padded_offset(hp, 2) == 10 * 20 + 7 * 8
    assert L.itc_plan_padded_offset(hp, 3) < 0
    assert L.itc_chamfer(hp, 0x100000, 0x2008, None) == itc.ITC_ERR_INVALID_ARG    # unaligned output
    assert L.itc_chamfer(hp, None, 0x2000, None) == itc.ITC_ERR_INVALID_ARG
    rc, buf, ws = _plan(L, [(16, 1100)], [2], _p())
    assert L.itc_chamfer(ctypes.cast(buf, ctypes.c_void_p), 0x100000, 0x2000, None) == itc.ITC_ERR_UNSUPPORTED
    imgs = (itc.ItcImage * 1)(itc.ItcImage(2, 16, 16, 1, 16, itc.ITC_F32, 0x10000, None))
    M = (ctypes.c_int * 1)(2)
    ps = (itc.ItcParams * 1)(_p())
    nb = L.itc_plan_bytes(1)
    b2 = ctypes.create_string_buffer(nb)
    wsz = ctypes.c_size_t(0)
    assert L.itc_plan(1, imgs, M, ps, 0, ctypes.cast(b2, ctypes.c_void_p), nb, ctypes.byref(wsz)) == 0
    assert L.itc_chamfer(ctypes.cast(b2, ctypes.c_void_p), 0x100000, 0x2000, None) == itc.ITC_ERR_INVALID_ARG


def test_recursive_flag_checks(L):
    img = itc.ItcImage(2, 64, 64, 1, 64, itc.ITC_U8, 0x1000, None)
    p = itc.make_params(40.0, 3.0, flags=itc.ITC_RECURSIVE)     # far beyond the masks, fine when recursive
    assert L.itc_fields(ctypes.byref(img), ctypes.byref(p), 0x2000, None, 0x4000, 1 << 20, None) == itc.ITC_ERR_UNSUPPORTED
    g = itc.ItcImage(3, 64, 64, 16, 64, itc.ITC_U8, 0x1000, None)
    assert L.itc_fields(ctypes.byref(g), ctypes.byref(itc.make_params((2.0, 2.0, 2.0), 3.0, flags=itc.ITC_RECURSIVE)),
                        0x2000, None, 0x4000, 1 << 20, None) == itc.ITC_ERR_UNSUPPORTED
    rc, buf, ws = _plan(L, [(64, 64), (40, 50)], [4, 4], [p, _p()])
    assert rc == 0
    hp = ctypes.cast(buf, ctypes.c_void_p)
    st = ctypes.c_int()
    assert L.itc_plan_class(hp, 0, None, None, None, None, ctypes.byref(st), None, None) == 0 and st.value == 3
    assert L.itc_backward(hp, 0x100000, 0x1000, None, None, None, None, 0x4000, ws, None) == itc.ITC_ERR_UNSUPPORTED
    assert L.itc_plan_configure(hp, 0x100000, 0, 64, 0, 0, None) == itc.ITC_ERR_UNSUPPORTED


def test_staged_run_checks_the_image_buffer(L):
    rc, buf, ws = _plan(L, [(64, 64), (40, 50)], [4, 4], _p(iters=2))
    hp = ctypes.cast(buf, ctypes.c_void_p)
    # images sit at 0x10000 and 0x20000 (see _plan); a buffer that does not hold both is refused
    assert L.itc_run_staged(hp, 0x100000, 0x1000, 0x10000, 0x8000, 0x2000, None, 0x4000, ws, 2, None, None) == itc.ITC_ERR_INVALID_ARG
    assert L.itc_run_staged(hp, 0x100000, 0x1000, 0x10000, 0x20000, 0x2000, None, 0x4000, ws, 0, None, None) == itc.ITC_ERR_INVALID_ARG
    assert L.itc_run_staged(hp, 0x100000, None, 0x10000, 0x20000, 0x2000, None, 0x4000, ws, 2, None, None) == itc.ITC_ERR_INVALID_ARG


def test_budget_workspace_query_and_checks(L):
    """itc_plan_budget_bytes: the smallest budgeted workspace holds the batch's per-tile and
    per-image words plus the fields of its largest image (here the 300 x 513 one: 3 planes of
    rows of 516 floats), far less than the whole batch's fields; larger budgets are rounded down
    to 256 bytes; the budgeted calls reject workspaces below the smallest before any launch."""
    shapes = [(64, 64), (100, 70), (300, 513), (17, 9), (200, 200)]
    rc, buf, ws = _plan(L, shapes, [8, 16, 128, 3, 32], [_p(2.0), _p(3.0), _p(2.0), _p(4.0), _p(3.0)])
    assert rc == 0
    plan = ctypes.cast(buf, ctypes.c_void_p)
    least = L.itc_plan_budget_bytes(plan, 0)
    largest = 3 * 300 * 516 * 4
    assert largest <= least < largest + (ws - sum(3 * h * ((w + 3) // 4 * 4) * 4 for h, w in shapes)) + 4096
    assert least < ws and least % 256 == 0
    assert L.itc_plan_budget_bytes(plan, least + 1000) == (least + 1000) // 256 * 256
    assert L.itc_plan_budget_bytes(plan, 10) == least
    bogus = ctypes.create_string_buffer(len(buf.raw))
    assert L.itc_plan_budget_bytes(ctypes.cast(bogus, ctypes.c_void_p), 0) == 0
    for fn in (lambda w, n: L.itc_run_budget(plan, 0x1000, 0x2000, None, w, n, None),
               lambda w, n: L.itc_backward_budget(plan, 0x1000, 0x2000, None, None, None, None, w, n, None)):
        assert fn(0x4000, least - 256) == itc.ITC_ERR_WORKSPACE
        assert fn(0x4010, least) == itc.ITC_ERR_WORKSPACE
        assert fn(None, least) == itc.ITC_ERR_WORKSPACE
