"""Pins of the oracle with separate kernel widths (xi for the data, omega for the codebook).

By the Gaussian product theorem (Sec. 2.1) the overlap integrals of Eq. (1) are Gaussian sums of
widths tau^2 = xi^2 + omega^2 (V(X;W)), rho^2 = 2 omega^2 (V(W)) and s^2 = 2 xi^2 (V(X)).  The
oracle's sums with the three widths and the normalising constant K are checked against dense
numerical quadrature of the normalised Parzen densities (Eq. (dens1)/(dens2)), for isotropic and
per-axis widths; Eq. (accupdate) evaluated by quadrature is checked against the oracle's
update, which pins both the step factor omega^2/tau^2 and the pair factor tau^2/rho^2 that
differentiating Eq. (1) gives (and that Eq. (origupdate) as printed lacks); the analytic
gradient is checked against central differences; a fixed point of the update is a stationary
point of D_cs; the lattice step on exact fields equals the continuous update at lattice W.
"""
import math

import numpy as np
import pytest

import oracle

PTS = np.array([[12.0, 12.0], [13.0, 15.0], [16.0, 13.0], [15.0, 16.0], [11.0, 17.0]])
HX = np.array([1.0, 0.6, 0.8, 0.3, 0.9])
W0 = np.array([[13.0, 13.0], [15.0, 15.0], [12.0, 16.0]])
SHAPE = (30, 30)
CASES = [((0.7, 0.7), (1.3, 1.3)), ((1.1, 1.1), (0.6, 0.6)), ((0.8, 1.2), (1.4, 0.9))]


def _grid(lo=-2.0, hi=30.0, step=0.02):
    t = np.arange(lo, hi, step)
    return np.meshgrid(t, t, indexing="ij")


def _G(U, V, c, s):
    """Normalised 2-D Gaussian with per-axis widths s at centre c."""
    return (np.exp(-(U - c[0]) ** 2 / (2 * s[0] ** 2) - (V - c[1]) ** 2 / (2 * s[1] ** 2))
            / (2 * np.pi * s[0] * s[1]))


def _densities(U, V, xi, om, W):
    p = sum(w * _G(U, V, x, xi) for x, w in zip(PTS, HX)) / HX.sum()
    q = sum(_G(U, V, w, om) for w in W) / len(W)
    return p, q


@pytest.mark.parametrize("xi,om", CASES)
def test_dcs_with_three_widths_equals_quadrature(xi, om):
    U, V = _grid()
    p, q = _densities(U, V, xi, om, W0)
    d_quad = -2 * math.log((p * q).sum()) + math.log((q * q).sum()) + math.log((p * p).sum())
    tau, rho, s, _ = oracle.widths(xi, om)
    d_orc = oracle.dcs(SHAPE, PTS, HX, tau, W0, R=(29, 29), rho=rho, s=s, Rs=(29, 29))
    assert abs(d_quad - d_orc) < 1e-9, (d_quad, d_orc)


def test_equal_widths_reduce_to_one_sigma():
    tau, rho, s, step = oracle.widths(0.9, 0.9)
    assert np.allclose(tau, rho) and np.allclose(tau, s) and abs(step - 0.5) < 1e-15
    assert abs(oracle.dcs_const(tau, rho, s)) < 1e-14
    a = oracle.dcs(SHAPE, PTS, HX, tau, W0, R=(8, 8))
    b = oracle.dcs(SHAPE, PTS, HX, tau, W0, R=(8, 8), rho=rho, s=s, Rs=(8, 8))
    assert abs(a - b) < 1e-12
    # K >= 0 (AM-GM on tau^4 = (xi^2 + omega^2)^2 >= 4 xi^2 omega^2), zero only for xi = omega
    for xi, om in CASES:
        t, r, ss, _ = oracle.widths(xi, om)
        assert oracle.dcs_const(t, r, ss) > 0


@pytest.mark.parametrize("xi,om", CASES)
def test_accupdate_by_quadrature_equals_oracle_update(xi, om):
    """Eq. (accupdate) with every integral done numerically against the oracle's continuous
    untruncated update at step omega^2/tau^2 with pair factor tau^2/rho^2."""
    U, V = _grid()
    p, q = _densities(U, V, xi, om, W0)
    c = (p * q).sum() / (q * q).sum()
    om = np.asarray(om)
    want = np.zeros_like(W0)
    for k, w in enumerate(W0):
        gk = _G(U, V, w, om)
        den = (p * gk).sum()
        for i, X in enumerate((U, V)):
            want[k, i] = ((p * gk * X).sum() - c * (q * gk * X).sum() + c * (q * gk).sum() * w[i]) / den
    tau, rho, s, step = oracle.widths(xi, om)
    full = oracle.original_step(PTS, tau, W0, HX, rho=rho, kappa_from_widths=True)
    got = W0 + step * (full - W0)
    assert np.abs(got - want).max() < 1e-9, np.abs(got - want).max()
    if not np.allclose(tau, rho):
        printed = oracle.original_step(PTS, tau, W0, HX, rho=rho, kappa_from_widths=False)
        assert np.abs(W0 + step * (printed - W0) - want).max() > 1e-3


@pytest.mark.parametrize("xi,om", CASES)
def test_gradient_with_three_widths_matches_central_differences(xi, om):
    tau, rho, s, _ = oracle.widths(xi, om)
    W = W0 + np.array([[0.2, -0.1], [0.1, 0.3], [-0.2, 0.1]])   # real W inside its lattice cells
    kw = dict(R=(6, 6), rho=rho, s=s, Rs=(5, 5))
    gW, gh = oracle.dcs_grad(SHAPE, PTS, HX, tau, W, **kw)
    e = 1e-5
    for k in range(len(W)):
        for i in range(2):
            Wp, Wm = W.copy(), W.copy()
            Wp[k, i] += e
            Wm[k, i] -= e
            fd = (oracle.dcs(SHAPE, PTS, HX, tau, Wp, **kw) - oracle.dcs(SHAPE, PTS, HX, tau, Wm, **kw)) / (2 * e)
            assert abs(fd - gW[k, i]) < 1e-7 * max(1.0, abs(fd)), (k, i, fd, gW[k, i])
    for n in range(len(PTS)):
        hp, hm = HX.copy(), HX.copy()
        hp[n] += e
        hm[n] -= e
        fd = (oracle.dcs(SHAPE, PTS, hp, tau, W, **kw) - oracle.dcs(SHAPE, PTS, hm, tau, W, **kw)) / (2 * e)
        assert abs(fd - gh[n]) < 1e-7 * max(1.0, abs(fd)), (n, fd, gh[n])


@pytest.mark.parametrize("xi,om", CASES)
def test_fixed_point_of_the_update_is_stationary(xi, om):
    """Iterating the update with the derived pair factor ends where dD/dW = 0; with the factor
    as printed in Eq. (origupdate) it does not (unless tau = rho)."""
    tau, rho, s, _ = oracle.widths(xi, om)
    kw = dict(R=(29, 29), rho=rho, s=s, Rs=(29, 29))
    W = oracle.original_run(PTS, tau, W0, 400, HX, rho=rho, kappa_from_widths=True)
    gW, _ = oracle.dcs_grad(SHAPE, PTS, HX, tau, W, with_h=False, **kw)
    assert np.abs(gW).max() < 1e-8, np.abs(gW).max()
    Wp = oracle.original_run(PTS, tau, W0, 400, HX, rho=rho, kappa_from_widths=False)
    gP, _ = oracle.dcs_grad(SHAPE, PTS, HX, tau, Wp, with_h=False, **kw)
    if not np.allclose(tau, rho):
        assert np.abs(gP).max() > 1e-4


@pytest.mark.parametrize("xi,om", CASES)
def test_lattice_step_on_exact_fields_equals_continuous_update(xi, om):
    """At lattice W with windows covering the whole image, the lattice step (fields at tau,
    pair sums at rho, no rounding) is the continuous update."""
    tau, rho, s, step = oracle.widths(xi, om)
    h = np.zeros(SHAPE)
    for (u, v), w in zip(PTS, HX):
        h[int(u), int(v)] = w
    A, Fu, Fv = oracle.fields2d(h, tau, R=(29, 29))
    Wn, raw, st = oracle.lattice_step(A, (Fu, Fv), tau, W0, step_scale=float(np.mean(step)), snap=False, rho=rho)
    if np.ptp(step) == 0:
        full = oracle.original_step(PTS, tau, W0, HX, rho=rho, kappa_from_widths=True)
        assert np.abs(raw - (W0 + step[0] * (full - W0))).max() < 1e-10
    sxw, sww, _ = oracle.dcs_sums(SHAPE, PTS, HX, tau, W0, R=(29, 29), rho=rho)
    assert abs(st["sxw"] - sxw) < 1e-12 * sxw and abs(st["sww"] - sww) < 1e-12 * sww


def test_lattice_run_dcs_includes_the_constant():
    xi, om = (0.9, 0.9), (1.5, 1.5)
    tau, rho, s, step = oracle.widths(xi, om)
    h = np.zeros(SHAPE)
    for (u, v), w in zip(PTS, HX):
        h[int(u), int(v)] = w
    A, Fu, Fv = oracle.fields2d(h, tau, R=(29, 29))
    As = oracle.fields2d(h, s, R=(29, 29))[0]
    K = oracle.dcs_const(tau, rho, s)
    W, d, _, t = oracle.lattice_run(A, (Fu, Fv), oracle.sxx(h, As), tau, W0, 3, step_scale=float(step[0]),
                                    rho=rho, dcs_const=K)
    want = oracle.dcs(SHAPE, PTS, HX, tau, W, R=(29, 29), rho=rho, s=s, Rs=(29, 29))
    assert abs(d[t] - want) < 1e-10
