"""FP64 CPU oracle for lattice information-theoretic clustering (arXiv:1310.7114).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference legs of ``bench.py`` may import this package.  The arithmetic lives in the plain C file
``itc_oracle.c`` (FP64 throughout); this module compiles it with gcc and marshals numpy arrays
to it.  It shares no code with the CUDA library and never calls it.

Function map (paper passage each one follows):

* :func:`fields2d`, :func:`fields2d_sites`, :func:`fields3d`, :func:`fields3d_sites` -- the data
  density p = h * G and its first moments as truncated lattice sums (Sec. 3.1, Sec. 5; 3-D gray
  lattice of Sec. 1 (ii)); ``method="direct"`` is the windowed definition, ``"separable"`` the
  two- (three-) pass form.
* :func:`lattice_step`, :func:`lattice_run` -- Algorithm 1 with Eq. (origupdate)'s constant c and
  Eq. (accupdate)'s data integrals read from the fields.
* :func:`original_step`, :func:`original_run` -- Eq. (origupdate), continuous, untruncated, O(N M).
* :func:`dcs`, :func:`dcs_sums`, :func:`dcs_grad`, :func:`dcs_grad2d_dense` -- Eq. (1) and its
  gradient with respect to the codebook and to the per-pixel weights (Sec. 5).

Parity status: every function is pinned by the ``-m "not gpu"`` tests in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "itc_oracle.c")
_SO = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile ``itc_oracle.c`` into ``oracle/_build/liboracle.so`` with gcc (-O2, FP64, no fast-math)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(_SO), exist_ok=True)
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        L.orc_radius.restype = ctypes.c_int
        L.orc_radius.argtypes = [ctypes.c_double, ctypes.c_double]
        L.orc_sxx.restype = ctypes.c_double
        L.orc_dcs.restype = ctypes.c_double
        L.orc_dcs_const.restype = ctypes.c_double
        L.orc_lattice_run.restype = ctypes.c_int
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(_D)


def _i(a):
    return a.ctypes.data_as(_I)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def radius(sigma: float, trunc: float = 3.0) -> int:
    """Filter-mask half width R = ceil(trunc * sigma) (Sec. 3.1)."""
    return lib().orc_radius(float(sigma), float(trunc))


def _radii(sigma, trunc):
    return [radius(s, trunc) for s in sigma]


# ------------------------------------------------------------------------------------ fields
def fields2d(h, sigma, trunc=3.0, absolute=False, method="separable", R=None):
    """A, F_u, F_v of a 2-D weight/occupancy image ``h`` (H x W); each H x W float64."""
    h = _f64(h)
    H, W = h.shape
    su, sv = (float(sigma), float(sigma)) if np.isscalar(sigma) else map(float, sigma)
    Ru, Rv = R if R is not None else _radii((su, sv), trunc)
    A, Fu, Fv = (np.zeros((H, W)) for _ in range(3))
    fn = lib().orc_fields2d_direct if method == "direct" else lib().orc_fields2d_separable
    fn(_d(h), H, W, ctypes.c_double(su), ctypes.c_double(sv), Ru, Rv, int(absolute), _d(A), _d(Fu), _d(Fv))
    return A, Fu, Fv


def fields2d_sites(h, sigma, sites, trunc=3.0, absolute=False, R=None):
    """Fields at the listed (u, v) sites only (direct sums); returns three length-n arrays."""
    h = _f64(h)
    H, W = h.shape
    su, sv = (float(sigma), float(sigma)) if np.isscalar(sigma) else map(float, sigma)
    Ru, Rv = R if R is not None else _radii((su, sv), trunc)
    sites = _i32(sites).reshape(-1, 2)
    n = sites.shape[0]
    A, Fu, Fv = (np.zeros(n) for _ in range(3))
    lib().orc_fields2d_sites(_d(h), H, W, ctypes.c_double(su), ctypes.c_double(sv), Ru, Rv,
                             int(absolute), n, _i(sites), _d(A), _d(Fu), _d(Fv))
    return A, Fu, Fv


def fields3d(gray, G=256, sigma=(3.0, 3.0, 8.0), trunc=3.0, hw=None, absolute=False, method="separable", R=None):
    """A, F_u, F_v, F_g of the [u, v, g] occupancy volume of a gray image; each G x H x W."""
    gray = _i32(gray)
    H, W = gray.shape
    sig = _f64(sigma)
    RR = _i32(R if R is not None else _radii(sigma, trunc))
    hw_keep = _f64(hw) if hw is not None else None
    hwp = _d(hw_keep) if hw_keep is not None else None
    out = [np.zeros((G, H, W)) for _ in range(4)]
    fn = lib().orc_fields3d_direct if method == "direct" else lib().orc_fields3d_separable
    fn(_i(gray), hwp, H, W, G, _d(sig), _i(RR), int(absolute), *[_d(o) for o in out])
    return tuple(out)


def fields3d_sites(gray, sites, G=256, sigma=(3.0, 3.0, 8.0), trunc=3.0, hw=None, absolute=False, R=None):
    """3-D fields at listed (u, v, g) sites; returns four length-n arrays."""
    gray = _i32(gray)
    H, W = gray.shape
    sig = _f64(sigma)
    RR = _i32(R if R is not None else _radii(sigma, trunc))
    hw_keep = _f64(hw) if hw is not None else None
    sites = _i32(sites).reshape(-1, 3)
    n = sites.shape[0]
    out = [np.zeros(n) for _ in range(4)]
    lib().orc_fields3d_sites(_i(gray), _d(hw_keep) if hw_keep is not None else None, H, W, G, _d(sig),
                             _i(RR), int(absolute), n, _i(sites), *[_d(o) for o in out])
    return tuple(out)


def sxx(h, A) -> float:
    """S_XX = sum_x h(x) A(x) (the V(X) term of Eq. (1))."""
    h, A = _f64(h).reshape(-1), _f64(A).reshape(-1)
    return lib().orc_sxx(_d(h), _d(A), ctypes.c_size_t(h.size))


# ------------------------------------------------------------------------- fixed-point step
def segment_q(tau, ndim=2):
    """q_i = 1/tau_i^2 rounded once to float (tau taken as the float of the parameters)."""
    t = np.asarray(np.broadcast_to(np.asarray(tau, np.float32), (ndim,)), np.float64)
    return (1.0 / (t * t)).astype(np.float32)


def segment2d(h, tau, W):
    """Segmentation reading (Figs. 3, 6): label of the codebook vector whose lattice site gives the
    smallest single-precision sum_i d_i^2 / tau_i^2 (lowest index on ties); -1 where h = 0."""
    h = _f64(h)
    H, Wd = h.shape
    q = np.ascontiguousarray(segment_q(tau, 2))
    Wc = _f64(W).reshape(-1, 2)
    lab = np.zeros((H, Wd), np.int32)
    lib().orc_segment2d(_d(h), H, Wd, q.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), Wc.shape[0], _d(Wc),
                        lab.ctypes.data_as(_I))
    return lab


def segment3d(gray, tau, W, G=256, hw=None):
    """Segmentation of a gray image's [u, v, g] lattice: one label per pixel (its voxel)."""
    gray = _i32(gray)
    H, Wd = gray.shape
    q = np.ascontiguousarray(segment_q(tau, 3))
    Wc = _f64(W).reshape(-1, 3)
    hwp = _f64(hw) if hw is not None else None
    lab = np.zeros((H, Wd), np.int32)
    lib().orc_segment3d(_i(gray), _d(hwp) if hwp is not None else None, H, Wd, G,
                        q.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), Wc.shape[0], _d(Wc), lab.ctypes.data_as(_I))
    return lab


def deriche_kernel(x):
    """The damped-sinusoid fit k(x) of exp(-x^2/2), x >= 0 (Deriche)."""
    lib().orc_deriche_kernel.restype = ctypes.c_double
    return np.array([lib().orc_deriche_kernel(ctypes.c_double(float(t))) for t in np.ravel(x)])


def deriche_filter(x, sigma):
    """(sum_m x[m] g(m-n), sum_m x[m] g(m-n)(m-n)) by Deriche's recursion, zero outside the signal."""
    x = _f64(x).ravel()
    y, yd = np.zeros_like(x), np.zeros_like(x)
    lib().orc_deriche_filter(_d(x), x.size, ctypes.c_double(sigma), _d(y), _d(yd))
    return y, yd


def fields2d_recursive(h, sigma, absolute=False):
    """(A, F_u, F_v) by the recursive Gaussian (large-sigma fields, Sec. 3.1)."""
    h = _f64(h)
    H, W = h.shape
    su, sv = (float(sigma), float(sigma)) if np.isscalar(sigma) else map(float, sigma)
    A, Fu, Fv = np.zeros_like(h), np.zeros_like(h), np.zeros_like(h)
    lib().orc_fields2d_recursive(_d(h), H, W, ctypes.c_double(su), ctypes.c_double(sv), int(absolute),
                                 _d(A), _d(Fu), _d(Fv))
    return A, Fu, Fv


def chamfer34(X):
    """Sec. 5 weighting: 3-4 chamfer distance of every foreground pixel to the nearest background
    pixel (outside of the image = background), by the two raster passes; H x W int32."""
    X = np.ascontiguousarray(np.asarray(X) != 0, dtype=np.uint8)
    H, W = X.shape
    T = np.zeros((H, W), np.int32)
    lib().orc_chamfer34(X.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)), H, W, T.ctypes.data_as(_I))
    return T


def _field_ptrs(F):
    F = [_f64(f) for f in F]
    arr = (_D * len(F))(*[_d(f) for f in F])
    return F, arr


def _vec(x, ndim):
    return None if x is None else _f64(np.broadcast_to(np.asarray(x, float), (ndim,)))


def widths(xi, omega):
    """Kernel widths of Sec. 2.1 from the Parzen widths xi (data) and omega (codebook), per axis:
    tau = sqrt(xi^2 + omega^2) (V(X;W)), rho = sqrt(2) omega (V(W)), s = sqrt(2) xi (V(X)), and
    the step factor omega^2 / tau^2 at which Eq. (accupdate), evaluated exactly, moves w_k."""
    xi, omega = np.asarray(xi, float), np.asarray(omega, float)
    tau = np.sqrt(xi ** 2 + omega ** 2)
    return tau, np.sqrt(2.0) * omega, np.sqrt(2.0) * xi, omega ** 2 / tau ** 2


def dcs_const(sigma, rho=None, s=None, ndim=2):
    """Normalisers of Eq. (1) left over when tau, rho, s differ: 1/2 sum log(tau^4/(rho^2 s^2))."""
    sig = _vec(sigma, ndim)
    return float(lib().orc_dcs_const(ndim, _d(sig), _d(_vec(rho, ndim)) if rho is not None else None,
                                     _d(_vec(s, ndim)) if s is not None else None))


def lattice_step(A, F, sigma, W, step_scale=1.0, snap=True, absolute=False, rho=None):
    """One lattice ITC iteration from oracle fields (Algorithm 1 steps 4-10).

    ``A``/``F`` are 2-D (H x W) or 3-D (G x H x W) arrays; ``W`` is M x ndim; ``rho`` is the
    width of the codebook pair sums (None = sigma).  Returns ``(W_new, W_raw, stats)`` with
    stats = dict(c, sxw, sww, empty, moved).
    """
    A = _f64(A)
    ndim = len(F)
    shape = _i32([A.shape[0], A.shape[1]] if ndim == 2 else [A.shape[1], A.shape[2], A.shape[0]])
    Fk, Fp = _field_ptrs(F)
    sig = _f64(np.broadcast_to(np.asarray(sigma, float), (ndim,)))
    W = _f64(W).reshape(-1, ndim)
    M = W.shape[0]
    Wo, Wr, st = np.zeros_like(W), np.zeros_like(W), np.zeros(5)
    rh = _vec(rho, ndim)
    lib().orc_lattice_step(ndim, _i(shape), _d(A), Fp, int(absolute), _d(sig), _d(rh) if rh is not None else None,
                           M, _d(W), ctypes.c_double(step_scale), int(snap), _d(Wo), _d(Wr), _d(st))
    return Wo, Wr, dict(c=st[0], sxw=st[1], sww=st[2], empty=int(st[3]), moved=int(st[4]))


def lattice_run(A, F, sxx_value, sigma, W, iters, step_scale=1.0, snap=True, absolute=False, stop_on_fixed=False,
                rho=None, dcs_const=0.0):
    """Algorithm 1 loop; returns (W_final, dcs[0..t], tie[0..t-1], t).  ``sxx_value`` is S_XX at
    the width of V(X); ``dcs_const`` the normalisers of Eq. (1) (see :func:`dcs_const`)."""
    A = _f64(A)
    ndim = len(F)
    shape = _i32([A.shape[0], A.shape[1]] if ndim == 2 else [A.shape[1], A.shape[2], A.shape[0]])
    Fk, Fp = _field_ptrs(F)
    sig = _f64(np.broadcast_to(np.asarray(sigma, float), (ndim,)))
    W = _f64(W).reshape(-1, ndim).copy()
    M = W.shape[0]
    dcs = np.zeros(iters + 1)
    tie = np.zeros(max(iters, 1))
    rh = _vec(rho, ndim)
    t = lib().orc_lattice_run(ndim, _i(shape), _d(A), Fp, int(absolute), ctypes.c_double(sxx_value),
                              _d(sig), _d(rh) if rh is not None else None, ctypes.c_double(dcs_const), M, _d(W),
                              ctypes.c_double(step_scale), int(snap), int(iters), int(stop_on_fixed), _d(dcs),
                              _d(tie))
    return W, dcs[: t + 1], tie[:t], t


def original_step(X, sigma, W, hx=None, rho=None, kappa_from_widths=True):
    """Eq. (origupdate): one continuous, untruncated O(N M) update over the point list X (N x d);
    data sums at width sigma (tau), pair sums at rho (None = sigma).  ``kappa_from_widths``
    gives the pair terms the factor tau^2/rho^2 that differentiating Eq. (1) yields; False is the
    equation as printed (the two agree when tau = rho)."""
    X = _f64(X)
    N, ndim = X.shape
    W = _f64(W).reshape(-1, ndim)
    Wo = np.zeros_like(W)
    hk = _f64(hx) if hx is not None else None
    sig = _f64(np.broadcast_to(np.asarray(sigma, float), (ndim,)))
    rh = _vec(rho, ndim)
    lib().orc_original_step(ndim, N, _d(X), _d(hk) if hk is not None else None, _d(sig),
                            _d(rh) if rh is not None else None, int(kappa_from_widths), W.shape[0], _d(W), _d(Wo))
    return Wo


def original_run(X, sigma, W, iters, hx=None, rho=None, kappa_from_widths=True):
    W = _f64(W)
    for _ in range(iters):
        W = original_step(X, sigma, W, hx, rho, kappa_from_widths)
    return W


# -------------------------------------------------------------- divergence and its gradient
def image_points(h):
    """Point list of a 2-D weight image: (X int coords N x 2, weights N) over sites with h != 0."""
    h = np.asarray(h)
    u, v = np.nonzero(h)
    return np.stack([u, v], 1).astype(np.float64), h[u, v].astype(np.float64)


def gray_points(gray, hw=None):
    """Point list of a gray image's [u, v, g] lattice: one voxel per pixel."""
    H, W = gray.shape
    u, v = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    X = np.stack([u.ravel(), v.ravel(), gray.ravel().astype(np.int64)], 1).astype(np.float64)
    w = np.ones(H * W) if hw is None else _f64(hw).ravel()
    keep = w != 0
    return X[keep], w[keep]


def _pts(shape, X, hx, sigma, trunc, R):
    X = _f64(X)
    ndim = X.shape[1]
    sig = _f64(sigma if not np.isscalar(sigma) else [sigma] * ndim)
    RR = _i32(R if R is not None else _radii(sig, trunc))
    return X, _f64(hx), sig, RR, _i32(shape)


def _widths_args(ndim, rho, s, trunc, Rs):
    """(rho, s, Rs) ctypes arguments; None stays NULL (= sigma, sigma, R)."""
    rh, ss = _vec(rho, ndim), _vec(s, ndim)
    RRs = None
    if ss is not None:
        RRs = _i32(Rs if Rs is not None else _radii(ss, trunc))
    return ((rh, ss, RRs), (_d(rh) if rh is not None else None, _d(ss) if ss is not None else None,
                            _i(RRs) if RRs is not None else None))


def dcs_sums(shape, X, hx, sigma, W, trunc=3.0, R=None, rho=None, s=None, Rs=None):
    """(S_XW, S_WW, S_XX) from their definitions; shape = lattice sizes per axis (u, v[, g]).
    S_XW at width sigma (tau) over the box R, S_WW at rho, S_XX at s over the box Rs."""
    X, hx, sig, RR, shp = _pts(shape, X, hx, sigma, trunc, R)
    keep, wa = _widths_args(X.shape[1], rho, s, trunc, Rs)
    W = _f64(W).reshape(-1, X.shape[1])
    out = np.zeros(3)
    lib().orc_dcs_sums(X.shape[1], _i(shp), X.shape[0], _d(X), _d(hx), _d(sig), _i(RR), *wa, W.shape[0], _d(W),
                       _d(out))
    return tuple(out)


def dcs(shape, X, hx, sigma, W, trunc=3.0, R=None, rho=None, s=None, Rs=None) -> float:
    """Cauchy-Schwarz divergence, Eq. (1): log S_WW + log S_XX - 2 log S_XW + K."""
    X, hx, sig, RR, shp = _pts(shape, X, hx, sigma, trunc, R)
    keep, wa = _widths_args(X.shape[1], rho, s, trunc, Rs)
    W = _f64(W).reshape(-1, X.shape[1])
    return lib().orc_dcs(X.shape[1], _i(shp), X.shape[0], _d(X), _d(hx), _d(sig), _i(RR), *wa, W.shape[0], _d(W))


def dcs_grad(shape, X, hx, sigma, W, trunc=3.0, R=None, with_h=True, rho=None, s=None, Rs=None):
    """(dD/dW [M x d], dD/dh [N] or None) from the analytic formulas."""
    X, hx, sig, RR, shp = _pts(shape, X, hx, sigma, trunc, R)
    keep, wa = _widths_args(X.shape[1], rho, s, trunc, Rs)
    W = _f64(W).reshape(-1, X.shape[1])
    gW = np.zeros_like(W)
    gh = np.zeros(X.shape[0]) if with_h else None
    lib().orc_dcs_grad(X.shape[1], _i(shp), X.shape[0], _d(X), _d(hx), _d(sig), _i(RR), *wa, W.shape[0], _d(W),
                       _d(gW), _d(gh) if gh is not None else None)
    return gW, gh


def dcs_grad2d_dense(h, sigma, W, trunc=3.0, R=None, A=None, with_h=True, rho=None, s=None):
    """Dense-image gradient of Eq. (1): (gW [M x 2], gh [H x W] or None, (S_XW, S_WW, S_XX)).
    ``A`` is the field of h at the width s of V(X) (computed here when None)."""
    h = _f64(h)
    H, Wd = h.shape
    su, sv = (float(sigma), float(sigma)) if np.isscalar(sigma) else map(float, sigma)
    pu, pv = (su, sv) if rho is None else ((float(rho), float(rho)) if np.isscalar(rho) else map(float, rho))
    Ru, Rv = R if R is not None else _radii((su, sv), trunc)
    if A is None:
        A = fields2d(h, (su, sv) if s is None else s, trunc)[0]
    A = _f64(A)
    s_xx = sxx(h, A)
    W = _f64(W).reshape(-1, 2)
    gW = np.zeros_like(W)
    gh = np.zeros((H, Wd)) if with_h else None
    sums = np.zeros(3)
    lib().orc_dcs_grad2d_dense(_d(h), _d(A), H, Wd, ctypes.c_double(su), ctypes.c_double(sv), Ru, Rv,
                               ctypes.c_double(pu), ctypes.c_double(pv), ctypes.c_double(s_xx), W.shape[0],
                               _d(W), _d(gW), _d(gh) if gh is not None else None, _d(sums))
    return gW, gh, tuple(sums)


def dcs2d_dense(h, sigma, W, trunc=3.0, R=None, A=None, rho=None, s=None) -> float:
    """Eq. (1) for a dense 2-D weight image, from oracle fields (S_XX = sum h A_s) and the direct
    window and pair sums at the real codebook W (the same sums as :func:`dcs_sums`)."""
    _, _, (sxw, sww, s_xx) = dcs_grad2d_dense(h, sigma, W, trunc, R, A, with_h=False, rho=rho, s=s)
    return float(np.log(sww) + np.log(s_xx) - 2.0 * np.log(sxw) + dcs_const(sigma, rho, s, 2))
