"""Helpers shared by the GPU parity tests (marshalling between numpy, torch and the oracle)."""
import numpy as np

import oracle


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def radii(sigma, trunc=3.0, ndim=2):
    s = [sigma] * ndim if np.isscalar(sigma) else list(sigma)
    return [oracle.radius(x, trunc) for x in s]


def assert_fields_close(gpu, ref, R, absolute=False, what=""):
    """GPU FP32 fields vs FP64 oracle fields.

    A: |dA| <= 1e-5 A_ref, and exact zeros where the window holds no data.  The bound follows
    from the arithmetic: each A is a sum of non-negative products with FP32 taps (one rounding
    each) accumulated by two passes of 2R+1 FMAs, so its relative error is below
    (2(2R+1)+3) 2^-24 < 4e-6 for R <= 12.
    Centred moments F_i: the same products carry |x_i - y_i| <= R_i, so |dF_i| <= 1e-5 R_i A_ref.
    Absolute moments B_i (non-negative terms): relative 1e-5.
    """
    A, Aref = gpu[0], ref[0]
    assert np.all((Aref == 0) == (A == 0)), f"{what}: zero pattern of A differs"
    err = np.abs(A - Aref)
    assert np.all(err <= 1e-5 * Aref), f"{what}: A max rel err {np.max(err / np.maximum(Aref, 1e-300)):.3e}"
    for i in range(1, len(ref)):
        e = np.abs(gpu[i] - ref[i])
        tol = 1e-5 * np.abs(ref[i]) if absolute else 1e-5 * R[i - 1] * Aref
        bad = e > tol
        assert not bad.any(), f"{what}: field {i} worst {e[bad].max():.3e} vs tol {tol[bad].min():.3e} ({bad.sum()} sites)"


def half_integer_distance(raw):
    f = raw - np.floor(raw)
    return np.abs(f - 0.5)


def assert_lattice_equal_except_ties(Wg, Wref, raw, eps=1e-4, what=""):
    """Identical lattice positions except coordinates whose oracle value is within eps of a
    half-integer (a rounding tie that FP32 may resolve either way).  Returns the tie count."""
    Wg, Wref, raw = (np.asarray(x, np.float64) for x in (Wg, Wref, raw))
    ties = half_integer_distance(raw) < eps
    bad = (Wg != Wref) & ~ties
    assert not bad.any(), f"{what}: {bad.sum()} coordinates differ: gpu {Wg[bad][:6]} oracle {Wref[bad][:6]} raw {raw[bad][:6]}"
    return int(ties.sum())


def assert_grad_h_close(gh, h, A_s, sums, gh_ref, gD=1.0, c=3e-5, what=""):
    """Element-wise bound on dD/dh(x) = s1 A_s(x) - s2 S(x), s1 = 2 gD / S_XX, s2 = 2 gD / S_XW,
    S(x) = sum_k g(x - w_k) over the boxes that hold x (the transposed stamp of the codebook).

    The GPU value is the FP32 combination of FP32 terms: A_s within 1e-5 relative (the fields
    bound), S_XX and S_XW within 1e-5 relative (sums of those fields), and the stamp a sum of at
    most M non-negative products of two ex2.approx factors (2^-22 each, plus the rounding of the
    exponent and of each product and partial sum: below (M + 4) 2^-23 < 2e-5 for M <= 128).  So
    |delta| <= c (|s1 A_s| + |s2 S|) with c = 3e-5, where both terms are taken from the oracle:
    s1 A_s from A_s and S_XX, and s2 S = s1 A_s - dD/dh.  Exact zeros (pixels whose windows
    hold no data and that no box covers) must be zero."""
    gh = np.asarray(gh, np.float64)
    t1 = 2.0 * gD * np.asarray(A_s, np.float64) / sums[2]
    t2 = t1 - np.asarray(gh_ref, np.float64)
    tol = c * (np.abs(t1) + np.abs(t2))
    err = np.abs(gh - gh_ref)
    bad = err > tol
    assert not bad.any(), (f"{what}: {bad.sum()} pixels of dD/dh outside the element-wise bound, worst "
                           f"{(err[bad] / np.maximum(tol[bad], 1e-300)).max():.2f}x at {np.argwhere(bad)[:4].tolist()}")


# D = log S_WW + log S_XX - 2 log S_XW; each sum carries at most 1e-5 relative error, which is an
# absolute error of at most 1e-5 in its log, so |dD| <= (1 + 1 + 2) 1e-5.
DCS_ATOL = 4e-5


def one_iteration(p):
    """A copy of itc_params ``p`` with a single iteration (for lockstep plans)."""
    import ctypes
    from paper_1310_7114_gb300 import itc
    q = itc.ItcParams()
    ctypes.memmove(ctypes.byref(q), ctypes.byref(p), ctypes.sizeof(q))
    q.iters = 1
    return q


def plan_lockstep(images, Ms, params, W0s, iters, oracle_step, ndims=None, Gs=None, weights=None, what="lockstep"):
    """Lockstep through the batched plan itself (not through itc_step): a plan over the same
    images with one iteration per call, its fields computed once.  Every call starts each image
    from the oracle's codebooks of that iteration and must give the oracle's next codebooks
    except coordinates within 1e-4 of a half-integer.  The iteration CTAs are grouped as in the
    full run (the groups depend on M and, through the launch order, only on the images'
    relative cost, which is unchanged when every image has one iteration).
    ``oracle_step(b, W) -> (W_next, W_raw)``; ``params`` one ItcParams or one per image.
    Returns the tie count."""
    import torch
    from paper_1310_7114_gb300 import itc
    B = len(images)
    ps = [params] * B if not isinstance(params, (list, tuple)) else list(params)
    ts = [to_dev(im) for im in images]
    ws = [None if w is None else to_dev(np.asarray(w, np.float32)) for w in (weights or [None] * B)]
    plan = itc.Plan(ts, Ms, [one_iteration(p) for p in ps], ndims=ndims, Gs=Gs, weights=ws)
    itc.run_fields(plan)
    Wc = [np.asarray(w, np.float64) for w in W0s]
    ties = 0
    for t in range(iters):
        W = plan.pack_W([w.astype(np.float32) for w in Wc])
        st = itc.new_stats(B, W.device)
        itc.run_iterate(plan, W, st)
        torch.cuda.synchronize()
        got = plan.unpack_W(W)
        for b in range(B):
            Wn, raw = oracle_step(b, Wc[b])
            ties += assert_lattice_equal_except_ties(got[b], Wn, raw, what=f"{what}: image {b} iteration {t}")
            Wc[b] = Wn
    return ties


def assert_nearest_sites(X, lab, W, shape, tau, what=""):
    """Segment labels against exact arithmetic, independently of the single-precision metric
    both the kernel and the oracle evaluate: every point's codebook site is at most a few FP32
    roundings (8 u, relative) farther than the nearest under sum_i (x_i - r_i)^2 / tau_i^2, and
    where the nearest site is unique by more than that, the label is that site.  X: N x d points
    (int), lab: N labels, W: M x d codebook (sites by rounding and clamping to shape)."""
    u = 2.0 ** -24
    R = np.clip(np.floor(np.asarray(W, np.float64) + 0.5), 0, np.asarray(shape) - 1).astype(np.int64)
    t2 = np.asarray(np.broadcast_to(np.asarray(tau, np.float32), (X.shape[1],)), np.float64) ** 2
    for s in range(0, len(X), 4096):   # chunks of points: N x M metrics stay small
        Xc, lc = X[s:s + 4096].astype(np.int64), np.asarray(lab[s:s + 4096])
        d = Xc[:, None, :] - R[None, :, :]
        D = ((d * d) / t2).sum(-1)
        best = D.min(1)
        got = D[np.arange(len(Xc)), lc]
        assert np.all(got <= best * (1 + 8 * u)), f"{what}: a label farther than the nearest site"
        if D.shape[1] > 1:
            srt = np.partition(D, 1, axis=1)[:, :2]
            clear = srt[:, 1] > srt[:, 0] * (1 + 8 * u)
            assert np.all(lc[clear] == D.argmin(1)[clear]), f"{what}: not the unique nearest site"
