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


# D = log S_WW + log S_XX - 2 log S_XW; each sum carries at most 1e-5 relative error, which is an
# absolute error of at most 1e-5 in its log, so |dD| <= (1 + 1 + 2) 1e-5.
DCS_ATOL = 4e-5
