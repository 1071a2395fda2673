"""ctypes binding of ``libitc.so`` (declared in ``include/itc.h``).

Argument marshalling only: every step of the method runs in the library's CUDA kernels.  The
functions named ``itc_*`` are the C entry points with their C signatures; the lower-case helpers
below them build the C structs from torch tensors (device memory comes from PyTorch) and call
them on the current torch stream.  There is no CPU fallback: if the library cannot be loaded,
every call raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

from . import build as _build

ITC_OK = 0
ITC_WARN_EMPTY_SUPPORT = 1
ITC_ERR_INVALID_ARG = -1
ITC_ERR_CUDA = -2
ITC_ERR_TIMEOUT = -3
ITC_ERR_NONFINITE = -4
ITC_ERR_WORKSPACE = -5
ITC_ERR_UNSUPPORTED = -6
ITC_U8 = 0
ITC_F32 = 1
ITC_CONTINUOUS = 1
ITC_FIELDS_ABSOLUTE = 2
ITC_STOP_ON_FIXED = 4
ITC_RECURSIVE = 8
ITC_TEST_STALL_WAIT = 256

# every symbol include/itc.h declares
EXPORTS = (
    "itc_field_pitch", "itc_fields_bytes", "itc_fields_workspace_bytes", "itc_status_string",
    "itc_fields", "itc_step", "itc_plan_bytes", "itc_plan", "itc_plan_pixels", "itc_plan_offsets",
    "itc_run", "itc_run_fields", "itc_run_iterate", "itc_run_fields_range", "itc_run_iterate_range",
    "itc_run_pipelined", "itc_backward", "itc_fields_noalloc", "itc_autotune", "itc_plan_classes",
    "itc_plan_class", "itc_plan_configure", "itc_params_parzen", "itc_segment",
    "itc_plan_padded_offset", "itc_chamfer", "itc_run_staged", "itc_plan_budget_bytes", "itc_run_budget",
    "itc_backward_budget",
)


class ItcImage(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("H", ctypes.c_int), ("W", ctypes.c_int), ("G", ctypes.c_int),
                ("pitch", ctypes.c_int), ("dtype", ctypes.c_int), ("data", ctypes.c_void_p),
                ("weight", ctypes.c_void_p)]


class ItcParams(ctypes.Structure):
    _fields_ = [("sigma", ctypes.c_float * 3), ("trunc", ctypes.c_float), ("iters", ctypes.c_int),
                ("step_scale", ctypes.c_float), ("flags", ctypes.c_int), ("sigma_pair", ctypes.c_float * 3),
                ("sigma_self", ctypes.c_float * 3)]


class ItcStats(ctypes.Structure):
    _fields_ = [("dcs", ctypes.c_double), ("sxw", ctypes.c_double), ("sww", ctypes.c_double),
                ("sxx", ctypes.c_double), ("c", ctypes.c_double), ("empty", ctypes.c_int),
                ("moved", ctypes.c_int), ("iters_done", ctypes.c_int), ("status", ctypes.c_int)]


STATS_DTYPE = np.dtype([("dcs", "f8"), ("sxw", "f8"), ("sww", "f8"), ("sxx", "f8"), ("c", "f8"),
                        ("empty", "i4"), ("moved", "i4"), ("iters_done", "i4"), ("status", "i4")])
assert STATS_DTYPE.itemsize == ctypes.sizeof(ItcStats)

_lib = None
_P = ctypes.c_void_p
_SZ = ctypes.c_size_t


class ItcError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {status_string(code)} ({code})")
        self.code = code


def library_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = False) -> ctypes.CDLL:
    """Load libitc.so (raises if it is missing; the package never computes without it)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if build_if_missing:
            path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is not built (run paper_1310_7114_gb300.build.build())")
        L = ctypes.CDLL(path)
        L.itc_field_pitch.restype = ctypes.c_int
        L.itc_field_pitch.argtypes = [ctypes.c_int]
        L.itc_fields_bytes.restype = _SZ
        L.itc_fields_bytes.argtypes = [ctypes.POINTER(ItcImage)]
        L.itc_fields_workspace_bytes.restype = _SZ
        L.itc_fields_workspace_bytes.argtypes = [ctypes.POINTER(ItcImage)]
        L.itc_status_string.restype = ctypes.c_char_p
        L.itc_status_string.argtypes = [ctypes.c_int]
        L.itc_fields.restype = ctypes.c_int
        L.itc_fields.argtypes = [ctypes.POINTER(ItcImage), ctypes.POINTER(ItcParams), _P, _P, _P, _SZ, _P]
        L.itc_fields_noalloc.restype = ctypes.c_int
        L.itc_fields_noalloc.argtypes = [ctypes.POINTER(ItcImage), ctypes.POINTER(ItcParams), _P, _P, _P]
        L.itc_step.restype = ctypes.c_int
        L.itc_step.argtypes = [ctypes.POINTER(ItcImage), ctypes.POINTER(ItcParams), _P, _P, ctypes.c_int,
                               _P, _P, _P, _P, _P]
        L.itc_plan_bytes.restype = _SZ
        L.itc_plan_bytes.argtypes = [ctypes.c_int]
        L.itc_plan.restype = ctypes.c_int
        L.itc_plan.argtypes = [ctypes.c_int, ctypes.POINTER(ItcImage), ctypes.POINTER(ctypes.c_int),
                               ctypes.POINTER(ItcParams), ctypes.c_int, _P, _SZ, ctypes.POINTER(_SZ)]
        L.itc_plan_pixels.restype = _SZ
        L.itc_plan_pixels.argtypes = [_P]
        L.itc_plan_offsets.restype = ctypes.c_int
        L.itc_plan_offsets.argtypes = [_P, ctypes.c_int, ctypes.POINTER(_SZ), ctypes.POINTER(_SZ), ctypes.POINTER(_SZ)]
        L.itc_run.restype = ctypes.c_int
        L.itc_run.argtypes = [_P, _P, _P, _P, _P, _SZ, _P]
        L.itc_run_fields.restype = ctypes.c_int
        L.itc_run_fields.argtypes = [_P, _P, _P, _SZ, _P]
        L.itc_run_iterate.restype = ctypes.c_int
        L.itc_run_iterate.argtypes = [_P, _P, _P, _P, _P, _SZ, _P]
        L.itc_run_fields_range.restype = ctypes.c_int
        L.itc_run_fields_range.argtypes = [_P, _P, ctypes.c_int, ctypes.c_int, _P, _SZ, _P]
        L.itc_run_iterate_range.restype = ctypes.c_int
        L.itc_run_iterate_range.argtypes = [_P, _P, ctypes.c_int, ctypes.c_int, _P, _P, _P, _SZ, _P]
        L.itc_run_pipelined.restype = ctypes.c_int
        L.itc_run_pipelined.argtypes = [_P, _P, _P, _P, _P, _SZ, _P, _P, ctypes.c_int]
        L.itc_autotune.restype = ctypes.c_int
        L.itc_autotune.argtypes = [_P, _P, _P, _SZ, ctypes.c_int, _P]
        L.itc_run_staged.restype = ctypes.c_int
        L.itc_run_staged.argtypes = [_P, _P, _P, _P, _SZ, _P, _P, _P, _SZ, ctypes.c_int, _P, _P]
        L.itc_plan_padded_offset.restype = ctypes.c_longlong
        L.itc_plan_padded_offset.argtypes = [_P, ctypes.c_int]
        L.itc_chamfer.restype = ctypes.c_int
        L.itc_chamfer.argtypes = [_P, _P, _P, _P]
        L.itc_segment.restype = ctypes.c_int
        L.itc_segment.argtypes = [_P, _P, _P, _P, _P]
        L.itc_params_parzen.restype = ctypes.c_int
        L.itc_params_parzen.argtypes = [ctypes.c_int, _P, _P, ctypes.c_double, ctypes.c_int, ctypes.c_float,
                                        ctypes.c_int, ctypes.c_int, ctypes.c_int, _P]
        L.itc_plan_configure.restype = ctypes.c_int
        L.itc_plan_configure.argtypes = [_P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P]
        L.itc_plan_classes.restype = ctypes.c_int
        L.itc_plan_classes.argtypes = [_P]
        _I = ctypes.POINTER(ctypes.c_int)
        _F = ctypes.POINTER(ctypes.c_float)
        L.itc_plan_class.restype = ctypes.c_int
        L.itc_plan_class.argtypes = [_P, ctypes.c_int, _I, _F, _I, _I, _I, _I, _F]
        L.itc_backward.restype = ctypes.c_int
        L.itc_backward.argtypes = [_P, _P, _P, _P, _P, _P, _P, _P, _SZ, _P]
        L.itc_plan_budget_bytes.restype = _SZ
        L.itc_plan_budget_bytes.argtypes = [_P, _SZ]
        L.itc_run_budget.restype = ctypes.c_int
        L.itc_run_budget.argtypes = [_P, _P, _P, _P, _P, _SZ, _P]
        L.itc_backward_budget.restype = ctypes.c_int
        L.itc_backward_budget.argtypes = [_P, _P, _P, _P, _P, _P, _P, _P, _SZ, _P]
        _lib = L
    return _lib


def status_string(code: int) -> str:
    return lib().itc_status_string(int(code)).decode()


def _check(rc: int, what: str) -> int:
    if rc < 0:
        raise ItcError(rc, what)
    return rc


# ----------------------------------------------------------------------------- torch marshalling
def _torch():
    import torch
    return torch


def _ptr(t) -> Optional[int]:
    return None if t is None else t.data_ptr()


def _stream(stream=None) -> int:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _width3(x, fill):
    if x is None:
        return [0.0] * 3
    return [float(x)] * 3 if np.isscalar(x) else [float(v) for v in x] + [fill] * (3 - len(x))


def make_params(sigma, trunc: float = 3.0, iters: int = 0, step_scale: float = 1.0, flags: int = 0,
                sigma_pair=None, sigma_self=None) -> ItcParams:
    """itc_params; ``sigma_pair`` (rho) and ``sigma_self`` (s) default to sigma (stored as 0)."""
    s = _width3(sigma, 1.0)
    return ItcParams((ctypes.c_float * 3)(*s), float(trunc), int(iters), float(step_scale), int(flags),
                     (ctypes.c_float * 3)(*_width3(sigma_pair, 0.0)), (ctypes.c_float * 3)(*_width3(sigma_self, 0.0)))


def params_parzen(ndim: int, xi=None, omega=None, mass: float = 0.0, M: int = 0, trunc: float = 3.0,
                  iters: int = 0, form: int = 0, flags: int = 0) -> ItcParams:
    """itc_params_parzen: parameters from the Parzen widths (xi, omega) or, with mass and M, from
    the schedule omega = sqrt(mass/M)/2, xi = omega/2."""
    def arr(x):
        if x is None:
            return None
        v = [float(x)] * ndim if np.isscalar(x) else [float(t) for t in x]
        return (ctypes.c_float * 3)(*(v + [0.0] * (3 - len(v))))
    out = ItcParams()
    _check(lib().itc_params_parzen(int(ndim), arr(xi), arr(omega), ctypes.c_double(mass), int(M), ctypes.c_float(trunc),
                                   int(iters), int(form), int(flags), ctypes.byref(out)), "itc_params_parzen")
    return out


def make_image(data, ndim: int = 2, G: int = 1, weight=None) -> ItcImage:
    """Descriptor of a device tensor: 2-D uint8 occupancy / float32 weights, or (ndim 3) uint8 gray."""
    torch = _torch()
    if data.dim() != 2 or data.stride(1) != 1 or not data.is_cuda:
        raise ValueError("image must be a 2-D CUDA tensor with unit column stride")
    dt = ITC_U8 if data.dtype == torch.uint8 else (ITC_F32 if data.dtype == torch.float32 else None)
    if dt is None:
        raise ValueError("image dtype must be uint8 or float32")
    if weight is not None and (weight.dtype != torch.float32 or weight.stride(0) != data.stride(0)):
        raise ValueError("weight must be float32 with the image's row pitch")
    H, W = data.shape
    return ItcImage(int(ndim), int(H), int(W), int(G if ndim == 3 else 1), int(data.stride(0)), dt,
                    data.data_ptr(), _ptr(weight))


def field_pitch(W: int) -> int:
    return lib().itc_field_pitch(int(W))


def itc_fields(img: ItcImage, p: ItcParams, fields_ptr, sxx_ptr, ws_ptr, ws_bytes, stream):
    return lib().itc_fields(ctypes.byref(img), ctypes.byref(p), fields_ptr, sxx_ptr, ws_ptr, ws_bytes, stream)


def itc_fields_noalloc(img: ItcImage, p: ItcParams, fields_ptr, sxx_ptr, stream):
    return lib().itc_fields_noalloc(ctypes.byref(img), ctypes.byref(p), fields_ptr, sxx_ptr, stream)


def itc_step(img, p, fields_ptr, sxx_ptr, M, W_in, W_out, W_lat, stats, stream):
    return lib().itc_step(ctypes.byref(img), ctypes.byref(p), fields_ptr, sxx_ptr, int(M), W_in, W_out, W_lat,
                          stats, stream)


def itc_run(plan_host, plan_dev, W, stats, ws, ws_bytes, stream):
    return lib().itc_run(plan_host, plan_dev, W, stats, ws, ws_bytes, stream)


def itc_backward(plan_host, plan_dev, W, grad_dcs, grad_W, grad_h, stats, ws, ws_bytes, stream):
    return lib().itc_backward(plan_host, plan_dev, W, grad_dcs, grad_W, grad_h, stats, ws, ws_bytes, stream)


def stats_to_numpy(t) -> np.ndarray:
    """Copy a device stats buffer (uint8 tensor of n * sizeof(itc_stats)) to a numpy record array."""
    return np.frombuffer(t.cpu().numpy().tobytes(), dtype=STATS_DTYPE)


def fields(data, sigma, trunc: float = 3.0, absolute: bool = False, ndim: int = 2, G: int = 1, weight=None,
           stream=None, sigma_self=None):
    """Fields of one image; returns (fields [nf, G, H, fpitch] float32, S_XX float64 tensor [1]).
    S_XX is taken at ``sigma_self`` (the width of V(X)) when given."""
    torch = _torch()
    img = make_image(data, ndim, G, weight)
    p = make_params(sigma, trunc, flags=ITC_FIELDS_ABSOLUTE if absolute else 0, sigma_self=sigma_self)
    nbytes = lib().itc_fields_bytes(ctypes.byref(img))
    if nbytes == 0:
        raise ItcError(ITC_ERR_INVALID_ARG, "itc_fields_bytes")
    wsb = lib().itc_fields_workspace_bytes(ctypes.byref(img))
    dev = data.device
    out = torch.empty(nbytes // 4, dtype=torch.float32, device=dev)
    ws = torch.empty(max(wsb, 256), dtype=torch.uint8, device=dev)
    sxx = torch.empty(1, dtype=torch.float64, device=dev)
    _check(itc_fields(img, p, out.data_ptr(), sxx.data_ptr(), ws.data_ptr(), ws.numel(), _stream(stream)),
           "itc_fields")
    nf = ndim + 1
    return out.view(nf, img.G, img.H, field_pitch(img.W)), sxx


def step(data, fields_t, sxx, W, sigma, trunc: float = 3.0, step_scale: float = 1.0, flags: int = 0,
         ndim: int = 2, G: int = 1, weight=None, stream=None, sigma_pair=None, sigma_self=None):
    """One update (itc_step); returns (W_out float32 [M, d], W_lattice int32 [M, d], stats record)."""
    torch = _torch()
    img = make_image(data, ndim, G, weight)
    p = make_params(sigma, trunc, 1, step_scale, flags, sigma_pair=sigma_pair, sigma_self=sigma_self)
    W = W.contiguous()
    M = W.shape[0]
    Wo = torch.empty_like(W)
    Wl = torch.empty(W.shape, dtype=torch.int32, device=W.device)
    st = torch.empty(ctypes.sizeof(ItcStats), dtype=torch.uint8, device=W.device)
    _check(itc_step(img, p, fields_t.data_ptr(), sxx.data_ptr(), M, W.data_ptr(), Wo.data_ptr(), Wl.data_ptr(),
                    st.data_ptr(), _stream(stream)), "itc_step")
    return Wo, Wl, st


class Plan:
    """A batch plan (itc_plan) with its host blob, device copy and workspace.

    images: list of 2-D CUDA tensors (uint8 occupancy, float32 weights, or uint8 gray for ndim 3)
    M: codebook count per image; params: one ItcParams or one per image; ndims / Gs / weights: per
    image (defaults 2 / 1 / None).
    """

    def __init__(self, images: Sequence, M: Sequence[int], params, ndims=None, Gs=None, weights=None,
                 device=None, allocate_ws: bool = True):
        torch = _torch()
        B = len(images)
        ndims = list(ndims) if ndims is not None else [2] * B
        Gs = list(Gs) if Gs is not None else [1] * B
        weights = list(weights) if weights is not None else [None] * B
        self.B = B
        self.ndims = ndims
        self._G = Gs
        self.M = [int(m) for m in M]
        self.shapes = [tuple(im.shape) for im in images]
        imgs = (ItcImage * B)(*[make_image(images[b], ndims[b], Gs[b], weights[b]) for b in range(B)])
        Ms = (ctypes.c_int * B)(*self.M)
        if isinstance(params, ItcParams):
            ps, stride = (ItcParams * 1)(params), 0
        else:
            ps, stride = (ItcParams * B)(*params), 1
        nbytes = lib().itc_plan_bytes(B)
        self.host = ctypes.create_string_buffer(nbytes)
        ws = _SZ(0)
        _check(lib().itc_plan(B, imgs, Ms, ps, stride, ctypes.cast(self.host, _P), nbytes, ctypes.byref(ws)),
               "itc_plan")
        dev = device if device is not None else images[0].device
        blob = np.frombuffer(self.host.raw, dtype=np.uint8)
        self.dev = torch.from_numpy(blob.copy()).to(dev)
        self.ws_bytes = int(ws.value)
        # the whole batch's fields; a plan used only through the budgeted calls needs none of it
        self.ws = torch.empty(max(self.ws_bytes, 256), dtype=torch.uint8, device=dev) if allocate_ws else None
        self.pixels = int(lib().itc_plan_pixels(ctypes.cast(self.host, _P)))
        self.w_offsets = np.concatenate([[0], np.cumsum([m * d for m, d in zip(self.M, ndims)])]).astype(np.int64)
        self.gh_offsets = np.concatenate([[0], np.cumsum([h * w for h, w in self.shapes])]).astype(np.int64)
        self._keep = (images, weights)

    @property
    def host_ptr(self):
        return ctypes.cast(self.host, _P)

    def budget_bytes(self, budget_bytes: int = 0) -> int:
        """itc_plan_budget_bytes: workspace of the budgeted calls within ``budget_bytes`` in all
        (raised to the smallest they accept; 0 gives that smallest)."""
        return int(lib().itc_plan_budget_bytes(self.host_ptr, int(budget_bytes)))

    def offsets(self, b: int):
        """(field byte offset in ws, W float offset, grad_h float offset) of image b (itc_plan_offsets)."""
        f, w, g = _SZ(0), _SZ(0), _SZ(0)
        _check(lib().itc_plan_offsets(self.host_ptr, int(b), ctypes.byref(f), ctypes.byref(w), ctypes.byref(g)),
               "itc_plan_offsets")
        return int(f.value), int(w.value), int(g.value)

    def autotune(self, reps: int = 3, stream=None):
        """itc_autotune: time the fields configurations per class and keep the fastest (updates both
        plan copies; overwrites the workspace)."""
        _check(lib().itc_autotune(self.host_ptr, self.dev.data_ptr(), self.ws.data_ptr(), self.ws.numel(), int(reps),
                                  _stream(stream)), "itc_autotune")
        return self.classes()

    def configure(self, c: int, tile_h: int, ctas_per_sm: int = 0, staging: str = "tma", stream=None):
        """itc_plan_configure: pin class c's fields configuration."""
        _check(lib().itc_plan_configure(self.host_ptr, self.dev.data_ptr(), int(c), int(tile_h), int(ctas_per_sm),
                                        1 if staging == "tma" else 0, _stream(stream)), "itc_plan_configure")

    def classes(self):
        """Configuration of every parameter class (itc_plan_class)."""
        out = []
        for c in range(lib().itc_plan_classes(self.host_ptr)):
            nd, th, gp, st, ni = (ctypes.c_int() for _ in range(5))
            sig, ms = (ctypes.c_float * 3)(), ctypes.c_float()
            _check(lib().itc_plan_class(self.host_ptr, c, ctypes.byref(nd), sig, ctypes.byref(th), ctypes.byref(gp),
                                        ctypes.byref(st), ctypes.byref(ni), ctypes.byref(ms)), "itc_plan_class")
            out.append(dict(ndim=nd.value, sigma=[round(x, 4) for x in sig[:nd.value]], tile_h=th.value,
                            ctas_per_sm=gp.value, staging={0: "plain", 1: "tma", 2: "self", 3: "recursive"}[st.value], images=ni.value,
                            tuned_ms=ms.value))
        return out

    def fields_of(self, b: int):
        """View of image b's fields inside the workspace: [ndim+1, G, H, fpitch] float32."""
        f, _, _ = self.offsets(b)
        H, W = self.shapes[b]
        G = self._G[b] if self.ndims[b] == 3 else 1
        n = (self.ndims[b] + 1) * G * H * field_pitch(W)
        return self.ws[f:f + 4 * n].view(_torch().float32).view(self.ndims[b] + 1, G, H, field_pitch(W))

    def pack_W(self, Ws: Sequence) -> "object":
        """Concatenate per-image codebooks ([M_b, d_b] arrays) into the plan's ragged device layout."""
        torch = _torch()
        flat = np.concatenate([np.asarray(w, np.float32).reshape(-1) for w in Ws])
        return torch.from_numpy(flat).to(self.dev.device)

    def unpack_W(self, flat) -> list:
        a = flat.detach().cpu().numpy() if hasattr(flat, "detach") else np.asarray(flat)
        return [a[self.w_offsets[b]:self.w_offsets[b + 1]].reshape(self.M[b], self.ndims[b]) for b in range(self.B)]

    def unpack_pixels(self, flat) -> list:
        a = flat.detach().cpu().numpy() if hasattr(flat, "detach") else np.asarray(flat)
        return [a[self.gh_offsets[b]:self.gh_offsets[b + 1]].reshape(self.shapes[b]) for b in range(self.B)]


def run(plan: Plan, W, stats=None, stream=None):
    """itc_run on a plan: W (ragged device float32) is updated in place; stats (uint8 device buffer
    of B * sizeof(itc_stats)) receives the per-image results."""
    _check(itc_run(plan.host_ptr, plan.dev.data_ptr(), W.data_ptr(), _ptr(stats), plan.ws.data_ptr(),
                   plan.ws.numel(), _stream(stream)), "itc_run")
    return W


def chamfer(plan: Plan, out=None, stream=None, views: bool = True):
    """itc_chamfer: the Sec. 5 weights of every binary image of the plan; returns (buffer, list of
    [H, W] float32 views with rows of field_pitch(W) floats, ready to be the images of a weighted
    plan; None with views=False)."""
    torch = _torch()
    if out is None:
        total = int(lib().itc_plan_padded_offset(plan.host_ptr, plan.B))
        out = torch.zeros(max(total, 4), dtype=torch.float32, device=plan.dev.device)
    _check(lib().itc_chamfer(plan.host_ptr, plan.dev.data_ptr(), out.data_ptr(), _stream(stream)), "itc_chamfer")
    if not views:
        return out, None
    views = []
    for b, (H, W) in enumerate(plan.shapes):
        o = int(lib().itc_plan_padded_offset(plan.host_ptr, b))
        fp = field_pitch(W)
        views.append(out[o:o + H * fp].view(H, fp)[:, :W])
    return out, views


def segment(plan: Plan, W, labels=None, stream=None):
    """itc_segment: int16 label per pixel (plan.pixels, image b at its pixel offset), -1 without data."""
    torch = _torch()
    if labels is None:
        labels = torch.empty(plan.pixels, dtype=torch.int16, device=W.device)
    _check(lib().itc_segment(plan.host_ptr, plan.dev.data_ptr(), W.data_ptr(), labels.data_ptr(), _stream(stream)),
           "itc_segment")
    return labels


def run_staged(plan: Plan, host_buf, dev_buf, W, stats=None, chunks: int = 8, stream=None, copy_stream=None):
    """itc_run_staged: copy the images from the pinned host tensor ``host_buf`` into ``dev_buf``
    (the buffer the plan's images live in) range by range on ``copy_stream`` while the fields and
    iterations of the ranges already copied run on ``stream``."""
    nbytes = dev_buf.numel() * dev_buf.element_size()
    if host_buf.numel() * host_buf.element_size() != nbytes:
        raise ValueError("host and device image buffers differ in size")
    _check(lib().itc_run_staged(plan.host_ptr, plan.dev.data_ptr(), host_buf.data_ptr(), dev_buf.data_ptr(), nbytes,
                                W.data_ptr(), _ptr(stats), plan.ws.data_ptr(), plan.ws.numel(), int(chunks),
                                _stream(stream), _stream(copy_stream) if copy_stream is not None else None),
           "itc_run_staged")


def run_fields(plan: Plan, stream=None):
    """itc_run_fields: the fields pass of itc_run alone."""
    _check(lib().itc_run_fields(plan.host_ptr, plan.dev.data_ptr(), plan.ws.data_ptr(), plan.ws.numel(),
                                _stream(stream)), "itc_run_fields")


def run_iterate(plan: Plan, W, stats=None, stream=None):
    """itc_run_iterate: the iterations of itc_run on the fields already in the workspace."""
    _check(lib().itc_run_iterate(plan.host_ptr, plan.dev.data_ptr(), W.data_ptr(), _ptr(stats), plan.ws.data_ptr(),
                                 plan.ws.numel(), _stream(stream)), "itc_run_iterate")
    return W


def run_pipelined(plan: Plan, W, stats=None, stream2=None, chunks: int = 4, stream=None):
    """itc_run_pipelined: fields of image range k+1 overlap the iterations of range k on stream2."""
    torch = _torch()
    s2 = stream2 if stream2 is not None else torch.cuda.Stream(device=W.device)
    _check(lib().itc_run_pipelined(plan.host_ptr, plan.dev.data_ptr(), W.data_ptr(), _ptr(stats), plan.ws.data_ptr(),
                                   plan.ws.numel(), _stream(stream), s2.cuda_stream, int(chunks)), "itc_run_pipelined")
    return W


def backward(plan: Plan, W, grad_dcs=None, grad_W=None, grad_h=None, stats=None, stream=None):
    """itc_backward on a plan (after itc_run on the same plan filled the workspace fields)."""
    _check(itc_backward(plan.host_ptr, plan.dev.data_ptr(), W.data_ptr(), _ptr(grad_dcs), _ptr(grad_W),
                        _ptr(grad_h), _ptr(stats), plan.ws.data_ptr(), plan.ws.numel(), _stream(stream)),
           "itc_backward")
    return grad_W, grad_h


def budget_workspace(plan: Plan, budget_bytes: int = 0):
    """A device workspace for the budgeted calls, of itc_plan_budget_bytes(plan, budget_bytes)."""
    return _torch().empty(plan.budget_bytes(budget_bytes), dtype=_torch().uint8, device=plan.dev.device)


def run_budget(plan: Plan, W, ws, stats=None, stream=None):
    """itc_run_budget: itc_run with the fields recomputed range by range inside ``ws``."""
    _check(lib().itc_run_budget(plan.host_ptr, plan.dev.data_ptr(), W.data_ptr(), _ptr(stats), ws.data_ptr(),
                                ws.numel(), _stream(stream)), "itc_run_budget")
    return W


def backward_budget(plan: Plan, W, ws, grad_dcs=None, grad_W=None, grad_h=None, stats=None, stream=None):
    """itc_backward_budget: the gradient with A and S_XX recomputed range by range inside ``ws``."""
    _check(lib().itc_backward_budget(plan.host_ptr, plan.dev.data_ptr(), W.data_ptr(), _ptr(grad_dcs),
                                     _ptr(grad_W), _ptr(grad_h), _ptr(stats), ws.data_ptr(), ws.numel(),
                                     _stream(stream)), "itc_backward_budget")
    return grad_W, grad_h


def new_stats(n: int, device):
    torch = _torch()
    return torch.zeros(n * ctypes.sizeof(ItcStats), dtype=torch.uint8, device=device)


def pack_images(images: Sequence[np.ndarray], device, align: int = 16):
    """Copy host images into one device buffer, rows padded to ``align`` elements and every image
    starting on a 256-byte boundary; returns (buffer, list of 2-D strided views)."""
    torch = _torch()
    dtype = images[0].dtype
    esize = np.dtype(dtype).itemsize
    offs, views, total = [], [], 0
    for im in images:
        H, W = im.shape
        pitch = (W + align - 1) // align * align
        total = (total + 255) // 256 * 256
        offs.append((total, H, W, pitch))
        total += H * pitch * esize
    host = np.zeros(max(total, 1) // esize + 1, dtype=dtype)
    for (o, H, W, pitch), im in zip(offs, images):
        host[o // esize: o // esize + H * pitch].reshape(H, pitch)[:, :W] = im
    buf = torch.from_numpy(host).to(device)
    for (o, H, W, pitch) in offs:
        views.append(buf[o // esize: o // esize + H * pitch].view(H, pitch)[:, :W])
    return buf, views
