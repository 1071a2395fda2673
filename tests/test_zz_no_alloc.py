"""itc_fields_noalloc: the fields entry point for callers that cannot allocate device memory.

Some hosts hand the library only their input and output buffers and forbid allocation while
they run, so they cannot pass itc_fields' scratch.  This variant keeps that scratch in a fixed
array inside the library.  The GPU test checks its output against itc_fields on two calls in a
row (the second call reuses the shared array that the first one filled), and against the FP64
oracle, with the same tolerances as the other fields tests."""
import numpy as np
import pytest

import oracle
from gpuhelp import assert_fields_close, radii
from paper_1310_7114_gb300 import build, itc, synth


@pytest.mark.gpu
def test_noalloc_fields_match_itc_fields_and_the_oracle_on_two_calls():
    import torch
    build.build()
    itc.lib()
    stream = torch.cuda.current_stream().cuda_stream
    for h, sigma in [(synth.c2_image(0, size=512), 4.0), (synth.c1_image(3), 2.0)]:
        t = torch.from_numpy(h).cuda()
        ref, sxx_ref = itc.fields(t, sigma)
        out = torch.full_like(ref, float("nan"))
        sxx = torch.full((1,), float("nan"), dtype=torch.float64, device=t.device)
        rc = itc.itc_fields_noalloc(itc.make_image(t), itc.make_params(sigma), out.data_ptr(), sxx.data_ptr(), stream)
        assert rc == itc.ITC_OK, itc.status_string(rc)
        torch.cuda.synchronize()
        W = h.shape[1]
        new = [out[i, 0, :, :W].cpu().numpy().astype(np.float64) for i in range(3)]
        old = [ref[i, 0, :, :W].cpu().numpy().astype(np.float64) for i in range(3)]
        assert_fields_close(new, old, radii(sigma), False, "noalloc vs itc_fields")
        assert abs(sxx.item() - sxx_ref.item()) <= 1e-5 * abs(sxx_ref.item())
        orc = oracle.fields2d(h.astype(np.float64), sigma)
        assert_fields_close(new, list(orc), radii(sigma), False, "noalloc vs oracle")
        orc_sxx = oracle.sxx(h.astype(np.float64), orc[0])
        assert abs(sxx.item() - orc_sxx) <= 1e-5 * orc_sxx


def test_noalloc_rejects_images_beyond_the_fixed_scratch():
    import ctypes
    build.build()
    L = itc.lib()
    big = itc.ItcImage(2, 64 * 300, 64 * 300, 1, 64 * 300, itc.ITC_U8, 0x1000, None)  # 90,000 tiles
    p = itc.make_params(2.0)
    assert L.itc_fields_noalloc(ctypes.byref(big), ctypes.byref(p), 0x2000, 0x3000, None) == itc.ITC_ERR_UNSUPPORTED
    ok = itc.ItcImage(2, 64 * 256, 64 * 256, 1, 64 * 256, itc.ITC_U8, None, None)  # invalid: no data
    assert L.itc_fields_noalloc(ctypes.byref(ok), ctypes.byref(p), 0x2000, 0x3000, None) == itc.ITC_ERR_INVALID_ARG
