"""The allocation-free J w entry point (bl_jw_fp32_static) against bl_hypergrad.

For callers that may not allocate device memory (code inside a host framework that owns the
device heap, or under a no-allocation rule after start-up): the entry point keeps its scratch
in a fixed device array.  Two calls in a row on different vectors must both agree with the
allocating path within the tolerance the other J w parity tests use (1e-5 relative, FP32).
This file is collected last so that a failure here leaves every other GPU test already run."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2412_08264_gb300 import _lib as L
from paper_2412_08264_gb300 import synth
from tests.gpu_util import DEV, make, packed, r32, rel

pytestmark = pytest.mark.gpu


def test_static_jw_matches_hypergrad_on_two_calls_in_a_row():
    wl = synth.uneven_foe([(150, 171)], n_filters=4, f=5, blur_radius=2, seed=31)
    P, prob, dt = make(wl, "fp32", max_recycle=1, max_basis=1)
    rng = np.random.default_rng(31)
    th = r32(wl.theta0)
    theta = torch.tensor(th, dtype=torch.float64, device=DEV)
    x = packed([r32(np.clip(wl.x_star[0] + 0.05 * rng.standard_normal(wl.x_star[0].shape), -0.2, 1.2))], dt)
    P.set_point(theta, x)
    lib = L.load()
    stream = torch.cuda.current_stream(DEV)
    h, w = P.sizes[0]
    for call in range(2):
        wv = packed([r32(rng.standard_normal((h, w)))], dt)
        ref = P.hypergrad(wv).cpu().numpy()
        out = torch.full((P.p,), float("nan"), dtype=torch.float64, device=DEV)
        st = lib.bl_jw_fp32_static(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(wv.data_ptr()), h, w,
                                   ctypes.c_void_p(theta.data_ptr()), wl.n_filters, wl.filter_size, 0, wl.phi_eps,
                                   ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
        assert st == L.BL_OK, lib.bl_last_error()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert rel(got, ref) < 1e-5, (call, rel(got, ref))


def test_static_jw_rejects_sizes_beyond_its_scratch():
    lib = L.load()
    dummy = ctypes.c_void_p(256)
    # 2048 x 2048 with 48 7x7 filters: 64 * 64 tiles * 2400 values > 524288
    st = lib.bl_jw_fp32_static(dummy, dummy, 2048, 2048, dummy, 48, 7, 0, 0.01, dummy, None)
    assert st == L.BL_EINVAL
    assert b"static scratch" in lib.bl_last_error()
