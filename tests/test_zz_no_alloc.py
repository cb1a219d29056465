"""The allocation-free J w entry point (bl_jw_fp32_static).

Some callers cannot allocate device memory once they run: code inside a host framework that owns
the whole device heap, or a service under a no-allocation rule after start-up.  They cannot create
a bl_problem (its set-up allocates), so bl_jw_fp32_static computes J w for one FP32 image with its
scratch in a fixed device array of the library.

Checked here, on two calls in a row on different vectors, for every filter size and penalty:
  - against the FP64 checker's J w (oracle.functional.LowerLevel.Jw) on the same FP32-rounded
    inputs, within the 1e-5 relative bar of the other J w parity tests, with a per-element bar;
  - against the allocating path (bl_hypergrad on a bl_problem) within the same bar;
  - that the calls leave the device's free memory unchanged (no allocation).
This file is collected last, so a failure here leaves every other GPU test already run."""
import ctypes

import numpy as np
import pytest
import torch

from oracle.functional import LowerLevel
from paper_2412_08264_gb300 import _lib as L
from paper_2412_08264_gb300 import synth
from tests.gpu_util import DEV, make, max_elem, packed, r32, rel

pytestmark = pytest.mark.gpu

TOL = 1e-5
PHI = ["charbonnier", "sq", "log1p"]


def _call(lib, x, wv, h, w, theta, wl, out, stream):
    return lib.bl_jw_fp32_static(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(wv.data_ptr()), h, w,
                                 ctypes.c_void_p(theta.data_ptr()), wl.n_filters, wl.filter_size,
                                 L.BL_PHI[wl.phi], wl.phi_eps, ctypes.c_void_p(out.data_ptr()),
                                 ctypes.c_void_p(stream.cuda_stream))


@pytest.mark.parametrize("f, phi, size", [(1, "charbonnier", (40, 33)), (3, "sq", (7, 13)), (5, "charbonnier", (150, 171)),
                                          (5, "log1p", (96, 64)), (7, "log1p", (70, 45)), (7, "charbonnier", (31, 97)),
                                          (3, "charbonnier", (65, 1))])
def test_static_jw_matches_checker_and_hypergrad_on_two_calls_in_a_row(f, phi, size):
    h, w = size
    wl = synth.uneven_foe([size], n_filters=4, f=f, blur_radius=2, seed=31 + f)
    wl.phi = phi
    P, prob, dt = make(wl, "fp32", max_recycle=1, max_basis=1)
    rng = np.random.default_rng(31 + f)
    th = r32(wl.theta0)
    theta = torch.tensor(th, dtype=torch.float64, device=DEV)
    xh = r32(np.clip(wl.x_star[0] + 0.05 * rng.standard_normal((h, w)), -0.2, 1.2))
    x = packed([xh], dt)
    P.set_point(theta, x)
    ll = LowerLevel(prob.ys[0], None, "foe", wl.n_filters, f, phi, wl.phi_eps, wl.l2_eps)
    lib = L.load()
    stream = torch.cuda.current_stream(DEV)
    out = torch.empty(P.p, dtype=torch.float64, device=DEV)
    # a first call looks up the scratch array's device address (and loads the library's module)
    wv = packed([r32(rng.standard_normal((h, w)))], dt)
    assert _call(lib, x, wv, h, w, theta, wl, out, stream) == L.BL_OK, lib.bl_last_error()
    torch.cuda.synchronize()
    vecs = [r32(rng.standard_normal((h, w))) for _ in range(2)]
    refs_alloc = [P.hypergrad(packed([v], dt)).cpu().numpy() for v in vecs]
    wvs = [packed([v], dt) for v in vecs]
    outs = [torch.full((P.p,), float("nan"), dtype=torch.float64, device=DEV) for _ in range(2)]
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info(DEV)
    for call in range(2):
        st = _call(lib, x, wvs[call], h, w, theta, wl, outs[call], stream)
        assert st == L.BL_OK, lib.bl_last_error()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info(DEV)
    assert free1 == free0, f"device free memory changed by {free0 - free1} bytes across the calls"
    for call in range(2):
        got = outs[call].cpu().numpy()
        assert np.all(np.isfinite(got))
        ref = ll.Jw(xh, th, vecs[call])
        assert rel(got, ref) < TOL, (call, rel(got, ref))
        assert max_elem(got, ref) < TOL, (call, max_elem(got, ref))
        assert rel(got, refs_alloc[call]) < TOL, (call, rel(got, refs_alloc[call]))
