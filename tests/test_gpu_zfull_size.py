"""GPU parity at the full sizes of the benchmark configurations, on outputs the FP64 checker
evaluates one by one (tests/crops.py: exact crop evaluations, pinned against full-image results
in tests/test_oracle_crops.py).

  64-pair batch, in the problem configuration the bench times (FP32, recycle dimension 16, 32
  stored basis vectors): the GPU lower solve meets the first-order condition on the checker's
  FP64 gradient (smallest pairs); Hessian actions at sampled pixels (corners, edges, halo rims,
  random points) of one pair of every size; plain CG to the bench's tolerance, its residual
  recomputed by the checker; J w of whole pairs and of patch-supported w on every size.
  8 x 1024^2 with 24 7x7 filters, and 2048^2 with 48 7x7 filters and a 9x9 blur: Hessian actions
  at sampled pixels and J w for patch-supported w, at a point near x*.

Bars as for the small cases: 1e-5 relative on Hessian actions (over the sampled values) and J w,
FP32 inputs rounded identically on both sides."""
import numpy as np
import pytest
import torch

from paper_2412_08264_gb300 import synth
from tests import crops
from tests.gpu_util import DEV, make, packed, r32, rel, split

pytestmark = pytest.mark.gpu


def check_hvp_and_patch_jw(P, prob, dt, th, xs, pairs, rng, n_random):
    theta = torch.tensor(th, dtype=torch.float64, device=DEV)
    P.set_point(theta, packed(xs, dt))
    vs = [r32(rng.standard_normal(x.shape)) for x in xs]
    hv = split(P.hvp(packed(vs, dt)), P.sizes)
    got, ref = [], []
    for k in pairs:
        ll = prob.lowers[k]
        pix = crops.sample_pixels(rng, ll.h, ll.w, n_random)
        got += [hv[k][i, j] for i, j in pix]
        ref += list(crops.hvp_at(ll, xs[k], th, vs[k], pix))
    assert rel(got, ref) < 1e-5, rel(got, ref)
    ws, pts = [], []
    for k, ll in enumerate(prob.lowers):
        patch = crops.patches(ll.h, ll.w)[k % 3]      # corner, edge and interior patches in turn
        pts.append(patch)
        ws.append(r32(crops.patch_vector(rng, ll.h, ll.w, patch)))
    _, per = P.hypergrad(packed(ws, dt), per_pair=True)
    per = per.cpu().numpy()
    for k in pairs:
        ref_k = crops.jw_patch(prob.lowers[k], xs[k], th, ws[k], pts[k])
        assert rel(per[k], ref_k) < 1e-5, (k, rel(per[k], ref_k))


def test_batch64_in_the_bench_configuration():
    wl = synth.batch_64()
    P, prob, dt = make(wl, "fp32", max_recycle=16, max_basis=32)
    th = r32(wl.theta0)
    theta = torch.tensor(th, dtype=torch.float64, device=DEV)
    x = P.zeros()
    info = P.lower_solve(theta, x, gtol=1e-5, relative=True, max_iters=2000, allow_noconv=True)
    xs = split(x, P.sizes)
    order = sorted(range(len(wl.pairs)), key=lambda k: wl.pairs[k].height)
    small = order[:2]
    for k in small:
        ll = prob.lowers[k]
        g0 = np.linalg.norm(ll.grad(np.zeros_like(xs[k]), th))
        gk = np.linalg.norm(ll.grad(xs[k], th))
        # the GPU's FP32 gradient norm is the checker's FP64 one at the same x^ (cancellation at
        # convergence leaves FP32 rounding of ~1e-7 ||grad Phi(0)||), and converged pairs meet the
        # relative tolerance
        assert abs(gk - info[k]["gnorm"]) <= 0.1 * gk + 1e-6 * g0, (k, gk, info[k])
        if info[k]["status"] == 0:
            assert gk <= 3e-5 * g0, (k, gk / g0, info[k])
    one_per_size = {}
    for k in order:
        one_per_size.setdefault(wl.pairs[k].height, k)
    rng = np.random.default_rng(64)
    check_hvp_and_patch_jw(P, prob, dt, th, xs, sorted(one_per_size.values()), rng, 12)
    # the bench's Hessian solve (plain CG to rtol 1e-4) at the lower-solve point
    P.set_point(theta, x)
    w = P.zeros()
    P.hessian_solve(w, recycle=False, tol=1e-4, relative=True, maxit=3000, store_basis=False, warm_start=False)
    W = split(w, P.sizes)
    for k in small:
        g = prob.rhs(k, xs[k])
        r = g - prob.apply_H(k, xs[k], th)(W[k].ravel())
        # recursive FP32 residual below 1e-4; the true FP64 residual within 3x of it
        assert np.linalg.norm(r) <= 3e-4 * np.linalg.norm(g), (k, np.linalg.norm(r) / np.linalg.norm(g))
    _, per = P.hypergrad(w, per_pair=True)
    per = per.cpu().numpy()
    for k in [small[0], one_per_size[256]]:
        assert rel(per[k], prob.Jw(k, xs[k], th, W[k])) < 1e-5


@pytest.mark.parametrize("name", ["batch8_1024_foe_n24f7", "large2048_foe_n48f7"])
def test_large_configurations_sampled(name):
    wl = synth.WORKLOADS[name]()
    P, prob, dt = make(wl, "fp32", max_recycle=1, max_basis=4)
    th = r32(wl.theta0)
    rng = np.random.default_rng(7)
    xs = [r32(x + 0.02 * rng.standard_normal(x.shape)) for x in wl.x_star]
    pairs = list(range(min(3, len(wl.pairs))))
    check_hvp_and_patch_jw(P, prob, dt, th, xs, pairs, rng, 16)
