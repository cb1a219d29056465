"""Python binding of libbl: one object per batch of training pairs.

Thin marshalling over include/bl.h.  Image tensors are CUDA tensors (float32
for FP32 problems, float64 for FP64 problems) holding the listed pairs packed
back to back; theta and hypergradients are float64 CUDA tensors.  The library
runs on the CUDA stream that is current when the problem is created.
"""
from __future__ import annotations

import ctypes as C
from typing import Optional, Sequence

import numpy as np
import torch

from . import _lib as L
from .strategy import Strategy, parse


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else C.c_void_p(t.data_ptr())


class Problem:
    def __init__(self, pairs: Sequence, reg: str, y: torch.Tensor, x_star: torch.Tensor, n_filters: int = 0,
                 filter_size: int = 0, phi: str = "charbonnier", phi_eps: float = 0.01, l2_eps: float = 1e-6,
                 precision: str = "fp32", max_recycle: int = 0, max_basis: int = 0):
        """pairs: sequence of (height, width, blur_sigma, blur_radius) for blur pairs, or
        (height, width, blur_sigma, blur_radius, mask) with mask an (height, width) array of
        measured pixels (non-zero) for inpainting pairs (blur fields then ignored)."""
        if reg not in ("tv", "foe"):
            raise ValueError(f"unknown regulariser {reg!r} (expected 'tv' or 'foe')")
        if precision not in ("fp32", "fp64"):
            raise ValueError(f"unknown precision {precision!r} (expected 'fp32' or 'fp64')")
        if phi not in L.BL_PHI:
            raise ValueError(f"unknown phi {phi!r} (expected one of {sorted(L.BL_PHI)})")
        self.lib = L.load()
        self.K = len(pairs)
        self.sizes = [(int(p[0]), int(p[1])) for p in pairs]
        self.dtype = torch.float32 if precision == "fp32" else torch.float64
        self.device = y.device
        masks = []       # kept alive until bl_problem_create has copied them
        descs = []
        for p in pairs:
            h, w, s, r = p[:4]
            m = p[4] if len(p) > 4 else None
            ptr = None
            if m is not None:
                m = np.ascontiguousarray((np.asarray(m) != 0).astype(np.uint8))
                if m.shape != (int(h), int(w)):
                    raise ValueError(f"mask shape {m.shape} does not match the image size {(h, w)}")
                masks.append(m)
                ptr = m.ctypes.data
            descs.append(L.PairDesc(int(h), int(w), float(s), int(r), ptr))
        arr = (L.PairDesc * self.K)(*descs)
        rd = L.RegDesc(L.BL_REG_TV if reg == "tv" else L.BL_REG_FOE, int(n_filters), int(filter_size),
                       L.BL_PHI[phi], float(phi_eps), float(l2_eps),
                       L.BL_FP32 if precision == "fp32" else L.BL_FP64, int(max_recycle), int(max_basis))
        self._check_images(y)
        self._check_images(x_star)
        self.stream = torch.cuda.current_stream(y.device)
        h = C.c_void_p()
        L.check(self.lib.bl_problem_create(arr, self.K, C.byref(rd), _ptr(y), _ptr(x_star),
                                           C.c_void_p(self.stream.cuda_stream), C.byref(h)), "bl_problem_create")
        self.h = h
        self.p = self.lib.bl_num_params(self.h)
        self.max_recycle = max_recycle

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and h.value:
            self.lib.bl_problem_destroy(h)
            self.h = None

    # ---- helpers -----------------------------------------------------------------------
    def _pairs(self, pairs):
        idx = list(range(self.K)) if pairs is None else [int(i) for i in pairs]
        return (C.c_int32 * len(idx))(*idx), len(idx), idx

    def n_pixels(self, pairs=None) -> int:
        return sum(self.sizes[i][0] * self.sizes[i][1] for i in (range(self.K) if pairs is None else pairs))

    def _check_images(self, t: torch.Tensor, pairs=None):
        if not t.is_cuda or not t.is_contiguous():
            raise ValueError("image buffers must be contiguous CUDA tensors")
        if t.device != self.device:
            raise ValueError(f"image buffer on {t.device}, the problem lives on {self.device}")
        if t.dtype != self.dtype:
            raise ValueError(f"expected {self.dtype}, got {t.dtype}")
        if t.numel() != self.n_pixels(pairs):
            raise ValueError(f"packed buffer has {t.numel()} elements, pairs need {self.n_pixels(pairs)}")

    def _check_theta(self, theta: torch.Tensor):
        if not theta.is_cuda or theta.dtype != torch.float64 or theta.numel() != self.p or not theta.is_contiguous():
            raise ValueError(f"theta must be a contiguous float64 CUDA tensor of {self.p} values")
        if theta.device != self.device:
            raise ValueError(f"theta on {theta.device}, the problem lives on {self.device}")

    def empty(self, pairs=None) -> torch.Tensor:
        return torch.empty(self.n_pixels(pairs), dtype=self.dtype, device=self.device)

    def zeros(self, pairs=None) -> torch.Tensor:
        return torch.zeros(self.n_pixels(pairs), dtype=self.dtype, device=self.device)

    # ---- entry points ------------------------------------------------------------------
    def set_data(self, y: torch.Tensor, x_star: torch.Tensor, pairs=None):
        pa, n, idx = self._pairs(pairs)
        self._check_images(y, idx)
        self._check_images(x_star, idx)
        L.check(self.lib.bl_set_data(self.h, pa, n, _ptr(y), _ptr(x_star)), "bl_set_data")

    def forward(self, x: torch.Tensor, pairs=None) -> torch.Tensor:
        pa, n, idx = self._pairs(pairs)
        self._check_images(x, idx)
        out = self.empty(idx)
        L.check(self.lib.bl_forward(self.h, pa, n, _ptr(x), _ptr(out)), "bl_forward")
        return out

    def set_point(self, theta: torch.Tensor, xhat: torch.Tensor, pairs=None):
        pa, n, idx = self._pairs(pairs)
        self._check_theta(theta)
        self._check_images(xhat, idx)
        L.check(self.lib.bl_set_point(self.h, pa, n, _ptr(theta), _ptr(xhat)), "bl_set_point")

    def lower_solve(self, theta: torch.Tensor, xhat: torch.Tensor, pairs=None, gtol: float = 1e-5,
                    relative: bool = True, max_iters: int = 5000, history: int = 10, max_backtrack: int = 30,
                    armijo_slack: Optional[float] = None, allow_noconv: bool = False, graph: bool = True):
        pa, n, idx = self._pairs(pairs)
        self._check_theta(theta)
        self._check_images(xhat, idx)
        if armijo_slack is None:
            armijo_slack = 1e-6 if self.dtype == torch.float32 else 0.0
        opts = L.LbfgsOpts(int(max_iters), int(history), float(gtol), 1 if relative else 0, int(max_backtrack),
                           float(armijo_slack), 1 if graph else 0)
        info = (L.SolveInfo * n)()
        allow = (L.BL_OK, L.BL_ENOCONV) if allow_noconv else (L.BL_OK,)
        L.check(self.lib.bl_lower_solve(self.h, pa, n, _ptr(theta), C.byref(opts), _ptr(xhat), info),
                "bl_lower_solve", allow)
        return [dict(iters=i.iters, status=i.status, gnorm=i.resid, value=i.nsc_est, gtol=i.rhs_norm) for i in info]

    def gradient(self, theta: torch.Tensor, x: torch.Tensor, pairs=None):
        pa, n, idx = self._pairs(pairs)
        self._check_theta(theta)
        self._check_images(x, idx)
        g = self.empty(idx)
        vals = torch.empty(n, dtype=torch.float64, device=self.device)
        L.check(self.lib.bl_gradient(self.h, pa, n, _ptr(theta), _ptr(x), _ptr(g), _ptr(vals)), "bl_gradient")
        return g, vals

    def hvp(self, v: torch.Tensor, pairs=None) -> torch.Tensor:
        pa, n, idx = self._pairs(pairs)
        self._check_images(v, idx)
        out = self.empty(idx)
        L.check(self.lib.bl_hvp(self.h, pa, n, _ptr(v), _ptr(out)), "bl_hvp")
        return out

    def ritz_update(self, strategy, s: int, pairs=None, variant: str = "outer", allow_breakdown: bool = True):
        """variant "outer": project W with the current Hessian (eq. (3.3)); "inner": with the Hessian
        of the last solve, rebuilt from its Lanczos record (eq. (3.4); that solve must have used
        store_basis="lanczos").

        A pair whose projected matrix is not positive definite (RGSV needs T^{-1}; CholeskyQR of
        C = H U needs a full-rank U) gets an empty recycle space, so its next solve is plain CG,
        while the other pairs are refreshed; the library reports this as BL_EBREAKDOWN.  With
        allow_breakdown (the default) that status is not raised: the return value is False when
        some pair was left without a recycle space, True otherwise."""
        st = parse(strategy) if isinstance(strategy, str) else strategy
        if not st.recycles:
            return True
        pa, n, _ = self._pairs(pairs)
        o = L.RecycleOpts(L.BL_RECYCLE[st.kind], L.BL_SIZE[st.size], L.BL_SIDE[st.side], int(s),
                          L.BL_REFRESH[variant])
        allow = (L.BL_OK, L.BL_EBREAKDOWN) if allow_breakdown else (L.BL_OK,)
        status = L.check(self.lib.bl_ritz_update(self.h, pa, n, C.byref(o)), "bl_ritz_update", allow)
        return status == L.BL_OK

    def hessian_solve(self, w: torch.Tensor, g: Optional[torch.Tensor] = None, pairs=None, recycle: bool = True,
                      nsc: bool = False, tol: float = 1e-4, relative: bool = True, maxit: int = 2000,
                      store_basis: bool = True, warm_start: bool = True, nsc_scale=None, allow_noconv=False,
                      graph: bool = True, method: str = "cg"):
        """method "cg": (recycled) CG, SPD Hessians; "minres": (recycled) MINRES (Algorithm 3),
        symmetric indefinite Hessians.  store_basis: False, True (the most recent basis vectors, for
        the outer refresh) or "lanczos" (CG: the first basis vectors with the CG coefficients, for
        the inner refresh)."""
        pa, n, idx = self._pairs(pairs)
        self._check_images(w, idx)
        if g is not None:
            self._check_images(g, idx)
        if method not in ("cg", "minres"):
            raise ValueError(f"unknown Krylov method {method!r}")
        if method == "cg":
            meth = L.BL_SOLVE_RCG if recycle else L.BL_SOLVE_CG
        else:
            meth = L.BL_SOLVE_RMINRES if recycle else L.BL_SOLVE_MINRES
        store = (L.BL_STORE_LANCZOS if store_basis == "lanczos"
                 else (L.BL_STORE_RECENT if store_basis else L.BL_STORE_NONE))
        o = L.KrylovOpts(meth, L.BL_STOP_NSC if nsc else L.BL_STOP_RESID,
                         float(tol), 1 if relative else 0, int(maxit), store,
                         1 if warm_start else 0, 1 if graph else 0)
        sc = None
        if nsc_scale is not None:
            vals = [float(v) for v in nsc_scale]
            if len(vals) != n:
                raise ValueError(f"nsc_scale needs one value per solved pair ({n}), got {len(vals)}")
            sc = (C.c_double * n)(*vals)
        info = (L.SolveInfo * n)()
        allow = (L.BL_OK, L.BL_ENOCONV) if allow_noconv else (L.BL_OK,)
        L.check(self.lib.bl_hessian_solve(self.h, pa, n, C.byref(o), _ptr(g), _ptr(w), sc, info),
                "bl_hessian_solve", allow)
        return [dict(iters=i.iters, status=i.status, resid=i.resid, nsc=i.nsc_est, rhs_norm=i.rhs_norm)
                for i in info]

    def hypergrad(self, w: torch.Tensor, pairs=None, per_pair: bool = False, loss: bool = False):
        pa, n, idx = self._pairs(pairs)
        self._check_images(w, idx)
        mean = torch.empty(self.p, dtype=torch.float64, device=self.device)
        grads = torch.empty((n, self.p), dtype=torch.float64, device=self.device) if per_pair else None
        lv = C.c_double(0.0)
        L.check(self.lib.bl_hypergrad(self.h, pa, n, _ptr(w), _ptr(grads), _ptr(mean),
                                      C.byref(lv) if loss else None), "bl_hypergrad")
        out = [mean]
        if per_pair:
            out.append(grads)
        if loss:
            out.append(lv.value)
        return out[0] if len(out) == 1 else tuple(out)

    def recycle_dim(self, pair: int) -> int:
        return self.lib.bl_recycle_dim(self.h, int(pair))

    def basis_size(self, pair: int) -> int:
        return self.lib.bl_basis_size(self.h, int(pair))

    def recycle_export(self, pair: int) -> bytes:
        nbytes = C.c_size_t(0)
        L.check(self.lib.bl_recycle_export(self.h, int(pair), None, C.byref(nbytes)), "bl_recycle_export")
        buf = C.create_string_buffer(nbytes.value)
        L.check(self.lib.bl_recycle_export(self.h, int(pair), buf, C.byref(nbytes)), "bl_recycle_export")
        return buf.raw[:nbytes.value]

    def recycle_import(self, pair: int, data: bytes):
        buf = C.create_string_buffer(data, len(data))
        L.check(self.lib.bl_recycle_import(self.h, int(pair), buf, len(data)), "bl_recycle_import")

    def graph_used(self) -> bool:
        return bool(self.lib.bl_graph_used(self.h))

    def hvp_tma(self) -> bool:
        """Whether the FP32 Hessian action runs the TMA-staged kernel (else the generic one)."""
        return bool(self.lib.bl_hvp_tma(self.h))

    def hvp_tile(self, pair: int) -> int:
        """Output tile side of the TMA-staged Hessian action for a pair (0: generic kernel)."""
        return int(self.lib.bl_hvp_tile(self.h, int(pair)))

    def set_hvp_tile(self, pair: int, side: int):
        L.check(self.lib.bl_set_hvp_tile(self.h, int(pair), int(side)), "bl_set_hvp_tile")

    def launch_count(self) -> int:
        return int(self.lib.bl_launch_count(self.h))

    def profile(self, enable: bool = True):
        L.check(self.lib.bl_profile_enable(self.h, 1 if enable else 0), "bl_profile_enable")

    def profile_read(self) -> dict:
        """Per kernel class: total milliseconds, launches, pixels processed and (vector passes) algorithmic
        bytes moved since profile()."""
        out = {}
        for i, name in enumerate(L.KERNEL_CLASSES):
            ms, n, px = C.c_double(), C.c_int64(), C.c_int64()
            L.check(self.lib.bl_profile_read(self.h, i, C.byref(ms), C.byref(n), C.byref(px)), "bl_profile_read")
            nb = C.c_int64()
            L.check(self.lib.bl_profile_read_bytes(self.h, i, C.byref(nb)), "bl_profile_read_bytes")
            out[name] = dict(ms=ms.value, launches=n.value, pixels=px.value, bytes=nb.value)
        return out


def from_workload(wl, y: torch.Tensor, x_star: torch.Tensor, **kw) -> Problem:
    """Problem for a synth.Workload with given packed measurements and ground truths."""
    masks = (list(getattr(wl, "masks", None) or []) + [None] * len(wl.pairs))[:len(wl.pairs)]
    pairs = [(p.height, p.width, p.blur_sigma, p.blur_radius, m) for p, m in zip(wl.pairs, masks)]
    args = dict(reg=wl.reg, n_filters=wl.n_filters, filter_size=wl.filter_size, phi=wl.phi,
                phi_eps=wl.phi_eps, l2_eps=wl.l2_eps, precision=wl.precision)
    args.update(kw)
    return Problem(pairs, y=y, x_star=x_star, **args)
