"""Python binding of libkpdhg: a Plan object whose methods carry the C ABI's names.

Every method only checks and marshals torch tensors (device pointers, sizes, the current
CUDA stream) into one C call; all arithmetic runs in the library's CUDA kernels.
Complex storage: torch.complex64 tensors map to KP_C64; float16 / bfloat16 tensors with a
trailing dimension of 2 (re, im) map to KP_C32_FP16 / KP_C32_BF16.
"""
from __future__ import annotations

import ctypes
import math

import torch

from . import _lib as L

_REG = {"l2": L.KP_REG_L2, "l1_wavelet": L.KP_REG_L1_WAVELET, "tv": L.KP_REG_TV}


def _stream(device):
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _ctype_of(t: torch.Tensor):
    if t.dtype == torch.complex64:
        return L.KP_C64
    if t.dtype == torch.float16 and t.shape[-1] == 2:
        return L.KP_C32_FP16
    if t.dtype == torch.bfloat16 and t.shape[-1] == 2:
        return L.KP_C32_BF16
    raise TypeError(f"unsupported complex storage {t.dtype} {tuple(t.shape)}")


def _ptr(t: torch.Tensor):
    return ctypes.c_void_p(t.data_ptr())


def to_storage(t: torch.Tensor, kind: str) -> torch.Tensor:
    """complex64 -> storage tensor of the given kind ('c64', 'bf16', 'fp16')."""
    if kind == "c64":
        return t.to(torch.complex64).contiguous()
    r = torch.view_as_real(t.to(torch.complex64).contiguous())
    return r.to(torch.bfloat16 if kind == "bf16" else torch.float16).contiguous()


class Plan:
    """A reconstruction plan for one image size, coil count and sample count (kp_plan)."""

    def __init__(self, img_shape, ncoils, nsamples, oversamp=1.25, kernel_width=4, wavelet_levels=0,
                 device="cuda"):
        self.lib = L.load()
        self.device = torch.device(device)
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        self.img_shape = tuple(int(n) for n in img_shape)
        self.ncoils = int(ncoils)
        self.nsamples = int(nsamples)
        self.ndim = len(self.img_shape)
        prm = L.KpParams()
        prm.ndim = self.ndim
        for d, n in enumerate(self.img_shape):
            prm.img[d] = n
        prm.ncoils = self.ncoils
        prm.nsamples = self.nsamples
        prm.oversamp = float(oversamp)
        prm.kernel_width = int(kernel_width)
        prm.wavelet_levels = int(wavelet_levels)
        self._h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            L.check(self.lib.kp_plan_create(ctypes.byref(self._h), ctypes.byref(prm), _stream(self.device)),
                    "kp_plan_create")

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self.lib.kp_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _dev(self, t, name):
        """Check placement and layout; materialise lazy conjugate / negative views (autograd
        hands those to backward functions), whose raw memory is not the tensor's value."""
        if not t.is_cuda or t.device != self.device:
            raise ValueError(f"{name} must be on {self.device}")
        if t.is_conj() or t.is_neg():
            t = t.resolve_conj().resolve_neg()
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        return t

    @property
    def N(self):
        return math.prod(self.img_shape)

    # -------------------------------------------------------------- set-up
    def set_trajectory(self, traj):
        """traj: float32 [M, ndim] in cycles/FOV on the plan's device."""
        t = self._dev(traj, "traj")
        if t.dtype != torch.float32 or tuple(t.shape) != (self.nsamples, self.ndim):
            raise ValueError("traj must be float32 [M, ndim]")
        L.check(self.lib.kp_plan_set_trajectory(self._h, _ptr(t), _stream(self.device)), "kp_plan_set_trajectory")
        self.trajectory = t.detach().clone()
        return self

    def set_maps(self, maps):
        """maps: [C, *img] complex64, or [C, *img, 2] float16/bfloat16."""
        m = self._dev(maps, "maps")
        kind = _ctype_of(m)
        L.check(self.lib.kp_plan_set_maps(self._h, _ptr(m), kind, _stream(self.device)), "kp_plan_set_maps")
        self._maps_ref = m
        return self

    def set_profiling(self, enable=True):
        L.check(self.lib.kp_plan_set_profiling(self._h, int(bool(enable))), "kp_plan_set_profiling")
        return self

    def launch_count(self):
        n = ctypes.c_int64()
        L.check(self.lib.kp_plan_launch_count(self._h, ctypes.byref(n)), "kp_plan_launch_count")
        return n.value

    def tile_stats(self):
        nt, mx = ctypes.c_int64(), ctypes.c_int64()
        L.check(self.lib.kp_plan_tile_stats(self._h, ctypes.byref(nt), ctypes.byref(mx)), "kp_plan_tile_stats")
        return nt.value, mx.value

    def spread_config(self):
        """Autotuned spreading choice: dict(variant, chunk, items, split_tiles)."""
        v, c, ni, ns = ctypes.c_int(), ctypes.c_int(), ctypes.c_int64(), ctypes.c_int64()
        L.check(self.lib.kp_plan_spread_config(self._h, ctypes.byref(v), ctypes.byref(c), ctypes.byref(ni),
                                               ctypes.byref(ns)), "kp_plan_spread_config")
        return dict(variant=v.value, chunk=c.value, items=ni.value, split_tiles=ns.value)

    # -------------------------------------------------------------- operators
    def sense_forward(self, x, out=None, storage="c64"):
        """y = A x: x complex64 [*img] -> y [C, M] (complex64 or half storage)."""
        x = self._dev(x, "x")
        if x.dtype != torch.complex64 or x.numel() != self.N:
            raise ValueError("x must be complex64 of the image size")
        if out is None:
            if storage == "c64":
                out = torch.empty((self.ncoils, self.nsamples), dtype=torch.complex64, device=self.device)
            else:
                dt = torch.bfloat16 if storage == "bf16" else torch.float16
                out = torch.empty((self.ncoils, self.nsamples, 2), dtype=dt, device=self.device)
        self._dev(out, "out")
        L.check(self.lib.kp_sense_forward(self._h, _ptr(x), _ptr(out), _ctype_of(out), _stream(self.device)),
                "kp_sense_forward")
        return out

    def sense_adjoint(self, y, out=None):
        """x = A^H y: y [C, M] -> complex64 [*img]."""
        y = self._dev(y, "y")
        if out is None:
            out = torch.empty(self.img_shape, dtype=torch.complex64, device=self.device)
        out = self._dev(out, "out")
        L.check(self.lib.kp_sense_adjoint(self._h, _ptr(y), _ctype_of(y), _ptr(out), _stream(self.device)),
                "kp_sense_adjoint")
        return out

    def make_preconditioner(self, multichannel=True, out=None):
        """Diagonal k-space preconditioner p [C, M] float32 (multi- or single-channel)."""
        if out is None:
            out = torch.empty((self.ncoils, self.nsamples), dtype=torch.float32, device=self.device)
        self._dev(out, "out")
        L.check(self.lib.kp_make_preconditioner(self._h, int(bool(multichannel)), _ptr(out), _stream(self.device)),
                "kp_make_preconditioner")
        return out

    def max_eig(self, p=None, v0=None, iters=30):
        """lambda_max(P A A^H) by the power method."""
        lm = ctypes.c_double()
        p = self._dev(p, "p") if p is not None else None
        v0 = self._dev(v0, "v0") if v0 is not None else None
        pp = _ptr(p) if p is not None else None
        vv = _ptr(v0) if v0 is not None else None
        L.check(self.lib.kp_max_eig(self._h, pp, vv, int(iters), ctypes.byref(lm), _stream(self.device)),
                "kp_max_eig")
        return lm.value

    def sense_forward_traj_grad(self, x, gy):
        """dL/dtraj [M, ndim] through y = A x for the upstream gradient gy."""
        out = torch.empty((self.nsamples, self.ndim), dtype=torch.float32, device=self.device)
        x, gy = self._dev(x, "x"), self._dev(gy, "gy")
        L.check(self.lib.kp_sense_forward_traj_grad(self._h, _ptr(x), _ptr(gy),
                                                    _ptr(out), _stream(self.device)), "kp_sense_forward_traj_grad")
        return out

    def sense_adjoint_traj_grad(self, u, gx):
        """dL/dtraj [M, ndim] through x = A^H u for the upstream gradient gx."""
        out = torch.empty((self.nsamples, self.ndim), dtype=torch.float32, device=self.device)
        u, gx = self._dev(u, "u"), self._dev(gx, "gx")
        L.check(self.lib.kp_sense_adjoint_traj_grad(self._h, _ptr(u), _ptr(gx),
                                                    _ptr(out), _stream(self.device)), "kp_sense_adjoint_traj_grad")
        return out

    def unrolled_forward(self, y, p=None, lam=0.0, iters=10, lmax=0.0):
        """Unrolled l2 PDHG keeping per-iteration checkpoints; returns x_K.  The checkpoints of
        an earlier call are replaced (tape_id counts the calls)."""
        self.tape_id = getattr(self, "tape_id", 0) + 1
        x = torch.empty(self.img_shape, dtype=torch.complex64, device=self.device)
        p = self._dev(p, "p") if p is not None else None
        y = self._dev(y, "y")
        pp = _ptr(p) if p is not None else None
        L.check(self.lib.kp_unrolled_forward(self._h, _ptr(y), pp, float(lam), int(iters), float(lmax),
                                             _ptr(x), _stream(self.device)), "kp_unrolled_forward")
        return x

    def unrolled_backward(self, gx, want_y=True, want_traj=True):
        """Reverse sweep of the last unrolled_forward: (dL/dy, dL/dlambda, dL/dtraj)."""
        gy = torch.empty((self.ncoils, self.nsamples), dtype=torch.complex64, device=self.device) if want_y else None
        gt = torch.empty((self.nsamples, self.ndim), dtype=torch.float32, device=self.device) if want_traj else None
        gl = ctypes.c_double()
        gx = self._dev(gx.contiguous(), "gx")
        L.check(self.lib.kp_unrolled_backward(self._h, _ptr(gx),
                                              _ptr(gy) if gy is not None else None, ctypes.byref(gl),
                                              _ptr(gt) if gt is not None else None, _stream(self.device)),
                "kp_unrolled_backward")
        return gy, gl.value, gt

    def wavelet(self, x, forward=True, out=None):
        x = self._dev(x, "x")
        if out is None:
            out = torch.empty_like(x)
        L.check(self.lib.kp_wavelet(self._h, _ptr(x), _ptr(out), int(bool(forward)), _stream(self.device)),
                "kp_wavelet")
        return out

    def dual_l2_solve(self, y, p=None, lam=1.0, iters=50):
        """l2 reconstruction through the dual: (A A^H + lam I) w = lam y by conjugate gradients
        with p (complex64 y [C, M]; float32 p [C, M] or None) as preconditioner, x = A^H w / lam.
        Returns (x, residual norms before and after each iteration)."""
        yd = self._dev(y, "y")
        if yd.dtype != torch.complex64 or tuple(yd.shape) != (self.ncoils, self.nsamples):
            raise ValueError("y must be complex64 [C, M]")
        pd = self._dev(p, "p") if p is not None else None
        x = torch.empty(self.img_shape, dtype=torch.complex64, device=self.device)
        tr = (ctypes.c_double * (int(iters) + 1))()
        L.check(self.lib.kp_dual_l2_solve(self._h, _ptr(yd), _ptr(pd) if pd is not None else None, float(lam),
                                          int(iters), _ptr(x), tr, _stream(self.device)), "kp_dual_l2_solve")
        return x, list(tr)

    def pdhg_solve(self, y, p=None, reg="l2", lam=0.0, iters=30, lmax=0.0, trace=False, out=None, state=None,
                   return_state=False):
        """Preconditioned PDHG; reg is "l2", "l1_wavelet" (Sec. 4.1) or "tv" (Sec. 4.2).  y may
        live on the host (it is then copied in, and x copied back to the host; page-locked y is
        copied in by the library while the set-up runs, and a page-locked host `out` receives x).  state: None to
        start from zero, or a dict (x, xbar, u, v, k) returned by an earlier call with
        return_state=True, to continue that run (kp_pdhg_solve_ex).  Returns (x, objective trace
        or None, stats dict), plus the state dict after the last iteration when return_state."""
        host = not y.is_cuda
        if host and y.is_pinned() and y.is_contiguous() and state is None and not return_state:
            # page-locked host measurements: the library copies them in while the set-up runs
            ct = _ctype_of(y)
            if y.numel() * y.element_size() != self.ncoils * self.nsamples * (8 if ct == L.KP_C64 else 4):
                raise ValueError("y must hold [C, M] complex values")
            pd = self._dev(p, "p") if p is not None and p.is_cuda else (
                p.to(self.device, non_blocking=True) if p is not None else None)
            xd = torch.empty(self.img_shape, dtype=torch.complex64, device=self.device)
            tr = (ctypes.c_double * max(int(iters), 1))() if trace else None
            st = L.KpStats()
            L.check(self.lib.kp_pdhg_solve_host(self._h, _ptr(y), _ctype_of(y), _ptr(pd) if pd is not None else None,
                                                _REG[reg], float(lam), int(iters), float(lmax), _ptr(xd), tr,
                                                ctypes.byref(st), _stream(self.device)), "kp_pdhg_solve_host")
            stats = dict(iters=st.iters, lmax=st.lmax, pmin=st.pmin, sigma_last=st.sigma_last,
                         tau_last=st.tau_last, final_obj=st.final_obj,
                         phase_ms={n: st.phase_ms[i] for i, n in enumerate(L.PHASES)})
            if out is not None and not out.is_cuda and out.is_pinned():
                # a page-locked result buffer of the caller: one asynchronous copy
                out.copy_(xd, non_blocking=True)
                torch.cuda.current_stream(self.device).synchronize()
                xh = out
            else:
                xh = xd.to("cpu")
            return xh, (list(tr)[: int(iters)] if trace else None), stats
        yd = y.to(self.device, non_blocking=True) if host else y
        yd = self._dev(yd, "y")
        pd = None
        if p is not None:
            pd = p.to(self.device, non_blocking=True) if not p.is_cuda else p
            pd = self._dev(pd, "p")
        x = torch.empty(self.img_shape, dtype=torch.complex64, device=self.device) if out is None or host else out
        tr = (ctypes.c_double * max(int(iters), 1))() if trace else None
        st = L.KpStats()
        start = None
        if state is not None:
            sx, sxb, su = (self._dev(state[k], k) for k in ("x", "xbar", "u"))
            sv = self._dev(state["v"], "v") if state.get("v") is not None else None
            start = L.KpState(sx.data_ptr(), sxb.data_ptr(), su.data_ptr(), sv.data_ptr() if sv is not None else None,
                              int(state["k"]))
        new_state = None
        if return_state:
            new_state = {"x": x, "xbar": torch.empty_like(x),
                         "u": torch.empty((self.ncoils, self.nsamples), dtype=torch.complex64, device=self.device),
                         "v": torch.empty((self.ndim,) + self.img_shape, dtype=torch.complex64, device=self.device)
                         if reg == "tv" else None}
        end = L.KpState(x.data_ptr(), new_state["xbar"].data_ptr() if new_state else None,
                        new_state["u"].data_ptr() if new_state else None,
                        new_state["v"].data_ptr() if new_state and new_state["v"] is not None else None, 0)
        status = self.lib.kp_pdhg_solve_ex(self._h, _ptr(yd), _ctype_of(yd), _ptr(pd) if pd is not None else None,
                                           _REG[reg], float(lam), int(iters), float(lmax),
                                           ctypes.byref(start) if start is not None else None, ctypes.byref(end),
                                           tr, ctypes.byref(st), _stream(self.device))
        L.check(status, "kp_pdhg_solve_ex")
        if host:
            x = x.to("cpu")
        stats = dict(iters=st.iters, lmax=st.lmax, pmin=st.pmin, sigma_last=st.sigma_last,
                     tau_last=st.tau_last, final_obj=st.final_obj,
                     phase_ms={n: st.phase_ms[i] for i, n in enumerate(L.PHASES)})
        out_t = (x, (list(tr)[: int(iters)] if trace else None), stats)
        if return_state:
            new_state["k"] = end.k
            return out_t + (new_state,)
        return out_t

    def circulant_preconditioner(self):
        """Eigenvalues (float32 [*img]) of the App. B l2-optimised circulant preconditioner."""
        out = torch.empty(self.img_shape, dtype=torch.float32, device=self.device)
        L.check(self.lib.kp_make_circulant_preconditioner(self._h, _ptr(out), _stream(self.device)),
                "kp_make_circulant_preconditioner")
        return out

    def cg_l2_solve(self, y, lam, iters, circulant=False, trace=True):
        """CG on (A^H A + lam I) x = A^H y, plain or circulant-preconditioned (App. B).
        Returns (x, objective trace or None)."""
        yd = self._dev(y, "y")
        if yd.dtype != torch.complex64 or tuple(yd.shape) != (self.ncoils, self.nsamples):
            raise ValueError("y must be complex64 [C, M]")
        x = torch.empty(self.img_shape, dtype=torch.complex64, device=self.device)
        tr = (ctypes.c_double * max(int(iters), 1))() if trace else None
        L.check(self.lib.kp_cg_l2_solve(self._h, _ptr(yd), float(lam), int(iters), int(bool(circulant)), _ptr(x), tr,
                                        _stream(self.device)), "kp_cg_l2_solve")
        return x, (list(tr)[: int(iters)] if trace else None)

    def fista_solve(self, y, reg, lam, iters, lmax=0.0, trace=True):
        """FISTA for reg "l2" or "l1_wavelet" with step 1/lmax (lmax <= 0: estimated).
        Returns (x, objective trace or None)."""
        yd = self._dev(y, "y")
        if yd.dtype != torch.complex64 or tuple(yd.shape) != (self.ncoils, self.nsamples):
            raise ValueError("y must be complex64 [C, M]")
        x = torch.empty(self.img_shape, dtype=torch.complex64, device=self.device)
        tr = (ctypes.c_double * max(int(iters), 1))() if trace else None
        L.check(self.lib.kp_fista_solve(self._h, _ptr(yd), _REG[reg], float(lam), int(iters), float(lmax), _ptr(x), tr,
                                        _stream(self.device)), "kp_fista_solve")
        return x, (list(tr)[: int(iters)] if trace else None)

    def set_wait_limit(self, cycles):
        """Limit (SM clock cycles) of every bounded device wait of this plan's kernels."""
        L.check(self.lib.kp_plan_set_wait_limit(self._h, int(cycles)), "kp_plan_set_wait_limit")
        return self

    def sync(self):
        """Wait for the plan's stream work and report recorded device-side timeouts."""
        L.check(self.lib.kp_plan_sync(self._h, _stream(self.device)), "kp_plan_sync")


BATCH_FORMS = {"per_case": 0, "phases": 1}


class Batch:
    """Independent cases (one Plan each, any sizes) solved together: per-case set-up, then one
    CUDA graph per iteration advancing every case (kp_batch).  form "per_case" puts each case's
    own kernels on its own stream; "phases" issues one launch per phase over all cases."""

    def __init__(self, plans, form="per_case"):
        self.lib = L.load()
        self.plans = list(plans)
        if not self.plans:
            raise ValueError("a batch needs at least one plan")
        self.device = self.plans[0].device
        if any(p.device != self.device for p in self.plans):
            raise ValueError("all plans of a batch must be on one device")
        n = len(self.plans)
        arr = (ctypes.c_void_p * n)(*[p._h.value for p in self.plans])
        self._h = ctypes.c_void_p()
        L.check(self.lib.kp_batch_create(ctypes.byref(self._h), arr, n), "kp_batch_create")
        self.set_form(form)

    def set_form(self, form):
        if form not in BATCH_FORMS:
            raise ValueError(f"batch form must be one of {sorted(BATCH_FORMS)}")
        L.check(self.lib.kp_batch_set_form(self._h, BATCH_FORMS[form]), "kp_batch_set_form")
        self.form = form
        return self

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self.lib.kp_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, ys, ps=None, regs="l2", lams=0.0, iters=30):
        """ys: list of [C_i, M_i] device tensors; ps: list (entries may be None) or None;
        regs / lams: one value or one per case.  Returns the list of complex64 images."""
        n = len(self.plans)
        if len(ys) != n:
            raise ValueError("one y per case")
        regs = [regs] * n if isinstance(regs, str) else list(regs)
        lams = [lams] * n if isinstance(lams, (int, float)) else list(lams)
        ys = [pl._dev(y, "y") for pl, y in zip(self.plans, ys)]
        ps = [None] * n if ps is None else [pl._dev(p, "p") if p is not None else None for pl, p in zip(self.plans, ps)]
        xs = [torch.empty(pl.img_shape, dtype=torch.complex64, device=self.device) for pl in self.plans]
        VP = ctypes.c_void_p * n
        st = self.lib.kp_batch_solve(
            self._h, VP(*[y.data_ptr() for y in ys]), (ctypes.c_int * n)(*[_ctype_of(y) for y in ys]),
            VP(*[p.data_ptr() if p is not None else None for p in ps]),
            (ctypes.c_int * n)(*[_REG[r] for r in regs]), (ctypes.c_float * n)(*[float(v) for v in lams]),
            int(iters), VP(*[x.data_ptr() for x in xs]), _stream(self.device))
        L.check(st, "kp_batch_solve")
        return xs


def bounds_report():
    """Out-of-range accesses the bounds-checked build recorded since the last call
    (kp_bounds_report): dict(checked, count, first_site, first_index); checked is False and
    count 0 for the release build."""
    lib = L.load()
    ck, n, site, idx = ctypes.c_int(), ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_int64()
    L.check(lib.kp_bounds_report(ctypes.byref(ck), ctypes.byref(n), ctypes.byref(site), ctypes.byref(idx)),
            "kp_bounds_report")
    return dict(checked=bool(ck.value), count=int(n.value), first_site=int(site.value), first_index=int(idx.value))
