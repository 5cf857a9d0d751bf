"""Torch-facing wrapper of the C ABI: device memory and streams come from
PyTorch, every computation from the CUDA library (no fallback path).

  Engine(...)                 one context = one grid / frequency set / dt
  .fwd_model(rho, src, rec)   -> d_syn [S, R, F] complex128 (+ E volumes)
  .estimate_adjoint_basis()   -> B+ [nt, 2F] float64 (device), fit residual
  .adjoint_model(rho, rec, resid, basis) -> conj(v) volumes
  .gradient(rho, E, V, wrt)   -> [nz, ny, nx]
  .gradient_td(rho, src, rec, resid, wrt) -> [nz, ny, nx] by the time-domain adjoint
  misfit(d_obs, d_syn, w)     -> phi (0-d tensor), resid
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Optional

import numpy as np
import torch

from . import _capi


def _stream():
    return ctypes_void(torch.cuda.current_stream().cuda_stream)


def ctypes_void(v):
    import ctypes
    return ctypes.c_void_p(v)


def _ptr(t: Optional[torch.Tensor]):
    import ctypes
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


class Engine:
    """One context: grid, frequencies, dt/nt, precision, batch capacity.

    vti=True: a VTI medium (Sec. 2); models are (2, nz, ny, nx) = (rho_h, rho_v) and
    gradients (2, nz, ny, nx) = (h, v) (Sec. 3.1, Eq. 15).  order=4: four-point staggered
    differences on the non-uniform grid instead of the two-point Yee ones."""

    def __init__(self, xn, yn, zn, npml, freqs, f0=1.0, rho_max=1.0, precision=32, kahan=1,
                 max_src=1, max_rec=0, nt=0, dt=0.0, device=None, autotune=True, vti=False, order=2,
                 ring_slots=0):
        if not torch.cuda.is_available():
            raise RuntimeError("the CSEM engine needs a CUDA device")
        self.device = torch.device(device or "cuda")
        with torch.cuda.device(self.device):
            self.ctx = _capi.create(xn, yn, zn, npml, freqs, f0=f0, rho_max=rho_max, dt=dt, nt=nt,
                                    precision=precision, kahan=kahan, max_src=max_src, max_rec=max_rec,
                                    anisotropy=1 if vti else 0, order=order, ring_slots=ring_slots)
        info = _capi.get_info(self.ctx)
        self.info = info
        self.nx, self.ny, self.nz = info.nx, info.ny, info.nz
        self.pitch, self.vol = info.pitch, info.vol_elems
        self.dt, self.nt = info.dt, info.nt
        self.precision = precision
        self.rho_max = float(rho_max)
        self.vti = bool(vti)
        self.order = info.order
        self.freqs = np.asarray(freqs, np.float64)
        self.nf = self.freqs.size
        self.f0 = f0
        self.real = torch.float32 if precision == 32 else torch.float64
        self.cplx = torch.complex64 if precision == 32 else torch.complex128
        self._wavelet = None
        self.early_stop_tol = 0.0
        self.kz = _capi.autotune(self.ctx, max_src, _stream()) if autotune else None

    @classmethod
    def from_workload(cls, wl, max_src=None, max_rec=None, nt=None, **kw):
        return cls(wl.xn, wl.yn, wl.zn, wl.npml, wl.freqs, f0=wl.f0, rho_max=wl.rho_max,
                   precision=kw.pop("precision", wl.precision), kahan=kw.pop("kahan", wl.kahan),
                   max_src=max_src or wl.src.n, max_rec=max_rec if max_rec is not None else wl.rec.n,
                   nt=nt if nt is not None else (wl.nt or 0), **kw)

    def close(self):
        self._td_work = None
        if getattr(self, "ctx", None):
            _capi.destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- shapes ------------------------------------------------------------
    def volume_shape(self, n_src):
        return (n_src, 3, self.nf, self.nz + 1, self.ny + 1, self.pitch)

    @property
    def model_shape(self):
        """Shape of a model or gradient: (nz, ny, nx), or (2, nz, ny, nx) for VTI."""
        return ((2,) if self.vti else ()) + (self.nz, self.ny, self.nx)

    def _model(self, rho):
        """The model a call passes to the library: on this device, contiguous, of model_shape."""
        same_device = torch.is_tensor(rho) and rho.is_cuda and \
            (self.device.index is None or rho.device.index == self.device.index)
        if not same_device or tuple(rho.shape) != self.model_shape or rho.dtype != self.real \
                or not rho.is_contiguous():
            raise ValueError(f"expected a contiguous {self.real} model of shape {self.model_shape} on {self.device}")
        return rho

    def model_tensor(self, rho) -> torch.Tensor:
        t = torch.as_tensor(np.asarray(rho), dtype=self.real) if not torch.is_tensor(rho) else rho.to(self.real)
        if tuple(t.shape) != self.model_shape:
            raise ValueError(f"model of shape {tuple(t.shape)}, expected {self.model_shape}")
        return t.to(self.device).contiguous()

    # -- C-ABI calls ---------------------------------------------------------
    def fwd_model(self, rho: torch.Tensor, src, rec, keep_volume=False, trace=False):
        S = src.n
        d = torch.zeros((S, rec.n, self.nf), dtype=torch.complex128, device=self.device)
        vol = torch.empty(self.volume_shape(S), dtype=self.cplx, device=self.device) if keep_volume else None
        tr = None
        if trace:
            tr = torch.zeros((S, rec.n, self.nt), dtype=torch.float64, device=self.device)
            _capi.set_trace(self.ctx, _ptr(tr))
        try:
            _capi.fwd_model(self.ctx, _ptr(self._model(rho)), src, rec, _ptr(d) if rec.n else None, _ptr(vol),
                            _stream())
        finally:
            if trace:
                _capi.set_trace(self.ctx, None)
        out = [d]
        if keep_volume:
            out.append(vol)
        if trace:
            out.append(tr)
        return out[0] if len(out) == 1 else tuple(out)

    def set_early_stop(self, tol=0.0):
        """Forward data runs (no volumes) end once the receiver spectra change by at most
        tol (relative) over 64 steps (Sec. 2); 0 turns it off."""
        _capi.set_early_stop(self.ctx, tol)
        self.early_stop_tol = float(tol)

    def set_early_stop_volumes(self, tol=0.0, floor=1e-4):
        """Forward runs with volumes and adjoint runs end once every entry of the volumetric
        transform changes over 64 steps by at most tol times the larger of its magnitude and
        `floor` times its frequency's largest magnitude (Sec. 2, csem_set_early_stop_volumes)."""
        _capi.set_early_stop_volumes(self.ctx, tol, floor)

    def last_run_steps(self) -> int:
        """Steps the last fwd_model or adjoint_model run included (synchronises the current stream)."""
        return _capi.last_run_steps(self.ctx, _stream())

    def set_wavelet(self, wavelet=None):
        _capi.set_wavelet(self.ctx, wavelet)

    def estimate_adjoint_basis(self, gamma=1e-12, relative=True, max_iter=200, tol=1e-14, fit_target=None):
        """B+ (Sec. 3.3).  fit_target: with a relative gamma, divide gamma by 100 (down to 1e-16)
        until the fit residual max |B B+ - I| is at most fit_target (the Gram matrix of many
        widely spaced frequencies is ill-conditioned and needs less regularisation)."""
        basis = torch.empty((self.nt, 2 * self.nf), dtype=torch.float64, device=self.device)
        while True:
            fit, its = _capi.estimate_adjoint_basis(self.dt, self.nt, self.freqs, self.f0, gamma, int(relative),
                                                    max_iter, tol, _ptr(basis), _stream())
            if fit_target is None or not relative or fit <= fit_target or gamma <= 1e-16 * 1.0001:
                break
            gamma = max(gamma / 100.0, 1e-16)
        self.basis_gamma = gamma
        return basis, fit, its

    def adjoint_model(self, rho, rec, resid: torch.Tensor, basis: torch.Tensor):
        S = resid.shape[0]
        assert resid.dtype == torch.complex128 and resid.shape[1:] == (rec.n, self.nf)
        vol = torch.empty(self.volume_shape(S), dtype=self.cplx, device=self.device)
        _capi.adjoint_model(self.ctx, _ptr(self._model(rho)), rec, S, _ptr(resid.contiguous()), _ptr(basis),
                            _ptr(vol), _stream())
        return vol

    def gradient(self, rho, Evol, Vvol, wrt="lnrho", out=None):
        if out is None:
            out = torch.zeros(self.model_shape, dtype=self.real, device=self.device)
        self._model(out)
        vs = self.volume_shape(Evol.shape[0])
        if tuple(Evol.shape) != vs or tuple(Vvol.shape) != vs:
            raise ValueError(f"volumes of shape {vs} expected")
        _capi.gradient(self.ctx, _ptr(self._model(rho)), _ptr(Evol), _ptr(Vvol), Evol.shape[0],
                       1 if wrt == "lnrho" else 0, _ptr(out), _stream())
        return out

    def td_plan(self, n_src, n_rec, budget_bytes=0, segment=0):
        """(segment length, workspace bytes) of gradient_td; budget_bytes > 0 picks the
        segment with the fewest replayed forward steps that fits it."""
        return _capi.td_plan(self.ctx, n_src, n_rec, budget_bytes, segment)

    def gradient_td(self, rho, src, rec, resid: torch.Tensor, wrt="lnrho", segment=0, budget_bytes=None, out=None,
                    work=None):
        """Gradient by the time-domain adjoint (appendix): the reversed-time run of the
        scheme driven by the residual, correlated with the forward field replayed from
        checkpoints.  budget_bytes: workspace limit (default: 80% of the free memory);
        work: a uint8 device tensor to use as the workspace (else one is allocated)."""
        S = src.n
        if resid.dtype != torch.complex128 or tuple(resid.shape) != (S, rec.n, self.nf):
            raise ValueError(f"resid of shape {(S, rec.n, self.nf)} complex128 expected")
        if out is None:
            out = torch.zeros(self.model_shape, dtype=self.real, device=self.device)
        self._model(out)
        cached = getattr(self, "_td_work", None)
        if budget_bytes is None:     # the engine's own cached workspace counts as free
            held = cached.numel() if (cached is not None and work is None) else 0
            budget_bytes = int(0.8 * (torch.cuda.mem_get_info(self.device)[0] + held))
        seg, nbytes = _capi.td_plan(self.ctx, S, rec.n, budget_bytes if segment <= 0 else 0, segment)
        if work is None:
            if cached is not None and cached.numel() >= nbytes + 256:
                work = cached
            else:
                self._td_work = cached = None
                work = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
                self._td_work = work     # kept for the next call (released by close())
        off = (-work.data_ptr()) % 256
        if work.dtype != torch.uint8 or not work.is_cuda or work.numel() < nbytes + off:
            raise ValueError(f"workspace of at least {nbytes + off} bytes (uint8, on the device) expected")
        _capi.gradient_td(self.ctx, _ptr(self._model(rho)), src, rec, _ptr(resid.contiguous()), seg,
                          1 if wrt == "lnrho" else 0, _ptr(out), ctypes_void(work.data_ptr() + off), nbytes,
                          _stream())
        self.last_td = dict(segment=seg, workspace_bytes=nbytes)
        return out

    def check(self):
        _capi.check(self.ctx, _stream())

    def set_copy_fault(self, extra_bytes=16):
        """Test hook (csem_set_copy_fault): the bulk-copy kernels' first stage waits for
        extra_bytes that never come, so their bounded waits run out; 0 turns it off."""
        _capi.set_copy_fault(self.ctx, extra_bytes)

    def set_launch(self, kz_h=4, mb_h=4, kz_e=4, mb_e=4, fused_kz=0, flush_mode=0, block=16, vec_h=0, vec_e=0,
                   tma_h=0, tma_e=0, lean_h=0, lean_e=0, onepass=None, wspec=None, wave=None):
        """Pins a launch configuration (see csem_set_launch); launch_config() then reports it.
        onepass = (z planes, rows per block, resident blocks per SM) selects the fused
        one-pass step kernel (code 10000 + planes * 100 + rows * 10 + blocks); wspec = (z planes,
        rows per block, resident blocks per SM) the warp-specialised fused step (code 30000 + ...);
        wave = (lag in z blocks, z planes, resident blocks per SM) the wave-ordered step
        (code 50000 + lag * 100 + planes * 10 + blocks)."""
        if onepass:
            kz, by, mb = onepass
            fused_kz = 10000 + kz * 100 + by * 10 + mb
        elif wspec:
            kz, by, mb = wspec
            fused_kz = 30000 + kz * 100 + by * 10 + mb
        elif wave:
            lag, kz, mb = wave
            fused_kz = 50000 + lag * 100 + kz * 10 + mb
        _capi.set_launch(self.ctx, kz_h, mb_h, kz_e, mb_e, fused_kz, flush_mode, block, vec_h, vec_e, tma_h, tma_e,
                         lean_h, lean_e)
        self.kz = (kz_h * 16 + mb_h + 256 * vec_h + 1024 * tma_h + 8192 * lean_h,
                   kz_e * 16 + mb_e + 256 * vec_e + 1024 * tma_e + 8192 * lean_e,
                   block * 4 + flush_mode, fused_kz)

    def flush_block(self) -> int:
        """Snapshots per damped-transform flush chosen by the autotuner (16 if untuned)."""
        return self.kz[2] // 4 if self.kz else 16

    def launch_config(self) -> dict:
        if not self.kz:
            return {}
        h, e, f, fz = self.kz
        def one(code):
            if code >= 8192:
                return {"kernel": "lean", "cells_per_thread": code // 8192, "z_planes": (code % 256) // 16,
                        "blocks_per_sm": code % 16}
            if code >= 1024:
                return {"kernel": "bulk-copy staged", "rows_per_block": code // 1024, "z_planes": (code % 1024) // 16}
            return {"kernel": "four cells per thread" if code >= 256 else "one cell per thread",
                    "z_planes": (code % 256) // 16, "blocks_per_sm": code % 16}
        if fz >= 50000:
            c = fz - 50000
            step = {"kernel": "wave-ordered H+E", "lag": c // 100, "z_planes": (c // 10) % 10,
                    "blocks_per_sm": c % 10}
        elif fz >= 10000:
            c = fz - (30000 if fz >= 30000 else 10000)
            step = {"kernel": "fused warp-specialised H+E" if fz >= 30000 else "fused one-pass H+E",
                    "z_planes": c // 100, "rows_per_block": (c // 10) % 10, "blocks_per_sm": c % 10}
        elif fz:
            step = {"kernel": "fused H+E", "z_planes": fz}
        else:
            step = {"kernel": "split", "h": one(h), "e": one(e)}
        return {"step": step, "flush": {"snapshots": f // 4, "kernel": "bulk-copy" if f % 2 == 1 else "register",
                                        "overlapped": f % 4 >= 2}}


def misfit(d_obs: torch.Tensor, d_syn: torch.Tensor, weight: Optional[torch.Tensor] = None):
    """phi = 1/2 sum |w (d_obs - d_syn)|^2 and resid = w^2 (d_obs - d_syn), on the device."""
    d_obs = d_obs.contiguous()
    d_syn = d_syn.contiguous()
    resid = torch.empty_like(d_syn)
    phi = torch.empty((), dtype=torch.float64, device=d_syn.device)
    _capi.misfit(d_syn.numel(), _ptr(d_obs), _ptr(d_syn), _ptr(weight.contiguous()) if weight is not None else None,
                 _ptr(resid), _ptr(phi), _stream())
    return phi, resid
