"""The forward solve as a torch.autograd.Function whose backward is the
adjoint time stepping (Sec. 3.2-3.3) plus the gradient kernel (Sec. 3.1, 3.5).

forward(ln_rho)  -> d_syn [S, R, F] complex128, keeping the normalised E volumes
backward(g)      -> d L / d ln_rho
(or, with route="td", the appendix's time-domain adjoint in backward and no volumes kept)

PyTorch hands a real loss's gradient with respect to a complex output as
g = dL/dRe(d) + i dL/dIm(d).  For L = 1/2 |d_obs - d_syn|^2 this is
-(d_obs - d_syn), so the weighted residual that drives the adjoint is r = -g;
any other real loss works the same way (dL = Re(conj(g) dd)).

Batches larger than `chunk` sources are processed chunk by chunk; the forward
volumes of a chunk are recomputed in backward when `recompute` is set, so the
device holds only one chunk's volumes at a time.
"""
from __future__ import annotations

import torch

from .engine import Engine


class CsemForward(torch.autograd.Function):
    @staticmethod
    def forward(ctx, ln_rho, engine: Engine, src, rec, basis, chunk, recompute, route="basis"):
        rho = torch.exp(ln_rho).to(engine.real).contiguous()
        S = src.n
        chunk = chunk or S
        ds, vols = [], []
        tol = engine.early_stop_tol
        if route == "td" and tol > 0:
            engine.set_early_stop(0.0)     # the gradient belongs to the full run: so must the data
        for s0 in range(0, S, chunk):
            sub = src.subset(list(range(s0, min(S, s0 + chunk))))
            if route == "td" or (recompute and chunk < S):
                ds.append(engine.fwd_model(rho, sub, rec))
                vols.append(None)
            else:
                d, v = engine.fwd_model(rho, sub, rec, keep_volume=True)
                ds.append(d)
                vols.append(v)
        if route == "td" and tol > 0:
            engine.set_early_stop(tol)
        ctx.engine, ctx.src, ctx.rec, ctx.basis, ctx.chunk, ctx.route = engine, src, rec, basis, chunk, route
        ctx.vols = vols
        ctx.in_dtype = ln_rho.dtype
        ctx.save_for_backward(rho)
        return torch.cat(ds, dim=0)

    @staticmethod
    def backward(ctx, grad_d):
        (rho,) = ctx.saved_tensors
        eng = ctx.engine
        S = ctx.src.n
        g = torch.zeros(eng.model_shape, dtype=eng.real, device=rho.device)
        resid = (-grad_d).to(torch.complex128).contiguous()
        for ci, s0 in enumerate(range(0, S, ctx.chunk)):
            idx = list(range(s0, min(S, s0 + ctx.chunk)))
            if ctx.route == "td":      # time-domain adjoint: replays the forward itself (appendix)
                eng.gradient_td(rho, ctx.src.subset(idx), ctx.rec, resid[s0:s0 + len(idx)].contiguous(), out=g)
                continue
            E = ctx.vols[ci]
            if E is None:
                _, E = eng.fwd_model(rho, ctx.src.subset(idx), ctx.rec, keep_volume=True)
            V = eng.adjoint_model(rho, ctx.rec, resid[s0:s0 + len(idx)].contiguous(), ctx.basis)
            eng.gradient(rho, E, V, wrt="lnrho", out=g)
            del E, V
        ctx.vols = None
        return g.to(ctx.in_dtype), None, None, None, None, None, None, None


def forward_data(ln_rho, engine, src, rec, basis, chunk=None, recompute=False, route="basis"):
    """d_syn = F(ln rho) with the adjoint-state gradient attached.  route: "basis" (Sec. 3.2-3.3:
    forward volumes kept, adjoint run from the basis estimate) or "td" (appendix: the forward
    keeps no volumes and backward runs the time-domain adjoint with checkpointed replay; basis
    may be None).  Without a gradient to attach (grad mode off, or ln_rho not requiring one)
    the runs keep no volumes, so the engine's early end of data runs (Engine.set_early_stop)
    applies."""
    if not (torch.is_grad_enabled() and ln_rho.requires_grad):
        rho = torch.exp(ln_rho).to(engine.real).contiguous()
        S = src.n
        chunk = chunk or S
        return torch.cat([engine.fwd_model(rho, src.subset(list(range(s0, min(S, s0 + chunk)))), rec)
                          for s0 in range(0, S, chunk)], dim=0)
    if route not in ("basis", "td"):
        raise ValueError("route is 'basis' or 'td'")
    return CsemForward.apply(ln_rho, engine, src, rec, basis, chunk, recompute, route)
