"""Outer inversion loop (Sec. 3.5) on the device, driven by the adjoint-state
gradient through autograd.

  phi(m) = phi_d(m) + beta_k phi_m(m),  m = ln(rho) on the free cells;
  phi_d = 1/2 sum |W (d_obs - d(m))|^2 (W: data weights, e.g. an offset mute);
  phi_m = 1/2 || grad^alpha (m - m_ref) ||^2, first-order differences
          alpha_a (m_q - m_p) / (distance of the centres) between neighbouring
          free cells along each axis a;
  the direction from l-BFGS (two-loop recursion), the step from a backtracking
  search with sufficient decrease; after the first failed l-BFGS search the
  loop restarts from the steepest-descent direction, a later failure ends it;
  m stays inside [m_min, m_max] (m_max at most ln of the resistivity that fixes
  the context's CFL step, above which the stepping would not be stable).

Choices where the paper leaves the details open: beta_k = beta_0 cool^k; a
steepest-descent trial step moves the largest cell by `step0` in ln(rho), an
l-BFGS trial is the unit step; up to `max_backtracks` halvings, c1 = 1e-4;
pairs with s.y <= 0 are dropped.
"""
from __future__ import annotations

import math
from typing import Optional

import numpy as np
import torch

from .autograd import forward_data


def centre_distances(nodes) -> torch.Tensor:
    c = 0.5 * (np.asarray(nodes[1:], float) + np.asarray(nodes[:-1], float))
    return torch.as_tensor(np.diff(c))


class Tikhonov:
    """phi_m = 1/2 sum_a alpha_a^2 sum_{free pairs along a} ((dm_q - dm_p) / dc_a)^2, dm = m - m_ref."""

    def __init__(self, xn, yn, zn, free: torch.Tensor, m_ref: torch.Tensor, alpha=(1.0, 1.0, 0.1)):
        dev = free.device
        self.m_ref = m_ref
        self.terms = []
        lead = free.dim() - 3
        for axis, nodes, a in ((lead + 2, xn, alpha[0]), (lead + 1, yn, alpha[1]), (lead, zn, alpha[2])):
            dc = centre_distances(nodes).to(device=dev, dtype=torch.float64)
            shape = [1] * free.dim()
            shape[axis] = dc.numel()
            n = free.shape[axis]
            pair = free.narrow(axis, 1, n - 1) & free.narrow(axis, 0, n - 1)
            self.terms.append((axis, float(a), dc.reshape(shape), pair))

    def __call__(self, m: torch.Tensor) -> torch.Tensor:
        dm = m - self.m_ref
        phi = m.new_zeros(())
        for axis, a, dc, pair in self.terms:
            n = dm.shape[axis]
            slope = (dm.narrow(axis, 1, n - 1) - dm.narrow(axis, 0, n - 1)) / dc
            phi = phi + 0.5 * a * a * torch.sum(torch.where(pair, slope, torch.zeros_like(slope)) ** 2)
        return phi


class Inversion:
    """Minimises phi over m = ln(rho) on the free cells with the engine's forward
    and adjoint runs (one gradient per iteration, one forward per trial step).
    route: "basis" (Sec. 3.2-3.3) or "td" (the appendix's time-domain adjoint)."""

    def __init__(self, engine, src, rec, d_obs: torch.Tensor, rho_fixed, free, basis: torch.Tensor,
                 weights: Optional[torch.Tensor] = None, m_ref=None, alpha=(1.0, 1.0, 0.1), xn=None, yn=None,
                 zn=None, beta0=0.01, cool=0.7, m_min=math.log(0.1), m_max=math.log(1e3), memory=5, step0=0.5,
                 max_backtracks=6, chunk=None, recompute=False, route="basis"):
        dev = engine.device
        self.eng, self.src, self.rec, self.basis = engine, src, rec, basis
        self.d_obs = d_obs.to(dev)
        self.w = None if weights is None else torch.as_tensor(weights, dtype=torch.float64, device=dev)
        self.free = torch.as_tensor(np.asarray(free, bool), device=dev)
        self.ln_fixed = torch.log(torch.as_tensor(np.asarray(rho_fixed, float), dtype=torch.float64, device=dev))
        self.m_ref = self.ln_fixed.clone() if m_ref is None else \
            torch.as_tensor(np.asarray(m_ref, float), dtype=torch.float64, device=dev)
        self.reg = Tikhonov(xn, yn, zn, self.free, self.m_ref, alpha) if xn is not None else None
        self.beta0, self.cool = beta0, cool
        self.m_min = m_min
        self.m_max = min(m_max, math.log(engine.rho_max))
        self.memory, self.step0, self.max_backtracks = memory, step0, max_backtracks
        self.chunk, self.recompute, self.route = chunk, recompute, route

    def _phi_d(self, m: torch.Tensor) -> torch.Tensor:
        ln_rho = torch.where(self.free, m, self.ln_fixed)
        d = forward_data(ln_rho, self.eng, self.src, self.rec, self.basis, chunk=self.chunk,
                         recompute=self.recompute, route=self.route)
        res = self.d_obs - d
        if self.w is not None:
            res = res * self.w
        return 0.5 * torch.sum(res.real ** 2 + res.imag ** 2)

    def objective(self, m: torch.Tensor, beta: float, with_grad: bool):
        """(phi, phi_d, phi_m, gradient on the free cells or None)."""
        if not with_grad:
            with torch.no_grad():
                pd = self._phi_d(m)
                pm = self.reg(m) if self.reg is not None else m.new_zeros(())
            return float(pd + beta * pm), float(pd), float(pm), None
        mm = m.detach().clone().requires_grad_(True)
        pd = self._phi_d(mm)
        pm = self.reg(mm) if self.reg is not None else mm.new_zeros(())
        total = pd + beta * pm
        total.backward()
        g = torch.where(self.free, mm.grad, torch.zeros_like(mm.grad))
        return float(total.detach()), float(pd.detach()), float(pm.detach()), g

    @staticmethod
    def _dot(a, b) -> float:
        return float(torch.sum(a * b))

    def _direction(self, g, pairs):
        """-H g, two-loop recursion; H0 = (s.y / y.y) I from the newest pair."""
        q = g.clone()
        saved = []
        for s, y in reversed(pairs):
            r = 1.0 / self._dot(y, s)
            a = r * self._dot(s, q)
            saved.append((a, r, s, y))
            q -= a * y
        s, y = pairs[-1]
        q *= self._dot(s, y) / self._dot(y, y)
        for a, r, s, y in reversed(saved):
            q += (a - r * self._dot(y, q)) * s
        return -q

    def run(self, m0: torch.Tensor, iters: int):
        """Returns (m, history); m0 = ln(rho) of the start model (its fixed cells are ignored)."""
        m = torch.clamp(torch.as_tensor(m0, dtype=torch.float64, device=self.eng.device), self.m_min, self.m_max)
        pairs, history = [], []
        restarted = False
        g_prev = m_prev = None
        for it in range(iters):
            beta = self.beta0 * self.cool ** it
            phi, pd, pm, g = self.objective(m, beta, True)
            if g_prev is not None:
                s, y = m - m_prev, g - g_prev
                if self._dot(s, y) > 0.0:
                    pairs = (pairs + [(s, y)])[-self.memory:]

            def search(d, steepest):
                slope = self._dot(d, g)
                step = self.step0 / max(float(d.abs().max()), 1e-300) if steepest else 1.0
                for _ in range(self.max_backtracks + 1):
                    trial = torch.clamp(m + step * d, self.m_min, self.m_max)
                    if self.objective(trial, beta, False)[0] <= phi + 1e-4 * step * slope:
                        return True, step, trial
                    step *= 0.5
                return False, 0.0, m

            steepest = not pairs
            d = -g if steepest else self._direction(g, pairs)
            if self._dot(d, g) >= 0.0:
                d, steepest = -g, True
            ok, step, m_new = search(d, steepest)
            if not ok and not steepest and not restarted:
                restarted, pairs, steepest = True, [], True
                ok, step, m_new = search(-g, True)
            history.append(dict(iter=it, phi=phi, phi_d=pd, phi_m=pm, beta=beta, step=step,
                                direction="steepest" if steepest else "lbfgs", accepted=ok))
            if not ok:
                break
            g_prev, m_prev = g, m
            m = m_new
        return m, history
