"""Reference outer inversion loop (test infrastructure, FP64 numpy; only the
tests, the smoke check and the bench's CPU baseline may use it).

Follows Sec. 3.5 ("The final algorithm") in its order:
  phi(m) = phi_d(m) + beta phi_m(m), m = ln(rho) on the free cells;
  phi_m = 1/2 || grad^alpha (m - m_ref) ||^2 with the first-order differences
  alpha_x d/dx, alpha_y d/dy, alpha_z d/dz between neighbouring cells (divided by
  the distance of their centres; only pairs of two free cells count);
  the descent direction from l-BFGS (two-loop recursion, memory `memory`),
  the step from a backtracking line search (sufficient decrease), and l-BFGS
  restarted from the steepest-descent direction after the first line-search
  failure; m kept inside [m_min, m_max] by projection; data within an offset
  `mute` of the source weighted out of phi_d (Sec. 4 examples).

Readings where the paper does not fix the details (also listed in the design
notes): beta decreases geometrically, beta_k = beta_0 * cool^k; the first
trial step of a steepest-descent iteration moves the largest cell by `step0`
in ln(rho), an l-BFGS iteration tries the unit step; backtracking halves the
step up to `max_backtracks` times with c1 = 1e-4; curvature pairs with
s.y <= 0 are not stored; a failed steepest-descent search ends the loop.
"""
from __future__ import annotations

import numpy as np

from . import fdtd


def centre_spacings(nodes):
    """Distances between neighbouring cell centres along one axis."""
    c = 0.5 * (nodes[1:] + nodes[:-1])
    return np.diff(c)


def tikhonov(m, m_ref, free, xn, yn, zn, alpha):
    """phi_m = 1/2 sum over axes a and neighbouring free pairs (p, q) of
    (alpha_a (dm_q - dm_p) / dc_a)^2 with dm = m - m_ref; returns (phi_m, gradient).

    m, m_ref, free: (nz, ny, nx) or (2, nz, ny, nx) (VTI, each part regularised alone).
    """
    dm = np.asarray(m, float) - np.asarray(m_ref, float)
    free = np.asarray(free, bool)
    lead = dm.ndim - 3
    grad = np.zeros_like(dm)
    phi = 0.0
    for axis, (nodes, a) in enumerate(((zn, alpha[2]), (yn, alpha[1]), (xn, alpha[0]))):
        ax = lead + axis
        dc = centre_spacings(np.asarray(nodes, float))
        shape = [1] * dm.ndim
        shape[ax] = dc.size
        dc = dc.reshape(shape)
        n = dm.shape[ax]
        lo = [slice(None)] * dm.ndim
        hi = [slice(None)] * dm.ndim
        lo[ax] = slice(0, n - 1)
        hi[ax] = slice(1, n)
        lo, hi = tuple(lo), tuple(hi)
        pair = free[lo] & free[hi]
        diff = np.where(pair, a * (dm[hi] - dm[lo]) / dc, 0.0)
        phi += 0.5 * float(np.sum(diff ** 2))
        flux = a * diff / dc
        grad[hi] += flux
        grad[lo] -= flux
    return phi, grad


def mute_weights(src, rec, n_freq, offset):
    """W[s, r, k] = 0 where the horizontal source-receiver offset is below `offset`, else 1."""
    dx = rec.x[None, :] - src.x[:, None]
    dy = rec.y[None, :] - src.y[:, None]
    w = (np.hypot(dx, dy) >= offset).astype(float)
    return np.repeat(w[:, :, None], n_freq, axis=2)


class DataTerm:
    """phi_d and its gradient in m = ln(rho) on the free cells, from the FP64 oracle."""

    def __init__(self, pb, src, rec, d_obs, weights, rho_fixed, free):
        self.pb, self.src, self.rec, self.d_obs, self.w = pb, src, rec, d_obs, weights
        self.rho_fixed = np.asarray(rho_fixed, float)
        self.free = np.asarray(free, bool)
        self.Bp, _ = fdtd.adjoint_basis(pb, 1e-12)

    def model(self, m):
        return np.where(self.free, np.exp(m), self.rho_fixed)

    def value(self, m):
        d = fdtd.forward(self.pb, self.model(m), self.src, self.rec)
        return fdtd.misfit(self.d_obs, d, self.w)[0]

    def __call__(self, m):
        rho = self.model(m)
        d, E = fdtd.forward(self.pb, rho, self.src, self.rec, keep_volume=True)
        phi, r = fdtd.misfit(self.d_obs, d, self.w)
        V = fdtd.adjoint(self.pb, rho, self.rec, r, self.Bp)
        g = fdtd.gradient(self.pb, rho, E, V, wrt="lnrho")
        return phi, np.where(self.free, g, 0.0)


def lbfgs_direction(g, pairs):
    """-H g by the two-loop recursion over the stored (s, y) pairs, oldest first;
    H0 = (s.y / y.y) I from the newest pair."""
    q = g.copy()
    coefs = []
    for s, y in reversed(pairs):
        rho_i = 1.0 / float(np.sum(y * s))
        a = rho_i * float(np.sum(s * q))
        coefs.append((a, rho_i, s, y))
        q -= a * y
    if pairs:
        s, y = pairs[-1]
        q *= float(np.sum(s * y)) / float(np.sum(y * y))
    for a, rho_i, s, y in reversed(coefs):
        b = rho_i * float(np.sum(y * q))
        q += (a - b) * s
    return -q


def invert(objective, m0, free, iters, m_min, m_max, memory=5, step0=0.5, max_backtracks=6,
           beta0=0.01, cool=0.7, reg=None):
    """Minimise phi = phi_d + beta_k phi_m over m (free cells only).

    objective(m) -> (phi_d, grad phi_d) and objective.value(m) -> phi_d;
    reg(m) -> (phi_m, grad phi_m), or None for no regularisation.
    Returns (m, history) with one record per iteration.
    """
    free = np.asarray(free, bool)
    m = np.clip(np.asarray(m0, float), m_min, m_max)
    pairs = []
    history = []
    restarted = False
    g_prev = m_prev = None
    for it in range(iters):
        beta = beta0 * cool ** it

        def total(mm, with_grad):
            pd, gd = objective(mm) if with_grad else (objective.value(mm), None)
            pm, gm = reg(mm) if reg is not None else (0.0, np.zeros_like(mm))
            g = None if gd is None else np.where(free, gd + beta * gm, 0.0)
            return pd + beta * pm, pd, pm, g

        phi, pd, pm, g = total(m, True)
        if g_prev is not None:
            s, y = m - m_prev, g - g_prev
            if float(np.sum(s * y)) > 0.0:
                pairs = (pairs + [(s, y)])[-memory:]

        def search(d, use_sd):
            slope = float(np.sum(d * g))
            step = step0 / max(float(np.max(np.abs(d))), 1e-300) if use_sd else 1.0
            for _ in range(max_backtracks + 1):
                m_try = np.clip(m + step * d, m_min, m_max)
                if total(m_try, False)[0] <= phi + 1e-4 * step * slope:
                    return True, step, m_try
                step *= 0.5
            return False, 0.0, m

        use_sd = not pairs
        d = -g if use_sd else lbfgs_direction(g, pairs)
        if float(np.sum(d * g)) >= 0.0:          # not a descent direction: steepest descent
            d, use_sd = -g, True
        ok, step, m_new = search(d, use_sd)
        if not ok and not use_sd and not restarted:
            restarted = True                     # first failure: restart from steepest descent
            pairs = []
            use_sd = True
            ok, step, m_new = search(-g, True)
        history.append(dict(iter=it, phi=phi, phi_d=pd, phi_m=pm, beta=beta, step=step,
                            direction="steepest" if use_sd else "lbfgs", accepted=ok))
        if not ok:
            break
        g_prev, m_prev = g, m
        m = m_new
    return m, history
