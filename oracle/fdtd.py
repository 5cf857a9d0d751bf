"""FP64 oracle of the fictitious-wave forward / adjoint / gradient path.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Each function follows
a passage of the paper (Yang, "3D fictitious wave domain CSEM inversion by
adjoint source estimation"):

  Sec. 2, Eq. 2-3  sigma = 2 w0 eps, J' = k J, E' = E, k = sqrt(-i w / 2 w0)
  Sec. 2, Eq. 4    fictitious-time Maxwell system, leap-frog on a staggered grid
  Sec. 2, Eq. 6    on-the-fly damped transform, no dt factor, n = 0..nt-1
  Sec. 2           early end of a forward run once the receiver spectra stop changing
  Sec. 3.1, Eq. 7  misfit 1/2 ||W (d - R u)||^2
  Sec. 3.1         gradient -Re sum_s sum_w conj(v_E) . E, scaled by cell volume
  Sec. 3.2, Eq. 14 conj(v) from the same engine with conjugated residual sources
  Sec. 3.3         adjoint time series from the basis functions
  Sec. 3.5         m = ln(rho): dphi/dm = -(1/rho) dphi/dsigma
  Appendix          time-domain adjoint: the same scheme run in reversed time,
                   driven at the receivers by the transpose of the data functional,
                   and the gradient as the time correlation of the two fields
  Sec. 2, Sec. 3.1 Eq. 15  VTI medium: sigma_h = sigma_xx = sigma_yy on the x and y edges,
                   sigma_v = sigma_zz on the z edges; dphi/dsigma_h collects the x and y
                   edges, dphi/dsigma_v the z edges

Readings where the paper is silent (each listed in the design notes):
  * second-order Yee stencil (order 2), or four-point staggered differences exact
    for cubics on the non-uniform nodes, two-point rows next to the outer boundary
    (order 4); tangential E = 0 on the outer boundary;
  * cell-centred rho; edge conductivity = volume-weighted mean of the (up to
    four) cells sharing the edge; gradient mapped back by the transpose;
  * CFL step dt = s / (v_max sqrt(max_cells sum 1/h^2)), v = sqrt(2 w0 rho / mu0),
    rho_max frozen for a problem; nt = ceil(35 / (a_min dt)) unless given;
  * CPML: d = d0 (xi/L)^2, d0 = -3 v_pml ln(R) / (2 L), R = 1e-6, kappa = 1,
    alpha = pi f0 (1 - xi/L), b = exp(-(d + alpha) dt), a = d (b - 1)/(d + alpha),
    profiles evaluated where each derivative lives;
  * E at t_n = n dt, H and J' at t_{n+1/2}; a unit impulse J'_0 = 1/dt forward;
    E(w_k) = k_k Ehat_k / What_k with What_k the transform of the wavelet at
    the injection times;
  * point sources / receivers: trilinear weights on the component's lattice,
    injection = transpose of sampling divided by the edge's dual volume;
  * adjoint: target spectrum c_k = k_k conj(r_k) / dt for an E residual r
    (an electric current conj(r) at the receiver), conj(v) = dt * Vhat_k.
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass
from typing import Optional

import numpy as np

from . import basis as _basis
from ._build import build_oracle

MU0 = 4e-7 * np.pi
C_R = 1e-6          # CPML theoretical reflection
CFL_SAFETY = 0.99
DECAY_SPAN = 35.0   # nt covers exp(-35) of the slowest transform weight


# --------------------------------------------------------------------------
# grid, materials, time step
# --------------------------------------------------------------------------

def spacings(xn: np.ndarray):
    """Primal widths h_{i+1/2} = x_{i+1} - x_i (len n) and dual widths
    h~_i = (h_{i-1/2} + h_{i+1/2}) / 2 at nodes (len n+1, half cells at the ends)."""
    h = np.diff(xn)
    ht = np.empty(h.size + 1)
    ht[1:-1] = 0.5 * (h[:-1] + h[1:])
    ht[0] = 0.5 * h[0]
    ht[-1] = 0.5 * h[-1]
    return h, ht


def omega0(f0: float) -> float:
    return 2 * np.pi * f0


def wave_speed(rho, f0: float):
    """Fictitious speed 1/sqrt(mu0 eps) with eps = sigma / (2 w0)  (Eq. 2)."""
    return np.sqrt(2 * omega0(f0) * np.asarray(rho) / MU0)


def cfl_dt(xn, yn, zn, rho_max: float, f0: float, safety: float = CFL_SAFETY) -> float:
    hx, hy, hz = np.diff(xn), np.diff(yn), np.diff(zn)
    s = 1 / hz[:, None, None] ** 2 + 1 / hy[None, :, None] ** 2 + 1 / hx[None, None, :] ** 2
    return float(safety / (wave_speed(rho_max, f0) * np.sqrt(s.max())))


def fd_weights(x0: float, xs) -> np.ndarray:
    """Weights w with sum_i w_i f(xs_i) = f'(x0) for every polynomial f of degree < len(xs):
    the derivative of the Lagrange interpolant through the points (moment conditions
    sum_i w_i (xs_i - x0)^m = [m == 1], m = 0 .. len(xs) - 1)."""
    d = np.asarray(xs, float) - x0
    A = np.vander(d, d.size, increasing=True).T          # A[m, i] = d_i^m
    rhs = np.zeros(d.size)
    rhs[1] = 1.0
    return np.linalg.solve(A, rhs)


def staggered_weights(xn):
    """Fourth-order staggered difference weights on one non-uniform axis (Sec. 2: high-order
    differences on the non-uniform grid; the paper prints no coefficients).

    H rows (derivative at the half node p from the nodes p-1 .. p+2) and E rows (derivative
    at the node q from the half nodes q-2 .. q+1) are each the weights of fd_weights at
    their own point, so both are exact for cubics on any node spacing.  Rows whose four
    points would leave the lattice (the first and last half node, the nodes 1 and n-1)
    keep the two-point difference of the second-order scheme.
    Returns wh [n][4] (nodes p-1 .. p+2) and wn [n+1][4] (half nodes q-2 .. q+1).
    """
    xn = np.asarray(xn, float)
    n = xn.size - 1
    h, ht = spacings(xn)
    xh = 0.5 * (xn[1:] + xn[:-1])
    wh = np.zeros((n, 4))
    for p in range(n):
        if 1 <= p <= n - 2:
            wh[p] = fd_weights(xh[p], xn[p - 1:p + 3])
        else:
            wh[p, 1], wh[p, 2] = -1.0 / h[p], 1.0 / h[p]
    wn = np.zeros((n + 1, 4))
    for q in range(1, n):
        if 2 <= q <= n - 2:
            wn[q] = fd_weights(xn[q], xh[q - 2:q + 2])
        else:
            wn[q, 1], wn[q, 2] = -1.0 / ht[q], 1.0 / ht[q]
    return wh, wn


def cfl_dt_order4(xn, yn, zn, rho_max: float, f0: float, safety: float = CFL_SAFETY) -> float:
    """Leap-frog limit for the four-point scheme: dt = 2 s / (v sqrt(max_cells sum_a S_a^2)),
    S_a the largest absolute row sum of the weights touching the cell along axis a (the
    largest symbol of the staggered difference; two-point rows give 2/h, the Yee limit)."""
    S = []
    for g in (xn, yn, zn):
        wh, wn = staggered_weights(g)
        rh = np.abs(wh).sum(axis=1)
        rn = np.abs(wn).sum(axis=1)
        S.append(np.maximum(rh, np.maximum(rn[:-1], rn[1:])))
    sx, sy, sz = S
    tot = sz[:, None, None] ** 2 + sy[None, :, None] ** 2 + sx[None, None, :] ** 2
    return float(2.0 * safety / (wave_speed(rho_max, f0) * np.sqrt(tot.max())))


def default_nt(dt: float, freqs, f0: float) -> int:
    return int(math.ceil(DECAY_SPAN / (_basis.decay_rates(freqs, f0).min() * dt)))


def cell_volumes(xn, yn, zn):
    hx, hy, hz = np.diff(xn), np.diff(yn), np.diff(zn)
    return hz[:, None, None] * hy[None, :, None] * hx[None, None, :]


def _edge_sums(A):
    """Sum of a cell array over the cells sharing each E edge, per component.

    A has shape (nz, ny, nx); output (3, nz+1, ny+1, nx+1) on the node lattice.
    Ex(i,j,k) touches cells (i, j-1..j, k-1..k); Ey(i,j,k): (i-1..i, j, k-1..k);
    Ez(i,j,k): (i-1..i, j-1..j, k).
    """
    nz, ny, nx = A.shape
    P = np.zeros((nz + 2, ny + 2, nx + 2))
    P[1:-1, 1:-1, 1:-1] = A
    kk0, kk1 = slice(0, nz + 1), slice(1, nz + 2)
    jj0, jj1 = slice(0, ny + 1), slice(1, ny + 2)
    ii0, ii1 = slice(0, nx + 1), slice(1, nx + 2)
    sx = P[kk0, jj0, ii1] + P[kk1, jj0, ii1] + P[kk0, jj1, ii1] + P[kk1, jj1, ii1]
    sy = P[kk0, jj1, ii0] + P[kk1, jj1, ii0] + P[kk0, jj1, ii1] + P[kk1, jj1, ii1]
    sz = P[kk1, jj0, ii0] + P[kk1, jj1, ii0] + P[kk1, jj0, ii1] + P[kk1, jj1, ii1]
    return np.stack([sx, sy, sz])


def is_vti(rho) -> bool:
    """A model of shape (2, nz, ny, nx) holds (rho_h, rho_v) of a VTI medium."""
    return np.ndim(rho) == 4 and np.shape(rho)[0] == 2


def edge_conductivity(rho, xn, yn, zn):
    """sigma_e = sum_c V_c sigma_c / sum_c V_c over the cells sharing edge e.

    rho is (nz, ny, nx) for an isotropic medium or (2, nz, ny, nx) = (rho_h, rho_v)
    for a VTI medium (Sec. 2): the x and y edges average sigma_h = 1/rho_h, the z
    edges sigma_v = 1/rho_v.
    """
    V = cell_volumes(xn, yn, zn)
    rho = np.asarray(rho, float)
    if is_vti(rho):
        num = _edge_sums(V / rho[0])
        num[2] = _edge_sums(V / rho[1])[2]
    else:
        num = _edge_sums(V / rho)
    den = _edge_sums(V)
    out = np.zeros_like(num)
    np.divide(num, den, out=out, where=den > 0)
    return out


def edge_dual_volumes(xn, yn, zn):
    """dV of each E edge: its length times the dual face area, shape (3, nz+1, ny+1, nx+1)."""
    hx, hxt = spacings(xn)
    hy, hyt = spacings(yn)
    hz, hzt = spacings(zn)
    nx, ny, nz = hx.size, hy.size, hz.size
    out = np.zeros((3, nz + 1, ny + 1, nx + 1))
    out[0, :, :, :nx] = hzt[:, None, None] * hyt[None, :, None] * hx[None, None, :]
    out[1, :, :ny, :] = hzt[:, None, None] * hy[None, :, None] * hxt[None, None, :]
    out[2, :nz, :, :] = hz[:, None, None] * hyt[None, :, None] * hxt[None, None, :]
    return out


# --------------------------------------------------------------------------
# CPML (Komatitsch & Martin 2007) on the outer npml cells of each axis
# --------------------------------------------------------------------------

def cpml_profiles(xn, npml: int, dt: float, v_pml: float, f0: float):
    """Recursion coefficients (b, a) at half nodes and at nodes for one axis."""
    n = xn.size - 1
    xh = 0.5 * (xn[1:] + xn[:-1])

    def coeffs(p):
        b = np.zeros_like(p)
        a = np.zeros_like(p)
        if npml == 0:
            return b, a
        lo, hi = xn[npml], xn[n - npml]
        L_lo, L_hi = lo - xn[0], xn[n] - hi
        for side, L, xi in (("lo", L_lo, lo - p), ("hi", L_hi, p - hi)):
            m = xi > 0
            d0 = -3.0 * v_pml * np.log(C_R) / (2.0 * L)
            d = d0 * (xi[m] / L) ** 2
            alpha = np.pi * f0 * (1.0 - xi[m] / L)
            bb = np.exp(-(d + alpha) * dt)
            b[m] = bb
            a[m] = d * (bb - 1.0) / (d + alpha)
        return b, a

    bh, ah = coeffs(xh)
    bn, an = coeffs(xn.astype(np.float64))
    return bh, ah, bn, an


# --------------------------------------------------------------------------
# point sources / receivers
# --------------------------------------------------------------------------

def _lattice(xn, staggered: bool):
    return 0.5 * (xn[1:] + xn[:-1]) if staggered else xn


def trilinear_taps(xn, yn, zn, x, y, z, comp):
    """(k, j, i, weight) of the 8 lattice points around a point on comp's lattice.

    Ex lives at (x half nodes, y nodes, z nodes), Ey at (nodes, half, nodes),
    Ez at (nodes, nodes, half).  Weights are the tensor product of 1D linear
    interpolation weights; they sum to one.
    """
    out = []
    axes = []
    for ax_i, (g_nodes, p) in enumerate(((xn, x), (yn, y), (zn, z))):
        g = _lattice(g_nodes, staggered=(ax_i == comp))
        m = int(np.clip(np.searchsorted(g, p, side="right") - 1, 0, g.size - 2))
        t = (p - g[m]) / (g[m + 1] - g[m])
        if t < -1e-12 or t > 1 + 1e-12:
            raise ValueError("point outside the grid")
        axes.append(((m, 1.0 - t), (m + 1, t)))
    for (i, wi) in axes[0]:
        for (j, wj) in axes[1]:
            for (k, wk) in axes[2]:
                out.append((k, j, i, wi * wj * wk))
    return out


# --------------------------------------------------------------------------
# the ctypes bridge to the C stepper
# --------------------------------------------------------------------------

_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)


class _Model(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int)] + \
        [(n, _D) for n in ("ihx_h", "ihx_n", "ihy_h", "ihy_n", "ihz_h", "ihz_n",
                           "bx_h", "ax_h", "bx_n", "ax_n", "by_h", "ay_h", "by_n", "ay_n",
                           "bz_h", "az_h", "bz_n", "az_n")] + \
        [("cH", ctypes.c_double), ("cE", _D), ("order", ctypes.c_int)] + \
        [(n, _D) for n in ("wx_h", "wx_n", "wy_h", "wy_n", "wz_h", "wz_n")]


class _IO(ctypes.Structure):
    _fields_ = [("n_inj", ctypes.c_int), ("comp", _I), ("i", _I), ("j", _I), ("k", _I), ("emitter", _I),
                ("w", _D), ("series", _D),
                ("n_tap", ctypes.c_int), ("n_rec", ctypes.c_int),
                ("tcomp", _I), ("ti", _I), ("tj", _I), ("tk", _I), ("trec", _I), ("tw", _D), ("trace", _D),
                ("n_freq", ctypes.c_int), ("dft_re", _D), ("dft_im", _D), ("vol_re", _D), ("vol_im", _D),
                ("nt", ctypes.c_int)]


_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        _LIB = ctypes.CDLL(build_oracle())
        _LIB.orc_run.argtypes = [ctypes.POINTER(_Model), ctypes.POINTER(_IO), _D, _D, ctypes.c_int, ctypes.c_int]
        _LIB.orc_run.restype = ctypes.c_int
        _LIB.orc_set_threads.argtypes = [ctypes.c_int]
        _LIB.orc_set_threads.restype = None
        _LIB.orc_get_threads.argtypes = []
        _LIB.orc_get_threads.restype = ctypes.c_int
    return _LIB


def set_threads(n: int):
    """OpenMP threads of the C stepper (timing only)."""
    _lib().orc_set_threads(int(n))


def get_threads() -> int:
    return int(_lib().orc_get_threads())


def _dp(a):
    return None if a is None else a.ctypes.data_as(_D)


def _ip(a):
    return None if a is None else a.ctypes.data_as(_I)


# --------------------------------------------------------------------------
# problem set-up
# --------------------------------------------------------------------------

@dataclass
class Problem:
    xn: np.ndarray
    yn: np.ndarray
    zn: np.ndarray
    npml: int
    freqs: np.ndarray
    f0: float
    dt: float
    nt: int
    rho_max: float
    v_pml: float
    order: int = 2

    @property
    def shape_nodes(self):
        return (self.zn.size, self.yn.size, self.xn.size)

    @property
    def N(self):
        return self.zn.size * self.yn.size * self.xn.size

    @property
    def a(self):
        return _basis.decay_rates(self.freqs, self.f0)

    @property
    def k(self):
        """k_k = sqrt(-i w_k / (2 w0)) on the principal branch = (1 - i)/2 sqrt(w_k / w0)  (Eq. 3)."""
        return np.sqrt(-1j * 2 * np.pi * self.freqs / (2 * omega0(self.f0)))

    def dft_weights(self):
        """w_{n,k} = exp((-1 + i) a_k n dt), n = 0..nt-1  (Eq. 6)."""
        t = np.arange(self.nt)[:, None] * self.dt
        return np.exp((-1 + 1j) * self.a[None, :] * t)

    def wavelet_spectrum(self, wavelet):
        """What_k = sum_n wavelet_n exp((-1 + i) a_k (n + 1/2) dt)."""
        t = (np.arange(self.nt)[:, None] + 0.5) * self.dt
        return (wavelet[:, None] * np.exp((-1 + 1j) * self.a[None, :] * t)).sum(axis=0)

    def impulse(self):
        w = np.zeros(self.nt)
        w[0] = 1.0 / self.dt
        return w


def make_problem(xn, yn, zn, npml, freqs, f0=1.0, rho_max=1.0, nt=None, dt=None, v_pml=None,
                 order=2) -> Problem:
    if order not in (2, 4):
        raise ValueError("spatial order 2 or 4")
    if dt is None:
        dt = cfl_dt(xn, yn, zn, rho_max, f0) if order == 2 else cfl_dt_order4(xn, yn, zn, rho_max, f0)
    if nt is None:
        nt = default_nt(dt, freqs, f0)
    if v_pml is None:
        v_pml = float(wave_speed(rho_max, f0))
    return Problem(np.asarray(xn, float), np.asarray(yn, float), np.asarray(zn, float), int(npml),
                   np.asarray(freqs, float), float(f0), float(dt), int(nt), float(rho_max), float(v_pml),
                   int(order))


def problem_from_workload(wl, nt=None, order=2) -> Problem:
    return make_problem(wl.xn, wl.yn, wl.zn, wl.npml, wl.freqs, wl.f0, wl.rho_max,
                        nt if nt is not None else wl.nt, order=order)


class Stepper:
    """Holds the coefficient arrays of one (problem, model) pair and runs the C loop."""

    def __init__(self, pb: Problem, rho: np.ndarray):
        self.pb = pb
        xn, yn, zn = pb.xn, pb.yn, pb.zn
        self.hx, self.hxt = spacings(xn)
        self.hy, self.hyt = spacings(yn)
        self.hz, self.hzt = spacings(zn)
        sig_e = edge_conductivity(np.asarray(rho, float), xn, yn, zn)
        eps_e = sig_e / (2 * omega0(pb.f0))
        self.cE = np.zeros_like(sig_e)
        np.divide(pb.dt, eps_e, out=self.cE, where=eps_e > 0)
        self.cE = np.ascontiguousarray(self.cE)
        self.dV = edge_dual_volumes(xn, yn, zn)
        self.cpml = [cpml_profiles(g, pb.npml, pb.dt, pb.v_pml, pb.f0) for g in (xn, yn, zn)]
        inv = lambda v: np.ascontiguousarray(np.where(v > 0, 1.0 / np.where(v > 0, v, 1.0), 0.0))
        self._keep = [inv(self.hx), inv(self.hxt), inv(self.hy), inv(self.hyt), inv(self.hz), inv(self.hzt)]
        prof = []
        for (bh, ah, bn, an) in self.cpml:
            prof += [np.ascontiguousarray(v) for v in (bh, ah, bn, an)]
        self._keep += prof
        m = _Model()
        m.nx, m.ny, m.nz = xn.size - 1, yn.size - 1, zn.size - 1
        for name, arr in zip(("ihx_h", "ihx_n", "ihy_h", "ihy_n", "ihz_h", "ihz_n"), self._keep[:6]):
            setattr(m, name, _dp(arr))
        names = ("bx_h", "ax_h", "bx_n", "ax_n", "by_h", "ay_h", "by_n", "ay_n", "bz_h", "az_h", "bz_n", "az_n")
        for name, arr in zip(names, prof):
            setattr(m, name, _dp(arr))
        m.cH = pb.dt / MU0
        m.cE = _dp(self.cE)
        m.order = pb.order
        if pb.order == 4:
            ws = []
            for g in (xn, yn, zn):
                ws += [np.ascontiguousarray(w) for w in staggered_weights(g)]
            self._keep += ws
            for name, arr in zip(("wx_h", "wx_n", "wy_h", "wy_n", "wz_h", "wz_n"), ws):
                setattr(m, name, _dp(arr))
        self._model = m

    def new_state(self):
        N = self.pb.N
        return np.zeros(6 * N), np.zeros(12 * N)

    def run(self, fields, psi, n0, n1, inj=None, series=None, taps=None, n_rec=0, trace=None,
            dft=None, vol_re=None, vol_im=None):
        """Advance steps n0..n1-1.  inj: list of (comp,k,j,i,w,emitter); taps: (comp,k,j,i,w,rec)."""
        io = _IO()
        io.nt = self.pb.nt
        keep = []
        if inj:
            arr = np.array(inj, dtype=np.float64)
            ci = [np.ascontiguousarray(arr[:, c].astype(np.int32)) for c in (0, 3, 2, 1, 5)]
            wv = np.ascontiguousarray(arr[:, 4])
            ser = np.ascontiguousarray(np.asarray(series, np.float64))
            keep += ci + [wv, ser]
            io.n_inj = len(inj)
            io.comp, io.i, io.j, io.k, io.emitter = (_ip(c) for c in ci)
            io.w, io.series = _dp(wv), _dp(ser)
        if taps:
            arr = np.array(taps, dtype=np.float64)
            ci = [np.ascontiguousarray(arr[:, c].astype(np.int32)) for c in (0, 3, 2, 1, 5)]
            wv = np.ascontiguousarray(arr[:, 4])
            keep += ci + [wv]
            io.n_tap, io.n_rec = len(taps), n_rec
            io.tcomp, io.ti, io.tj, io.tk, io.trec = (_ip(c) for c in ci)
            io.tw = _dp(wv)
            io.trace = _dp(trace)
        if dft is not None:
            dre = np.ascontiguousarray(dft.real)
            dim = np.ascontiguousarray(dft.imag)
            keep += [dre, dim]
            io.n_freq = dft.shape[1]
            io.dft_re, io.dft_im = _dp(dre), _dp(dim)
            io.vol_re, io.vol_im = _dp(vol_re), _dp(vol_im)
        rc = _lib().orc_run(ctypes.byref(self._model), ctypes.byref(io), _dp(fields), _dp(psi), int(n0), int(n1))
        if rc != 0:
            raise RuntimeError("oracle stepper failed")
        return keep


# --------------------------------------------------------------------------
# forward / adjoint / misfit / gradient
# --------------------------------------------------------------------------

def point_taps(pb: Problem, pts, idx, scale_by_dV: Optional[np.ndarray] = None, tag=None):
    """Trilinear taps of point idx of `pts`; with dV given, weights are divided by it (injection)."""
    out = []
    c = int(pts.comp[idx])
    for (k, j, i, w) in trilinear_taps(pb.xn, pb.yn, pb.zn, pts.x[idx], pts.y[idx], pts.z[idx], c):
        if scale_by_dV is not None:
            w = w / scale_by_dV[c, k, j, i]
        out.append((c, k, j, i, w, idx if tag is None else tag))
    return out


def forward(pb: Problem, rho, src, rec, keep_volume=False, wavelet=None, nt_run=None, return_trace=False):
    """Receiver spectra E(x_r, w_k) for every source (and optionally the E volumes).

    Returns d [n_src, n_rec, n_freq] complex and, with keep_volume, the
    normalised volumes [n_src, 3, n_freq, nz+1, ny+1, nx+1] complex.
    """
    st = Stepper(pb, rho)
    nt = pb.nt if nt_run is None else nt_run
    wav = pb.impulse() if wavelet is None else np.asarray(wavelet, float)
    What = pb.wavelet_spectrum(wav)
    norm = pb.k / What
    W = pb.dft_weights()
    taps = []
    for r in range(rec.n):
        taps += point_taps(pb, rec, r)
    d = np.zeros((src.n, rec.n, pb.freqs.size), complex)
    vols = np.zeros((src.n, 3, pb.freqs.size) + pb.shape_nodes, complex) if keep_volume else None
    traces = np.zeros((src.n, rec.n, pb.nt))
    for s in range(src.n):
        fields, psi = st.new_state()
        inj = point_taps(pb, src, s, scale_by_dV=st.dV, tag=0)
        trace = np.zeros(rec.n * pb.nt)
        vre = vim = None
        if keep_volume:
            vre = np.zeros(3 * pb.freqs.size * pb.N)
            vim = np.zeros_like(vre)
        st.run(fields, psi, 0, nt, inj=inj, series=wav[None, :], taps=taps, n_rec=rec.n, trace=trace,
               dft=W if keep_volume else None, vol_re=vre, vol_im=vim)
        tr = trace.reshape(rec.n, pb.nt)
        traces[s] = tr
        d[s] = (tr @ W) * norm[None, :]
        if keep_volume:
            v = (vre + 1j * vim).reshape((3, pb.freqs.size) + pb.shape_nodes)
            vols[s] = v * norm[None, :, None, None, None]
    out = [d]
    if keep_volume:
        out.append(vols)
    if return_trace:
        out.append(traces)
    return out[0] if len(out) == 1 else tuple(out)


def forward_early_stop(pb: Problem, rho, src, rec, tol: float, chunk: int = 64, wavelet=None):
    """Receiver spectra with the early end of Sec. 2 (stepping ends once the frequency-domain
    field has reached its steady state, checked regularly during the run).

    All sources advance together in chunks of `chunk` steps.  After chunk c the running
    transform R_c[s, r, k] = sum_{n < chunk (c+1)} w_{k,n} E^n(x_r) is compared with R_{c-1};
    the run ends after the first chunk c >= 1 with |R_c - R_{c-1}| <= tol |R_c| for every
    source, receiver and frequency, or at nt.  Returns (d = alpha_k R, steps run).
    """
    st = Stepper(pb, rho)
    nt = pb.nt
    wav = pb.impulse() if wavelet is None else np.asarray(wavelet, float)
    norm = pb.k / pb.wavelet_spectrum(wav)
    W = pb.dft_weights()
    taps = []
    for r in range(rec.n):
        taps += point_taps(pb, rec, r)
    states = [st.new_state() for _ in range(src.n)]
    injs = [point_taps(pb, src, s, scale_by_dV=st.dV, tag=0) for s in range(src.n)]
    traces = [np.zeros(rec.n * nt) for _ in range(src.n)]
    prev = None
    n1 = 0
    for c in range((nt + chunk - 1) // chunk):
        n0, n1 = c * chunk, min(nt, (c + 1) * chunk)
        for s in range(src.n):
            fields, psi = states[s]
            st.run(fields, psi, n0, n1, inj=injs[s], series=wav[None, :], taps=taps, n_rec=rec.n,
                   trace=traces[s])
        R = np.stack([tr.reshape(rec.n, nt)[:, :n1] @ W[:n1] for tr in traces])
        if n1 == nt:
            break
        if prev is not None and np.all(np.abs(R - prev) <= tol * np.abs(R)):
            break
        prev = R
    return R * norm[None, None, :], n1


def volume_tail_factor(pb: Problem, chunk: int) -> np.ndarray:
    """Per frequency: what the rest of an endless run adds, relative to the last chunk's
    change, when the field stays as it was over that chunk -- the weights fall by the
    factor q = exp((-1 + i) a_k chunk dt) from one chunk to the next (Eq. 6), so the
    remainder is the geometric tail |q| / |1 - q| times the change."""
    q = np.exp((-1.0 + 1.0j) * pb.a * chunk * pb.dt)
    return np.abs(q) / np.abs(1.0 - q)


def _volume_converged(V, prev, prev_max, tol, floor_frac, tail):
    """The early end of runs with volumes (Sec. 2: stop once the frequency-domain field is
    steady): converged when, for every entry of every source, component and frequency k,
    the remainder estimated from its change since the previous check, tail[k] |V - prev|,
    is at most tol * max(|V|, floor_frac * prev_max[k]), with prev_max[k] the largest
    |prev| of frequency k -- entries of at least floor_frac of the largest are held to a
    relative bound, smaller ones to an absolute one.  The decision is taken in single
    precision.  V, prev: [n_src][3][n_freq][N] complex."""
    f32 = np.float32
    a = np.abs(V).astype(f32)
    d = np.abs(V - prev).astype(f32) * tail.astype(f32)[None, None, :, None]
    floor = f32(floor_frac) * prev_max.astype(f32)[None, None, :, None]
    return bool(np.all(d <= f32(tol) * np.maximum(a, floor)))


def _volumes_in_chunks(pb, st, runs, tol, chunk, floor_frac):
    """Steps every source's run (fields, psi, inj, series) together in chunks, with the
    volumetric transform; ends after the first chunk c >= 1 that passes _volume_converged,
    or at nt.  Returns the raw transforms [n_src][3][n_freq][N] and the steps run."""
    nt, nf, N = pb.nt, pb.freqs.size, pb.N
    W = pb.dft_weights()
    vre = [np.zeros(3 * nf * N) for _ in runs]
    vim = [np.zeros(3 * nf * N) for _ in runs]
    prev = None
    n1 = 0
    for c in range((nt + chunk - 1) // chunk):
        n0, n1 = c * chunk, min(nt, (c + 1) * chunk)
        for s, (fields, psi, inj, series, extra) in enumerate(runs):
            st.run(fields, psi, n0, n1, inj=inj, series=series, dft=W, vol_re=vre[s], vol_im=vim[s], **extra)
        V = np.stack([(vre[s] + 1j * vim[s]).reshape(3, nf, N) for s in range(len(runs))])
        if n1 == nt:
            break
        if prev is not None and tol > 0:
            prev_max = np.abs(prev).astype(np.float32).max(axis=(0, 1, 3))
            if _volume_converged(V, prev, prev_max, tol, floor_frac, volume_tail_factor(pb, chunk)):
                break
        prev = V
    return V, n1


def forward_volumes_early_stop(pb: Problem, rho, src, rec, tol: float, chunk: int = 64, floor_frac: float = 1e-4):
    """Forward run with volumes and the early end of Sec. 2 applied to the volumetric
    transform (all sources together, checked every `chunk` steps).  Returns (d, volumes,
    steps) with d and the volumes normalised as in forward()."""
    st = Stepper(pb, rho)
    wav = pb.impulse()
    norm = pb.k / pb.wavelet_spectrum(wav)
    W = pb.dft_weights()
    taps = []
    for r in range(rec.n):
        taps += point_taps(pb, rec, r)
    traces = [np.zeros(rec.n * pb.nt) for _ in range(src.n)]
    runs = []
    for s in range(src.n):
        fields, psi = st.new_state()
        runs.append((fields, psi, point_taps(pb, src, s, scale_by_dV=st.dV, tag=0), wav[None, :],
                     dict(taps=taps, n_rec=rec.n, trace=traces[s])))
    V, steps = _volumes_in_chunks(pb, st, runs, tol, chunk, floor_frac)
    d = np.stack([(tr.reshape(rec.n, pb.nt)[:, :steps] @ W[:steps]) * norm[None, :] for tr in traces])
    vols = V.reshape((src.n, 3, pb.freqs.size) + pb.shape_nodes) * norm[None, None, :, None, None, None]
    return d, vols, steps


def adjoint_early_stop(pb: Problem, rho, rec, resid, Bp, tol: float, chunk: int = 64, floor_frac: float = 1e-4):
    """adjoint() with the early end of Sec. 2 applied to the volumetric transform.
    Returns (conj(v) volumes, steps)."""
    st = Stepper(pb, rho)
    inj = []
    for r in range(rec.n):
        inj += point_taps(pb, rec, r, scale_by_dV=st.dV, tag=r)
    runs = []
    for s in range(resid.shape[0]):
        coef = pb.k[None, :] * np.conj(resid[s]) / pb.dt
        fields, psi = st.new_state()
        runs.append((fields, psi, inj, _basis.synthesize(Bp, coef), {}))
    V, steps = _volumes_in_chunks(pb, st, runs, tol, chunk, floor_frac)
    return pb.dt * V.reshape((resid.shape[0], 3, pb.freqs.size) + pb.shape_nodes), steps


def misfit(d_obs, d_syn, weights=None):
    """phi = 1/2 sum |W (d_obs - d_syn)|^2 and the weighted residual r = W^T W (d_obs - d_syn)  (Eq. 7)."""
    w = 1.0 if weights is None else weights
    res = d_obs - d_syn
    phi = 0.5 * float(np.sum(np.abs(w * res) ** 2))
    return phi, (w * w) * res


def adjoint_basis(pb: Problem, gamma_rel=1e-12):
    B = _basis.basis_matrix(pb.dt, pb.nt, pb.freqs, pb.f0)
    gamma = _basis.gamma_from_relative(B, gamma_rel)
    Bp = _basis.pinv_pushthrough(B, gamma)
    return Bp, _basis.fit_residual(B, Bp)


def adjoint(pb: Problem, rho, rec, resid, Bp, nt_run=None):
    """conj(v) volumes [n_src, 3, n_freq, nodes] for E residuals r at the receivers.

    The adjoint system (Eq. 14) is the forward system with an electric
    current conj(r) at each receiver; in the fictitious domain its spectrum is
    k_k conj(r_k) (Eq. 3).  The series injected is B+ [Re c; Im c] with
    c_k = k_k conj(r_k) / dt, so that the no-dt transform of the field times dt
    is conj(v).
    """
    st = Stepper(pb, rho)
    W = pb.dft_weights()
    n_src = resid.shape[0]
    out = np.zeros((n_src, 3, pb.freqs.size) + pb.shape_nodes, complex)
    for s in range(n_src):
        coef = pb.k[None, :] * np.conj(resid[s]) / pb.dt          # [n_rec, n_freq]
        series = _basis.synthesize(Bp, coef)                       # [n_rec, nt]
        inj = []
        for r in range(rec.n):
            inj += point_taps(pb, rec, r, scale_by_dV=st.dV, tag=r)
        fields, psi = st.new_state()
        vre = np.zeros(3 * pb.freqs.size * pb.N)
        vim = np.zeros_like(vre)
        st.run(fields, psi, 0, pb.nt if nt_run is None else nt_run, inj=inj, series=series, dft=W, vol_re=vre,
               vol_im=vim)
        out[s] = pb.dt * (vre + 1j * vim).reshape((3, pb.freqs.size) + pb.shape_nodes)
    return out


def gradient(pb: Problem, rho, Evol, Vvol, wrt="lnrho"):
    """Cell gradient of the misfit.

    Edge form (Sec. 3.1, isotropic): dphi/dsigma_e = -Re sum_s sum_k conj(v)_e E_e dV_e.
    Cell form: dphi/dsigma_c = sum_{e touching c} dphi/dsigma_e * V_c / sum_{c' at e} V_c'.
    ln rho (Sec. 3.5): dphi/dln(rho_c) = -sigma_c dphi/dsigma_c.
    VTI (Sec. 3.1, Eq. 15): dphi/dsigma_h collects the x and y edges of the cell,
    dphi/dsigma_v its z edges; the result is (2, nz, ny, nx) = (h, v).
    """
    dV = edge_dual_volumes(pb.xn, pb.yn, pb.zn)
    g_edge = -np.real(np.sum(Vvol * Evol, axis=(0, 2))) * dV         # [3, nodes]
    return _edge_to_cells(pb, np.asarray(rho, float), g_edge, wrt)


def _edge_to_cells(pb: Problem, rho, g_edge, wrt):
    """dphi/dsigma per edge [3, nodes] -> per cell (h, v parts for VTI), in sigma or ln rho."""
    xn, yn, zn = pb.xn, pb.yn, pb.zn
    V = cell_volumes(xn, yn, zn)
    den = _edge_sums(V)
    ratio = np.zeros_like(g_edge)
    np.divide(g_edge, den, out=ratio, where=den > 0)
    nz, ny, nx = V.shape
    # transpose of the edge averaging: each cell collects from its 12 edges
    gx = ratio[0]
    gy = ratio[1]
    gz = ratio[2]
    acc_h = np.zeros((nz, ny, nx))
    acc_v = np.zeros((nz, ny, nx))
    for dk in (0, 1):
        for dj in (0, 1):
            acc_h += gx[dk:dk + nz, dj:dj + ny, 0:nx]              # Ex(i, j+dj, k+dk)
    for dk in (0, 1):
        for di in (0, 1):
            acc_h += gy[dk:dk + nz, 0:ny, di:di + nx]              # Ey(i+di, j, k+dk)
    for dj in (0, 1):
        for di in (0, 1):
            acc_v += gz[0:nz, dj:dj + ny, di:di + nx]              # Ez(i+di, j+dj, k)
    if is_vti(rho):
        g_sigma = np.stack([acc_h * V, acc_v * V])
    else:
        g_sigma = (acc_h + acc_v) * V
    if wrt == "sigma":
        return g_sigma
    return -g_sigma / rho

def gradient_time_domain(pb: Problem, rho, src, rec, resid, wrt="lnrho", wavelet=None):
    """Cell gradient by the appendix's time-domain adjoint (full storage; small grids).

    With d_k = norm_k sum_n w_{k,n} tr^n (tr^n: E^n sampled at the receivers,
    norm_k = k_k / What_k) the data functional's derivative is
    d phi / d tr^n = -q^n, q^n = Re sum_k conj(r_k) norm_k w_{k,n}.  The adjoint of
    the leap-frog scheme is the same scheme run in reversed time, m = nt - 1 - n,
    driven by q^{nt-1-m} injected at the receivers like a source; with its field
    Et^m the gradient on each edge is
        dphi/dsigma_e = -1 / (2 w0 dt) sum_n dV_e Et_e^{nt-1-n} (E_e^{n+1} - E_e^n)
    (Appendix: dphi/dsigma = -(1 / 2 w0) int Et . d_t E dt', sigma = 2 w0 eps),
    mapped to cells like the frequency-domain gradient.  resid: r [n_src, n_rec, n_freq].
    """
    st = Stepper(pb, rho)
    N, nt = pb.N, pb.nt
    wav = pb.impulse() if wavelet is None else np.asarray(wavelet, float)
    norm = pb.k / pb.wavelet_spectrum(wav)
    W = pb.dft_weights()
    dV = edge_dual_volumes(pb.xn, pb.yn, pb.zn).reshape(-1)
    rinj = []
    for r in range(rec.n):
        rinj += point_taps(pb, rec, r, scale_by_dV=st.dV, tag=r)
    corr = np.zeros(3 * N)
    for s in range(src.n):
        fields, psi = st.new_state()
        inj = point_taps(pb, src, s, scale_by_dV=st.dV, tag=0)
        E = np.zeros((nt + 1, 3 * N))
        for n in range(nt):
            st.run(fields, psi, n, n + 1, inj=inj, series=wav[None, :])
            E[n + 1] = fields[:3 * N]
        q = np.real((np.conj(resid[s]) * norm[None, :]) @ W.T)          # [n_rec, nt]
        series = np.ascontiguousarray(q[:, ::-1])
        fa, pa = st.new_state()
        Et = np.zeros(3 * N)
        for m in range(nt):
            n = nt - 1 - m
            corr += Et * (E[n + 1] - E[n])                               # Et = adjoint field after m steps
            st.run(fa, pa, m, m + 1, inj=rinj, series=series)
            Et = fa[:3 * N].copy()
    g_edge = (-(1.0 / (2 * omega0(pb.f0) * pb.dt)) * corr * dV).reshape((3,) + pb.shape_nodes)
    return _edge_to_cells(pb, np.asarray(rho, float), g_edge, wrt)
