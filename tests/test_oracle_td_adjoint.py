"""Pins of the time-domain adjoint gradient (appendix) in the oracle:

  T1  it matches central differences of the misfit in ln(rho) on the cells
      with the largest gradient (it is the exact adjoint of the discrete
      scheme, so only the difference quotient's own error remains);
  T2  it agrees with the fictitious-wave-domain gradient of Sec. 3.1 (basis
      adjoint) on the whole model, up to that method's regularised fit.

A dropped 1/dt, a conjugated normalisation, an off-by-one in the time
alignment of the two fields (E^{n+1} - E^n against the adjoint field of step
nt-1-n) or a wrong sign each moves T1 and T2 by orders of magnitude.
"""
import numpy as np
import pytest

from oracle import fdtd
from paper_2211_16665_gb300.workloads import small_box


@pytest.fixture(scope="module")
def case():
    wl = small_box(n_core=10, h=100.0, npml=5, ratio=1.0, n_st=0, n_rec=4, n_freq=2)
    pb = fdtd.problem_from_workload(wl)
    d_obs = fdtd.forward(pb, wl.rho_true, wl.src, wl.rec)
    d, E = fdtd.forward(pb, wl.rho, wl.src, wl.rec, keep_volume=True)
    phi, r = fdtd.misfit(d_obs, d)
    g_td = fdtd.gradient_time_domain(pb, wl.rho, wl.src, wl.rec, r)
    return wl, pb, d_obs, E, r, g_td


def test_td_gradient_matches_central_differences(case):
    wl, pb, d_obs, _, _, g_td = case
    m = np.log(wl.rho)
    h = 1e-4
    for c in np.argsort(-np.abs(g_td).ravel())[:3]:
        vals = []
        for sgn in (1.0, -1.0):
            mm = m.copy()
            mm.flat[c] += sgn * h
            vals.append(fdtd.misfit(d_obs, fdtd.forward(pb, np.exp(mm), wl.src, wl.rec))[0])
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(g_td.flat[c] - fd) <= 1e-5 * abs(fd), (c, g_td.flat[c], fd)


def test_td_gradient_agrees_with_basis_gradient(case):
    wl, pb, _, E, r, g_td = case
    Bp, _ = fdtd.adjoint_basis(pb, 1e-12)
    V = fdtd.adjoint(pb, wl.rho, wl.rec, r, Bp)
    g_fw = fdtd.gradient(pb, wl.rho, E, V, wrt="lnrho")
    assert np.linalg.norm(g_td - g_fw) <= 1e-4 * np.linalg.norm(g_fw)


def test_td_gradient_vti_agrees_with_basis_gradient():
    wl = small_box(n_core=10, h=100.0, npml=5, ratio=1.0, n_st=0, n_rec=4, n_freq=2)
    pb = fdtd.problem_from_workload(wl)
    rho = np.stack([wl.rho, np.minimum(2.0 * wl.rho, 50.0)])        # (h, v)
    d_obs = fdtd.forward(pb, np.stack([wl.rho_true, wl.rho_true]), wl.src, wl.rec)
    d, E = fdtd.forward(pb, rho, wl.src, wl.rec, keep_volume=True)
    _, r = fdtd.misfit(d_obs, d)
    g_td = fdtd.gradient_time_domain(pb, rho, wl.src, wl.rec, r)
    Bp, _ = fdtd.adjoint_basis(pb, 1e-12)
    g_fw = fdtd.gradient(pb, rho, E, fdtd.adjoint(pb, rho, wl.rec, r, Bp), wrt="lnrho")
    assert g_td.shape == (2,) + wl.rho.shape
    for part in (0, 1):
        assert np.linalg.norm(g_td[part] - g_fw[part]) <= 1e-4 * np.linalg.norm(g_fw[part])


def test_td_gradient_vti_central_differences():
    """Both parts of the VTI time-domain gradient against central differences in ln rho_h and ln rho_v."""
    wl = small_box(n_core=10, h=100.0, npml=5, ratio=1.0, n_st=0, n_rec=4, n_freq=2)
    pb = fdtd.problem_from_workload(wl)
    rho = np.stack([wl.rho, np.minimum(2.0 * wl.rho, 50.0)])
    d_obs = fdtd.forward(pb, np.stack([wl.rho_true, wl.rho_true]), wl.src, wl.rec)
    _, r = fdtd.misfit(d_obs, fdtd.forward(pb, rho, wl.src, wl.rec))
    g = fdtd.gradient_time_domain(pb, rho, wl.src, wl.rec, r)
    m = np.log(rho)
    h = 1e-4
    for part in (0, 1):
        c = int(np.argmax(np.abs(g[part])))
        vals = []
        for sgn in (1.0, -1.0):
            mm = m.copy()
            mm[part].flat[c] += sgn * h
            vals.append(fdtd.misfit(d_obs, fdtd.forward(pb, np.exp(mm), wl.src, wl.rec))[0])
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(g[part].flat[c] - fd) <= 1e-5 * abs(fd), (part, g[part].flat[c], fd)
