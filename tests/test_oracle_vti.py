"""Pins of the oracle's VTI medium (Sec. 2: sigma_h = sigma_xx = sigma_yy,
sigma_v = sigma_zz; Sec. 3.1, Eq. 15: dphi/dsigma_h from the x and y edges,
dphi/dsigma_v from the z edges).

  V1  with rho_h = rho_v the VTI oracle is the isotropic one: the same
      receivers bit for bit, and g_h + g_v is the isotropic gradient (Eq. 16 is
      Eq. 15 summed);
  V2  TE decoupling: a horizontal current loop (four unit edge dipoles around
      one z face, a vertical magnetic dipole) in a horizontally layered medium
      drives a purely horizontal E field, so its response does not depend on
      sigma_v, while an electric dipole's does.  A planted mistake that puts
      sigma_v on the x edges breaks it;
  V3  the split gradient against central differences of the misfit in ln rho_h
      and ln rho_v separately;
  V4  reciprocity holds in the VTI medium (the conductivity tensor is symmetric).
"""
import numpy as np
import pytest

from oracle import fdtd
from paper_2211_16665_gb300.workloads import Points, small_box


@pytest.fixture(scope="module")
def box():
    wl = small_box(n_core=16, h=100.0, npml=8, ratio=1.0, n_st=0, n_rec=5, n_freq=2)
    return wl, fdtd.problem_from_workload(wl)


def vti_model(rho, k_from, factor, cap=20.0):
    """(rho_h, rho_v) with rho_v = factor * rho below plane k_from, at most cap (the
    resistivity that fixes the CFL step of the box)."""
    r = np.stack([rho, rho.copy()])
    r[1][k_from:] = np.minimum(r[1][k_from:] * factor, cap)
    return r


def loop_and_receivers(wl):
    xn, yn, zn = wl.xn, wl.yn, wl.zn
    i0, j0, k0 = wl.nx // 2, wl.ny // 2, wl.nz // 2 - 2
    xc = lambda i: 0.5 * (xn[i] + xn[i + 1])
    yc = lambda j: 0.5 * (yn[j] + yn[j + 1])
    # circulation around the z face of cell (i0, j0) in node plane k0, each dipole on an edge centre
    loop = Points.make([[xc(i0), yn[j0], zn[k0]], [xn[i0 + 1], yc(j0), zn[k0]],
                        [xc(i0), yn[j0 + 1], zn[k0]], [xn[i0], yc(j0), zn[k0]]], [0, 1, 0, 1])
    sign = np.array([1.0, 1.0, -1.0, -1.0])
    rec = Points.make([[xc(i0 + 4), yn[j0 + 3], zn[k0 + 3]], [xc(i0 - 5), yn[j0 + 2], zn[k0 - 2]]], [0, 0])
    hed = Points.make([[xc(i0), yn[j0], zn[k0]]], [0])
    return loop, sign, rec, hed, k0


def loop_response(pb, model, loop, sign, rec):
    return np.tensordot(sign, fdtd.forward(pb, model, loop, rec), axes=(0, 0))


def test_isotropic_reduction(box):
    wl, pb = box
    iso = fdtd.forward(pb, wl.rho, wl.src, wl.rec)
    vti = fdtd.forward(pb, np.stack([wl.rho, wl.rho]), wl.src, wl.rec)
    assert np.array_equal(iso, vti)
    d_obs = fdtd.forward(pb, wl.rho_true, wl.src, wl.rec)
    d, E = fdtd.forward(pb, wl.rho, wl.src, wl.rec, keep_volume=True)
    _, r = fdtd.misfit(d_obs, d)
    Bp, _ = fdtd.adjoint_basis(pb, 1e-12)
    V = fdtd.adjoint(pb, wl.rho, wl.rec, r, Bp)
    V2 = fdtd.adjoint(pb, np.stack([wl.rho, wl.rho]), wl.rec, r, Bp)
    assert np.array_equal(V, V2)
    for wrt in ("sigma", "lnrho"):
        g_iso = fdtd.gradient(pb, wl.rho, E, V, wrt=wrt)
        g_hv = fdtd.gradient(pb, np.stack([wl.rho, wl.rho]), E, V, wrt=wrt)
        assert g_hv.shape == (2,) + wl.rho.shape
        np.testing.assert_allclose(g_hv[0] + g_hv[1], g_iso, rtol=0, atol=1e-13 * np.abs(g_iso).max())
        assert np.abs(g_hv[1]).max() > 1e-3 * np.abs(g_hv[0]).max()   # both parts carry signal


def test_te_loop_does_not_see_rho_v(box):
    wl, pb = box
    loop, sign, rec, hed, k0 = loop_and_receivers(wl)
    a = loop_response(pb, vti_model(wl.rho, k0 - 1, 1.0), loop, sign, rec)
    b = loop_response(pb, vti_model(wl.rho, k0 - 1, 3.0), loop, sign, rec)
    assert np.abs(a).max() > 0
    assert np.abs(b - a).max() <= 1e-11 * np.abs(a).max()
    e1 = fdtd.forward(pb, vti_model(wl.rho, k0 - 1, 1.0), hed, rec)
    e3 = fdtd.forward(pb, vti_model(wl.rho, k0 - 1, 3.0), hed, rec)
    assert np.abs(e3 - e1).max() >= 0.1 * np.abs(e1).max()


def test_te_pin_detects_sigma_v_on_the_wrong_edges(box, monkeypatch):
    wl, pb = box
    loop, sign, rec, hed, k0 = loop_and_receivers(wl)
    right = fdtd.edge_conductivity

    def swapped(rho, xn, yn, zn):   # planted mistake: sigma_v on the x edges, sigma_h on the z edges
        out = right(rho, xn, yn, zn)
        if fdtd.is_vti(rho):
            rr = np.asarray(rho)
            sv = right(np.stack([rr[1], rr[1]]), xn, yn, zn)
            sh = right(np.stack([rr[0], rr[0]]), xn, yn, zn)
            out = np.stack([sv[0], sh[1], sh[2]])
        return out

    monkeypatch.setattr(fdtd, "edge_conductivity", swapped)
    a = loop_response(pb, vti_model(wl.rho, k0 - 1, 1.0), loop, sign, rec)
    b = loop_response(pb, vti_model(wl.rho, k0 - 1, 3.0), loop, sign, rec)
    assert np.abs(b - a).max() >= 1e-3 * np.abs(a).max()


def test_vti_gradient_matches_central_differences(box):
    wl, pb = box
    k_sed = int(np.argmax(wl.rho[:, 0, 0] > 0.5))          # first sediment layer
    model = vti_model(wl.rho, k_sed, 2.0)
    true = vti_model(wl.rho_true, k_sed, 2.0)
    d_obs = fdtd.forward(pb, true, wl.src, wl.rec)
    d, E = fdtd.forward(pb, model, wl.src, wl.rec, keep_volume=True)
    _, r = fdtd.misfit(d_obs, d)
    Bp, fit = fdtd.adjoint_basis(pb, 1e-12)
    assert fit < 1e-8
    V = fdtd.adjoint(pb, model, wl.rec, r, Bp)
    g = fdtd.gradient(pb, model, E, V, wrt="lnrho")
    lnm = np.log(model)
    h = 1e-3
    for comp in (0, 1):
        order = np.argsort(-np.abs(g[comp]).ravel())
        for c in (order[0], order[30]):
            phis = []
            for sgn in (1, -1):
                m = lnm.copy()
                m[comp].flat[c] += sgn * h
                phis.append(fdtd.misfit(d_obs, fdtd.forward(pb, np.exp(m), wl.src, wl.rec))[0])
            fd = (phis[0] - phis[1]) / (2 * h)
            assert abs(g[comp].flat[c] - fd) <= 1e-3 * abs(fd), (comp, c, g[comp].flat[c], fd)


def test_vti_reciprocity(box):
    wl, pb = box
    model = vti_model(wl.rho_true, wl.nz // 2, 2.5)
    A = Points.make([[130.0, -220.0, 777.0]], 2)
    B = Points.make([[-480.0, 310.0, 1120.0]], 0)
    d_ab = fdtd.forward(pb, model, B, A)
    d_ba = fdtd.forward(pb, model, A, B)
    assert np.abs(d_ab - d_ba).max() <= 1e-9 * np.abs(d_ab).max()
