"""Pin G1: the oracle's adjoint-state gradient against central finite
differences of the misfit (Sec. 3.1-3.5), FP64, dt and CPML frozen.

This pins every convention of the adjoint chain at once: the placement and
scaling of the conjugated residual source (Eq. 14 read as an electric current
conj(r) at each receiver), the basis synthesis of the time series (Sec. 3.3),
the dual-volume factor, the transpose of the edge averaging and the
ln(rho) chain rule.  The expected gap is the basis fit plus the
O((|w'| dt)^2 / 24) difference between the leap-frog operator and the
continuous one.
"""
import numpy as np
import pytest

from oracle import fdtd
from paper_2211_16665_gb300.workloads import small_box


@pytest.fixture(scope="module")
def grad_case():
    wl = small_box(n_core=16, h=100.0, npml=8, ratio=1.0, n_st=0, n_rec=5, n_freq=2)
    pb = fdtd.problem_from_workload(wl)
    d_obs = fdtd.forward(pb, wl.rho_true, wl.src, wl.rec)
    d_syn, Ev = fdtd.forward(pb, wl.rho, wl.src, wl.rec, keep_volume=True)
    phi, r = fdtd.misfit(d_obs, d_syn)
    Bp, fit = fdtd.adjoint_basis(pb, 1e-12)
    Vv = fdtd.adjoint(pb, wl.rho, wl.rec, r, Bp)
    g = fdtd.gradient(pb, wl.rho, Ev, Vv, wrt="lnrho")
    return wl, pb, d_obs, g, fit


def test_gradient_matches_central_differences(grad_case):
    wl, pb, d_obs, g, fit = grad_case
    assert fit < 1e-8
    lnr = np.log(wl.rho)
    order = np.argsort(-np.abs(g).ravel())
    cells = list(order[:6:2]) + list(order[40:200:80])
    h = 1e-3
    for c in cells:
        phis = []
        for sgn in (1, -1):
            m = lnr.ravel().copy()
            m[c] += sgn * h
            d = fdtd.forward(pb, np.exp(m.reshape(lnr.shape)), wl.src, wl.rec)
            phis.append(fdtd.misfit(d_obs, d)[0])
        fd = (phis[0] - phis[1]) / (2 * h)
        assert abs(g.ravel()[c] - fd) <= 1e-3 * abs(fd), (c, g.ravel()[c], fd)

