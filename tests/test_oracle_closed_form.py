"""Pin P1: the oracle against the closed-form field of an electric dipole in a
homogeneous conductive whole space (diffusive Maxwell system of paper Eq. 1,
time convention exp(-i w t), reached through the fictitious-wave correspondence
of Eq. 2-3 and the damped transform of Eq. 6).

Whole-space field of an x-directed unit current dipole (textbook result, e.g.
Ward & Hohmann 1988), re-derived here from E = i w mu0 (I + grad grad / k^2) g,
g = exp(i k r) / (4 pi r), k^2 = i w mu0 sigma, Im k > 0:
    E_x = (k^2 g + d^2 g / dx^2) / sigma
        = exp(i k r) / (4 pi sigma r^3) [ (x/r)^2 (3 - 3 i k r - k^2 r^2) - (1 - i k r - k^2 r^2) ].
The tests also check that expression against a numerical second derivative of g
and against its DC limit, so the pin does not rest on a retyped formula alone.
"""
import numpy as np
import pytest

from oracle import fdtd
from paper_2211_16665_gb300.workloads import Points, stretched_axis

MU0 = 4e-7 * np.pi


def wavenumber(f, sigma):
    k = np.sqrt(1j * 2 * np.pi * f * MU0 * sigma)
    return k if k.imag > 0 else -k


def ex_closed_form(x, y, z, f, sigma):
    k = wavenumber(f, sigma)
    r = np.sqrt(x * x + y * y + z * z)
    kr = k * r
    return np.exp(1j * kr) / (4 * np.pi * sigma * r ** 3) * (
        (x * x / r ** 2) * (3 - 3j * kr - kr * kr) - (1 - 1j * kr - kr * kr))


def ex_from_green(x, y, z, f, sigma, dx=1.0):
    k = wavenumber(f, sigma)

    def g(xx):
        r = np.sqrt(xx * xx + y * y + z * z)
        return np.exp(1j * k * r) / (4 * np.pi * r)

    d2 = (-g(x + 2 * dx) + 16 * g(x + dx) - 30 * g(x) + 16 * g(x - dx) - g(x - 2 * dx)) / (12 * dx * dx)
    return (k * k * g(x) + d2) / sigma


def test_closed_form_matches_green_function_and_dc_limit():
    for (x, y, z) in [(700.0, 0.0, 0.0), (0.0, 900.0, 0.0), (500.0, 400.0, 300.0)]:
        for f in (0.25, 1.0):
            a = ex_closed_form(x, y, z, f, 1.0)
            b = ex_from_green(x, y, z, f, 1.0)
            assert abs(a - b) <= 1e-7 * abs(a)
        r = np.sqrt(x * x + y * y + z * z)
        dc = (3 * x * x / r ** 2 - 1) / (4 * np.pi * 1.0 * r ** 3)
        assert abs(ex_closed_form(x, y, z, 1e-9, 1.0) - dc) <= 1e-4 * abs(dc)


def _run(h):
    ncore = int(round(4000 / h))
    # x nodes shifted so that x = 50 + 100 m is an Ex edge centre at both h
    xn = stretched_axis(h, ncore, 0, 0, 10, 1.0, -2000.0 + 50.0 - h / 2)
    ax = stretched_axis(h, ncore, 0, 0, 10, 1.0, -2000.0)
    rho = np.ones((ax.size - 1,) * 3)
    pb = fdtd.make_problem(xn, ax, ax, 10, [0.25, 1.0], 1.0, rho_max=1.0)
    # source and receivers on Ex edge centres: the point operators are exact there
    src = Points.make([[50.0, 0.0, 0.0]], 0)
    offs = np.arange(300.0, 1501.0, 100.0)
    pts = [[50.0 + o, 0.0, 0.0] for o in offs] + [[50.0, o, 0.0] for o in offs] + \
          [[50.0, 0.0, o] for o in offs]
    rec = Points.make(pts, 0)
    d = fdtd.forward(pb, rho, src, rec)[0]
    ref = np.array([[ex_closed_form(px - 50.0, py, pz, f, 1.0) for (px, py, pz) in pts] for f in (0.25, 1.0)]).T
    return offs, d, ref


@pytest.fixture(scope="module")
def runs():
    return {h: _run(h) for h in (100.0, 50.0)}


def test_whole_space_dipole_amplitude_and_phase(runs):
    offs, d, ref = runs[100.0]
    # A second-order point dipole carries an O((h/r)^2) near-field error and an
    # O((h/skin depth)^2) one; at r >= 10 h both are a few per cent.  0.25 Hz has
    # 10 cells per skin depth at h = 100 m, 1 Hz only 5.
    far = np.concatenate([offs >= 1000.0] * 3)
    for fi, (amp_tol, ph_tol) in enumerate(((0.03, 2.0), (0.04, 2.5))):
        ratio = d[far, fi] / ref[far, fi]
        assert np.abs(np.abs(ratio) - 1).max() <= amp_tol
        assert np.abs(np.degrees(np.angle(ratio))).max() <= ph_tol


def test_whole_space_dipole_second_order_convergence(runs):
    _, d1, ref = runs[100.0]
    _, d2, _ = runs[50.0]
    e1 = np.abs(d1 / ref - 1)
    e2 = np.abs(d2 / ref - 1)
    # the error falls by ~4 when h halves (2nd-order Yee), everywhere 3h..15h
    assert np.median(e1 / e2) >= 3.5
    assert (e1 / e2).min() >= 3.0
    offs = runs[50.0][0]
    assert np.abs(d2 / ref - 1)[np.concatenate([offs >= 600.0] * 3)].max() <= 0.03
