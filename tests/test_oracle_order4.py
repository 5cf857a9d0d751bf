"""Pins of the fourth-order staggered differences (Sec. 2: the paper's engine uses
high-order differences over the non-uniform grid and prints no coefficients):

  O1  fd_weights differentiates every cubic exactly at any point from four
      arbitrary nodes (checked against the analytic derivative) and misses a
      quartic; on a uniform grid the weights are the textbook staggered pair
      (1/24, -9/8, 9/8, -1/24) / h, for both the H rows and the E rows;
  O2  on a stretched axis every four-point row of staggered_weights is exact for
      cubics and the rows next to the boundary are the two-point differences;
  O3  the CFL step on a uniform grid is 6/7 of the Yee step (the symbol of the
      four-point difference peaks at 7/6 of the two-point one);
  O4  the whole-space dipole (closed form of the Yee pin) is matched to a few
      parts in 10^3 at h = 100 m, with errors at least five times smaller than
      the Yee scheme's on the same grid;
  O5  a long lossless run on a strongly stretched grid with PEC walls and a
      random model stays bounded;
  O6  the gradient through the adjoint run agrees with central differences of
      the misfit on a stretched box (the rows are not the exact transpose of
      one another on stretched axes, so within the scheme's consistency error).
"""
import numpy as np

from oracle import fdtd
from paper_2211_16665_gb300.workloads import Points, small_box, stretched_axis

from test_oracle_closed_form import ex_closed_form


def test_fd_weights_exact_for_cubics_and_textbook_values():
    rng = np.random.default_rng(11)
    for _ in range(20):
        xs = np.sort(rng.uniform(-3.0, 3.0, 4))
        if np.min(np.diff(xs)) < 0.05:
            continue
        x0 = rng.uniform(xs[0], xs[-1])
        w = fdtd.fd_weights(x0, xs)
        for deg in range(4):
            c = rng.standard_normal(deg + 1)
            f = np.polynomial.Polynomial(c)
            assert abs(w @ f(xs) - f.deriv()(x0)) <= 1e-10 * (1 + abs(f.deriv()(x0))) * np.abs(c).sum()
        assert abs(w @ xs ** 4 - 4 * x0 ** 3) > 1e-8
    h = 37.0
    xn = np.arange(12) * h
    wh, wn = fdtd.staggered_weights(xn)
    ref = np.array([1 / 24, -9 / 8, 9 / 8, -1 / 24]) / h
    np.testing.assert_allclose(wh[1:-1], np.broadcast_to(ref, wh[1:-1].shape), rtol=1e-12)
    np.testing.assert_allclose(wn[2:-2], np.broadcast_to(ref, wn[2:-2].shape), rtol=1e-12)


def test_stretched_rows_exact_for_cubics_and_boundary_rows():
    xn = stretched_axis(50.0, 10, 6, 8, 4, 1.15, -400.0)
    n = xn.size - 1
    h, ht = fdtd.spacings(xn)
    xh = 0.5 * (xn[1:] + xn[:-1])
    wh, wn = fdtd.staggered_weights(xn)
    f = np.polynomial.Polynomial([0.3, -1.1, 0.7, 0.25])
    scale = lambda x: f(x / 500.0)                       # noqa: E731
    dscale = lambda x: f.deriv()(x / 500.0) / 500.0      # noqa: E731
    for p in range(1, n - 1):
        assert abs(wh[p] @ scale(xn[p - 1:p + 3]) - dscale(xh[p])) <= 1e-9 * abs(dscale(xh[p])) + 1e-15
    for q in range(2, n - 1):
        assert abs(wn[q] @ scale(xh[q - 2:q + 2]) - dscale(xn[q])) <= 1e-9 * abs(dscale(xn[q])) + 1e-15
    for p in (0, n - 1):
        np.testing.assert_allclose(wh[p], [0, -1 / h[p], 1 / h[p], 0], rtol=1e-14)
    for q in (1, n - 1):
        np.testing.assert_allclose(wn[q], [0, -1 / ht[q], 1 / ht[q], 0], rtol=1e-14)
    assert np.all(wn[0] == 0) and np.all(wn[n] == 0)


def test_cfl_uniform_grid_ratio():
    ax = np.arange(21) * 80.0
    d2 = fdtd.cfl_dt(ax, ax, ax, 3.0, 1.0)
    d4 = fdtd.cfl_dt_order4(ax, ax, ax, 3.0, 1.0)
    assert abs(d4 / d2 - 6.0 / 7.0) <= 1e-12


def _dipole(order, h=100.0):
    ncore = int(round(4000 / h))
    xn = stretched_axis(h, ncore, 0, 0, 10, 1.0, -2000.0 + 50.0 - h / 2)
    ax = stretched_axis(h, ncore, 0, 0, 10, 1.0, -2000.0)
    rho = np.ones((ax.size - 1,) * 3)
    pb = fdtd.make_problem(xn, ax, ax, 10, [0.25, 1.0], 1.0, rho_max=1.0, order=order)
    src = Points.make([[50.0, 0.0, 0.0]], 0)
    offs = np.arange(300.0, 1501.0, 100.0)
    pts = [[50.0 + o, 0.0, 0.0] for o in offs] + [[50.0, o, 0.0] for o in offs] + \
          [[50.0, 0.0, o] for o in offs]
    d = fdtd.forward(pb, rho, src, Points.make(pts, 0))[0]
    ref = np.array([[ex_closed_form(px - 50.0, py, pz, f, 1.0) for (px, py, pz) in pts] for f in (0.25, 1.0)]).T
    return offs, d / ref


def test_whole_space_dipole_fourth_order():
    offs, r4 = _dipole(4)
    _, r2 = _dipole(2)
    far = np.concatenate([offs >= 1000.0] * 3)
    for fi, (amp_tol, ph_tol) in enumerate(((0.002, 0.1), (0.006, 0.3))):
        assert np.abs(np.abs(r4[far, fi]) - 1).max() <= amp_tol
        assert np.abs(np.degrees(np.angle(r4[far, fi]))).max() <= ph_tol
        assert np.median(np.abs(r2[far, fi] - 1)) >= 5 * np.median(np.abs(r4[far, fi] - 1))


def test_long_lossless_run_stays_bounded_on_a_stretched_grid():
    rng = np.random.default_rng(3)
    xn = stretched_axis(100.0, 10, 3, 4, 0, 1.1, 0.0)
    yn = stretched_axis(80.0, 9, 2, 3, 0, 1.2, 0.0)
    zn = stretched_axis(120.0, 8, 4, 2, 0, 1.05, 0.0)
    nx, ny, nz = xn.size - 1, yn.size - 1, zn.size - 1
    rho = 10 ** rng.uniform(-0.5, 1.5, (nz, ny, nx))
    pb = fdtd.make_problem(xn, yn, zn, 0, [0.5], 1.0, rho_max=rho.max(), nt=400, order=4)
    st = fdtd.Stepper(pb, rho)
    fields, psi = st.new_state()
    F = fields.reshape((6,) + pb.shape_nodes)
    F[0][1:nz, 1:ny, :nx] = rng.standard_normal((nz - 1, ny - 1, nx))
    F[1][1:nz, :ny, 1:nx] = rng.standard_normal((nz - 1, ny, nx - 1))
    F[2][:nz, 1:ny, 1:nx] = rng.standard_normal((nz, ny - 1, nx - 1))
    norms = []
    for _ in range(8):
        st.run(fields, psi, 0, 1000)
        norms.append(np.linalg.norm(fields))    # E and H after the energy has spread to H
    assert np.all(np.isfinite(norms)) and max(norms) <= 1.2 * norms[0]


def test_fourth_order_gradient_central_differences():
    wl = small_box(n_core=10, h=100.0, npml=5, ratio=1.08, n_st=3, n_rec=4, n_freq=2)
    pb = fdtd.problem_from_workload(wl, order=4)
    d_obs = fdtd.forward(pb, wl.rho_true, wl.src, wl.rec)
    d, E = fdtd.forward(pb, wl.rho, wl.src, wl.rec, keep_volume=True)
    _, r = fdtd.misfit(d_obs, d)
    Bp, _ = fdtd.adjoint_basis(pb, 1e-12)
    g = fdtd.gradient(pb, wl.rho, E, fdtd.adjoint(pb, wl.rho, wl.rec, r, Bp), wrt="lnrho")
    g_td = fdtd.gradient_time_domain(pb, wl.rho, wl.src, wl.rec, r)
    assert np.linalg.norm(g - g_td) <= 1e-4 * np.linalg.norm(g)
    m = np.log(wl.rho)
    h = 1e-4
    for c in np.argsort(-np.abs(g).ravel())[:3]:
        vals = []
        for sgn in (1.0, -1.0):
            mm = m.copy()
            mm.flat[c] += sgn * h
            vals.append(fdtd.misfit(d_obs, fdtd.forward(pb, np.exp(mm), wl.src, wl.rec))[0])
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(g.flat[c] - fd) <= 5e-4 * abs(fd)
