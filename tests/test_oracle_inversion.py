"""Pins of the reference inversion loop (Sec. 3.5); all but the last are independent of
any modelling:

  I1  the Tikhonov term on a linear ramp m = c x (stretched grid) is
      1/2 alpha_x^2 c^2 per x pair and zero along y and z; its gradient matches
      central differences on random models and free masks (isotropic and VTI);
  I2  the two-loop recursion satisfies the newest secant condition H y = s;
  I3  l-BFGS with the backtracking search minimises an SPD quadratic, with the
      iterates kept inside the bounds;
  I4  after the first failed l-BFGS line search the loop restarts from the
      steepest-descent direction, and a second failure ends it;
  I5  the offset mute zeroes exactly the pairs closer than the offset, and the
      data term with the mute and a free-cell mask matches central differences.
"""
import numpy as np

from oracle import inversion as inv
from paper_2211_16665_gb300.workloads import Points, stretched_axis


def grid():
    xn = stretched_axis(100.0, 6, 2, 2, 2, 1.2, -600.0)
    yn = stretched_axis(80.0, 5, 1, 1, 2, 1.1, -400.0)
    zn = stretched_axis(50.0, 4, 1, 2, 1, 1.3, 0.0)
    return xn, yn, zn


def test_tikhonov_ramp_closed_form():
    xn, yn, zn = grid()
    nx, ny, nz = xn.size - 1, yn.size - 1, zn.size - 1
    xc = 0.5 * (xn[1:] + xn[:-1])
    c = 0.37
    m = np.broadcast_to(c * xc, (nz, ny, nx)).copy()
    alpha = (1.0, 1.0, 0.1)
    phi, g = inv.tikhonov(m, np.zeros_like(m), np.ones_like(m, bool), xn, yn, zn, alpha)
    assert abs(phi - 0.5 * alpha[0] ** 2 * c ** 2 * (nx - 1) * ny * nz) <= 1e-12 * phi
    ramp_z = np.broadcast_to(c * (0.5 * (zn[1:] + zn[:-1]))[:, None, None], (nz, ny, nx))
    phi_z, _ = inv.tikhonov(ramp_z, np.zeros_like(m), np.ones_like(m, bool), xn, yn, zn, alpha)
    assert abs(phi_z - 0.5 * alpha[2] ** 2 * c ** 2 * nx * ny * (nz - 1)) <= 1e-12 * phi_z


def test_tikhonov_gradient_central_differences():
    xn, yn, zn = grid()
    shape = (zn.size - 1, yn.size - 1, xn.size - 1)
    rng = np.random.default_rng(5)
    for lead in ((), (2,)):
        m = rng.normal(size=lead + shape)
        ref = rng.normal(size=lead + shape)
        free = rng.random(lead + shape) > 0.3
        phi, g = inv.tikhonov(m, ref, free, xn, yn, zn, (1.0, 0.7, 0.1))
        h = 1e-6
        for c in rng.choice(m.size, 12, replace=False):
            mp, mm = m.copy(), m.copy()
            mp.flat[c] += h
            mm.flat[c] -= h
            fd = (inv.tikhonov(mp, ref, free, xn, yn, zn, (1.0, 0.7, 0.1))[0] -
                  inv.tikhonov(mm, ref, free, xn, yn, zn, (1.0, 0.7, 0.1))[0]) / (2 * h)
            assert abs(g.flat[c] - fd) <= 1e-6 * max(1.0, abs(fd))


def test_two_loop_secant_condition():
    rng = np.random.default_rng(1)
    n = 7
    Q = rng.normal(size=(n, n))
    A = Q @ Q.T + n * np.eye(n)
    pairs = []
    for _ in range(4):
        s = rng.normal(size=n)
        pairs.append((s, A @ s))
    s_new, y_new = pairs[-1]
    np.testing.assert_allclose(inv.lbfgs_direction(y_new, pairs), -s_new, rtol=1e-10, atol=1e-12)


class Quadratic:
    def __init__(self, A, b):
        self.A, self.b = A, b

    def value(self, x):
        return 0.5 * float(x @ self.A @ x) - float(self.b @ x)

    def __call__(self, x):
        return Quadratic.value(self, x), self.A @ x - self.b


def test_lbfgs_minimises_a_bounded_quadratic():
    rng = np.random.default_rng(2)
    n = 12
    Q = rng.normal(size=(n, n))
    A = Q @ Q.T + np.diag(np.linspace(1.0, 20.0, n))
    x_star = rng.uniform(-0.8, 0.8, size=n)
    f = Quadratic(A, A @ x_star)
    x, hist = inv.invert(f, np.zeros(n), np.ones(n, bool), 60, -1.0, 1.0, step0=0.5)
    assert np.abs(x - x_star).max() <= 1e-6
    phis = [h["phi"] for h in hist]
    assert all(b <= a + 1e-12 for a, b in zip(phis, phis[1:]))
    assert hist[0]["direction"] == "steepest" and any(h["direction"] == "lbfgs" for h in hist)
    # a minimiser outside the box: the iterates stay inside it and the objective still decreases
    f2 = Quadratic(A, A @ (3.0 * np.ones(n)))
    x2, hist2 = inv.invert(f2, np.zeros(n), np.ones(n, bool), 40, -1.0, 1.0)
    assert x2.max() <= 1.0 and x2.min() >= -1.0 and x2.max() == 1.0
    phis2 = [h["phi"] for h in hist2]
    assert all(b <= a + 1e-12 for a, b in zip(phis2, phis2[1:])) and f2.value(x2) < phis2[0]


class Trapped(Quadratic):
    """Rejects every trial point of the line searches it is told to (planted failures)."""

    def __init__(self, A, b, fail_iters):
        super().__init__(A, b)
        self.fail_iters, self.grad_calls, self.value_calls_this_iter = set(fail_iters), 0, 0

    def __call__(self, x):
        self.grad_calls += 1
        self.value_calls_this_iter = 0
        return super().__call__(x)

    def value(self, x):
        self.value_calls_this_iter += 1
        it = self.grad_calls - 1
        # in a trapped iteration the first search (7 trials) fails; the retry, if any, does not
        if it in self.fail_iters and self.value_calls_this_iter <= 7:
            return np.inf
        return super().value(x)


def test_restart_after_the_first_line_search_failure():
    rng = np.random.default_rng(3)
    n = 10
    Q = rng.normal(size=(n, n))
    A = Q @ Q.T + n * np.eye(n)
    f = Trapped(A, A @ rng.uniform(-0.5, 0.5, n), fail_iters={2})
    x, hist = inv.invert(f, np.zeros(n), np.ones(n, bool), 6, -1.0, 1.0, max_backtracks=6)
    assert [h["direction"] for h in hist[:3]] == ["steepest", "lbfgs", "steepest"]
    assert all(h["accepted"] for h in hist)
    assert hist[3]["direction"] == "lbfgs"
    # a second failure (here in a later l-BFGS iteration) ends the loop
    g = Trapped(A, A @ rng.uniform(-0.5, 0.5, n), fail_iters={2, 4})
    _, hist2 = inv.invert(g, np.zeros(n), np.ones(n, bool), 8, -1.0, 1.0, max_backtracks=6)
    assert len(hist2) == 5 and not hist2[-1]["accepted"]


def test_offset_mute():
    src = Points.make([[0.0, 0.0, 900.0], [500.0, 0.0, 900.0]], 0)
    rec = Points.make([[x, 0.0, 1000.0] for x in (-700.0, 0.0, 400.0, 1200.0)], 0)
    w = inv.mute_weights(src, rec, 3, 600.0)
    assert w.shape == (2, 4, 3)
    np.testing.assert_array_equal(w[0, :, 0], [1, 0, 0, 1])
    np.testing.assert_array_equal(w[1, :, 0], [1, 0, 0, 1])
    assert np.all(w[..., 1] == w[..., 0])


def test_data_term_with_mute_and_free_mask_matches_central_differences():
    from oracle import fdtd
    from paper_2211_16665_gb300.workloads import small_box
    wl = small_box(n_core=16, h=100.0, npml=8, ratio=1.0, n_st=0, n_rec=5, n_freq=2)
    pb = fdtd.problem_from_workload(wl)
    d_obs = fdtd.forward(pb, wl.rho_true, wl.src, wl.rec)
    w = inv.mute_weights(wl.src, wl.rec, wl.freqs.size, 300.0)
    assert 0 < w.sum() < w.size
    free = wl.rho > 0.5                               # the sediment; the water is fixed
    dt = inv.DataTerm(pb, wl.src, wl.rec, d_obs, w, wl.rho, free)
    m = np.log(wl.rho)
    phi, g = dt(m)
    assert np.all(g[~free] == 0.0) and abs(phi - dt.value(m)) <= 1e-12 * phi
    c = int(np.argmax(np.abs(g)))
    h = 1e-3
    mp, mm = m.copy(), m.copy()
    mp.flat[c] += h
    mm.flat[c] -= h
    fd = (dt.value(mp) - dt.value(mm)) / (2 * h)
    assert abs(g.flat[c] - fd) <= 1e-3 * abs(fd)
