"""Pin P6: the adjoint-source basis of Sec. 3.3 (oracle side).

  * exact push-through B+ = B^T (B B^T + gamma I)^-1 equals the brute-force
    dense (B^T B + gamma I)^-1 B^T of Eq. 11 on small N_t;
  * CGNR reaches the same columns and, since B^T B + gamma I has at most
    2 N_w + 1 distinct eigenvalues, converges in that many iterations;
  * feeding unit spectra reproduces the columns (Sec. 3.3, bullet list);
  * the paper's worked example (golden/basis_example_sec33.json): error
    below 1e-8 within 15 CG iterations, basis decaying with time.
"""
import json
import os

import numpy as np
import pytest

from oracle import basis

GOLD = os.path.join(os.path.dirname(__file__), "golden", "basis_example_sec33.json")


def test_pushthrough_equals_dense_bruteforce():
    for (dt, nt, freqs, gamma_rel) in ((0.004, 400, [0.25, 0.75], 1e-6), (0.01, 1500, [0.1, 0.3, 1.0], 1e-5)):
        B = basis.basis_matrix(dt, nt, freqs, 1.0)
        g = basis.gamma_from_relative(B, gamma_rel)
        a = basis.pinv_pushthrough(B, g)
        b = basis.pinv_dense(B, g)
        # the dense solve has condition ~ 1/gamma_rel, so it is exact to ~1e-10 here
        assert np.abs(a - b).max() <= 1e-9 * np.abs(b).max()


def test_basis_rows_are_the_damped_transform():
    # B s must be the real / imaginary parts of the no-dt damped transform at t_{n+1/2}
    dt, nt, f = 0.003, 300, [0.3, 1.1]
    B = basis.basis_matrix(dt, nt, f, 1.0)
    rng = np.random.default_rng(1)
    s = rng.standard_normal(nt)
    a = np.sqrt(2 * np.pi * np.array(f) * 2 * np.pi)
    t = (np.arange(nt) + 0.5) * dt
    spec = np.array([np.sum(s * np.exp(-ak * t) * np.exp(1j * ak * t)) for ak in a])
    Bs = B @ s
    assert np.allclose(Bs[:2], spec.real, rtol=1e-13, atol=1e-13)
    assert np.allclose(Bs[2:], spec.imag, rtol=1e-13, atol=1e-13)


def test_cgnr_matches_exact_within_2nw_plus_1_iterations():
    dt, nt, freqs = 0.004, 1000, [0.25, 0.5, 1.0]
    B = basis.basis_matrix(dt, nt, freqs, 1.0)
    g = basis.gamma_from_relative(B, 1e-6)
    exact = basis.pinv_pushthrough(B, g)
    for j in range(6):
        # exact arithmetic: done after 2 N_w + 1 = 7 steps; FP64 needs one more for 1e-10
        x, hist = basis.cgnr(B, g, np.eye(6)[j], max_iter=2 * 3 + 1, tol=0.0)
        assert np.abs(x - exact[:, j]).max() <= 1e-6 * np.abs(exact[:, j]).max()
        x, hist = basis.cgnr(B, g, np.eye(6)[j], max_iter=2 * 3 + 2, tol=0.0)
        assert np.abs(x - exact[:, j]).max() <= 1e-10 * np.abs(exact[:, j]).max()
    # and it has not converged after 2 N_w steps: the count is not an accident
    x, hist = basis.cgnr(B, g, np.eye(6)[0], max_iter=2 * 3 - 1, tol=0.0)
    assert np.abs(x - exact[:, 0]).max() > 1e-4 * np.abs(exact[:, 0]).max()


def test_unit_spectra_reproduce_columns_and_synthesis_is_linear():
    B = basis.basis_matrix(0.004, 800, [0.25, 0.75], 1.0)
    Bp = basis.pinv_pushthrough(B, basis.gamma_from_relative(B, 1e-10))
    cols = basis.basis_by_cgnr(B, basis.gamma_from_relative(B, 1e-10), max_iter=50)
    assert np.abs(cols - Bp).max() <= 1e-7 * np.abs(Bp).max()
    c = np.array([[1.0 + 0j, 0], [0, 0], [0, 1j]])
    s = basis.synthesize(Bp, c)
    assert np.allclose(s[0], Bp[:, 0]) and np.allclose(s[1], 0) and np.allclose(s[2], Bp[:, 3])
    # a small gamma reproduces any spectrum: B B+ ~ I
    assert basis.fit_residual(B, Bp) <= 1e-6


def test_paper_worked_example():
    gold = json.load(open(GOLD))
    pr, rd = gold["printed"], gold["reading"]
    for dt in (pr["dt_text"], pr["dt_caption"]):
        B = basis.basis_matrix(dt, pr["nt"], rd["freqs_hz"], pr["f0"])
        assert B.shape == (2 * pr["n_freq"], pr["nt"])
        exact = basis.pinv_pushthrough(B, pr["gamma"])
        for j in range(2 * pr["n_freq"]):
            x, hist = basis.cgnr(B, pr["gamma"], np.eye(2 * pr["n_freq"])[j], max_iter=pr["cg_iterations"], tol=0.0)
            assert min(hist) < pr["cg_error_below"]
            assert np.abs(x - exact[:, j]).max() < pr["cg_error_below"] * np.abs(exact[:, j]).max()
    B = basis.basis_matrix(pr["dt_caption"], pr["nt"], rd["freqs_hz"], pr["f0"])
    Bp = basis.pinv_pushthrough(B, pr["gamma"])
    tail = int(0.9 * pr["nt"])
    assert np.all(np.abs(Bp[tail:]).max(axis=0) < 1e-2 * np.abs(Bp).max(axis=0))


def test_eight_log_spaced_frequencies_need_less_regularisation():
    """The reading behind the fit target: for 8 log-spaced frequencies over 0.1-1.5 Hz and
    19 492 steps the Gram matrix B B^T has a condition number near 1e12, so gamma = 1e-12
    relative leaves a fit residual near 0.2, while 1e-16 fits to ~1e-4 with B+ entries only
    about twice as large; 4 frequencies over 0.25-1 Hz fit at 1e-12 already."""
    from oracle import basis as B
    from oracle import fdtd
    from paper_2211_16665_gb300 import workloads as W
    large = fdtd.problem_from_workload(W.large_gradient())
    M = B.basis_matrix(large.dt, large.nt, large.freqs, large.f0)
    ev = np.linalg.eigvalsh(M @ M.T)
    assert 1e11 < ev.max() / ev.min() < 1e13
    fits, amps = {}, {}
    for g in (1e-12, 1e-16):
        Bp = B.pinv_pushthrough(M, B.gamma_from_relative(M, g))
        fits[g], amps[g] = B.fit_residual(M, Bp), np.abs(Bp).max()
    assert fits[1e-12] > 0.1 and fits[1e-16] < 1e-3 and amps[1e-16] < 3 * amps[1e-12]
    thin = fdtd.problem_from_workload(W.thin_reservoir())
    Mt = B.basis_matrix(thin.dt, thin.nt, thin.freqs, thin.f0)
    assert B.fit_residual(Mt, B.pinv_pushthrough(Mt, B.gamma_from_relative(Mt, 1e-12))) < 1e-3
