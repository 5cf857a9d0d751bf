"""Adjoint-source basis of paper Sec. 3.2-3.3 in plain FP64 numpy (test infrastructure only).

The time series s(t'_n) whose damped transform matches a few frequency
samples s(w_k) minimises (Eq. 8)
    Psi = || s(w) - B s(t') ||^2 + gamma || s(t') ||^2,
with B (2 N_w x N_t) holding the rows exp(-a_k t_n) cos(a_k t_n) and then
exp(-a_k t_n) sin(a_k t_n), a_k = sqrt(w_k w0) (Eq. 9-10).  Its solution is
s(t) = B+ s(w) with B+ = (B^T B + gamma I)^-1 B^T (Eq. 11), whose 2 N_w
columns are the basis functions (Eq. 12-13), each obtained from a unit
right-hand side.

Reading used here: the time samples are the source-injection times
t_n = (n + 1/2) dt of the leap-frog scheme (the source term enters the E
update half way between E samples), so that the transform of the injected
series is exactly the quantity the forward normalisation divides by.
"""
from __future__ import annotations

import numpy as np


def decay_rates(freqs, f0: float) -> np.ndarray:
    """a_k = sqrt(w_k w0) with w = 2 pi f (Eq. 5-6)."""
    return np.sqrt(2 * np.pi * np.asarray(freqs, np.float64) * 2 * np.pi * f0)


def basis_matrix(dt: float, nt: int, freqs, f0: float) -> np.ndarray:
    """B of Eq. 10 at t_n = (n + 1/2) dt; shape (2 N_w, nt)."""
    a = decay_rates(freqs, f0)[:, None]
    t = (np.arange(nt) + 0.5) * dt
    env = np.exp(-a * t)
    return np.concatenate([env * np.cos(a * t), env * np.sin(a * t)], axis=0)


def gamma_from_relative(B: np.ndarray, gamma_rel: float) -> float:
    """gamma = gamma_rel * largest eigenvalue of B B^T."""
    return float(gamma_rel * np.linalg.eigvalsh(B @ B.T).max())


def pinv_pushthrough(B: np.ndarray, gamma: float) -> np.ndarray:
    """B+ = (B^T B + gamma I)^-1 B^T = B^T (B B^T + gamma I)^-1, shape (nt, 2 N_w).

    The second form is the same matrix (push-through identity) and needs only
    the small 2 N_w x 2 N_w Gram system.
    """
    m = B.shape[0]
    G = B @ B.T + gamma * np.eye(m)
    return B.T @ np.linalg.solve(G, np.eye(m))


def pinv_dense(B: np.ndarray, gamma: float) -> np.ndarray:
    """Brute force: solve the nt x nt regularised normal equations of Eq. 11."""
    nt = B.shape[1]
    return np.linalg.solve(B.T @ B + gamma * np.eye(nt), B.T)


def cgnr(B: np.ndarray, gamma: float, rhs: np.ndarray, max_iter: int = 100, tol: float = 1e-14):
    """Conjugate gradients on the regularised normal equations (CGNR), Sec. 3.3.

    Solves (B^T B + gamma I) x = B^T rhs without forming B^T B, using only
    products with B and B^T.  Returns (x, list of relative residual norms).
    """
    x = np.zeros(B.shape[1])
    r = rhs.astype(np.float64).copy()          # data residual  rhs - B x
    s = B.T @ r - gamma * x                    # normal-equation residual
    p = s.copy()
    gam = float(s @ s)
    hist = [1.0]
    g0 = np.sqrt(gam)
    for _ in range(max_iter):
        if np.sqrt(gam) <= tol * g0:
            break
        q = B @ p
        delta = float(q @ q) + gamma * float(p @ p)
        alpha = gam / delta
        x += alpha * p
        r -= alpha * q
        s = B.T @ r - gamma * x
        gam_new = float(s @ s)
        hist.append(np.sqrt(gam_new) / g0)
        p = s + (gam_new / gam) * p
        gam = gam_new
    return x, hist


def basis_by_cgnr(B: np.ndarray, gamma: float, max_iter: int = 100, tol: float = 1e-14) -> np.ndarray:
    """Columns of B+ from the 2 N_w unit right-hand sides (Sec. 3.3, bullet list)."""
    m = B.shape[0]
    cols = [cgnr(B, gamma, np.eye(m)[j], max_iter, tol)[0] for j in range(m)]
    return np.stack(cols, axis=1)


def fit_residual(B: np.ndarray, Bp: np.ndarray) -> float:
    """max |B B+ - I|: how well the basis reproduces unit spectra."""
    return float(np.abs(B @ Bp - np.eye(B.shape[0])).max())


def synthesize(Bp: np.ndarray, coef: np.ndarray) -> np.ndarray:
    """Eq. 13: s(t) = sum_k Re c_k b_k + Im c_k b_{k+N_w}; coef (..., N_w) complex -> (..., nt)."""
    nw = coef.shape[-1]
    return coef.real @ Bp[:, :nw].T + coef.imag @ Bp[:, nw:].T
