"""Pins of the early end of a forward run (Sec. 2: stepping can end once the
frequency-domain field has reached its steady state):

  S1  with tol = 0 no chunk qualifies (the late increments are never exactly zero):
      all nt steps run and the spectra equal the plain forward run;
  S2  the chunked run reproduces the plain run's traces, so the stop chunk is the
      first chunk whose 64-step increment of the running transform, computed from
      the plain run's traces, is within tol of the running value everywhere;
  S3  the spectra after the early end differ from the full run by no more than a
      small multiple of tol (the damped weights shrink the later increments), and a
      smaller tol runs more steps.
"""
import numpy as np

from oracle import fdtd
from paper_2211_16665_gb300.workloads import small_box


def case():
    wl = small_box(n_core=10, h=100.0, npml=5, ratio=1.0, n_st=0, n_rec=4, n_freq=2)
    return wl, fdtd.problem_from_workload(wl)


def test_zero_tolerance_runs_everything():
    wl, pb = case()
    d_full = fdtd.forward(pb, wl.rho, wl.src, wl.rec)
    d, steps = fdtd.forward_early_stop(pb, wl.rho, wl.src, wl.rec, 0.0)
    assert steps == pb.nt
    np.testing.assert_allclose(d, d_full, rtol=1e-13, atol=0)


def test_stop_chunk_from_the_plain_run_and_error_bound():
    wl, pb = case()
    d_full, _, tr = fdtd.forward(pb, wl.rho, wl.src, wl.rec, keep_volume=True, return_trace=True)
    W = pb.dft_weights()
    norm = pb.k / pb.wavelet_spectrum(pb.impulse())
    prev_steps = 0
    for tol in (1e-4, 1e-6, 1e-8):
        d, steps = fdtd.forward_early_stop(pb, wl.rho, wl.src, wl.rec, tol)
        # first qualifying chunk from the plain run's traces
        expect = pb.nt
        prev = None
        for c in range((pb.nt + 63) // 64):
            n1 = min(pb.nt, 64 * (c + 1))
            R = tr[:, :, :n1] @ W[:n1]
            if n1 < pb.nt and prev is not None and np.all(np.abs(R - prev) <= tol * np.abs(R)):
                expect = n1
                break
            prev = R
        assert steps == expect < pb.nt
        assert steps > prev_steps
        prev_steps = steps
        assert np.abs(d - d_full).max() <= 20 * tol * np.abs(d_full).max()
        np.testing.assert_allclose(d, (tr[:, :, :steps] @ W[:steps]) * norm, rtol=1e-12)


def test_volume_early_end():
    """V1 tol = 0 reproduces forward() and adjoint(); V2 the stop chunk is the first one
    where, in a plain run's chunked transforms, every entry moved by at most tol times the
    larger of its magnitude and 1e-4 of its frequency's largest magnitude at the
    previous check (single precision); V3 the truncated gradient stays close to the full
    one."""
    wl, pb = case()
    d_full, E_full = fdtd.forward(pb, wl.rho, wl.src, wl.rec, keep_volume=True)
    d0, E0, steps0 = fdtd.forward_volumes_early_stop(pb, wl.rho, wl.src, wl.rec, 0.0)
    assert steps0 == pb.nt
    np.testing.assert_allclose(d0, d_full, rtol=1e-13)
    np.testing.assert_allclose(E0, E_full, rtol=1e-12, atol=1e-12 * np.abs(E_full).max())
    d_obs = fdtd.forward(pb, wl.rho_true, wl.src, wl.rec)
    _, r = fdtd.misfit(d_obs, d_full)
    Bp, _ = fdtd.adjoint_basis(pb, 1e-12)
    V_full = fdtd.adjoint(pb, wl.rho, wl.rec, r, Bp)
    V0, sa0 = fdtd.adjoint_early_stop(pb, wl.rho, wl.rec, r, Bp, 0.0)
    assert sa0 == pb.nt
    np.testing.assert_allclose(V0, V_full, rtol=1e-12, atol=1e-12 * np.abs(V_full).max())
    g_full = fdtd.gradient(pb, wl.rho, E_full, V_full)
    tol = 1e-6
    d, E, steps = fdtd.forward_volumes_early_stop(pb, wl.rho, wl.src, wl.rec, tol)
    V, sa = fdtd.adjoint_early_stop(pb, wl.rho, wl.rec, r, Bp, tol)
    assert steps < pb.nt and sa < pb.nt
    # the stop chunk from plain chunked transforms (brute force on the running sum)
    st = fdtd.Stepper(pb, wl.rho)
    W = pb.dft_weights()
    fields, psi = st.new_state()
    inj = fdtd.point_taps(pb, wl.src, 0, scale_by_dV=st.dV, tag=0)
    vre, vim = np.zeros(3 * 2 * pb.N), np.zeros(3 * 2 * pb.N)
    prev, expect = None, pb.nt
    for c in range((pb.nt + 63) // 64):
        n0, n1 = 64 * c, min(pb.nt, 64 * (c + 1))
        st.run(fields, psi, n0, n1, inj=inj, series=pb.impulse()[None, :], dft=W, vol_re=vre, vol_im=vim)
        R = (vre + 1j * vim).reshape(3, 2, pb.N)
        if n1 < pb.nt and prev is not None:
            f32 = np.float32
            floor = f32(1e-4) * np.abs(prev).astype(f32).max(axis=(0, 2))          # per frequency
            bound = f32(tol) * np.maximum(np.abs(R).astype(f32), floor[None, :, None])
            # what later chunks add if the field stays as it was: the weights of Eq. 6 summed
            # chunk by chunk, sum_{m >= 1} exp((-1 + i) a_k 64 dt m), by brute force
            tail = np.array([abs(sum(np.exp((-1 + 1j) * pb.a[k] * 64 * pb.dt * m) for m in range(1, 4000)))
                             for k in range(2)])
            moved = np.abs(R - prev).astype(f32) * tail.astype(f32)[None, :, None]
            if np.all(moved <= bound):
                expect = n1
                break
        prev = R.copy()
    assert steps == expect
    g = fdtd.gradient(pb, wl.rho, E, V)
    assert np.linalg.norm(g - g_full) <= 1e-4 * np.linalg.norm(g_full)
