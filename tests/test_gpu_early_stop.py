"""GPU parity of the early end of forward data runs (Sec. 2) against the oracle's
chunked run on the same inputs: the same stop step in FP64, within one 64-step
chunk in FP32 (the decision compares running transforms computed in different
precisions), and the data equal to the oracle's transform truncated at the step
the device stopped at (1e-10 FP64, 1e-5 FP32).  Two sources end together.
"""
import dataclasses

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from oracle import fdtd  # noqa: E402
from paper_2211_16665_gb300 import workloads as W  # noqa: E402
from paper_2211_16665_gb300.engine import Engine  # noqa: E402


def rel_l2(a, b):
    return float(np.linalg.norm((np.asarray(a) - b).ravel()) / np.linalg.norm(np.asarray(b).ravel()))


@pytest.fixture(scope="module")
def case():
    wl = W.small_box(n_core=12, h=100.0, npml=6, ratio=1.05, n_st=2, n_rec=5, n_freq=3)
    wl = dataclasses.replace(wl, src=W.Points.make([[30.0, 0.0, wl.src.z[0]], [-240.0, 60.0, wl.src.z[0]]], 0))
    pb = fdtd.problem_from_workload(wl)
    _, _, tr = fdtd.forward(pb, wl.rho, wl.src, wl.rec, keep_volume=True, return_trace=True)
    Wt = pb.dft_weights()
    norm = pb.k / pb.wavelet_spectrum(pb.impulse())
    partial = lambda steps: (tr[:, :, :steps] @ Wt[:steps]) * norm          # noqa: E731
    ref = {tol: fdtd.forward_early_stop(pb, wl.rho, wl.src, wl.rec, tol) for tol in (1e-4, 1e-6)}
    return wl, pb, partial, ref


@pytest.mark.parametrize("precision", [64, 32])
def test_early_end_matches_oracle(case, precision):
    wl, pb, partial, ref = case
    eng = Engine.from_workload(wl, precision=precision, kahan=1)
    rho = eng.model_tensor(wl.rho)
    for tol in (1e-4, 1e-6):
        eng.set_early_stop(tol)
        d = eng.fwd_model(rho, wl.src, wl.rec)
        steps = eng.last_run_steps()
        d_ref, steps_ref = ref[tol]
        assert steps_ref < pb.nt
        if precision == 64:
            assert steps == steps_ref
        else:
            assert abs(steps - steps_ref) <= 64 and steps % 64 == 0
        assert rel_l2(d.cpu().numpy(), partial(steps)) <= (1e-10 if precision == 64 else 1e-5)
    # off, and runs that keep volumes, take every step
    eng.set_early_stop(0.0)
    d_full = eng.fwd_model(rho, wl.src, wl.rec)
    assert eng.last_run_steps() == pb.nt
    eng.set_early_stop(1e-6)
    d_vol, _ = eng.fwd_model(rho, wl.src, wl.rec, keep_volume=True)
    assert eng.last_run_steps() == pb.nt
    assert rel_l2(d_vol.cpu().numpy(), d_full.cpu().numpy()) <= 1e-12 + (0 if precision == 64 else 1e-6)
    eng.close()


def test_forward_data_without_gradient_uses_the_early_end(case):
    from paper_2211_16665_gb300.autograd import forward_data
    wl, pb, partial, ref = case
    eng = Engine.from_workload(wl, precision=64)
    eng.set_early_stop(1e-6)
    m = torch.log(eng.model_tensor(wl.rho)).double()
    basis, _, _ = eng.estimate_adjoint_basis()
    with torch.no_grad():
        d = forward_data(m, eng, wl.src, wl.rec, basis)
    assert eng.last_run_steps() == ref[1e-6][1]
    assert rel_l2(d.cpu().numpy(), ref[1e-6][0]) <= 1e-10
    d2 = forward_data(m.clone().requires_grad_(True), eng, wl.src, wl.rec, basis)
    assert eng.last_run_steps() == pb.nt and d2.requires_grad
    eng.close()


def gpu_volume(eng, v):
    return v.cpu().numpy()[..., : eng.nx + 1].astype(np.complex128)


@pytest.mark.parametrize("precision,floor", [(64, 1e-2), (32, 1e-2), (64, 1e-4)])
def test_volume_early_end_matches_oracle(case, precision, floor):
    """Forward (with volumes) and adjoint runs ending on the volumetric transform: the same
    stop steps as the oracle in FP64 (within a chunk in FP32); volumes and gradient equal to
    the oracle's truncated at the device's steps; the gradient within 1e-5 of the full one."""
    wl, pb, partial, ref = case
    tol = 1e-6
    d_obs = fdtd.forward(pb, wl.rho_true, wl.src, wl.rec)
    d_full, E_full = fdtd.forward(pb, wl.rho, wl.src, wl.rec, keep_volume=True)
    _, r = fdtd.misfit(d_obs, d_full)
    Bp, _ = fdtd.adjoint_basis(pb, 1e-12)
    _, _, steps_ref = fdtd.forward_volumes_early_stop(pb, wl.rho, wl.src, wl.rec, tol, floor_frac=floor)
    _, sa_ref = fdtd.adjoint_early_stop(pb, wl.rho, wl.rec, r, Bp, tol, floor_frac=floor)
    assert steps_ref < pb.nt and sa_ref < pb.nt

    eng = Engine.from_workload(wl, precision=precision, kahan=1)
    rho = eng.model_tensor(wl.rho)
    basis, _, _ = eng.estimate_adjoint_basis(gamma=1e-12, relative=True)
    rg = torch.as_tensor(r, dtype=torch.complex128, device=eng.device)
    E_all, V_all = eng.fwd_model(rho, wl.src, wl.rec, keep_volume=True)[1], eng.adjoint_model(rho, wl.rec, rg, basis)
    g_all = eng.gradient(rho, E_all, V_all).double().cpu().numpy()
    eng.set_early_stop_volumes(tol, floor)
    d, E = eng.fwd_model(rho, wl.src, wl.rec, keep_volume=True)
    steps = eng.last_run_steps()
    V = eng.adjoint_model(rho, wl.rec, rg, basis)
    sa = eng.last_run_steps()
    g = eng.gradient(rho, E, V).double().cpu().numpy()
    if precision == 64:
        assert (steps, sa) == (steps_ref, sa_ref)
    else:
        assert abs(steps - steps_ref) <= 64 and abs(sa - sa_ref) <= 64
    tol_v = 1e-10 if precision == 64 else 1e-3
    d_t, E_t = fdtd.forward(pb, wl.rho, wl.src, wl.rec, keep_volume=True, nt_run=steps)
    V_t = fdtd.adjoint(pb, wl.rho, wl.rec, r, Bp, nt_run=sa)
    assert rel_l2(d.cpu().numpy(), d_t) <= (1e-10 if precision == 64 else 1e-5)
    assert rel_l2(gpu_volume(eng, E), E_t) <= tol_v
    assert rel_l2(gpu_volume(eng, V), V_t) <= (1e-9 if precision == 64 else 1e-3)
    assert rel_l2(g, fdtd.gradient(pb, wl.rho, E_t, V_t)) <= (1e-9 if precision == 64 else 1e-3)
    assert rel_l2(g, g_all) <= 1e-5
    eng.close()
