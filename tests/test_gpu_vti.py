"""GPU parity of the VTI medium (Sec. 2: sigma_h on the x and y edges, sigma_v on
the z edges; Sec. 3.1, Eq. 15: the gradient split into sigma_h and sigma_v parts)
through the C ABI, against the FP64 oracle on the same seeded box.

Tolerances as for the isotropic path: FP64 1e-10 (receivers, volumes) and 1e-9
(gradient); FP32 receivers 1e-5, volumes and gradients 1e-3 relative L2.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from oracle import fdtd  # noqa: E402
from paper_2211_16665_gb300 import workloads as W  # noqa: E402
from paper_2211_16665_gb300.autograd import forward_data  # noqa: E402
from paper_2211_16665_gb300.engine import Engine, misfit  # noqa: E402


def rel_l2(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def gpu_volume(eng, v):
    return v.cpu().numpy()[..., : eng.nx + 1].astype(np.complex128)


def vti(rho, k_from, factor, cap):
    r = np.stack([rho, rho.copy()])
    r[1][k_from:] = np.minimum(r[1][k_from:] * factor, cap)
    return r


@pytest.fixture(scope="module")
def case():
    wl = W.small_box(n_core=24, h=100.0, npml=8, ratio=1.08, n_st=4, n_rec=6, n_freq=2)
    pb = fdtd.problem_from_workload(wl)
    k_sed = int(np.argmax(wl.rho[:, 0, 0] > 0.5))
    model = vti(wl.rho, k_sed, 2.0, wl.rho_max)
    true = vti(wl.rho_true, k_sed, 2.0, wl.rho_max)
    d_obs = fdtd.forward(pb, true, wl.src, wl.rec)
    d, E = fdtd.forward(pb, model, wl.src, wl.rec, keep_volume=True)
    phi, r = fdtd.misfit(d_obs, d)
    Bp, fit = fdtd.adjoint_basis(pb, 1e-12)
    V = fdtd.adjoint(pb, model, wl.rec, r, Bp)
    g = fdtd.gradient(pb, model, E, V, wrt="lnrho")
    gs = fdtd.gradient(pb, model, E, V, wrt="sigma")
    return wl, pb, model, dict(d_obs=d_obs, d=d, E=E, V=V, g=g, gs=gs)


@pytest.mark.parametrize("precision", [64, 32])
def test_vti_forward_adjoint_gradient_match_oracle(case, precision):
    wl, pb, model, o = case
    eng = Engine.from_workload(wl, precision=precision, kahan=1, vti=True)
    assert eng.info.anisotropy == 1 and eng.model_shape == (2, wl.nz, wl.ny, wl.nx)
    rho = eng.model_tensor(model)
    d, E = eng.fwd_model(rho, wl.src, wl.rec, keep_volume=True)
    tol_r, tol_v, tol_g = (1e-10, 1e-10, 1e-9) if precision == 64 else (1e-5, 1e-3, 1e-3)
    assert rel_l2(d.cpu().numpy(), o["d"]) <= tol_r
    assert rel_l2(gpu_volume(eng, E), o["E"]) <= tol_v
    phi, r = misfit(torch.as_tensor(o["d_obs"], device=eng.device), d)
    basis, _, _ = eng.estimate_adjoint_basis(gamma=1e-12, relative=True)
    V = eng.adjoint_model(rho, wl.rec, r, basis)
    assert rel_l2(gpu_volume(eng, V), o["V"]) <= tol_v
    g = eng.gradient(rho, E, V, wrt="lnrho").cpu().numpy()
    gs = eng.gradient(rho, E, V, wrt="sigma").cpu().numpy()
    assert g.shape == (2, wl.nz, wl.ny, wl.nx)
    for part in (0, 1):        # sigma_h and sigma_v parts, each against the oracle
        assert rel_l2(g[part], o["g"][part]) <= tol_g
        assert rel_l2(gs[part], o["gs"][part]) <= tol_g
    eng.check()
    eng.close()


@pytest.mark.parametrize("launch", [dict(onepass=(8, 4, 4), flush_mode=1, block=32),
                                    dict(wspec=(8, 4, 3), flush_mode=1, block=32),
                                    dict(wave=(2, 4, 8), flush_mode=1, block=32)])
def test_vti_onepass_step_matches_oracle(case, launch):
    """The fused one-pass step averages sigma_v on the z edges from its own per-cell values;
    the warp-specialised fused step and the wave-ordered step read the edges' dt/eps."""
    wl, pb, model, o = case
    eng = Engine.from_workload(wl, precision=32, kahan=1, vti=True, autotune=False)
    eng.set_launch(**launch)
    rho = eng.model_tensor(model)
    d, E = eng.fwd_model(rho, wl.src, wl.rec, keep_volume=True)
    assert rel_l2(d.cpu().numpy(), o["d"]) <= 1e-5
    assert rel_l2(gpu_volume(eng, E), o["E"]) <= 1e-3
    phi, r = misfit(torch.as_tensor(o["d_obs"], device=eng.device), d)
    basis, _, _ = eng.estimate_adjoint_basis(gamma=1e-12, relative=True)
    V = eng.adjoint_model(rho, wl.rec, r, basis)
    assert rel_l2(gpu_volume(eng, V), o["V"]) <= 1e-3
    g = eng.gradient(rho, E, V, wrt="lnrho").cpu().numpy()
    for part in (0, 1):
        assert rel_l2(g[part], o["g"][part]) <= 1e-3
    eng.check()
    eng.close()


@pytest.mark.parametrize("onepass", [None, (8, 4, 4), "wspec"])
def test_vti_with_equal_parts_is_the_isotropic_engine(case, onepass):
    wl, pb, model, o = case
    iso = Engine.from_workload(wl, precision=32, kahan=1, autotune=False)
    ani = Engine.from_workload(wl, precision=32, kahan=1, autotune=False, vti=True)
    if onepass == "wspec":
        iso.set_launch(wspec=(8, 4, 3))
        ani.set_launch(wspec=(8, 4, 3))
    elif onepass:
        iso.set_launch(onepass=onepass)
        ani.set_launch(onepass=onepass)
    rho = iso.model_tensor(wl.rho)
    rho2 = ani.model_tensor(np.stack([wl.rho, wl.rho]))
    d1, E1 = iso.fwd_model(rho, wl.src, wl.rec, keep_volume=True)
    d2, E2 = ani.fwd_model(rho2, wl.src, wl.rec, keep_volume=True)
    assert torch.equal(d1, d2) and torch.equal(E1, E2)
    phi, r = misfit(torch.as_tensor(o["d_obs"], device=iso.device), d1)
    basis, _, _ = iso.estimate_adjoint_basis()
    V1 = iso.adjoint_model(rho, wl.rec, r, basis)
    V2 = ani.adjoint_model(rho2, wl.rec, r, basis)
    assert torch.equal(V1, V2)
    g1 = iso.gradient(rho, E1, V1).double()
    g2 = ani.gradient(rho2, E2, V2).double()
    assert rel_l2((g2[0] + g2[1]).cpu().numpy(), g1.cpu().numpy()) <= 1e-6
    with pytest.raises(ValueError):
        ani.fwd_model(rho, wl.src, wl.rec)                 # an isotropic model on a VTI context
    iso.close()
    ani.close()


def test_vti_autograd_gradient_is_the_engine_gradient(case):
    wl, pb, model, o = case
    eng = Engine.from_workload(wl, precision=32, kahan=1, vti=True)
    basis, _, _ = eng.estimate_adjoint_basis()
    d_obs = torch.as_tensor(o["d_obs"], device=eng.device)
    ln_rho = torch.tensor(np.log(model), dtype=torch.float64, device="cuda", requires_grad=True)
    d = forward_data(ln_rho, eng, wl.src, wl.rec, basis)
    (0.5 * (d_obs - d).abs().pow(2).sum()).backward()
    rho = eng.model_tensor(model)
    dd, E = eng.fwd_model(rho, wl.src, wl.rec, keep_volume=True)
    phi, r = misfit(d_obs, dd)
    V = eng.adjoint_model(rho, wl.rec, r, basis)
    g = eng.gradient(rho, E, V).double()
    assert ln_rho.grad.shape == (2, wl.nz, wl.ny, wl.nx)
    assert rel_l2(ln_rho.grad.cpu().numpy(), g.cpu().numpy()) <= 1e-6
    eng.close()
