"""GPU parity of the fourth-order staggered scheme through the C ABI against the
FP64 oracle with the same weights (derived independently on each side), on the
same seeded inputs.

Tolerances as for the Yee scheme: FP64 1e-10 (traces, receivers, volumes),
1e-9 (adjoint volumes, gradients); FP32 1e-4 traces, 1e-5 receivers, 1e-3
volumes and gradients.  The box is 48 x 41 x 39 cells with stretched padding:
ragged for 32 x 8 thread blocks and 4-plane z blocks, and every row type of the
weights (two-point next to the boundary, four-point on stretched and uniform
stretches) is exercised.
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
from paper_2211_16665_gb300.engine import Engine, misfit  # noqa: E402
from paper_2211_16665_gb300._capi import CsemError  # noqa: E402


def rel_l2(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def gpu_volume(eng, v):
    return v.cpu().numpy()[..., : eng.nx + 1].astype(np.complex128)


@pytest.fixture(scope="module")
def box():
    wl = W.small_box(n_core=24, h=100.0, npml=8, ratio=1.08, n_st=4, n_rec=6, n_freq=2, n_core_y=17, n_core_z=15)
    pb = fdtd.problem_from_workload(wl, order=4)
    d_obs = fdtd.forward(pb, wl.rho_true, wl.src, wl.rec)
    d, E, tr = fdtd.forward(pb, wl.rho, wl.src, wl.rec, keep_volume=True, return_trace=True)
    phi, r = fdtd.misfit(d_obs, d)
    Bp, _ = fdtd.adjoint_basis(pb, 1e-12)
    V = fdtd.adjoint(pb, wl.rho, wl.rec, r, Bp)
    g = fdtd.gradient(pb, wl.rho, E, V, wrt="lnrho")
    return wl, pb, dict(d_obs=d_obs, d=d, E=E, tr=tr, phi=phi, r=r, V=V, g=g)


@pytest.mark.parametrize("precision", [64, 32])
def test_forward_order4(box, precision):
    wl, pb, o = box
    eng = Engine.from_workload(wl, precision=precision, kahan=1, order=4)
    assert eng.order == 4 and eng.nt == pb.nt and abs(eng.dt - pb.dt) <= 1e-14 * pb.dt
    rho = eng.model_tensor(wl.rho)
    d, E, tr = eng.fwd_model(rho, wl.src, wl.rec, keep_volume=True, trace=True)
    torch.cuda.synchronize()
    assert rel_l2(tr.cpu().numpy(), o["tr"]) <= (1e-10 if precision == 64 else 1e-4)
    assert rel_l2(d.cpu().numpy(), o["d"]) <= (1e-10 if precision == 64 else 1e-5)
    assert rel_l2(gpu_volume(eng, E), o["E"]) <= (1e-10 if precision == 64 else 1e-3)
    eng.check()
    eng.close()


@pytest.mark.parametrize("precision", [64, 32])
def test_adjoint_and_gradient_order4(box, precision):
    wl, pb, o = box
    eng = Engine.from_workload(wl, precision=precision, kahan=1, order=4)
    rho = eng.model_tensor(wl.rho)
    d, E = eng.fwd_model(rho, wl.src, wl.rec, keep_volume=True)
    phi, r = misfit(torch.as_tensor(o["d_obs"], device=eng.device), d)
    assert abs(phi.item() - o["phi"]) <= (1e-10 if precision == 64 else 1e-4) * o["phi"]
    basis, _, _ = eng.estimate_adjoint_basis(gamma=1e-12, relative=True)
    V = eng.adjoint_model(rho, wl.rec, r, basis)
    tol = 1e-9 if precision == 64 else 1e-3
    assert rel_l2(gpu_volume(eng, V), o["V"]) <= tol
    g = eng.gradient(rho, E, V, wrt="lnrho")
    assert rel_l2(g.cpu().numpy(), o["g"]) <= tol
    eng.close()


ORDER4_FP32_LAUNCH = [
    dict(flush_mode=1, block=32),                                                     # plain kernels
    dict(lean_h=2, kz_h=4, mb_h=6, lean_e=2, kz_e=4, mb_e=6, flush_mode=1, block=32),
    dict(lean_h=2, kz_h=2, mb_h=8, flush_mode=0, block=16),                           # lean H, plain E
    dict(lean_e=2, kz_e=8, mb_e=4, flush_mode=3, block=16),                           # plain H, lean E
    dict(lean_h=2, kz_h=8, mb_h=4, lean_e=2, kz_e=2, mb_e=8, flush_mode=1, block=16),
]


@pytest.mark.parametrize("variant", range(len(ORDER4_FP32_LAUNCH)))
def test_order4_fp32_launch_variants(box, variant):
    """The lean fourth-order kernels (two cells per thread, z window, branch-free boundary
    rows) and the plain ones, alone or mixed per half, against the FP64 oracle."""
    wl, pb, o = box
    eng = Engine.from_workload(wl, precision=32, kahan=1, order=4, autotune=False)
    eng.set_launch(**ORDER4_FP32_LAUNCH[variant])
    rho = eng.model_tensor(wl.rho)
    d, E, tr = eng.fwd_model(rho, wl.src, wl.rec, keep_volume=True, trace=True)
    assert rel_l2(tr.cpu().numpy(), o["tr"]) <= 1e-4
    assert rel_l2(d.cpu().numpy(), o["d"]) <= 1e-5
    assert rel_l2(gpu_volume(eng, E), o["E"]) <= 1e-3
    assert torch.count_nonzero(E[..., eng.nx + 1:]) == 0
    phi, r = misfit(torch.as_tensor(o["d_obs"], device=eng.device), d)
    basis, _, _ = eng.estimate_adjoint_basis(gamma=1e-12, relative=True)
    V = eng.adjoint_model(rho, wl.rec, r, basis)
    assert rel_l2(gpu_volume(eng, V), o["V"]) <= 1e-3
    assert rel_l2(eng.gradient(rho, E, V, wrt="lnrho").cpu().numpy(), o["g"]) <= 1e-3
    eng.check()
    eng.close()


@pytest.mark.parametrize("precision,launch", [(64, None), (32, None),
                                              (32, dict(lean_h=2, kz_h=4, mb_h=6, lean_e=2, kz_e=8, mb_e=4))])
def test_td_gradient_order4(precision, launch):
    wl = W.small_box(n_core=20, h=100.0, npml=6, ratio=1.08, n_st=2, n_rec=5, n_freq=2, n_core_y=14, n_core_z=10,
                     nt=1000)
    wl = dataclasses.replace(wl, src=W.Points.make([[30.0, 0.0, wl.src.z[0]], [-250.0, 40.0, wl.src.z[0]]], 0))
    pb = fdtd.problem_from_workload(wl, order=4)
    d_obs = fdtd.forward(pb, wl.rho_true, wl.src, wl.rec)
    _, r = fdtd.misfit(d_obs, fdtd.forward(pb, wl.rho, wl.src, wl.rec))
    g_ref = fdtd.gradient_time_domain(pb, wl.rho, wl.src, wl.rec, r)
    eng = Engine.from_workload(wl, precision=precision, kahan=1, order=4, autotune=launch is None)
    if launch:
        eng.set_launch(**launch)
    rg = torch.as_tensor(r, dtype=torch.complex128, device=eng.device)
    _, nbytes = eng.td_plan(wl.src.n, wl.rec.n, segment=128)
    work = torch.full((nbytes + 256,), 0xFF, dtype=torch.uint8, device=eng.device)
    g = eng.gradient_td(eng.model_tensor(wl.rho), wl.src, wl.rec, rg, segment=128, work=work)
    assert rel_l2(g.cpu().numpy(), g_ref) <= (1e-9 if precision == 64 else 1e-3)
    eng.close()


def test_order4_refuses_other_kernel_families(box):
    wl, _, _ = box
    eng = Engine.from_workload(wl, precision=32, kahan=1, order=4, autotune=False)
    for bad in (dict(lean_h=1, kz_h=1, mb_h=6), dict(fused_kz=4), dict(vec_e=1), dict(tma_h=1, kz_h=4),
                dict(lean_h=2, kz_h=16, mb_h=4), dict(lean_e=2, kz_e=4, mb_e=5)):
        with pytest.raises(CsemError):
            eng.set_launch(**bad)
    eng.set_launch(flush_mode=1, block=32)
    eng.close()


def test_order4_vti_gradient():
    """Fourth-order stepping in a VTI medium: the two features combine (FP32 against the oracle)."""
    wl = W.small_box(n_core=16, h=100.0, npml=6, ratio=1.05, n_st=2, n_rec=5, n_freq=2, n_core_y=12, n_core_z=10)
    rho = np.stack([wl.rho, np.minimum(2.0 * wl.rho, 15.0)])
    rho_true = np.stack([wl.rho_true, np.minimum(2.0 * wl.rho_true, 15.0)])
    wl = dataclasses.replace(wl, rho_max=float(rho_true.max()))
    pb = fdtd.problem_from_workload(wl, order=4)
    d_obs = fdtd.forward(pb, rho_true, wl.src, wl.rec)
    d, E = fdtd.forward(pb, rho, wl.src, wl.rec, keep_volume=True)
    _, r = fdtd.misfit(d_obs, d)
    Bp, _ = fdtd.adjoint_basis(pb, 1e-12)
    g_ref = fdtd.gradient(pb, rho, E, fdtd.adjoint(pb, rho, wl.rec, r, Bp), wrt="lnrho")
    eng = Engine.from_workload(wl, precision=32, kahan=1, order=4, vti=True)
    rt = eng.model_tensor(rho)
    dg, Eg = eng.fwd_model(rt, wl.src, wl.rec, keep_volume=True)
    assert rel_l2(dg.cpu().numpy(), d) <= 1e-5
    _, rg = misfit(torch.as_tensor(d_obs, device=eng.device), dg)
    basis, _, _ = eng.estimate_adjoint_basis(gamma=1e-12, relative=True)
    g = eng.gradient(rt, Eg, eng.adjoint_model(rt, wl.rec, rg, basis)).cpu().numpy()
    for part in (0, 1):
        assert rel_l2(g[part], g_ref[part]) <= 1e-3
    eng.close()
