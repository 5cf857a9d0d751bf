"""GPU parity of the time-domain adjoint gradient (appendix) through the C ABI
against the FP64 oracle's reversed-time adjoint, on the same residual.

Tolerances (relative L2 over the cell gradient): FP64 stencil 1e-9 (the same
arithmetic, only the summation order of the time correlation differs); FP32
stencil 1e-3 (the gradient target of the hot path).  The box is 36 x 30 x 26
cells (ragged for 32-wide rows and 4-row / z blocks), two sources, a run of
1000 steps (15 graph chunks and a ragged 40-step tail); the segment lengths
cover one segment (no replay), 64 (16 segments, a short last one), 128
(adjoint sub-blocks of 64 and 40) and 2 (a checkpoint every other step).
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
from paper_2211_16665_gb300._capi import CsemError  # noqa: E402


def rel_l2(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def make_box(vti=False):
    wl = W.small_box(n_core=20, h=100.0, npml=6, ratio=1.08, n_st=2, n_rec=5, n_freq=2, n_core_y=14, n_core_z=10,
                     nt=1000)
    src = W.Points.make([[30.0, 0.0, wl.src.z[0]], [-250.0, 40.0, wl.src.z[0]]], 0)
    wl = dataclasses.replace(wl, src=src)
    rho, rho_true = wl.rho, wl.rho_true
    if vti:
        rho = np.stack([wl.rho, np.minimum(2.0 * wl.rho, 15.0)])
        rho_true = np.stack([wl.rho_true, np.minimum(2.0 * wl.rho_true, 15.0)])
        wl = dataclasses.replace(wl, rho_max=float(rho_true.max()))
    pb = fdtd.problem_from_workload(wl)
    d_obs = fdtd.forward(pb, rho_true, wl.src, wl.rec)
    _, r = fdtd.misfit(d_obs, fdtd.forward(pb, rho, wl.src, wl.rec))
    g = fdtd.gradient_time_domain(pb, rho, wl.src, wl.rec, r)
    return wl, rho, r, g


@pytest.fixture(scope="module")
def box():
    return make_box()


@pytest.mark.parametrize("precision,segment", [(64, 0), (64, 64), (32, 0), (32, 64), (32, 128), (32, 2)])
def test_td_gradient_matches_oracle(box, precision, segment):
    wl, rho, r, g_ref = box
    eng = Engine.from_workload(wl, precision=precision, kahan=1)
    assert eng.nt == 1000
    rg = torch.as_tensor(r, dtype=torch.complex128, device=eng.device)
    # a workspace full of NaN bit patterns: nothing may be read before it is written
    seg, nbytes = eng.td_plan(wl.src.n, wl.rec.n, budget_bytes=1 << 40 if segment == 0 else 0, segment=segment)
    work = torch.full((nbytes + 256,), 0xFF, dtype=torch.uint8, device=eng.device)
    g = eng.gradient_td(eng.model_tensor(rho), wl.src, wl.rec, rg, segment=segment, budget_bytes=1 << 40, work=work)
    torch.cuda.synchronize()
    if segment == 0:
        assert eng.last_td["segment"] >= eng.nt        # the whole run fits: no replay
    else:
        assert eng.last_td["segment"] == segment
    err = rel_l2(g.cpu().numpy(), g_ref)
    assert err <= (1e-9 if precision == 64 else 1e-3), (err, eng.launch_config())
    eng.check()
    eng.close()


TD_VARIANTS = [
    dict(kz_h=1, mb_h=6, lean_h=1, kz_e=1, mb_e=8, lean_e=1),
    dict(kz_h=2, mb_h=4, lean_h=2, kz_e=4, mb_e=6, lean_e=2),
    dict(fused_kz=4),
    dict(kz_h=2, mb_h=4, kz_e=1, mb_e=6, vec_h=1, vec_e=1),
    dict(kz_h=4, mb_h=4, kz_e=2, mb_e=4, tma_h=4, tma_e=4),
    dict(kz_h=8, mb_h=4, kz_e=2, mb_e=4),
    dict(onepass=(8, 4, 4)),
    dict(onepass=(16, 8, 3)),
    dict(wspec=(8, 4, 3)),
    dict(wspec=(16, 8, 2)),
    dict(wave=(2, 4, 8)),
    dict(wave=(1, 2, 6)),
]


@pytest.mark.parametrize("variant", range(len(TD_VARIANTS)))
def test_td_gradient_launch_variants(box, variant):
    """Checkpoints keep every state the chosen kernels carry (the second H buffer of
    the fused step, the CPML memory of the lean kernels) across the replay."""
    wl, rho, r, g_ref = box
    eng = Engine.from_workload(wl, precision=32, kahan=1, autotune=False)
    eng.set_launch(**TD_VARIANTS[variant])
    rg = torch.as_tensor(r, dtype=torch.complex128, device=eng.device)
    _, nbytes = eng.td_plan(wl.src.n, wl.rec.n, segment=192)
    work = torch.full((nbytes + 256,), 0xFF, dtype=torch.uint8, device=eng.device)
    g = eng.gradient_td(eng.model_tensor(rho), wl.src, wl.rec, rg, segment=192, work=work)
    assert rel_l2(g.cpu().numpy(), g_ref) <= 1e-3
    eng.close()


@pytest.mark.parametrize("precision", [64, 32])
def test_td_gradient_vti(precision):
    wl, rho, r, g_ref = make_box(vti=True)
    eng = Engine.from_workload(wl, precision=precision, kahan=1, vti=True)
    rg = torch.as_tensor(r, dtype=torch.complex128, device=eng.device)
    g = eng.gradient_td(eng.model_tensor(rho), wl.src, wl.rec, rg, segment=128)
    g = g.cpu().numpy()
    assert g.shape == g_ref.shape == (2,) + wl.rho.shape
    for part in (0, 1):
        assert rel_l2(g[part], g_ref[part]) <= (1e-9 if precision == 64 else 1e-3)
    eng.close()


def test_td_plan_and_workspace_checks(box):
    wl, rho, r, _ = box
    eng = Engine.from_workload(wl, precision=32, kahan=1)
    seg_min, bytes_min = eng.td_plan(2, wl.rec.n)
    seg_all, bytes_all = eng.td_plan(2, wl.rec.n, budget_bytes=1 << 40)
    assert seg_all >= eng.nt and bytes_all >= bytes_min and seg_min % 64 == 0 and seg_min < eng.nt
    seg_mid, bytes_mid = eng.td_plan(2, wl.rec.n, budget_bytes=(bytes_min + bytes_all) // 2)
    assert bytes_min <= bytes_mid <= (bytes_min + bytes_all) // 2 and seg_min <= seg_mid <= seg_all
    with pytest.raises(CsemError):
        eng.td_plan(2, wl.rec.n, budget_bytes=bytes_min // 2)
    with pytest.raises(CsemError):
        eng.td_plan(2, wl.rec.n, segment=63)
    # a workspace below the plan is refused before anything is launched
    from paper_2211_16665_gb300 import _capi
    from paper_2211_16665_gb300.engine import _ptr, _stream
    rg = torch.as_tensor(r, dtype=torch.complex128, device=eng.device)
    out = torch.zeros(eng.model_shape, dtype=eng.real, device=eng.device)
    work = torch.empty(1 << 20, dtype=torch.uint8, device=eng.device)
    with pytest.raises(CsemError):
        _capi.gradient_td(eng.ctx, _ptr(eng.model_tensor(rho)), wl.src, wl.rec, _ptr(rg), 64, 1, _ptr(out),
                          _ptr(work), work.numel(), _stream())
    eng.close()
