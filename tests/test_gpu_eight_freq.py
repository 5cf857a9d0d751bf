"""GPU parity with the largest frequency set (eight frequencies, the flush kernels'
widest padding) through the C ABI against the FP64 oracle, on the same seeded inputs.

The box is 70 x 39 x 37 cells: ragged for the 64-wide x tiles of the two-cell
kernels, for 8-row blocks and for 16-plane z blocks.  Every transform flush
kernel runs: the register kernel at 16, 32, 64 and 128 snapshots per block (its
weights for all snapshots and frequencies staged in shared memory at once), the
bulk-copy kernel at 16 and 32, the streamed kernel at 64 and 128, in order and
overlapped.  The adjoint runs from the oracle's 16-column basis, so the adjoint
parity does not depend on the conditioning of the basis fit.

Tolerances as for the two-frequency box: FP64 1e-10 (receivers, volumes) and
1e-9 (adjoint, gradient); FP32 receivers 1e-5, volumes and gradients 1e-3.
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


def rel_l2(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def gpu_volume(eng, v):
    return v.cpu().numpy()[..., : eng.nx + 1].astype(np.complex128)


@pytest.fixture(scope="module")
def eight():
    wl = W.small_box(n_core=46, h=100.0, npml=8, ratio=1.08, n_st=4, n_rec=6, n_freq=2, n_core_y=15, n_core_z=13)
    wl = dataclasses.replace(wl, freqs=np.linspace(0.25, 1.5, 8))
    pb = fdtd.problem_from_workload(wl)
    d_obs = fdtd.forward(pb, wl.rho_true, wl.src, wl.rec)
    d, E = fdtd.forward(pb, wl.rho, wl.src, wl.rec, keep_volume=True)
    phi, r = fdtd.misfit(d_obs, d)
    Bp, _ = fdtd.adjoint_basis(pb, 1e-12)
    V = fdtd.adjoint(pb, wl.rho, wl.rec, r, Bp)
    g = fdtd.gradient(pb, wl.rho, E, V, wrt="lnrho")
    return wl, pb, dict(d_obs=d_obs, d=d, E=E, Bp=Bp, V=V, g=g)


FLUSHES_FP32 = [(0, 16), (0, 32), (0, 64), (0, 128), (1, 16), (1, 32), (1, 64), (1, 128), (2, 32), (3, 64)]
FLUSHES_FP64 = [(0, 16), (0, 64), (0, 128), (2, 32)]


@pytest.mark.parametrize("precision,flush", [(32, f) for f in FLUSHES_FP32] + [(64, f) for f in FLUSHES_FP64])
def test_every_flush_kernel_with_eight_frequencies(eight, precision, flush):
    wl, pb, o = eight
    fm, m = flush
    eng = Engine.from_workload(wl, precision=precision, kahan=1, autotune=False)
    assert eng.nt == pb.nt and eng.nf == 8
    eng.set_launch(kz_h=4, mb_h=4, kz_e=4, mb_e=4, flush_mode=fm, block=m)
    rho = eng.model_tensor(wl.rho)
    d, E = eng.fwd_model(rho, wl.src, wl.rec, keep_volume=True)
    assert rel_l2(d.cpu().numpy(), o["d"]) <= (1e-10 if precision == 64 else 1e-5)
    assert rel_l2(gpu_volume(eng, E), o["E"]) <= (1e-10 if precision == 64 else 1e-3)
    eng.check()
    eng.close()


@pytest.mark.parametrize("precision", [32, 64])
def test_autotuned_gradient_with_eight_frequencies(eight, precision):
    """The autotuner times every step and flush candidate on this grid (all of them
    staging eight frequencies), then forward, adjoint and gradient match the oracle."""
    wl, pb, o = eight
    eng = Engine.from_workload(wl, precision=precision, kahan=1)
    rho = eng.model_tensor(wl.rho)
    d, E = eng.fwd_model(rho, wl.src, wl.rec, keep_volume=True)
    tol = 1e-10 if precision == 64 else 1e-3
    assert rel_l2(d.cpu().numpy(), o["d"]) <= (1e-10 if precision == 64 else 1e-5)
    assert rel_l2(gpu_volume(eng, E), o["E"]) <= tol
    _, r = misfit(torch.as_tensor(o["d_obs"], device=eng.device), d)
    basis = torch.as_tensor(o["Bp"], dtype=torch.float64, device=eng.device)
    V = eng.adjoint_model(rho, wl.rec, r, basis)
    tol = 1e-9 if precision == 64 else 1e-3
    assert rel_l2(gpu_volume(eng, V), o["V"]) <= tol
    assert rel_l2(eng.gradient(rho, E, V, wrt="lnrho").cpu().numpy(), o["g"]) <= tol
    eng.check()
    eng.close()
