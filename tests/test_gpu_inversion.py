"""GPU parity of the outer inversion loop (Sec. 3.5): the device loop (FP64
engine, gradient through autograd) against the reference loop on the FP64
oracle, same data, weights, free cells, Tikhonov term and bounds, for three
iterations: the same directions and accepted steps, phi per iteration within
1e-6 and the final model within 1e-6 in ln(rho).
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from oracle import fdtd  # noqa: E402
from oracle import inversion as ref  # noqa: E402
from paper_2211_16665_gb300 import workloads as W  # noqa: E402
from paper_2211_16665_gb300.engine import Engine  # noqa: E402
from paper_2211_16665_gb300.inversion import Inversion  # noqa: E402


def test_device_loop_follows_the_reference_loop():
    wl = W.small_box(n_core=16, h=100.0, npml=8, ratio=1.0, n_st=0, n_rec=5, n_freq=2)
    pb = fdtd.problem_from_workload(wl)
    d_obs = fdtd.forward(pb, wl.rho_true, wl.src, wl.rec)
    mute = ref.mute_weights(wl.src, wl.rec, wl.freqs.size, 300.0)
    w = mute / (0.05 * np.abs(d_obs) + 1e-3 * np.abs(d_obs).max())
    free = wl.rho > 0.5
    m0 = np.log(wl.rho)
    alpha, beta0, cool, lo, hi = (1.0, 1.0, 0.1), 0.01, 0.7, math.log(0.1), math.log(wl.rho_max)
    kw = dict(memory=5, step0=0.5, max_backtracks=6, beta0=beta0, cool=cool)

    data = ref.DataTerm(pb, wl.src, wl.rec, d_obs, w, wl.rho, free)
    reg = lambda m: ref.tikhonov(m, m0, free, wl.xn, wl.yn, wl.zn, alpha)
    m_ref, h_ref = ref.invert(data, m0, free, 3, lo, hi, reg=reg, **kw)

    eng = Engine.from_workload(wl, precision=64, kahan=0)
    basis, _, _ = eng.estimate_adjoint_basis(gamma=1e-12, relative=True)
    inv = Inversion(eng, wl.src, wl.rec, torch.as_tensor(d_obs), wl.rho, free, basis, weights=w,
                    alpha=alpha, xn=wl.xn, yn=wl.yn, zn=wl.zn, m_min=lo, m_max=hi, **kw)
    m_gpu, h_gpu = inv.run(torch.as_tensor(m0), 3)
    eng.close()

    assert len(h_gpu) == len(h_ref) == 3
    for a, b in zip(h_gpu, h_ref):
        assert a["direction"] == b["direction"] and a["accepted"] == b["accepted"]
        assert abs(a["step"] - b["step"]) <= 1e-6 * b["step"]
        assert abs(a["phi"] - b["phi"]) <= 1e-6 * b["phi"]
        assert abs(a["phi_m"] - b["phi_m"]) <= 1e-6 * max(b["phi_m"], 1e-30)
    assert h_ref[-1]["phi"] < h_ref[0]["phi"]
    assert np.abs(m_gpu.cpu().numpy()[free] - m_ref[free]).max() <= 1e-6
