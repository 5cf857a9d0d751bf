"""The autograd function's time-domain route (appendix) against the basis route and
the oracle's time-domain gradient, and the inversion loop on it (FP64 engine)."""
import dataclasses

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from oracle import fdtd  # noqa: E402
from paper_2211_16665_gb300 import workloads as W  # noqa: E402
from paper_2211_16665_gb300.autograd import forward_data  # noqa: E402
from paper_2211_16665_gb300.engine import Engine  # noqa: E402


def rel_l2(a, b):
    return float(np.linalg.norm((np.asarray(a) - b).ravel()) / np.linalg.norm(np.asarray(b).ravel()))


def test_autograd_td_route_matches_oracle_and_basis_route():
    wl = W.small_box(n_core=16, h=100.0, npml=6, ratio=1.05, n_st=2, n_rec=5, n_freq=2, nt=900)
    wl = dataclasses.replace(wl, src=W.Points.make([[30.0, 0.0, wl.src.z[0]], [-250.0, 40.0, wl.src.z[0]]], 0))
    pb = fdtd.problem_from_workload(wl)
    d_obs = fdtd.forward(pb, wl.rho_true, wl.src, wl.rec)
    _, r = fdtd.misfit(d_obs, fdtd.forward(pb, wl.rho, wl.src, wl.rec))
    g_ref = fdtd.gradient_time_domain(pb, wl.rho, wl.src, wl.rec, r)
    eng = Engine.from_workload(wl, precision=64)
    eng.set_early_stop(1e-3)                       # the td route's data must still be the full run's
    dobs = torch.as_tensor(d_obs, device=eng.device)
    grads = {}
    for route in ("td", "basis"):
        basis = None if route == "td" else eng.estimate_adjoint_basis()[0]
        m = torch.tensor(np.log(wl.rho), dtype=torch.float64, device=eng.device, requires_grad=True)
        d = forward_data(m, eng, wl.src, wl.rec, basis, route=route, chunk=1)
        (0.5 * (dobs - d).abs().pow(2).sum()).backward()
        grads[route] = m.grad.cpu().numpy()
    assert rel_l2(grads["td"], g_ref) <= 1e-9
    assert rel_l2(grads["basis"], grads["td"]) <= 1e-3
    eng.close()
