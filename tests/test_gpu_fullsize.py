"""Full-size GPU checks.

* thin_reservoir (128x128x96, nt from CFL, 4 frequencies): the CUDA path
  against FP64 oracle values stored by tests/golden/make_thin_reservoir_golden.py
  -- receivers rel-L2 <= 1e-5, gradient rel-L2 <= 1e-3 on 600 stored cells;
* the autograd-wrapped FP32 gradient against central finite differences of
  the misfit computed with the FP64 engine on 20 seeded cells;
* batched_towline (256x256x128, 32 sources): one batched launch equals
  single-source launches bit for bit (a property that holds at any size);
* source chunks recomputed in backward give the unchunked gradient;
* large_gradient (400x400x200, 8 frequencies): the source-chunked autograd path
  with recomputation gives the chunked path that keeps the forward volumes, bit
  for bit, at the full grid size (nt shortened; a property that holds at any nt);
* heterogeneous (512x512x256, Gaussian random field model): a two-source batch
  equals single-source runs bit for bit, receivers and volumes, at the full grid.
"""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2211_16665_gb300 import workloads as W  # noqa: E402
from paper_2211_16665_gb300.autograd import forward_data  # noqa: E402
from paper_2211_16665_gb300.engine import Engine, misfit  # noqa: E402

GOLD = os.path.join(os.path.dirname(__file__), "golden", "thin_reservoir_oracle.json")


def rel_l2(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def cplx(d):
    return np.asarray(d["re"]) + 1j * np.asarray(d["im"])


@pytest.fixture(scope="module")
def gold():
    return json.load(open(GOLD))


@pytest.fixture(scope="module")
def thin():
    wl = W.thin_reservoir()
    eng = Engine.from_workload(wl)
    yield wl, eng
    eng.close()


def test_thin_reservoir_matches_oracle(thin, gold):
    wl, eng = thin
    assert eng.nt == gold["nt"] and abs(eng.dt - gold["dt"]) <= 1e-12 * gold["dt"]
    d_obs = eng.fwd_model(eng.model_tensor(wl.rho_true), wl.src, wl.rec)
    e_obs = rel_l2(d_obs[0].cpu().numpy(), cplx(gold["d_obs"]))
    assert e_obs <= 1e-5
    rho = eng.model_tensor(wl.rho)
    d_syn, E = eng.fwd_model(rho, wl.src, wl.rec, keep_volume=True)
    e_syn = rel_l2(d_syn[0].cpu().numpy(), cplx(gold["d_syn"]))
    assert e_syn <= 1e-5
    d_obs_noisy = torch.as_tensor(cplx(gold["d_obs_noisy"])[None], device="cuda")
    phi, r = misfit(d_obs_noisy, d_syn)
    assert abs(phi.item() - gold["phi"]) <= 1e-4 * gold["phi"]
    basis, fit, _ = eng.estimate_adjoint_basis()
    assert abs(fit - gold["basis_fit"]) <= 1e-3 * gold["basis_fit"] + 1e-9
    V = eng.adjoint_model(rho, wl.rec, r, basis)
    g = eng.gradient(rho, E, V).double().cpu().numpy().ravel()
    cells = np.asarray(gold["grad_cells"])
    e_g = rel_l2(g[cells], gold["grad_values"])
    e_n = abs(np.linalg.norm(g) - gold["grad_norm"]) / gold["grad_norm"]
    print(f"\nthin_reservoir vs oracle: d_obs {e_obs:.2e}, d_syn {e_syn:.2e}, phi "
          f"{abs(phi.item() - gold['phi']) / gold['phi']:.2e}, gradient (600 cells) {e_g:.2e}, norm {e_n:.2e}")
    assert e_g <= 1e-3
    assert e_n <= 1e-3


def test_thin_reservoir_autograd_matches_central_differences(thin, gold):
    wl, eng = thin
    basis, _, _ = eng.estimate_adjoint_basis()
    d_obs = torch.as_tensor(cplx(gold["d_obs_noisy"])[None], device="cuda")
    ln_rho = torch.tensor(np.log(wl.rho), dtype=torch.float64, device="cuda", requires_grad=True)
    d = forward_data(ln_rho, eng, wl.src, wl.rec, basis)
    loss = 0.5 * (d_obs - d).abs().pow(2).sum()
    loss.backward()
    g = ln_rho.grad.cpu().numpy()

    eng64 = Engine.from_workload(wl, precision=64, kahan=0)
    flat = np.abs(g).ravel()
    strong = np.flatnonzero(flat >= 1e-2 * flat.max())
    cells = np.random.default_rng(42).choice(strong, size=20, replace=False)
    h = 1e-3
    errs = []
    for c in cells:
        phis = []
        for sgn in (1.0, -1.0):
            m = np.log(wl.rho).ravel().copy()
            m[c] += sgn * h
            dd = eng64.fwd_model(eng64.model_tensor(np.exp(m.reshape(wl.rho.shape))), wl.src, wl.rec)
            phis.append(0.5 * float((d_obs - dd).abs().pow(2).sum()))
        fd = (phis[0] - phis[1]) / (2 * h)
        errs.append(abs(g.ravel()[c] - fd) / abs(fd))
    eng64.close()
    print(f"\nautograd vs central differences (20 cells): max rel {max(errs):.2e}, median {np.median(errs):.2e}")
    assert max(errs) <= 1e-2, errs


def test_batched_towline_batched_equals_single_source():
    wl = W.batched_towline()
    eng = Engine.from_workload(wl, nt=1024)
    rho = eng.model_tensor(wl.rho)
    d_all, E_all = eng.fwd_model(rho, wl.src, wl.rec, keep_volume=True)
    for s in (0, 13, 31):
        d1, E1 = eng.fwd_model(rho, wl.src.subset([s]), wl.rec, keep_volume=True)
        assert torch.equal(d1[0], d_all[s])
        assert torch.equal(E1[0], E_all[s])
    eng.close()


def test_chunked_recompute_gives_the_unchunked_gradient():
    wl = W.small_box(n_core=20, h=100.0, npml=8, ratio=1.05, n_st=3, n_rec=6, n_freq=2)
    src = W.Points.make([[x, 0.0, wl.src.z[0]] for x in (-300.0, -100.0, 100.0, 300.0)], 0)
    eng = Engine.from_workload(wl, max_src=4)
    basis, _, _ = eng.estimate_adjoint_basis()
    d_obs = eng.fwd_model(eng.model_tensor(wl.rho_true), src, wl.rec)
    grads = []
    for chunk, recompute in ((4, False), (2, True), (1, True)):
        ln_rho = torch.tensor(np.log(wl.rho), dtype=torch.float64, device="cuda", requires_grad=True)
        d = forward_data(ln_rho, eng, src, wl.rec, basis, chunk=chunk, recompute=recompute)
        (0.5 * (d_obs - d).abs().pow(2).sum()).backward()
        grads.append(ln_rho.grad.cpu().numpy())
    for g in grads[1:]:
        assert rel_l2(g, grads[0]) <= 1e-6
    eng.close()


def test_large_gradient_chunked_recompute_at_full_size():
    wl = W.large_gradient()
    src = wl.src.subset([0, 21, 40, 63])
    eng = Engine.from_workload(wl, max_src=2, nt=192)
    basis, _, _ = eng.estimate_adjoint_basis()
    ln_true = torch.tensor(np.log(wl.rho_true), dtype=torch.float64, device="cuda")
    with torch.no_grad():
        d_obs = 0.9 * forward_data(ln_true, eng, src, wl.rec, basis, chunk=2, recompute=True)
    grads = []
    for recompute in (False, True):
        ln_rho = ln_true.clone().requires_grad_(True)
        d = forward_data(ln_rho, eng, src, wl.rec, basis, chunk=2, recompute=recompute)
        (0.5 * (d_obs - d).abs().pow(2).sum()).backward()
        grads.append(ln_rho.grad)
    eng.check()
    eng.close()
    g = grads[0]
    assert torch.isfinite(g).all() and g.abs().max() > 0
    assert torch.equal(grads[1], g)


def test_heterogeneous_full_grid_batched_equals_single_source():
    wl = W.heterogeneous()
    src = wl.src.subset([0, 9])
    eng = Engine.from_workload(wl, max_src=2, nt=128)
    rho = eng.model_tensor(wl.rho)
    d2, E2 = eng.fwd_model(rho, src, wl.rec, keep_volume=True)
    assert torch.isfinite(E2).all() and E2.abs().max() > 0
    for s in (0, 1):
        d1, E1 = eng.fwd_model(rho, src.subset([s]), wl.rec, keep_volume=True)
        assert torch.equal(d1[0], d2[s])
        assert torch.equal(E1[0], E2[s])
        del E1
    eng.check()
    eng.close()
