"""Precision stress on the heterogeneous model (log10 rho a Gaussian random
field, 0.5-100 ohm-m, under 0.3 ohm-m water) cropped to 116^3 cells: the FP32
stencil with a plain volumetric transform, the FP32 stencil with the
Kahan-compensated transform, and the FP64 stencil, each against the FP64 oracle
(values stored by tests/golden/make_heterogeneous_crop_golden.py) on the
receiver fields and on the ln(rho) gradient.  The receiver transforms are FP64
in every mode; the volumetric transform precision shows in the gradient."""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2211_16665_gb300 import workloads as W  # noqa: E402
from paper_2211_16665_gb300.engine import Engine, misfit  # noqa: E402

GOLD = os.path.join(os.path.dirname(__file__), "golden", "heterogeneous_crop_oracle.json")


def rel_l2(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def cplx(d):
    return np.asarray(d["re"]) + 1j * np.asarray(d["im"])


# both FP32 modes step with one launch configuration, so their fields are the same bit for
# bit and only the volumetric transform differs between them
FP32_LAUNCH = dict(kz_h=2, mb_h=6, lean_h=2, kz_e=2, mb_e=6, lean_e=2, flush_mode=1, block=32)


def run_mode(wl, src, gold, precision, kahan):
    eng = Engine.from_workload(wl, precision=precision, kahan=kahan, max_src=src.n, autotune=precision != 32)
    if precision == 32:
        eng.set_launch(**FP32_LAUNCH)
    rho = eng.model_tensor(wl.rho)
    d, E = eng.fwd_model(rho, src, wl.rec, keep_volume=True)
    phi, r = misfit(torch.as_tensor(cplx(gold["d_obs"]), device="cuda"), d)
    basis, fit, _ = eng.estimate_adjoint_basis()
    V = eng.adjoint_model(rho, wl.rec, r, basis)
    g = eng.gradient(rho, E, V).double().cpu().numpy().ravel()
    eng.close()
    cells = np.asarray(gold["grad_cells"])
    return rel_l2(d.cpu().numpy(), cplx(gold["d_syn"])), rel_l2(g[cells], gold["grad_values"])


def test_plain_kahan_fp64_against_oracle():
    gold = json.load(open(GOLD))
    wl = W.heterogeneous_crop96()
    src = wl.src.subset([0, 1])
    res = {name: run_mode(wl, src, gold, prec, kahan)
           for name, prec, kahan in (("fp32_plain", 32, 0), ("fp32_kahan", 32, 1), ("fp64", 64, 0))}
    print("\nprecision stress (receiver rel-L2, gradient rel-L2 at 600 cells): " +
          ", ".join(f"{k} ({v[0]:.2e}, {v[1]:.2e})" for k, v in res.items()))
    assert res["fp64"][0] <= 1e-9 and res["fp64"][1] <= 1e-7
    assert res["fp32_kahan"][0] <= 1e-5 and res["fp32_kahan"][1] <= 1e-3
    assert res["fp32_plain"][0] <= 1e-5 and res["fp32_plain"][1] <= 1e-2
    # compensation does not make the gradient worse than the plain transform, beyond the FP32
    # stepping floor both share (the error of the common fields can cancel either transform's)
    assert res["fp32_kahan"][1] <= res["fp32_plain"][1] * 1.05 + 2e-6
