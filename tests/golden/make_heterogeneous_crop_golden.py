"""Writes heterogeneous_crop_oracle.json: FP64 oracle outputs for the
heterogeneous (Gaussian random field) model cropped to 116^3 cells, used by
the precision-stress GPU test (plain FP32 vs Kahan-compensated FP32 vs FP64).

Calls only `oracle/` (and the seeded input generators).  Stored for the first
two of the workload's sources: receiver spectra, and the ln(rho) gradient of
the misfit against data from the same model with every resistivity scaled by
1.2 (at 600 cells: the 300 largest |g| and 300 seeded random core cells, plus
the global L2 norm).  Takes ~45 min on 8 cores.

    python tests/golden/make_heterogeneous_crop_golden.py
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import fdtd  # noqa: E402
from paper_2211_16665_gb300 import workloads as W  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "heterogeneous_crop_oracle.json")


def cplx(a):
    a = np.asarray(a)
    return {"re": a.real.tolist(), "im": a.imag.tolist()}


def main():
    t0 = time.time()
    wl = W.heterogeneous_crop96()
    src = wl.src.subset([0, 1])
    pb = fdtd.problem_from_workload(wl)
    rho_obs = wl.rho * 1.2
    d_obs = fdtd.forward(pb, rho_obs, src, wl.rec)
    d_syn, E = fdtd.forward(pb, wl.rho, src, wl.rec, keep_volume=True)
    phi, r = fdtd.misfit(d_obs, d_syn)
    Bp, fit = fdtd.adjoint_basis(pb, 1e-12)
    V = fdtd.adjoint(pb, wl.rho, wl.rec, r, Bp)
    g = fdtd.gradient(pb, wl.rho, E, V, wrt="lnrho")
    flat = g.ravel()
    top = np.argsort(-np.abs(flat))[:300]
    rng = np.random.default_rng(0)
    nz, ny, nx = g.shape
    core, topset = [], set(top.tolist())
    while len(core) < 300:
        k, j, i = rng.integers(10, nz - 10), rng.integers(10, ny - 10), rng.integers(10, nx - 10)
        c = int((k * ny + j) * nx + i)
        if c not in core and c not in topset:
            core.append(c)
    cells = [int(c) for c in top] + core
    out = {"what": "FP64 oracle, heterogeneous model cropped to 116^3, sources 0 and 1",
           "dt": pb.dt, "nt": pb.nt, "freqs": wl.freqs.tolist(),
           "d_obs": cplx(d_obs), "d_syn": cplx(d_syn), "phi": phi, "basis_fit": fit,
           "grad_cells": cells, "grad_values": flat[cells].tolist(), "grad_norm": float(np.linalg.norm(flat)),
           "seconds": time.time() - t0}
    json.dump(out, open(OUT, "w"))
    print(f"wrote {OUT} in {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
